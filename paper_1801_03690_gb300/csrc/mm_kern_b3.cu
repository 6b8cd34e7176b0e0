// Batched solver kernel for at least 3 resident blocks per SM.
#include "mm_solver_body.cuh"

namespace mm {
const void* solver_batch_kernel_3() { return (const void*)k_solver_batch<3>; }
}  // namespace mm
