// Batched solver kernel for at least 4 resident blocks per SM.
#include "mm_solver_body.cuh"

namespace mm {
const void* solver_batch_kernel_4() { return (const void*)k_solver_batch<4>; }
}  // namespace mm
