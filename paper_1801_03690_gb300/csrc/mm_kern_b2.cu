// Batched solver kernel for at least 2 resident blocks per SM.
#include "mm_solver_body.cuh"

namespace mm {
const void* solver_batch_kernel_2() { return (const void*)k_solver_batch<2>; }
}  // namespace mm
