// The batched solver's device code at 512 threads per CTA (see batched.cuh).
#include "batched.cuh"

namespace mds {
namespace batch {
namespace bt512 {
constexpr int kBT = 512;
#include "batched_dev.cuh"

KernelFn kernel() { return batched_solve_kernel; }
unsigned smem_bytes(int N, int m, int np, int P4) { return smem_layout(N, m, np, P4).total; }
}  // namespace bt512
}  // namespace batch
}  // namespace mds
