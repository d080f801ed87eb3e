// The batched solver's device code at 128 threads per CTA (see batched.cuh).
#include "batched.cuh"

namespace mds {
namespace batch {
namespace bt128 {
constexpr int kBT = 128;
#include "batched_dev.cuh"

KernelFn kernel() { return batched_solve_kernel; }
unsigned smem_bytes(int N, int m, int np, int P4) { return smem_layout(N, m, np, P4).total; }
}  // namespace bt128
}  // namespace batch
}  // namespace mds
