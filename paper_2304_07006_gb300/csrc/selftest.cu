// Self-test of the bounded device waits that every tensor-core kernel relies on: a wait whose
// barrier nothing completes must give up after its limit, record an error code for the host and
// let the kernel return, leaving the context usable.
#include "ptx_sm100.cuh"
#include "xtc_internal.cuh"

namespace xtc {
namespace {

__global__ void wait_timeout_selftest_kernel(int* err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  // the phase of parity 0 never completes: no thread arrives on bar
  if (threadIdx.x == 0) mbar_wait(&bar, 0, &abort_flag, err, DEV_ERR_TIMEOUT_SELFTEST, limit_ns);
  __syncthreads();
}

}  // namespace

void launch_wait_timeout_selftest(int* err, unsigned long long limit_ns, cudaStream_t st) {
  wait_timeout_selftest_kernel<<<1, 32, 0, st>>>(err, limit_ns);
}

}  // namespace xtc
