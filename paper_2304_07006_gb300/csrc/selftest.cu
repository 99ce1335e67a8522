// Self-tests of device building blocks: the bounded device waits that every tensor-core kernel
// relies on (a wait whose barrier nothing completes must give up after its limit, record an error
// code for the host and let the kernel return, leaving the context usable), and the refined
// reciprocal square root and reciprocal of the gradient kernel.
#include "ptx_sm100.cuh"
#include "simt_pack.cuh"
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

__global__ void recip_selftest_kernel(const float* __restrict__ x, int64_t n, float* __restrict__ y_rsqrt,
                                      float* __restrict__ y_rcp) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  // the packed forms used by the gradient kernel, on (x, x) pairs; both halves and the scalar
  // form must agree
  const f32x2 r2 = rsqrt_nr2(x[i], x[i]);
  const f32x2 c2 = rcp_nr2(x[i], x[i]);
  float ra, rb, ca, cb;
  up2(r2, ra, rb);
  up2(c2, ca, cb);
  const float rs = rsqrt_nr(x[i]), rc = rcp_nr(x[i]);
  y_rsqrt[i] = (ra == rb && ra == rs) ? rs : __int_as_float(0x7fc00000);  // NaN flags a mismatch
  y_rcp[i] = (ca == cb && ca == rc) ? rc : __int_as_float(0x7fc00000);
}

}  // namespace

void launch_wait_timeout_selftest(int* err, unsigned long long limit_ns, cudaStream_t st) {
  wait_timeout_selftest_kernel<<<1, 32, 0, st>>>(err, limit_ns);
}

void launch_recip_selftest(const float* x, int64_t n, float* y_rsqrt, float* y_rcp, cudaStream_t st) {
  if (n <= 0) return;
  recip_selftest_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(x, n, y_rsqrt, y_rcp);
}

}  // namespace xtc
