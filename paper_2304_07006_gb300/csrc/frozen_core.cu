// Frozen-core folding of the xTC corrections (xTC-FC, Results section "Frozen core approximation"):
// the corrections are built for the whole orbital space and the doubly occupied core orbitals C
// are frozen afterwards with the standard closed-shell equations,
//   E_core      = sum_c 2 h_cc + sum_{c,d} [2 U(cc|dd) - U(cd|dc)]
//   h^FC_pq     = h_pq + sum_c [2 U(pq|cc) - U(pc|cq)]          p, q active
//   U^FC(pq|rs) = U(pq|rs)                                      p, q, r, s active,
// applied to h = Delta h and U = Delta U (chemists' order, U(pq|rs) = U(rs|pq)).  The folding is
// linear, so the caller adds the folding of its own one- and two-electron integrals.
//
// All three parts read Delta U in FP64.  The one-body part and the core energy touch
// O(n_act^2 n_core) and O(n_core^2) elements; the two-body part is a gather of n_act^4 elements
// (16 bytes of HBM traffic each), one warp per (p, q, r) row so that the reads of a row are one
// contiguous run wherever the active orbitals are.
#include "xtc_internal.cuh"

namespace xtc {
namespace {

__global__ void fc_onebody_kernel(const double* __restrict__ dU, const double* __restrict__ dh, int N,
                                  FcIndex ix, double* __restrict__ dh_fc) {
  const int a = blockIdx.x;
  const int64_t p = ix.act[a];
  const int64_t n = N;
  for (int b = threadIdx.x; b < ix.n_act; b += blockDim.x) {
    const int64_t q = ix.act[b];
    double s = dh[p * n + q];
    for (int k = 0; k < ix.n_core; ++k) {
      const int64_t c = ix.core[k];
      const double coulomb = dU[((p * n + q) * n + c) * n + c];
      const double exchange = dU[((p * n + c) * n + c) * n + q];
      s += 2.0 * coulomb - exchange;
    }
    dh_fc[static_cast<int64_t>(a) * ix.n_act + b] = s;
  }
}

constexpr int FC_E_THREADS = 256;

// One block; a fixed reduction tree, so the result does not depend on timing.
__global__ void fc_core_energy_kernel(const double* __restrict__ dU, const double* __restrict__ dh, int N,
                                      FcIndex ix, double* __restrict__ e_core) {
  __shared__ double part[FC_E_THREADS];
  const int64_t n = N;
  const int nc = ix.n_core;
  double s = 0.0;
  for (int t = threadIdx.x; t < nc * nc; t += FC_E_THREADS) {
    const int64_t c = ix.core[t / nc], d = ix.core[t % nc];
    s += 2.0 * dU[((c * n + c) * n + d) * n + d] - dU[((c * n + d) * n + d) * n + c];
  }
  for (int t = threadIdx.x; t < nc; t += FC_E_THREADS) {
    const int64_t c = ix.core[t];
    s += 2.0 * dh[c * n + c];
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = FC_E_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *e_core = part[0];
}

constexpr int FC_G_THREADS = 256;

__global__ void __launch_bounds__(FC_G_THREADS) fc_gather_kernel(const double* __restrict__ dU, int N, FcIndex ix,
                                                                 double* __restrict__ dU_act) {
  __shared__ int act[FC_MAX_ORB];
  for (int t = threadIdx.x; t < ix.n_act; t += FC_G_THREADS) act[t] = ix.act[t];
  __syncthreads();
  const int na = ix.n_act;
  const int lane = threadIdx.x & 31;
  const int64_t n = N;
  const int64_t rows = static_cast<int64_t>(na) * na * na;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (FC_G_THREADS / 32);
  for (int64_t row = blockIdx.x * static_cast<int64_t>(FC_G_THREADS / 32) + (threadIdx.x >> 5); row < rows;
       row += warps) {
    const int r = static_cast<int>(row % na);
    const int64_t pq = row / na;
    const int q = static_cast<int>(pq % na), p = static_cast<int>(pq / na);
    const double* src = dU + ((act[p] * n + act[q]) * n + act[r]) * n;
    double* dst = dU_act + row * na;
    for (int s = lane; s < na; s += 32) dst[s] = __ldcs(src + act[s]);
  }
}

}  // namespace

void launch_frozen_core(const double* dU, const double* dh, int N, const FcIndex& ix, double* dh_fc,
                        double* dU_act, double* e_core, int n_sm, cudaStream_t st) {
  fc_core_energy_kernel<<<1, FC_E_THREADS, 0, st>>>(dU, dh, N, ix, e_core);
  if (ix.n_act == 0) return;
  fc_onebody_kernel<<<ix.n_act, 128, 0, st>>>(dU, dh, N, ix, dh_fc);
  if (dU_act) {
    const int64_t rows = static_cast<int64_t>(ix.n_act) * ix.n_act * ix.n_act;
    const int64_t want = (rows + FC_G_THREADS / 32 - 1) / (FC_G_THREADS / 32);
    const int64_t cap = static_cast<int64_t>(n_sm) * 8;  // 8 resident blocks of 256 threads per SM
    fc_gather_kernel<<<static_cast<unsigned>(want < cap ? want : cap), FC_G_THREADS, 0, st>>>(dU, N, ix, dU_act);
  }
}

}  // namespace xtc
