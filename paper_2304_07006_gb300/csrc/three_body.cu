// The explicit three-body tensor of eq. Ldecomp ("Decomposition of two-body correction") for small
// orbital sets, as a validation aid for full transcorrelated codes:
//     L_prt^qsu = sum_i [ rho_pq(i) V_rs(i).V_tu(i) + rho_rs(i) V_pq(i).V_tu(i) + rho_tu(i) V_pq(i).V_rs(i) ],
//     rho_pq(i) = w_i phi_p(i) phi_q(i),   V_rs(i) the vector pair field of step (b).
// With packed pairs a, b, c the three terms are one tensor read three ways:
//     T[a][b][c] = sum_i rho_a(i) X_bc(i),   X_bc(i) = V_b(i).V_c(i),
//     L_prt^qsu = T[pq][rs][tu] + T[rs][pq][tu] + T[tu][pq][rs].
// T is an FP64 product of rho^T (pairs x points) with X (points x pair pairs), tiled through shared
// memory with X formed while staging; L is then written densely, L[p][r][t][q][s][u].
#include <algorithm>

#include "xtc_internal.cuh"

namespace xtc {
namespace {

constexpr int TB_TA = 32;  // pairs a per CTA
constexpr int TB_TM = 64;  // (b, c) combinations per CTA
constexpr int TB_KC = 16;  // outer points per shared-memory stage

__device__ __forceinline__ int tb_pair(int p, int q, int N) {
  const int a = min(p, q), b = max(p, q);
  return a * N - a * (a - 1) / 2 + (b - a);
}

// T[a][m], m = b * NP + c: each thread owns 2 rows a x 4 columns m of the CTA's 32 x 64 tile.
__global__ void __launch_bounds__(256)
    three_body_t_kernel(const double* __restrict__ phi, const double* __restrict__ w, int64_t i0, int64_t n_i,
                        int N, int NP, const int* __restrict__ pair_p, const int* __restrict__ pair_q,
                        const double* __restrict__ V, double* __restrict__ T) {
  __shared__ double As[TB_KC][TB_TA];
  __shared__ double Bs[TB_KC][TB_TM];
  const int a0 = blockIdx.y * TB_TA;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * TB_TM;
  const int64_t NP2 = static_cast<int64_t>(NP) * NP;
  const int t = threadIdx.x;
  const int ta = (t / 16) * 2, tm = (t % 16) * 4;
  double acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  for (int64_t k0 = 0; k0 < n_i; k0 += TB_KC) {
    for (int e = t; e < TB_KC * TB_TA; e += blockDim.x) {
      const int kk = e / TB_TA, a = a0 + e % TB_TA;
      const int64_t k = k0 + kk;
      double v = 0.0;
      if (k < n_i && a < NP) {
        const int64_t g = i0 + k;
        v = w[g] * phi[g * N + pair_p[a]] * phi[g * N + pair_q[a]];
      }
      As[kk][e % TB_TA] = v;
    }
    for (int e = t; e < TB_KC * TB_TM; e += blockDim.x) {
      const int kk = e / TB_TM;
      const int64_t k = k0 + kk, m = m0 + e % TB_TM;
      double v = 0.0;
      if (k < n_i && m < NP2) {
        const int b = static_cast<int>(m / NP), c = static_cast<int>(m % NP);
        const double* Vk = V + k * 3 * NP;  // V[k][x][pair]
        v = Vk[b] * Vk[c] + Vk[NP + b] * Vk[NP + c] + Vk[2 * NP + b] * Vk[2 * NP + c];
      }
      Bs[kk][e % TB_TM] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TB_KC; ++kk) {
      const double x0 = As[kk][ta], x1 = As[kk][ta + 1];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const double y = Bs[kk][tm + j];
        acc[0][j] = fma(x0, y, acc[0][j]);
        acc[1][j] = fma(x1, y, acc[1][j]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int a = a0 + ta + r;
    if (a >= NP) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t m = m0 + tm + j;
      if (m < NP2) T[static_cast<int64_t>(a) * NP2 + m] = acc[r][j];
    }
  }
}

// L[p][r][t][q][s][u] = T[pq][rs][tu] + T[rs][pq][tu] + T[tu][pq][rs]
__global__ void three_body_unpack_kernel(const double* __restrict__ T, int N, int NP, double* __restrict__ L) {
  const int64_t n3 = static_cast<int64_t>(N) * N * N;
  const int64_t total = n3 * n3;
  const int64_t NP2 = static_cast<int64_t>(NP) * NP;
  for (int64_t o = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; o < total;
       o += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t r_ = o;
    const int u = static_cast<int>(r_ % N); r_ /= N;
    const int s = static_cast<int>(r_ % N); r_ /= N;
    const int q = static_cast<int>(r_ % N); r_ /= N;
    const int tt = static_cast<int>(r_ % N); r_ /= N;
    const int r = static_cast<int>(r_ % N); r_ /= N;
    const int p = static_cast<int>(r_);
    const int64_t a = tb_pair(p, q, N), b = tb_pair(r, s, N), c = tb_pair(tt, u, N);
    L[o] = T[a * NP2 + b * NP + c] + T[b * NP2 + a * NP + c] + T[c * NP2 + a * NP + b];
  }
}

}  // namespace

void launch_three_body_t(const double* phi, const double* w, int64_t i0, int64_t n_i, int n_orb, const int* pair_p,
                         const int* pair_q, const double* V, double* T, cudaStream_t st) {
  const int NP = n_orb * (n_orb + 1) / 2;
  const int64_t NP2 = static_cast<int64_t>(NP) * NP;
  dim3 grid(static_cast<unsigned>((NP2 + TB_TM - 1) / TB_TM), static_cast<unsigned>((NP + TB_TA - 1) / TB_TA));
  three_body_t_kernel<<<grid, 256, 0, st>>>(phi, w, i0, n_i, n_orb, NP, pair_p, pair_q, V, T);
}

void launch_three_body_unpack(const double* T, int n_orb, double* L, cudaStream_t st) {
  const int NP = n_orb * (n_orb + 1) / 2;
  const int64_t n3 = static_cast<int64_t>(n_orb) * n_orb * n_orb;
  const int64_t blocks = std::min<int64_t>((n3 * n3 + 255) / 256, 152 * 32);
  three_body_unpack_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(T, n_orb, NP, L);
}

}  // namespace xtc
