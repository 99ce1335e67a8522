// The two-body transcorrelated integrals K (Theory section, next to the Coulomb integrals V):
//     K_pr^qs = 1/2 <pr| P12 [ lap_1 u + (grad_1 u)^2 + 2 grad_1 u . grad_1 ] |qs>,
//     P12 f(1,2) = f(1,2) + f(2,1),
// on the quadrature grid, for real spatial orbitals.  Written out with the vector pair field
// V_rs(i) = sum_j w_j grad_1 u(r_i, r_j) phi_r(j) phi_s(j) of step (b) and the scalar field
//     W_rs(i) = sum_j w_j F(r_i, r_j) phi_r(j) phi_s(j),   F = lap_1 u + |grad_1 u|^2,
// the f(1,2) part is
//     sum_i [ rho_pq(i) W_rs(i) + 2 psi_pq(i) . V_rs(i) ],  rho_pq = w phi_p phi_q,  psi_pq = w phi_p grad phi_q,
// and the f(2,1) part is the same expression with (pq) and (rs) exchanged (relabel i <-> j; u is
// symmetric).  So with
//     S[pq][rs] = sum_i [ 1/2 rho_pq(i) W_rs(i) + psi_pq(i) . V_rs(i) ]      (pq: all N^2, rs: pairs)
// the integrals are K[p][q][r][s] = S[pq][rs] + S[rs][pq].
//
// Per chunk of outer points: F w_j as a table (FP64, inner points x outer points), W = that table
// times the pair products (an FP64 GEMM with the pair products formed while staging), then S
// accumulates an FP64 GEMM over K = 4 x outer points whose left operand (rho / 2, psi_x) is formed
// from phi, grad phi and w while staging.
#include <algorithm>

#include "xtc_internal.cuh"

namespace xtc {
namespace {

constexpr double K_EPS = 1e-14;

// F(r1, r2) = lap_1 u + |grad_1 u|^2 for u = sum_I sum_t c (a1^m a2^n + a1^n a2^m) b^o,
// a = r / (1 + r) for the electron-nucleus distances, b the same for r12.  Each term is P(a1) Q(b):
// lap(P Q) = Q lap P + P lap Q + 2 grad P . grad Q, and a function f(a(r)) of one distance has
// lap f = f_aa a'^2 + f_a (a'' + 2 a'/r) with a' = (1+r)^-2, a'' = -2 (1+r)^-3.  Unit vectors and
// the 2 a'/r terms are 0 below 1e-14 bohr and everything else is kept, as for the gradient of
// step (a): at a coincident pair (j = i) the electron-nucleus parts stay in the sums.
__device__ double lap_plus_square(const JastrowParams& jp, double x1, double y1, double z1, double x2, double y2,
                                  double z2) {
  const double dx = x1 - x2, dy = y1 - y2, dz = z1 - z2;
  const double r12 = sqrt(dx * dx + dy * dy + dz * dz);
  const double i12 = r12 < K_EPS ? 0.0 : 1.0 / r12;
  const double e12x = dx * i12, e12y = dy * i12, e12z = dz * i12;
  const double s12 = 1.0 / (1.0 + r12);
  const double b = r12 * s12, bp = s12 * s12, bpp = -2.0 * bp * s12;
  const double pb[3] = {1.0, b, b * b};
  double gx = 0.0, gy = 0.0, gz = 0.0, lap = 0.0;
  for (int I = 0; I < jp.n_nuc; ++I) {
    const double vx = x1 - jp.nuc[I][0], vy = y1 - jp.nuc[I][1], vz = z1 - jp.nuc[I][2];
    const double d1 = sqrt(vx * vx + vy * vy + vz * vz);
    const double inv1 = d1 < K_EPS ? 0.0 : 1.0 / d1;
    const double e1x = vx * inv1, e1y = vy * inv1, e1z = vz * inv1;
    const double s1 = 1.0 / (1.0 + d1);
    const double a1 = d1 * s1, ap = s1 * s1, app = -2.0 * ap * s1;
    const double ux = x2 - jp.nuc[I][0], uy = y2 - jp.nuc[I][1], uz = z2 - jp.nuc[I][2];
    const double d2 = sqrt(ux * ux + uy * uy + uz * uz);
    const double a2 = d2 / (1.0 + d2);
    const double p1[3] = {1.0, a1, a1 * a1};
    const double p2[3] = {1.0, a2, a2 * a2};
    const double cosang = e1x * e12x + e1y * e12y + e1z * e12z;
    const double radial1 = app + 2.0 * ap * inv1;   // a'' + 2 a'/r for r1I
    const double radial12 = bpp + 2.0 * bp * i12;   // the same for r12
    const int set = jp.set[I];
    for (int t = 0; t < jp.n_terms; ++t) {
      const int m = jp.mno[t][0], n = jp.mno[t][1], o = jp.mno[t][2];
      const double c = jp.coef[set][t];
      const double P = c * (p1[m] * p2[n] + p1[n] * p2[m]);
      const double Pa = c * ((m > 0 ? m * p1[m - 1] : 0.0) * p2[n] + (n > 0 ? n * p1[n - 1] : 0.0) * p2[m]);
      const double Paa = c * ((m > 1 ? m * (m - 1) * p1[m - 2] : 0.0) * p2[n] +
                              (n > 1 ? n * (n - 1) * p1[n - 2] : 0.0) * p2[m]);
      const double Q = pb[o];
      const double Qb = o > 0 ? o * pb[o - 1] : 0.0;
      const double Qbb = o > 1 ? o * (o - 1) * pb[o - 2] : 0.0;
      const double gP = Pa * ap, gQ = Qb * bp;  // radial derivatives along e1 and e12
      gx += Q * gP * e1x + P * gQ * e12x;
      gy += Q * gP * e1y + P * gQ * e12y;
      gz += Q * gP * e1z + P * gQ * e12z;
      lap += Q * (Paa * ap * ap + Pa * radial1) + P * (Qbb * bp * bp + Qb * radial12) + 2.0 * gP * gQ * cosang;
    }
  }
  return lap + gx * gx + gy * gy + gz * gz;
}

// Ft[j][il] = w_j F(r_{i0+il}, r_j) for j < n_grid, il < n_i (il contiguous).
__global__ void __launch_bounds__(256) kfield_table_kernel(const double* __restrict__ grid,
                                                           const double* __restrict__ w,
                                                           const JastrowParams* __restrict__ jp, int64_t n_grid,
                                                           int64_t i0, int64_t n_i, double* __restrict__ Ft) {
  const int64_t total = n_grid * n_i;
  for (int64_t o = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; o < total;
       o += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t j = o / n_i, il = o - j * n_i;
    const double* ri = grid + 3 * (i0 + il);
    const double* rj = grid + 3 * j;
    Ft[o] = w[j] * lap_plus_square(*jp, ri[0], ri[1], ri[2], rj[0], rj[1], rj[2]);
  }
}

// ------------------------------------------------------------------ FP64 SIMT GEMM
// C[m][n] (+)= sum_k A(k, m) B(k, n) with both operands produced element by element by Op while
// staging: 64 x 64 tiles, 16-deep K steps, 4 x 4 results per thread.  blockIdx.z selects a slice
// [z kslice, (z+1) kslice) of K and an output block C + z zstride (split K for small outputs).
constexpr int KG_T = 64, KG_K = 16;

// W[i][rs] = sum_j Ft[j][i] phi_r(j) phi_s(j)   (m: outer point of the chunk, n: pair, k: inner point)
struct WOperands {
  const double* Ft;
  int64_t ldf;
  const double* phi;
  int n_orb;
  const int* pair_p;
  const int* pair_q;
  __device__ double a(int64_t k, int64_t m) const { return Ft[k * ldf + m]; }
  __device__ double b(int64_t k, int64_t n) const {
    const double* row = phi + k * n_orb;
    return row[pair_p[n]] * row[pair_q[n]];
  }
};

// S[pq][rs] += sum_i sum_c L_c(i, pq) R_c(i, rs), k = 4 i + c:
//   c = 0: L = w phi_p phi_q / 2, R = W_rs;   c = 1..3: L = w phi_p d_x phi_q, R = V_x,rs.
struct SOperands {
  const double* phi;
  const double* dphi;
  const double* w;
  int64_t i0;
  int n_orb, n_pair;
  const double* W;
  const double* V;
  __device__ double a(int64_t k, int64_t m) const {
    const int64_t g = i0 + (k >> 2);
    const int c = static_cast<int>(k & 3);
    const int p = static_cast<int>(m / n_orb), q = static_cast<int>(m - static_cast<int64_t>(p) * n_orb);
    const double wp = w[g] * phi[g * n_orb + p];
    return c == 0 ? 0.5 * wp * phi[g * n_orb + q] : wp * dphi[(g * n_orb + q) * 3 + (c - 1)];
  }
  __device__ double b(int64_t k, int64_t n) const {
    const int64_t i = k >> 2;
    const int c = static_cast<int>(k & 3);
    return c == 0 ? W[i * n_pair + n] : V[(i * 3 + (c - 1)) * n_pair + n];
  }
};

template <class Op, bool ACC>
__global__ void __launch_bounds__(256) gemm_f64_kernel(Op op, int64_t M, int64_t Nn, int64_t K, int64_t kslice,
                                                       double* __restrict__ C, int64_t ldc, int64_t zstride) {
  __shared__ double As[KG_K][KG_T];
  __shared__ double Bs[KG_K][KG_T];
  const int t = threadIdx.x;
  const int tn = t & 15, tm = t >> 4;
  const int64_t m0 = static_cast<int64_t>(blockIdx.y) * KG_T, n0 = static_cast<int64_t>(blockIdx.x) * KG_T;
  const int64_t kb = static_cast<int64_t>(blockIdx.z) * kslice;
  const int64_t ke = kb + kslice < K ? kb + kslice : K;
  C += static_cast<int64_t>(blockIdx.z) * zstride;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (int64_t k0 = kb; k0 < ke; k0 += KG_K) {
    for (int e = t; e < KG_K * KG_T; e += 256) {
      const int kk = e / KG_T, c = e % KG_T;
      const int64_t k = k0 + kk;
      As[kk][c] = (k < ke && m0 + c < M) ? op.a(k, m0 + c) : 0.0;
      Bs[kk][c] = (k < ke && n0 + c < Nn) ? op.b(k, n0 + c) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KG_K; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][tm * 4 + u];
        b[u] = Bs[kk][tn * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t row = m0 + tm * 4 + u;
    if (row >= M) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t col = n0 + tn * 4 + v;
      if (col >= Nn) continue;
      if (ACC)
        C[row * ldc + col] += acc[u][v];
      else
        C[row * ldc + col] = acc[u][v];
    }
  }
}

// Index of the pair (min(p,q), max(p,q)) in the packed order p-major, q >= p (the order of the
// pair tables that V and S use).
__device__ __forceinline__ int64_t k_pair(int p, int q, int N) {
  const int a = min(p, q), b = max(p, q);
  return static_cast<int64_t>(a) * N - static_cast<int64_t>(a) * (a - 1) / 2 + (b - a);
}

// K[p][q][r][s] = S[pq][rs] + S[rs][pq]
__global__ void k_unpack_kernel(const double* __restrict__ S, int N, int NP, double* __restrict__ K) {
  const int64_t n2 = static_cast<int64_t>(N) * N;
  const int64_t total = n2 * n2;
  for (int64_t o = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; o < total;
       o += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t left = o / n2, right = o - left * n2;  // (p, q) and (r, s)
    const int p = static_cast<int>(left / N), q = static_cast<int>(left % N);
    const int r = static_cast<int>(right / N), s = static_cast<int>(right % N);
    K[o] = S[left * NP + k_pair(r, s, N)] + S[right * NP + k_pair(p, q, N)];
  }
}

// C[m][n] (+)= sum_z P[z][m][n], the slices in order (the same result for the same split).
template <bool ACC>
__global__ void slice_sum_kernel(const double* __restrict__ P, int splits, int64_t M, int64_t Nn,
                                 double* __restrict__ C, int64_t ldc) {
  const int64_t total = M * Nn;
  for (int64_t o = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; o < total;
       o += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double sum = 0.0;
    for (int z = 0; z < splits; ++z) sum += P[z * total + o];
    const int64_t m = o / Nn, n = o - m * Nn;
    if (ACC)
      C[m * ldc + n] += sum;
    else
      C[m * ldc + n] = sum;
  }
}

// One GEMM; when its output has fewer tiles than two per SM, K is split into slices (at most 64,
// each at least 8 K steps) whose partial results go to `partial` (room for partial_elems
// doubles) and are summed in order afterwards.
template <class Op, bool ACC>
void launch_gemm(const Op& op, int64_t M, int64_t Nn, int64_t K, double* C, int64_t ldc, double* partial,
                 int64_t partial_elems, int n_sm, cudaStream_t st) {
  const int64_t tm = (M + KG_T - 1) / KG_T, tn = (Nn + KG_T - 1) / KG_T, tiles = tm * tn;
  int64_t splits = 1;
  if (partial && tiles < 2 * static_cast<int64_t>(n_sm))
    splits = std::min<int64_t>(std::min<int64_t>((2 * n_sm + tiles - 1) / tiles, (K + 8 * KG_K - 1) / (8 * KG_K)),
                               64);
  while (splits > 1 && splits * M * Nn > partial_elems) --splits;
  int64_t kslice = K;
  if (splits > 1) {
    kslice = ((K + splits - 1) / splits + KG_K - 1) / KG_K * KG_K;
    splits = (K + kslice - 1) / kslice;
  }
  dim3 grid(static_cast<unsigned>(tn), static_cast<unsigned>(tm), static_cast<unsigned>(splits));
  if (splits <= 1) {
    gemm_f64_kernel<Op, ACC><<<grid, 256, 0, st>>>(op, M, Nn, K, K, C, ldc, 0);
    return;
  }
  gemm_f64_kernel<Op, false><<<grid, 256, 0, st>>>(op, M, Nn, K, kslice, partial, Nn, M * Nn);
  const int64_t blocks = std::min<int64_t>((M * Nn + 255) / 256, static_cast<int64_t>(n_sm) * 16);
  slice_sum_kernel<ACC><<<static_cast<unsigned>(blocks), 256, 0, st>>>(partial, static_cast<int>(splits), M, Nn, C,
                                                                      ldc);
}

}  // namespace

void launch_k_chunk(const double* grid, const double* w, const double* phi, const double* dphi,
                    const JastrowParams* jp_dev, int64_t n_grid, int n_orb, const int* pair_p, const int* pair_q,
                    int64_t i0, int64_t n_i, const double* V, double* Ft, double* W, double* S, double* partial,
                    int64_t partial_elems, int n_sm, cudaStream_t st) {
  const int NP = n_orb * (n_orb + 1) / 2;
  const int64_t total = n_grid * n_i;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, static_cast<int64_t>(n_sm) * 16);
  kfield_table_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(grid, w, jp_dev, n_grid, i0, n_i, Ft);
  const WOperands wop{Ft, n_i, phi, n_orb, pair_p, pair_q};
  launch_gemm<WOperands, false>(wop, n_i, NP, n_grid, W, NP, partial, partial_elems, n_sm, st);
  const SOperands sop{phi, dphi, w, i0, n_orb, NP, W, V};
  launch_gemm<SOperands, true>(sop, static_cast<int64_t>(n_orb) * n_orb, NP, 4 * n_i, S, NP, partial, partial_elems,
                               n_sm, st);
}

void launch_k_unpack(const double* S, int n_orb, double* K, int n_sm, cudaStream_t st) {
  const int NP = n_orb * (n_orb + 1) / 2;
  const int64_t n2 = static_cast<int64_t>(n_orb) * n_orb;
  const int64_t blocks = std::min<int64_t>((n2 * n2 + 255) / 256, static_cast<int64_t>(n_sm) * 32);
  k_unpack_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(S, n_orb, NP, K);
}

}  // namespace xtc
