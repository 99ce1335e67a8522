// Step (c): the per-point intermediates of Appendix B ("Restricted closed-shell working
// equations"), from the vector pair fields V of step (b):
//     rho_pq = w phi_p phi_q            Wt  = 2 rho_tu gamma_tu
//     W_x    = 2 V_x,tu gamma_tu        Vt  = W . V
//     X_x    = gamma V_x                Zt  = V_x . X_x  (= sum_x V_x gamma V_x)
//     Y_x    = V_x gamma                Z_x = rho X_x + Y_x rho
//     A      = Vt - Zt                  B_x = 1/2 Wt V_x - Z_x
// and of Appendix A (restricted open shell) for electron-2 spin t: the same with the direct
// density 2 gamma replaced by gamma^a + gamma^b (in W, Wt) and the exchange density gamma by
// gamma^t (in X, Y, Zt, Z).  The library factorises both on the host over one set of vectors c_k:
// g_d = sum_k lamd_k c_k c_k^T (direct), gamma_x = sum_k lam_k c_k c_k^T (exchange), so that the N^3
// products become rank-r updates: H_xk = V_x c_k, Zt = sum_xk lam_k H_xk H_xk^T,
// W_x = sum_k lamd_k c_k.H_xk, h_x = V_x gamma_x phi = sum_k lam_k (c_k.phi) H_xk,
// Z_x = w (phi h_x^T + h_x phi^T), Wt = w sum_k lamd_k (c_k.phi)^2.  (Exact reformulation.)
// A spin build runs one pass for both spins of electron 2 (SPIN): the factors of gamma^a and
// gamma^b together carry the direct weights (gamma^a + gamma^b), a.lam the alpha exchange weights
// and a.lam2 the beta ones (zero on the other spin's factors); L is written once, R for alpha and
// R2 for beta.
//
// A CTA owns `pts` (8 or fewer) consecutive outer points of one block of V (v_index: the block
// holds the whole N x N matrices of its points, a row p of them one contiguous run) and all orbital
// pairs; lanes run over the points, so a warp reads whole 32-byte pieces of a row.  H for its
// points lives in shared memory.  Outputs, per point and pair, are L = (rho, Vx, Vy, Vz) and R = (A, Bx, By, Bz), written
// as the operands of step (d): FP32 rows [pq][4*gcp], FP64 [4*gcp][pq] or three bf16 parts
// [part][pq][4*gcp].  L does not depend on the density and R is linear in its factors, so a
// density of more factors than one pass holds runs several passes: the first writes L and R, the
// next ones add their R (FP32 and FP64 outputs).
// Points past the chunk end are written as zeros.
#include <cuda_bf16.h>

#include "xtc_internal.cuh"

namespace xtc {
namespace {

constexpr int THREADS = 256;
constexpr int RMAX = 16;
constexpr int U1 = 4;  // phase 1: columns per group (3 V loads each in flight)
constexpr int U2 = 2;  // phase 2: pairs per iteration

template <typename TC>
struct FieldsSmem {
  TC* phis;  // [N][P]
  TC* ws;    // [P]
  TC* cs;    // [R][N]
  TC* lam;   // [R]
  TC* lamd;  // [R]
  TC* cph;   // [R][P]
  TC* Hs;    // [3][R][N][P]
  TC* hs;    // [3][N][P]
  TC* Wv;    // [3][P]
  TC* Wt;    // [P]
  TC* part;  // [3][R][P]
  TC* lam2;  // [R]        (SPIN)
  TC* hs2;   // [3][N][P]  (SPIN)
};

template <typename TC>
__host__ __device__ inline size_t carve(FieldsSmem<TC>* s, uint8_t* base, int N, int R, int P, bool spin) {
  size_t off = 0;
  TC* p[13];
  const size_t n[13] = {static_cast<size_t>(N) * P,
                        static_cast<size_t>(P),
                        static_cast<size_t>(R) * N,
                        static_cast<size_t>(R),
                        static_cast<size_t>(R),
                        static_cast<size_t>(R) * P,
                        static_cast<size_t>(3) * R * N * P,
                        static_cast<size_t>(3) * N * P,
                        static_cast<size_t>(3) * P,
                        static_cast<size_t>(P),
                        static_cast<size_t>(3) * R * P,
                        spin ? static_cast<size_t>(R) : 0,
                        spin ? static_cast<size_t>(3) * N * P : 0};
  for (int k = 0; k < 13; ++k) {
    p[k] = reinterpret_cast<TC*>(base + off);
    off += ((n[k] * sizeof(TC) + 15) / 16) * 16;
  }
  if (s) *s = FieldsSmem<TC>{p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], p[8], p[9], p[10], p[11], p[12]};
  return off;
}

template <typename TV>
__device__ __forceinline__ TV vload(const TV* V, int splits, int64_t split_stride, int64_t idx) {
  // V is read-only while this kernel runs: the non-coherent path lets loads run ahead of stores
  TV v = __ldg(V + idx);
  for (int z = 1; z < splits; ++z) v += __ldg(V + z * split_stride + idx);
  return v;
}

__device__ __forceinline__ void split3_bf16(float v, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// add: FP64 and FP32 outputs are added to what the buffer holds (the R of a further group of
// density factors; R is linear in the factors), else stored.
template <typename TC, int OUT_PARTS>
__device__ __forceinline__ void write4(void* base, int64_t n_pair, int64_t gcp, int q, int64_t il,
                                       const TC (&v)[4], bool add = false) {
  if (OUT_PARTS == 0) {
    double* o = static_cast<double*>(base);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double* e = o + (4 * il + c) * n_pair + q;
      *e = add ? *e + static_cast<double>(v[c]) : static_cast<double>(v[c]);
    }
  } else if (OUT_PARTS == 1) {
    // FP32 rows [pq][4*gcp] (split afterwards with a per-row scale)
    float* o = static_cast<float*>(base) + static_cast<int64_t>(q) * 4 * gcp + 4 * il;
    float4 w = make_float4(static_cast<float>(v[0]), static_cast<float>(v[1]), static_cast<float>(v[2]),
                           static_cast<float>(v[3]));
    if (add) {
      const float4 old = *reinterpret_cast<const float4*>(o);
      w.x += old.x;
      w.y += old.y;
      w.z += old.z;
      w.w += old.w;
    }
    *reinterpret_cast<float4*>(o) = w;
  } else {
    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(base);
    __nv_bfloat16 h[4], m[4], l[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) split3_bf16(static_cast<float>(v[c]), h[c], m[c], l[c]);
    const int64_t part_stride = n_pair * 4 * gcp;
    const int64_t off = static_cast<int64_t>(q) * 4 * gcp + 4 * il;
    uint2 uh, um, ul;
    uh.x = static_cast<uint32_t>(__bfloat16_as_ushort(h[0])) | (static_cast<uint32_t>(__bfloat16_as_ushort(h[1])) << 16);
    uh.y = static_cast<uint32_t>(__bfloat16_as_ushort(h[2])) | (static_cast<uint32_t>(__bfloat16_as_ushort(h[3])) << 16);
    um.x = static_cast<uint32_t>(__bfloat16_as_ushort(m[0])) | (static_cast<uint32_t>(__bfloat16_as_ushort(m[1])) << 16);
    um.y = static_cast<uint32_t>(__bfloat16_as_ushort(m[2])) | (static_cast<uint32_t>(__bfloat16_as_ushort(m[3])) << 16);
    ul.x = static_cast<uint32_t>(__bfloat16_as_ushort(l[0])) | (static_cast<uint32_t>(__bfloat16_as_ushort(l[1])) << 16);
    ul.y = static_cast<uint32_t>(__bfloat16_as_ushort(l[2])) | (static_cast<uint32_t>(__bfloat16_as_ushort(l[3])) << 16);
    *reinterpret_cast<uint2*>(o + off) = uh;
    *reinterpret_cast<uint2*>(o + part_stride + off) = um;
    *reinterpret_cast<uint2*>(o + 2 * part_stride + off) = ul;
  }
}

template <typename TV, typename TC, int OUT_PARTS, bool SPIN>
__global__ void __launch_bounds__(THREADS) fields_kernel(const FieldsArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int N = a.n_orb, R = a.rank, P = a.pts;
  FieldsSmem<TC> sm;
  carve<TC>(&sm, smem_raw, N, R, P, SPIN);
  const int t = threadIdx.x;
  const int pt = t % P, sub = t / P, nsub = THREADS / P;
  const int64_t il = static_cast<int64_t>(blockIdx.x) * P + pt;  // chunk-local outer point
  const bool live = il < a.n_i;
  const TV* V = static_cast<const TV*>(a.V);
  const int64_t sstride = v_slice(a.gcp, N);  // split slices of V

  // ---------------------------------------------------------------- phase 0: orbitals and gamma factors
  for (int k = t; k < N * P; k += THREADS) {
    const int p = k / P, q = k % P;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * P + q;
    sm.phis[k] = i < a.n_i ? static_cast<TC>(a.phiT[static_cast<int64_t>(p) * a.ldphi + a.i0 + i]) : TC(0);
  }
  for (int k = t; k < P; k += THREADS) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * P + k;
    sm.ws[k] = i < a.n_i ? static_cast<TC>(a.w[a.i0 + i]) : TC(0);
  }
  for (int k = t; k < R * N; k += THREADS) sm.cs[k] = static_cast<TC>(a.evec[k]);
  for (int k = t; k < R; k += THREADS) {
    sm.lam[k] = static_cast<TC>(a.lam[k]);
    sm.lamd[k] = static_cast<TC>(a.lamd[k]);
    if (SPIN) sm.lam2[k] = static_cast<TC>(a.lam2[k]);
  }
  __syncthreads();
  for (int k = t; k < R * P; k += THREADS) {
    const int kk = k / P, q = k % P;
    TC acc = 0;
    for (int p = 0; p < N; ++p) acc += sm.cs[kk * N + p] * sm.phis[p * P + q];
    sm.cph[k] = acc;
  }
  __syncthreads();
  for (int q = t; q < P; q += THREADS) {
    TC acc = 0;
    for (int kk = 0; kk < R; ++kk) acc += sm.lamd[kk] * sm.cph[kk * P + q] * sm.cph[kk * P + q];
    sm.Wt[q] = sm.ws[q] * acc;
  }

  // ---------------------------------------------------------------- phase 1: H_xk = V_x c_k, h_x
  // A thread takes row p of the three V_x of its point, one contiguous run of the point block
  // (v_index), U1 columns s at a time (their loads issued before the products), s = 0..N-1 in order.
  const TV* vrow0 = V + (il / VB) * static_cast<int64_t>(N) * N * 3 * VB + (il % VB);
  for (int p = sub; p < N; p += nsub) {
    TC acc[3][RMAX];
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
      for (int kk = 0; kk < RMAX; ++kk) acc[x][kk] = 0;
    const TV* vrow = vrow0 + static_cast<int64_t>(p) * N * 3 * VB;
    for (int s0 = 0; s0 < N; s0 += U1) {
      TC v[U1][3];
#pragma unroll
      for (int u = 0; u < U1; ++u) {
        const int s = s0 + u;
#pragma unroll
        for (int x = 0; x < 3; ++x)
          v[u][x] = (live && s < N) ? static_cast<TC>(vload<TV>(vrow, a.splits, sstride, s * 3 * VB + x * VB)) : TC(0);
      }
#pragma unroll
      for (int u = 0; u < U1; ++u) {
        const int s = min(s0 + u, N - 1);  // v[u] = 0 past the last orbital
#pragma unroll
        for (int kk = 0; kk < RMAX; ++kk)
          if (kk < R) {
            const TC c = sm.cs[kk * N + s];
#pragma unroll
            for (int x = 0; x < 3; ++x) acc[x][kk] += v[u][x] * c;
          }
      }
    }
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      TC h = 0, h2 = 0;
#pragma unroll
      for (int kk = 0; kk < RMAX; ++kk)
        if (kk < R) {
          sm.Hs[((x * R + kk) * N + p) * P + pt] = acc[x][kk];
          h += sm.lam[kk] * sm.cph[kk * P + pt] * acc[x][kk];
          if (SPIN) h2 += sm.lam2[kk] * sm.cph[kk * P + pt] * acc[x][kk];
        }
      sm.hs[(x * N + p) * P + pt] = h;
      if (SPIN) sm.hs2[(x * N + p) * P + pt] = h2;
    }
  }
  __syncthreads();
  // W_x = sum_k lamd_k sum_p c_k[p] H_xk[p]  (deterministic two-level sum)
  for (int k = t; k < 3 * R * P; k += THREADS) {
    const int q = k % P, xk = k / P, kk = xk % R;
    TC acc = 0;
    for (int p = 0; p < N; ++p) acc += sm.cs[kk * N + p] * sm.Hs[(xk * N + p) * P + q];
    sm.part[k] = sm.lamd[kk] * acc;
  }
  __syncthreads();
  for (int k = t; k < 3 * P; k += THREADS) {
    const int x = k / P, q = k % P;
    TC acc = 0;
    for (int kk = 0; kk < R; ++kk) acc += sm.part[(x * R + kk) * P + q];
    sm.Wv[k] = acc;
  }
  __syncthreads();

  // ---------------------------------------------------------------- phase 2: pair outputs
  const TC w = sm.ws[pt];
  const TC wt = sm.Wt[pt];
  const TC W0 = sm.Wv[pt], W1 = sm.Wv[P + pt], W2 = sm.Wv[2 * P + pt];
  // U2 pairs per iteration, their V loads issued first
  for (int q0 = sub; q0 < a.n_pair; q0 += U2 * nsub) {
    TC v[U2][3];
    int pp[U2], ss[U2];
#pragma unroll
    for (int j = 0; j < U2; ++j) {
      const int q = q0 + j * nsub;
      const bool ok = live && q < a.n_pair;
      pp[j] = ok ? __ldg(a.pair_p + q) : 0;
      ss[j] = ok ? __ldg(a.pair_q + q) : 0;
      const int64_t vo = (static_cast<int64_t>(pp[j]) * N + ss[j]) * 3 * VB;
#pragma unroll
      for (int x = 0; x < 3; ++x)
        v[j][x] = ok ? static_cast<TC>(vload<TV>(vrow0, a.splits, sstride, vo + x * VB)) : TC(0);
    }
#pragma unroll
    for (int j = 0; j < U2; ++j) {
      const int q = q0 + j * nsub;
      if (q >= a.n_pair) break;
      TC Lv[4] = {0, 0, 0, 0}, Rv[4] = {0, 0, 0, 0}, R2v[4] = {0, 0, 0, 0};
      if (live) {
        const int p = pp[j], s = ss[j];
        TC zt = 0, zt2 = 0;
        for (int x = 0; x < 3; ++x) {
          const TC* Hp = sm.Hs + (x * R * N + p) * P + pt;
          const TC* Hq = sm.Hs + (x * R * N + s) * P + pt;
#pragma unroll 4
          for (int kk = 0; kk < R; ++kk) {
            if (SPIN) {
              const TC hh = Hp[kk * N * P] * Hq[kk * N * P];
              zt += sm.lam[kk] * hh;
              zt2 += sm.lam2[kk] * hh;
            } else {
              zt += sm.lam[kk] * Hp[kk * N * P] * Hq[kk * N * P];
            }
          }
        }
        const TC vt = W0 * v[j][0] + W1 * v[j][1] + W2 * v[j][2];
        const TC php = sm.phis[p * P + pt], phs = sm.phis[s * P + pt];
        Lv[0] = w * php * phs;
        Lv[1] = v[j][0];
        Lv[2] = v[j][1];
        Lv[3] = v[j][2];
        Rv[0] = vt - zt;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          const TC zx = w * (php * sm.hs[(x * N + s) * P + pt] + sm.hs[(x * N + p) * P + pt] * phs);
          Rv[1 + x] = TC(0.5) * wt * v[j][x] - zx;
        }
        if (SPIN) {
          R2v[0] = vt - zt2;
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            const TC zx = w * (php * sm.hs2[(x * N + s) * P + pt] + sm.hs2[(x * N + p) * P + pt] * phs);
            R2v[1 + x] = TC(0.5) * wt * v[j][x] - zx;
          }
        }
      }
      if (a.write_L) write4<TC, OUT_PARTS>(a.L, a.n_pair, a.gcp, q, il, Lv);
      write4<TC, OUT_PARTS>(a.R, a.n_pair, a.gcp, q, il, Rv, a.add_R);
      if (SPIN) write4<TC, OUT_PARTS>(a.R2, a.n_pair, a.gcp, q, il, R2v, a.add_R);
    }
  }
}

template <typename TV, typename TC, int OUT, bool SPIN>
void launch_t(const FieldsArgs& a, cudaStream_t st) {
  const size_t smem = fields_smem_bytes(a.n_orb, a.rank, a.pts, sizeof(TC) == 8, SPIN);
  auto kern = fields_kernel<TV, TC, OUT, SPIN>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem());
  const int blocks = static_cast<int>(a.gcp / a.pts);
  kern<<<blocks, THREADS, smem, st>>>(a);
}

}  // namespace

size_t fields_smem_bytes(int n_orb, int rank, int pts, bool f64, bool spin) {
  return f64 ? carve<double>(nullptr, nullptr, n_orb, rank, pts, spin)
             : carve<float>(nullptr, nullptr, n_orb, rank, pts, spin);
}

template <bool SPIN>
void launch_spin_t(const FieldsArgs& a, bool f64, cudaStream_t st) {
  if (f64)
    launch_t<double, double, 0, SPIN>(a, st);
  else if (a.out_parts == 1)
    launch_t<float, float, 1, SPIN>(a, st);
  else
    launch_t<float, float, 3, SPIN>(a, st);
}

void launch_fields(const FieldsArgs& a, bool f64, cudaStream_t st) {
  if (a.R2)
    launch_spin_t<true>(a, f64, st);
  else
    launch_spin_t<false>(a, f64, st);
}

}  // namespace xtc
