// Preparation kernels, the FP64 SIMT twins of steps (a)+(b) and (d), and the final kernels
// (Delta U unpacking, the one-body correction and the constant of Appendix B).
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "jastrow_coef.cuh"
#include "simt_pack.cuh"
#include "xtc_internal.cuh"

namespace xtc {
namespace {

__device__ __forceinline__ int pair_of(int p, int q, int N) {
  // packed index of the unordered pair {p, q}
  const int a = min(p, q), b = max(p, q);
  return a * N - a * (a - 1) / 2 + (b - a);
}

// ------------------------------------------------------------------ inner-point tables
__global__ void jtab_kernel(const double* __restrict__ grid, int64_t n_grid, int64_t n_pad,
                            const JastrowParams* __restrict__ jp, int n_nuc, int js, float* __restrict__ jtab) {
  const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (j >= n_pad) return;
  double x = 1.0e3, y = 1.0e3, z = 1.0e3;  // padding points: far away and finite (their rho is zero)
  if (j < n_grid) {
    x = grid[3 * j];
    y = grid[3 * j + 1];
    z = grid[3 * j + 2];
  }
  // Points j = 2k and 2k+1 share a record of 2 js floats, each field stored as an adjacent (even,
  // odd) pair so that one 16-byte load yields two packed fields:
  //   x_hi y_hi | z_hi x_lo | y_lo z_lo | a_0 a_1 | a_2 a_3 | ...      (each entry = [j even, j odd])
  // with x = x_hi + x_lo (differences of nearby points keep FP64-level accuracy in FP32) and
  // a_I = |r_j - R_I| / (1 + |r_j - R_I|); js = 12 holds 4 nuclei, js = 16 holds 8 (+ 2 zero
  // fields); entries past the last nucleus are zero.
  float* o = jtab + (j >> 1) * 2 * js + (j & 1);
  const float xh = static_cast<float>(x), yh = static_cast<float>(y), zh = static_cast<float>(z);
  float f[16] = {xh, yh, zh, static_cast<float>(x - static_cast<double>(xh)),
                 static_cast<float>(y - static_cast<double>(yh)), static_cast<float>(z - static_cast<double>(zh))};
  for (int k = 6; k < 16; ++k) f[k] = 0.0f;
  for (int I = 0; I < n_nuc && I < js - 6 && I < 8; ++I) {
    const double dx = x - jp->nuc[I][0], dy = y - jp->nuc[I][1], dz = z - jp->nuc[I][2];
    const double d = sqrt(dx * dx + dy * dy + dz * dz);
    f[6 + I] = static_cast<float>(d / (1.0 + d));
  }
  for (int k = 0; k < js && k < 16; ++k) o[2 * k] = f[k];
}

__global__ void transpose_phi_kernel(const double* __restrict__ phi, int64_t n_grid, int64_t n_pad, int N,
                                     double* __restrict__ phiT) {
  __shared__ double tile[32][33];
  const int64_t j0 = blockIdx.x * 32ll;
  const int p0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t j = j0 + k;
    const int p = p0 + threadIdx.x;
    tile[k][threadIdx.x] = (j < n_grid && p < N) ? phi[j * N + p] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int p = p0 + k;
    const int64_t j = j0 + threadIdx.x;
    if (p < N && j < n_pad) phiT[p * n_pad + j] = tile[threadIdx.x][k];
  }
}

__global__ void check_finite_kernel(const double* __restrict__ x, int64_t n, int* flag) {
  int bad = 0;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x)
    bad |= !isfinite(x[k]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

// ------------------------------------------------------------------ pair products rho
// colmax[pq] = max_j |w_j phi_p(j) phi_q(j)| (as float bits; values are non-negative)
// power-of-2 exponent that brings the column maximum near 2^14 (fp16 split); 0 when unscaled
__device__ __forceinline__ int col_exponent(const unsigned int* colmax, int pq, bool scale) {
  if (!scale) return 0;
  const float m = __uint_as_float(colmax[pq]);
  if (!(m > 0.0f)) return 0;
  int e;
  frexpf(m, &e);           // m = f * 2^e, f in [0.5, 1)
  return min(max(14 - e, -60), 60);
}

// Orbitals and weights as FP32 pairs hi + lo (hi = the value rounded to FP32, lo = the FP32
// rounding of the rest): row r < n_orb of dst is phi_r, row n_orb the weights; dst[part][row][j].
__global__ void split_phi_f32_kernel(const double* __restrict__ phiT, const double* __restrict__ w, int64_t n_grid,
                                     int64_t n_pad, int n_orb, float* __restrict__ dst) {
  const int64_t rows = static_cast<int64_t>(n_orb) + 1, total = rows * n_pad;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < total;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = k / n_pad, j = k % n_pad;
    const double v = r < n_orb ? phiT[k] : (j < n_grid ? w[j] : 0.0);
    const float hi = static_cast<float>(v);
    dst[k] = hi;
    dst[total + k] = static_cast<float>(v - static_cast<double>(hi));
  }
}

// w phi_p phi_q from the FP32 pairs of split_phi_f32_kernel as an unevaluated sum rh + rl (error-
// free products by fma, then one renormalisation): about 2^-44 of the value, on the FP32 pipes.
__device__ __forceinline__ void rho_pair_f32(const float* __restrict__ f32, int64_t total, int64_t n_pad, int n_orb,
                                             int p, int q, int64_t j, float& rh, float& rl) {
  const float ah = f32[p * n_pad + j], al = f32[total + p * n_pad + j];
  const float bh = f32[q * n_pad + j], bl = f32[total + q * n_pad + j];
  const float wh = f32[n_orb * n_pad + j], wl = f32[total + n_orb * n_pad + j];
  const float xh = ah * bh;
  const float xl = fmaf(ah, bh, -xh) + fmaf(ah, bl, al * bh);
  const float yh = xh * wh;
  const float yl = fmaf(xh, wh, -yh) + fmaf(xh, wl, xl * wh);
  rh = yh + yl;
  rl = yl - (rh - yh);
}

// Largest |rho| of each pair over the grid (FP32; it only picks the pair's power-of-2 scale).
__global__ void rho_colmax_f32_kernel(const float* __restrict__ f32, int64_t n_grid, int64_t n_pad, int n_orb,
                                      const int* __restrict__ pp, const int* __restrict__ pq_,
                                      unsigned int* __restrict__ colmax) {
  const int pq = blockIdx.y;
  const int p = pp[pq], q = pq_[pq];
  const int64_t total = (static_cast<int64_t>(n_orb) + 1) * n_pad;
  float m = 0.0f;
  for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n_grid;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float rh, rl;
    rho_pair_f32(f32, total, n_pad, n_orb, p, q, j, rh, rl);
    m = fmaxf(m, fabsf(rh));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(colmax + pq, __float_as_uint(m));
}

// fp16 (2 parts, exact split): warp w of the CTA handles pair pq = 8 * blockIdx.y + w over one
// accumulation range of the GEMM, points j0 + lane + 32 s (s < kd, j0 = 32 kd blockIdx.x); the
// range shares one quantum (largest |value| of the range, `bits` bits).  rho = rh + rl in FP32
// pairs (rho_pair_f32); hi = rh rounded to the quantum (exact), lo = fp16((rh - hi) + rl), whose
// rounding error is far below fp16's.  Layout: the two parts of a 32-point block share one 128-byte
// row, [pq][j / 32][part][j % 32]; then the plane [pq][j] of the value rounded to fp16.
__global__ void rho_split_f16_kernel(const float* __restrict__ f32, int64_t n_grid, int64_t n_pad, int n_orb,
                                     int n_pair, const int* __restrict__ pp, const int* __restrict__ pq_,
                                     const unsigned int* __restrict__ colmax, int kd, int bits,
                                     int* __restrict__ colexp, uint16_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int pq = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (pq >= n_pair) return;  // whole warp
  const int e = col_exponent(colmax, pq, true);
  if (blockIdx.x == 0 && lane == 0) colexp[pq] = e;
  const int p = pp[pq], q = pq_[pq];
  const int64_t j0 = static_cast<int64_t>(blockIdx.x) * 32 * kd;
  const int64_t total = (static_cast<int64_t>(n_orb) + 1) * n_pad;
  const float sc = pow2f(e);  // |e| <= 60: exact scaling
  float vh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, vl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  float m = 0.0f;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int64_t j = j0 + 32 * s + lane;
    if (s < kd && j < n_grid) {
      float rh, rl;
      rho_pair_f32(f32, total, n_pad, n_orb, p, q, j, rh, rl);
      vh[s] = rh * sc;
      vl[s] = rl * sc;
    }
    m = fmaxf(m, fabsf(vh[s]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int qe = exact_quantum(m, bits);
  uint16_t* out16 = out + static_cast<int64_t>(n_pair) * 2 * n_pad;  // the fp16(rho) plane
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int64_t j = j0 + 32 * s + lane;
    if (s >= kd || j >= n_pad) break;
    float h = 0.0f;
    if (qe >= -24) h = rintf(vh[s] * pow2f(-qe)) * pow2f(qe);  // both products exact (powers of 2)
    const int64_t o = static_cast<int64_t>(pq) * 2 * n_pad + (j >> 5) * 64 + (j & 31);
    out[o] = __half_as_ushort(__float2half_rn(h));                      // exact: at most 10 bits
    out[o + 32] = __half_as_ushort(__float2half_rn((vh[s] - h) + vl[s]));  // vh - h is exact
    out16[static_cast<int64_t>(pq) * n_pad + j] = __half_as_ushort(__float2half_rn(vh[s]));
  }
}

// bf16 (3 parts): per-element split with a plain power-of-2 scale of 1 (no exact ranges), one
// plane per part: [part][pq][j].
__global__ void rho_split_bf16_kernel(const double* __restrict__ phiT, const double* __restrict__ w, int64_t n_grid,
                                      int64_t n_pad, int n_pair, const int* __restrict__ pp,
                                      const int* __restrict__ pq_, int* __restrict__ colexp,
                                      uint16_t* __restrict__ out) {
  const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int pq0 = blockIdx.y * 8;
  const int64_t part_stride = static_cast<int64_t>(n_pair) * n_pad;
  for (int u = 0; u < 8; ++u) {
    const int pq = pq0 + u;
    if (pq >= n_pair) break;
    if (j == 0) colexp[pq] = 0;
    if (j >= n_pad) continue;
    const int p = pp[pq], q = pq_[pq];
    const double v = j < n_grid ? w[j] * phiT[p * n_pad + j] * phiT[q * n_pad + j] : 0.0;
    const int64_t o = static_cast<int64_t>(pq) * n_pad + j;
    const __nv_bfloat16 h = __double2bfloat16(v);
    const double r1 = v - static_cast<double>(__bfloat162float(h));
    const __nv_bfloat16 mm = __double2bfloat16(r1);
    const __nv_bfloat16 l = __double2bfloat16(r1 - static_cast<double>(__bfloat162float(mm)));
    out[o] = __bfloat16_as_ushort(h);
    out[part_stride + o] = __bfloat16_as_ushort(mm);
    out[2 * part_stride + o] = __bfloat16_as_ushort(l);
  }
}

// One CTA per row of a step (d) operand: the row maximum sets a power-of-2 scale, then the scaled
// row is split exactly into fp16 hi + lo (simt_pack.cuh), one quantum per accumulation range of kd
// blocks of 32 values (`bits` bits).  With kc = 4 the source row holds kc values per outer point
// (k = kc * i + c) and the split row is written component-major (k' = c * (kdim / kc) + i), so that
// a range never mixes components; with kc = 1 the order is kept.
__global__ void __launch_bounds__(256) lr_split_kernel(const float* __restrict__ src, int64_t kdim, int kc, int kd,
                                                       int bits, uint16_t* __restrict__ dst, int* __restrict__ exps,
                                                       uint16_t* __restrict__ dst16) {
  __shared__ float red[8];
  const int64_t r = blockIdx.x;
  const float* s = src + r * kdim;
  float m = 0.0f;
  for (int64_t k = threadIdx.x * 4; k < kdim; k += blockDim.x * 4) {
    const float4 v = *reinterpret_cast<const float4*>(s + k);
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = red[0];
  for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
  int e = 0;
  if (m > 0.0f) {
    int em;
    frexpf(m, &em);  // m = f * 2^em, f in [0.5, 1)
    e = min(max(14 - em, -100), 100);
  }
  if (threadIdx.x == 0) exps[r] = e;
  const float scale = ldexpf(1.0f, e);  // exact power of 2 (|e| <= 100)
  uint16_t* d = dst + r * 2 * kdim;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t per_c = kdim / kc;           // outer points (kc = 4) or values (kc = 1) per component
  // warp g handles the source points 32 kd g .. 32 kd (g + 1) - 1 (all kc components of each)
  for (int64_t g = warp; g < per_c / (32 * kd); g += 8) {
    float v[4][4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int64_t i = 32 * (kd * g + t) + lane;
      v[t][0] = v[t][1] = v[t][2] = v[t][3] = 0.0f;
      if (t >= kd) continue;
      if (kc == 4) {
        const float4 q4 = *reinterpret_cast<const float4*>(s + 4 * i);
        v[t][0] = q4.x * scale;
        v[t][1] = q4.y * scale;
        v[t][2] = q4.z * scale;
        v[t][3] = q4.w * scale;
      } else {
        v[t][0] = s[i] * scale;
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (c >= kc) break;
      float bm = 0.0f;
#pragma unroll
      for (int t = 0; t < 4; ++t) bm = fmaxf(bm, fabsf(v[t][c]));
      for (int o = 16; o > 0; o >>= 1) bm = fmaxf(bm, __shfl_xor_sync(0xffffffffu, bm, o));
      const int qe = exact_quantum(bm, bits);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (t >= kd) break;
        __half h, l;
        split_exact(v[t][c], qe, h, l);
        const int64_t kk = c * per_c + 32 * (kd * g + t);  // first value of the 32-value block
        const int64_t blk = kk >> 5;
        d[blk * 64 + lane] = __half_as_ushort(h);
        d[blk * 64 + 32 + lane] = __half_as_ushort(l);
        if (dst16) dst16[r * kdim + kk + lane] = __half_as_ushort(__float2half_rn(v[t][c]));
      }
    }
  }
}

__global__ void rho_f64_kernel(const double* __restrict__ phi, const double* __restrict__ w, int64_t n_grid,
                               int64_t n_pad, int N, int n_pair, const int* __restrict__ pp,
                               const int* __restrict__ pq_, double* __restrict__ rho) {
  const int64_t j = blockIdx.x;
  for (int pq = blockIdx.y * blockDim.x + threadIdx.x; pq < n_pair; pq += gridDim.y * blockDim.x) {
    double v = 0.0;
    if (j < n_grid) v = w[j] * phi[j * N + pp[pq]] * phi[j * N + pq_[pq]];
    rho[j * n_pair + pq] = v;
  }
}

// ------------------------------------------------------------------ step (a) alone, FP64
__global__ void jastrow_grad_kernel(const JastrowParams* __restrict__ jp, const double* __restrict__ r1,
                                    const double* __restrict__ r2, int64_t n, double* __restrict__ out) {
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= n) return;
  double pc[PT_COEF];
  double nc[MAX_NUC * NUC_COEF];
  double aj[MAX_NUC];
  point_coefs<double>(*jp, r1[3 * k], r1[3 * k + 1], r1[3 * k + 2], 1.0, pc, nc, 0, jp->n_nuc);
  const double x = r2[3 * k], y = r2[3 * k + 1], z = r2[3 * k + 2];
  for (int I = 0; I < jp->n_nuc; ++I) {
    const double dx = x - jp->nuc[I][0], dy = y - jp->nuc[I][1], dz = z - jp->nuc[I][2];
    const double d = sqrt(dx * dx + dy * dy + dz * dz);
    aj[I] = d / (1.0 + d);
  }
  double gx, gy, gz;
  pair_grad_f64(pc, nc, jp->n_nuc, x, y, z, aj, gx, gy, gz);
  out[3 * k] = gx;
  out[3 * k + 1] = gy;
  out[3 * k + 2] = gz;
}

// ------------------------------------------------------------------ steps (a)+(b), FP64 SIMT
// CTA: 32 outer points x 64 pairs x 3 components; K steps of 16 inner points.  The gradient
// tile is generated in shared memory from per-point coefficients (computed once per CTA) and a
// per-inner-point FP64 table (x, y, z, a_jI...).
constexpr int F64_TI = 32, F64_TP = 64, F64_KJ = 16;

__global__ void jtab64_kernel(const double* __restrict__ grid, int64_t n_grid, int64_t n_pad,
                              const JastrowParams* __restrict__ jp, int n_nuc, double* __restrict__ jtab) {
  const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (j >= n_pad) return;
  double x = 1.0e3, y = 1.0e3, z = 1.0e3;
  if (j < n_grid) {
    x = grid[3 * j];
    y = grid[3 * j + 1];
    z = grid[3 * j + 2];
  }
  double* o = jtab + j * (3 + n_nuc);
  o[0] = x;
  o[1] = y;
  o[2] = z;
  for (int I = 0; I < n_nuc; ++I) {
    const double dx = x - jp->nuc[I][0], dy = y - jp->nuc[I][1], dz = z - jp->nuc[I][2];
    const double d = sqrt(dx * dx + dy * dy + dz * dz);
    o[3 + I] = d / (1.0 + d);
  }
}

__global__ void __launch_bounds__(256) vfield_f64_kernel(const double* __restrict__ grid,
                                                          const JastrowParams* __restrict__ jp,
                                                          const double* __restrict__ jtab64,
                                                          const double* __restrict__ rho, int64_t n_pad, int n_pair,
                                                          int64_t i0, int64_t n_i, int64_t gcp,
                                                          const int* __restrict__ pair_p,
                                                          const int* __restrict__ pair_q, int n_orb,
                                                          double* __restrict__ V) {
  extern __shared__ double sm64[];
  const int n_nuc = jp->n_nuc;
  const int cstride = PT_COEF + NUC_COEF * n_nuc;
  double* coef = sm64;                                  // [TI][cstride]
  double* Gs = coef + F64_TI * cstride;                 // [KJ][3][TI]
  double* Rs = Gs + F64_KJ * 3 * F64_TI;                // [KJ][TP]
  const int t = threadIdx.x;
  const int64_t ib = static_cast<int64_t>(blockIdx.x) * F64_TI;
  const int pb = blockIdx.y * F64_TP;
  if (t < F64_TI) {
    const int64_t il = ib + t;
    const int64_t ig = i0 + (il < n_i ? il : n_i - 1);
    double* c = coef + t * cstride;
    point_coefs<double>(*jp, grid[3 * ig], grid[3 * ig + 1], grid[3 * ig + 2], 1.0, c, c + PT_COEF, 0, n_nuc);
  }
  __syncthreads();
  const int tx = t & 31, ty = t >> 5;  // pairs tx, tx+32; points ty*4 .. ty*4+3
  double acc[4][2][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int x = 0; x < 3; ++x) acc[a][b][x] = 0.0;
  const int js = 3 + n_nuc;
  for (int64_t j0 = 0; j0 < n_pad; j0 += F64_KJ) {
    for (int k = t; k < F64_KJ * F64_TI; k += 256) {
      const int jj = k / F64_TI, ii = k % F64_TI;
      const double* jr = jtab64 + (j0 + jj) * js;
      const double* c = coef + ii * cstride;
      double gx, gy, gz;
      pair_grad_f64(c, c + PT_COEF, n_nuc, jr[0], jr[1], jr[2], jr + 3, gx, gy, gz);
      Gs[(jj * 3 + 0) * F64_TI + ii] = gx;
      Gs[(jj * 3 + 1) * F64_TI + ii] = gy;
      Gs[(jj * 3 + 2) * F64_TI + ii] = gz;
    }
    for (int k = t; k < F64_KJ * F64_TP; k += 256) {
      const int jj = k / F64_TP, pp = k % F64_TP;
      Rs[k] = (pb + pp < n_pair) ? rho[(j0 + jj) * n_pair + pb + pp] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < F64_KJ; ++jj) {
      const double r0 = Rs[jj * F64_TP + tx], r1 = Rs[jj * F64_TP + tx + 32];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          const double g = Gs[(jj * 3 + x) * F64_TI + ty * 4 + a];
          acc[a][0][x] = fma(g, r0, acc[a][0][x]);
          acc[a][1][x] = fma(g, r1, acc[a][1][x]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t il = ib + ty * 4 + a;
    if (il >= n_i) continue;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int pq = pb + tx + 32 * b;
      if (pq >= n_pair) continue;
      const int p = pair_p[pq], q = pair_q[pq];
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        V[v_index(il, p, q, x, n_orb)] = acc[a][b][x];
        V[v_index(il, q, p, x, n_orb)] = acc[a][b][x];
      }
    }
  }
}

// ------------------------------------------------------------------ step (d), FP64 SIMT
// M[pq][rs] += sum_k L[k][pq] R[k][rs]; 64 x 64 tiles, 16-deep K steps, 4 x 4 per thread.
__global__ void __launch_bounds__(256) assemble_f64_kernel(const double* __restrict__ L,
                                                            const double* __restrict__ R, int n_pair, int kdim,
                                                            int ldm, double* __restrict__ M) {
  __shared__ double Ls[16][64];
  __shared__ double Rs[16][64];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < kdim; k0 += 16) {
    for (int k = t; k < 16 * 64; k += 256) {
      const int kk = k / 64, c = k % 64;
      const int64_t row = static_cast<int64_t>(k0 + kk) * n_pair;
      Ls[kk][c] = (k0 + kk < kdim && m0 + c < n_pair) ? L[row + m0 + c] : 0.0;
      Rs[kk][c] = (k0 + kk < kdim && n0 + c < n_pair) ? R[row + n0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = Ls[kk][ty * 4 + u];
        b[u] = Rs[kk][tx * 4 + u];
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
    const int row = m0 + ty * 4 + u;
    if (row >= n_pair) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int col = n0 + tx * 4 + v;
      if (col < n_pair) M[static_cast<int64_t>(row) * ldm + col] += acc[u][v];
    }
  }
}

// ------------------------------------------------------------------ final kernels
// In place: M <- Delta U = -(M + M^T) (packed pairs), one CTA per pair of 32 x 32 tiles.
__global__ void symmetrize_kernel(double* __restrict__ M, int n_pair, int ldm) {
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj < bi) return;
  __shared__ double A[32][33], B[32][33];
  const int i0 = bi * 32, j0 = bj * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int ri = i0 + r, rj = j0 + r, ci = j0 + threadIdx.x, cj = i0 + threadIdx.x;
    A[r][threadIdx.x] = (ri < n_pair && ci < n_pair) ? M[static_cast<int64_t>(ri) * ldm + ci] : 0.0;
    B[r][threadIdx.x] = (rj < n_pair && cj < n_pair) ? M[static_cast<int64_t>(rj) * ldm + cj] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int ri = i0 + r, ci = j0 + threadIdx.x;
    if (ri < n_pair && ci < n_pair) M[static_cast<int64_t>(ri) * ldm + ci] = -(A[r][threadIdx.x] + B[threadIdx.x][r]);
    const int rj = j0 + r, cj = i0 + threadIdx.x;
    if (bi != bj && rj < n_pair && cj < n_pair)
      M[static_cast<int64_t>(rj) * ldm + cj] = -(B[r][threadIdx.x] + A[threadIdx.x][r]);
  }
}

// dU[p][q][r][s] = U[pair(p,q)][pair(r,s)]
__global__ void unpack_kernel(const double* __restrict__ U, int N, int ldm, double* __restrict__ dU,
                              float* __restrict__ dU32) {
  const int64_t n2 = static_cast<int64_t>(N) * N;
  const int64_t rs = blockIdx.y * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t pqi = blockIdx.x;
  if (rs >= n2) return;
  const int p = static_cast<int>(pqi / N), q = static_cast<int>(pqi % N);
  const int r = static_cast<int>(rs / N), s = static_cast<int>(rs % N);
  const double v = U[static_cast<int64_t>(pair_of(p, q, N)) * ldm + pair_of(r, s, N)];
  const int64_t o = pqi * n2 + rs;
  if (dU) dU[o] = v;
  if (dU32) dU32[o] = static_cast<float>(v);
}

// Delta h_pq = -1/2 (2 sum_rs U(pq|rs) gamma_rs - sum_rs U(ps|rq) gamma_rs), one CTA per (p, q).
__global__ void onebody_kernel(const double* __restrict__ U, const double* __restrict__ gamma, int N, int ldm,
                               double* __restrict__ dh) {
  const int p = blockIdx.y, q = blockIdx.x;
  const int pq = pair_of(p, q, N);
  double acc = 0.0;
  for (int k = threadIdx.x; k < N * N; k += blockDim.x) {
    const int r = k / N, s = k % N;
    const double g = gamma[k];
    acc += g * (2.0 * U[static_cast<int64_t>(pq) * ldm + pair_of(r, s, N)] -
                U[static_cast<int64_t>(pair_of(p, s, N)) * ldm + pair_of(r, q, N)]);
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) dh[p * N + q] = -0.5 * red[0];
}

// Spin builds (Appendix A): U[pq][rs] = -(Fb[pq][rs] + Fa[rs][pq]) = Delta U^{ab}(pq|rs), where
// Ft[pq][rs] = sum_i rho_pq A^t_rs + V_pq.B^t_rs; one CTA per 32 x 32 tile of U.
__global__ void spin_cross_kernel(const double* __restrict__ Fb, const double* __restrict__ Fa, int n_pair, int ldm,
                                  double* __restrict__ U) {
  __shared__ double T[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int ra = j0 + r, ca = i0 + threadIdx.x;  // T[r][x] = Fa[j0 + r][i0 + x]
    T[r][threadIdx.x] = (ra < n_pair && ca < n_pair) ? Fa[static_cast<int64_t>(ra) * ldm + ca] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int row = i0 + r, col = j0 + threadIdx.x;
    if (row < n_pair && col < n_pair)
      U[static_cast<int64_t>(row) * ldm + col] = -(Fb[static_cast<int64_t>(row) * ldm + col] + T[threadIdx.x][r]);
  }
}

// Delta h^s_pq = -1/2 (sum_rs U^{ss}(pq|rs) g^s_rs + sum_rs U^{st}(pq|rs) g^t_rs - sum_rs U^{ss}(ps|rq) g^s_rs),
// t the other spin, U^{ba}(pq|rs) = U^{ab}(rs|pq) (Appendix A); one CTA per (p, q, s).
__global__ void onebody_spin_kernel(const double* __restrict__ Uaa, const double* __restrict__ Uab,
                                    const double* __restrict__ Ubb, const double* __restrict__ ga,
                                    const double* __restrict__ gb, int N, int ldm, double* __restrict__ dh_a,
                                    double* __restrict__ dh_b) {
  const int p = blockIdx.y, q = blockIdx.x, sp = blockIdx.z;
  const double* Us = sp ? Ubb : Uaa;
  const double* gs = sp ? gb : ga;
  const double* go = sp ? ga : gb;
  const int pq = pair_of(p, q, N);
  double acc = 0.0;
  for (int k = threadIdx.x; k < N * N; k += blockDim.x) {
    const int r = k / N, s = k % N;
    const int rs = pair_of(r, s, N);
    const double cross = sp ? Uab[static_cast<int64_t>(rs) * ldm + pq] : Uab[static_cast<int64_t>(pq) * ldm + rs];
    acc += gs[k] * (Us[static_cast<int64_t>(pq) * ldm + rs] -
                    Us[static_cast<int64_t>(pair_of(p, s, N)) * ldm + pair_of(r, q, N)]) +
           go[k] * cross;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) (sp ? dh_b : dh_a)[p * N + q] = -0.5 * red[0];
}

// e0 = -1/3 sum_pq (Delta h^a_pq gamma^a_pq + Delta h^b_pq gamma^b_pq)  (Appendix A)
__global__ void constant_spin_kernel(const double* __restrict__ dh_a, const double* __restrict__ ga,
                                     const double* __restrict__ dh_b, const double* __restrict__ gb, int n2,
                                     double* __restrict__ e0) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < n2; k += blockDim.x) acc += dh_a[k] * ga[k] + dh_b[k] * gb[k];
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *e0 = -1.0 / 3.0 * red[0];
}

// e0 = -2/3 sum_pq Delta h_pq gamma_pq
__global__ void constant_kernel(const double* __restrict__ dh, const double* __restrict__ gamma, int n2,
                                double* __restrict__ e0) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < n2; k += blockDim.x) acc += dh[k] * gamma[k];
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *e0 = -2.0 / 3.0 * red[0];
}

template <typename TV>
__global__ void vfield_export_kernel(const TV* __restrict__ V, int splits, int n_pair, int n_orb,
                                     const int* __restrict__ pair_p, const int* __restrict__ pair_q, int64_t n_i,
                                     int64_t gcp, double* __restrict__ out) {
  const int64_t total = n_i * 3 * n_pair;
  const int64_t sstride = v_slice(gcp, n_orb);
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < total;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t pq = k % n_pair, i = k / (3 * n_pair);
    const int x = static_cast<int>((k / n_pair) % 3);
    const int64_t idx = v_index(i, pair_p[pq], pair_q[pq], x, n_orb);
    double v = 0.0;
    for (int z = 0; z < splits; ++z) v += static_cast<double>(V[z * sstride + idx]);
    out[k] = v;
  }
}

inline unsigned int blocks_for(int64_t n, int bs) { return static_cast<unsigned int>((n + bs - 1) / bs); }

}  // namespace

// ------------------------------------------------------------------ launchers
void launch_jtab(const double* grid, int64_t n_grid, int64_t n_pad, const JastrowParams* jp, int n_nuc, int js,
                 float* jtab, cudaStream_t st) {
  jtab_kernel<<<blocks_for(n_pad, 256), 256, 0, st>>>(grid, n_grid, n_pad, jp, n_nuc, js, jtab);
}

void launch_transpose_phi(const double* phi, int64_t n_grid, int64_t n_pad, int N, double* phiT, cudaStream_t st) {
  dim3 grid(blocks_for(n_pad, 32), blocks_for(N, 32));
  transpose_phi_kernel<<<grid, dim3(32, 8), 0, st>>>(phi, n_grid, n_pad, N, phiT);
}

void launch_check_finite(const double* x, int64_t n, int* flag, cudaStream_t st) {
  if (n <= 0) return;
  const unsigned int b = std::min<unsigned int>(blocks_for(n, 256), 4096u);
  check_finite_kernel<<<b, 256, 0, st>>>(x, n, flag);
}

void launch_rho_split(const double* phiT, const double* w, int64_t n_grid, int64_t n_pad, int n_orb, int parts, int kd,
                      const int* pp, const int* pq, unsigned int* colmax, int* colexp, float* phi32, void* out,
                      cudaStream_t st) {
  const int n_pair = n_orb * (n_orb + 1) / 2;
  if (parts == 2) {
    const int64_t total = (static_cast<int64_t>(n_orb) + 1) * n_pad;
    split_phi_f32_kernel<<<std::min<unsigned int>(blocks_for(total, 256), 8192u), 256, 0, st>>>(phiT, w, n_grid,
                                                                                                n_pad, n_orb, phi32);
    cudaMemsetAsync(colmax, 0, sizeof(unsigned int) * n_pair, st);
    dim3 g(std::min<unsigned int>(blocks_for(n_grid, 256), 64u), n_pair);
    rho_colmax_f32_kernel<<<g, 256, 0, st>>>(phi32, n_grid, n_pad, n_orb, pp, pq, colmax);
    dim3 g2(static_cast<unsigned int>(n_pad / (32 * kd)), blocks_for(n_pair, 8));
    rho_split_f16_kernel<<<g2, 256, 0, st>>>(phi32, n_grid, n_pad, n_orb, n_pair, pp, pq, colmax, kd,
                                              gemm_bits_b(kd), colexp, static_cast<uint16_t*>(out));
  } else {
    dim3 g2(blocks_for(n_pad, 256), blocks_for(n_pair, 8));
    rho_split_bf16_kernel<<<g2, 256, 0, st>>>(phiT, w, n_grid, n_pad, n_pair, pp, pq, colexp,
                                               static_cast<uint16_t*>(out));
  }
}

void launch_lr_split(const float* src, int rows, int64_t kdim, int kc, int kd, uint16_t* dst, int* exps,
                     uint16_t* dst16, cudaStream_t st) {
  if (rows <= 0) return;
  lr_split_kernel<<<rows, 256, 0, st>>>(src, kdim, kc, kd, gemm_bits_lr(kd), dst, exps, dst16);
}

void launch_rho_f64(const double* phi, const double* w, int64_t n_grid, int64_t n_pad, int n_orb, const int* pp,
                    const int* pq, double* rho, cudaStream_t st) {
  const int n_pair = n_orb * (n_orb + 1) / 2;
  dim3 g(static_cast<unsigned int>(n_pad), std::min<unsigned int>(blocks_for(n_pair, 256), 65535u));
  rho_f64_kernel<<<g, 256, 0, st>>>(phi, w, n_grid, n_pad, n_orb, n_pair, pp, pq, rho);
}

void launch_jastrow_grad(const JastrowParams* jp, const double* r1, const double* r2, int64_t n, double* out,
                         cudaStream_t st) {
  jastrow_grad_kernel<<<blocks_for(n, 64), 64, 0, st>>>(jp, r1, r2, n, out);
}

void launch_jtab64(const double* grid, int64_t n_grid, int64_t n_pad, const JastrowParams* jp, int n_nuc,
                   double* jtab, cudaStream_t st) {
  jtab64_kernel<<<blocks_for(n_pad, 256), 256, 0, st>>>(grid, n_grid, n_pad, jp, n_nuc, jtab);
}

void launch_vfield_f64_impl(const double* grid, const JastrowParams* jp, int n_nuc, const double* jtab64,
                            const double* rho, int64_t n_pad, int n_pair, int64_t i0, int64_t n_i, int64_t gcp,
                            const int* pair_p, const int* pair_q, int n_orb, double* V, cudaStream_t st) {
  const size_t smem = sizeof(double) * (F64_TI * (PT_COEF + NUC_COEF * n_nuc) + F64_KJ * 3 * F64_TI + F64_KJ * F64_TP);
  cudaFuncSetAttribute(vfield_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn_smem());
  dim3 g(blocks_for(n_i, F64_TI), blocks_for(n_pair, F64_TP));
  vfield_f64_kernel<<<g, 256, smem, st>>>(grid, jp, jtab64, rho, n_pad, n_pair, i0, n_i, gcp, pair_p, pair_q, n_orb,
                                          V);
}

void launch_assemble_f64(const double* L, const double* R, int n_pair, int kdim, double* M, cudaStream_t st) {
  const int ldm = static_cast<int>(m_stride(n_pair));
  dim3 g(blocks_for(n_pair, 64), blocks_for(n_pair, 64));
  assemble_f64_kernel<<<g, 256, 0, st>>>(L, R, n_pair, kdim, ldm, M);
}

void launch_unpack(const double* M, int n_orb, int n_pair, double* dU, float* dU32, cudaStream_t st) {
  const int ldm = static_cast<int>(m_stride(n_pair));
  if (dU || dU32) {
    dim3 g(static_cast<unsigned int>(n_orb) * n_orb, blocks_for(static_cast<int64_t>(n_orb) * n_orb, 256));
    unpack_kernel<<<g, 256, 0, st>>>(M, n_orb, ldm, dU, dU32);
  }
}

void launch_symmetrize(double* M, int n_pair, cudaStream_t st) {
  const int ldm = static_cast<int>(m_stride(n_pair));
  dim3 g(blocks_for(n_pair, 32), blocks_for(n_pair, 32));
  symmetrize_kernel<<<g, dim3(32, 8), 0, st>>>(M, n_pair, ldm);
}

void launch_onebody(const double* M, const double* gamma, int n_orb, int n_pair, double* dh, double* e0,
                    cudaStream_t st) {
  const int ldm = static_cast<int>(m_stride(n_pair));
  onebody_kernel<<<dim3(n_orb, n_orb), 256, 0, st>>>(M, gamma, n_orb, ldm, dh);
  constant_kernel<<<1, 256, 0, st>>>(dh, gamma, n_orb * n_orb, e0);
}

void launch_spin_cross(const double* Fb, const double* Fa, int n_pair, double* U, cudaStream_t st) {
  const int ldm = static_cast<int>(m_stride(n_pair));
  dim3 g(blocks_for(n_pair, 32), blocks_for(n_pair, 32));
  spin_cross_kernel<<<g, dim3(32, 8), 0, st>>>(Fb, Fa, n_pair, ldm, U);
}

void launch_onebody_spin(const double* Uaa, const double* Uab, const double* Ubb, const double* ga, const double* gb,
                         int n_orb, int n_pair, double* dh_a, double* dh_b, double* e0, cudaStream_t st) {
  const int ldm = static_cast<int>(m_stride(n_pair));
  onebody_spin_kernel<<<dim3(n_orb, n_orb, 2), 256, 0, st>>>(Uaa, Uab, Ubb, ga, gb, n_orb, ldm, dh_a, dh_b);
  constant_spin_kernel<<<1, 256, 0, st>>>(dh_a, ga, dh_b, gb, n_orb * n_orb, e0);
}

void launch_vfield_export(const void* V, bool f64, int splits, int n_pair, int n_orb, const int* pair_p,
                          const int* pair_q, int64_t n_i, int64_t gcp, double* out, cudaStream_t st) {
  const unsigned int b = std::min<unsigned int>(blocks_for(n_i * 3 * n_pair, 256), 8192u);
  if (f64)
    vfield_export_kernel<double><<<b, 256, 0, st>>>(static_cast<const double*>(V), splits, n_pair, n_orb, pair_p,
                                                    pair_q, n_i, gcp, out);
  else
    vfield_export_kernel<float><<<b, 256, 0, st>>>(static_cast<const float*>(V), splits, n_pair, n_orb, pair_p,
                                                   pair_q, n_i, gcp, out);
}

}  // namespace xtc
