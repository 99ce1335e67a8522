// Jastrow gradient nabla_1 u(r_i, r_j) split into per-outer-point coefficients and a
// per-pair polynomial (step (a) of the path).
//
// u(r1, r2) = sum_I sum_t c[set(I)][t] (a1^m a2^n + a1^n a2^m) b^o,
//   a_k = |r_k - R_I| / (1 + |r_k - R_I|),  b = r12 / (1 + r12),  0 <= m, n, o <= 2.
// By the chain rule (a'(r) = b'(r) = 1/(1+r)^2):
//   nabla_1 u = sum_I E_I(a2, b) g_I + H(a2, b) (1+r12)^-2 (r1 - r2)/r12,
//   g_I = (1+r1I)^-2 (r1 - R_I)/r1I,
//   E_I = sum_{o,k} alpha_I[o][k] a2I^k b^o,  alpha_I[o][k] = sum_{t: o_t=o} c (m a1^(m-1) [n=k] + n a1^(n-1) [m=k]),
//   H   = sum_I sum_{o>=1,k} beta_I[o][k] a2I^k b^(o-1),  beta_I[o][k] = sum_{t: o_t=o} c o (a1^m [n=k] + a1^n [m=k]).
// Everything that depends on the outer point alone (g_I, alpha, beta) is computed once per
// outer point; the k = 0 pieces are summed over nuclei into K_o (vectors) and Hc_o:
//   E . g summed = K0 + b K1 + b^2 K2 + sum_I a2I t_I g_I,
//   t_I = (a01 + a02 a2) + b ((a11 + a12 a2) + b (a21 + a22 a2)),
//   H   = (Hc1 + sum_I a2I (b11 + b12 a2I)) + b (Hc2 + sum_I a2I (b21 + b22 a2I)).
// A zero-length unit vector (point on a nucleus, or r12 = 0) contributes zero.
#pragma once
#include "xtc_internal.cuh"

namespace xtc {

// pc[PT_COEF]: x y z K0[3] K1[3] K2[3] Hc1 Hc2 ; nc[I*NUC_COEF + ...]: g[3] a01 a02 a11 a12 a21 a22 b11 b12 b21 b22
// The E part (K, g) and the H part (beta, Hc) are multiplied by `scale`.
template <typename T>
__device__ inline void point_coefs(const JastrowParams& jp, double x, double y, double z, double scale,
                                   T* pc, T* nc, int nuc_lo, int nuc_hi) {
  double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double Hc1 = 0.0, Hc2 = 0.0;
  for (int I = 0; I < jp.n_nuc; ++I) {
    const double vx = x - jp.nuc[I][0], vy = y - jp.nuc[I][1], vz = z - jp.nuc[I][2];
    const double d = sqrt(vx * vx + vy * vy + vz * vz);
    const double a1 = d / (1.0 + d);
    const double ap = 1.0 / ((1.0 + d) * (1.0 + d));
    const double ginv = d < 1e-14 ? 0.0 : ap / d;
    const double g[3] = {vx * ginv, vy * ginv, vz * ginv};
    double al[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double be[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const double pw[3] = {1.0, a1, a1 * a1};
    const int s = jp.set[I];
    for (int t = 0; t < jp.n_terms; ++t) {
      const int m = jp.mno[t][0], n = jp.mno[t][1], o = jp.mno[t][2];
      const double c = jp.coef[s][t];
      if (m >= 1) al[o][n] += c * m * pw[m - 1];
      if (n >= 1) al[o][m] += c * n * pw[n - 1];
      if (o >= 1) {
        be[o][n] += c * o * pw[m];
        be[o][m] += c * o * pw[n];
      }
    }
    for (int o = 0; o < 3; ++o)
      for (int x3 = 0; x3 < 3; ++x3) K[o][x3] += al[o][0] * g[x3];
    Hc1 += be[1][0];
    Hc2 += be[2][0];
    if (I >= nuc_lo && I < nuc_hi) {
      T* q = nc + (I - nuc_lo) * NUC_COEF;
      q[0] = (T)(g[0] * scale); q[1] = (T)(g[1] * scale); q[2] = (T)(g[2] * scale);
      q[3] = (T)al[0][1]; q[4] = (T)al[0][2];
      q[5] = (T)al[1][1]; q[6] = (T)al[1][2];
      q[7] = (T)al[2][1]; q[8] = (T)al[2][2];
      q[9] = (T)(be[1][1] * scale); q[10] = (T)(be[1][2] * scale);
      q[11] = (T)(be[2][1] * scale); q[12] = (T)(be[2][2] * scale);
    }
  }
  pc[0] = (T)x; pc[1] = (T)y; pc[2] = (T)z;
  for (int o = 0; o < 3; ++o)
    for (int x3 = 0; x3 < 3; ++x3) pc[3 + 3 * o + x3] = (T)(K[o][x3] * scale);
  pc[12] = (T)(Hc1 * scale);
  pc[13] = (T)(Hc2 * scale);
}

// Same coefficients for a compile-time number of nuclei NN, written into fixed-size arrays with
// compile-time indices (so that a kernel can keep them in registers).
struct NucTerms {
  double g[3];
  double al[3][3];
  double be[3][3];
};

__device__ inline void nuc_terms(const JastrowParams& jp, int I, double x, double y, double z, NucTerms& r) {
  const double vx = x - jp.nuc[I][0], vy = y - jp.nuc[I][1], vz = z - jp.nuc[I][2];
  const double d = sqrt(vx * vx + vy * vy + vz * vz);
  const double a1 = d / (1.0 + d);
  const double ap = 1.0 / ((1.0 + d) * (1.0 + d));
  const double ginv = d < 1e-14 ? 0.0 : ap / d;
  r.g[0] = vx * ginv;
  r.g[1] = vy * ginv;
  r.g[2] = vz * ginv;
  for (int o = 0; o < 3; ++o)
    for (int k = 0; k < 3; ++k) r.al[o][k] = r.be[o][k] = 0.0;
  const double pw[3] = {1.0, a1, a1 * a1};
  const int s = jp.set[I];
  for (int t = 0; t < jp.n_terms; ++t) {
    const int m = jp.mno[t][0], n = jp.mno[t][1], o = jp.mno[t][2];
    const double c = jp.coef[s][t];
    if (m >= 1) r.al[o][n] += c * m * pw[m - 1];
    if (n >= 1) r.al[o][m] += c * n * pw[n - 1];
    if (o >= 1) {
      r.be[o][n] += c * o * pw[m];
      r.be[o][m] += c * o * pw[n];
    }
  }
}

template <typename T, int NN>
__device__ inline void point_coefs_fixed(const JastrowParams& jp, double x, double y, double z, double scale,
                                         T (&pc)[PT_COEF], T (&nc)[NN * NUC_COEF]) {
  double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double Hc1 = 0.0, Hc2 = 0.0;
#pragma unroll
  for (int I = 0; I < NN; ++I) {
    // an instance with fewer nuclei than NN: the extra slots get zero coefficients
    if (I >= jp.n_nuc) {
#pragma unroll
      for (int k = 0; k < NUC_COEF; ++k) nc[I * NUC_COEF + k] = (T)0;
      continue;
    }
    NucTerms t;
    nuc_terms(jp, I, x, y, z, t);
#pragma unroll
    for (int o = 0; o < 3; ++o)
#pragma unroll
      for (int x3 = 0; x3 < 3; ++x3) K[o][x3] += t.al[o][0] * t.g[x3];
    Hc1 += t.be[1][0];
    Hc2 += t.be[2][0];
    nc[I * NUC_COEF + 0] = (T)(t.g[0] * scale);
    nc[I * NUC_COEF + 1] = (T)(t.g[1] * scale);
    nc[I * NUC_COEF + 2] = (T)(t.g[2] * scale);
    nc[I * NUC_COEF + 3] = (T)t.al[0][1];
    nc[I * NUC_COEF + 4] = (T)t.al[0][2];
    nc[I * NUC_COEF + 5] = (T)t.al[1][1];
    nc[I * NUC_COEF + 6] = (T)t.al[1][2];
    nc[I * NUC_COEF + 7] = (T)t.al[2][1];
    nc[I * NUC_COEF + 8] = (T)t.al[2][2];
    nc[I * NUC_COEF + 9] = (T)(t.be[1][1] * scale);
    nc[I * NUC_COEF + 10] = (T)(t.be[1][2] * scale);
    nc[I * NUC_COEF + 11] = (T)(t.be[2][1] * scale);
    nc[I * NUC_COEF + 12] = (T)(t.be[2][2] * scale);
  }
  pc[0] = (T)x;
  pc[1] = (T)y;
  pc[2] = (T)z;
#pragma unroll
  for (int o = 0; o < 3; ++o)
#pragma unroll
    for (int x3 = 0; x3 < 3; ++x3) pc[3 + 3 * o + x3] = (T)(K[o][x3] * scale);
  pc[12] = (T)(Hc1 * scale);
  pc[13] = (T)(Hc2 * scale);
}

// The per-pair polynomial in FP64 (also the reference form for the FP32 producer).
// aj[I] = a_jI for every nucleus.
__device__ inline void pair_grad_f64(const double* pc, const double* nc, int n_nuc, double xj, double yj,
                                     double zj, const double* aj, double& gx, double& gy, double& gz) {
  const double dx = pc[0] - xj, dy = pc[1] - yj, dz = pc[2] - zj;
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double r = sqrt(r2);
  const double q = 1.0 / (1.0 + r);
  const double b = r * q;
  const double s = r2 > 1e-28 ? q * q / r : 0.0;
  double ex = pc[3] + b * (pc[6] + b * pc[9]);
  double ey = pc[4] + b * (pc[7] + b * pc[10]);
  double ez = pc[5] + b * (pc[8] + b * pc[11]);
  double h1 = pc[12], h2 = pc[13];
  for (int I = 0; I < n_nuc; ++I) {
    const double* c = nc + I * NUC_COEF;
    const double a = aj[I];
    const double t = (c[3] + c[4] * a) + b * ((c[5] + c[6] * a) + b * (c[7] + c[8] * a));
    const double at = a * t;
    ex += at * c[0];
    ey += at * c[1];
    ez += at * c[2];
    h1 += a * (c[9] + c[10] * a);
    h2 += a * (c[11] + c[12] * a);
  }
  const double hs = (h1 + b * h2) * s;
  gx = ex + hs * dx;
  gy = ey + hs * dy;
  gz = ez + hs * dz;
}

}  // namespace xtc
