// Internal declarations shared by the xTC library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda.h>
#include <stdint.h>

namespace xtc {

constexpr int MAX_NUC = 64;
constexpr int MAX_TERMS = 27;   // (m, n, o) in {0,1,2}^3
constexpr int MAX_SETS = 64;

// Jastrow parameters as copied to the device (global memory).
struct JastrowParams {
  int n_nuc, n_terms, n_sets, pad;
  double nuc[MAX_NUC][3];
  int set[MAX_NUC];
  int mno[MAX_TERMS][3];
  double coef[MAX_SETS][MAX_TERMS];
};

// Per (outer point, nucleus) coefficients of the pair formula (see jastrow_coef.cuh).
constexpr int NUC_COEF = 13;    // g[3], a01 a02 a11 a12 a21 a22, b11 b12 b21 b22
constexpr int PT_COEF = 14;     // x y z, K0[3] K1[3] K2[3], Hc1 Hc2

// Tile shapes of the tensor-core kernels.
constexpr int VF_BM = 128;      // outer points per tile (TMEM lanes)
// orbital pairs per tensor-core tile (B rows): the fp16 engine keeps two pairs of TMEM accumulators
// of 128 columns (exact hi x hi and cross products per issuer), 7 pipeline stages of 32 KB; the bf16
// engine two accumulators of 160 columns, 4 stages of 54 KB; each drain thread holds a running sum
// of half a tile row in registers
__host__ __device__ constexpr int vf_bn(int parts) { return parts == 2 ? 128 : 160; }
constexpr int VF_BK = 32;       // inner points per pipeline stage (64-byte rows, SWIZZLE_64B)
constexpr int AS_BM = 128;      // step (d) tile rows (pairs pq)
constexpr int AS_BN = 128;      // step (d) tile columns (pairs rs)
constexpr int AS_BK = 32;
constexpr int CHUNK_ALIGN = 128;
// fp16 engine: exact hi x hi accumulation over ranges of kd K-blocks of VF_BK values needs
// kd * VF_BK * 2^(bits_a + bits_b) <= 2^24.  Step (b) (kd <= 2): G carries GEMM_BITS_A bits and
// rho^T gemm_bits_b(kd) on per-range quanta; step (d): L and R both gemm_bits_lr(kd) per range.
constexpr int GEMM_BITS_A = 9;
__host__ __device__ constexpr int log2_kd(int kd) { return kd >= 8 ? 3 : kd >= 4 ? 2 : kd >= 2 ? 1 : 0; }
__host__ __device__ constexpr int gemm_bits_b(int kd) { return 24 - 5 - GEMM_BITS_A - log2_kd(kd); }
__host__ __device__ constexpr int gemm_bits_lr(int kd) { return (24 - 5 - log2_kd(kd)) / 2; }
static_assert(GEMM_BITS_A + gemm_bits_b(4) + 5 + 2 <= 24 && 2 * gemm_bits_lr(4) + 5 + 2 <= 24, "exact ranges");

// Error codes written by kernels into the context's device error word.
constexpr int DEV_ERR_TIMEOUT_VF = 1;
constexpr int DEV_ERR_TIMEOUT_AS = 2;
constexpr int DEV_ERR_TIMEOUT_SELFTEST = 3;
// Self-test of the bounded waits: one CTA waits on an mbarrier that nothing arrives on, with the
// kernels' own wait routine and a limit of limit_ns, and records DEV_ERR_TIMEOUT_SELFTEST in err.
void launch_wait_timeout_selftest(int* err, unsigned long long limit_ns, cudaStream_t st);
// Self-test of the gradient kernel's refined 1/sqrt(x) and 1/x (simt_pack.cuh) on x[0..n).
void launch_recip_selftest(const float* x, int64_t n, float* y_rsqrt, float* y_rcp, cudaStream_t st);

// Frozen-core folding (frozen_core.cu): core and active orbital lists, passed by value.
constexpr int FC_MAX_ORB = 320;
struct FcIndex {
  int n_core, n_act;
  int core[FC_MAX_ORB];
  int act[FC_MAX_ORB];
};
// e_core (one FP64), dh_fc [n_act]^2 and, unless NULL, dU_act [n_act]^4 from the device arrays
// dU [N]^4 and dh [N]^2.
void launch_frozen_core(const double* dU, const double* dh, int N, const FcIndex& ix, double* dh_fc,
                        double* dU_act, double* e_core, int n_sm, cudaStream_t st);

// V of a chunk (written by step (b), read by step (c)): blocks of VB consecutive outer points, each
// holding the whole symmetric N x N matrix of the three components, V_x,ps(i) at
// [i / VB][p][s][x][i % VB]; both (p, s) and (s, p) are written.  A row p of a block is one
// contiguous run of 3 * VB * N values, so step (c) streams rows instead of gathering pairs.  One
// split slice holds gcp * N * N * 3 values.
constexpr int VB = 8;
__host__ __device__ inline int64_t v_index(int64_t i, int p, int s, int x, int n_orb) {
  return (((i / VB) * n_orb + p) * n_orb + s) * (3 * VB) + x * VB + (i % VB);
}
__host__ __device__ inline int64_t v_slice(int64_t gcp, int n_orb) {
  return gcp * static_cast<int64_t>(n_orb) * n_orb * 3;
}

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
// Row stride of the FP64 accumulator M[pq][rs]: a multiple of 32 (the bf16 step (d) kernel writes
// whole 32-column groups of its 128-column tiles) with room for every pair.
inline int64_t m_stride(int64_t n_pair) { return round_up(n_pair, 384); }

// The current device's opt-in maximum of dynamic shared memory per CTA.  Kernels whose dynamic
// shared memory varies from call to call set their limit to this one value (not to the call's
// size): the limit is per function and process-wide, and batch lanes launch from several host
// threads, so a per-call value set by one thread could undercut another thread's launch.
inline int max_dyn_smem() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 48 * 1024;
  return v;
}

// Floats per inner point in the gradient producer's table: 12 for up to 4 nuclei, 16 for 5..8.
inline int jtab_stride(int n_nuc) { return n_nuc <= 4 ? 12 : 16; }

// ---------------------------------------------------------------- launchers

// Per-inner-point table for the producer: stride js floats per point:
// x, y, z, a_j0, a_j1, ...  (a_jI = |r_j - R_I| / (1 + |r_j - R_I|)), padded points far away.
void launch_jtab(const double* grid, int64_t n_grid, int64_t n_grid_pad, const JastrowParams* jp_dev,
                 int n_nuc, int js, float* jtab, cudaStream_t st);

// Pair products rho^T[pq][j] = w_j phi_p(j) phi_q(j) split into parts.  fp16 (2 parts): each pair's
// row scaled by a power of 2 (colexp[pq] receives the exponent; colmax is scratch) and split exactly
// with one quantum per range of kd blocks of 32 points (gemm_bits_b(kd) bits), the two parts of a
// block in one 128-byte row: [pq][j / 32][part][j % 32], followed by a plane of the scaled value
// rounded to fp16, [pq][j] (2 x n_pair x n_pad values, then n_pair x n_pad); the products are
// taken in FP32 pairs hi + lo from phi32, scratch of 2 (n_orb + 1) n_pad floats.  bf16 (3 parts):
// per-element split, unscaled (colexp = 0), [part][pq][j].  n_pad must be a multiple of 32 kd.
void launch_rho_split(const double* phiT, const double* w, int64_t n_grid, int64_t n_pad, int n_orb, int parts, int kd,
                      const int* pair_p, const int* pair_q, unsigned int* colmax, int* colexp, float* phi32,
                      void* out, cudaStream_t st);

// FP64 pair products rho[j][pq] for the FP64 path (n_grid_pad rows, zero padded).
void launch_rho_f64(const double* phi, const double* w, int64_t n_grid, int64_t n_grid_pad, int n_orb,
                    const int* pair_p, const int* pair_q, double* rho, cudaStream_t st);

// Transposed orbitals phiT[p][j] (FP64), zero padded to n_grid_pad.
void launch_transpose_phi(const double* phi, int64_t n_grid, int64_t n_grid_pad, int n_orb, double* phiT,
                          cudaStream_t st);

// Finite check: sets *flag non-zero if any of n values is NaN/Inf.
void launch_check_finite(const double* x, int64_t n, int* flag, cudaStream_t st);

// Step (a), tensor-core path: the split Jastrow gradient of the outer points [i0, i0 + n_i) and every
// padded inner point, K-major, row x * gcp + il: fp16 (2 parts) G[row][j / 32][part][j % 32] stored
// as 128-byte-swizzled TMA tiles (box 64 x 32); bf16 (3 parts) G[part][row][j] as 64-byte-swizzled
// tiles (box 32 x 32).  Rows up to n_tiles * 32 are written (past n_i they repeat the last point).
struct GfieldArgs {
  const double* grid;          // outer-point coordinates (global index space)
  const JastrowParams* jp;
  const float* jtab;           // pair-interleaved inner-point table (launch_jtab, 12 floats per point)
  int64_t i0, n_i;             // outer range of this chunk
  int64_t gcp;                 // padded chunk length (rows per component)
  int n_tiles;                 // 32-row outer tiles to write (multiple of 4)
  int n_kb, kb_per_seg, n_seg; // inner K-blocks (32 points), K-blocks per warp unit, units along K
  int n_nuc;
  float g_scale;               // 2^sG folded into the gradient
  int range_blocks;            // fp16: K-blocks per exact range of the step (b) GEMM (1 or 2)
};
void launch_gfield(const CUtensorMap* tm_g_store, const GfieldArgs& a, int parts, cudaStream_t st);

// Step (b), tensor cores.  V[z][pq][x][il] (FP32, il = i - i0 < gcp) for the outer points of the
// chunk, from the G table (tm_g: box rows 128) and the split rho^T (tm_rho: box rows vf_bn(parts)).
struct VfieldArgs {
  const int* colexp;           // per-pair exponent of the rho scaling (0 when unscaled)
  float* V;                    // output base (mode 0), layout v_index
  const int* pair_p;           // mode 0: orbitals (p, s) of pair pq
  const int* pair_q;
  int n_orb;
  double* Vacc;                // FP64 partial sums, [splits][grid CTAs][BN][128] (used when flush > 0)
  int flush;                   // ranges summed in FP32 registers between FP64 flushes (0: no flush)
  int64_t n_i;                 // outer points of this chunk
  int64_t gcp;                 // padded chunk length (row stride of V and of G per component)
  int mt_per_x;                // 128-row tiles per component: ceil(n_i / 128)
  int n_tiles;                 // column tiles: ceil(n_pair / vf_bn(parts))
  int n_pair;
  int kb_per_split, n_kb;      // inner K-blocks per split slice, total K-blocks
  int kd;                      // K-blocks per TMEM accumulation range (then added to the FP32 running sum);
                               // fp16 engine: 1, 2 or 4, the range of the operands' exact split
  int xper;                    // fp16 engine: K-blocks between drains of the cross-product accumulator
  float unscale_g;             // 2^-sG
  int* err;
  // mode 1 (step d with fp16 x2 operands): A = L split rows (rows_a of them), B = R split rows
  // (n_pair), K = 32 * n_kb; the tile sums (FP64, Vacc, flush > 0 required) are added, unscaled by
  // 2^-(exp_a[pq] + exp_b[rs]), into M[pq * ldm + rs]
  int mode;
  int rows_a;
  double* M;
  int64_t ldm;
  const int* exp_a;
  const int* exp_b;
};
bool vfield_tc_supported(int n_nuc);
// Launches the GEMM.
// tm_rho16: the fp16(rho^T) plane of the fp16 precision (box 32 x 128, 64-byte swizzle); step (d)
// (mode 1) and the bf16 precision ignore it.
void launch_vfield_tc(const CUtensorMap* tm_g, const CUtensorMap* tm_rho, const CUtensorMap* tm_rho16,
                      const VfieldArgs& a, int parts, int splits, cudaStream_t st);
// Then, with FP64 sums (a.flush > 0): mode 0 writes V from them, mode 1 adds the tiles into M.
void launch_vfield_tc_finalize(const VfieldArgs& a, int parts, int splits, cudaStream_t st);

// Steps (a)+(b), FP64 SIMT twin.  V in the layout of v_index (FP64).  jtab64[n_grid_pad][3 + n_nuc].
void launch_jtab64(const double* grid, int64_t n_grid, int64_t n_pad, const JastrowParams* jp, int n_nuc,
                   double* jtab, cudaStream_t st);
void launch_vfield_f64_impl(const double* grid, const JastrowParams* jp, int n_nuc, const double* jtab64,
                            const double* rho, int64_t n_pad, int n_pair, int64_t i0, int64_t n_i, int64_t gcp,
                            const int* pair_p, const int* pair_q, int n_orb, double* V, cudaStream_t st);

// Step (a) alone in FP64.
void launch_jastrow_grad(const JastrowParams* jp, const double* r1, const double* r2, int64_t n, double* out,
                         cudaStream_t st);

// Step (c).  Reads V (T = float or double, [splits] slices in the layout of v_index), writes L = (rho, Vx, Vy, Vz) and
// R = (A, Bx, By, Bz) per outer point, either as split parts [part][pq][4*gcp] (fp16/bf16) or as FP64
// [4*gcp][pq].
struct FieldsArgs {
  const void* V;
  int splits;
  const double* phiT;          // [n_orb][ldphi], global grid index
  int64_t ldphi;
  const double* w;
  const double* evec;          // [rank][n_orb]: factors c_k of the densities
  const double* lam;           // [rank]: exchange weights, gamma_x = sum_k lam_k c_k c_k^T (X, Y, Zt, Z)
  const double* lamd;          // [rank]: direct weights, g_d = sum_k lamd_k c_k c_k^T (W = V.g_d, Wt = rho.g_d);
                               // closed shell: lamd = 2 lam; spin t: g_d = gamma^a + gamma^b, gamma_x = gamma^t
  int rank;
  int64_t i0, n_i, gcp;
  int n_orb, n_pair;
  int pts;                     // outer points per CTA
  const int* pair_p;
  const int* pair_q;
  void* L;                     // outputs
  void* R;
  void* R2;                    // spin builds: R for electron-2 spin beta (R is alpha); nullptr otherwise
  const double* lam2;          // spin builds: beta exchange weights (lam holds the alpha ones)
  int out_parts;               // 0 = FP64 [4*gcp][pq]; 1 = FP32 [pq][4*gcp]; 3 = bf16 x3 split [part][pq][4*gcp]
  int write_L;                 // write L (the first pass over a density's factors)
  int add_R;                   // add R (and R2) to the buffer's contents (later passes; out_parts 0 or 1)
};
size_t fields_smem_bytes(int n_orb, int rank, int pts, bool f64, bool spin);
void launch_fields(const FieldsArgs& a, bool f64, cudaStream_t st);  // f64: FP64 V, compute and output

// Step (d) operands in fp16 x2: each FP32 row src[r][0..kdim) is scaled by 2^exps[r] (largest
// magnitude in [2^13, 2^14)) and split exactly into hi + lo fp16 with one quantum per range of kd
// blocks of 32 values (gemm_bits_lr(kd) bits), both parts of a block in one 128-byte row:
// dst[r][k' / 32][part][k' % 32].  kc = 4: the source holds 4 values per outer point (k = 4 i + c)
// and k' = c * kdim / 4 + i (component-major, so that a range never mixes components); kc = 1:
// k' = k.  kdim / kc must be a multiple of 32 kd.  dst16 (or NULL): the scaled values rounded to
// fp16, dst16[r][k'] (the plane of the B operand, for the lo x fp16(B) product).
void launch_lr_split(const float* src, int rows, int64_t kdim, int kc, int kd, uint16_t* dst, int* exps,
                     uint16_t* dst16, cudaStream_t st);

// Step (d), tensor cores, bf16 x3: M[pq][rs] += sum_k L[pq][k] R[rs][k] over k < kdim (FP64 accumulator).
void launch_assemble_tc(const CUtensorMap* tm_L, const CUtensorMap* tm_R, int n_pair, int kdim, int kd, double* M,
                        int* err, cudaStream_t st);

// Step (d), FP64 SIMT twin: M[pq][rs] += sum_k L[k][pq] R[k][rs].
void launch_assemble_f64(const double* L, const double* R, int n_pair, int kdim, double* M, cudaStream_t st);

// Final: M <- Delta U = -(M + M^T) in place; unpacking; Delta h; e0.  M row stride round_up(n_pair, AS_BN).
void launch_symmetrize(double* M, int n_pair, cudaStream_t st);
void launch_unpack(const double* M, int n_orb, int n_pair, double* dU, float* dU32, cudaStream_t st);
// Explicit three-body L (eq. Ldecomp), FP64: T[a][b][c] = sum_k rho_a(i0 + k) V[k].b . V[k].c over
// k < n_i with V[k][x][pair] (the layout of xtc_vfield), then L[p][r][t][q][s][u] from T.
void launch_three_body_t(const double* phi, const double* w, int64_t i0, int64_t n_i, int n_orb, const int* pair_p,
                         const int* pair_q, const double* V, double* T, cudaStream_t st);
void launch_three_body_unpack(const double* T, int n_orb, double* L, cudaStream_t st);
// Two-body integrals K: one chunk of outer points [i0, i0 + n_i) adds into S (N^2 x n_pair, FP64)
// from V of the chunk ([n_i][3][n_pair]); Ft (n_grid x n_i), W (n_i x n_pair) and partial
// (split-K slices of small GEMMs, partial_elems doubles; 4 x n_sm x 4096 suffice) are workspace.
void launch_k_chunk(const double* grid, const double* w, const double* phi, const double* dphi,
                    const JastrowParams* jp_dev, int64_t n_grid, int n_orb, const int* pair_p, const int* pair_q,
                    int64_t i0, int64_t n_i, const double* V, double* Ft, double* W, double* S, double* partial,
                    int64_t partial_elems, int n_sm, cudaStream_t st);
// K[p][q][r][s] = S[pq][rs] + S[rs][pq].
void launch_k_unpack(const double* S, int n_orb, double* K, int n_sm, cudaStream_t st);
// Spin builds: U = Delta U^{ab} = -(Fb + Fa^T) (packed pairs, row stride m_stride(n_pair)).
void launch_spin_cross(const double* Fb, const double* Fa, int n_pair, double* U, cudaStream_t st);
// Spin builds: Delta h^a, Delta h^b and e0 from Delta U^{aa}, ^{ab}, ^{bb} and the two densities.
void launch_onebody_spin(const double* Uaa, const double* Uab, const double* Ubb, const double* ga, const double* gb,
                         int n_orb, int n_pair, double* dh_a, double* dh_b, double* e0, cudaStream_t st);
void launch_onebody(const double* M, const double* gamma, int n_orb, int n_pair, double* dh, double* e0,
                    cudaStream_t st);

// V (FP32 or FP64, [splits] slices in the layout of v_index) -> FP64 [n_i][3][pq] (for xtc_vfield).
void launch_vfield_export(const void* V, bool f64, int splits, int n_pair, int n_orb, const int* pair_p,
                          const int* pair_q, int64_t n_i, int64_t gcp, double* out, cudaStream_t st);

// Read-only view of a context for entry points implemented outside xtc_api.cu.
struct CtxView {
  int device;
  cudaStream_t stream;
  int precision;
  int n_sm;
  bool jastrow_set;
  int n_nuc;
  double g_bound;
  int vf_kd;
  const JastrowParams* jp_dev;
  void* encode_tiled;  // PFN_cuTensorMapEncodeTiled_v12000
};

}  // namespace xtc

struct xtc_ctx;
// Fills *v from ctx; false for a null context.
bool xtc_internal_ctx_view(const xtc_ctx* ctx, xtc::CtxView* v);
// Records a failure message on ctx and returns code.
int xtc_internal_fail(xtc_ctx* ctx, int code, const char* msg);
