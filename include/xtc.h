/*
 * xtc.h -- C ABI of the GB300 (sm_103a) grid-quadrature build of the xTC
 * corrections (arXiv 2304.07006).
 *
 * The library computes, on one GPU and without ever forming the six-index
 * three-body tensor L, the three outputs of eq. (xTC):
 *
 *   dU[p][q][r][s] = Delta U_pr^qs        two-body correction, chemists' (pq|rs) order
 *   dh[p][q]       = Delta h_p^q          one-body correction
 *   e0             = <Phi0|L|Phi0>        constant added to E_nuc
 *
 * for a closed-shell reference with real orbitals, using the restricted
 * closed-shell working equations of Appendix B together with the intermediate
 * V_rs(i) = sum_j w_j phi_r(j) nabla_1 u(r_i, r_j) phi_s(j) of the section
 * "Decomposition of two-body correction" (eq. Ldecomp).  The path has four
 * steps, all in the library's own CUDA kernels:
 *   (a) the Jastrow gradient nabla_1 u over grid-point pairs,
 *   (b) the vector pair fields V (a dense contraction over the inner grid index),
 *   (c) the density-contracted intermediates rho, W, Vt, X, Zt, Wt, Y, Z, A, B,
 *   (d) Delta U = -P^(pq)_(rs) sum_i (rho_pq A_rs + V_pq . B_rs), then
 *       Delta h = -1/2 (2 Delta U_pr^qs gamma_rs - Delta U_pr^sq gamma_rs) and
 *       e0 = -2/3 Delta h_pq gamma_pq.
 *
 * Beside this closed-shell build the library offers the build for separate alpha and beta
 * densities of Appendix A (xtc_build_1b2b_rohf), a batched build of many instances
 * (xtc_build_1b2b_batched), the frozen-core folding of the corrections (xtc_frozen_core_fold),
 * the explicit L of eq. Ldecomp for small orbital sets as a validation aid (xtc_three_body_L),
 * the two-body integrals K of the similarity-transformed Hamiltonian (xtc_two_body_K),
 * steps (a) and (b) alone (xtc_jastrow_grad, xtc_vfield, and xtc_vfield_noalloc, which allocates
 * nothing) and a chunk autotuner (xtc_autotune_chunk).
 *
 * Units are Hartree atomic units (bohr, Eh).  Conventions:
 *   - gamma is the per-spin (alpha) density matrix; the spin factor 2 is explicit
 *     in the equations (Appendix B).  It must be symmetric.
 *   - The Jastrow factor is u(r1,r2) = sum_I sum_t c[set(I)][t]
 *       (a1^m a2^n + a1^n a2^m) b^o, a_k = |r_k - R_I|/(1 + |r_k - R_I|),
 *       b = r12/(1 + r12), t = (m, n, o) with 0 <= m, n, o <= 2.
 *   - Where a unit vector is undefined (r12 = 0, including the grid diagonal
 *     j = i, or a point on a nucleus) its contribution to nabla_1 u is zero.
 *
 * Ownership and memory: the caller owns every input and output buffer.  Each
 * pointer may address host memory or device memory of the context's device;
 * the library detects which.  The library owns only its device workspace,
 * allocated on first use, reused by later calls of the same sizes, and released
 * by xtc_destroy.  Calls are synchronous with respect to the host: when a call
 * returns XTC_OK its outputs are complete (device outputs included).  All
 * device work is issued on the stream given in xtc_params.  One context must
 * not be used by two host threads at once.
 *
 * Errors: every function returns an xtc_status (0 = success).  Nothing throws
 * across the ABI.  xtc_strerror gives a static message; xtc_last_error_detail
 * gives a per-context message describing the last failure.
 */
#ifndef XTC_H
#define XTC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define XTC_API __attribute__((visibility("default")))
#else
#define XTC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xtc_ctx xtc_ctx;

typedef enum {
  XTC_OK = 0,
  XTC_ERR_ARG = -1,           /* bad size, null pointer where one is required, term out of range */
  XTC_ERR_NOT_SYMMETRIC = -2, /* gamma is not symmetric to 1e-12 relative */
  XTC_ERR_NONFINITE = -3,     /* NaN or Inf in an input */
  XTC_ERR_OOM = -4,           /* device workspace allocation failed */
  XTC_ERR_CUDA = -5,          /* a CUDA runtime or driver call failed */
  XTC_ERR_TIMEOUT = -6,       /* a bounded device-side wait gave up (kernel returned early) */
  XTC_ERR_STATE = -7,         /* xtc_set_jastrow not called, or context unusable */
  XTC_ERR_UNSUPPORTED = -8    /* device is not sm_103 / sm_100 class, or > 8 nuclei on tensor cores */
} xtc_status;

typedef enum {
  XTC_PREC_FP64 = 0,   /* all four steps in FP64 (SIMT) */
  XTC_PREC_FP16X2 = 1, /* steps (b) and (d): range-exact 2-term FP16 split with power-of-2 scaling
                          (per pair column of rho in step b, per row of L and R in step d): per
                          accumulation range (range_stages blocks of 32 inner values, default 2)
                          hi = an integer times the range's power-of-2 quantum (step b: 9 bits for
                          the gradient, 10 - log2(range) for rho; step d: (19 - log2(range)) / 2
                          each), lo = the FP16 remainder, so the hi x hi products of a range sum
                          exactly in the tensor core's FP32 accumulator (no truncation bias); the
                          cross products hi x lo and lo x FP16(B) (B = rho in step b, R in step d)
                          accumulate apart.  FP32 running sums (round to
                          nearest) flushed to FP64 every 8,192 inner points; FP64 accumulation of
                          Delta U across grid chunks, of Delta h and of e0 */
  XTC_PREC_BF16X3 = 2  /* steps (b) and (d): 3-term BF16 split (6 products) accumulated in the tensor
                          cores over short ranges (range_stages), otherwise as FP16X2; its FP32
                          accumulation truncates toward zero at every MMA, a one-signed error that
                          grows with the grid */
} xtc_precision;

typedef struct {
  int device;          /* CUDA device ordinal */
  void* stream;        /* cudaStream_t for all device work; NULL = the legacy default stream */
  int precision;       /* xtc_precision */
  int64_t grid_chunk;  /* outer grid points per chunk (multiple of 128); 0 = automatic */
  int split_k;         /* inner-grid slices of step (b) accumulated separately (1..16); 0 = automatic */
  int timing;          /* non-zero: record CUDA events around every kernel (see xtc_get_timings) */
  int range_stages;    /* stages of 32 inner points per tensor-core accumulation range, 1..4;
                          0 = default (2).  XTC_PREC_FP16X2: the range of the exact hi x hi sums
                          (1, 2 or 4: the hi parts carry fewer bits on longer ranges so that every
                          range sum stays exact; longer ranges mean fewer drains and larger lo
                          parts).  XTC_PREC_BF16X3: stages accumulated in the tensor cores before a
                          round-to-nearest FP32 add (at most 2 in step b and 3 in step d); that
                          accumulator truncates toward zero, so the error grows with the range */
  /* Caller allocator for the device workspace (for instance a framework's caching allocator), or
   * both NULL for cudaMalloc / cudaFree.  alloc returns `bytes` of device memory of p->device
   * usable on p->stream, or NULL when it cannot (the call then fails with XTC_ERR_OOM); release
   * takes back a pointer that alloc returned, after the context's stream has finished with it.
   * Workspace is allocated on first use, grown when a call needs more (old block released
   * first) and released by xtc_destroy.  Callbacks may run on the library's batch-lane threads. */
  void* (*alloc)(size_t bytes, void* user);
  void (*release)(void* ptr, void* user);
  void* alloc_user;    /* passed to alloc and release */
} xtc_params;

/* Fills *p with defaults: device 0, default stream, XTC_PREC_FP16X2, automatic chunking. */
XTC_API void xtc_default_params(xtc_params* p);

/* Creates a context bound to p->device.  *out receives the handle (NULL on failure).
 * Errors: XTC_ERR_ARG (null), XTC_ERR_CUDA, XTC_ERR_UNSUPPORTED (compute capability < 10.0). */
XTC_API int xtc_create(xtc_ctx** out, const xtc_params* p);

/* Releases the context and its device workspace.  Accepts NULL. */
XTC_API int xtc_destroy(xtc_ctx* ctx);

/* Static message for a status code. */
XTC_API const char* xtc_strerror(int status);

/* Detail of the last error on this context (static storage owned by the context). */
XTC_API const char* xtc_last_error_detail(const xtc_ctx* ctx);

/* Jastrow factor (Results, "Computational details" gives the paper's DTN form; this
 * library takes the polynomial form in the header comment).  Host arrays, copied.
 *   n_nuc    >= 1        nuclei (any number for XTC_PREC_FP64; at most 8 for the tensor-core
 *                        precisions, else xtc_build_1b2b returns XTC_ERR_UNSUPPORTED)
 *   nuc_xyz  [n_nuc][3]  bohr
 *   nuc_set  [n_nuc]     centre-set index of each nucleus, 0 <= nuc_set[I] < n_sets
 *   n_terms  >= 1, mno [n_terms][3] = (m, n, o), each in 0..2
 *   coef     [n_sets][n_terms]
 * Errors: XTC_ERR_ARG, XTC_ERR_NONFINITE. */
XTC_API int xtc_set_jastrow(xtc_ctx* ctx, int n_nuc, const double* nuc_xyz, const int* nuc_set, int n_sets,
                    int n_terms, const int* mno, const double* coef);

/* Restricts the outer grid sum over i (eqs. Ldecomp, tcmf:2el) to points
 * [begin, end); end < 0 means n_grid.  The inner sum over j always covers the
 * whole grid.  The outputs are linear in the outer sum, so disjoint ranges add
 * up to the full result.  Default: the whole grid. */
XTC_API int xtc_set_outer_range(xtc_ctx* ctx, int64_t begin, int64_t end);

/* The xTC build (steps a-d).
 *   n_grid >= 1, n_orb >= 1
 *   grid_xyz [n_grid][3], weights [n_grid], phi [n_grid][n_orb] (row-major, real MOs),
 *   gamma [n_orb][n_orb] symmetric per-spin density           -- inputs, FP64
 *   dU     [n_orb]^4 FP64 or NULL; dU_f32 [n_orb]^4 FP32 or NULL -- dU[p][q][r][s] = Delta U_pr^qs
 *   dh     [n_orb][n_orb] FP64 (required), e0 [1] FP64 (required)
 * The outer grid is processed in chunks (xtc_params.grid_chunk, automatic by default: at most
 * 16 GB of gradient table and 12 GB of V and step (d) operands per chunk).  With several chunks
 * and room for a second gradient table, step (a) of the next chunk runs on a second stream of the
 * library's own while the current chunk finishes (ordered by events; the results do not depend on
 * it); at N=120 and 100,000 points the workspace is about 50 GB.
 * Errors: XTC_ERR_ARG, XTC_ERR_STATE, XTC_ERR_NOT_SYMMETRIC, XTC_ERR_NONFINITE,
 *         XTC_ERR_OOM, XTC_ERR_CUDA, XTC_ERR_TIMEOUT. */
XTC_API int xtc_build_1b2b(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz, const double* weights,
                   const double* phi, const double* gamma, double* dU, float* dU_f32, double* dh, double* e0);

/* The xTC build for two spin densities (Appendix A, "Restricted open-shell working equations"):
 * both spins share the real orbitals phi and the Jastrow factor, so steps (a) and (b) are
 * spin-free; steps (c) and (d) run once per spin of electron 2, with the direct terms (W, Wt)
 * from gamma_a + gamma_b and the exchange terms from that spin's density.
 *   n_grid, n_orb, grid_xyz, weights, phi           -- as in xtc_build_1b2b
 *   gamma_a, gamma_b [n_orb][n_orb] symmetric alpha and beta densities (occupied = 1), FP64
 *   dU_aa, dU_ab, dU_bb [n_orb]^4 FP64, each may be NULL -- dU_st[p][q][r][s] = [Delta U_pr^qs]^{st},
 *                        electron 1 (p, q) of spin s, electron 2 (r, s) of spin t; the beta-alpha
 *                        block is dU_ba[p][q][r][s] = dU_ab[r][s][p][q]
 *   dh_a, dh_b [n_orb][n_orb] FP64 (required): [Delta h_p^q]^a and ^b
 *   e0 [1] FP64 (required): <Psi0|L|Psi0> = -1/3 sum_s dh_s . gamma_s
 * With gamma_a = gamma_b = gamma every block equals xtc_build_1b2b's Delta U, dh_a = dh_b its
 * Delta h and e0 its constant (to rounding).  Pointers may be host or device memory; the call
 * returns when the outputs are complete.  Workspace: two more N_pair^2 FP64 accumulators than
 * xtc_build_1b2b.  Errors: as xtc_build_1b2b. */
XTC_API int xtc_build_1b2b_rohf(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz,
                        const double* weights, const double* phi, const double* gamma_a, const double* gamma_b,
                        double* dU_aa, double* dU_ab, double* dU_bb, double* dh_a, double* dh_b, double* e0);

/* Step (a) alone: out[k][0..2] = nabla_1 u(r1[k], r2[k]) in FP64 arithmetic on the device.
 * r1, r2 [n][3], out [n][3]. */
XTC_API int xtc_jastrow_grad(xtc_ctx* ctx, int64_t n, const double* r1, const double* r2, double* out);

/* Steps (a)+(b) alone, in the context's precision, for the outer points [outer_begin, outer_end):
 * V[k][x][pq] = V_pq(i = outer_begin + k) component x, pq the packed index of p <= q
 * (pq = p*n_orb - p*(p-1)/2 + (q - p)).  V has (outer_end - outer_begin) * 3 * n_orb(n_orb+1)/2 doubles. */
XTC_API int xtc_vfield(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz, const double* weights,
               const double* phi, int64_t outer_begin, int64_t outer_end, double* V);

/* Self-test of failure detection (no counterpart in the paper): every wait inside the library's
 * tensor-core kernels is bounded; when it runs out, the kernel records an error code and returns,
 * and the call reports XTC_ERR_TIMEOUT.  This call runs one such wait on a barrier that nothing
 * completes, with a limit of limit_ms (1..4000), and returns what a timed-out build would:
 * XTC_ERR_TIMEOUT.  The context stays usable.  XTC_ERR_ARG for a limit out of range. */
XTC_API int xtc_selftest_wait_timeout(xtc_ctx* ctx, int limit_ms);

/* Frozen-core folding of the xTC corrections, xTC-FC (Results section "Frozen core
 * approximation"): the corrections of the whole orbital space are folded over a set C of doubly
 * occupied core orbitals with the standard closed-shell frozen-core equations,
 *   e_core        = sum_{c in C} 2 dh[c][c] + sum_{c,d in C} (2 dU[c][c][d][d] - dU[c][d][d][c])
 *   dh_fc[a][b]   = dh[p][q] + sum_{c in C} (2 dU[p][q][c][c] - dU[p][c][c][q])
 *   dU_act[a][b][e][f] = dU[p][q][r][s]
 * where p = act[a], q = act[b], r = act[e], s = act[f] and act lists the orbitals outside C in
 * ascending order (n_act = n_orb - n_core of them).  The folding is linear in (dh, dU): these are
 * the xTC parts of the folded one-body integrals, two-body integrals and core energy, and the
 * caller adds the folding of its own one-electron integrals and of V - K the same way.  The
 * equations need only the pair symmetry dU[p][q][r][s] = dU[r][s][p][q], so they also fold a
 * caller's non-hermitian integrals.  (FC-xTC, the other convention of that section, is
 * xtc_build_1b2b run on the active orbitals alone.)
 *   n_orb  1..320
 *   dU     [n_orb]^4 FP64, dh [n_orb][n_orb] FP64 -- e.g. the outputs of xtc_build_1b2b
 *   core   [n_core] distinct orbital indices in 0..n_orb-1, host memory; 0 <= n_core <= n_orb
 *   dh_fc  [n_act][n_act] FP64 (required unless n_act = 0)
 *   dU_act [n_act]^4 FP64 or NULL
 *   e_core [1] FP64 (required)
 * dU, dh, dh_fc, dU_act and e_core may be host or device memory; host inputs are staged through
 * the context's workspace (n_orb^4 doubles for dU).  Returns when the outputs are complete.
 * Every sum is taken in FP64, the core energy in a fixed order.  Errors: XTC_ERR_ARG (sizes, null
 * pointers, a core index out of range or repeated), XTC_ERR_OOM, XTC_ERR_CUDA. */
XTC_API int xtc_frozen_core_fold(xtc_ctx* ctx, int n_orb, const double* dU, const double* dh, int n_core,
                                 const int* core, double* dh_fc, double* dU_act, double* e_core);

/* Self-test of the reciprocal square root and reciprocal that the tensor-core precisions use in
 * step (a) (the unit vectors and the b = r12/(1+r12) factors of nabla_1 u): the hardware
 * approximation refined by one Newton-Raphson step, in the packed and the scalar form.  Reads
 * x[0..n) (positive normal FP32 values; host or device memory) and writes y_rsqrt[k] ~ 1/sqrt(x[k])
 * and y_rcp[k] ~ 1/x[k], or NaN where the packed and scalar forms disagree.  n <= 2^26.
 * Errors: XTC_ERR_ARG, XTC_ERR_OOM, XTC_ERR_CUDA. */
XTC_API int xtc_selftest_reciprocals(xtc_ctx* ctx, int64_t n, const float* x, float* y_rsqrt, float* y_rcp);

/* Chunk autotuner (no counterpart in the paper; the chunk is this library's streaming unit):
 * times xtc_build_1b2b on this problem's first outer points, min(n_grid, 2 x the rule's chunk) of
 * them, with up to three chunk lengths (the rule's choice, and the rule under 3/4 and 1/2 of its
 * memory budgets, each fitted to whole waves of the step (b) GEMM), after one warm-up, and keeps
 * the fastest as the context's grid_chunk for later builds; *chunk receives it.  The outer range
 * set by xtc_set_outer_range is restored.  Inputs as in xtc_build_1b2b (Delta U is not formed).
 * XTC_PREC_FP64 contexts take the rule's choice without timing.  Errors: as xtc_build_1b2b. */
XTC_API int xtc_autotune_chunk(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz,
                       const double* weights, const double* phi, const double* gamma, int64_t* chunk);

/* The explicit three-body tensor of eq. Ldecomp ("Decomposition of two-body correction"), for
 * validating full transcorrelated codes on small orbital sets:
 *   L[p][r][t][q][s][u] = L_prt^qsu = sum_i [ rho_pq V_rs.V_tu + rho_rs V_pq.V_tu + rho_tu V_pq.V_rs ](i),
 *   rho_pq(i) = w_i phi_p(i) phi_q(i), V_rs(i) the vector pair field of step (b) (xtc_vfield),
 * summed over the context's outer range (xtc_set_outer_range; the whole grid by default).
 *   n_grid >= 1, 1 <= n_orb <= XTC_THREE_BODY_MAX_ORB; grid_xyz, weights, phi as in xtc_build_1b2b
 *   L [n_orb]^6 FP64, host or device memory (n_orb = 24: 1.5 GB)
 * V is formed in the context's precision (steps a and b); the products and sums over i are FP64.
 * Requires xtc_set_jastrow.  Errors: XTC_ERR_ARG, XTC_ERR_STATE, XTC_ERR_OOM, XTC_ERR_CUDA and
 * those of xtc_vfield. */
#define XTC_THREE_BODY_MAX_ORB 24
XTC_API int xtc_three_body_L(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz, const double* weights,
                     const double* phi, double* L);

/* The non-hermitian two-body integrals K of the similarity-transformed Hamiltonian (Theory
 * section, next to the Coulomb integrals V; the combined two-body integrals are U = V - K):
 *   K[p][q][r][s] = K_pr^qs = 1/2 <pr| P12 [ lap_1 u + (grad_1 u)^2 + 2 grad_1 u . grad_1 ] |qs>,
 *   P12 f(1,2) = f(1,2) + f(2,1),
 * on the quadrature grid for real spatial orbitals (electron 1: p -> q, electron 2: r -> s; the
 * index order of Delta U), with u the Jastrow factor of xtc_set_jastrow.  K has the pair-swap
 * symmetry K[p][q][r][s] = K[r][s][p][q] and is not hermitian.  Coincident grid points contribute
 * nothing.  Summed over the context's outer range (xtc_set_outer_range): the results of disjoint
 * ranges add up to the whole grid's.
 *   n_grid >= 1, 1 <= n_orb <= XTC_TWO_BODY_K_MAX_ORB; grid_xyz, weights, phi as in xtc_build_1b2b
 *   dphi [n_grid][n_orb][3]  gradients of the orbitals at the grid points (bohr^-1), host or device
 *   K    [n_orb]^4 FP64, host or device memory (n_orb = 120: 1.66 GB)
 * The vector pair field V (steps a and b) is formed in the context's precision; the Laplacian
 * table, its product with the pair densities and the contraction are FP64 (SIMT).  Workspace:
 * n_orb^2 x n_pair doubles plus about 6 GB per chunk of outer points (the context's grid_chunk,
 * else chosen by that budget).  Synchronous.  Requires xtc_set_jastrow.  Errors: XTC_ERR_ARG,
 * XTC_ERR_STATE, XTC_ERR_NONFINITE (grid, weights, orbitals or their gradients), XTC_ERR_OOM,
 * XTC_ERR_CUDA and those of xtc_vfield. */
#define XTC_TWO_BODY_K_MAX_ORB 200
XTC_API int xtc_two_body_K(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz, const double* weights,
                           const double* phi, const double* dphi, double* K);

/* One instance of a batched build: the arguments of xtc_set_jastrow and xtc_build_1b2b, with the
 * same meanings, layouts and ownership; status receives the instance's own status. */
typedef struct xtc_instance {
  int64_t n_grid;
  int n_orb;
  const double* grid_xyz;   /* [n_grid][3] bohr */
  const double* weights;    /* [n_grid] */
  const double* phi;        /* [n_grid][n_orb] */
  const double* gamma;      /* [n_orb][n_orb] per spin, symmetric */
  int n_nuc;
  const double* nuc_xyz;    /* [n_nuc][3] bohr */
  const int* nuc_set;       /* [n_nuc] */
  int n_sets;
  int n_terms;
  const int* mno;           /* [n_terms][3] */
  const double* coef;       /* [n_sets][n_terms] */
  double* dU;               /* [n_orb]^4 or NULL */
  float* dU_f32;            /* [n_orb]^4 or NULL */
  double* dh;               /* [n_orb][n_orb] */
  double* e0;               /* scalar */
  int status;               /* out */
} xtc_instance;

/* Batched build of many molecules (or Jastrow parameter sets) of uneven size: every instance is
 * computed exactly as by xtc_set_jastrow + xtc_build_1b2b on a context with ctx's parameters (the
 * results are bitwise identical).  The instances are spread over n_lanes lanes (0 = automatic,
 * at most 4; at most 16), each a context with its own stream and workspace driven by its own host
 * thread, largest instances first, so that the kernels of small instances overlap on the GPU.
 * Lane contexts are kept in ctx for later batches and released by xtc_destroy.  Inputs written
 * on ctx's stream are waited for first; the call returns when every instance is done (or has
 * failed: the first failing instance's status is returned and named in xtc_last_error_detail).
 * Each lane holds the workspace of its largest instance.  The outer range of ctx does not apply.
 * Lanes are created with ctx's parameters, so a grid_chunk set on ctx (by the caller or by
 * xtc_autotune_chunk for another problem) applies to every instance: leave it 0 for batches of
 * uneven sizes. */
XTC_API int xtc_build_1b2b_batched(xtc_ctx* ctx, int n_inst, xtc_instance* inst, int n_lanes);

/* Kernel timers of the last build (requires params.timing != 0).  Kernel ids: */
enum {
  XTC_K_PREP = 0,     /* per-grid-point tables, orbital transposition, pair products rho (split) */
  XTC_K_VFIELD = 1,   /* step (b) GEMM alone (tensor-core precisions); steps (a)+(b) (XTC_PREC_FP64) */
  XTC_K_FIELDS = 2,   /* step (c) */
  XTC_K_ASSEMBLE = 3, /* step (d): Delta U accumulation (the GEMM alone) */
  XTC_K_FINAL = 4,    /* Delta U unpacking, Delta h, e0 */
  XTC_K_GRAD = 5,     /* step (a) gradient table of the tensor-core precisions */
  XTC_K_AUX = 6,      /* around the tensor-core GEMMs: the kernels that write V or add into M from
                         the FP64 tile sums, and the fp16 row splits of step (d) */
  XTC_N_KERNELS = 7
};
/* ms[k] = summed device milliseconds of kernel class k over the last build, launches[k] = launch
 * count; either pointer may be NULL.  n = array length (>= XTC_N_KERNELS). */
XTC_API int xtc_get_timings(xtc_ctx* ctx, double* ms, int64_t* launches, int n);

/* Revision number of the tensor-core GEMM engine (steps (b) and (d)), raised whenever its code
 * changes.  Profiler counters recorded for one revision (DRAM traffic per launch, for instance)
 * describe that revision only.  Needs no GPU and no context. */
XTC_API int xtc_engine_revision(void);

/* Allocation-free variant of xtc_vfield, for callers that must not allocate device memory (for
 * instance code that runs inside a host framework owning every allocation, or a loop that may
 * not call cudaMalloc).  The paper has no counterpart; it is a deployment convenience.
 * Same computation and output layout as xtc_vfield (steps (a)+(b) in the context's precision), but:
 *   - grid_xyz, weights, phi and V must be device (or managed) pointers on the context's device
 *     (else XTC_ERR_ARG, also for memory of another GPU); nothing is staged through host memory;
 *   - the tensor-core precisions keep their running sums in FP32 for the whole inner sum (no
 *     FP64 flush every 8,192 inner points, which xtc_vfield does), so results differ from
 *     xtc_vfield by FP32 rounding that grows with n_grid;
 *   - all workspace comes from one fixed device array of XTC_NOALLOC_SCRATCH_MIB MiB built into
 *     the library (every GPU that loads the library holds it until the process exits); problems
 *     whose workspace does not fit (with P = 2 parts for fp16x2, 3 for bf16x3, 4 for FP64:
 *     about n_grid * P * (n_orb^2 + 800) bytes for the pair and gradient tables) are rejected
 *     with XTC_ERR_ARG before any device work;
 *   - the call makes no device allocation (no cudaMalloc, cudaFree or allocating library call).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress).
 * Every call reuses the same array, which keeps the
 * last call's contents: calls that overlap on the GPU race with each other, so serialise them.
 * The call is synchronous with respect to the host, like the others: it synchronises the
 * context's stream before returning.  The calling thread's current device is restored. */
#define XTC_NOALLOC_SCRATCH_MIB 64
XTC_API int xtc_vfield_noalloc(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz,
                               const double* weights, const double* phi, int64_t outer_begin, int64_t outer_end,
                               double* V);

#ifdef __cplusplus
}
#endif
#endif /* XTC_H */
