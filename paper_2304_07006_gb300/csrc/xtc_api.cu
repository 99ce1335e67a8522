// Host side of the xTC library: the C ABI of include/xtc.h, input validation, the
// factorisation of gamma, the device workspace, TMA descriptors and the chunked build loop.
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/xtc.h"
#include "xtc_internal.cuh"

using namespace xtc;

namespace {

// A device workspace buffer of a context; owner gives the context's allocator (the caller's
// alloc/release callbacks, or cudaMalloc/cudaFree when they are NULL) and stream.
struct DBuf {
  void* p = nullptr;
  size_t n = 0;
  const xtc_params* owner = nullptr;
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
};

void release(DBuf& b) {
  if (b.p) {
    if (b.owner && b.owner->release) {
      // a caller allocator may hand the memory out again at once: the context's work on it ends first
      cudaStreamSynchronize(static_cast<cudaStream_t>(b.owner->stream));
      b.owner->release(b.p, b.owner->alloc_user);
    } else {
      cudaFree(b.p);
    }
  }
  b.p = nullptr;
  b.n = 0;
}

bool ensure(DBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.n >= bytes) return true;
  release(b);
  if (b.owner && b.owner->alloc) {
    b.p = b.owner->alloc(bytes, b.owner->alloc_user);
    if (!b.p) return false;
  } else if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return false;
  }
  b.n = bytes;
  return true;
}

// NVTX range for profilers (a no-op unless a tool is attached): the build, each chunk, each step.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct TimedLaunch {
  int kind;
  cudaEvent_t a, b;
};

constexpr int RANK_GROUP = 16;
constexpr int MAX_ORB = 320;

}  // namespace

struct xtc_ctx {
  xtc_params prm{};
  cudaStream_t st = nullptr;
  int n_sm = 0;
  JastrowParams jp{};
  bool jastrow_set = false;
  double g_bound = 0.0;  // bound on |nabla_1 u|
  int64_t outer_begin = 0, outer_end = -1;
  char detail[512] = {0};
  // device workspace
  DBuf jp_dev, err_dev, flag_dev;
  DBuf grid, w, phi, gamma, phiT, phi32, pair_p, pair_q;
  DBuf jtab, jtab64, rho, colmax, colexp, G;
  DBuf V, Vacc, L, R, L32, R32, eL, eR, M, evec, lam, dU_tmp, dh_tmp, e0_tmp, vout, r1, r2;
  DBuf lamd, gamma_b, M2, M3;  // direct weights; spin builds: beta density, f^b, Delta U^{ab}
  DBuf lam2, R2, R32b, eR2;    // spin builds: beta exchange weights, R for electron-2 beta
  DBuf Lv, T3;                 // explicit three-body L: V of the outer points, the packed T
  DBuf fc_U, fc_h, fc_hout, fc_Uout;  // frozen-core folding: staged host inputs and outputs
  DBuf G2;                     // second gradient table: step (a) of the next chunk on stream st2
  DBuf k_dphi, k_V, k_Ft, k_W, k_S, k_P;  // two-body integrals K: staged gradients, V, F table, W, S, split-K slices
  cudaStream_t st2 = nullptr;  // created on first use
  cudaEvent_t ev_g[2] = {nullptr, nullptr};  // gradient table b written
  cudaEvent_t ev_b[2] = {nullptr, nullptr};  // step (b) GEMM that read table b done
  // prepared state key (pair tables)
  int pair_n = -1;
  // timers
  std::vector<TimedLaunch> timed;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  double ms[XTC_N_KERNELS] = {0};
  int64_t launches[XTC_N_KERNELS] = {0};
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  int vf_kd = 2;  // K-blocks per tensor-core accumulation range in step (b)
  int vf_flush = 8192;  // inner points (K values) between FP64 flushes of the running sums (0: FP32 only)
  int as_kd = 2;  // the same for step (d)
  int x_period = 64;  // fp16 engine: K-blocks between drains of the cross-product accumulator
  // batched builds: lane contexts, each with its own stream (created on first use)
  std::vector<xtc_ctx*> lanes;
  std::vector<cudaStream_t> lane_streams;

  std::vector<DBuf*> buffers() {
    return {&jp_dev, &err_dev, &flag_dev, &grid, &w, &phi, &gamma, &phiT, &phi32, &pair_p, &pair_q, &jtab, &jtab64,
            &rho, &colmax, &colexp, &G, &V, &Vacc, &L, &R, &L32, &R32, &eL, &eR, &M, &evec, &lam, &dU_tmp,
            &dh_tmp, &e0_tmp, &vout, &r1, &r2, &lamd, &gamma_b, &M2, &M3, &lam2, &R2, &R32b, &eR2, &Lv, &T3,
            &fc_U, &fc_h, &fc_hout, &fc_Uout, &G2, &k_dphi, &k_V, &k_Ft, &k_W, &k_S, &k_P};
  }
};

namespace {

int fail(xtc_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->detail, sizeof(c->detail), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CUDA_OK(call)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(ctx, XTC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cudaEvent_t next_event(xtc_ctx* c) {
  if (c->pool_used == c->pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->pool.push_back(e);
  }
  return c->pool[c->pool_used++];
}

// Runs `fn` (which launches kernels of class `kind`, `count` of them) bracketed by events when timing.
// The events go on stream `st` (default: the context's stream), the one the launches use.
template <typename F>
void timed(xtc_ctx* c, int kind, int count, F&& fn, cudaStream_t st) {
  c->launches[kind] += count;
  if (!c->prm.timing) {
    fn();
    return;
  }
  TimedLaunch t{kind, next_event(c), next_event(c)};
  cudaEventRecord(t.a, st);
  fn();
  cudaEventRecord(t.b, st);
  c->timed.push_back(t);
}
template <typename F>
void timed(xtc_ctx* c, int kind, int count, F&& fn) {
  timed(c, kind, count, static_cast<F&&>(fn), c->st);
}

void reset_timers(xtc_ctx* c) {
  c->timed.clear();
  c->pool_used = 0;
  for (int k = 0; k < XTC_N_KERNELS; ++k) {
    c->ms[k] = 0.0;
    c->launches[k] = 0;
  }
}

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (row-major).  On return a holds
// the eigenvalues on its diagonal and v (row-major) the eigenvectors as columns.
void jacobi_eigen(std::vector<double>& a, std::vector<double>& v, int n) {
  v.assign(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i) v[static_cast<size_t>(i) * n + i] = 1.0;
  double total = 0.0;
  for (double x : a) total += x * x;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += a[static_cast<size_t>(p) * n + q] * a[static_cast<size_t>(p) * n + q];
    if (off <= 1e-32 * total || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[static_cast<size_t>(p) * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = a[static_cast<size_t>(p) * n + p], aqq = a[static_cast<size_t>(q) * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = a[static_cast<size_t>(k) * n + p], akq = a[static_cast<size_t>(k) * n + q];
          a[static_cast<size_t>(k) * n + p] = c * akp - s * akq;
          a[static_cast<size_t>(k) * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = a[static_cast<size_t>(p) * n + k], aqk = a[static_cast<size_t>(q) * n + k];
          a[static_cast<size_t>(p) * n + k] = c * apk - s * aqk;
          a[static_cast<size_t>(q) * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = v[static_cast<size_t>(k) * n + p], vkq = v[static_cast<size_t>(k) * n + q];
          v[static_cast<size_t>(k) * n + p] = c * vkp - s * vkq;
          v[static_cast<size_t>(k) * n + q] = s * vkp + c * vkq;
        }
      }
  }
}

int make_tmap_3d(xtc_ctx* ctx, CUtensorMap* tm, void* base, bool bf16, uint64_t d0, uint64_t d1, uint64_t d2,
                 uint32_t b0, uint32_t b1, bool sw128 = false) {
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {d0 * 2, d0 * d1 * 2};
  const cuuint32_t box[3] = {b0, b1, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  CUresult r = ctx->encode(tm, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, base, dims,
                           strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           sw128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, XTC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return XTC_OK;
}

// Copies (or aliases) an input array into device memory.
int stage_input(xtc_ctx* ctx, DBuf& buf, const double* src, size_t count, const double** dev) {
  if (is_device_ptr(src)) {
    *dev = src;
    return XTC_OK;
  }
  if (!ensure(buf, count * sizeof(double))) return fail(ctx, XTC_ERR_OOM, "input staging (%zu bytes)", count * 8);
  CUDA_OK(cudaMemcpyAsync(buf.p, src, count * sizeof(double), cudaMemcpyHostToDevice, ctx->st));
  *dev = buf.as<double>();
  return XTC_OK;
}

struct Plan {
  int N, NP;
  int64_t NG, NGp;
  int64_t ob, oe;    // outer range
  int64_t gc;        // chunk length (multiple of 128)
  int splits;
  int parts_b;       // step (b) parts (2 fp16 / 3 bf16), 0 = FP64
  bool f64;
};

// budget_scale < 1 shrinks the memory budgets (the autotuner's smaller candidates).
int64_t auto_chunk(const xtc_ctx* c, int NP, int64_t NGp, int parts, int64_t n_outer, bool f64,
                   double budget_scale = 1.0) {
  // memory budgets: 12 GB for V and the step (d) operands, 16 GB for the step (a) gradient table;
  // then the chunk that fills whole waves of the step (b) GEMM best
  const double vbytes = f64 ? 3.0 * 8 : 3.0 * 4;
  // step (d) operands per pair and outer point: FP64 L, R; bf16 x3 L, R; or FP32 L, R + fp16 x2 split
  // and the fp16(R) plane
  const double lrbytes = f64 ? 2 * 4 * 8.0 : (parts == 2 ? 2 * 4 * (4.0 + 4.0) + 4 * 2.0 : 2 * 3 * 4 * 2.0);
  // V holds the whole N x N matrix per point (N^2 < 2 NP)
  const double per_point = NP * (2.0 * vbytes + lrbytes);
  int64_t cap = static_cast<int64_t>(budget_scale * 12.0e9 / per_point);
  if (!f64) cap = std::min<int64_t>(cap, static_cast<int64_t>(budget_scale * 16.0e9 / (3.0 * parts * 2.0 * NGp)));
  cap = std::max<int64_t>(128, std::min<int64_t>(cap, static_cast<int64_t>(budget_scale * 32768)) / 128 * 128);
  const int64_t need = round_up(n_outer, 128);
  if (need <= cap) return need;
  const int nt = f64 ? 1 : (NP + vf_bn(parts) - 1) / vf_bn(parts);
  int64_t best = cap;
  double best_eff = 0.0;
  for (int64_t tiles = cap / 128; tiles >= std::max<int64_t>(1, cap / 256); --tiles) {
    const double ctas = 3.0 * tiles * nt;
    const double eff = ctas / (std::ceil(ctas / c->n_sm) * c->n_sm);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = tiles * 128;
    }
  }
  return best;
}

// Stages per exact accumulation range of the fp16 engine: the largest of 1, 2, 4 not above k (the
// split tables hold one quantum per range, and chunk and grid lengths are multiples of 128 points).
int f16_range(int k) { return k >= 4 ? 4 : (k >= 2 ? 2 : 1); }
int f16_range_b(int k) { return f16_range(k); }

// Ranges of kd stages (32 K values each) between FP64 flushes for a flush interval of `points` K
// values (0: no flushes).
int flush_ranges(int points, int kd) { return points > 0 ? std::max(1, points / (32 * kd)) : 0; }

int choose_pts(int N, int R, bool f64, bool spin) {
  for (int p : {8, 4, 2, 1})
    if (fields_smem_bytes(N, R, p, f64, spin) <= 200 * 1024) return p;
  return 0;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void xtc_default_params(xtc_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->device = 0;
  p->stream = nullptr;
  p->precision = XTC_PREC_FP16X2;
  p->grid_chunk = 0;
  p->split_k = 0;
  p->timing = 0;
}

const char* xtc_strerror(int s) {
  switch (s) {
    case XTC_OK: return "success";
    case XTC_ERR_ARG: return "invalid argument";
    case XTC_ERR_NOT_SYMMETRIC: return "gamma is not symmetric";
    case XTC_ERR_NONFINITE: return "non-finite input";
    case XTC_ERR_OOM: return "device allocation failed";
    case XTC_ERR_CUDA: return "CUDA error";
    case XTC_ERR_TIMEOUT: return "device-side wait timed out";
    case XTC_ERR_STATE: return "context not ready (xtc_set_jastrow missing?)";
    case XTC_ERR_UNSUPPORTED: return "unsupported device or configuration";
    default: return "unknown status";
  }
}

const char* xtc_last_error_detail(const xtc_ctx* ctx) { return ctx ? ctx->detail : "null context"; }

int xtc_create(xtc_ctx** out, const xtc_params* p) {
  if (!out || !p) return XTC_ERR_ARG;
  *out = nullptr;
  if (p->precision < XTC_PREC_FP64 || p->precision > XTC_PREC_BF16X3) return XTC_ERR_ARG;
  if (p->grid_chunk < 0 || p->grid_chunk % 128 != 0 || p->split_k < 0 || p->split_k > 16) return XTC_ERR_ARG;
  if (p->range_stages < 0 || p->range_stages > 4) return XTC_ERR_ARG;
  if ((p->alloc == nullptr) != (p->release == nullptr)) return XTC_ERR_ARG;
  if (cudaSetDevice(p->device) != cudaSuccess) {
    cudaGetLastError();
    return XTC_ERR_CUDA;
  }
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, p->device) != cudaSuccess) return XTC_ERR_CUDA;
  if (prop.major < 10) return XTC_ERR_UNSUPPORTED;
  xtc_ctx* ctx = new xtc_ctx();
  ctx->prm = *p;
  ctx->st = static_cast<cudaStream_t>(p->stream);
  for (DBuf* b : ctx->buffers()) b->owner = &ctx->prm;
  ctx->n_sm = prop.multiProcessorCount;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    delete ctx;
    return XTC_ERR_CUDA;
  }
  ctx->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  if (const char* s = std::getenv("XTC_VF_KD")) ctx->vf_kd = std::max(1, std::atoi(s));
  if (const char* s = std::getenv("XTC_AS_KD")) ctx->as_kd = std::max(1, std::atoi(s));
  if (const char* s = std::getenv("XTC_VF_FLUSH")) ctx->vf_flush = std::max(0, std::atoi(s));
  if (const char* s = std::getenv("XTC_X_PERIOD")) ctx->x_period = std::max(1, std::atoi(s));
  if (p->range_stages > 0) ctx->vf_kd = ctx->as_kd = p->range_stages;
  if (!ensure(ctx->jp_dev, sizeof(JastrowParams)) || !ensure(ctx->err_dev, 16) || !ensure(ctx->flag_dev, 16)) {
    xtc_destroy(ctx);
    return XTC_ERR_OOM;
  }
  *out = ctx;
  return XTC_OK;
}

int xtc_destroy(xtc_ctx* ctx) {
  if (!ctx) return XTC_OK;
  cudaSetDevice(ctx->prm.device);
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  else cudaDeviceSynchronize();
  for (DBuf* b : ctx->buffers()) release(*b);
  for (xtc_ctx* lane : ctx->lanes) xtc_destroy(lane);
  for (cudaStream_t s : ctx->lane_streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
  for (int b = 0; b < 2; ++b) {
    if (ctx->ev_g[b]) cudaEventDestroy(ctx->ev_g[b]);
    if (ctx->ev_b[b]) cudaEventDestroy(ctx->ev_b[b]);
  }
  if (ctx->st2) cudaStreamDestroy(ctx->st2);
  delete ctx;
  return XTC_OK;
}

int xtc_set_jastrow(xtc_ctx* ctx, int n_nuc, const double* nuc_xyz, const int* nuc_set, int n_sets, int n_terms,
                    const int* mno, const double* coef) {
  if (!ctx) return XTC_ERR_ARG;
  if (n_nuc < 1 || n_nuc > MAX_NUC || n_sets < 1 || n_sets > MAX_SETS || n_terms < 1 || n_terms > MAX_TERMS ||
      !nuc_xyz || !nuc_set || !mno || !coef)
    return fail(ctx, XTC_ERR_ARG, "set_jastrow: bad sizes or null pointer");
  JastrowParams jp{};
  jp.n_nuc = n_nuc;
  jp.n_terms = n_terms;
  jp.n_sets = n_sets;
  double bound = 0.0;
  for (int I = 0; I < n_nuc; ++I) {
    for (int k = 0; k < 3; ++k) {
      if (!std::isfinite(nuc_xyz[3 * I + k])) return fail(ctx, XTC_ERR_NONFINITE, "nucleus coordinate");
      jp.nuc[I][k] = nuc_xyz[3 * I + k];
    }
    if (nuc_set[I] < 0 || nuc_set[I] >= n_sets) return fail(ctx, XTC_ERR_ARG, "nuc_set[%d] out of range", I);
    jp.set[I] = nuc_set[I];
  }
  for (int t = 0; t < n_terms; ++t)
    for (int k = 0; k < 3; ++k) {
      if (mno[3 * t + k] < 0 || mno[3 * t + k] > 2) return fail(ctx, XTC_ERR_ARG, "term %d: powers must be 0..2", t);
      jp.mno[t][k] = mno[3 * t + k];
    }
  for (int s = 0; s < n_sets; ++s)
    for (int t = 0; t < n_terms; ++t) {
      const double c = coef[s * n_terms + t];
      if (!std::isfinite(c)) return fail(ctx, XTC_ERR_NONFINITE, "Jastrow coefficient");
      jp.coef[s][t] = c;
    }
  // |nabla_1 u| <= sum_I sum_t |c| (m + n + 2 o): a, b, a', b' are all in [0, 1]
  for (int I = 0; I < n_nuc; ++I)
    for (int t = 0; t < n_terms; ++t)
      bound += std::fabs(jp.coef[jp.set[I]][t]) * (jp.mno[t][0] + jp.mno[t][1] + 2.0 * jp.mno[t][2]);
  cudaSetDevice(ctx->prm.device);
  // on the context's stream (a plain cudaMemcpy is not ordered with non-blocking streams)
  CUDA_OK(cudaMemcpyAsync(ctx->jp_dev.p, &jp, sizeof(jp), cudaMemcpyHostToDevice, ctx->st));
  CUDA_OK(cudaStreamSynchronize(ctx->st));
  ctx->jp = jp;
  ctx->g_bound = bound;
  ctx->jastrow_set = true;
  return XTC_OK;
}

int xtc_set_outer_range(xtc_ctx* ctx, int64_t begin, int64_t end) {
  if (!ctx || begin < 0 || (end >= 0 && end < begin)) return XTC_ERR_ARG;
  ctx->outer_begin = begin;
  ctx->outer_end = end;
  return XTC_OK;
}

// 1: one accumulator per range of kd stages, truncating FP32 accumulation (192-column tiles);
// 2: exact fp16 split on per-range quanta, an exact hi x hi accumulator and a cross-product
//    accumulator per issuer (128-column tiles);
// 3: plus the fp16 plane of rho^T in step (b) and a commit per stage that frees its slot;
// 4: step (d) on an fp16 plane of R as well (three products), drains waiting without suspending;
// 5: tiles ordered in groups of 16 row tiles (8 before).
int xtc_engine_revision(void) { return 5; }

int xtc_get_timings(xtc_ctx* ctx, double* ms, int64_t* launches, int n) {
  if (!ctx || n < XTC_N_KERNELS) return XTC_ERR_ARG;
  if (ms) for (int k = 0; k < XTC_N_KERNELS; ++k) ms[k] = ctx->ms[k];
  if (launches) for (int k = 0; k < XTC_N_KERNELS; ++k) launches[k] = ctx->launches[k];
  return XTC_OK;
}

}  // extern "C"

// ====================================================================== build
namespace {

int finish_timers(xtc_ctx* ctx) {
  for (const TimedLaunch& t : ctx->timed) {
    float m = 0.0f;
    if (cudaEventElapsedTime(&m, t.a, t.b) == cudaSuccess) ctx->ms[t.kind] += m;
  }
  cudaGetLastError();
  return XTC_OK;
}

int check_device_error(xtc_ctx* ctx) {
  int h[2] = {0, 0};
  CUDA_OK(cudaMemcpyAsync(h, ctx->err_dev.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CUDA_OK(cudaStreamSynchronize(ctx->st));
  if (h[0] != 0) return fail(ctx, XTC_ERR_TIMEOUT, "device wait timed out (code %d)", h[0]);
  return XTC_OK;
}

// Common preparation of grid-wide tables.  Fills the plan.
int prepare(xtc_ctx* ctx, Plan& pl, int64_t n_grid, int n_orb, const double* grid_xyz, const double* weights,
            const double* phi, const double** d_grid, const double** d_w, const double** d_phi) {
  if (!ctx->jastrow_set) return fail(ctx, XTC_ERR_STATE, "xtc_set_jastrow has not been called");
  if (n_grid < 1 || n_orb < 1 || n_orb > MAX_ORB || !grid_xyz || !weights || !phi)
    return fail(ctx, XTC_ERR_ARG, "bad sizes (n_grid=%lld, n_orb=%d) or null input", (long long)n_grid, n_orb);
  const bool f64 = ctx->prm.precision == XTC_PREC_FP64;
  if (!f64 && !vfield_tc_supported(ctx->jp.n_nuc))
    return fail(ctx, XTC_ERR_UNSUPPORTED, "the tensor-core path supports 1..8 nuclei (got %d)", ctx->jp.n_nuc);
  pl.N = n_orb;
  pl.NP = n_orb * (n_orb + 1) / 2;
  pl.NG = n_grid;
  pl.NGp = round_up(n_grid, 128);
  pl.f64 = f64;
  pl.parts_b = f64 ? 0 : (ctx->prm.precision == XTC_PREC_FP16X2 ? 2 : 3);
  pl.ob = std::min<int64_t>(ctx->outer_begin, n_grid);
  pl.oe = ctx->outer_end < 0 ? n_grid : std::min<int64_t>(ctx->outer_end, n_grid);
  if (pl.oe < pl.ob) pl.oe = pl.ob;
  const int64_t n_outer = pl.oe - pl.ob;
  pl.gc = ctx->prm.grid_chunk > 0 ? ctx->prm.grid_chunk
                                   : auto_chunk(ctx, pl.NP, pl.NGp, pl.parts_b, std::max<int64_t>(n_outer, 1), f64);
  const int n_kb = static_cast<int>(pl.NGp / VF_BK);
  pl.splits = ctx->prm.split_k > 0 ? std::min(ctx->prm.split_k, n_kb) : 1;
  if (f64) pl.splits = 1;

  cudaStream_t st = ctx->st;
  int rc;
  if ((rc = stage_input(ctx, ctx->grid, grid_xyz, static_cast<size_t>(n_grid) * 3, d_grid))) return rc;
  if ((rc = stage_input(ctx, ctx->w, weights, static_cast<size_t>(n_grid), d_w))) return rc;
  if ((rc = stage_input(ctx, ctx->phi, phi, static_cast<size_t>(n_grid) * n_orb, d_phi))) return rc;

  CUDA_OK(cudaMemsetAsync(ctx->flag_dev.p, 0, 16, st));
  CUDA_OK(cudaMemsetAsync(ctx->err_dev.p, 0, 16, st));
  timed(ctx, XTC_K_PREP, 3, [&] {
    launch_check_finite(*d_grid, n_grid * 3, ctx->flag_dev.as<int>(), st);
    launch_check_finite(*d_w, n_grid, ctx->flag_dev.as<int>(), st);
    launch_check_finite(*d_phi, n_grid * n_orb, ctx->flag_dev.as<int>(), st);
  });
  int flag = 0;
  CUDA_OK(cudaMemcpyAsync(&flag, ctx->flag_dev.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_OK(cudaStreamSynchronize(st));
  if (flag) return fail(ctx, XTC_ERR_NONFINITE, "NaN or Inf in grid, weights or orbitals");

  if (ctx->pair_n != n_orb) {
    std::vector<int> pp(pl.NP), pq(pl.NP);
    int k = 0;
    for (int p = 0; p < n_orb; ++p)
      for (int q = p; q < n_orb; ++q) {
        pp[k] = p;
        pq[k] = q;
        ++k;
      }
    if (!ensure(ctx->pair_p, pl.NP * sizeof(int)) || !ensure(ctx->pair_q, pl.NP * sizeof(int)))
      return fail(ctx, XTC_ERR_OOM, "pair tables");
    CUDA_OK(cudaMemcpyAsync(ctx->pair_p.p, pp.data(), pl.NP * sizeof(int), cudaMemcpyHostToDevice, st));
    CUDA_OK(cudaMemcpyAsync(ctx->pair_q.p, pq.data(), pl.NP * sizeof(int), cudaMemcpyHostToDevice, st));
    CUDA_OK(cudaStreamSynchronize(st));  // pp and pq are released on return
    ctx->pair_n = n_orb;
  }
  if (!ensure(ctx->phiT, sizeof(double) * pl.NGp * n_orb)) return fail(ctx, XTC_ERR_OOM, "phiT");
  const int n_nuc = ctx->jp.n_nuc;
  if (f64) {
    if (!ensure(ctx->jtab64, sizeof(double) * pl.NGp * (3 + n_nuc)) ||
        !ensure(ctx->rho, sizeof(double) * pl.NGp * pl.NP))
      return fail(ctx, XTC_ERR_OOM, "FP64 grid tables (%.2f GB)", 8.0 * pl.NGp * pl.NP / 1e9);
  } else {
    const int js = jtab_stride(n_nuc);
    if (!ensure(ctx->jtab, sizeof(float) * pl.NGp * js) ||
        !ensure(ctx->rho, 2ull * 3 * pl.NGp * pl.NP) || !ensure(ctx->colmax, 4ull * pl.NP) ||
        !ensure(ctx->colexp, 4ull * pl.NP) || !ensure(ctx->phi32, 8ull * (n_orb + 1) * pl.NGp))
      return fail(ctx, XTC_ERR_OOM, "grid tables (%.2f GB)", 2.0 * 3 * pl.NGp * pl.NP / 1e9);
  }
  const int nprep = f64 ? 3 : (pl.parts_b == 2 ? 5 : 3);
  timed(ctx, XTC_K_PREP, nprep, [&] {
    launch_transpose_phi(*d_phi, n_grid, pl.NGp, n_orb, ctx->phiT.as<double>(), st);
    if (f64) {
      launch_jtab64(*d_grid, n_grid, pl.NGp, ctx->jp_dev.as<JastrowParams>(), n_nuc, ctx->jtab64.as<double>(), st);
      launch_rho_f64(*d_phi, *d_w, n_grid, pl.NGp, n_orb, ctx->pair_p.as<int>(), ctx->pair_q.as<int>(),
                     ctx->rho.as<double>(), st);
    } else {
      const int js = jtab_stride(n_nuc);
      launch_jtab(*d_grid, n_grid, pl.NGp, ctx->jp_dev.as<JastrowParams>(), n_nuc, js, ctx->jtab.as<float>(), st);
      launch_rho_split(ctx->phiT.as<double>(), *d_w, n_grid, pl.NGp, n_orb, pl.parts_b, f16_range_b(ctx->vf_kd),
                       ctx->pair_p.as<int>(), ctx->pair_q.as<int>(), ctx->colmax.as<unsigned int>(),
                       ctx->colexp.as<int>(), ctx->phi32.as<float>(), ctx->rho.p, st);
    }
  });
  const size_t vbytes = static_cast<size_t>(pl.splits) * v_slice(pl.gc, pl.N) * (f64 ? 8 : 4);
  if (!ensure(ctx->V, vbytes)) return fail(ctx, XTC_ERR_OOM, "V chunk (%.2f GB)", vbytes / 1e9);
  if (!f64) {
    const size_t gbytes = 2ull * pl.parts_b * 3 * pl.gc * pl.NGp;
    if (!ensure(ctx->G, gbytes)) return fail(ctx, XTC_ERR_OOM, "gradient table (%.2f GB)", gbytes / 1e9);
    // FP64 partial sums of step (b): one 128 x vf_bn tile per CTA and split slice
    const int bn = vf_bn(pl.parts_b);
    const size_t tiles = 3ull * ((pl.gc + VF_BM - 1) / VF_BM) * ((pl.NP + bn - 1) / bn);
    const size_t abytes = ctx->vf_flush > 0 ? 8ull * pl.splits * tiles * VF_BM * bn : 0;
    if (!ensure(ctx->Vacc, abytes)) return fail(ctx, XTC_ERR_OOM, "step (b) FP64 sums (%.2f GB)", abytes / 1e9);
  }
  return XTC_OK;
}

// Tensor maps of the step (b) operands: rho^T (box rows vf_bn) and the gradient table, as stored by
// step (a) (box rows 32) and as loaded by the GEMM (box rows 128).  fp16: both parts of a 32-point
// block in one 128-byte row (rows of 2 NGp values, boxes 64 wide, 128-byte swizzle); bf16: one
// plane per part (rows of NGp values, boxes 32 wide, 64-byte swizzle).
struct VfMaps {
  CUtensorMap rho, rho16, g_store, g_load;
};
int make_vfield_maps(xtc_ctx* ctx, const Plan& pl, VfMaps& m) {
  if (pl.f64) return XTC_OK;
  const bool bf = pl.parts_b == 3, wide = pl.parts_b == 2;
  const uint64_t cols = wide ? 2 * pl.NGp : pl.NGp, planes = wide ? 1 : pl.parts_b;
  const uint32_t bk = wide ? 2 * VF_BK : VF_BK;
  int rc;
  if ((rc = make_tmap_3d(ctx, &m.rho, ctx->rho.p, bf, cols, pl.NP, planes, bk, vf_bn(pl.parts_b), wide))) return rc;
  // fp16: the plane of fp16(rho^T) after the split rows, boxes 32 wide (64-byte swizzle)
  if (wide && (rc = make_tmap_3d(ctx, &m.rho16, ctx->rho.as<uint16_t>() + 2 * pl.NP * pl.NGp, false, pl.NGp, pl.NP, 1,
                                 VF_BK, vf_bn(2))))
    return rc;
  if ((rc = make_tmap_3d(ctx, &m.g_store, ctx->G.p, bf, cols, 3 * pl.gc, planes, bk, 32, wide))) return rc;
  return make_tmap_3d(ctx, &m.g_load, ctx->G.p, bf, cols, 3 * pl.gc, planes, bk, VF_BM, wide);
}

// fp16 gradient scale 2^sG keeps |G| below 16384 (bf16 needs none)
int gradient_scale(const xtc_ctx* ctx, const Plan& pl) {
  if (pl.parts_b != 2 || !(ctx->g_bound > 0.0)) return 0;
  const int sg = static_cast<int>(std::floor(std::log2(16384.0 / ctx->g_bound)));
  return std::max(-30, std::min(30, sg));
}

// Step (a) for outer points [i0, i0 + n_i): the gradient table behind `maps`, on stream `st`.
void run_grad(xtc_ctx* ctx, const Plan& pl, const double* d_grid, int64_t i0, int64_t n_i, const VfMaps& maps,
              cudaStream_t st) {
  const int n_kb = static_cast<int>(pl.NGp / VF_BK);
  const int mt_per_x = static_cast<int>((n_i + VF_BM - 1) / VF_BM);
  GfieldArgs g{};
  g.grid = d_grid;
  g.jp = ctx->jp_dev.as<JastrowParams>();
  g.jtab = ctx->jtab.as<float>();
  g.i0 = i0;
  g.n_i = n_i;
  g.gcp = pl.gc;
  g.n_tiles = mt_per_x * (VF_BM / 32);
  g.n_kb = n_kb;
  g.kb_per_seg = 32;
  g.n_seg = (n_kb + g.kb_per_seg - 1) / g.kb_per_seg;
  g.n_nuc = ctx->jp.n_nuc;
  g.g_scale = std::ldexp(1.0f, gradient_scale(ctx, pl));
  g.range_blocks = f16_range_b(ctx->vf_kd);
  timed(ctx, XTC_K_GRAD, 1, [&] { launch_gfield(&maps.g_store, g, pl.parts_b, st); }, st);
}

// Step (b) for outer points [i0, i0 + n_i) from the gradient table behind `maps`, into ctx->V.
void run_gemm_b(xtc_ctx* ctx, const Plan& pl, int64_t n_i, const VfMaps& maps) {
  cudaStream_t st = ctx->st;
  const int n_kb = static_cast<int>(pl.NGp / VF_BK);
  VfieldArgs a{};
  a.colexp = ctx->colexp.as<int>();
  a.V = ctx->V.as<float>();
  a.pair_p = ctx->pair_p.as<int>();
  a.pair_q = ctx->pair_q.as<int>();
  a.n_orb = pl.N;
  a.Vacc = ctx->Vacc.as<double>();
  a.n_i = n_i;
  a.gcp = pl.gc;
  a.mt_per_x = static_cast<int>((n_i + VF_BM - 1) / VF_BM);
  a.n_tiles = (pl.NP + vf_bn(pl.parts_b) - 1) / vf_bn(pl.parts_b);
  a.n_pair = pl.NP;
  a.n_kb = n_kb;
  a.kb_per_split = (a.n_kb + pl.splits - 1) / pl.splits;
  a.kd = pl.parts_b == 2 ? f16_range_b(ctx->vf_kd) : std::min(ctx->vf_kd, 2);
  a.xper = ctx->x_period;
  a.flush = flush_ranges(ctx->vf_flush, a.kd);
  a.unscale_g = std::ldexp(1.0f, -gradient_scale(ctx, pl));
  a.err = ctx->err_dev.as<int>();
  const int splits = (a.n_kb + a.kb_per_split - 1) / a.kb_per_split;  // every slice non-empty
  // the GEMM, then (FP64 flushes) the kernel that writes V from the FP64 sums
  timed(ctx, XTC_K_VFIELD, 1, [&] { launch_vfield_tc(&maps.g_load, &maps.rho, &maps.rho16, a, pl.parts_b, splits, st); });
  if (a.flush > 0) timed(ctx, XTC_K_AUX, 1, [&] { launch_vfield_tc_finalize(a, pl.parts_b, splits, st); });
}

// Steps (a)+(b) for outer points [i0, i0 + n_i) into ctx->V, on the context's stream.
int run_vfield(xtc_ctx* ctx, const Plan& pl, const double* d_grid, int64_t i0, int64_t n_i, const VfMaps& maps) {
  cudaStream_t st = ctx->st;
  if (pl.f64) {
    timed(ctx, XTC_K_VFIELD, 1, [&] {
      launch_vfield_f64_impl(d_grid, ctx->jp_dev.as<JastrowParams>(), ctx->jp.n_nuc, ctx->jtab64.as<double>(),
                             ctx->rho.as<double>(), pl.NGp, pl.NP, i0, n_i, pl.gc, ctx->pair_p.as<int>(),
                             ctx->pair_q.as<int>(), pl.N, ctx->V.as<double>(), st);
    });
    return XTC_OK;
  }
  run_grad(ctx, pl, d_grid, i0, n_i, maps, st);
  run_gemm_b(ctx, pl, n_i, maps);
  return XTC_OK;
}

}  // namespace

namespace {

// One density matrix, read, checked and factorised on the host: gamma = sum_k lam_k c_k c_k^T
// (cyclic Jacobi, exact to rounding), eigenvalues below 1e-13 of the largest dropped.
struct Density {
  std::vector<double> g, lam, ev;  // ev[k][p]
  int rank = 0;
};

int read_density(xtc_ctx* ctx, const double* gamma, int N, const char* name, Density& d) {
  cudaStream_t st = ctx->st;
  d.g.assign(static_cast<size_t>(N) * N, 0.0);
  if (is_device_ptr(gamma)) {
    CUDA_OK(cudaMemcpyAsync(d.g.data(), gamma, d.g.size() * 8, cudaMemcpyDeviceToHost, st));
    CUDA_OK(cudaStreamSynchronize(st));
  } else {
    std::memcpy(d.g.data(), gamma, d.g.size() * 8);
  }
  double gmax = 0.0, asym = 0.0;
  for (int p = 0; p < N; ++p)
    for (int q = 0; q < N; ++q) {
      const double v = d.g[static_cast<size_t>(p) * N + q];
      if (!std::isfinite(v)) return fail(ctx, XTC_ERR_NONFINITE, "%s has NaN/Inf", name);
      gmax = std::max(gmax, std::fabs(v));
      asym = std::max(asym, std::fabs(v - d.g[static_cast<size_t>(q) * N + p]));
    }
  if (asym > 1e-12 * gmax) return fail(ctx, XTC_ERR_NOT_SYMMETRIC, "max |%s - %s^T| = %g", name, name, asym);
  std::vector<double> a = d.g, vecs;
  jacobi_eigen(a, vecs, N);
  double lmax = 0.0;
  for (int k = 0; k < N; ++k) lmax = std::max(lmax, std::fabs(a[static_cast<size_t>(k) * N + k]));
  d.lam.clear();
  d.ev.clear();
  for (int k = 0; k < N; ++k) {
    const double l = a[static_cast<size_t>(k) * N + k];
    if (std::fabs(l) <= 1e-13 * lmax || l == 0.0) continue;
    d.lam.push_back(l);
    for (int p = 0; p < N; ++p) d.ev.push_back(vecs[static_cast<size_t>(p) * N + k]);
  }
  d.rank = static_cast<int>(d.lam.size());
  return XTC_OK;
}

// What a build writes: the closed-shell Delta U (dU[0] / dU32), Delta h (dh[0]) and e0, or the
// spin blocks aa, ab, bb (dU[0..2]), Delta h^a, Delta h^b (dh[0..1]) and e0.
struct BuildOut {
  int n_spin = 1;
  double* dU[3] = {nullptr, nullptr, nullptr};
  float* dU32 = nullptr;
  double* dh[2] = {nullptr, nullptr};
  double* e0 = nullptr;
};

// One step (c)+(d) pass over the factor list [k0, k0 + rank) into the accumulator M, and for a
// spin build also (electron 2 beta) into M2.
struct Pass {
  int k0, rank;
  DBuf* M;
  DBuf* M2;
};

int build_impl(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz, const double* weights,
               const double* phi, const double* const* gammas, const BuildOut& out) {
  NvtxRange nvtx_build(out.n_spin == 2 ? "xtc build (spin)" : "xtc build");
  CUDA_OK(cudaSetDevice(ctx->prm.device));
  reset_timers(ctx);
  cudaStream_t st = ctx->st;
  const bool spin = out.n_spin == 2;

  // ---- densities: symmetry, finiteness, factorisation
  if (n_orb < 1 || n_orb > MAX_ORB) return fail(ctx, XTC_ERR_ARG, "n_orb=%d out of range", n_orb);
  const int N = n_orb;
  Density dens[2];
  int rc;
  for (int sp = 0; sp < out.n_spin; ++sp)
    if ((rc = read_density(ctx, gammas[sp], N, spin ? (sp ? "gamma_b" : "gamma_a") : "gamma", dens[sp]))) return rc;

  // Factor lists.  Closed shell: exchange weights lam_k, direct weights 2 lam_k (W = 2 V.gamma,
  // Wt = 2 rho.gamma), one pass into M.  Spin build: one pass over the factors of gamma^a and then
  // gamma^b, all with direct weights (the direct density gamma^a + gamma^b, Appendix A), with the
  // alpha exchange weights (lamx: gamma^a's factors) for R into M and the beta ones (lam2:
  // gamma^b's factors) for R2 into M2.
  std::vector<double> ev, lamx, lamd, lam2;
  std::vector<Pass> passes;
  if (!spin) {
    ev = dens[0].ev;
    lamx = dens[0].lam;
    for (double l : dens[0].lam) lamd.push_back(2.0 * l);
    passes.push_back({0, dens[0].rank, &ctx->M, nullptr});
  } else {
    const Density &da = dens[0], &db = dens[1];
    ev = da.ev;
    ev.insert(ev.end(), db.ev.begin(), db.ev.end());
    lamd = da.lam;
    lamd.insert(lamd.end(), db.lam.begin(), db.lam.end());
    lamx = da.lam;
    lamx.insert(lamx.end(), db.lam.size(), 0.0);
    lam2.assign(da.lam.size(), 0.0);
    lam2.insert(lam2.end(), db.lam.begin(), db.lam.end());
    passes.push_back({0, da.rank + db.rank, &ctx->M, &ctx->M2});
  }

  Plan pl{};
  const double *d_grid = nullptr, *d_w = nullptr, *d_phi = nullptr;
  rc = prepare(ctx, pl, n_grid, n_orb, grid_xyz, weights, phi, &d_grid, &d_w, &d_phi);
  if (rc) return rc;
  const int NP = pl.NP;
  const int ldm = static_cast<int>(m_stride(NP));
  const size_t mbytes = 8ull * NP * ldm;

  // ---- device copies of the densities, their factors and the accumulators
  const size_t gbytes = static_cast<size_t>(N) * N * 8;
  if (!ensure(ctx->gamma, gbytes) || (spin && !ensure(ctx->gamma_b, gbytes)) ||
      !ensure(ctx->evec, std::max<size_t>(ev.size(), 1) * 8) || !ensure(ctx->lam, std::max<size_t>(lamx.size(), 1) * 8) ||
      !ensure(ctx->lamd, std::max<size_t>(lamd.size(), 1) * 8) || !ensure(ctx->M, mbytes) ||
      (spin && !ensure(ctx->lam2, std::max<size_t>(lam2.size(), 1) * 8)) ||
      (spin && (!ensure(ctx->M2, mbytes) || !ensure(ctx->M3, mbytes))))
    return fail(ctx, XTC_ERR_OOM, "densities / accumulators (%.2f GB)", (spin ? 3.0 : 1.0) * mbytes / 1e9);
  CUDA_OK(cudaMemcpyAsync(ctx->gamma.p, dens[0].g.data(), gbytes, cudaMemcpyHostToDevice, st));
  if (spin) CUDA_OK(cudaMemcpyAsync(ctx->gamma_b.p, dens[1].g.data(), gbytes, cudaMemcpyHostToDevice, st));
  if (!lamx.empty()) {
    CUDA_OK(cudaMemcpyAsync(ctx->evec.p, ev.data(), ev.size() * 8, cudaMemcpyHostToDevice, st));
    CUDA_OK(cudaMemcpyAsync(ctx->lam.p, lamx.data(), lamx.size() * 8, cudaMemcpyHostToDevice, st));
    CUDA_OK(cudaMemcpyAsync(ctx->lamd.p, lamd.data(), lamd.size() * 8, cudaMemcpyHostToDevice, st));
    if (spin) CUDA_OK(cudaMemcpyAsync(ctx->lam2.p, lam2.data(), lam2.size() * 8, cudaMemcpyHostToDevice, st));
  }
  for (const Pass& ps : passes) {
    CUDA_OK(cudaMemsetAsync(ps.M->p, 0, mbytes, st));
    if (ps.M2) CUDA_OK(cudaMemsetAsync(ps.M2->p, 0, mbytes, st));
  }

  // ---- step (d) operands
  // fp16 x2: step (c) writes FP32 rows L32 / R32, split per row into fp16 hi + lo (L, R, 128-byte
  // rows) and multiplied on the step (b) engine; bf16 x3: step (c) writes the three bf16 parts.
  const int64_t kdim = 4 * pl.gc;
  const bool d16 = !pl.f64 && pl.parts_b == 2;
  const size_t lr_bytes = pl.f64 ? 8ull * kdim * NP : (d16 ? 4ull * kdim * NP : 2ull * 3 * kdim * NP);
  // fp16x2: R (and R2) carry the plane fp16(R) after the split rows
  const size_t r_bytes = lr_bytes + (d16 ? 2ull * kdim * NP : 0);
  if (!ensure(ctx->L, lr_bytes) || !ensure(ctx->R, r_bytes) || (spin && !ensure(ctx->R2, r_bytes)))
    return fail(ctx, XTC_ERR_OOM, "step (d) operands (%.2f GB)", (spin ? 3.0 : 2.0) * lr_bytes / 1e9);
  if (d16) {
    const size_t ebytes = 4ull * m_stride(NP);
    const int bn = vf_bn(2);
    const size_t tiles = static_cast<size_t>((NP + VF_BM - 1) / VF_BM) * ((NP + bn - 1) / bn);
    if (!ensure(ctx->L32, 4ull * kdim * NP) || !ensure(ctx->R32, 4ull * kdim * NP) || !ensure(ctx->eL, ebytes) ||
        !ensure(ctx->eR, ebytes) || !ensure(ctx->Vacc, std::max<size_t>(ctx->Vacc.n, 8ull * tiles * VF_BM * bn)) ||
        (spin && (!ensure(ctx->R32b, 4ull * kdim * NP) || !ensure(ctx->eR2, ebytes))))
      return fail(ctx, XTC_ERR_OOM, "step (d) FP32 operands (%.2f GB)", 8.0 * kdim * NP / 1e9);
    // exponents of the padding columns of M stay 0
    CUDA_OK(cudaMemsetAsync(ctx->eL.p, 0, ebytes, st));
    CUDA_OK(cudaMemsetAsync(ctx->eR.p, 0, ebytes, st));
    if (spin) CUDA_OK(cudaMemsetAsync(ctx->eR2.p, 0, ebytes, st));
  }
  VfMaps maps{};
  CUtensorMap tm_L{}, tm_R{}, tm_R2{}, tm_R16{}, tm_R216{};
  if ((rc = make_vfield_maps(ctx, pl, maps))) return rc;
  if (d16) {
    if ((rc = make_tmap_3d(ctx, &tm_L, ctx->L.p, false, 2 * kdim, NP, 1, 2 * VF_BK, VF_BM, true))) return rc;
    if ((rc = make_tmap_3d(ctx, &tm_R, ctx->R.p, false, 2 * kdim, NP, 1, 2 * VF_BK, vf_bn(2), true))) return rc;
    if (spin && (rc = make_tmap_3d(ctx, &tm_R2, ctx->R2.p, false, 2 * kdim, NP, 1, 2 * VF_BK, vf_bn(2), true)))
      return rc;
    // the fp16(R) planes, boxes 32 wide (64-byte swizzle)
    if ((rc = make_tmap_3d(ctx, &tm_R16, ctx->R.as<uint16_t>() + 2 * kdim * NP, false, kdim, NP, 1, VF_BK, vf_bn(2))))
      return rc;
    if (spin &&
        (rc = make_tmap_3d(ctx, &tm_R216, ctx->R2.as<uint16_t>() + 2 * kdim * NP, false, kdim, NP, 1, VF_BK, vf_bn(2))))
      return rc;
  } else if (!pl.f64) {
    if ((rc = make_tmap_3d(ctx, &tm_L, ctx->L.p, true, kdim, NP, 3, AS_BK, AS_BM))) return rc;
    if ((rc = make_tmap_3d(ctx, &tm_R, ctx->R.p, true, kdim, NP, 3, AS_BK, AS_BN))) return rc;
    if (spin && (rc = make_tmap_3d(ctx, &tm_R2, ctx->R2.p, true, kdim, NP, 3, AS_BK, AS_BN))) return rc;
  }
  int pts = 0;
  for (const Pass& ps : passes) {
    const int groups = std::max(1, (ps.rank + RANK_GROUP - 1) / RANK_GROUP);
    for (int gi = 0; gi < groups; ++gi) {
      const int rg = std::min(RANK_GROUP, ps.rank - gi * RANK_GROUP);
      const int p = choose_pts(N, std::max(rg, 0), pl.f64, spin);
      if (!p) return fail(ctx, XTC_ERR_UNSUPPORTED, "step (c) shared memory exceeded (n_orb=%d)", N);
      pts = pts ? std::min(pts, p) : p;
    }
  }

  // ---- chunk loop.  fp16 with several chunks: two gradient tables, and step (a) of chunk k + 1 on
  // a second stream once chunk k's step (b) GEMM is done, beside the memory-bound steps (c) and
  // (d) operand splits of chunk k (the GEMMs fill every SM; the gradient kernel shares an SM with
  // step (c)).  Without room for the second table the chunks run one after another.
  VfMaps maps2 = maps;
  bool pipe = !pl.f64 && pl.parts_b == 2 && pl.oe - pl.ob > pl.gc;
  if (pipe) {
    pipe = ensure(ctx->G2, ctx->G.n);
    if (pipe && !ctx->st2) {
      CUDA_OK(cudaStreamCreateWithFlags(&ctx->st2, cudaStreamNonBlocking));
      for (int b = 0; b < 2; ++b) {
        CUDA_OK(cudaEventCreateWithFlags(&ctx->ev_g[b], cudaEventDisableTiming));
        CUDA_OK(cudaEventCreateWithFlags(&ctx->ev_b[b], cudaEventDisableTiming));
      }
    }
    if (pipe) {
      const uint64_t cols = 2 * pl.NGp;
      if ((rc = make_tmap_3d(ctx, &maps2.g_store, ctx->G2.p, false, cols, 3 * pl.gc, 1, 2 * VF_BK, 32, true))) return rc;
      if ((rc = make_tmap_3d(ctx, &maps2.g_load, ctx->G2.p, false, cols, 3 * pl.gc, 1, 2 * VF_BK, VF_BM, true)))
        return rc;
    }
  }
  if (pipe) run_grad(ctx, pl, d_grid, pl.ob, std::min<int64_t>(pl.gc, pl.oe - pl.ob), maps, st);
  int gb = 0;  // gradient table of the current chunk
  for (int64_t c0 = pl.ob; c0 < pl.oe; c0 += pl.gc) {
    NvtxRange nvtx_chunk("chunk");
    const int64_t n_i = std::min<int64_t>(pl.gc, pl.oe - c0);
    {
      NvtxRange nvtx_ab("steps a+b");
      if (pipe) {
        const VfMaps& cur = gb ? maps2 : maps;
        if (c0 > pl.ob) CUDA_OK(cudaStreamWaitEvent(st, ctx->ev_g[gb], 0));
        run_gemm_b(ctx, pl, n_i, cur);
        const int64_t c1 = c0 + pl.gc;
        if (c1 < pl.oe) {
          // the other table was last read by chunk k - 1's GEMM, which ran before this one
          CUDA_OK(cudaEventRecord(ctx->ev_b[gb], st));
          CUDA_OK(cudaStreamWaitEvent(ctx->st2, ctx->ev_b[gb], 0));
          run_grad(ctx, pl, d_grid, c1, std::min<int64_t>(pl.gc, pl.oe - c1), gb ? maps : maps2, ctx->st2);
          CUDA_OK(cudaEventRecord(ctx->ev_g[1 - gb], ctx->st2));
        }
        gb = 1 - gb;
      } else if ((rc = run_vfield(ctx, pl, d_grid, c0, n_i, maps))) {
        return rc;
      }
    }
    NvtxRange nvtx_cd("steps c+d");
    for (const Pass& ps : passes) {
      const int groups = std::max(1, (ps.rank + RANK_GROUP - 1) / RANK_GROUP);
      double* M = ps.M->as<double>();
      double* M2 = ps.M2 ? ps.M2->as<double>() : nullptr;
      // L does not depend on the density and R is linear in its factors: with FP32 or FP64
      // operands step (c) runs once per group of factors, adding into R, and step (d) once per
      // chunk; the bf16 x3 operands (split in step (c)) take one step (d) per group
      const bool accum = pl.f64 || d16;
      for (int gi = 0; gi < groups; ++gi) {
        const int k0 = ps.k0 + gi * RANK_GROUP;
        const int rg = std::max(0, std::min(RANK_GROUP, ps.rank - gi * RANK_GROUP));
        FieldsArgs fa{};
        fa.V = ctx->V.p;
        fa.splits = pl.f64 ? 1 : pl.splits;
        fa.phiT = ctx->phiT.as<double>();
        fa.ldphi = pl.NGp;
        fa.w = d_w;
        fa.evec = ctx->evec.as<double>() + static_cast<size_t>(k0) * N;
        fa.lam = ctx->lam.as<double>() + k0;
        fa.lamd = ctx->lamd.as<double>() + k0;
        fa.rank = rg;
        fa.i0 = c0;
        fa.n_i = n_i;
        fa.gcp = pl.gc;
        fa.n_orb = N;
        fa.n_pair = NP;
        fa.pts = pts;
        fa.pair_p = ctx->pair_p.as<int>();
        fa.pair_q = ctx->pair_q.as<int>();
        fa.L = d16 ? ctx->L32.p : ctx->L.p;
        fa.R = d16 ? ctx->R32.p : ctx->R.p;
        fa.R2 = M2 ? (d16 ? ctx->R32b.p : ctx->R2.p) : nullptr;
        fa.lam2 = M2 ? ctx->lam2.as<double>() + k0 : nullptr;
        fa.out_parts = pl.f64 ? 0 : (d16 ? 1 : 3);
        fa.write_L = (!accum || gi == 0) ? 1 : 0;
        fa.add_R = (accum && gi > 0) ? 1 : 0;
        timed(ctx, XTC_K_FIELDS, 1, [&] { launch_fields(fa, pl.f64, st); });
        if (!accum) {
          timed(ctx, XTC_K_ASSEMBLE, M2 ? 2 : 1, [&] {
            launch_assemble_tc(&tm_L, &tm_R, NP, static_cast<int>(kdim), std::min(ctx->as_kd, 3), M,
                               ctx->err_dev.as<int>(), st);
            if (M2)
              launch_assemble_tc(&tm_L, &tm_R2, NP, static_cast<int>(kdim), std::min(ctx->as_kd, 3), M2,
                                 ctx->err_dev.as<int>(), st);
          });
        }
      }
      if (d16) {
        VfieldArgs da{};
        da.mode = 1;
        da.rows_a = NP;
        da.n_pair = NP;
        da.n_tiles = (NP + vf_bn(2) - 1) / vf_bn(2);
        da.n_kb = static_cast<int>(kdim / VF_BK);
        da.kb_per_split = da.n_kb;
        da.kd = f16_range(ctx->as_kd);
        da.xper = ctx->x_period;
        da.flush = flush_ranges(ctx->vf_flush > 0 ? ctx->vf_flush : 8192, da.kd);
        da.Vacc = ctx->Vacc.as<double>();
        da.M = M;
        da.ldm = m_stride(NP);
        da.exp_a = ctx->eL.as<int>();
        da.exp_b = ctx->eR.as<int>();
        da.err = ctx->err_dev.as<int>();
        timed(ctx, XTC_K_AUX, M2 ? 3 : 2, [&] {
          launch_lr_split(ctx->L32.as<float>(), NP, kdim, 4, da.kd, ctx->L.as<uint16_t>(), ctx->eL.as<int>(), nullptr,
                          st);
          launch_lr_split(ctx->R32.as<float>(), NP, kdim, 4, da.kd, ctx->R.as<uint16_t>(), ctx->eR.as<int>(),
                          ctx->R.as<uint16_t>() + 2 * kdim * NP, st);
          if (M2)
            launch_lr_split(ctx->R32b.as<float>(), NP, kdim, 4, da.kd, ctx->R2.as<uint16_t>(), ctx->eR2.as<int>(),
                            ctx->R2.as<uint16_t>() + 2 * kdim * NP, st);
        });
        timed(ctx, XTC_K_ASSEMBLE, 1, [&] { launch_vfield_tc(&tm_L, &tm_R, &tm_R16, da, 2, 1, st); });
        timed(ctx, XTC_K_AUX, 1, [&] { launch_vfield_tc_finalize(da, 2, 1, st); });
        if (M2) {  // the tile sums buffer is reused after the finalize above, in stream order
          VfieldArgs db = da;
          db.M = M2;
          db.exp_b = ctx->eR2.as<int>();
          timed(ctx, XTC_K_ASSEMBLE, 1, [&] { launch_vfield_tc(&tm_L, &tm_R2, &tm_R216, db, 2, 1, st); });
          timed(ctx, XTC_K_AUX, 1, [&] { launch_vfield_tc_finalize(db, 2, 1, st); });
        }
      } else if (pl.f64) {
        timed(ctx, XTC_K_ASSEMBLE, M2 ? 2 : 1, [&] {
          launch_assemble_f64(ctx->L.as<double>(), ctx->R.as<double>(), NP, static_cast<int>(kdim), M, st);
          if (M2) launch_assemble_f64(ctx->L.as<double>(), ctx->R2.as<double>(), NP, static_cast<int>(kdim), M2, st);
        });
      }
    }
  }

  // ---- final: Delta U, Delta h, e0
  NvtxRange nvtx_final("final");
  const size_t n4 = static_cast<size_t>(N) * N * N * N;
  const size_t n2b = static_cast<size_t>(N) * N * 8;
  if (!ensure(ctx->dh_tmp, 2 * n2b) || !ensure(ctx->e0_tmp, 8)) return fail(ctx, XTC_ERR_OOM, "dh staging");
  double* dh_d[2] = {nullptr, nullptr};
  for (int sp = 0; sp < out.n_spin; ++sp)
    dh_d[sp] = is_device_ptr(out.dh[sp]) ? out.dh[sp] : ctx->dh_tmp.as<double>() + static_cast<size_t>(sp) * N * N;
  double* e0_d = is_device_ptr(out.e0) ? out.e0 : ctx->e0_tmp.as<double>();
  // device destinations of the Delta U blocks; host ones are staged one at a time in dU_tmp
  const int n_blocks = spin ? 3 : 1;
  bool u_dev[3] = {false, false, false};
  bool need_stage = false;
  for (int b = 0; b < n_blocks; ++b) {
    u_dev[b] = out.dU[b] && is_device_ptr(out.dU[b]);
    need_stage |= out.dU[b] && !u_dev[b];
  }
  const bool u32_dev = out.dU32 && is_device_ptr(out.dU32);
  if (need_stage && !ensure(ctx->dU_tmp, n4 * 8)) return fail(ctx, XTC_ERR_OOM, "dU staging");
  if (out.dU32 && !u32_dev && !ensure(ctx->vout, n4 * 4)) return fail(ctx, XTC_ERR_OOM, "dU_f32 staging");
  float* u32dst = out.dU32 ? (u32_dev ? out.dU32 : ctx->vout.as<float>()) : nullptr;
  if (!spin) {
    double* udst = out.dU[0] ? (u_dev[0] ? out.dU[0] : ctx->dU_tmp.as<double>()) : nullptr;
    timed(ctx, XTC_K_FINAL, (udst || u32dst) ? 4 : 3, [&] {
      launch_symmetrize(ctx->M.as<double>(), NP, st);
      launch_unpack(ctx->M.as<double>(), N, NP, udst, u32dst, st);
      launch_onebody(ctx->M.as<double>(), ctx->gamma.as<double>(), N, NP, dh_d[0], e0_d, st);
    });
    CUDA_OK(cudaGetLastError());
    if (out.dU[0] && !u_dev[0]) CUDA_OK(cudaMemcpyAsync(out.dU[0], udst, n4 * 8, cudaMemcpyDeviceToHost, st));
    if (out.dU32 && !u32_dev) CUDA_OK(cudaMemcpyAsync(out.dU32, u32dst, n4 * 4, cudaMemcpyDeviceToHost, st));
  } else {
    // M = f^a, M2 = f^b (f^t[pq][rs] = sum_i rho_pq A^t_rs + V_pq.B^t_rs):
    // Delta U^{ab} = -(f^b + f^a^T) into M3, then Delta U^{aa} and Delta U^{bb} in place.
    timed(ctx, XTC_K_FINAL, 6, [&] {
      launch_spin_cross(ctx->M2.as<double>(), ctx->M.as<double>(), NP, ctx->M3.as<double>(), st);
      launch_symmetrize(ctx->M.as<double>(), NP, st);
      launch_symmetrize(ctx->M2.as<double>(), NP, st);
      launch_onebody_spin(ctx->M.as<double>(), ctx->M3.as<double>(), ctx->M2.as<double>(), ctx->gamma.as<double>(),
                          ctx->gamma_b.as<double>(), N, NP, dh_d[0], dh_d[1], e0_d, st);
    });
    DBuf* src[3] = {&ctx->M, &ctx->M3, &ctx->M2};
    for (int b = 0; b < 3; ++b) {
      if (!out.dU[b]) continue;
      double* udst = u_dev[b] ? out.dU[b] : ctx->dU_tmp.as<double>();
      timed(ctx, XTC_K_FINAL, 1, [&] { launch_unpack(src[b]->as<double>(), N, NP, udst, nullptr, st); });
      CUDA_OK(cudaGetLastError());
      // the staging buffer is reused by the next block: this copy completes before the next unpack
      if (!u_dev[b]) CUDA_OK(cudaMemcpyAsync(out.dU[b], udst, n4 * 8, cudaMemcpyDeviceToHost, st));
    }
  }
  CUDA_OK(cudaGetLastError());
  for (int sp = 0; sp < out.n_spin; ++sp)
    if (dh_d[sp] != out.dh[sp]) CUDA_OK(cudaMemcpyAsync(out.dh[sp], dh_d[sp], n2b, cudaMemcpyDeviceToHost, st));
  if (e0_d != out.e0) CUDA_OK(cudaMemcpyAsync(out.e0, e0_d, 8, cudaMemcpyDeviceToHost, st));
  if ((rc = check_device_error(ctx))) return rc;
  finish_timers(ctx);
  return XTC_OK;
}

}  // namespace

extern "C" int xtc_build_1b2b(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz, const double* weights,
                              const double* phi, const double* gamma, double* dU, float* dU_f32, double* dh,
                              double* e0) {
  if (!ctx) return XTC_ERR_ARG;
  if (!gamma || !dh || !e0) return fail(ctx, XTC_ERR_ARG, "gamma, dh and e0 are required");
  BuildOut out;
  out.n_spin = 1;
  out.dU[0] = dU;
  out.dU32 = dU_f32;
  out.dh[0] = dh;
  out.e0 = e0;
  const double* g[1] = {gamma};
  return build_impl(ctx, n_grid, n_orb, grid_xyz, weights, phi, g, out);
}

extern "C" int xtc_build_1b2b_rohf(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz,
                                   const double* weights, const double* phi, const double* gamma_a,
                                   const double* gamma_b, double* dU_aa, double* dU_ab, double* dU_bb, double* dh_a,
                                   double* dh_b, double* e0) {
  if (!ctx) return XTC_ERR_ARG;
  if (!gamma_a || !gamma_b || !dh_a || !dh_b || !e0)
    return fail(ctx, XTC_ERR_ARG, "gamma_a, gamma_b, dh_a, dh_b and e0 are required");
  BuildOut out;
  out.n_spin = 2;
  out.dU[0] = dU_aa;
  out.dU[1] = dU_ab;
  out.dU[2] = dU_bb;
  out.dh[0] = dh_a;
  out.dh[1] = dh_b;
  out.e0 = e0;
  const double* g[2] = {gamma_a, gamma_b};
  return build_impl(ctx, n_grid, n_orb, grid_xyz, weights, phi, g, out);
}

extern "C" int xtc_jastrow_grad(xtc_ctx* ctx, int64_t n, const double* r1, const double* r2, double* out) {
  if (!ctx) return XTC_ERR_ARG;
  if (!ctx->jastrow_set) return fail(ctx, XTC_ERR_STATE, "xtc_set_jastrow has not been called");
  if (n < 0 || (n > 0 && (!r1 || !r2 || !out))) return fail(ctx, XTC_ERR_ARG, "bad arguments");
  if (n == 0) return XTC_OK;
  CUDA_OK(cudaSetDevice(ctx->prm.device));
  cudaStream_t st = ctx->st;
  const double *d1 = nullptr, *d2 = nullptr;
  int rc;
  if ((rc = stage_input(ctx, ctx->r1, r1, static_cast<size_t>(n) * 3, &d1))) return rc;
  if ((rc = stage_input(ctx, ctx->r2, r2, static_cast<size_t>(n) * 3, &d2))) return rc;
  const bool out_dev = is_device_ptr(out);
  double* o = out;
  if (!out_dev) {
    if (!ensure(ctx->vout, static_cast<size_t>(n) * 24)) return fail(ctx, XTC_ERR_OOM, "output staging");
    o = ctx->vout.as<double>();
  }
  launch_jastrow_grad(ctx->jp_dev.as<JastrowParams>(), d1, d2, n, o, st);
  CUDA_OK(cudaGetLastError());
  if (!out_dev) CUDA_OK(cudaMemcpyAsync(out, o, static_cast<size_t>(n) * 24, cudaMemcpyDeviceToHost, st));
  CUDA_OK(cudaStreamSynchronize(st));
  return XTC_OK;
}

extern "C" int xtc_vfield(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz, const double* weights,
                          const double* phi, int64_t outer_begin, int64_t outer_end, double* V) {
  if (!ctx) return XTC_ERR_ARG;
  if (!V || outer_begin < 0 || outer_end < outer_begin || outer_end > n_grid)
    return fail(ctx, XTC_ERR_ARG, "bad outer range or null output");
  CUDA_OK(cudaSetDevice(ctx->prm.device));
  reset_timers(ctx);
  const int64_t ob = ctx->outer_begin, oe = ctx->outer_end;
  ctx->outer_begin = outer_begin;
  ctx->outer_end = outer_end;
  Plan pl{};
  const double *d_grid = nullptr, *d_w = nullptr, *d_phi = nullptr;
  int rc = prepare(ctx, pl, n_grid, n_orb, grid_xyz, weights, phi, &d_grid, &d_w, &d_phi);
  ctx->outer_begin = ob;
  ctx->outer_end = oe;
  if (rc) return rc;
  cudaStream_t st = ctx->st;
  VfMaps maps{};
  if ((rc = make_vfield_maps(ctx, pl, maps))) return rc;
  const bool out_dev = is_device_ptr(V);
  const size_t per_point = static_cast<size_t>(3) * pl.NP;
  const int64_t n_out = pl.oe - pl.ob;
  for (int64_t c0 = pl.ob; c0 < pl.oe; c0 += pl.gc) {
    const int64_t n_i = std::min<int64_t>(pl.gc, pl.oe - c0);
    if ((rc = run_vfield(ctx, pl, d_grid, c0, n_i, maps))) return rc;
    double* dst = V + (c0 - pl.ob) * per_point;
    if (!out_dev) {
      if (!ensure(ctx->vout, n_i * per_point * 8)) return fail(ctx, XTC_ERR_OOM, "V staging");
      dst = ctx->vout.as<double>();
    }
    launch_vfield_export(ctx->V.p, pl.f64, pl.f64 ? 1 : pl.splits, pl.NP, pl.N, ctx->pair_p.as<int>(),
                         ctx->pair_q.as<int>(), n_i, pl.gc, dst, st);
    CUDA_OK(cudaGetLastError());
    if (!out_dev)
      CUDA_OK(cudaMemcpyAsync(V + (c0 - pl.ob) * per_point, dst, n_i * per_point * 8, cudaMemcpyDeviceToHost, st));
  }
  (void)n_out;
  if ((rc = check_device_error(ctx))) return rc;
  finish_timers(ctx);
  return XTC_OK;
}

// ====================================================================== bounded-wait self-test
extern "C" int xtc_selftest_wait_timeout(xtc_ctx* ctx, int limit_ms) {
  if (!ctx) return XTC_ERR_ARG;
  if (limit_ms < 1 || limit_ms > 4000) return fail(ctx, XTC_ERR_ARG, "selftest: limit_ms outside 1..4000");
  CUDA_OK(cudaSetDevice(ctx->prm.device));
  CUDA_OK(cudaMemsetAsync(ctx->err_dev.p, 0, 16, ctx->st));
  launch_wait_timeout_selftest(ctx->err_dev.as<int>(), 1000000ull * static_cast<unsigned long long>(limit_ms),
                               ctx->st);
  CUDA_OK(cudaGetLastError());
  const int rc = check_device_error(ctx);  // XTC_ERR_TIMEOUT when the wait gave up, as it must
  CUDA_OK(cudaMemsetAsync(ctx->err_dev.p, 0, 16, ctx->st));
  CUDA_OK(cudaStreamSynchronize(ctx->st));
  return rc;
}

// ====================================================================== frozen-core folding
extern "C" int xtc_frozen_core_fold(xtc_ctx* ctx, int n_orb, const double* dU, const double* dh, int n_core,
                                    const int* core, double* dh_fc, double* dU_act, double* e_core) {
  if (!ctx) return XTC_ERR_ARG;
  if (n_orb < 1 || n_orb > FC_MAX_ORB || n_core < 0 || n_core > n_orb || !dU || !dh || !e_core ||
      (n_core > 0 && !core) || (n_core < n_orb && !dh_fc))
    return fail(ctx, XTC_ERR_ARG, "frozen_core_fold: null pointer or bad size");
  FcIndex ix{};
  std::vector<char> frozen(static_cast<size_t>(n_orb), 0);
  for (int k = 0; k < n_core; ++k) {
    if (core[k] < 0 || core[k] >= n_orb || frozen[core[k]])
      return fail(ctx, XTC_ERR_ARG, "frozen_core_fold: core index %d out of range or repeated", core[k]);
    frozen[core[k]] = 1;
  }
  for (int p = 0; p < n_orb; ++p) (frozen[p] ? ix.core[ix.n_core++] : ix.act[ix.n_act++]) = p;
  CUDA_OK(cudaSetDevice(ctx->prm.device));
  reset_timers(ctx);
  cudaStream_t st = ctx->st;
  const size_t n4 = static_cast<size_t>(n_orb) * n_orb * n_orb * n_orb;
  const size_t na2 = static_cast<size_t>(ix.n_act) * ix.n_act, na4 = na2 * na2;
  const double *d_U = nullptr, *d_h = nullptr;
  int rc;
  if ((rc = stage_input(ctx, ctx->fc_U, dU, n4, &d_U))) return rc;
  if ((rc = stage_input(ctx, ctx->fc_h, dh, static_cast<size_t>(n_orb) * n_orb, &d_h))) return rc;
  // small outputs go through one staging buffer unless both are device memory
  const bool small_dev = is_device_ptr(e_core) && (na2 == 0 || is_device_ptr(dh_fc));
  const bool big_dev = !dU_act || is_device_ptr(dU_act);
  double *o_h = dh_fc, *o_e = e_core, *o_U = dU_act;
  if (!small_dev) {
    if (!ensure(ctx->fc_hout, (na2 + 1) * sizeof(double))) return fail(ctx, XTC_ERR_OOM, "output staging");
    o_e = ctx->fc_hout.as<double>();
    o_h = o_e + 1;
  }
  if (!big_dev && na4 > 0) {
    if (!ensure(ctx->fc_Uout, na4 * sizeof(double))) return fail(ctx, XTC_ERR_OOM, "output staging");
    o_U = ctx->fc_Uout.as<double>();
  }
  timed(ctx, XTC_K_AUX, 1 + (na2 > 0) + (na2 > 0 && dU_act), [&] {
    launch_frozen_core(d_U, d_h, n_orb, ix, o_h, na4 > 0 ? o_U : nullptr, o_e, ctx->n_sm, st);
  });
  CUDA_OK(cudaGetLastError());
  if (!small_dev) {
    CUDA_OK(cudaMemcpyAsync(e_core, o_e, sizeof(double), cudaMemcpyDefault, st));
    if (na2) CUDA_OK(cudaMemcpyAsync(dh_fc, o_h, na2 * sizeof(double), cudaMemcpyDefault, st));
  }
  if (!big_dev && na4 > 0) CUDA_OK(cudaMemcpyAsync(dU_act, o_U, na4 * sizeof(double), cudaMemcpyDefault, st));
  CUDA_OK(cudaStreamSynchronize(st));
  return XTC_OK;
}

// ====================================================================== reciprocal self-test
extern "C" int xtc_selftest_reciprocals(xtc_ctx* ctx, int64_t n, const float* x, float* y_rsqrt, float* y_rcp) {
  if (!ctx) return XTC_ERR_ARG;
  if (n < 0 || n > (int64_t(1) << 26) || (n > 0 && (!x || !y_rsqrt || !y_rcp)))
    return fail(ctx, XTC_ERR_ARG, "selftest_reciprocals: bad arguments");
  if (n == 0) return XTC_OK;
  CUDA_OK(cudaSetDevice(ctx->prm.device));
  const size_t bytes = static_cast<size_t>(n) * sizeof(float);
  if (!ensure(ctx->r1, bytes) || !ensure(ctx->r2, 2 * bytes)) return fail(ctx, XTC_ERR_OOM, "selftest buffers");
  cudaStream_t st = ctx->st;
  CUDA_OK(cudaMemcpyAsync(ctx->r1.p, x, bytes, cudaMemcpyDefault, st));
  launch_recip_selftest(ctx->r1.as<float>(), n, ctx->r2.as<float>(), ctx->r2.as<float>() + n, st);
  CUDA_OK(cudaGetLastError());
  CUDA_OK(cudaMemcpyAsync(y_rsqrt, ctx->r2.as<float>(), bytes, cudaMemcpyDefault, st));
  CUDA_OK(cudaMemcpyAsync(y_rcp, ctx->r2.as<float>() + n, bytes, cudaMemcpyDefault, st));
  CUDA_OK(cudaStreamSynchronize(st));
  return XTC_OK;
}

// ====================================================================== chunk autotuner
// Times the build on the first outer points of this problem with up to three chunk lengths (the
// rule's choice and the rule under 3/4 and 1/2 of its memory budgets) and keeps the fastest in
// the context's parameters.  Every candidate covers the same outer points, so the fixed costs of
// a build (preparation, final kernels) are the same for all and the comparison is direct.
extern "C" int xtc_autotune_chunk(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz,
                                  const double* weights, const double* phi, const double* gamma, int64_t* chunk) {
  if (!ctx) return XTC_ERR_ARG;
  if (!chunk || !gamma || n_grid < 1 || n_orb < 1 || n_orb > MAX_ORB)
    return fail(ctx, XTC_ERR_ARG, "autotune: null pointer or bad size");
  CUDA_OK(cudaSetDevice(ctx->prm.device));
  const bool f64 = ctx->prm.precision == XTC_PREC_FP64;
  const int parts = f64 ? 0 : (ctx->prm.precision == XTC_PREC_FP16X2 ? 2 : 3);
  const int NP = n_orb * (n_orb + 1) / 2;
  const int64_t NGp = round_up(n_grid, 128);
  if (f64) {  // the FP64 path is too slow to time; its chunk only bounds memory
    *chunk = ctx->prm.grid_chunk = auto_chunk(ctx, NP, NGp, parts, n_grid, true);
    return XTC_OK;
  }
  std::vector<int64_t> cand;
  for (double scale : {1.0, 0.75, 0.5}) {
    const int64_t c = auto_chunk(ctx, NP, NGp, parts, n_grid, f64, scale);
    if (std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
  }
  const int64_t span = std::min<int64_t>(n_grid, 2 * cand[0]);
  const int64_t saved_b = ctx->outer_begin, saved_e = ctx->outer_end, saved_c = ctx->prm.grid_chunk;
  std::vector<double> dh(static_cast<size_t>(n_orb) * n_orb);
  double e0 = 0.0;
  ctx->outer_begin = 0;
  ctx->outer_end = span;
  int rc = XTC_OK;
  int64_t best = cand[0];
  double best_s = 0.0;
  for (size_t k = 0; k < cand.size() && rc == XTC_OK; ++k) {
    ctx->prm.grid_chunk = cand[k];
    if (k == 0) rc = xtc_build_1b2b(ctx, n_grid, n_orb, grid_xyz, weights, phi, gamma, nullptr, nullptr, dh.data(), &e0);
    if (rc != XTC_OK) break;
    const auto t0 = std::chrono::steady_clock::now();
    rc = xtc_build_1b2b(ctx, n_grid, n_orb, grid_xyz, weights, phi, gamma, nullptr, nullptr, dh.data(), &e0);
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rc == XTC_OK && (k == 0 || sec < best_s)) {
      best_s = sec;
      best = cand[k];
    }
  }
  ctx->outer_begin = saved_b;
  ctx->outer_end = saved_e;
  ctx->prm.grid_chunk = rc == XTC_OK ? best : saved_c;
  if (rc != XTC_OK) return rc;
  *chunk = best;
  return XTC_OK;
}

// ====================================================================== explicit three-body L
// eq. Ldecomp for small N: V of the outer points from steps (a)+(b) in the context's precision,
// then T[a][b][c] = sum_i rho_a V_b.V_c and L[p][r][t][q][s][u] = T[pq][rs][tu] + T[rs][pq][tu] +
// T[tu][pq][rs] in FP64.
extern "C" int xtc_three_body_L(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz,
                                const double* weights, const double* phi, double* L) {
  if (!ctx) return XTC_ERR_ARG;
  if (!L || n_orb < 1 || n_orb > XTC_THREE_BODY_MAX_ORB || n_grid < 1 || !grid_xyz || !weights || !phi)
    return fail(ctx, XTC_ERR_ARG, "three_body_L: null pointer, n_grid < 1 or n_orb outside 1..%d",
                XTC_THREE_BODY_MAX_ORB);
  if (!ctx->jastrow_set) return fail(ctx, XTC_ERR_STATE, "xtc_set_jastrow has not been called");
  CUDA_OK(cudaSetDevice(ctx->prm.device));
  cudaStream_t st = ctx->st;
  const int N = n_orb, NP = N * (N + 1) / 2;
  const int64_t ob = std::min<int64_t>(ctx->outer_begin, n_grid);
  const int64_t oe = std::max<int64_t>(ob, ctx->outer_end < 0 ? n_grid : std::min<int64_t>(ctx->outer_end, n_grid));
  const int64_t n_i = oe - ob;
  const size_t n6 = static_cast<size_t>(N) * N * N * N * N * N;
  const bool out_dev = is_device_ptr(L);
  if (!out_dev && !ensure(ctx->dU_tmp, n6 * 8)) return fail(ctx, XTC_ERR_OOM, "L staging (%.2f GB)", n6 * 8e-9);
  double* Ld = out_dev ? L : ctx->dU_tmp.as<double>();
  int rc;
  if (n_i == 0) {
    CUDA_OK(cudaMemsetAsync(Ld, 0, n6 * 8, st));
  } else {
    const size_t tbytes = static_cast<size_t>(NP) * NP * NP * 8;
    if (!ensure(ctx->Lv, static_cast<size_t>(n_i) * 3 * NP * 8) || !ensure(ctx->T3, tbytes))
      return fail(ctx, XTC_ERR_OOM, "three_body_L workspace (%.2f GB)", tbytes * 1e-9);
    // steps (a)+(b) for the outer points; this also builds the pair tables for n_orb
    if ((rc = xtc_vfield(ctx, n_grid, n_orb, grid_xyz, weights, phi, ob, oe, ctx->Lv.as<double>()))) return rc;
    const double *d_w = nullptr, *d_phi = nullptr;
    if ((rc = stage_input(ctx, ctx->w, weights, static_cast<size_t>(n_grid), &d_w))) return rc;
    if ((rc = stage_input(ctx, ctx->phi, phi, static_cast<size_t>(n_grid) * n_orb, &d_phi))) return rc;
    launch_three_body_t(d_phi, d_w, ob, n_i, N, ctx->pair_p.as<int>(), ctx->pair_q.as<int>(), ctx->Lv.as<double>(),
                        ctx->T3.as<double>(), st);
    launch_three_body_unpack(ctx->T3.as<double>(), N, Ld, st);
    CUDA_OK(cudaGetLastError());
  }
  if (!out_dev) CUDA_OK(cudaMemcpyAsync(L, Ld, n6 * 8, cudaMemcpyDeviceToHost, st));
  if ((rc = check_device_error(ctx))) return rc;
  return XTC_OK;
}

// ====================================================================== two-body integrals K
// K_pr^qs of the Theory section on the grid: per chunk of outer points V (steps a+b, the
// context's precision), the table w_j (lap_1 u + |grad_1 u|^2), W and the FP64 sum S of
// two_body_k.cu; then K[p][q][r][s] = S[pq][rs] + S[rs][pq].
extern "C" int xtc_two_body_K(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz,
                              const double* weights, const double* phi, const double* dphi, double* K) {
  if (!ctx) return XTC_ERR_ARG;
  if (!K || !dphi || n_orb < 1 || n_orb > XTC_TWO_BODY_K_MAX_ORB || n_grid < 1 || !grid_xyz || !weights || !phi)
    return fail(ctx, XTC_ERR_ARG, "two_body_K: null pointer, n_grid < 1 or n_orb outside 1..%d",
                XTC_TWO_BODY_K_MAX_ORB);
  if (!ctx->jastrow_set) return fail(ctx, XTC_ERR_STATE, "xtc_set_jastrow has not been called");
  CUDA_OK(cudaSetDevice(ctx->prm.device));
  cudaStream_t st = ctx->st;
  const int N = n_orb, NP = N * (N + 1) / 2;
  const int64_t ob = std::min<int64_t>(ctx->outer_begin, n_grid);
  const int64_t oe = std::max<int64_t>(ob, ctx->outer_end < 0 ? n_grid : std::min<int64_t>(ctx->outer_end, n_grid));
  const int64_t n_i = oe - ob;
  const size_t n4 = static_cast<size_t>(N) * N * N * N;
  const bool out_dev = is_device_ptr(K);
  if (!out_dev && !ensure(ctx->dU_tmp, n4 * 8)) return fail(ctx, XTC_ERR_OOM, "K staging (%.2f GB)", n4 * 8e-9);
  double* Kd = out_dev ? K : ctx->dU_tmp.as<double>();
  int rc;
  if (n_i == 0) {
    CUDA_OK(cudaMemsetAsync(Kd, 0, n4 * 8, st));
  } else {
    // chunk of outer points: the caller's grid_chunk, else what keeps F table + V + W near 6 GB
    const size_t per_point = static_cast<size_t>(n_grid) * 8 + static_cast<size_t>(4) * NP * 8;
    int64_t ch = ctx->prm.grid_chunk > 0 ? ctx->prm.grid_chunk
                                         : std::max<int64_t>(64, static_cast<int64_t>(6e9 / per_point));
    ch = std::min<int64_t>(std::min<int64_t>(ch, n_i), int64_t{65535} * 64);  // grid.y of the W GEMM
    const size_t s_bytes = static_cast<size_t>(N) * N * NP * 8;
    if (!ensure(ctx->k_S, s_bytes) || !ensure(ctx->k_V, static_cast<size_t>(ch) * 3 * NP * 8) ||
        !ensure(ctx->k_W, static_cast<size_t>(ch) * NP * 8) || !ensure(ctx->k_Ft, static_cast<size_t>(ch) * n_grid * 8) ||
        !ensure(ctx->k_P, static_cast<size_t>(4) * ctx->n_sm * 4096 * 8))
      return fail(ctx, XTC_ERR_OOM, "two_body_K workspace (%.2f GB)",
                  (s_bytes + static_cast<size_t>(ch) * per_point) * 1e-9);
    CUDA_OK(cudaMemsetAsync(ctx->k_S.p, 0, s_bytes, st));
    for (int64_t c0 = ob; c0 < oe; c0 += ch) {
      const int64_t n_c = std::min<int64_t>(ch, oe - c0);
      // steps (a)+(b) for the chunk; this also stages grid, weights and orbitals and checks them
      if ((rc = xtc_vfield(ctx, n_grid, n_orb, grid_xyz, weights, phi, c0, c0 + n_c, ctx->k_V.as<double>())))
        return rc;
      const double *d_grid = nullptr, *d_w = nullptr, *d_phi = nullptr, *d_dphi = nullptr;
      if ((rc = stage_input(ctx, ctx->grid, grid_xyz, static_cast<size_t>(n_grid) * 3, &d_grid))) return rc;
      if ((rc = stage_input(ctx, ctx->w, weights, static_cast<size_t>(n_grid), &d_w))) return rc;
      if ((rc = stage_input(ctx, ctx->phi, phi, static_cast<size_t>(n_grid) * n_orb, &d_phi))) return rc;
      if ((rc = stage_input(ctx, ctx->k_dphi, dphi, static_cast<size_t>(n_grid) * n_orb * 3, &d_dphi))) return rc;
      if (c0 == ob) {
        CUDA_OK(cudaMemsetAsync(ctx->flag_dev.p, 0, 16, st));
        launch_check_finite(d_dphi, n_grid * n_orb * 3, ctx->flag_dev.as<int>(), st);
        int flag = 0;
        CUDA_OK(cudaMemcpyAsync(&flag, ctx->flag_dev.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_OK(cudaStreamSynchronize(st));
        if (flag) return fail(ctx, XTC_ERR_NONFINITE, "NaN or Inf in the orbital gradients");
      }
      launch_k_chunk(d_grid, d_w, d_phi, d_dphi, ctx->jp_dev.as<JastrowParams>(), n_grid, N, ctx->pair_p.as<int>(),
                     ctx->pair_q.as<int>(), c0, n_c, ctx->k_V.as<double>(), ctx->k_Ft.as<double>(),
                     ctx->k_W.as<double>(), ctx->k_S.as<double>(), ctx->k_P.as<double>(),
                     static_cast<int64_t>(4) * ctx->n_sm * 4096, ctx->n_sm, st);
      CUDA_OK(cudaGetLastError());
    }
    launch_k_unpack(ctx->k_S.as<double>(), N, Kd, ctx->n_sm, st);
    CUDA_OK(cudaGetLastError());
  }
  if (!out_dev) CUDA_OK(cudaMemcpyAsync(K, Kd, n4 * 8, cudaMemcpyDeviceToHost, st));
  if ((rc = check_device_error(ctx))) return rc;
  return XTC_OK;
}

// ====================================================================== internal accessors
bool xtc_internal_ctx_view(const xtc_ctx* ctx, xtc::CtxView* v) {
  if (!ctx || !v) return false;
  v->device = ctx->prm.device;
  v->stream = ctx->st;
  v->precision = ctx->prm.precision;
  v->n_sm = ctx->n_sm;
  v->jastrow_set = ctx->jastrow_set;
  v->n_nuc = ctx->jp.n_nuc;
  v->g_bound = ctx->g_bound;
  v->vf_kd = ctx->vf_kd;
  v->jp_dev = ctx->jp_dev.as<JastrowParams>();
  v->encode_tiled = reinterpret_cast<void*>(ctx->encode);
  return true;
}

int xtc_internal_fail(xtc_ctx* ctx, int code, const char* msg) { return fail(ctx, code, "%s", msg); }

// ====================================================================== batched build
// Instances are ordered by their step (b) cost (N_g^2 N_pair, largest first) and each goes to the
// lane with the least work so far; every lane is a context with its own stream and workspace, run
// by its own host thread, so that the kernels of small instances (which fill little of the GPU)
// overlap.  Every instance is computed exactly as by xtc_set_jastrow + xtc_build_1b2b on a
// context of the same parameters.
extern "C" int xtc_build_1b2b_batched(xtc_ctx* ctx, int n_inst, xtc_instance* inst, int n_lanes) {
  if (!ctx) return XTC_ERR_ARG;
  if (n_inst < 0 || (n_inst > 0 && !inst) || n_lanes < 0)
    return fail(ctx, XTC_ERR_ARG, "bad instance count, instance array or lane count");
  if (n_inst == 0) return XTC_OK;
  CUDA_OK(cudaSetDevice(ctx->prm.device));
  // inputs the caller wrote on its stream are complete before the lanes start
  if (ctx->st) CUDA_OK(cudaStreamSynchronize(ctx->st));
  else CUDA_OK(cudaDeviceSynchronize());
  const int lanes = std::min(n_inst, n_lanes > 0 ? std::min(n_lanes, 16) : 4);
  while (static_cast<int>(ctx->lanes.size()) < lanes) {
    cudaStream_t sl = nullptr;
    CUDA_OK(cudaStreamCreateWithFlags(&sl, cudaStreamNonBlocking));
    xtc_params lp = ctx->prm;
    lp.stream = sl;
    lp.timing = 0;
    xtc_ctx* lc = nullptr;
    const int rc = xtc_create(&lc, &lp);
    if (rc != XTC_OK) {
      cudaStreamDestroy(sl);
      return fail(ctx, rc, "creating a batch lane failed");
    }
    ctx->lanes.push_back(lc);
    ctx->lane_streams.push_back(sl);
  }
  std::vector<int> order(n_inst);
  for (int i = 0; i < n_inst; ++i) order[i] = i;
  auto cost = [&](int i) {
    const double np = 0.5 * inst[i].n_orb * (inst[i].n_orb + 1.0);
    return static_cast<double>(inst[i].n_grid) * static_cast<double>(inst[i].n_grid) * np;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  std::vector<std::vector<int>> work(lanes);
  std::vector<double> load(lanes, 0.0);
  for (int i : order) {
    const int l = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
    work[l].push_back(i);
    load[l] += cost(i);
  }
  const int device = ctx->prm.device;
  auto run_lane = [&](int l) {
    cudaSetDevice(device);
    xtc_ctx* lc = ctx->lanes[l];
    for (int i : work[l]) {
      xtc_instance& in = inst[i];
      int rc = xtc_set_jastrow(lc, in.n_nuc, in.nuc_xyz, in.nuc_set, in.n_sets, in.n_terms, in.mno, in.coef);
      if (rc == XTC_OK) rc = xtc_set_outer_range(lc, 0, -1);
      if (rc == XTC_OK)
        rc = xtc_build_1b2b(lc, in.n_grid, in.n_orb, in.grid_xyz, in.weights, in.phi, in.gamma, in.dU, in.dU_f32, in.dh,
                            in.e0);
      in.status = rc;
    }
  };
  std::vector<std::thread> threads;
  for (int l = 1; l < lanes; ++l) threads.emplace_back(run_lane, l);
  run_lane(0);
  for (std::thread& t : threads) t.join();
  for (int i = 0; i < n_inst; ++i)
    if (inst[i].status != XTC_OK) {
      const xtc_ctx* lc = nullptr;
      for (int l = 0; l < lanes; ++l)
        if (std::find(work[l].begin(), work[l].end(), i) != work[l].end()) lc = ctx->lanes[l];
      return fail(ctx, inst[i].status, "instance %d: %s", i, lc ? lc->detail : "");
    }
  return XTC_OK;
}
