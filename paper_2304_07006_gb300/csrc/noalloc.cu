// Allocation-free variant of steps (a)+(b) (xtc_vfield) for callers that cannot allocate device
// memory: code running where the memory is owned by someone else (a host framework with its own
// pool, a real-time loop that must not call cudaMalloc) can still evaluate the vector pair fields
// V of small problems.  All workspace lives in one file-scope device array of fixed size; the
// caller passes device buffers for the inputs and the output.
//
// The array's device address is obtained with cudaGetSymbolAddress on the first call on each
// device (with that device current).  Every call reuses the same array and it keeps the last
// call's contents, so calls that overlap on the GPU (other streams, other threads, other contexts
// of this process on the same device) race with each other and must be serialised by the caller.
// The tensor-core GEMM
// runs with FP32 running sums only (no FP64 flush: the array has no room for the FP64 tile sums),
// so over long inner sums its rounding differs slightly from xtc_vfield's.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/xtc.h"
#include "xtc_internal.cuh"

using namespace xtc;

namespace {

constexpr size_t kScratchBytes = static_cast<size_t>(XTC_NOALLOC_SCRATCH_MIB) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, looked up once (under the mutex) and then read lock-free.
std::atomic<void*> g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

void* scratch_address(int device) {
  void* p = g_scratch_addr[device].load(std::memory_order_acquire);
  if (p) return p;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  p = g_scratch_addr[device].load(std::memory_order_relaxed);
  if (p) return p;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return nullptr;
  }
  g_scratch_addr[device].store(p, std::memory_order_release);
  return p;
}

// Restores the calling thread's current device when the call returns.
struct DeviceGuard {
  int saved = -1;
  DeviceGuard() {
    if (cudaGetDevice(&saved) != cudaSuccess) {
      cudaGetLastError();
      saved = -1;
    }
  }
  ~DeviceGuard() {
    if (saved >= 0) cudaSetDevice(saved);
  }
};

__global__ void pair_table_kernel(int n_orb, int* pp, int* pq) {
  const int p = blockIdx.x;
  const int base = p * n_orb - p * (p - 1) / 2;
  for (int q = p + threadIdx.x; q < n_orb; q += blockDim.x) {
    pp[base + q - p] = p;
    pq[base + q - p] = q;
  }
}

// True for managed memory and for device memory of `device` (memory of another GPU is refused:
// the kernels on `device` would read it through a peer mapping, or fault without one).
bool on_device(const void* p, int device) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == device);
}

// Carves 256-byte aligned pieces out of the scratch array.
struct Carver {
  unsigned char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base + off);
    off += (count * sizeof(T) + 255) / 256 * 256;
    return p;
  }
};

}  // namespace

extern "C" XTC_API int xtc_vfield_noalloc(xtc_ctx* ctx, int64_t n_grid, int n_orb, const double* grid_xyz,
                                          const double* weights, const double* phi, int64_t outer_begin,
                                          int64_t outer_end, double* V) {
  CtxView cv{};
  if (!xtc_internal_ctx_view(ctx, &cv)) return XTC_ERR_ARG;
  if (!cv.jastrow_set) return xtc_internal_fail(ctx, XTC_ERR_STATE, "xtc_set_jastrow has not been called");
  if (n_grid < 1 || n_orb < 1 || n_orb > 320 || outer_begin < 0 || outer_end < outer_begin || outer_end > n_grid)
    return xtc_internal_fail(ctx, XTC_ERR_ARG, "noalloc: bad sizes or outer range");
  const bool f64 = cv.precision == XTC_PREC_FP64;
  if (!f64 && !vfield_tc_supported(cv.n_nuc))
    return xtc_internal_fail(ctx, XTC_ERR_UNSUPPORTED, "noalloc: the tensor-core path supports 1..8 nuclei");
  if (cv.device < 0 || cv.device >= kMaxDevices)
    return xtc_internal_fail(ctx, XTC_ERR_ARG, "noalloc: device ordinal out of range");
  DeviceGuard restore_device;
  if (cudaSetDevice(cv.device) != cudaSuccess) {
    cudaGetLastError();
    return xtc_internal_fail(ctx, XTC_ERR_CUDA, "noalloc: cudaSetDevice failed");
  }
  if (!on_device(grid_xyz, cv.device) || !on_device(weights, cv.device) || !on_device(phi, cv.device) ||
      !on_device(V, cv.device))
    return xtc_internal_fail(ctx, XTC_ERR_ARG, "noalloc: inputs and output must be device pointers on the context's device");

  // ---- the scratch array's device address, once per device
  void* scratch = scratch_address(cv.device);
  if (!scratch)
    return xtc_internal_fail(ctx, XTC_ERR_CUDA, "noalloc: cudaGetSymbolAddress of the scratch array failed");

  // ---- plan and carve (sizes checked before any device work)
  const int N = n_orb, NP = N * (N + 1) / 2, n_nuc = cv.n_nuc;
  const int64_t NGp = round_up(n_grid, 128);
  const int64_t n_outer = outer_end - outer_begin;
  const int parts = f64 ? 0 : (cv.precision == XTC_PREC_FP16X2 ? 2 : 3);
  const int kd_b = cv.vf_kd >= 2 ? 2 : 1;  // exact range of the fp16 step (b) engine
  // bytes the layout below carves for a chunk of gc outer points (same order and rounding)
  auto need = [&](int64_t gc) {
    Carver c{nullptr};
    c.take<int>(4);
    c.take<int>(NP);
    c.take<int>(NP);
    if (f64) {
      c.take<double>(static_cast<size_t>(NGp) * (3 + n_nuc));
      c.take<double>(static_cast<size_t>(NGp) * NP);
      c.take<double>(static_cast<size_t>(v_slice(gc, N)));
    } else {
      c.take<double>(static_cast<size_t>(N) * NGp);
      c.take<float>(static_cast<size_t>(NGp) * jtab_stride(n_nuc));
      c.take<uint16_t>(static_cast<size_t>(3) * NP * NGp);
      c.take<unsigned int>(NP);
      c.take<int>(NP);
      c.take<float>(static_cast<size_t>(2) * (N + 1) * NGp);
      c.take<float>(static_cast<size_t>(v_slice(gc, N)));
      c.take<uint16_t>(static_cast<size_t>(parts) * 3 * gc * NGp);
    }
    return c.off;
  };
  int64_t gc = round_up(std::max<int64_t>(n_outer, 1), 128);
  while (gc > 128 && need(gc) > kScratchBytes) gc -= 128;
  if (need(gc) > kScratchBytes) {
    char msg[200];
    snprintf(msg, sizeof msg, "noalloc: problem needs %.1f MiB of workspace, the fixed scratch holds %d MiB",
             need(128) / 1048576.0, XTC_NOALLOC_SCRATCH_MIB);
    return xtc_internal_fail(ctx, XTC_ERR_ARG, msg);
  }
  Carver cz{static_cast<unsigned char*>(scratch)};
  int* err = cz.take<int>(4);
  int* pair_p = cz.take<int>(NP);
  int* pair_q = cz.take<int>(NP);
  cudaStream_t st = cv.stream;
  if (n_outer == 0) return XTC_OK;

  // ---- what must start at zero: the device error word (the column maxima are cleared by their launcher)
  if (cudaMemsetAsync(err, 0, 16, st) != cudaSuccess)
    return xtc_internal_fail(ctx, XTC_ERR_CUDA, "noalloc: clearing the error word failed");
  pair_table_kernel<<<N, 128, 0, st>>>(N, pair_p, pair_q);

  CUtensorMap tm{}, tm16{}, tm_gs{}, tm_gl{};
  double* jtab64 = nullptr;
  double* rho64 = nullptr;
  float* jtab = nullptr;
  void* rho = nullptr;
  int* colexp = nullptr;
  void* Vbuf = nullptr;
  if (f64) {
    jtab64 = cz.take<double>(static_cast<size_t>(NGp) * (3 + n_nuc));
    rho64 = cz.take<double>(static_cast<size_t>(NGp) * NP);
    Vbuf = cz.take<double>(static_cast<size_t>(v_slice(gc, N)));
    launch_jtab64(grid_xyz, n_grid, NGp, cv.jp_dev, n_nuc, jtab64, st);
    launch_rho_f64(phi, weights, n_grid, NGp, N, pair_p, pair_q, rho64, st);
  } else {
    double* phiT = cz.take<double>(static_cast<size_t>(N) * NGp);
    jtab = cz.take<float>(static_cast<size_t>(NGp) * jtab_stride(n_nuc));
    rho = cz.take<uint16_t>(static_cast<size_t>(3) * NP * NGp);  // fp16: split rows + fp16 plane
    unsigned int* colmax = cz.take<unsigned int>(NP);
    colexp = cz.take<int>(NP);
    float* phi32 = cz.take<float>(static_cast<size_t>(2) * (N + 1) * NGp);
    Vbuf = cz.take<float>(static_cast<size_t>(v_slice(gc, N)));
    void* G = cz.take<uint16_t>(static_cast<size_t>(parts) * 3 * gc * NGp);
    launch_transpose_phi(phi, n_grid, NGp, N, phiT, st);
    launch_jtab(grid_xyz, n_grid, NGp, cv.jp_dev, n_nuc, jtab_stride(n_nuc), jtab, st);
    launch_rho_split(phiT, weights, n_grid, NGp, N, parts, kd_b, pair_p, pair_q, colmax, colexp, phi32, rho, st);
    // rho^T (box rows vf_bn) and the gradient table [part][x * gc + il][j] (boxes 32 x 32
    // for the step (a) stores and 32 x 128 for the step (b) loads)
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(cv.encode_tiled);
    // (fp16: both parts of a 32-point block in one 128-byte row; bf16: one plane per part)
    const bool wide = parts == 2;
    const int64_t cols = wide ? 2 * NGp : NGp, planes = wide ? 1 : parts;
    auto map = [&](CUtensorMap* m, void* base, int64_t rows, uint32_t box_rows) {
      const cuuint64_t dims[3] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows),
                                  static_cast<cuuint64_t>(planes)};
      const cuuint64_t strides[2] = {static_cast<cuuint64_t>(cols) * 2, static_cast<cuuint64_t>(cols) * rows * 2};
      const cuuint32_t box[3] = {static_cast<cuuint32_t>(wide ? 2 * VF_BK : VF_BK), box_rows, 1};
      const cuuint32_t es[3] = {1, 1, 1};
      return encode(m, parts == 3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, base, dims,
                    strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    wide ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (!map(&tm, rho, NP, vf_bn(parts)) || !map(&tm_gs, G, 3 * gc, 32) || !map(&tm_gl, G, 3 * gc, VF_BM))
      return xtc_internal_fail(ctx, XTC_ERR_CUDA, "noalloc: cuTensorMapEncodeTiled failed");
    if (wide) {
      // the fp16(rho^T) plane after the split rows: [pq][j], boxes 32 x vf_bn (64-byte swizzle)
      const cuuint64_t dims[3] = {static_cast<cuuint64_t>(NGp), static_cast<cuuint64_t>(NP), 1};
      const cuuint64_t strides[2] = {static_cast<cuuint64_t>(NGp) * 2, static_cast<cuuint64_t>(NGp) * NP * 2};
      const cuuint32_t box[3] = {static_cast<cuuint32_t>(VF_BK), static_cast<cuuint32_t>(vf_bn(2)), 1};
      const cuuint32_t es[3] = {1, 1, 1};
      if (encode(&tm16, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, static_cast<uint16_t*>(rho) + 2 * static_cast<size_t>(NP) * NGp,
                 dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return xtc_internal_fail(ctx, XTC_ERR_CUDA, "noalloc: cuTensorMapEncodeTiled failed");
    }
  }

  // ---- chunks of outer points: steps (a)+(b), then V -> caller's buffer [k][x][pq] (FP64)
  const int n_kb = static_cast<int>(NGp / VF_BK);
  for (int64_t c0 = outer_begin; c0 < outer_end; c0 += gc) {
    const int64_t n_i = std::min<int64_t>(gc, outer_end - c0);
    if (f64) {
      launch_vfield_f64_impl(grid_xyz, cv.jp_dev, n_nuc, jtab64, rho64, NGp, NP, c0, n_i, gc, pair_p, pair_q, N,
                             static_cast<double*>(Vbuf), st);
    } else {
      int sg = 0;
      if (parts == 2 && cv.g_bound > 0.0)
        sg = std::max(-30, std::min(30, static_cast<int>(std::floor(std::log2(16384.0 / cv.g_bound)))));
      const int mt_per_x = static_cast<int>((n_i + VF_BM - 1) / VF_BM);
      GfieldArgs g{};
      g.grid = grid_xyz;
      g.jp = cv.jp_dev;
      g.jtab = jtab;
      g.i0 = c0;
      g.n_i = n_i;
      g.gcp = gc;
      g.n_tiles = mt_per_x * (VF_BM / 32);
      g.n_kb = n_kb;
      g.kb_per_seg = 32;
      g.n_seg = (n_kb + g.kb_per_seg - 1) / g.kb_per_seg;
      g.n_nuc = n_nuc;
      g.g_scale = std::ldexp(1.0f, sg);
      g.range_blocks = kd_b;
      launch_gfield(&tm_gs, g, parts, st);
      VfieldArgs a{};
      a.colexp = colexp;
      a.V = static_cast<float*>(Vbuf);
      a.pair_p = pair_p;
      a.pair_q = pair_q;
      a.n_orb = N;
      a.Vacc = nullptr;
      a.flush = 0;  // FP32 running sums only: the fixed scratch has no room for FP64 tiles
      a.n_i = n_i;
      a.gcp = gc;
      a.mt_per_x = mt_per_x;
      a.n_tiles = (NP + vf_bn(parts) - 1) / vf_bn(parts);
      a.n_pair = NP;
      a.n_kb = n_kb;
      a.kb_per_split = n_kb;
      a.kd = parts == 2 ? kd_b : std::min(cv.vf_kd, 2);
      a.xper = 64;
      a.unscale_g = std::ldexp(1.0f, -sg);
      a.err = err;
      launch_vfield_tc(&tm_gl, &tm, &tm16, a, parts, 1, st);
    }
    launch_vfield_export(Vbuf, f64, 1, NP, N, pair_p, pair_q, n_i, gc, V + (c0 - outer_begin) * 3 * NP, st);
  }
  if (cudaGetLastError() != cudaSuccess) return xtc_internal_fail(ctx, XTC_ERR_CUDA, "noalloc: kernel launch failed");
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return xtc_internal_fail(ctx, XTC_ERR_CUDA, "noalloc: stream synchronisation failed");
  if (h) return xtc_internal_fail(ctx, XTC_ERR_TIMEOUT, "noalloc: a device-side wait timed out");
  return XTC_OK;
}
