// Steps (a)+(b) on the tensor cores: the vector pair fields of the "Decomposition of two-body
// correction" section,
//     V_x[i][pq] = sum_j G_x(i, j) rho^T[pq][j],   G_x(i, j) = d/dx_i u(r_i, r_j),
//     rho^T[pq][j] = w_j phi_p(j) phi_q(j),
// as a GEMM whose A operand (the Jastrow gradient) is generated on the fly.
//
// CTA tile: 32 outer points x 3 components = 96 A rows (row x*32 + point; rows 96..127 stay zero)
// x 160 orbital pairs, 32 inner points per pipeline stage (64-byte rows, 64-byte swizzle, K-major).
//   * warp 0 (one lane): per stage, TMA loads of the rho^T tile of each split part (160 x 64 B)
//     and a bulk copy of the 32-point inner table (coordinates hi/lo and a_jI) into shared memory;
//   * warps 2..9: two groups of four warps take alternate stages; in a stage, warp c of a group
//     evaluates nabla_1 u in FP32 for its 8 inner points (one 16-byte chunk of every row) and all
//     32 outer points (one per lane, coefficients in registers), splits it into fp16 (2 parts)
//     or bf16 (3 parts) and stores the swizzled A tiles;
//   * warp 1 (one lane): tcgen05.mma for every split product into one of two TMEM accumulators;
//   * warps 10..13: every `kd` stages they add the finished accumulator into an FP32 running sum
//     kept in TMEM (tcgen05.ld / st) while the MMA fills the other accumulator, and at the end
//     store the sum, unscaled, as V[pq][x][i].
// The tensor-core accumulator truncates toward zero at each MMA, which biases a long inner sum.
// Each range is short (default two stages), its MMAs issue the small cross products of all its
// stages first so that only the hi x hi products meet a large accumulator, and the ranges are
// summed with round-to-nearest FP32 adds.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "jastrow_coef.cuh"
#include "ptx_sm100.cuh"
#include "xtc_internal.cuh"

namespace xtc {
namespace {

constexpr int TP = 32;               // outer points per tile
constexpr int PROD_WARPS = 8;        // two groups of four, alternate stages
constexpr int GROUP_WARPS = 4;       // one per 16-byte chunk (8 inner points) of a stage
constexpr int DRAIN_WARPS = 4;
constexpr int THREADS = (2 + PROD_WARPS + DRAIN_WARPS) * 32;
constexpr int A_TILE = 128 * 64;     // bytes per part tile (128 rows of 64 B)
constexpr int B_TILE = VF_BN * 64;   // bytes per part tile (160 rows of 64 B)
constexpr int JT_BYTES = VF_BK * 12 * 4;
constexpr int D_COLS = VF_BN;        // accumulator columns
constexpr uint32_t S_COL = 2 * D_COLS;  // running-sum columns start

template <int PARTS>
struct VfCfg {
  static constexpr int STAGES = PARTS == 2 ? 5 : 3;
  static constexpr int NPROD = PARTS == 2 ? 3 : 6;
  static constexpr int A_BYTES = PARTS * A_TILE;
  static constexpr int B_BYTES = PARTS * B_TILE;
  static constexpr int STAGE_BYTES = ((A_BYTES + B_BYTES + JT_BYTES + 1023) / 1024) * 1024;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};

// (A part, B part) of each split product in issue order: the small cross products first and
// hi x hi last, so that the truncations of the early MMAs act on a small accumulator.
template <int PARTS>
__device__ __forceinline__ void prod_parts(int p, int& pa, int& pb) {
  if (PARTS == 2) {
    constexpr int a[3] = {0, 1, 0};
    constexpr int b[3] = {1, 0, 0};
    pa = a[p];
    pb = b[p];
  } else {
    constexpr int a[6] = {1, 0, 2, 0, 1, 0};
    constexpr int b[6] = {1, 2, 0, 1, 0, 0};
    pa = a[p];
    pb = b[p];
  }
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <bool BF16>
__device__ __forceinline__ void split_pair(float a, float b, uint32_t* out) {
  if (!BF16) {
    __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    out[0] = *reinterpret_cast<uint32_t*>(&h);
    out[1] = *reinterpret_cast<uint32_t*>(&l);
  } else {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const float ra = a - hf.x, rb = b - hf.y;
    __nv_bfloat162 m = __floats2bfloat162_rn(ra, rb);
    const float2 mf = __bfloat1622float2(m);
    __nv_bfloat162 l = __floats2bfloat162_rn(ra - mf.x, rb - mf.y);
    out[0] = *reinterpret_cast<uint32_t*>(&h);
    out[1] = *reinterpret_cast<uint32_t*>(&m);
    out[2] = *reinterpret_cast<uint32_t*>(&l);
  }
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ float4 ld_shared_f4(uint32_t addr) {
  float4 r;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "r"(addr));
  return r;
}
// Two FP32 values packed in a 64-bit register, processed by Blackwell's paired FP32 instructions.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float a, float b) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void up2(f32x2 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ void ld_shared_2x64(uint32_t addr, f32x2& a, f32x2& b) {
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr));
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_st_32x32b_x32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

template <int PARTS, int NNUC>
__global__ void __launch_bounds__(THREADS, 1)
    vfield_tc_kernel(const __grid_constant__ CUtensorMap tm_rho, const VfieldArgs args) {
  using Cfg = VfCfg<PARTS>;
  constexpr bool BF16 = PARTS == 3;
  constexpr int STAGES = Cfg::STAGES;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * Cfg::STAGE_BYTES);
  uint64_t* tma_full = bars;                 // [STAGES]
  uint64_t* g_full = bars + STAGES;          // [STAGES]
  uint64_t* empty = bars + 2 * STAGES;       // [STAGES]
  uint64_t* d_full = bars + 3 * STAGES;      // [2]
  uint64_t* d_free = bars + 3 * STAGES + 2;  // [2]
  uint64_t* fin_bar = bars + 3 * STAGES + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_tile = blockIdx.x, n_tile = blockIdx.y, split = blockIdx.z;
  const int kb0 = split * args.kb_per_split;
  const int kb1 = min(args.n_kb, kb0 + args.kb_per_split);
  const int n_it = kb1 - kb0;
  const int kd = args.kd;
  const int n_ranges = (n_it + kd - 1) / kd;

  // rows 96..127 of every A tile are never written by the producers: zero them once
  for (int s = 0; s < STAGES; ++s)
    for (int p = 0; p < PARTS; ++p) {
      uint4* z = reinterpret_cast<uint4*>(smem + s * Cfg::STAGE_BYTES + p * A_TILE + 96 * 64);
      for (int k = threadIdx.x; k < 32 * 64 / 16; k += THREADS) z[k] = make_uint4(0, 0, 0, 0);
    }
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&tma_full[s], 1);
      mbar_init(&g_full[s], GROUP_WARPS);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&d_full[b], 1);
      mbar_init(&d_free[b], DRAIN_WARPS);
    }
    mbar_init(fin_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_desc(&tm_rho);
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t smem_base = smem_u32(smem);

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------------- TMA / bulk-copy producer
      int issued_end = kb0;
      for (int kb = kb0; kb < kb1; ++kb) {
        const int it = kb - kb0, s = it % STAGES, n = it / STAGES;
        if (n > 0 && !mbar_wait(&empty[s], (n - 1) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF)) break;
        mbar_arrive_expect_tx(&tma_full[s], PARTS * B_TILE + JT_BYTES);
        uint8_t* st = smem + s * Cfg::STAGE_BYTES;
        for (int p = 0; p < PARTS; ++p)
          tma_load_3d(st + Cfg::A_BYTES + p * B_TILE, &tm_rho, &tma_full[s], kb * VF_BK, n_tile * VF_BN, p);
        bulk_g2s(st + Cfg::A_BYTES + Cfg::B_BYTES, args.jtab + static_cast<int64_t>(kb) * VF_BK * 12, JT_BYTES,
                 &tma_full[s]);
        issued_end = kb + 1;
      }
      int zero = 0;
      for (int kb = max(kb0, issued_end - STAGES); kb < issued_end; ++kb) {
        const int it = kb - kb0;
        mbar_wait(&tma_full[it % STAGES], (it / STAGES) & 1, reinterpret_cast<volatile int*>(&zero), args.err,
                  DEV_ERR_TIMEOUT_VF);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------------------------------------------------------- MMA issuer
      // A range of kd stages goes into one TMEM accumulator: first every cross product of all its
      // stages (the accumulator is still small), then every hi x hi product.
      constexpr uint32_t idesc = idesc_f16(128, VF_BN, BF16);
      bool alive = true;
      for (int r = 0; r < n_ranges && alive; ++r) {
        const int it0 = r * kd, it1 = min(n_it, it0 + kd);
        const int b = r & 1, u = r >> 1;
        if (u >= 1 && !mbar_wait(&d_free[b], (u - 1) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF)) break;
        for (int it = it0; it < it1 && alive; ++it) {
          const int s = it % STAGES, n = it / STAGES;
          alive = mbar_wait(&tma_full[s], n & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF) &&
                  mbar_wait(&g_full[s], n & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF);
        }
        if (!alive) break;
        tc_fence_after();
        for (int pass = 0; pass < 2; ++pass) {
          for (int it = it0; it < it1; ++it) {
            const uint32_t sa = smem_base + (it % STAGES) * Cfg::STAGE_BYTES;
            const uint32_t sb = sa + Cfg::A_BYTES;
#pragma unroll
            for (int p = 0; p < Cfg::NPROD; ++p) {
              if ((p == Cfg::NPROD - 1) != (pass == 1)) continue;
              int pa, pb;
              prod_parts<PARTS>(p, pa, pb);
#pragma unroll
              for (int ks = 0; ks < 2; ++ks) {
                const uint64_t ad = sdesc_kmajor_sw64(sa + pa * A_TILE + ks * 32);
                const uint64_t bd = sdesc_kmajor_sw64(sb + pb * B_TILE + ks * 32);
                tc_mma_f16(tmem + b * D_COLS, ad, bd, idesc, (it == it0 && p == 0 && ks == 0) ? 0u : 1u);
              }
            }
          }
        }
        for (int it = it0; it < it1; ++it) tc_commit(&empty[it % STAGES]);
        tc_commit(&d_full[b]);
      }
      // every MMA issued by this thread has completed once fin_bar fires
      tc_commit(fin_bar);
      int zero = 0;
      mbar_wait(fin_bar, 0, reinterpret_cast<volatile int*>(&zero), args.err, DEV_ERR_TIMEOUT_VF);
    }
  } else if (warp < 2 + PROD_WARPS) {
    // ------------------------------------------------------------------ gradient producers
    const int group = (warp - 2) >> 2;  // stages it = group, group + 2, ...
    const int c = (warp - 2) & 3;       // inner points 8c .. 8c+7 of the stage
    const int pt = lane;                // outer point of the tile
    const int64_t il = static_cast<int64_t>(m_tile) * TP + pt;
    const int64_t ig = args.i0 + (il < args.n_i ? il : args.n_i - 1);
    float pc[PT_COEF];
    float nc[NNUC * NUC_COEF];
    const double gx = args.grid[3 * ig], gy = args.grid[3 * ig + 1], gz = args.grid[3 * ig + 2];
    point_coefs_fixed<float, NNUC>(*args.jp, gx, gy, gz, static_cast<double>(args.g_scale), pc, nc);
    const float xl = static_cast<float>(gx - static_cast<double>(pc[0]));
    const float yl = static_cast<float>(gy - static_cast<double>(pc[1]));
    const float zl = static_cast<float>(gz - static_cast<double>(pc[2]));
    uint32_t row_off[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) row_off[x] = sw64_offset(x * TP + pt, c);
    // the same constants duplicated in both halves of a packed pair (paired FP32 path, <= 2 nuclei)
    f32x2 PC[NNUC <= 2 ? PT_COEF : 1], NC[NNUC <= 2 ? NNUC * NUC_COEF : 1], XL = 0, YL = 0, ZL = 0;
    if constexpr (NNUC <= 2) {
#pragma unroll
      for (int k = 0; k < PT_COEF; ++k) PC[k] = pk2(pc[k], pc[k]);
#pragma unroll
      for (int k = 0; k < NNUC * NUC_COEF; ++k) NC[k] = pk2(nc[k], nc[k]);
      XL = pk2(xl, xl);
      YL = pk2(yl, yl);
      ZL = pk2(zl, zl);
    }

    for (int it = group; it < n_it; it += 2) {
      const int s = it % STAGES, n = it / STAGES;
      bool got = n == 0 || mbar_wait(&empty[s], (n - 1) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF);
      got = got && mbar_wait(&tma_full[s], n & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF);
      if (!__all_sync(0xffffffffu, got)) break;
      const uint32_t sa = smem_base + s * Cfg::STAGE_BYTES;
      const uint32_t jt = sa + Cfg::A_BYTES + Cfg::B_BYTES + c * 4 * 96;
      float gv[3][8];
#pragma unroll
      for (int v2 = 0; v2 < 4; ++v2) {
        // inner points j = 8c + 2 v2 (even) and + 1 (odd), one 96-byte record
        const uint32_t rec = jt + v2 * 96;
        if constexpr (NNUC <= 2) {
          f32x2 xh, yh, zh, xlo, ylo, zlo, a0, a1;
          ld_shared_2x64(rec, xh, yh);
          ld_shared_2x64(rec + 16, zh, xlo);
          ld_shared_2x64(rec + 32, ylo, zlo);
          ld_shared_2x64(rec + 48, a0, a1);
          const f32x2 dx = add2(sub2(PC[0], xh), sub2(XL, xlo));
          const f32x2 dy = add2(sub2(PC[1], yh), sub2(YL, ylo));
          const f32x2 dz = add2(sub2(PC[2], zh), sub2(ZL, zlo));
          const f32x2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
          float r2a, r2b;
          up2(r2, r2a, r2b);
          // unit vector of r1 - r2 taken as zero below 1e-14 bohr (coincident points)
          const float ria = r2a > 1e-28f ? rsqrt_approx(r2a) : 0.0f;
          const float rib = r2b > 1e-28f ? rsqrt_approx(r2b) : 0.0f;
          const f32x2 rinv = pk2(ria, rib);
          const f32x2 rr = mul2(r2, rinv);
          float ra, rb;
          up2(rr, ra, rb);
          const f32x2 q = pk2(rcp_approx(1.0f + ra), rcp_approx(1.0f + rb));
          const f32x2 b = mul2(rr, q);
          const f32x2 sfac = mul2(mul2(q, q), rinv);
          f32x2 ex = fma2(b, fma2(b, PC[9], PC[6]), PC[3]);
          f32x2 ey = fma2(b, fma2(b, PC[10], PC[7]), PC[4]);
          f32x2 ez = fma2(b, fma2(b, PC[11], PC[8]), PC[5]);
          f32x2 h1 = PC[12], h2 = PC[13];
#pragma unroll
          for (int I = 0; I < NNUC; ++I) {
            const f32x2* cf = NC + I * NUC_COEF;
            const f32x2 a = I == 0 ? a0 : a1;
            const f32x2 t = fma2(b, fma2(b, fma2(a, cf[8], cf[7]), fma2(a, cf[6], cf[5])), fma2(a, cf[4], cf[3]));
            const f32x2 at = mul2(a, t);
            ex = fma2(at, cf[0], ex);
            ey = fma2(at, cf[1], ey);
            ez = fma2(at, cf[2], ez);
            h1 = fma2(a, fma2(a, cf[10], cf[9]), h1);
            h2 = fma2(a, fma2(a, cf[12], cf[11]), h2);
          }
          const f32x2 hs = mul2(fma2(b, h2, h1), sfac);
          up2(fma2(hs, dx, ex), gv[0][2 * v2], gv[0][2 * v2 + 1]);
          up2(fma2(hs, dy, ey), gv[1][2 * v2], gv[1][2 * v2 + 1]);
          up2(fma2(hs, dz, ez), gv[2][2 * v2], gv[2][2 * v2 + 1]);
        } else {
          const float4 q0 = ld_shared_f4(rec), q1 = ld_shared_f4(rec + 16), q2 = ld_shared_f4(rec + 32);
          const float4 q3 = ld_shared_f4(rec + 48), q4 = ld_shared_f4(rec + 64);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float xh = h ? q0.y : q0.x, yh = h ? q0.w : q0.z, zh = h ? q1.y : q1.x;
            const float xlo = h ? q1.w : q1.z, ylo = h ? q2.y : q2.x, zlo = h ? q2.w : q2.z;
            float aj[NNUC];
            aj[0] = h ? q3.y : q3.x;
            aj[NNUC > 1 ? 1 : 0] = h ? q3.w : q3.z;
            if (NNUC > 2) aj[NNUC > 2 ? 2 : 0] = h ? q4.y : q4.x;
            if (NNUC > 3) aj[NNUC > 3 ? 3 : 0] = h ? q4.w : q4.z;
            const float dx = (pc[0] - xh) + (xl - xlo);
            const float dy = (pc[1] - yh) + (yl - ylo);
            const float dz = (pc[2] - zh) + (zl - zlo);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float rinv = r2 > 1e-28f ? rsqrt_approx(r2) : 0.0f;
            const float rr = r2 * rinv;
            const float q = rcp_approx(1.0f + rr);
            const float b = rr * q;
            const float sfac = q * q * rinv;
            float ex = fmaf(b, fmaf(b, pc[9], pc[6]), pc[3]);
            float ey = fmaf(b, fmaf(b, pc[10], pc[7]), pc[4]);
            float ez = fmaf(b, fmaf(b, pc[11], pc[8]), pc[5]);
            float h1 = pc[12], h2 = pc[13];
#pragma unroll
            for (int I = 0; I < NNUC; ++I) {
              const float* cf = nc + I * NUC_COEF;
              const float a = aj[I];
              const float t = fmaf(b, fmaf(b, fmaf(a, cf[8], cf[7]), fmaf(a, cf[6], cf[5])), fmaf(a, cf[4], cf[3]));
              const float at = a * t;
              ex = fmaf(at, cf[0], ex);
              ey = fmaf(at, cf[1], ey);
              ez = fmaf(at, cf[2], ez);
              h1 = fmaf(a, fmaf(a, cf[10], cf[9]), h1);
              h2 = fmaf(a, fmaf(a, cf[12], cf[11]), h2);
            }
            const float hs = fmaf(b, h2, h1) * sfac;
            gv[0][2 * v2 + h] = fmaf(hs, dx, ex);
            gv[1][2 * v2 + h] = fmaf(hs, dy, ey);
            gv[2][2 * v2 + h] = fmaf(hs, dz, ez);
          }
        }
      }
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        uint32_t w[4][PARTS];
#pragma unroll
        for (int h = 0; h < 4; ++h) split_pair<BF16>(gv[x][2 * h], gv[x][2 * h + 1], w[h]);
#pragma unroll
        for (int p = 0; p < PARTS; ++p) st_shared_v4(sa + p * A_TILE + row_off[x], w[0][p], w[1][p], w[2][p], w[3][p]);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&g_full[s]);
    }
  } else {
    // ------------------------------------------------------------------ range drains and epilogue
    const int quarter = warp & 3;
    const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
    bool ok = true;
    for (int r = 0; r < n_ranges && ok; ++r) {
      const int b = r & 1, u = r >> 1;
      ok = __all_sync(0xffffffffu, mbar_wait(&d_full[b], u & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF));
      __syncwarp();
      if (!ok) break;
      tc_fence_after();
#pragma unroll 1
      for (int c0 = 0; c0 < D_COLS; c0 += 32) {
        uint32_t d[32], sacc[32];
        tmem_ld_32x32b_x32(tmem + lane_base + b * D_COLS + c0, d);
        if (r > 0) tmem_ld_32x32b_x32(tmem + lane_base + S_COL + c0, sacc);
        tmem_wait_ld();
        if (r > 0) {
#pragma unroll
          for (int k = 0; k < 32; ++k) d[k] = __float_as_uint(__uint_as_float(sacc[k]) + __uint_as_float(d[k]));
        }
        tmem_st_32x32b_x32(tmem + lane_base + S_COL + c0, d);
      }
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&d_free[b]);
    }
    // store the running sum: row x*32 + pt of this tile -> V[split][pq][x][tile*32 + pt]
    const int row = quarter * 32 + lane;
    const int64_t il = static_cast<int64_t>(m_tile) * TP + (row & (TP - 1));
    const bool valid = ok && !*abort_flag && row < 3 * TP && il < args.n_i && n_it > 0;
    float* Vz = args.V + static_cast<int64_t>(split) * args.n_pair * 3 * args.gcp;
    const int64_t col_off = static_cast<int64_t>(row >> 5) * args.gcp + il;
    tc_fence_after();
#pragma unroll 1
    for (int c0 = 0; c0 < D_COLS; c0 += 32) {
      uint32_t sacc[32];
      tmem_ld_32x32b_x32(tmem + lane_base + S_COL + c0, sacc);
      tmem_wait_ld();
      if (valid) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const int pq = n_tile * VF_BN + c0 + k;
          if (pq < args.n_pair) {
            const float v = __uint_as_float(sacc[k]) * args.unscale_g;
            Vz[static_cast<int64_t>(pq) * 3 * args.gcp + col_off] = ldexpf(v, -__ldg(args.colexp + pq));
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

template <int PARTS, int NNUC>
void launch_t(const CUtensorMap* tm, const VfieldArgs& a, int splits, cudaStream_t st) {
  auto kern = vfield_tc_kernel<PARTS, NNUC>;
  constexpr int smem = VfCfg<PARTS>::SMEM;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int m_tiles = static_cast<int>((a.n_i + TP - 1) / TP);
  const int n_tiles = (a.n_pair + VF_BN - 1) / VF_BN;
  dim3 grid(m_tiles, n_tiles, splits);
  kern<<<grid, THREADS, smem, st>>>(*tm, a);
}

}  // namespace

bool vfield_tc_supported(int n_nuc) { return n_nuc >= 1 && n_nuc <= 4; }

void launch_vfield_tc(const CUtensorMap* tm_rho, const VfieldArgs& a, int parts, bool bf16, int splits,
                      cudaStream_t st) {
  (void)bf16;
  if (parts == 2) {
    switch (a.n_nuc) {
      case 1: launch_t<2, 1>(tm_rho, a, splits, st); break;
      case 2: launch_t<2, 2>(tm_rho, a, splits, st); break;
      case 3: launch_t<2, 3>(tm_rho, a, splits, st); break;
      default: launch_t<2, 4>(tm_rho, a, splits, st); break;
    }
  } else {
    switch (a.n_nuc) {
      case 1: launch_t<3, 1>(tm_rho, a, splits, st); break;
      case 2: launch_t<3, 2>(tm_rho, a, splits, st); break;
      case 3: launch_t<3, 3>(tm_rho, a, splits, st); break;
      default: launch_t<3, 4>(tm_rho, a, splits, st); break;
    }
  }
}

}  // namespace xtc
