// Steps (a)+(b) on the tensor cores: the vector pair fields of the "Decomposition of two-body
// correction" section,
//     V_x[i][pq] = sum_j G_x(i, j) rho^T[pq][j],   G_x(i, j) = d/dx_i u(r_i, r_j),
//     rho^T[pq][j] = w_j phi_p(j) phi_q(j),
// as one GEMM per outer-point tile with the Jastrow gradient generated on the fly.
//
// CTA tile: 128 outer points (TMEM lanes) x 160 orbital pairs x 3 components, three FP32
// accumulators of 160 TMEM columns each.  Per pipeline stage (32 inner points):
//   * warp 0 (one lane) TMA-loads the rho^T tile of each split part (160 rows x 64 B, 64-byte
//     swizzle) onto an mbarrier with a transaction count;
//   * warps 2..9 (256 threads, one outer point and 16 inner points each) evaluate nabla_1 u in
//     FP32, split every value into fp16 (2 parts) or bf16 (3 parts) and store the A tiles in the
//     same swizzled K-major layout, then arrive on a second mbarrier;
//   * warp 1 (one lane) issues tcgen05.mma for every component and every split product into the
//     TMEM accumulators and commits the stage back to the producers.
// After the last stage warps 2..5 read the accumulators with tcgen05.ld, undo the power-of-2
// scalings and store V[pq][x][i] (FP32, outer index contiguous).
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "jastrow_coef.cuh"
#include "ptx_sm100.cuh"
#include "xtc_internal.cuh"

namespace xtc {
namespace {

constexpr int PROD_WARPS = 8;
constexpr int VF_THREADS = 64 + PROD_WARPS * 32;
constexpr int A_TILE = VF_BM * 64;  // bytes per (component, part) tile
constexpr int B_TILE = VF_BN * 64;  // bytes per part tile

template <int PARTS>
struct VfCfg {
  static constexpr int STAGES = PARTS == 2 ? 3 : 2;
  static constexpr int NPROD = PARTS == 2 ? 3 : 6;
  static constexpr int A_BYTES = 3 * PARTS * A_TILE;
  static constexpr int STAGE_BYTES = A_BYTES + PARTS * B_TILE;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};

// (A part, B part) of each split product, in issue order.
__device__ __forceinline__ void prod_parts(int p, int& pa, int& pb) {
  constexpr int a[6] = {0, 0, 1, 0, 1, 2};
  constexpr int b[6] = {0, 1, 0, 2, 1, 0};
  pa = a[p];
  pb = b[p];
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
__device__ __forceinline__ void split_pair(float a, float b, uint32_t* out /*[PARTS]*/, int parts) {
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
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

template <int PARTS, int NNUC>
__global__ void __launch_bounds__(VF_THREADS, 1)
    vfield_tc_kernel(const __grid_constant__ CUtensorMap tm_rho, const VfieldArgs args) {
  using Cfg = VfCfg<PARTS>;
  constexpr bool BF16 = PARTS == 3;
  constexpr int STAGES = Cfg::STAGES;
  constexpr int JS = 12;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * Cfg::STAGE_BYTES);
  uint64_t* tma_full = bars;
  uint64_t* g_full = bars + STAGES;
  uint64_t* empty = bars + 2 * STAGES;
  uint64_t* acc_bar = bars + 3 * STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * STAGES + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_tile = blockIdx.x, n_tile = blockIdx.y, split = blockIdx.z;
  const int kb0 = split * args.kb_per_split;
  const int kb1 = min(args.n_kb, kb0 + args.kb_per_split);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&tma_full[s], 1);
      mbar_init(&g_full[s], PROD_WARPS);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_bar, 1);
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
      // ---------------------------------------------------------------- TMA producer
      int issued_end = kb0;
      for (int kb = kb0; kb < kb1; ++kb) {
        const int it = kb - kb0, s = it % STAGES, n = it / STAGES;
        if (n > 0 && !mbar_wait(&empty[s], (n - 1) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF)) break;
        mbar_arrive_expect_tx(&tma_full[s], PARTS * B_TILE);
        uint8_t* bdst = smem + s * Cfg::STAGE_BYTES + Cfg::A_BYTES;
        for (int p = 0; p < PARTS; ++p)
          tma_load_3d(bdst + p * B_TILE, &tm_rho, &tma_full[s], kb * VF_BK, n_tile * VF_BN, p);
        issued_end = kb + 1;
      }
      // make sure no bulk copy into this CTA's shared memory is still in flight
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
      constexpr uint32_t idesc = idesc_f16(VF_BM, VF_BN, BF16);
      for (int kb = kb0; kb < kb1; ++kb) {
        const int it = kb - kb0, s = it % STAGES, n = it / STAGES;
        if (!mbar_wait(&tma_full[s], n & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF)) break;
        if (!mbar_wait(&g_full[s], n & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF)) break;
        tc_fence_after();
        const uint32_t sa = smem_base + s * Cfg::STAGE_BYTES;
        const uint32_t sb = sa + Cfg::A_BYTES;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
#pragma unroll
          for (int p = 0; p < Cfg::NPROD; ++p) {
            int pa, pb;
            prod_parts(p, pa, pb);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint64_t ad = sdesc_kmajor_sw64(sa + (x * PARTS + pa) * A_TILE + ks * 32);
              const uint64_t bd = sdesc_kmajor_sw64(sb + pb * B_TILE + ks * 32);
              tc_mma_f16(tmem + x * VF_BN, ad, bd, idesc, (it > 0 || p > 0 || ks > 0) ? 1u : 0u);
            }
          }
        }
        tc_commit(&empty[s]);
      }
      tc_commit(acc_bar);  // also on an abort, so the accumulator wait below ends
    }
  } else {
    // ------------------------------------------------------------------ gradient producers
    const int pt = threadIdx.x - 64;
    const int row = pt & (VF_BM - 1);
    const int jh = pt >> 7;
    const int64_t il = static_cast<int64_t>(m_tile) * VF_BM + row;
    const int64_t ig = args.i0 + (il < args.n_i ? il : args.n_i - 1);
    float pc[PT_COEF];
    float nc[NNUC * NUC_COEF];
    const double gx = args.grid[3 * ig], gy = args.grid[3 * ig + 1], gz = args.grid[3 * ig + 2];
    point_coefs_fixed<float, NNUC>(*args.jp, gx, gy, gz, static_cast<double>(args.g_scale), pc, nc);
    // low parts of the outer point's coordinates (x = hi + lo)
    const float xl = static_cast<float>(gx - static_cast<double>(pc[0]));
    const float yl = static_cast<float>(gy - static_cast<double>(pc[1]));
    const float zl = static_cast<float>(gz - static_cast<double>(pc[2]));
    const int wgroup = warp - 2;

    for (int kb = kb0; kb < kb1; ++kb) {
      const int it = kb - kb0, s = it % STAGES, n = it / STAGES;
      const bool got = n == 0 || mbar_wait(&empty[s], (n - 1) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF);
      if (!__all_sync(0xffffffffu, got)) break;  // warp-uniform decision
      const uint32_t sa = smem_base + s * Cfg::STAGE_BYTES;
#pragma unroll
      for (int grp = 0; grp < 2; ++grp) {
        const int64_t jbase = static_cast<int64_t>(kb) * VF_BK + jh * 16 + grp * 8;
        float gv[3][8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float* jp = args.jtab + (jbase + u) * JS;
          const float4 p0 = __ldg(reinterpret_cast<const float4*>(jp));
          const float4 p1 = __ldg(reinterpret_cast<const float4*>(jp + 4));
          float aj[NNUC];
          aj[0] = p0.w;
          if (NNUC > 1) aj[NNUC > 1 ? 1 : 0] = p1.w;
          if (NNUC > 2) {
            const float4 p2 = __ldg(reinterpret_cast<const float4*>(jp + 8));
            aj[NNUC > 2 ? 2 : 0] = p2.x;
            if (NNUC > 3) aj[NNUC > 3 ? 3 : 0] = p2.y;
          }
          // (hi_i - hi_j) is exact for nearby points; the low parts restore the rest
          const float dx = (pc[0] - p0.x) + (xl - p1.x);
          const float dy = (pc[1] - p0.y) + (yl - p1.y);
          const float dz = (pc[2] - p0.z) + (zl - p1.z);
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          const float rinv = rsqrt_approx(fmaxf(r2, 1e-30f));
          const float r = r2 * rinv;
          const float q = rcp_approx(1.0f + r);
          const float b = r * q;
          const float sfac = r2 > 0.0f ? q * q * rinv : 0.0f;
          float ex = fmaf(b, fmaf(b, pc[9], pc[6]), pc[3]);
          float ey = fmaf(b, fmaf(b, pc[10], pc[7]), pc[4]);
          float ez = fmaf(b, fmaf(b, pc[11], pc[8]), pc[5]);
          float h1 = pc[12], h2 = pc[13];
#pragma unroll
          for (int I = 0; I < NNUC; ++I) {
            const float* c = nc + I * NUC_COEF;
            const float a = aj[I];
            const float t = fmaf(b, fmaf(b, fmaf(a, c[8], c[7]), fmaf(a, c[6], c[5])), fmaf(a, c[4], c[3]));
            const float at = a * t;
            ex = fmaf(at, c[0], ex);
            ey = fmaf(at, c[1], ey);
            ez = fmaf(at, c[2], ez);
            h1 = fmaf(a, fmaf(a, c[10], c[9]), h1);
            h2 = fmaf(a, fmaf(a, c[12], c[11]), h2);
          }
          const float hs = fmaf(b, h2, h1) * sfac;
          gv[0][u] = fmaf(hs, dx, ex);
          gv[1][u] = fmaf(hs, dy, ey);
          gv[2][u] = fmaf(hs, dz, ez);
        }
        const uint32_t off = sw64_offset(row, jh * 2 + grp);
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          uint32_t w[4][PARTS];
#pragma unroll
          for (int h = 0; h < 4; ++h) split_pair<BF16>(gv[x][2 * h], gv[x][2 * h + 1], w[h], PARTS);
#pragma unroll
          for (int p = 0; p < PARTS; ++p)
            st_shared_v4(sa + (x * PARTS + p) * A_TILE + off, w[0][p], w[1][p], w[2][p], w[3][p]);
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&g_full[s]);
    }

    // ------------------------------------------------------------------ epilogue (warps 2..5)
    if (wgroup < 4) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait(acc_bar, 0, abort_flag, args.err, DEV_ERR_TIMEOUT_VF));
      __syncwarp();
      tc_fence_after();
      const int quarter = warp & 3;
      const int erow = quarter * 32 + lane;
      const int64_t eil = static_cast<int64_t>(m_tile) * VF_BM + erow;
      const bool valid = ok && !*abort_flag && eil < args.n_i;
      float* Vz = args.V + static_cast<int64_t>(split) * args.n_pair * 3 * args.gcp;
#pragma unroll 1
      for (int x = 0; x < 3; ++x) {
#pragma unroll 1
        for (int c0 = 0; c0 < VF_BN; c0 += 32) {
          uint32_t r[32];
          tmem_ld_32x32b_x32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + x * VF_BN + c0, r);
          tmem_wait_ld();
          if (valid) {
#pragma unroll
            for (int k = 0; k < 32; ++k) {
              const int pq = n_tile * VF_BN + c0 + k;
              if (pq < args.n_pair) {
                const float v = __uint_as_float(r[k]) * args.unscale_g;
                Vz[(static_cast<int64_t>(pq) * 3 + x) * args.gcp + eil] = ldexpf(v, -__ldg(args.colexp + pq));
              }
            }
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
  const int m_tiles = static_cast<int>((a.n_i + VF_BM - 1) / VF_BM);
  const int n_tiles = (a.n_pair + VF_BN - 1) / VF_BN;
  dim3 grid(m_tiles, n_tiles, splits);
  kern<<<grid, VF_THREADS, smem, st>>>(*tm, a);
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
