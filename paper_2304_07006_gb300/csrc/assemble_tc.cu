// Step (d) on the tensor cores: the two-body assembly of Appendix B,
//     Delta U(pq|rs) = -sum_i [rho_pq A_rs + V_pq . B_rs + rho_rs A_pq + V_rs . B_pq]
// computed as M += L^T R with L[pq][k] = (rho, Vx, Vy, Vz) and R[rs][k] = (A, Bx, By, Bz) for
// k = (outer point, component); Delta U = -(M + M^T) is formed by the unpacking kernel.
//
// CTA tile 128 x 256 (one FP32 accumulator of 256 TMEM columns), 32-element K stages with both
// operands TMA-loaded in the 64-byte swizzle, three bf16 parts per operand and six split products
// (i + j <= 2).  Warp 0 issues the TMA loads, warp 1 the MMAs, warps 2..5 add the tile into the
// FP64 accumulator M in HBM (read-modify-write; every tile is owned by exactly one CTA).
#include "ptx_sm100.cuh"
#include "xtc_internal.cuh"

namespace xtc {
namespace {

constexpr int PARTS = 3;
constexpr int NPROD = 6;
constexpr int STAGES = 3;
constexpr int A_TILE = AS_BM * 64;
constexpr int B_TILE = AS_BN * 64;
constexpr int STAGE_BYTES = PARTS * (A_TILE + B_TILE);
constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int THREADS = 192;

__global__ void __launch_bounds__(THREADS, 1)
    assemble_tc_kernel(const __grid_constant__ CUtensorMap tm_L, const __grid_constant__ CUtensorMap tm_R,
                       int n_pair, int ldm, int n_kb, double* __restrict__ M, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* acc_bar = bars + 2 * STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_tile = blockIdx.x, n_tile = blockIdx.y;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_desc(&tm_L);
    tma_prefetch_desc(&tm_R);
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, 256);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t smem_base = smem_u32(smem);

  if (warp == 0) {
    if (lane == 0) {
      int issued_end = 0;
      for (int kb = 0; kb < n_kb; ++kb) {
        const int s = kb % STAGES, n = kb / STAGES;
        if (n > 0 && !mbar_wait(&empty[s], (n - 1) & 1, abort_flag, err, DEV_ERR_TIMEOUT_AS)) break;
        mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
        uint8_t* st = smem + s * STAGE_BYTES;
        for (int p = 0; p < PARTS; ++p) {
          tma_load_3d(st + p * A_TILE, &tm_L, &full[s], kb * AS_BK, m_tile * AS_BM, p);
          tma_load_3d(st + PARTS * A_TILE + p * B_TILE, &tm_R, &full[s], kb * AS_BK, n_tile * AS_BN, p);
        }
        issued_end = kb + 1;
      }
      int zero = 0;
      for (int kb = max(0, issued_end - STAGES); kb < issued_end; ++kb)
        mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, reinterpret_cast<volatile int*>(&zero), err,
                  DEV_ERR_TIMEOUT_AS);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(AS_BM, AS_BN, true);
      constexpr int pa_of[6] = {0, 0, 1, 0, 1, 2};
      constexpr int pb_of[6] = {0, 1, 0, 2, 1, 0};
      for (int kb = 0; kb < n_kb; ++kb) {
        const int s = kb % STAGES, n = kb / STAGES;
        if (!mbar_wait(&full[s], n & 1, abort_flag, err, DEV_ERR_TIMEOUT_AS)) break;
        tc_fence_after();
        const uint32_t sa = smem_base + s * STAGE_BYTES;
        const uint32_t sb = sa + PARTS * A_TILE;
#pragma unroll
        for (int p = 0; p < NPROD; ++p) {
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t ad = sdesc_kmajor_sw64(sa + pa_of[p] * A_TILE + ks * 32);
            const uint64_t bd = sdesc_kmajor_sw64(sb + pb_of[p] * B_TILE + ks * 32);
            tc_mma_f16(tmem, ad, bd, idesc, (kb > 0 || p > 0 || ks > 0) ? 1u : 0u);
          }
        }
        tc_commit(&empty[s]);
      }
      tc_commit(acc_bar);
    }
  } else {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(acc_bar, 0, abort_flag, err, DEV_ERR_TIMEOUT_AS));
    __syncwarp();
    tc_fence_after();
    const int quarter = warp & 3;
    const int row = m_tile * AS_BM + quarter * 32 + lane;
    const bool valid = ok && !*abort_flag && row < n_pair && n_kb > 0;
    double* Mrow = M + static_cast<int64_t>(row) * ldm;
#pragma unroll 1
    for (int c0 = 0; c0 < AS_BN; c0 += 32) {
      uint32_t r[32];
      tmem_ld_32x32b_x32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + c0, r);
      tmem_wait_ld();
      const int col0 = n_tile * AS_BN + c0;
      if (valid && col0 < n_pair) {
        double2* dst = reinterpret_cast<double2*>(Mrow + col0);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          double2 v = dst[k];
          v.x += static_cast<double>(__uint_as_float(r[2 * k]));
          v.y += static_cast<double>(__uint_as_float(r[2 * k + 1]));
          dst[k] = v;
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

}  // namespace

void launch_assemble_tc(const CUtensorMap* tm_L, const CUtensorMap* tm_R, int n_pair, int kdim, double* M,
                        int* err, cudaStream_t st) {
  // M has row stride ldm = round_up(n_pair, AS_BN) so every 32-column group of a tile is in bounds
  const int ldm = static_cast<int>(round_up(n_pair, AS_BN));
  cudaFuncSetAttribute(assemble_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  dim3 grid((n_pair + AS_BM - 1) / AS_BM, (n_pair + AS_BN - 1) / AS_BN);
  assemble_tc_kernel<<<grid, THREADS, SMEM, st>>>(*tm_L, *tm_R, n_pair, ldm, kdim / AS_BK, M, err);
}

}  // namespace xtc
