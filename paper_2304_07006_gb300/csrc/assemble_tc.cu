// Step (d) on the tensor cores: the two-body assembly of Appendix B,
//     Delta U(pq|rs) = -sum_i [rho_pq A_rs + V_pq . B_rs + rho_rs A_pq + V_rs . B_pq]
// computed as M += L^T R with L[pq][k] = (rho, Vx, Vy, Vz) and R[rs][k] = (A, Bx, By, Bz) for
// k = (outer point, component); Delta U = -(M + M^T) is formed by the final kernels.
//
// CTA tile 128 x 128, 32-element K stages with both operands TMA-loaded in the 64-byte swizzle,
// three bf16 parts per operand and six split products (i + j <= 2, smallest first).  Warp 0 issues
// the TMA loads, warp 1 the MMAs into one of two TMEM accumulators; every `kd` stages warps 2..5
// add the finished accumulator into a compensated FP32 running sum (sum and error term, Knuth's
// TwoSum, both in TMEM) while the MMA fills the other one, which keeps the tensor-core
// accumulation (truncating at each MMA) to short ranges.  A tcgen05.commit stalls the tensor pipe
// for a few hundred cycles, so each range ends with one commit, whose arrival both frees the
// range's stage slots (the TMA producer counts finished ranges in order) and starts the drain.
// At the end warps 2..5 add sum + error into the FP64 accumulator M in HBM (read-modify-write;
// every tile of M is owned by exactly one CTA).
#include "ptx_sm100.cuh"
#include "xtc_internal.cuh"

namespace xtc {
namespace {

constexpr int PARTS = 3;
constexpr int NPROD = 6;
constexpr int STAGES = 4;
constexpr int A_TILE = AS_BM * 64;
constexpr int B_TILE = AS_BN * 64;
constexpr int STAGE_BYTES = PARTS * (A_TILE + B_TILE);
constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int THREADS = 192;
constexpr int DRAIN_WARPS = 4;
constexpr uint32_t S_COL = 2 * AS_BN;  // running sum
constexpr uint32_t C_COL = 3 * AS_BN;  // its rounding-error term
constexpr int NRB = 8;                 // range barriers (range r uses r % NRB)
// a wait for range r must not alias range r + NRB (the producer waits for the range of stage
// k - STAGES before loading stage k)
static_assert(NRB > STAGES, "range barriers");

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

__global__ void __launch_bounds__(THREADS, 1)
    assemble_tc_kernel(const __grid_constant__ CUtensorMap tm_L, const __grid_constant__ CUtensorMap tm_R,
                       int n_pair, int ldm, int n_kb, int kd, double* __restrict__ M, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* full = bars;                     // [STAGES] the stage's loads landed
  uint64_t* rdone = bars + STAGES;           // [NRB] the MMAs of range r (r % NRB) completed
  uint64_t* d_free = bars + STAGES + NRB;    // [2] the drains released accumulator b
  uint64_t* fin_bar = bars + STAGES + NRB + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + STAGES + NRB + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_tile = blockIdx.x, n_tile = blockIdx.y;
  const int n_ranges = (n_kb + kd - 1) / kd;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
    for (int r = 0; r < NRB; ++r) mbar_init(&rdone[r], 1);
    for (int b = 0; b < 2; ++b) mbar_init(&d_free[b], DRAIN_WARPS);
    mbar_init(fin_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_desc(&tm_L);
    tma_prefetch_desc(&tm_R);
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
      int seen = 0;  // ranges known to have completed (their slots are free again)
      int issued_end = 0;
      for (int kb = 0; kb < n_kb; ++kb) {
        const int s = kb % STAGES;
        if (kb >= STAGES) {
          const int need = (kb - STAGES) / kd;  // range holding the slot's previous stage
          bool ok = true;
          for (; seen <= need && ok; ++seen)
            ok = mbar_wait(&rdone[seen % NRB], (seen / NRB) & 1, abort_flag, err, DEV_ERR_TIMEOUT_AS);
          if (!ok) break;
        }
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
      // small cross products first, hi x hi last, over all stages of a range (the early
      // truncations then act on a small accumulator)
      constexpr int pa_of[6] = {1, 0, 2, 0, 1, 0};
      constexpr int pb_of[6] = {1, 2, 0, 1, 0, 0};
      bool alive = true;
      for (int r = 0; r < n_ranges && alive; ++r) {
        const int kb0 = r * kd, kb1 = min(n_kb, kb0 + kd);
        const int b = r & 1, u = r >> 1;
        if (u >= 1 && !mbar_wait(&d_free[b], (u - 1) & 1, abort_flag, err, DEV_ERR_TIMEOUT_AS)) break;
        // cross products of each stage as it lands, then the hi x hi products of the range
        for (int pass = 0; pass < 2 && alive; ++pass) {
          for (int kb = kb0; kb < kb1; ++kb) {
            if (pass == 0) {
              if (!(alive = mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, abort_flag, err, DEV_ERR_TIMEOUT_AS)))
                break;
              tc_fence_after();
            }
            const uint32_t sa = smem_base + (kb % STAGES) * STAGE_BYTES;
            const uint32_t sb = sa + PARTS * A_TILE;
#pragma unroll
            for (int p = 0; p < NPROD; ++p) {
              if ((p == NPROD - 1) != (pass == 1)) continue;
#pragma unroll
              for (int ks = 0; ks < 2; ++ks) {
                const uint64_t ad = sdesc_kmajor_sw64(sa + pa_of[p] * A_TILE + ks * 32);
                const uint64_t bd = sdesc_kmajor_sw64(sb + pb_of[p] * B_TILE + ks * 32);
                tc_mma_f16(tmem + b * AS_BN, ad, bd, idesc, (kb == kb0 && p == 0 && ks == 0) ? 0u : 1u);
              }
            }
          }
        }
        if (!alive) break;
        tc_commit(&rdone[r % NRB]);
      }
      tc_commit(fin_bar);
      int zero = 0;
      mbar_wait(fin_bar, 0, reinterpret_cast<volatile int*>(&zero), err, DEV_ERR_TIMEOUT_AS);
    }
  } else {
    const int quarter = warp & 3;
    const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
    bool ok = true;
    for (int r = 0; r < n_ranges && ok; ++r) {
      const int b = r & 1;
      ok = __all_sync(0xffffffffu, mbar_wait(&rdone[r % NRB], (r / NRB) & 1, abort_flag, err, DEV_ERR_TIMEOUT_AS));
      __syncwarp();
      if (!ok) break;
      tc_fence_after();
#pragma unroll 1
      for (int c0 = 0; c0 < AS_BN; c0 += 32) {
        uint32_t d[32], sacc[32], cacc[32];
        tmem_ld_32x32b_x32(tmem + lane_base + b * AS_BN + c0, d);
        if (r > 0) {
          tmem_ld_32x32b_x32(tmem + lane_base + S_COL + c0, sacc);
          tmem_ld_32x32b_x32(tmem + lane_base + C_COL + c0, cacc);
        }
        tmem_wait_ld();
        if (r > 0) {
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            // TwoSum: s1 + e == x + y exactly
            const float x = __uint_as_float(sacc[k]), y = __uint_as_float(d[k]);
            const float s1 = __fadd_rn(x, y);
            const float yp = __fsub_rn(s1, x);
            const float xp = __fsub_rn(s1, yp);
            const float e = __fadd_rn(__fsub_rn(x, xp), __fsub_rn(y, yp));
            sacc[k] = __float_as_uint(s1);
            cacc[k] = __float_as_uint(__fadd_rn(__uint_as_float(cacc[k]), e));
          }
        } else {
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            sacc[k] = d[k];
            cacc[k] = 0u;
          }
        }
        tmem_st_32x32b_x32(tmem + lane_base + S_COL + c0, sacc);
        tmem_st_32x32b_x32(tmem + lane_base + C_COL + c0, cacc);
      }
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&d_free[b]);
    }
    const int row = m_tile * AS_BM + quarter * 32 + lane;
    const bool valid = ok && !*abort_flag && row < n_pair && n_kb > 0;
    double* Mrow = M + static_cast<int64_t>(row) * ldm;
    tc_fence_after();
#pragma unroll 1
    for (int c0 = 0; c0 < AS_BN; c0 += 32) {
      uint32_t sacc[32], cacc[32];
      tmem_ld_32x32b_x32(tmem + lane_base + S_COL + c0, sacc);
      tmem_ld_32x32b_x32(tmem + lane_base + C_COL + c0, cacc);
      tmem_wait_ld();
      const int col0 = n_tile * AS_BN + c0;
      if (valid && col0 < n_pair) {
        double2* dst = reinterpret_cast<double2*>(Mrow + col0);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          double2 v = dst[k];
          v.x += static_cast<double>(__uint_as_float(sacc[2 * k])) + static_cast<double>(__uint_as_float(cacc[2 * k]));
          v.y += static_cast<double>(__uint_as_float(sacc[2 * k + 1])) +
                 static_cast<double>(__uint_as_float(cacc[2 * k + 1]));
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
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace

void launch_assemble_tc(const CUtensorMap* tm_L, const CUtensorMap* tm_R, int n_pair, int kdim, int kd, double* M,
                        int* err, cudaStream_t st) {
  // M has row stride m_stride(n_pair) so every 32-column group of a tile is in bounds
  const int ldm = static_cast<int>(m_stride(n_pair));
  cudaFuncSetAttribute(assemble_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  dim3 grid((n_pair + AS_BM - 1) / AS_BM, (n_pair + AS_BN - 1) / AS_BN);
  assemble_tc_kernel<<<grid, THREADS, SMEM, st>>>(*tm_L, *tm_R, n_pair, ldm, kdim / AS_BK, kd, M, err);
}

}  // namespace xtc
