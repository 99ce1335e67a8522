// Step (b) on the tensor cores: the vector pair fields of the "Decomposition of two-body
// correction" section,
//     V_x[i][pq] = sum_j G_x(i, j) rho^T[pq][j],   G_x(i, j) = d/dx_i u(r_i, r_j),
//     rho^T[pq][j] = w_j phi_p(j) phi_q(j),
// as a split-precision GEMM over the inner points j: A = G (written by gfield.cu, rows x*gcp + il),
// B = rho^T (written by the rho split kernel), both split into fp16 (2 parts) or bf16 (3 parts).
//
// Tile: 128 A rows per CTA (128 outer points of one component) x BN orbital pairs (192 with 2
// parts, 160 with 3), 32 inner points per pipeline stage, K-major, all operands loaded by TMA.
// With 2 parts both parts of a row share one 128-byte row (128-byte swizzle; one TMA box per
// operand and stage); with 3 parts every part is a plane of 64-byte rows (64-byte swizzle).
//
// Every tcgen05.commit stalls the tensor pipe for a few hundred cycles (measured: a group of g
// back-to-back MMAs plus its commit takes about g x 96 + 300 cycles at N = 192), so the kernel
// commits once per accumulation range: that single arrival releases the range's stage slots to the
// TMA producer (which counts finished ranges in order) and hands the accumulator to the drains.
//
// Warp roles:
//   * warp 0 (one lane): TMA loads of the A and B tiles;
//   * warps 1 and 10 (one lane each): MMA issuers of the even and the odd ranges;
//   * warps 2..9: every `kd` stages they load the finished accumulator (tcgen05.ld) and add it into
//     an FP32 running sum held in their registers (two warps per TMEM lane quarter, BN/2 columns
//     each) while the MMA fills the other accumulator; at the end they store the sum, unscaled, as
//     V[pq][x][i].
// The tensor-core accumulator truncates toward zero at each MMA, which biases a long inner sum.
// Each range is short (default one stage), its MMAs issue the small cross products of all its
// stages first so that only the hi x hi products meet a large accumulator, and the ranges are
// summed with round-to-nearest FP32 adds.  Rounding of that FP32 sum grows with the number of
// ranges, so every `flush` ranges the drains add their FP32 partial sums into an FP64 accumulator
// in HBM, private to the CTA and column-major in its tile (each element belongs to one thread:
// plain read-modify-write, coalesced over the 32 rows of a warp); the final sum is written as V.
// Tiles are ordered in groups of GM row tiles so that the CTAs resident at one time share their A
// and B panels in L2.
//
// The same engine runs step (d) for the fp16 x2 precision (MODE 1): M += L^T R with A = the split
// rows L[pq] (rho, V) and B = the split rows R[rs] (A, B) of a chunk, K = 4 x chunk points, each
// row carrying its own power-of-2 scale; its tile-private FP64 sums are then added into M[pq][rs],
// unscaled, by assemble_finalize_kernel.
#include "ptx_sm100.cuh"
#include "xtc_internal.cuh"

namespace xtc {
namespace {

constexpr int DRAIN_WARPS = 8;       // two per TMEM lane quarter, BN/2 columns each
constexpr int MMA_WARPS = 2;         // issuers of the even / odd ranges (warps 1 and 2 + DRAIN_WARPS)
constexpr int THREADS = (1 + MMA_WARPS + DRAIN_WARPS) * 32;
constexpr int A_TILE = VF_BM * 64;   // bytes per part of an A tile (128 rows of 64 B)
constexpr int GM = 8;                // row tiles per group (L2 reuse)

constexpr int NRB = 8;               // range barriers (range r uses r % NRB)

template <int PARTS>
struct VfCfg {
  static constexpr int BN = vf_bn(PARTS);   // columns of the tile (TMEM accumulator width)
  static constexpr int B_TILE = BN * 64;    // bytes per part of a B tile
  static constexpr int HC = BN / 2;         // running-sum columns per drain thread
  static constexpr int NPROD = PARTS == 2 ? 3 : 6;
  static constexpr int A_BYTES = PARTS * A_TILE;
  static constexpr int B_BYTES = PARTS * B_TILE;
  static constexpr int STAGE_BYTES = ((A_BYTES + B_BYTES + 1023) / 1024) * 1024;
  static constexpr int STAGES = (220 * 1024) / STAGE_BYTES < 8 ? (220 * 1024) / STAGE_BYTES : 8;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};
static_assert(VfCfg<2>::SMEM <= 232448 && VfCfg<3>::SMEM <= 232448, "shared memory per CTA");
static_assert(VfCfg<2>::STAGES >= 4 && VfCfg<3>::STAGES >= 4, "pipeline depth");
// a wait for range r must not alias range r + NRB: the producer waits for the range of stage
// k - STAGES before loading stage k, and range r + NRB starts past stage k when NRB > STAGES
static_assert(NRB > VfCfg<2>::STAGES && NRB > VfCfg<3>::STAGES, "range barriers");
static_assert(2 * vf_bn(2) <= 512 && 2 * vf_bn(3) <= 512, "two accumulators in 512 TMEM columns");
static_assert(vf_bn(2) % 32 == 0 && vf_bn(3) % 32 == 0, "drain halves of whole 16-column chunks");

// Shared-memory descriptor of part p, K step ks (16 values) of an operand tile at `base`.
template <int PARTS>
__device__ __forceinline__ uint64_t op_desc(uint32_t base, int tile_bytes, int p, int ks) {
  if (PARTS == 2) return sdesc_kmajor_sw128(base + p * 64 + ks * 32);
  return sdesc_kmajor_sw64(base + p * tile_bytes + ks * 32);
}

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

__device__ __forceinline__ void red_add_f64(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns: thread t of the warp receives lane (base + t).
__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

template <int PARTS, int MODE>
__global__ void __launch_bounds__(THREADS, 1)
    vfield_tc_kernel(const __grid_constant__ CUtensorMap tm_g, const __grid_constant__ CUtensorMap tm_rho,
                     const VfieldArgs args) {
  using Cfg = VfCfg<PARTS>;
  constexpr bool BF16 = PARTS == 3;
  constexpr int BN = Cfg::BN, HC = Cfg::HC, STAGES = Cfg::STAGES;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * Cfg::STAGE_BYTES);
  uint64_t* tma_full = bars;                  // [STAGES] the stage's loads landed
  uint64_t* rdone = bars + STAGES;            // [NRB] the MMAs of range r (r % NRB) completed
  uint64_t* d_free = bars + STAGES + NRB;     // [2] the drains released accumulator b
  uint64_t* fin_bar = bars + STAGES + NRB + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + STAGES + NRB + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped tile order: GM row tiles x every column tile, row tile fastest
  const int m_tiles = MODE == 0 ? 3 * args.mt_per_x : (args.rows_a + VF_BM - 1) / VF_BM;
  const int L = blockIdx.x;
  const int group = L / (GM * args.n_tiles);
  const int first_m = group * GM;
  const int gm = min(GM, m_tiles - first_m);
  const int rem = L - group * GM * args.n_tiles;
  const int m_tile = first_m + rem % gm, n_tile = rem / gm;
  // mode 0: rows x * gcp + outer point of component x; mode 1: rows pq
  const int x = MODE == 0 ? m_tile / args.mt_per_x : 0;
  const int ib = MODE == 0 ? (m_tile - x * args.mt_per_x) * VF_BM : m_tile * VF_BM;
  const int row0 = MODE == 0 ? static_cast<int>(x * args.gcp) + ib : ib;
  const int split = blockIdx.y;
  const int kb0 = split * args.kb_per_split;
  const int kb1 = min(args.n_kb, kb0 + args.kb_per_split);
  const int n_it = kb1 - kb0;
  const int kd = args.kd;
  const int n_ranges = (n_it + kd - 1) / kd;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&tma_full[s], 1);
    for (int r = 0; r < NRB; ++r) mbar_init(&rdone[r], 1);
    for (int b = 0; b < 2; ++b) mbar_init(&d_free[b], DRAIN_WARPS);
    mbar_init(fin_bar, MMA_WARPS);
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_desc(&tm_g);
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
      int seen = 0;  // ranges known to have completed (their slots are free again)
      int issued_end = kb0;
      for (int kb = kb0; kb < kb1; ++kb) {
        const int it = kb - kb0, s = it % STAGES;
        if (it >= STAGES) {
          const int need = (it - STAGES) / kd;  // range holding the slot's previous stage
          bool ok = true;
          for (; seen <= need && ok; ++seen)
            ok = mbar_wait(&rdone[seen % NRB], (seen / NRB) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF);
          if (!ok) break;
        }
        mbar_arrive_expect_tx(&tma_full[s], Cfg::A_BYTES + Cfg::B_BYTES);
        uint8_t* st = smem + s * Cfg::STAGE_BYTES;
        if (PARTS == 2) {
          // one 128-byte-row box per operand holds both parts
          tma_load_3d(st, &tm_g, &tma_full[s], kb * 2 * VF_BK, row0, 0);
          tma_load_3d(st + Cfg::A_BYTES, &tm_rho, &tma_full[s], kb * 2 * VF_BK, n_tile * BN, 0);
        } else {
          for (int p = 0; p < PARTS; ++p) {
            tma_load_3d(st + p * A_TILE, &tm_g, &tma_full[s], kb * VF_BK, row0, p);
            tma_load_3d(st + Cfg::A_BYTES + p * Cfg::B_TILE, &tm_rho, &tma_full[s], kb * VF_BK, n_tile * BN, p);
          }
        }
        issued_end = kb + 1;
      }
      // the copies still in flight land before the CTA may exit
      int zero = 0;
      for (int kb = max(kb0, issued_end - STAGES); kb < issued_end; ++kb) {
        const int it = kb - kb0;
        mbar_wait(&tma_full[it % STAGES], (it / STAGES) & 1, reinterpret_cast<volatile int*>(&zero), args.err,
                  DEV_ERR_TIMEOUT_VF);
      }
    }
  } else if (warp == 1 || warp == 2 + DRAIN_WARPS) {
    if (lane == 0) {
      // ---------------------------------------------------------------- MMA issuers
      // A range of kd stages goes into one TMEM accumulator: first the cross products of each
      // stage as it lands (the accumulator is still small), then the hi x hi product of every
      // stage; one commit per range.  Warp 1 issues the even ranges (accumulator 0), the last warp
      // the odd ones (accumulator 1): a commit tracks only its own thread's MMAs, so while one
      // issuer's commit completes the other keeps the tensor pipe fed.
      constexpr uint32_t idesc = idesc_f16(VF_BM, BN, BF16);
      bool alive = true;
      for (int r = warp == 1 ? 0 : 1; r < n_ranges && alive; r += MMA_WARPS) {
        const int it0 = r * kd, it1 = min(n_it, it0 + kd);
        const int b = r & 1, u = r >> 1;
        const uint32_t d_tmem = tmem + b * BN;
        if (u >= 1 && !mbar_wait(&d_free[b], (u - 1) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF)) break;
        for (int it = it0; it < it1; ++it) {
          const int s = it % STAGES;
          if (!(alive = mbar_wait(&tma_full[s], (it / STAGES) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF))) break;
          tc_fence_after();
          const uint32_t sa = smem_base + s * Cfg::STAGE_BYTES;
          const uint32_t sb = sa + Cfg::A_BYTES;
#pragma unroll
          for (int p = 0; p < Cfg::NPROD - 1; ++p) {
            int pa, pb;
            prod_parts<PARTS>(p, pa, pb);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
              tc_mma_f16(d_tmem, op_desc<PARTS>(sa, A_TILE, pa, ks), op_desc<PARTS>(sb, Cfg::B_TILE, pb, ks), idesc,
                         (it == it0 && p == 0 && ks == 0) ? 0u : 1u);
          }
        }
        if (!alive) break;
        for (int it = it0; it < it1; ++it) {
          const uint32_t sa = smem_base + (it % STAGES) * Cfg::STAGE_BYTES;
          const uint32_t sb = sa + Cfg::A_BYTES;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks)
            tc_mma_f16(d_tmem, op_desc<PARTS>(sa, A_TILE, 0, ks), op_desc<PARTS>(sb, Cfg::B_TILE, 0, ks), idesc, 1u);
        }
        tc_commit(&rdone[r % NRB]);
      }
      // every MMA issued by both issuers has completed once fin_bar fires
      tc_commit(fin_bar);
      int zero = 0;
      mbar_wait(fin_bar, 0, reinterpret_cast<volatile int*>(&zero), args.err, DEV_ERR_TIMEOUT_VF);
    }
  } else {
    // ------------------------------------------------------------------ range drains and epilogue
    const int quarter = warp & 3;               // TMEM lanes 32*quarter .. +31 (hardware rule)
    const int half = (warp - 2) >> 2;           // columns HC*half .. +HC-1
    const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
    const uint32_t c_base = static_cast<uint32_t>(half * HC);
    float S[HC];
#pragma unroll
    for (int k = 0; k < HC; ++k) S[k] = 0.0f;
    // Adds the running sums into this thread's elements of the CTA-private FP64 accumulator,
    // column-major in the tile: Vacc[(split * gridDim.x + tile) * 128 * BN + column * 128 + row],
    // column = c_base + k (a store the first time, then fire-and-forget reductions, which need
    // no result registers), and clears them.
    int nflush = 0;
    auto flush_sums = [&]() {
      double* acc = args.Vacc + (static_cast<int64_t>(split) * gridDim.x + blockIdx.x) * VF_BM * BN +
                    static_cast<int64_t>(c_base) * VF_BM + quarter * 32 + lane;
      if (nflush == 0) {
#pragma unroll
        for (int k = 0; k < HC; ++k) acc[k * VF_BM] = static_cast<double>(S[k]);
      } else {
#pragma unroll
        for (int k = 0; k < HC; ++k) red_add_f64(acc + k * VF_BM, static_cast<double>(S[k]));
      }
#pragma unroll
      for (int k = 0; k < HC; ++k) S[k] = 0.0f;
      ++nflush;
    };
    bool ok = true;
    for (int r = 0; r < n_ranges && ok; ++r) {
      const int b = r & 1;
      ok = __all_sync(0xffffffffu,
                      mbar_wait(&rdone[r % NRB], (r / NRB) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF));
      __syncwarp();
      if (!ok) break;
      tc_fence_after();
      const uint32_t src = tmem + lane_base + b * BN + c_base;
#pragma unroll
      for (int c = 0; c < HC; c += 16) {
        uint32_t d0[16];
        tmem_ld_x16(src + c, d0);
        tmem_wait_ld();
#pragma unroll
        for (int k = 0; k < 16; ++k) S[c + k] += __uint_as_float(d0[k]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&d_free[b]);
      // FP64 flush of the partial sums (the accumulator is already handed back to the MMA)
      if (args.flush > 0 && (r + 1) % args.flush == 0) flush_sums();
    }
    if (args.flush > 0) {
      // the remaining sums join the FP64 accumulator; a finalize kernel writes V (mode 0) or adds
      // the tile into M (mode 1)
      if (ok && n_ranges % args.flush != 0) flush_sums();
    } else {
      // FP32 sums straight to V: row = outer point ib + row of component x -> V[split][pq][x][il]
      const int row = quarter * 32 + lane;
      const int64_t il = static_cast<int64_t>(ib) + row;
      const int64_t col_off = static_cast<int64_t>(x) * args.gcp + il;
      const int pq0 = n_tile * BN + static_cast<int>(c_base);
      if (ok && !*abort_flag && il < args.n_i && n_it > 0) {
        float* Vz = args.V + static_cast<int64_t>(split) * args.n_pair * 3 * args.gcp;
#pragma unroll
        for (int k = 0; k < HC; ++k) {
          const int pq = pq0 + k;
          if (pq < args.n_pair)
            Vz[static_cast<int64_t>(pq) * 3 * args.gcp + col_off] =
                ldexpf(S[k] * args.unscale_g, -__ldg(args.colexp + pq));
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

// V from the FP64 accumulator of the GEMM: one CTA per (tile, split), thread = tile row; the tile
// order is the GEMM's grouped order.
template <int BN>
__global__ void __launch_bounds__(VF_BM) vfield_finalize_kernel(const VfieldArgs args) {
  const int m_tiles = 3 * args.mt_per_x;
  const int L = blockIdx.x;
  const int group = L / (GM * args.n_tiles);
  const int first_m = group * GM;
  const int gm = min(GM, m_tiles - first_m);
  const int rem = L - group * GM * args.n_tiles;
  const int m_tile = first_m + rem % gm, n_tile = rem / gm;
  const int x = m_tile / args.mt_per_x;
  const int row = threadIdx.x;
  const int64_t il = static_cast<int64_t>(m_tile - x * args.mt_per_x) * VF_BM + row;
  if (il >= args.n_i) return;
  const double* acc = args.Vacc + (static_cast<int64_t>(blockIdx.y) * gridDim.x + L) * VF_BM * BN + row;
  float* v = args.V + static_cast<int64_t>(blockIdx.y) * args.n_pair * 3 * args.gcp + x * args.gcp + il;
  const int ncol = min(BN, args.n_pair - n_tile * BN);
  for (int c = 0; c < ncol; ++c) {
    const int pq = n_tile * BN + c;
    v[static_cast<int64_t>(pq) * 3 * args.gcp] =
        ldexpf(static_cast<float>(acc[static_cast<int64_t>(c) * VF_BM]) * args.unscale_g, -__ldg(args.colexp + pq));
  }
}

// M[pq][rs] += tile sum * 2^-(exp_a[pq] + exp_b[rs]) for one tile of the step (d) GEMM (mode 1);
// one CTA per tile, thread = row pq, columns in order (coalesced tile reads; each M element is
// owned by one tile).
template <int BN>
__global__ void __launch_bounds__(VF_BM) assemble_finalize_kernel(const VfieldArgs args) {
  const int m_tiles = (args.rows_a + VF_BM - 1) / VF_BM;
  const int L = blockIdx.x;
  const int group = L / (GM * args.n_tiles);
  const int first_m = group * GM;
  const int gm = min(GM, m_tiles - first_m);
  const int rem = L - group * GM * args.n_tiles;
  const int m_tile = first_m + rem % gm, n_tile = rem / gm;
  const int pq = m_tile * VF_BM + threadIdx.x;
  if (pq >= args.rows_a) return;
  const double* acc = args.Vacc + (static_cast<int64_t>(blockIdx.y) * gridDim.x + L) * VF_BM * BN + threadIdx.x;
  double* m = args.M + static_cast<int64_t>(pq) * args.ldm + n_tile * BN;
  const int ea = args.exp_a[pq];
  const int ncol = min(BN, args.n_pair - n_tile * BN);
  for (int c = 0; c < ncol; ++c) {
    const int e = ea + __ldg(args.exp_b + n_tile * BN + c);
    m[c] += acc[static_cast<int64_t>(c) * VF_BM] * __longlong_as_double(static_cast<long long>(1023 - e) << 52);
  }
}

template <int PARTS, int MODE>
void launch_t(const CUtensorMap* tm_g, const CUtensorMap* tm_rho, const VfieldArgs& a, int splits,
              cudaStream_t st) {
  auto kern = vfield_tc_kernel<PARTS, MODE>;
  constexpr int smem = VfCfg<PARTS>::SMEM;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int m_tiles = MODE == 0 ? 3 * a.mt_per_x : (a.rows_a + VF_BM - 1) / VF_BM;
  dim3 grid(static_cast<unsigned>(m_tiles * a.n_tiles), static_cast<unsigned>(splits));
  kern<<<grid, THREADS, smem, st>>>(*tm_g, *tm_rho, a);
}

template <int PARTS, int MODE>
void finalize_t(const VfieldArgs& a, int splits, cudaStream_t st) {
  const int m_tiles = MODE == 0 ? 3 * a.mt_per_x : (a.rows_a + VF_BM - 1) / VF_BM;
  dim3 grid(static_cast<unsigned>(m_tiles * a.n_tiles), static_cast<unsigned>(splits));
  if (MODE == 0 && a.flush > 0) vfield_finalize_kernel<VfCfg<PARTS>::BN><<<grid, VF_BM, 0, st>>>(a);
  if (MODE == 1) assemble_finalize_kernel<VfCfg<PARTS>::BN><<<grid, VF_BM, 0, st>>>(a);
}

}  // namespace

bool vfield_tc_supported(int n_nuc) { return n_nuc >= 1 && n_nuc <= 8; }

void launch_vfield_tc(const CUtensorMap* tm_g, const CUtensorMap* tm_rho, const VfieldArgs& a, int parts,
                      int splits, cudaStream_t st) {
  if (a.n_tiles <= 0 || splits <= 0) return;
  if (a.mode == 1) {
    if (a.rows_a > 0) launch_t<2, 1>(tm_g, tm_rho, a, splits, st);
    return;
  }
  if (a.mt_per_x <= 0) return;
  if (parts == 2)
    launch_t<2, 0>(tm_g, tm_rho, a, splits, st);
  else
    launch_t<3, 0>(tm_g, tm_rho, a, splits, st);
}

void launch_vfield_tc_finalize(const VfieldArgs& a, int parts, int splits, cudaStream_t st) {
  if (a.n_tiles <= 0 || splits <= 0) return;
  if (a.mode == 1) {
    if (a.rows_a > 0) finalize_t<2, 1>(a, splits, st);
    return;
  }
  if (a.mt_per_x <= 0 || a.flush <= 0) return;
  if (parts == 2)
    finalize_t<2, 0>(a, splits, st);
  else
    finalize_t<3, 0>(a, splits, st);
}

}  // namespace xtc
