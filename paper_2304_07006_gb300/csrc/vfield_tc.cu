// Step (b) on the tensor cores: the vector pair fields of the "Decomposition of two-body
// correction" section,
//     V_x[i][pq] = sum_j G_x(i, j) rho^T[pq][j],   G_x(i, j) = d/dx_i u(r_i, r_j),
//     rho^T[pq][j] = w_j phi_p(j) phi_q(j),
// as a split-precision GEMM over the inner points j: A = G (written by gfield.cu, rows x*gcp + il),
// B = rho^T (written by the rho split kernel), K-major, all operands loaded by TMA.  The same fp16
// engine runs step (d) of Appendix B (MODE 1): M += L^T R with A = the split rows L[pq]
// (rho, V) and B = the split rows R[rs] (A, B) of a chunk, K = 4 x chunk points, each row carrying
// its own power-of-2 scale; its tile sums are added into M[pq][rs] by assemble_finalize_kernel.
//
// fp16 x2 engine (xgemm_kernel).  Both operands are split exactly on per-range quanta (simt_pack.cuh):
// per row and accumulation range of kd stages (kd * 32 K values), hi = an integer times the row's
// power-of-2 quantum for that range (from the range's largest magnitude), lo = the fp16 remainder,
// with bit widths such that the range's hi x hi products sum within 2^24 units.
// The tensor core's FP32 accumulator truncates toward zero at every MMA, which biases a long sum
// by a relative ~2^-24 per MMA, always toward zero; the hi x hi sums of a range are exact, so they
// go, one range at a time, into an accumulator E, which the drain warps add into FP32 running sums
// (round to nearest) after every range.  The cross products (about 2^-9 of the total, signs that
// follow the rounding remainders rather than the data) go into a second accumulator X, drained
// every `xper` stages; their truncation is 2^-9 smaller and does not accumulate one-sided.  They
// must include lo_a x lo_b: where both operands hold values far below their range's maximum, hi is
// 0 and lo is the whole value.  Both steps issue hi_a x lo_b and lo_a x fp16(b), with fp16(b) a
// third plane of the B operand (rho^T in step (b), R in step (d)): lo_a x (hi_b + lo_b) to within
// fp16's rounding of b (a relative 2^-12 of a term that is itself 2^-10 of the product), one
// product where two would be needed.
//
// Tile 128 A rows x 128 columns, 32 K values per stage, both parts of a row of a block in one
// 128-byte row (128-byte swizzle; one TMA box per operand part and stage).  Measured
// on GB300: one thread issues a 128 x 128 x 16 MMA every ~50 cycles (the pipe takes 64), an MMA
// and its commit round-trip in ~360 cycles, and a range's round trip (its MMAs complete, the
// commit arrives, the drains read E, E is handed back) takes on the order of a thousand cycles.
// So ranges span two stages (12 MMAs), and two issuers alternate ranges, each with its own
// accumulator pair (TMEM: E0, X0, E1, X1 = 4 x 128 of 512 columns).  A stage holds 40 KB (A and B
// hi/lo, fp16(B)); 5 stages.  Warp roles:
//   * warp 0 (one lane): TMA loads; a slot is reloaded once the MMAs of its stage have completed;
//   * warps 1 and 2 (one lane each): the MMAs of the even / odd ranges, a commit per stage (it
//     frees the slot) and one per range (it starts the drains);
//   * warps 3..18: after every range, drains of E_k, and every `xper` stages of X_k, into FP32
//     running sums held in registers (four warps per TMEM lane quarter, 32 columns each).  The
//     sums move into an FP64 accumulator in HBM, private to the CTA and column-major in its tile,
//     one column per range in turn (each column at least once per `flush` ranges; each element
//     belongs to one thread); vfield_finalize_kernel writes V from it (MODE 0).
// Tiles are ordered in groups of GM row tiles so that the CTAs resident at one time share their A
// and B panels in L2.
//
// bf16 x3 engine (vfield_bf16_kernel, step (b) of the bf16 precision): three bf16 planes per
// operand (64-byte swizzle), six products (i + j <= 2) into one of two TMEM accumulators per range
// of `kd` stages, small cross products first, drained into FP32 running sums after every range.
// Its accumulation is not exact: the truncation bias is only kept small by the short ranges.
#include "ptx_sm100.cuh"
#include "xtc_internal.cuh"

namespace xtc {
namespace {

constexpr int DRAIN_WARPS = 8;       // two per TMEM lane quarter, half of the columns each
constexpr int GM = 16;               // row tiles per group (L2 reuse of the column panels)
constexpr int NRB = 8;               // per-stage / per-range barriers (stage or range r uses r % NRB)

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

// Tile coordinates of CTA L in the grouped order (GM row tiles x every column tile, row fastest).
struct TileXY {
  int m_tile, n_tile;
};
__device__ __forceinline__ TileXY grouped_tile(int L, int m_tiles, int n_tiles) {
  const int group = L / (GM * n_tiles);
  const int first_m = group * GM;
  const int gm = min(GM, m_tiles - first_m);
  const int rem = L - group * GM * n_tiles;
  return {first_m + rem % gm, rem / gm};
}

// =================================================================== fp16 x2 engine
constexpr int XB_BN = 128;                        // tile columns (TMEM accumulator width)
constexpr int XB_DRAIN_WARPS = 16;                // four per TMEM lane quarter, a quarter of the columns each
constexpr int XB_HC = XB_BN / 4;                  // running-sum columns per drain thread
constexpr int XB_A_BYTES = VF_BM * 128;           // 128 rows of 128 bytes (hi and lo of 32 values)
constexpr int XB_B_BYTES = XB_BN * 128;
constexpr int XB_B16_BYTES = XB_BN * 64;          // fp16(B) of the B rows, 64-byte rows
// stage bytes and pipeline depth: 40 KB (A, B hi/lo, B fp16) x 5
__host__ __device__ constexpr int xb_stage(int) { return XB_A_BYTES + XB_B_BYTES + XB_B16_BYTES; }
__host__ __device__ constexpr int xb_stages(int) { return 5; }
constexpr int XB_STAGES = 7;                      // the larger depth (barrier arrays)
constexpr int XB_WARP_I0 = 1, XB_WARP_I1 = 2;      // issuers of the even / odd ranges; drains 3..18
constexpr int XB_THREADS = (3 + XB_DRAIN_WARPS) * 32;  // TMA warp, two MMA warps, drains
__host__ __device__ constexpr int xb_smem(int mode) { return xb_stages(mode) * xb_stage(mode) + 1024 + 256; }
static_assert(XB_BN == vf_bn(2), "tile width of the fp16 engine");
static_assert(4 * XB_BN <= 512, "E0, X0, E1, X1 in 512 TMEM columns");
static_assert(XB_HC == 32, "drain columns per thread (one 32-column load)");
static_assert(xb_smem(0) <= 232448 && xb_smem(1) <= 232448, "shared memory per CTA");
static_assert(xb_stages(0) <= XB_STAGES && xb_stages(1) <= XB_STAGES, "barrier arrays");
// a wait for range r must not alias range r + NRB: the producer waits for the range of stage
// k - XB_STAGES before loading stage k, and range r + NRB starts past stage k
static_assert(NRB > XB_STAGES, "range barriers");
static_assert((XB_STAGES + NRB + 5) * 8 + 8 <= 256, "barrier area");

// Shared-memory descriptor of a K-major operand in the 128-byte swizzle, for a shared address
// below 2^18: the constant fields plus the address in 16-byte units (a plain add per stage and
// K step, no re-encoding in the issue loop).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) { return sdesc_kmajor_sw128(0) + (saddr >> 4); }
// The same for 64-byte rows in the 64-byte swizzle.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) { return sdesc_kmajor_sw64(0) + (saddr >> 4); }

template <int MODE>
__global__ void __launch_bounds__(XB_THREADS, 1)
    xgemm_kernel(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_b,
                 const __grid_constant__ CUtensorMap tm_b16, const VfieldArgs args) {
  constexpr int XB_STAGE = xb_stage(MODE), STAGES = xb_stages(MODE);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * XB_STAGE);
  uint64_t* tma_full = bars;                  // [XB_STAGES] the stage's loads landed
  uint64_t* rdone = bars + XB_STAGES;         // [NRB] every MMA of range r (r % NRB) completed
  uint64_t* e_free = rdone + NRB;             // [2] the drains released E_k (issuer k)
  uint64_t* x_free = e_free + 2;              // [2] the drains released X_k
  uint64_t* fin_bar = x_free + 2;             // every MMA of both issuers completed
  uint64_t* sfree = fin_bar + 1;              // [XB_STAGES] the stage's MMAs completed (slot free)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sfree + XB_STAGES);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m_tiles = MODE == 0 ? 3 * args.mt_per_x : (args.rows_a + VF_BM - 1) / VF_BM;
  const TileXY t = grouped_tile(blockIdx.x, m_tiles, args.n_tiles);
  // mode 0: rows x * gcp + outer point of component x; mode 1: rows pq
  const int x = MODE == 0 ? t.m_tile / args.mt_per_x : 0;
  const int ib = MODE == 0 ? (t.m_tile - x * args.mt_per_x) * VF_BM : t.m_tile * VF_BM;
  const int row0 = MODE == 0 ? static_cast<int>(x * args.gcp) + ib : ib;
  const int split = blockIdx.y;
  const int kb0 = split * args.kb_per_split;
  const int kb1 = min(args.n_kb, kb0 + args.kb_per_split);
  const int n_it = kb1 - kb0;
  const int kd = args.kd;                                  // stages per exact range (1, 2 or 4)
  const int n_ranges = (n_it + kd - 1) / kd;
  const int xr = max(1, args.xper / (2 * kd));             // ranges of one issuer per X drain

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&tma_full[s], 1);
      mbar_init(&sfree[s], 1);
    }
    for (int r = 0; r < NRB; ++r) mbar_init(&rdone[r], 1);
    for (int k = 0; k < 2; ++k) {
      mbar_init(&e_free[k], XB_DRAIN_WARPS);
      mbar_init(&x_free[k], XB_DRAIN_WARPS);
    }
    mbar_init(fin_bar, 2);
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_desc(&tm_a);
    tma_prefetch_desc(&tm_b);
    tma_prefetch_desc(&tm_b16);
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
      // a slot is refilled as soon as the MMAs of the stage it held have completed (one commit
      // per stage), not when the whole range has
      int issued = 0;
      for (int it = 0; it < n_it; ++it) {
        const int s = it % STAGES;
        if (it >= STAGES &&
            !mbar_wait(&sfree[s], ((it / STAGES) - 1) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF))
          break;
        mbar_arrive_expect_tx(&tma_full[s], XB_STAGE);
        uint8_t* st = smem + s * XB_STAGE;
        tma_load_3d(st, &tm_a, &tma_full[s], (kb0 + it) * 2 * VF_BK, row0, 0);
        tma_load_3d(st + XB_A_BYTES, &tm_b, &tma_full[s], (kb0 + it) * 2 * VF_BK, t.n_tile * XB_BN, 0);
        tma_load_3d(st + XB_A_BYTES + XB_B_BYTES, &tm_b16, &tma_full[s], (kb0 + it) * VF_BK, t.n_tile * XB_BN, 0);
        issued = it + 1;
      }
      // the copies still in flight land before the CTA may exit
      int zero = 0;
      for (int it = max(0, issued - STAGES); it < issued; ++it)
        mbar_wait(&tma_full[it % STAGES], (it / STAGES) & 1, reinterpret_cast<volatile int*>(&zero),
                  args.err, DEV_ERR_TIMEOUT_VF);
    }
  } else if (warp == XB_WARP_I0 || warp == XB_WARP_I1) {
    if (lane == 0) {
      // ---------------------------------------------------------------- MMA issuers
      // Issuer k takes the ranges r = k, k + 2, ...: per stage the hi x hi products into E_k (a
      // fresh, exact accumulation per range) and the cross products hi_a x lo_b, lo_a x fp16(b)
      // into X_k (restarted every xr of its ranges); a commit after each stage frees
      // its slot for the next load, one after each range starts the drains.  With two issuers
      // one's waits and commits overlap the other's MMAs, and neither waits for the other's drains.
      constexpr uint32_t idesc = idesc_f16(VF_BM, XB_BN, false);
      const int k = warp == XB_WARP_I0 ? 0 : 1;
      const uint32_t e_tmem = tmem + 2 * k * XB_BN, x_tmem = e_tmem + XB_BN;
      for (int r = k, u = 0; r < n_ranges; r += 2, ++u) {
        const int it0 = r * kd, it1 = min(n_it, it0 + kd);
        const bool x_start = u % xr == 0;
        if (u >= 1 && !mbar_spin(&e_free[k], (u - 1) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF)) break;
        if (x_start && u >= xr &&
            !mbar_spin(&x_free[k], ((u / xr) - 1) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF))
          break;
        bool alive = true;
        for (int it = it0; it < it1; ++it) {
          const int s = it % STAGES;
          if (!(alive = mbar_spin(&tma_full[s], (it / STAGES) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF)))
            break;
          tc_fence_after();
          const uint32_t sa = smem_base + s * XB_STAGE;
          const uint64_t da = sw128_desc(sa), db = da + (XB_A_BYTES >> 4);
          // K steps of 16 values advance 32 bytes (2 descriptor units); lo parts sit 64 bytes on
          tc_mma_f16(e_tmem, da, db, idesc, it > it0 ? 1u : 0u);
          tc_mma_f16(e_tmem, da + 2, db + 2, idesc, 1u);
          tc_mma_f16(x_tmem, da, db + 4, idesc, (x_start && it == it0) ? 0u : 1u);   // hi_a x lo_b
          tc_mma_f16(x_tmem, da + 2, db + 6, idesc, 1u);
          // lo_a x fp16(b): lo_a x (hi_b + lo_b) to within fp16(b)'s rounding, one product
          const uint64_t d16 = sw64_desc(sa + XB_A_BYTES + XB_B_BYTES);
          tc_mma_f16(x_tmem, da + 4, d16, idesc, 1u);
          tc_mma_f16(x_tmem, da + 6, d16 + 2, idesc, 1u);
          tc_commit(&sfree[s]);
        }
        if (!alive) break;
        tc_commit(&rdone[r % NRB]);
      }
      // every MMA issued by both issuers has completed once fin_bar fires
      tc_commit(fin_bar);
      int zero = 0;
      mbar_wait(fin_bar, 0, reinterpret_cast<volatile int*>(&zero), args.err, DEV_ERR_TIMEOUT_VF);
    }
  } else {
    // ------------------------------------------------------------------ drains and epilogue
    const int quarter = warp & 3;               // TMEM lanes 32*quarter .. +31 (hardware rule)
    const int group = (warp - 3) >> 2;          // columns XB_HC*group .. +XB_HC-1
    const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
    const uint32_t c_base = static_cast<uint32_t>(group * XB_HC);
    float S[XB_HC];
#pragma unroll
    for (int k = 0; k < XB_HC; ++k) S[k] = 0.0f;
    // S += this thread's 32 columns of the accumulator at TMEM column col
    auto add_acc = [&](uint32_t col) {
      uint32_t d[32];
      tmem_ld_32x32b_x32(tmem + lane_base + col + c_base, d);
      tmem_wait_ld();
#pragma unroll
      for (int k = 0; k < 32; ++k) S[k] += __uint_as_float(d[k]);
    };
    // The FP32 running sums move into the CTA-private FP64 accumulator, column-major in the tile:
    // Vacc[(split * gridDim.x + tile) * 128 * BN + column * 128 + row], column = c_base + c.  Column
    // c of every thread goes after range r when r % flush == c (staggered, so that no drain carries a
    // whole tile of FP64 adds at once): a store the first time (r < flush), then a fire-and-forget
    // reduction; every column is flushed at least once per `flush` ranges.
    double* acc = args.Vacc + (static_cast<int64_t>(split) * gridDim.x + blockIdx.x) * VF_BM * XB_BN +
                  static_cast<int64_t>(c_base) * VF_BM + quarter * 32 + lane;
    auto flush_col = [&](int c, bool first) {
#pragma unroll
      for (int k = 0; k < XB_HC; ++k)
        if (k == c) {
          if (first)
            acc[k * VF_BM] = static_cast<double>(S[k]);
          else
            red_add_f64(acc + k * VF_BM, static_cast<double>(S[k]));
          S[k] = 0.0f;
        }
    };
    bool ok = true;
    for (int r = 0; r < n_ranges && ok; ++r) {
      const int k = r & 1, u = r >> 1;
      // X_k is drained at the end of each of its periods and after issuer k's last range
      const bool x_end = u % xr == xr - 1 || r + 2 >= n_ranges;
      // a non-suspending wait: the drain's wake-up sits on the range round trip
      ok = __all_sync(0xffffffffu,
                      mbar_spin(&rdone[r % NRB], (r / NRB) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF));
      __syncwarp();
      if (!ok) break;
      tc_fence_after();
      add_acc(2 * k * XB_BN);
      if (x_end) add_acc((2 * k + 1) * XB_BN);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&e_free[k]);
        if (x_end) mbar_arrive(&x_free[k]);
      }
      // staggered FP64 flush (the accumulators are already handed back to the MMAs)
      if (args.flush > 0 && r % args.flush < XB_HC) flush_col(r % args.flush, r < args.flush);
    }
    if (args.flush > 0) {
      // the remaining sums join the FP64 accumulator (columns never flushed in the loop are
      // stored); a finalize kernel writes V (mode 0) or adds the tile into M (mode 1)
      if (ok) {
#pragma unroll
        for (int c = 0; c < XB_HC; ++c) {
          if (c < min(n_ranges, args.flush))
            red_add_f64(acc + c * VF_BM, static_cast<double>(S[c]));
          else
            acc[c * VF_BM] = static_cast<double>(S[c]);
        }
      }
    } else if (MODE == 0) {
      // FP32 sums straight to V: row = outer point ib + row of component x, both (p, s) and (s, p)
      const int row = quarter * 32 + lane;
      const int64_t il = static_cast<int64_t>(ib) + row;
      const int pq0 = t.n_tile * XB_BN + static_cast<int>(c_base);
      if (ok && !*abort_flag && il < args.n_i && n_it > 0) {
        float* Vz = args.V + split * v_slice(args.gcp, args.n_orb);
#pragma unroll
        for (int k = 0; k < XB_HC; ++k) {
          const int pq = pq0 + k;
          if (pq < args.n_pair) {
            const int p = __ldg(args.pair_p + pq), q = __ldg(args.pair_q + pq);
            const float v = ldexpf(S[k] * args.unscale_g, -__ldg(args.colexp + pq));
            Vz[v_index(il, p, q, x, args.n_orb)] = v;
            Vz[v_index(il, q, p, x, args.n_orb)] = v;
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

// =================================================================== bf16 x3 engine (step (b))
constexpr int BF_BN = 160;
constexpr int BF_HC = BF_BN / 2;
constexpr int BF_PARTS = 3;
constexpr int BF_A_TILE = VF_BM * 64;             // bytes per part of an A tile (128 rows of 64 B)
constexpr int BF_B_TILE = BF_BN * 64;
constexpr int BF_A_BYTES = BF_PARTS * BF_A_TILE;
constexpr int BF_B_BYTES = BF_PARTS * BF_B_TILE;
constexpr int BF_STAGE = ((BF_A_BYTES + BF_B_BYTES + 1023) / 1024) * 1024;
constexpr int BF_STAGES = 4;
constexpr int BF_MMA_WARPS = 2;                   // issuers of the even / odd ranges
constexpr int BF_THREADS = (1 + BF_MMA_WARPS + DRAIN_WARPS) * 32;
constexpr int BF_SMEM = BF_STAGES * BF_STAGE + 1024 + 256;
static_assert(BF_BN == vf_bn(3), "tile width of the bf16 engine");
static_assert(BF_SMEM <= 232448, "shared memory per CTA");
static_assert(NRB > BF_STAGES, "range barriers");
static_assert(2 * BF_BN <= 512 && BF_BN % 32 == 0, "two accumulators, drain halves of 16-column chunks");

__global__ void __launch_bounds__(BF_THREADS, 1)
    vfield_bf16_kernel(const __grid_constant__ CUtensorMap tm_g, const __grid_constant__ CUtensorMap tm_rho,
                       const VfieldArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + BF_STAGES * BF_STAGE);
  uint64_t* tma_full = bars;                  // [BF_STAGES] the stage's loads landed
  uint64_t* rdone = bars + BF_STAGES;         // [NRB] the MMAs of range r (r % NRB) completed
  uint64_t* d_free = bars + BF_STAGES + NRB;  // [2] the drains released accumulator b
  uint64_t* fin_bar = bars + BF_STAGES + NRB + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + BF_STAGES + NRB + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TileXY t = grouped_tile(blockIdx.x, 3 * args.mt_per_x, args.n_tiles);
  const int x = t.m_tile / args.mt_per_x;
  const int ib = (t.m_tile - x * args.mt_per_x) * VF_BM;
  const int row0 = static_cast<int>(x * args.gcp) + ib;
  const int split = blockIdx.y;
  const int kb0 = split * args.kb_per_split;
  const int kb1 = min(args.n_kb, kb0 + args.kb_per_split);
  const int n_it = kb1 - kb0;
  const int kd = args.kd;
  const int n_ranges = (n_it + kd - 1) / kd;

  if (threadIdx.x == 0) {
    for (int s = 0; s < BF_STAGES; ++s) mbar_init(&tma_full[s], 1);
    for (int r = 0; r < NRB; ++r) mbar_init(&rdone[r], 1);
    for (int b = 0; b < 2; ++b) mbar_init(&d_free[b], DRAIN_WARPS);
    mbar_init(fin_bar, BF_MMA_WARPS);
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
        const int it = kb - kb0, s = it % BF_STAGES;
        if (it >= BF_STAGES) {
          const int need = (it - BF_STAGES) / kd;  // range holding the slot's previous stage
          bool ok = true;
          for (; seen <= need && ok; ++seen)
            ok = mbar_wait(&rdone[seen % NRB], (seen / NRB) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF);
          if (!ok) break;
        }
        mbar_arrive_expect_tx(&tma_full[s], BF_A_BYTES + BF_B_BYTES);
        uint8_t* st = smem + s * BF_STAGE;
        for (int p = 0; p < BF_PARTS; ++p) {
          tma_load_3d(st + p * BF_A_TILE, &tm_g, &tma_full[s], kb * VF_BK, row0, p);
          tma_load_3d(st + BF_A_BYTES + p * BF_B_TILE, &tm_rho, &tma_full[s], kb * VF_BK, t.n_tile * BF_BN, p);
        }
        issued_end = kb + 1;
      }
      int zero = 0;
      for (int kb = max(kb0, issued_end - BF_STAGES); kb < issued_end; ++kb) {
        const int it = kb - kb0;
        mbar_wait(&tma_full[it % BF_STAGES], (it / BF_STAGES) & 1, reinterpret_cast<volatile int*>(&zero), args.err,
                  DEV_ERR_TIMEOUT_VF);
      }
    }
  } else if (warp == 1 || warp == 2 + DRAIN_WARPS) {
    if (lane == 0) {
      // ---------------------------------------------------------------- MMA issuers
      // A range of kd stages goes into one TMEM accumulator: first the cross products of each
      // stage as it lands (the accumulator is still small), then the hi x hi product of every
      // stage; one commit per range.  Warp 1 issues the even ranges (accumulator 0), the last warp
      // the odd ones (accumulator 1).
      constexpr uint32_t idesc = idesc_f16(VF_BM, BF_BN, true);
      constexpr int pa_of[5] = {1, 0, 2, 0, 1};   // (A part, B part) of the products before hi x hi
      constexpr int pb_of[5] = {1, 2, 0, 1, 0};
      bool alive = true;
      for (int r = warp == 1 ? 0 : 1; r < n_ranges && alive; r += BF_MMA_WARPS) {
        const int it0 = r * kd, it1 = min(n_it, it0 + kd);
        const int b = r & 1, u = r >> 1;
        const uint32_t d_tmem = tmem + b * BF_BN;
        if (u >= 1 && !mbar_wait(&d_free[b], (u - 1) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF)) break;
        for (int it = it0; it < it1; ++it) {
          const int s = it % BF_STAGES;
          if (!(alive = mbar_wait(&tma_full[s], (it / BF_STAGES) & 1, abort_flag, args.err, DEV_ERR_TIMEOUT_VF))) break;
          tc_fence_after();
          const uint32_t sa = smem_base + s * BF_STAGE;
          const uint32_t sb = sa + BF_A_BYTES;
#pragma unroll
          for (int p = 0; p < 5; ++p)
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
              tc_mma_f16(d_tmem, sdesc_kmajor_sw64(sa + pa_of[p] * BF_A_TILE + ks * 32),
                         sdesc_kmajor_sw64(sb + pb_of[p] * BF_B_TILE + ks * 32), idesc,
                         (it == it0 && p == 0 && ks == 0) ? 0u : 1u);
        }
        if (!alive) break;
        for (int it = it0; it < it1; ++it) {
          const uint32_t sa = smem_base + (it % BF_STAGES) * BF_STAGE;
          const uint32_t sb = sa + BF_A_BYTES;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks)
            tc_mma_f16(d_tmem, sdesc_kmajor_sw64(sa + ks * 32), sdesc_kmajor_sw64(sb + ks * 32), idesc, 1u);
        }
        tc_commit(&rdone[r % NRB]);
      }
      tc_commit(fin_bar);
      int zero = 0;
      mbar_wait(fin_bar, 0, reinterpret_cast<volatile int*>(&zero), args.err, DEV_ERR_TIMEOUT_VF);
    }
  } else {
    // ------------------------------------------------------------------ range drains and epilogue
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
    const uint32_t c_base = static_cast<uint32_t>(half * BF_HC);
    float S[BF_HC];
#pragma unroll
    for (int k = 0; k < BF_HC; ++k) S[k] = 0.0f;
    int nflush = 0;
    auto flush_sums = [&]() {
      double* acc = args.Vacc + (static_cast<int64_t>(split) * gridDim.x + blockIdx.x) * VF_BM * BF_BN +
                    static_cast<int64_t>(c_base) * VF_BM + quarter * 32 + lane;
      if (nflush == 0) {
#pragma unroll
        for (int k = 0; k < BF_HC; ++k) acc[k * VF_BM] = static_cast<double>(S[k]);
      } else {
#pragma unroll
        for (int k = 0; k < BF_HC; ++k) red_add_f64(acc + k * VF_BM, static_cast<double>(S[k]));
      }
#pragma unroll
      for (int k = 0; k < BF_HC; ++k) S[k] = 0.0f;
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
      const uint32_t src = tmem + lane_base + b * BF_BN + c_base;
#pragma unroll
      for (int c = 0; c < BF_HC; c += 16) {
        uint32_t d0[16];
        tmem_ld_x16(src + c, d0);
        tmem_wait_ld();
#pragma unroll
        for (int k = 0; k < 16; ++k) S[c + k] += __uint_as_float(d0[k]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&d_free[b]);
      if (args.flush > 0 && (r + 1) % args.flush == 0) flush_sums();
    }
    if (args.flush > 0) {
      if (ok && n_ranges % args.flush != 0) flush_sums();
    } else {
      const int row = quarter * 32 + lane;
      const int64_t il = static_cast<int64_t>(ib) + row;
      const int pq0 = t.n_tile * BF_BN + static_cast<int>(c_base);
      if (ok && !*abort_flag && il < args.n_i && n_it > 0) {
        float* Vz = args.V + split * v_slice(args.gcp, args.n_orb);
#pragma unroll
        for (int k = 0; k < BF_HC; ++k) {
          const int pq = pq0 + k;
          if (pq < args.n_pair) {
            const int p = __ldg(args.pair_p + pq), q = __ldg(args.pair_q + pq);
            const float v = ldexpf(S[k] * args.unscale_g, -__ldg(args.colexp + pq));
            Vz[v_index(il, p, q, x, args.n_orb)] = v;
            Vz[v_index(il, q, p, x, args.n_orb)] = v;
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

// =================================================================== finalize kernels
// V from the FP64 accumulator of the GEMM: one CTA per (tile, split), thread = tile row; the tile
// order is the GEMM's grouped order.
template <int BN>
__global__ void __launch_bounds__(VF_BM) vfield_finalize_kernel(const VfieldArgs args) {
  const TileXY t = grouped_tile(blockIdx.x, 3 * args.mt_per_x, args.n_tiles);
  const int x = t.m_tile / args.mt_per_x;
  const int row = threadIdx.x;
  const int64_t il = static_cast<int64_t>(t.m_tile - x * args.mt_per_x) * VF_BM + row;
  if (il >= args.n_i) return;
  const double* acc = args.Vacc + (static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x) * VF_BM * BN + row;
  float* v = args.V + blockIdx.y * v_slice(args.gcp, args.n_orb);
  const int ncol = min(BN, args.n_pair - t.n_tile * BN);
  for (int c = 0; c < ncol; ++c) {
    const int pq = t.n_tile * BN + c;
    const int p = __ldg(args.pair_p + pq), q = __ldg(args.pair_q + pq);
    const float val =
        ldexpf(static_cast<float>(acc[static_cast<int64_t>(c) * VF_BM]) * args.unscale_g, -__ldg(args.colexp + pq));
    v[v_index(il, p, q, x, args.n_orb)] = val;
    v[v_index(il, q, p, x, args.n_orb)] = val;
  }
}

// M[pq][rs] += tile sum * 2^-(exp_a[pq] + exp_b[rs]) for one tile of the step (d) GEMM (mode 1);
// one CTA per tile (each M element is owned by one tile), through shared memory in slabs of 32
// columns: read column-major from the tile sums (thread = row), added row-major into M (warp =
// row, lane = column), both coalesced.
template <int BN>
__global__ void __launch_bounds__(VF_BM) assemble_finalize_kernel(const VfieldArgs args) {
  __shared__ double slab[32][VF_BM + 1];
  const TileXY t = grouped_tile(blockIdx.x, (args.rows_a + VF_BM - 1) / VF_BM, args.n_tiles);
  const double* acc = args.Vacc + (static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x) * VF_BM * BN;
  const int ncol = min(BN, args.n_pair - t.n_tile * BN);
  const int row0 = t.m_tile * VF_BM, col0 = t.n_tile * BN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c0 = 0; c0 < ncol; c0 += 32) {
    for (int c = 0; c < 32; ++c)
      slab[c][threadIdx.x] = c0 + c < ncol ? acc[static_cast<int64_t>(c0 + c) * VF_BM + threadIdx.x] : 0.0;
    __syncthreads();
    const int c = c0 + lane;
    if (c < ncol) {
      const int eb = __ldg(args.exp_b + col0 + c);
      for (int r = warp; r < VF_BM && row0 + r < args.rows_a; r += VF_BM / 32) {
        const int pq = row0 + r;
        const int e = __ldg(args.exp_a + pq) + eb;
        double* m = args.M + static_cast<int64_t>(pq) * args.ldm + col0 + c;
        *m += slab[lane][r] * __longlong_as_double(static_cast<long long>(1023 - e) << 52);
      }
    }
    __syncthreads();
  }
}

int m_tiles_of(const VfieldArgs& a) { return a.mode == 0 ? 3 * a.mt_per_x : (a.rows_a + VF_BM - 1) / VF_BM; }

}  // namespace

bool vfield_tc_supported(int n_nuc) { return n_nuc >= 1 && n_nuc <= 8; }

void launch_vfield_tc(const CUtensorMap* tm_g, const CUtensorMap* tm_rho, const CUtensorMap* tm_rho16,
                      const VfieldArgs& a, int parts, int splits, cudaStream_t st) {
  if (a.n_tiles <= 0 || splits <= 0) return;
  if (a.mode == 1 ? a.rows_a <= 0 : a.mt_per_x <= 0) return;
  dim3 grid(static_cast<unsigned>(m_tiles_of(a) * a.n_tiles), static_cast<unsigned>(splits));
  if (a.mode == 1) {
    cudaFuncSetAttribute(xgemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, xb_smem(1));
    xgemm_kernel<1><<<grid, XB_THREADS, xb_smem(1), st>>>(*tm_g, *tm_rho, *tm_rho16, a);
  } else if (parts == 2) {
    cudaFuncSetAttribute(xgemm_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, xb_smem(0));
    xgemm_kernel<0><<<grid, XB_THREADS, xb_smem(0), st>>>(*tm_g, *tm_rho, *tm_rho16, a);
  } else {
    cudaFuncSetAttribute(vfield_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BF_SMEM);
    vfield_bf16_kernel<<<grid, BF_THREADS, BF_SMEM, st>>>(*tm_g, *tm_rho, a);
  }
}

void launch_vfield_tc_finalize(const VfieldArgs& a, int parts, int splits, cudaStream_t st) {
  if (a.n_tiles <= 0 || splits <= 0 || a.flush <= 0) return;
  if (a.mode == 1 ? a.rows_a <= 0 : a.mt_per_x <= 0) return;
  dim3 grid(static_cast<unsigned>(m_tiles_of(a) * a.n_tiles), static_cast<unsigned>(splits));
  if (a.mode == 1)
    assemble_finalize_kernel<XB_BN><<<grid, VF_BM, 0, st>>>(a);
  else if (parts == 2)
    vfield_finalize_kernel<XB_BN><<<grid, VF_BM, 0, st>>>(a);
  else
    vfield_finalize_kernel<BF_BN><<<grid, VF_BM, 0, st>>>(a);
}

}  // namespace xtc
