// Step (a) for the tensor-core path: the Jastrow gradient G_x(i, j) = d/dx_i u(r_i, r_j) of every
// (outer point i, inner point j) pair of a chunk (section "Decomposition of two-body correction",
// the factor that multiplies rho in V), split into fp16 (2 parts) or bf16 (3 parts) and stored
// K-major as the A operand of the step (b) GEMM, row x * gcp + il (il = i - i0):
//     fp16: G[row][j / 32][part][j % 32]  (both parts of a 32-point block in one 128-byte row,
//           128-byte swizzle tiles, so that one TMA row request moves 128 bytes);
//     bf16: G[part][row][j]               (one plane per part, 64-byte swizzle tiles).
// Computing G once per chunk, instead of inside every orbital-pair tile of the GEMM, removes the
// gradient from the GEMM's critical path; the table costs one HBM write and is then read through L2
// by the GEMM's tiles.
//
// One warp owns a unit of 32 outer points (one per lane, its per-point coefficients in registers)
// and a run of inner-point blocks of 32.  For each block it evaluates the gradient in FP32 (two
// inner points per packed FP32 instruction for up to two Jastrow centres; reciprocal square roots
// and reciprocals refined by a Newton-Raphson step, so that no one-signed error of the hardware
// approximations enters the gradient), splits
// it, writes the tiles of the three components (32 rows x 128 bytes, or 3 parts x 32 rows x 64
// bytes) into shared memory in their swizzle (conflict-free 16-byte stores) and one lane stores
// them with TMA.  The fp16 split is exact on a per-range quantum (simt_pack.cuh): for every row and
// accumulation range of the GEMM (RB blocks of 32 inner points), hi = an integer of at most 9
// bits times the range's quantum, lo = the fp16 remainder.  The lane first stages its RB x 32
// FP32 values per component in its own tile rows, then splits them with the quantum of their
// maximum; a warp then holds RB blocks of tiles, and a CTA GF_WARPS / RB warps.
// The gradient is taken with the pair formula of jastrow_coef.cuh: per-point coefficients times
// polynomials in b = r12 / (1 + r12) and a_jI = |r_j - R_I| / (1 + |r_j - R_I|).
#include "jastrow_coef.cuh"
#include "ptx_sm100.cuh"
#include "simt_pack.cuh"
#include "xtc_internal.cuh"

namespace xtc {
namespace {

constexpr int GF_WARPS = 8;
constexpr int GF_THREADS = GF_WARPS * 32;
constexpr int GF_TILE = 32 * 64;   // one part's share of a component tile: 32 rows of 64 bytes
// fp16: bits of the integer hi part of G on its range's quantum (|k| <= 2^9, exact in fp16)
constexpr int GF_EXACT_BITS = GEMM_BITS_A;

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, uint32_t src, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(src), "r"(c0), "r"(c1), "r"(c2)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Waits until the shared memory of every committed bulk store has been read.
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// Waits until every committed bulk store has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int PARTS, int NNUC, int RB>
__global__ void __launch_bounds__(GF_THREADS)
    gfield_kernel(const __grid_constant__ CUtensorMap tm_g, const GfieldArgs args) {
  constexpr bool BF16 = PARTS == 3;
  constexpr int JS = NNUC <= 4 ? 12 : 16;  // floats per inner point in the table (launch_jtab)
  constexpr int BLOCK_BYTES = 3 * PARTS * GF_TILE;  // the three component tiles of one block
  constexpr int WARP_BYTES = RB * BLOCK_BYTES;       // RB blocks: one exact range of the GEMM
  constexpr int WARPS = GF_WARPS / RB;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t unit = static_cast<int64_t>(blockIdx.x) * WARPS + warp;
  if (unit >= static_cast<int64_t>(args.n_tiles) * args.n_seg) return;  // whole warp; no block barrier below
  const int tile = static_cast<int>(unit / args.n_seg), seg = static_cast<int>(unit % args.n_seg);
  const int kb0 = seg * args.kb_per_seg, kb1 = min(args.n_kb, kb0 + args.kb_per_seg);
  const uint32_t buf = smem_u32(smem) + warp * WARP_BYTES;

  // coefficients of this lane's outer point (rows past the chunk repeat its last point)
  const int64_t il = static_cast<int64_t>(tile) * 32 + lane;
  const int64_t ig = args.i0 + (il < args.n_i ? il : args.n_i - 1);
  float pc[PT_COEF];
  float nc[NNUC * NUC_COEF];
  const double gx = args.grid[3 * ig], gy = args.grid[3 * ig + 1], gz = args.grid[3 * ig + 2];
  point_coefs_fixed<float, NNUC>(*args.jp, gx, gy, gz, static_cast<double>(args.g_scale), pc, nc);
  // low parts of the outer coordinates (the pair difference is taken in hi/lo FP32)
  const float xl = static_cast<float>(gx - static_cast<double>(pc[0]));
  const float yl = static_cast<float>(gy - static_cast<double>(pc[1]));
  const float zl = static_cast<float>(gz - static_cast<double>(pc[2]));
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
  const int row0 = tile * 32;
  float gmax[3] = {0.0f, 0.0f, 0.0f};  // fp16: largest |G| of the range per component

  for (int kr = kb0; kr < kb1; kr += RB) {
#pragma unroll 1
  for (int rb = 0; rb < RB; ++rb) {
    const int kb = kr + rb;
    const uint32_t bbuf = buf + rb * BLOCK_BYTES;
    // 16 records of two inner points each (the pair-interleaved table written by launch_jtab)
    const float* blk = args.jtab + static_cast<int64_t>(kb) * VF_BK * JS;
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
      float gv[3][8];
#pragma unroll
      for (int v2 = 0; v2 < 4; ++v2) {
        const float* rec = blk + (c * 4 + v2) * 2 * JS;  // inner points 8c + 2 v2 and + 1
        if constexpr (NNUC <= 2) {
          f32x2 xh, yh, zh, xlo, ylo, zlo, a0, a1;
          ldg_2x64(rec, xh, yh);
          ldg_2x64(rec + 4, zh, xlo);
          ldg_2x64(rec + 8, ylo, zlo);
          ldg_2x64(rec + 12, a0, a1);
          const f32x2 dx = add2(sub2(PC[0], xh), sub2(XL, xlo));
          const f32x2 dy = add2(sub2(PC[1], yh), sub2(YL, ylo));
          const f32x2 dz = add2(sub2(PC[2], zh), sub2(ZL, zlo));
          const f32x2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
          float r2a, r2b;
          up2(r2, r2a, r2b);
          // unit vector of r1 - r2 taken as zero below 1e-14 bohr (coincident points)
          f32x2 rinv = rsqrt_nr2(fmaxf(r2a, 1e-28f), fmaxf(r2b, 1e-28f));
          {
            float ia, ib;
            up2(rinv, ia, ib);
            rinv = pk2(r2a > 1e-28f ? ia : 0.0f, r2b > 1e-28f ? ib : 0.0f);
          }
          const f32x2 rr = mul2(r2, rinv);
          float ra, rb;
          up2(rr, ra, rb);
          const f32x2 q = rcp_nr2(1.0f + ra, 1.0f + rb);
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
          const float4 q0 = ldg_f4(rec), q1 = ldg_f4(rec + 4), q2 = ldg_f4(rec + 8);
          float2 ap[NNUC];  // a_jI of both points
#pragma unroll
          for (int I = 0; I < NNUC; ++I) ap[I] = __ldg(reinterpret_cast<const float2*>(rec + 12 + 2 * I));
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float xh = h ? q0.y : q0.x, yh = h ? q0.w : q0.z, zh = h ? q1.y : q1.x;
            const float xlo = h ? q1.w : q1.z, ylo = h ? q2.y : q2.x, zlo = h ? q2.w : q2.z;
            const float dx = (pc[0] - xh) + (xl - xlo);
            const float dy = (pc[1] - yh) + (yl - ylo);
            const float dz = (pc[2] - zh) + (zl - zlo);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float rinv = r2 > 1e-28f ? rsqrt_nr(r2) : 0.0f;
            const float rr = r2 * rinv;
            const float q = rcp_nr(1.0f + rr);
            const float b = rr * q;
            const float sfac = q * q * rinv;
            float ex = fmaf(b, fmaf(b, pc[9], pc[6]), pc[3]);
            float ey = fmaf(b, fmaf(b, pc[10], pc[7]), pc[4]);
            float ez = fmaf(b, fmaf(b, pc[11], pc[8]), pc[5]);
            float h1 = pc[12], h2 = pc[13];
#pragma unroll
            for (int I = 0; I < NNUC; ++I) {
              const float* cf = nc + I * NUC_COEF;
              const float a = h ? ap[I].y : ap[I].x;
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
      // the previous range's tiles must have been read by their TMA stores before they are overwritten
      if (c == 0 && rb == 0 && kr > kb0) {
        if (lane == 0) bulk_wait_read_all();
        __syncwarp();
      }
      if constexpr (PARTS == 2) {
        // FP32 staging in the lane's own 128-byte rows of the block's component tiles (16-byte
        // chunks b, b + 1 with b = 0, 4, 2, 6 for c = 0..3, so that the split below rewrites, for
        // each half of the block, exactly the chunks it has read), and the range maxima
        const int b = (c & 1) * 4 + (c >> 1) * 2;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
#pragma unroll
          for (int k = 0; k < 8; ++k) gmax[x] = fmaxf(gmax[x], fabsf(gv[x][k]));
          const uint32_t row = bbuf + x * 2 * GF_TILE;
          st_shared_v4(row + sw128_offset(lane, b), __float_as_uint(gv[x][0]), __float_as_uint(gv[x][1]),
                       __float_as_uint(gv[x][2]), __float_as_uint(gv[x][3]));
          st_shared_v4(row + sw128_offset(lane, b + 1), __float_as_uint(gv[x][4]), __float_as_uint(gv[x][5]),
                       __float_as_uint(gv[x][6]), __float_as_uint(gv[x][7]));
        }
      } else {
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          uint32_t w[4][PARTS];
#pragma unroll
          for (int h = 0; h < 4; ++h) split_pair<BF16>(gv[x][2 * h], gv[x][2 * h + 1], w[h]);
#pragma unroll
          for (int p = 0; p < PARTS; ++p)
            st_shared_v4(bbuf + (x * PARTS + p) * GF_TILE + sw64_offset(lane, c), w[0][p], w[1][p], w[2][p], w[3][p]);
        }
      }
    }
  }
    if constexpr (PARTS == 2) {
      // exact split of the lane's RB x 32 values per component on the range's quantum: hi of
      // points 8c .. 8c + 7 of a block goes to chunk c, lo to chunk 4 + c (component tile x of 32
      // rows x 128 bytes, the layout the GEMM loads)
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const int q = exact_quantum(gmax[x], GF_EXACT_BITS);
        gmax[x] = 0.0f;
#pragma unroll
        for (int rb = 0; rb < RB; ++rb) {
          const uint32_t row = buf + rb * BLOCK_BYTES + x * 2 * GF_TILE;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            // sub-blocks c = 2h (staged in chunks 2h, 2h + 1) and 2h + 1 (chunks 4 + 2h, 5 + 2h)
            uint32_t f[16];
            ld_shared_v4(row + sw128_offset(lane, 2 * h), f[0], f[1], f[2], f[3]);
            ld_shared_v4(row + sw128_offset(lane, 2 * h + 1), f[4], f[5], f[6], f[7]);
            ld_shared_v4(row + sw128_offset(lane, 4 + 2 * h), f[8], f[9], f[10], f[11]);
            ld_shared_v4(row + sw128_offset(lane, 5 + 2 * h), f[12], f[13], f[14], f[15]);
            uint32_t w[8][2];
#pragma unroll
            for (int k = 0; k < 8; ++k)
              split_pair_exact(__uint_as_float(f[2 * k]), __uint_as_float(f[2 * k + 1]), q, w[k]);
            st_shared_v4(row + sw128_offset(lane, 2 * h), w[0][0], w[1][0], w[2][0], w[3][0]);
            st_shared_v4(row + sw128_offset(lane, 2 * h + 1), w[4][0], w[5][0], w[6][0], w[7][0]);
            st_shared_v4(row + sw128_offset(lane, 4 + 2 * h), w[0][1], w[1][1], w[2][1], w[3][1]);
            st_shared_v4(row + sw128_offset(lane, 5 + 2 * h), w[4][1], w[5][1], w[6][1], w[7][1]);
          }
        }
      }
    }
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
#pragma unroll
      for (int rb = 0; rb < RB; ++rb) {
        const int kb = kr + rb;
        const uint32_t bbuf = buf + rb * BLOCK_BYTES;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          if (PARTS == 2) {
            tma_store_3d(&tm_g, bbuf + x * 2 * GF_TILE, kb * 2 * VF_BK, static_cast<int>(x * args.gcp) + row0, 0);
          } else {
#pragma unroll
            for (int p = 0; p < PARTS; ++p)
              tma_store_3d(&tm_g, bbuf + (x * PARTS + p) * GF_TILE, kb * VF_BK, static_cast<int>(x * args.gcp) + row0,
                           p);
          }
        }
      }
      bulk_commit();
    }
  }
  if (lane == 0) bulk_wait_all();
  __syncwarp();
}

template <int PARTS, int NNUC, int RB>
void launch_rb(const CUtensorMap* tm, const GfieldArgs& a, cudaStream_t st) {
  auto kern = gfield_kernel<PARTS, NNUC, RB>;
  constexpr int warps = GF_WARPS / RB;
  constexpr int smem = GF_WARPS * 3 * PARTS * GF_TILE + 1024;  // warps x RB blocks of three tiles
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int64_t units = static_cast<int64_t>(a.n_tiles) * a.n_seg;
  const unsigned blocks = static_cast<unsigned>((units + warps - 1) / warps);
  kern<<<blocks, warps * 32, smem, st>>>(*tm, a);
}
template <int PARTS, int NNUC>
void launch_t(const CUtensorMap* tm, const GfieldArgs& a, cudaStream_t st) {
  if (PARTS == 2 && a.range_blocks == 4)
    launch_rb<PARTS, NNUC, 4>(tm, a, st);
  else if (PARTS == 2 && a.range_blocks == 2)
    launch_rb<PARTS, NNUC, 2>(tm, a, st);
  else
    launch_rb<PARTS, NNUC, 1>(tm, a, st);
}

}  // namespace

void launch_gfield(const CUtensorMap* tm_g_store, const GfieldArgs& a, int parts, cudaStream_t st) {
  if (a.n_tiles <= 0 || a.n_seg <= 0) return;
  if (parts == 2) {
    switch (a.n_nuc) {
      case 1: launch_t<2, 1>(tm_g_store, a, st); break;
      case 2: launch_t<2, 2>(tm_g_store, a, st); break;
      case 3: launch_t<2, 3>(tm_g_store, a, st); break;
      case 4: launch_t<2, 4>(tm_g_store, a, st); break;
      default: launch_t<2, 8>(tm_g_store, a, st); break;  // 5..8 nuclei
    }
  } else {
    switch (a.n_nuc) {
      case 1: launch_t<3, 1>(tm_g_store, a, st); break;
      case 2: launch_t<3, 2>(tm_g_store, a, st); break;
      case 3: launch_t<3, 3>(tm_g_store, a, st); break;
      case 4: launch_t<3, 4>(tm_g_store, a, st); break;
      default: launch_t<3, 8>(tm_g_store, a, st); break;  // 5..8 nuclei
    }
  }
}

}  // namespace xtc
