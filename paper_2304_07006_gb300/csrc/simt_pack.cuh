// Device helpers shared by the SIMT producers: packed FP32 pair arithmetic, the fp16 / bf16 splits
// of an FP32 value (plain and block-exact), and vector shared-memory access.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace xtc {

// Two FP32 values are split into hi + lo fp16 parts (2 parts) or hi + mid + lo bf16 parts (3
// parts); out[p] holds part p of both values as one packed 32-bit word (a in the low half).
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
// ------------------------------------------------------------------ reciprocals
// 1/sqrt(x) and 1/x by the hardware approximation (relative error about 2^-23) followed by one
// Newton-Raphson step, y' = y + y (1 - x y^2) / 2 and y' = y + y (1 - x y): the step squares the
// approximation's error, so what remains is the rounding of the last fused multiply-add, about
// half an ulp and without the approximation's systematic part.  x must be a positive normal value.
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
__device__ __forceinline__ float rsqrt_nr(float x) {
  const float y = rsqrt_approx(x);
  const float e = fmaf(-x * y, y, 1.0f);
  return fmaf(0.5f * y, e, y);
}
__device__ __forceinline__ float rcp_nr(float x) {
  const float y = rcp_approx(x);
  return fmaf(y, fmaf(-x, y, 1.0f), y);
}
// The same for two values at once (packed FP32 pairs).
__device__ __forceinline__ f32x2 rsqrt_nr2(float xa, float xb) {
  const f32x2 y = pk2(rsqrt_approx(xa), rsqrt_approx(xb));
  const f32x2 e = fma2(mul2(pk2(-xa, -xb), y), y, pk2(1.0f, 1.0f));
  return fma2(mul2(pk2(0.5f, 0.5f), y), e, y);
}
__device__ __forceinline__ f32x2 rcp_nr2(float xa, float xb) {
  const f32x2 y = pk2(rcp_approx(xa), rcp_approx(xb));
  return fma2(y, fma2(pk2(-xa, -xb), y, pk2(1.0f, 1.0f)), y);
}

// ------------------------------------------------------------------ exact fp16 split
// The fp16 operands of the tensor-core GEMMs are split as x = hi + lo with
//     hi = k * 2^q,  k = rint(x / 2^q),  lo = fp16(x - hi),
// where 2^q is a quantum shared by every value of a row over one accumulation range of the GEMM
// (a run of K values), chosen so that |x| < 2^(q + bits): hi is an integer |k| <= 2^bits times the
// quantum, held exactly in fp16 (bits <= 11), and lo carries the remainder (|x - hi| <= 2^(q-1)) to
// fp16 precision.  A product hi_a * hi_b is then an integer below 2^(bits_a + bits_b) times
// 2^(qa + qb), and the products of a range of K values sum exactly in FP32 as long as
// K * 2^(bits_a + bits_b) <= 2^24, whatever rounding the tensor core's FP32 accumulator applies.
// Quanta below fp16's smallest step 2^-24 put everything into lo.  Inputs stay below 2^15.

// Quantum exponent q for a row range whose largest magnitude is m (a normal value or 0), with hi
// parts of `bits` bits: every |x| <= m is below 2^(q + bits).
__device__ __forceinline__ int exact_quantum(float m, int bits) {
  const int eb = (__float_as_int(m) >> 23) & 0xff;  // m in [2^(eb-127), 2^(eb-126)) for normal m
  return eb - 126 - bits;                            // 0 and subnormal m give q < -24: hi = 0
}
__device__ __forceinline__ int exact_quantum(double m, int bits) {
  const int eb = static_cast<int>((__double_as_longlong(m) >> 52) & 0x7ff);
  return eb - 1022 - bits;
}
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }  // -126 <= e <= 127

// hi and lo fp16 parts of x in a block of quantum exponent q.
__device__ __forceinline__ void split_exact(float x, int q, __half& hi, __half& lo) {
  float h = 0.0f;
  if (q >= -24) h = rintf(x * pow2f(-q)) * pow2f(q);  // both products are exact (powers of 2)
  hi = __float2half_rn(h);                              // exact: at most 11 significant bits
  lo = __float2half_rn(x - h);                          // x - h is exact in FP32
}
__device__ __forceinline__ void split_exact(double x, int q, __half& hi, __half& lo) {
  double h = 0.0;
  if (q >= -24) h = rint(x * __longlong_as_double(static_cast<long long>(1023 - q) << 52)) *
                    __longlong_as_double(static_cast<long long>(1023 + q) << 52);
  hi = __double2half(h);
  lo = __double2half(x - h);                            // one rounding, from FP64
}
// Two values of one range, packed as in split_pair: out[0] = hi parts, out[1] = lo parts.  hi is
// rounded to a multiple of 2^q (nearest, ties to even) by adding and subtracting 1.5 * 2^(q + 23):
// the sum then lies in [2^(q+23), 2^(q+24)), where the FP32 spacing is 2^q (here |x| < 2^(q+11)),
// so two round-to-nearest adds give exactly the rounded value, two values per packed instruction.
__device__ __forceinline__ void split_pair_exact(float a, float b, int q, uint32_t* out) {
  const f32x2 x = pk2(a, b);
  f32x2 h = pk2(0.0f, 0.0f);
  if (q >= -24) {
    const float m = 1.5f * pow2f(q + 23);
    const f32x2 mm = pk2(m, m);
    h = sub2(add2(x, mm), mm);
  }
  const f32x2 l = sub2(x, h);  // exact
  float h0, h1, l0, l1;
  up2(h, h0, h1);
  up2(l, l0, l1);
  const __half2 hh = __floats2half2_rn(h0, h1);   // exact: at most 11 significant bits
  const __half2 ll = __floats2half2_rn(l0, l1);
  out[0] = *reinterpret_cast<const uint32_t*>(&hh);
  out[1] = *reinterpret_cast<const uint32_t*>(&ll);
}

__device__ __forceinline__ void ld_shared_v4(uint32_t addr, uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) {
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(a), "=r"(b), "=r"(c), "=r"(d) : "r"(addr) : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// 16 bytes of global memory that every lane of the warp reads at the same address (read-only path).
__device__ __forceinline__ void ldg_2x64(const float* p, f32x2& a, f32x2& b) {
  asm("ld.global.nc.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
}
__device__ __forceinline__ float4 ldg_f4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}

}  // namespace xtc
