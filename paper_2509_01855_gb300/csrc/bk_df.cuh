// Double-float arithmetic for the FP64 transforms: a value is the unevaluated sum hi + lo of two
// binary32 numbers (|lo| <= ulp(hi) / 2), which carries 48 significand bits. On GB300 the FP32
// pipe runs 64 times as many lane operations per clock as the FP64 pipe, so a double-float
// butterfly of ~10 FP32 operations per FP64 operation still takes a fraction of the FP64 pipe's
// time.
//
// Sum: Knuth's TwoSum of the high parts, the low parts added to the error, and a
// renormalisation by Dekker's FastTwoSum (the "sloppy" double-word sum, Joldes, Muller and
// Popescu, ACM TOMS 44(2), 2017, Algorithm 5). Its error is below 2^-46 (|a| + |b|): small against
// the operands, not against the result when they cancel, which is the norm-wise bound an FFT
// needs. Product: TwoProd of the high parts by FMA (the exact error of a binary32 product),
// plus the cross terms, renormalised (Algorithm 11 of the same paper), relative error below
// 5 * 2^-48. The _rn intrinsics keep the compiler from contracting the error-free steps.
//
// Storage: the library's FP64 vectors stay IEEE binary64 in memory (the ABI's BK_F64 layout); a
// double converts to hi = rn(d), lo = rn(d - hi) exactly up to lo's rounding, and back as
// (double) hi + (double) lo. Scratch buffers and tables of a double-float plan hold dfl values
// (8 bytes, like a double).
#pragma once

#include <cuda_runtime.h>

namespace bk {

struct __align__(8) dfl {
  float hi, lo;
  __host__ __device__ constexpr dfl() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr dfl(float f) : hi(f), lo(0.f) {}
  __host__ __device__ constexpr dfl(int i) : dfl((double)i) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return df_fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { a = a + b; return a; }
__device__ __forceinline__ dfl& operator-=(dfl& a, dfl b) { a = a - b; return a; }
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) { a = a * b; return a; }

// Complex double-float (16 bytes, like double2).
struct __align__(16) dfl2 {
  dfl x, y;
};

// Read-only cached load of a complex value (float2, double2, dfl2).
template <typename C> __device__ __forceinline__ C ldg(const C* p) { return __ldg(p); }
template <> __device__ __forceinline__ dfl2 ldg<dfl2>(const dfl2* p) {
  const float4 f = __ldg(reinterpret_cast<const float4*>(p));
  dfl2 r;
  r.x = dfl(f.x, f.y);
  r.y = dfl(f.z, f.w);
  return r;
}

// Type of the caller's real vectors for arithmetic type T: T itself, except that double-float
// arithmetic serves binary64 vectors. Internal buffers (stage vectors between the DCTs) hold T.
template <typename T> struct User { typedef T t; };
template <> struct User<dfl> { typedef double t; };

// binary64 <-> double-float. GB300's FP64 pipe (which also converts between binary64 and
// binary32) runs 2 lane operations per clock per SM, so the conversions work on the bit fields
// with integer operations where the exponents allow it:
//   d2df: hi = x with its significand truncated to 24 bits (exact), lo = the remaining 29 bits,
//         an integer r < 2^29 times 2^(e - 1075), converted to binary32 (one rounding, relative
//         error 2^-24 of lo, i.e. 2^-48 of x) and scaled by that power of two, with x's sign.
//         Zeros, and exponents whose hi or lo would leave the normal binary32 range, take the
//         FP64 route: hi = rn(x), lo = rn(x - hi).
//   df2d: hi and lo widen exactly by moving their fields into binary64 (normal binary32 values;
//         others take the FP64 conversion), then one binary64 addition.
__device__ __forceinline__ dfl d2df(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7ff);
  if ((u << 1) == 0) return dfl(__uint_as_float((unsigned)(u >> 32)), 0.f);   // +-0
  if (e < 1023 - 126 + 53 || e > 1023 + 127) {   // tiny, huge or special: FP64 route
    const float h = __double2float_rn(x);
    return dfl(h, __double2float_rn(x - (double)h));
  }
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const unsigned long long m = u & 0xfffffffffffffull;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(m >> 29));
  const unsigned r = (unsigned)(m & 0x1fffffffu);
  const float scale = __uint_as_float((unsigned)(e - 1075 + 127) << 23);   // 2^(e - 1075), normal here
  const float lo = __fmul_rn(__uint2float_rn(r), scale);
  return dfl(hi, __uint_as_float(__float_as_uint(lo) | sign));
}
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ef = (b >> 23) & 0xff;
  if (ef == 0 || ef == 0xff) return (double)f;   // zero, subnormal, inf, nan
  const unsigned long long db = ((unsigned long long)(b & 0x80000000u) << 32) |
                                ((unsigned long long)(ef - 127 + 1023) << 52) |
                                ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)db);
}
__device__ __forceinline__ double df2d(dfl x) { return f2d_bits(x.hi) + f2d_bits(x.lo); }

// Warp shuffles of the arithmetic types (one per binary32 word for dfl).
__device__ __forceinline__ float shfl_up(float v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_up(double v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ dfl shfl_up(dfl v, int d) {
  return dfl(__shfl_up_sync(0xffffffffu, v.hi, d), __shfl_up_sync(0xffffffffu, v.lo, d));
}
__device__ __forceinline__ float shfl_down(float v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_down(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ dfl shfl_down(dfl v, int d) {
  return dfl(__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d));
}
__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ dfl shfl_xor(dfl v, int o) {
  return dfl(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

}  // namespace bk
