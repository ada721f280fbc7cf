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

// binary64 <-> double-float (one rounding each way; the FP64 pipe does the subtraction and the
// conversions, so these run once per element, in the first and the last kernel of a product)
__device__ __forceinline__ dfl d2df(double x) {
  const float h = __double2float_rn(x);
  return dfl(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df2d(dfl x) { return (double)x.hi + (double)x.lo; }

// Warp shuffles of the arithmetic types (one per binary32 word for dfl).
__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ dfl shfl_xor(dfl v, int o) {
  return dfl(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

}  // namespace bk
