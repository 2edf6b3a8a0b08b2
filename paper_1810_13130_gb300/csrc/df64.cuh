// Double-float ("DF64") arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, about 48 significant bits, computed entirely on
// the FP32 pipe.  On GB300 the FP32 pipe is ~58x faster than the FP64 pipe, so
// the contraction kernels run in DF64 to give FP64-level results (relative error
// ~1e-14) much faster than native FP64.
//
// Building blocks (error-free transformations):
//   two-sum (Knuth):  s = fl(a + b), e = (a - (s - v)) + (b - v) with v = s - a;
//                     then a + b = s + e exactly.
//   two-product:      p = fl(a b), e = fma(a, b, -p); then a b = p + e exactly.
// The __f*_rn intrinsics are never contracted into FMAs by the compiler, which
// would break the exactness of these sequences.
#pragma once

#include <cuda_runtime.h>

namespace tdks {

struct Df {
  float hi, lo;
};

__device__ __forceinline__ Df df_make(float h) { return Df{h, 0.0f}; }

// renormalize s + e into (hi, lo) (fast two-sum, |s| >= |e|)
__device__ __forceinline__ Df df_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return Df{h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ Df df_add(Df a, Df b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_norm(s, e);
}

__device__ __forceinline__ Df df_neg(Df a) { return Df{-a.hi, -a.lo}; }

__device__ __forceinline__ Df df_sub(Df a, Df b) { return df_add(a, df_neg(b)); }

// c * x (the lo * lo term, below 2^-48 relative, is dropped)
__device__ __forceinline__ Df df_mul(Df c, Df x) {
  const float p = __fmul_rn(c.hi, x.hi);
  float e = __fmaf_rn(c.hi, x.hi, -p);
  e = __fmaf_rn(c.hi, x.lo, e);
  e = __fmaf_rn(c.lo, x.hi, e);
  return df_norm(p, e);
}

// acc += c * x
__device__ __forceinline__ void df_madd(Df& acc, Df c, Df x) {
  const float p = __fmul_rn(c.hi, x.hi);
  float pe = __fmaf_rn(c.hi, x.hi, -p);
  pe = __fmaf_rn(c.hi, x.lo, pe);
  pe = __fmaf_rn(c.lo, x.hi, pe);
  const float s = __fadd_rn(acc.hi, p);
  const float v = __fsub_rn(s, acc.hi);
  float e = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, v)), __fsub_rn(p, v));
  e = __fadd_rn(e, __fadd_rn(acc.lo, pe));
  acc = df_norm(s, e);
}

// double -> Df on the integer pipe: hi = the double truncated to 24 significant
// bits, lo = the next 24 bits (rounded); the remaining 5 bits (2^-48 relative)
// are dropped.  Values below 2^-126 flush to 0; the lo part flushes when it
// would be subnormal.
__device__ __forceinline__ Df d2df_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned sign = hw & 0x80000000u;
  const int E = (int)((hw >> 20) & 0x7ffu);
  const int ef = E - 1023 + 127;
  if (ef <= 0) return Df{__uint_as_float(sign), 0.0f};
  if (ef >= 255) return Df{__uint_as_float(sign | 0x7f800000u), 0.0f};
  const unsigned m23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
  const float fhi = __uint_as_float(sign | ((unsigned)ef << 23) | m23);
  const unsigned R = lw & 0x1fffffffu;             // remainder, units of 2^(E-1075)
  const int k = E - 1075;                           // exponent of those units
  float flo = 0.0f;
  if (R != 0u && k >= -126 - 0) {
    const float scale = __uint_as_float((unsigned)(k + 127) << 23);
    flo = __fmul_rn(__uint2float_rn(R), scale);
  } else if (R != 0u && k >= -126 - 29) {
    // R < 2^29: scale in two exact steps so no intermediate is subnormal
    const float s1 = __uint_as_float((unsigned)(k + 29 + 127) << 23);
    flo = __fmul_rn(__fmul_rn(__uint2float_rn(R), 1.0f / 536870912.0f), s1);
  }
  if (sign) flo = -flo;
  return Df{fhi, flo};
}

}  // namespace tdks
