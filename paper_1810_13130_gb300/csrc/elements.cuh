// Device building blocks of the matrix-free element kernels.
//
// An element holds (p+1)^3 nodal values u[c][b][a] (a along x fastest).  Each
// CTA runs E elements side by side, one 2-D thread plane (P1 x P1 threads) per
// element.  In every stage each thread owns one complete 1-D line of the element
// cube (along z, y or x), applies a 1-D operator to it in registers and writes it
// back to shared memory.  With nq = p+1 Gauss points the "nodal -> Gauss point"
// map B is square, so forward (B (x) B (x) B) and backward (B^T (x) B^T (x) B^T)
// passes are three contractions each.
#pragma once

#include <cuda_runtime.h>

#include "df64.cuh"
#include "tdks_internal.h"

namespace tdks {

template <typename T>
struct Cx {
  T re, im;
};

// ---- conversions between double and float without the FP64 pipe ------------
// On GB300 the FP64 unit also executes double<->float conversions at the FP64
// rate; these bit-level versions run on the integer pipe instead.
// double -> float, round to nearest even; |x| below FLT_MIN flushes to signed 0.
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned sign = hw & 0x80000000u;
  const int E = (int)((hw >> 20) & 0x7ffu);
  int ef = E - 1023 + 127;
  if (E == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (((hw & 0xfffffu) | lw) ? 0x400000u : 0u));
  if (ef <= 0) return __uint_as_float(sign);
  unsigned m = ((hw & 0xfffffu) << 3) | (lw >> 29);       // top 23 mantissa bits
  const unsigned rest = lw & 0x1fffffffu;                  // 29 bits below them
  if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) {
    if (++m == 0x800000u) {
      m = 0;
      ++ef;
    }
  }
  if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)ef << 23) | m);
}

// float -> double (exact); float subnormals flush to signed 0.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0) return __longlong_as_double((long long)((unsigned long long)sign << 32));
  unsigned hw;
  if (e == 0xffu)
    hw = sign | 0x7ff00000u | ((u & 0x7fffffu) >> 3) | ((u & 0x7fffffu) ? 0x80000u : 0u);
  else
    hw = sign | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  const unsigned lw = (u & 0x7u) << 29;
  return __longlong_as_double((long long)(((unsigned long long)hw << 32) | lw));
}

template <typename T>
__device__ __forceinline__ void vzero(T& v) { v = T(0); }
__device__ __forceinline__ void vzero(Df& v) { v = Df{0.0f, 0.0f}; }
template <typename T>
__device__ __forceinline__ void vzero(Cx<T>& v) { v.re = T(0); v.im = T(0); }

template <typename T>
__device__ __forceinline__ void madd(T& acc, T c, const T& v) { acc = fma(c, v, acc); }
template <typename T>
__device__ __forceinline__ void madd(Cx<T>& acc, T c, const Cx<T>& v) {
  acc.re = fma(c, v.re, acc.re);
  acc.im = fma(c, v.im, acc.im);
}
template <typename T>
__device__ __forceinline__ T vadd(const T& a, const T& b) { return a + b; }
template <typename T>
__device__ __forceinline__ Cx<T> vadd(const Cx<T>& a, const Cx<T>& b) { return Cx<T>{a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ T vsub(const T& a, const T& b) { return a - b; }
template <typename T>
__device__ __forceinline__ Cx<T> vsub(const Cx<T>& a, const Cx<T>& b) { return Cx<T>{a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ T vscale(T c, const T& v) { return c * v; }

// ---- double-float overloads ------------------------------------------------
__device__ __forceinline__ void vzero(Cx<Df>& v) { v.re = Df{0.0f, 0.0f}; v.im = Df{0.0f, 0.0f}; }
__device__ __forceinline__ Cx<Df> vadd(const Cx<Df>& a, const Cx<Df>& b) {
  return Cx<Df>{df_add(a.re, b.re), df_add(a.im, b.im)};
}
__device__ __forceinline__ Cx<Df> vsub(const Cx<Df>& a, const Cx<Df>& b) {
  return Cx<Df>{df_sub(a.re, b.re), df_sub(a.im, b.im)};
}
__device__ __forceinline__ void madd(Cx<Df>& acc, Df c, const Cx<Df>& v) {
  df_madd(acc.re, c, v.re);
  df_madd(acc.im, c, v.im);
}
__device__ __forceinline__ Cx<Df> vscale(Df c, const Cx<Df>& v) {
  return Cx<Df>{df_mul(c, v.re), df_mul(c, v.im)};
}

// real double-float lines (the split form of the element kernel)
__device__ __forceinline__ Df vadd(const Df& a, const Df& b) { return df_add(a, b); }
__device__ __forceinline__ Df vsub(const Df& a, const Df& b) { return df_sub(a, b); }
__device__ __forceinline__ void madd(Df& acc, Df c, const Df& v) { df_madd(acc, c, v); }
__device__ __forceinline__ Df vscale(Df c, const Df& v) { return df_mul(c, v); }

// scalar conversions used in set-up code (not in the inner loops)
template <typename T>
__device__ __forceinline__ T from_d(double x) { return (T)x; }
template <>
__device__ __forceinline__ Df from_d<Df>(double x) {
  const float h = (float)x;
  return Df{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(Df x) { return (double)x.hi + (double)x.lo; }

// acc += Re(conj(a) b)
template <typename T>
__device__ __forceinline__ void dot_acc(T& acc, const Cx<T>& a, const Cx<T>& b) {
  acc = fma(a.re, b.re, fma(a.im, b.im, acc));
}
__device__ __forceinline__ void dot_acc(Df& acc, const Cx<Df>& a, const Cx<Df>& b) {
  df_madd(acc, a.re, b.re);
  df_madd(acc, a.im, b.im);
}
template <typename T>
__device__ __forceinline__ Cx<T> vscale(T c, const Cx<T>& v) { return Cx<T>{c * v.re, c * v.im}; }
// acc += a b (real lines)
__device__ __forceinline__ void dot_acc(float& acc, const float& a, const float& b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void dot_acc(Df& acc, const Df& a, const Df& b) { df_madd(acc, a, b); }

// out = M in for a centrosymmetric N x N matrix M stored folded (layout in
// tdks_internal.h): pairs (i, N-1-i) of the input are combined into even and odd
// parts e_i = in_i + in_{N-1-i}, o_i = in_i - in_{N-1-i}, so that
//   out_q = a_q + b_q,  out_{N-1-q} = a_q - b_q,  a_q = sum_i Me[q][i] e_i (+ M[q][h] in_h),
//   b_q = sum_i Mo[q][i] o_i,  out_h = sum_i M[h][i] e_i + M[h][h] in_h  (odd N):
// about N^2/2 multiply-adds instead of N^2.
template <int N, typename V, typename T>
__device__ __forceinline__ void cs_apply(const T* __restrict__ t, const V (&in)[N], V (&out)[N]) {
  constexpr int h = N / 2;
  constexpr int hh = h > 0 ? h : 1;
  const T* Me = t;
  const T* Mo = t + h * h;
  const T* Mc = t + 2 * h * h;
  const T* Mr = Mc + h;
  V e[hh], o[hh];
#pragma unroll
  for (int i = 0; i < h; ++i) {
    e[i] = vadd(in[i], in[N - 1 - i]);
    o[i] = vsub(in[i], in[N - 1 - i]);
  }
#pragma unroll
  for (int q = 0; q < h; ++q) {
    V a, b;
    vzero(a);
    vzero(b);
#pragma unroll
    for (int i = 0; i < h; ++i) {
      madd(a, Me[q * h + i], e[i]);
      madd(b, Mo[q * h + i], o[i]);
    }
    if (N & 1) madd(a, Mc[q], in[h]);
    out[q] = vadd(a, b);
    out[N - 1 - q] = vsub(a, b);
  }
  if (N & 1) {
    V c = vscale(Mr[h], in[h]);
#pragma unroll
    for (int i = 0; i < h; ++i) madd(c, Mr[i], e[i]);
    out[h] = c;
  }
}

// Double-float version: each dot product keeps an unnormalized (hi, err) pair --
// hi grows by exact two-sums, the rounding errors and product tails accumulate in
// err -- and is renormalized once, when the output pair is formed.
struct DfAcc {
  float hi, err;
};
__device__ __forceinline__ DfAcc dfa_first(Df c, Df x) {
  const float p = __fmul_rn(c.hi, x.hi);
  float pe = __fmaf_rn(c.hi, x.hi, -p);
  pe = __fmaf_rn(c.hi, x.lo, pe);
  pe = __fmaf_rn(c.lo, x.hi, pe);
  return DfAcc{p, pe};
}
__device__ __forceinline__ void dfa_madd(DfAcc& a, Df c, Df x) {
  const float p = __fmul_rn(c.hi, x.hi);
  float pe = __fmaf_rn(c.hi, x.hi, -p);
  pe = __fmaf_rn(c.hi, x.lo, pe);
  pe = __fmaf_rn(c.lo, x.hi, pe);
  const float s = __fadd_rn(a.hi, p);
  const float v = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(p, v));
  a.err = __fadd_rn(a.err, __fadd_rn(e, pe));
  a.hi = s;
}
// (a + b, a - b) of two accumulators, renormalized
__device__ __forceinline__ void dfa_pm(const DfAcc& a, const DfAcc& b, Df& plus, Df& minus) {
  float s = __fadd_rn(a.hi, b.hi);
  float v = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  plus = df_norm(s, __fadd_rn(e, __fadd_rn(a.err, b.err)));
  s = __fsub_rn(a.hi, b.hi);
  v = __fsub_rn(s, a.hi);
  e = __fsub_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fadd_rn(b.hi, v));
  minus = df_norm(s, __fadd_rn(e, __fsub_rn(a.err, b.err)));
}

template <int N>
__device__ __forceinline__ void cs_apply_df1(const Df* __restrict__ t, const Df (&in)[N], Df (&out)[N]) {
  constexpr int h = N / 2;
  constexpr int hh = h > 0 ? h : 1;
  const Df* Me = t;
  const Df* Mo = t + h * h;
  const Df* Mc = t + 2 * h * h;
  const Df* Mr = Mc + h;
  Df e[hh], o[hh];
#pragma unroll
  for (int i = 0; i < h; ++i) {
    e[i] = df_add(in[i], in[N - 1 - i]);
    o[i] = df_sub(in[i], in[N - 1 - i]);
  }
#pragma unroll
  for (int q = 0; q < h; ++q) {
    DfAcc a = dfa_first(Me[q * h], e[0]);
    DfAcc b = dfa_first(Mo[q * h], o[0]);
#pragma unroll
    for (int i = 1; i < h; ++i) {
      dfa_madd(a, Me[q * h + i], e[i]);
      dfa_madd(b, Mo[q * h + i], o[i]);
    }
    if (N & 1) dfa_madd(a, Mc[q], in[h]);
    dfa_pm(a, b, out[q], out[N - 1 - q]);
  }
  if (N & 1) {
    DfAcc c = dfa_first(Mr[h], in[h]);
#pragma unroll
    for (int i = 0; i < h; ++i) dfa_madd(c, Mr[i], e[i]);
    out[h] = df_norm(c.hi, c.err);
  }
}

// real double-float line
template <int N>
__device__ __forceinline__ void cs_apply(const Df* __restrict__ t, const Df (&in)[N], Df (&out)[N]) {
  if constexpr (N == 1) {
    out[0] = df_mul(t[0], in[0]);
  } else {
    cs_apply_df1<N>(t, in, out);
  }
}

template <int N>
__device__ __forceinline__ void cs_apply(const Df* __restrict__ t, const Cx<Df> (&in)[N],
                                         Cx<Df> (&out)[N]) {
  if constexpr (N == 1) {
    out[0] = vscale(t[0 + 2 * 0 + 0], in[0]);
  } else {
    Df ir[N], ii[N], orr[N], oi[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      ir[i] = in[i].re;
      ii[i] = in[i].im;
    }
    cs_apply_df1<N>(t, ir, orr);
    cs_apply_df1<N>(t, ii, oi);
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = Cx<Df>{orr[i], oi[i]};
  }
}

template <int N, typename V>
__device__ __forceinline__ void load_line(V (&r)[N], const V* src, int stride) {
#pragma unroll
  for (int i = 0; i < N; ++i) r[i] = src[i * stride];
}

template <int N, typename V>
__device__ __forceinline__ void store_line(const V (&r)[N], V* dst, int stride) {
#pragma unroll
  for (int i = 0; i < N; ++i) dst[i * stride] = r[i];
}

// Element of a parity colour: colour bits (cx, cy, cz) select ex = cx + 2 gx etc.
// Elements of one colour share no node, so a launch can read-modify-write its
// nodes without atomics; eight launches cover the mesh in a fixed order.
__device__ __forceinline__ bool color_elem(const Geom& g, int color, long long gidx, int& ex,
                                           int& ey, int& ez) {
  const int cx = color & 1, cy = (color >> 1) & 1, cz = (color >> 2) & 1;
  const int ncx = (g.nx - cx + 1) >> 1, ncy = (g.ny - cy + 1) >> 1, ncz = (g.nz - cz + 1) >> 1;
  const long long tot = (long long)ncx * ncy * ncz;
  if (gidx < 0 || gidx >= tot) return false;
  const int gx = (int)(gidx % ncx);
  const long long r = gidx / ncx;
  const int gy = (int)(r % ncy);
  const int gz = (int)(r / ncy);
  ex = cx + 2 * gx;
  ey = cy + 2 * gy;
  ez = cz + 2 * gz;
  return true;
}

__device__ __forceinline__ bool plain_elem(const Geom& g, long long gidx, int& ex, int& ey,
                                           int& ez) {
  const long long tot = (long long)g.nx * g.ny * g.nz;
  if (gidx < 0 || gidx >= tot) return false;
  ex = (int)(gidx % g.nx);
  const long long r = gidx / g.nx;
  ey = (int)(r % g.ny);
  ez = (int)(r / g.ny);
  return true;
}

// Deterministic block sum (fixed shuffle tree); result valid in thread 0.
// Works for block sizes that are not a multiple of 32: the last warp only
// combines the lanes that exist.  `red` needs one slot per warp.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  const int lane = tid & 31;
  const int wbase = tid & ~31;
  const int nin = (nthr - wbase) < 32 ? (nthr - wbase) : 32;
  const unsigned mask = nin == 32 ? 0xffffffffu : ((1u << nin) - 1u);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double t = __shfl_down_sync(mask, v, off);
    if (lane + off < nin) v += t;
  }
  if (lane == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (tid == 0) {
    const int nw = (nthr + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];
  }
  __syncthreads();
  return s;
}

// double -> contraction type on the integer pipe (float: round to nearest even; Df:
// the 48-bit split of d2df_bits), and back (the Df pair summed in FP64).
template <typename T>
__device__ __forceinline__ T d2t(double x);
template <>
__device__ __forceinline__ float d2t<float>(double x) { return d2f_bits(x); }
template <>
__device__ __forceinline__ Df d2t<Df>(double x) { return d2df_bits(x); }
__device__ __forceinline__ double t2d(float x) { return f2d_bits(x); }
__device__ __forceinline__ double t2d(Df x) { return f2d_bits(x.hi) + f2d_bits(x.lo); }

__device__ __forceinline__ float shfl_down_t(unsigned mask, float v, int off) {
  return __shfl_down_sync(mask, v, off);
}
__device__ __forceinline__ Df shfl_down_t(unsigned mask, Df v, int off) {
  return Df{__shfl_down_sync(mask, v.hi, off), __shfl_down_sync(mask, v.lo, off)};
}
__device__ __forceinline__ float add_t(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ Df add_t(Df a, Df b) { return df_add(a, b); }

// Block sum in float or double-float (the FP32 pipe), same fixed tree as block_sum;
// result valid in thread 0.  `red` needs one T per warp.
template <typename T>
__device__ __forceinline__ T block_sum_t(T v, T* red) {
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  const int lane = tid & 31;
  const int wbase = tid & ~31;
  const int nin = (nthr - wbase) < 32 ? (nthr - wbase) : 32;
  const unsigned mask = nin == 32 ? 0xffffffffu : ((1u << nin) - 1u);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const T t = shfl_down_t(mask, v, off);
    if (lane + off < nin) v = add_t(v, t);
  }
  if (lane == 0) red[tid >> 5] = v;
  __syncthreads();
  T s = red[0];
  if (tid == 0) {
    const int nw = (nthr + 31) >> 5;
    for (int i = 1; i < nw; ++i) s = add_t(s, red[i]);
  }
  __syncthreads();
  return s;
}

}  // namespace tdks
