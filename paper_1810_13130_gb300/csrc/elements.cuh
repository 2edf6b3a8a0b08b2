// Device building blocks of the matrix-free element kernels.
//
// An element holds (p+1)^3 nodal values u[c][b][a] (a along x fastest).  Each
// CTA runs E elements side by side, one 2-D thread plane (P1 x P1 threads) per
// element: thread (ta, tb) owns the z-column of values at (a = ta, b = tb) in
// registers.  A 1-D contraction along z is done in registers; along y and x the
// plane goes through shared memory.  With nq = p+1 Gauss points the "nodal ->
// Gauss point" map B is square, so forward (B (x) B (x) B) and backward
// (B^T (x) B^T (x) B^T) passes are three contractions each.
#pragma once

#include <cuda_runtime.h>

#include "tdks_internal.h"

namespace tdks {

template <typename T>
struct Cx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ void vzero(T& v) { v = T(0); }
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
__device__ __forceinline__ T vscale(T c, const T& v) { return c * v; }
template <typename T>
__device__ __forceinline__ Cx<T> vscale(T c, const Cx<T>& v) { return Cx<T>{c * v.re, c * v.im}; }

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

// Forward pass: column u[c] (registers) -> values at the Gauss points,
// returned as the z-column uq[qz] of thread (qx = ta, qy = tb).
template <int P1, typename V, typename T>
__device__ __forceinline__ void forward3(const V (&u)[P1], V (&uq)[P1], V* S1, V* S2,
                                         const T* sB, int ta, int tb) {
  constexpr int P2 = P1 * P1;
  V t[P1];
#pragma unroll
  for (int q = 0; q < P1; ++q) vzero(t[q]);
#pragma unroll
  for (int c = 0; c < P1; ++c)
#pragma unroll
    for (int q = 0; q < P1; ++q) madd(t[q], sB[q * P1 + c], u[c]);
#pragma unroll
  for (int q = 0; q < P1; ++q) S1[q * P2 + tb * P1 + ta] = t[q];
  __syncthreads();
  // y: thread (a = ta, qy = tb)
#pragma unroll
  for (int qz = 0; qz < P1; ++qz) {
    V acc;
    vzero(acc);
#pragma unroll
    for (int b = 0; b < P1; ++b) madd(acc, sB[tb * P1 + b], S1[qz * P2 + b * P1 + ta]);
    S2[qz * P2 + tb * P1 + ta] = acc;
  }
  __syncthreads();
  // x: thread (qx = ta, qy = tb)
#pragma unroll
  for (int qz = 0; qz < P1; ++qz) {
    V acc;
    vzero(acc);
#pragma unroll
    for (int a = 0; a < P1; ++a) madd(acc, sB[ta * P1 + a], S2[qz * P2 + tb * P1 + a]);
    uq[qz] = acc;
  }
}

// Backward pass: z-column r[qz] of thread (qx = ta, qy = tb) at the Gauss points
// -> nodal column y[c] of thread (a = ta, b = tb), y = (B^T (x) B^T (x) B^T) r.
// Starts with a barrier so that S1/S2 may still be in use on entry.
template <int P1, typename V, typename T>
__device__ __forceinline__ void backward3(const V (&r)[P1], V (&y)[P1], V* S1, V* S2,
                                          const T* sB, int ta, int tb) {
  constexpr int P2 = P1 * P1;
  V t[P1];
#pragma unroll
  for (int c = 0; c < P1; ++c) vzero(t[c]);
#pragma unroll
  for (int q = 0; q < P1; ++q)
#pragma unroll
    for (int c = 0; c < P1; ++c) madd(t[c], sB[q * P1 + c], r[q]);
  __syncthreads();
#pragma unroll
  for (int c = 0; c < P1; ++c) S1[c * P2 + tb * P1 + ta] = t[c];
  __syncthreads();
  // y: thread (qx = ta, b = tb)
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    V acc;
    vzero(acc);
#pragma unroll
    for (int q = 0; q < P1; ++q) madd(acc, sB[q * P1 + tb], S1[c * P2 + q * P1 + ta]);
    S2[c * P2 + tb * P1 + ta] = acc;
  }
  __syncthreads();
  // x: thread (a = ta, b = tb)
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    V acc;
    vzero(acc);
#pragma unroll
    for (int q = 0; q < P1; ++q) madd(acc, sB[q * P1 + ta], S2[c * P2 + tb * P1 + q]);
    y[c] = acc;
  }
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

}  // namespace tdks
