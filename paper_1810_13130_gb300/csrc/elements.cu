// Matrix-free element kernels on the tensor-product hexahedral mesh.
//
// Hbar psibar (Eqs. 15, 21).  On the affine element [hx, hy, hz] the form
//   1/2 int grad N_j . grad N_k + int V N_j N_k
// integrated with the tensor Gauss rule (nq = p+1 points per axis, Sec. VI.A) is
//   (B^T)^(x)3 [ cx Kq_x W_y W_z + cy W_x Kq_y W_z + cz W_x W_y Kq_z + J W^(x)3 V ] B^(x)3
// with B the GLL-Lagrange values at the Gauss points, W = diag(omega),
// Kq = Dg^T W Dg the 1-D stiffness in the Gauss-point Lagrange basis,
// J = hx hy hz / 8 and cx = hy hz / (4 hx) (the 1/2 included), etc.  Per element
// and real component this is 9 one-dimensional contractions of (p+1)^4
// multiply-adds: 3 forward, 3 for the kinetic operator at the Gauss points, 3
// backward.  The Loewdin scale M^-1/2 (diagonal, product of 1-D factors) is
// applied on load and on store.
//
// The Poisson stiffness K (Eq. 19) is applied in nodal form with the 1-D
// matrices K1 = D^T W D and Mg = B^T W B:
//   K = cx' K1 (x) Mg (x) Mg + cy' Mg (x) K1 (x) Mg + cz' Mg (x) Mg (x) K1,
// cx' = hy hz / (2 hx), factored as Mg_x (cy' K1_y Mg_z + cz' Mg_y K1_z) + cx' K1_x Mg_y Mg_z:
// 7 contractions per element.
//
// Assembly: elements are processed in 8 parity colours (one launch each); two
// elements of one colour never share a node, so the scatter is a plain
// read-modify-write and the summation order is fixed (deterministic results).
#include <cuda_bf16.h>

#include <cstdio>
#include <type_traits>

#include "elements.cuh"

using namespace tdks;

namespace {

template <int P1>
struct Cfg {
  static constexpr int P2 = P1 * P1;
  static constexpr int P3 = P2 * P1;
  static constexpr int E = (256 / P2) < 1 ? 1 : (256 / P2);   // elements per CTA
};

// Byte offset of the cp.async prefetch buffer (16-byte entries) in dynamic shared
// memory: the end of the element lines rounded up to 16 bytes.  With float lines
// that end is only 8-byte aligned for odd P1 (E * 2 * P1^3 * 4 bytes).
__host__ __device__ constexpr size_t pf_offset(size_t lines_end) { return (lines_end + 15) & ~size_t(15); }

// ---------------------------------------------------------------------------
// Hbar psibar, complex, contraction type T (double or float)
//
// Each thread of an element's P1 x P1 plane owns one full 1-D line in every
// stage (a z-column, a y-line or an x-line), applies the folded 1-D operator in
// registers and writes the line back to shared memory:
//   forward  z (gathered column) -> y -> x            : u~ = B^(x)3 u
//   x-line:  r = J W V u~ + cx W W (Kq u~)_x           (written to R)
//   y-line:  R += cy W W (Kq u~)_y;  z-line: r = R + cz W W (Kq u~)_z
//   backward z -> y -> x (B^T), scatter-add of the x-line with the Loewdin scale.
// ---------------------------------------------------------------------------
// Element body shared by the single-system and the batched kernels: the threads
// of row threadIdx.y handle element eidx (P1 x P1 lines each) for the orbitals
// [o_begin, o_end) that orb(o, in, sc) accepts (in: the orbital's input vector,
// sc: its scale); results go to ev, alpha partials to part[o][pslot].
// Shared tables (sB, sBT, sK, sw) must be loaded and synchronized by the caller.
// BF16-operand mode (kBF, T = float): every value that enters a contraction as an
// operand -- the gathered input, the 1-D operator coefficients (rounded in the
// table) and each contraction result that feeds the next contraction -- is rounded
// to bfloat16; products and sums stay FP32.  That is the arithmetic of a BF16
// tensor-core contraction with FP32 accumulation, run on the CUDA cores to measure
// its accuracy.
template <bool kBF, int N>
__device__ __forceinline__ void bf_round(Cx<float> (&v)[N]) {
  if constexpr (kBF) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      v[i].re = __bfloat162float(__float2bfloat16_rn(v[i].re));
      v[i].im = __bfloat162float(__float2bfloat16_rn(v[i].im));
    }
  }
}
template <bool kBF, int N, typename V>
__device__ __forceinline__ void bf_round(V (&)[N]) {}

template <int P1, typename T, class OrbFn, bool kBF = false>
__device__ __forceinline__ void hbar_elem_body(const Geom& g, const T* sB, const T* sBT, const T* sK,
                                               const T* sw, Cx<T>* S1, Cx<T>* S2, double* red,
                                               const double* __restrict__ vks, long long eidx,
                                               int o_begin, int o_end, OrbFn orb,
                                               Cx<T>* __restrict__ ev, double* part,
                                               int64_t part_stride, long long pslot) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3;
  typedef Cx<T> V;
  const int u = threadIdx.x % P1, v = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const bool valid = plain_elem(g, eidx, ex, ey, ez);
  const long long n_elem = (long long)g.nx * g.ny * g.nz;
  T fx = from_d<T>(0.0), fy = from_d<T>(0.0), fz = from_d<T>(0.0);
  T vx[P1];
#pragma unroll
  for (int q = 0; q < P1; ++q) vx[q] = from_d<T>(0.0);
  if (valid) {
    const double hx = g.brk[0][ex + 1] - g.brk[0][ex];
    const double hy = g.brk[1][ey + 1] - g.brk[1][ey];
    const double hz = g.brk[2][ez + 1] - g.brk[2][ez];
    const double J = 0.125 * hx * hy * hz;
    const double wl = to_d(sw[u]) * to_d(sw[v]);
    fx = from_d<T>(hy * hz / (4.0 * hx) * wl);
    fy = from_d<T>(hx * hz / (4.0 * hy) * wl);
    fz = from_d<T>(hx * hy / (4.0 * hz) * wl);
    const long long e = ex + (long long)g.nx * (ey + (long long)g.ny * ez);
    const double* vp = vks + e * P3 + v * P2 + u * P1;      // x-line (qy = u, qz = v)
#pragma unroll
    for (int q = 0; q < P1; ++q) vx[q] = from_d<T>(vp[q] * J * wl * to_d(sw[q]));
  }
  const long long plane = (long long)g.nix * g.niy;
  // gather: z-column (a = u, b = v); Loewdin scales of the column (once per CTA)
  constexpr bool kF32 = std::is_same<T, float>::value;
  constexpr bool kDF = std::is_same<T, Df>::value;
  const int Ig = ex * g.p + u, Jg = ey * g.p + v;
  const bool inG = valid && Ig >= 1 && Ig <= g.nix && Jg >= 1 && Jg <= g.niy;
  const long long baseG = inG ? (long long)(Ig - 1) + (long long)g.nix * (Jg - 1) : 0;
  T gsc[P1];
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    const int K = ez * g.p + c;
    gsc[c] = from_d<T>((inG && K >= 1 && K <= g.niz) ? g.s[0][Ig] * g.s[1][Jg] * g.s[2][K] : 0.0);
  }

  for (int o = o_begin; o < o_end; ++o) {
    const double2* in = nullptr;
    double sc = 1.0;
    if (!orb(o, in, sc)) continue;
    V col[P1], t[P1];
    T scT;
    if constexpr (kF32) scT = d2f_bits(sc);
    else scT = from_d<T>(sc);
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      const int K = ez * g.p + c;
      vzero(col[c]);
      if (inG && K >= 1 && K <= g.niz) {
        const double2 w2 = in[baseG + plane * (K - 1)];
        if constexpr (kF32) {   // no FP64 arithmetic in the FP32 path
          const float f = gsc[c] * scT;
          col[c].re = d2f_bits(w2.x) * f;
          col[c].im = d2f_bits(w2.y) * f;
        } else if constexpr (kDF) {   // split on the integer pipe, products in DF64
          const Df f = df_mul(gsc[c], scT);
          col[c].re = df_mul(d2df_bits(w2.x), f);
          col[c].im = df_mul(d2df_bits(w2.y), f);
        } else {
          const double f = gsc[c] * sc;
          col[c].re = w2.x * f;
          col[c].im = w2.y * f;
        }
      }
    }
    // forward z, y, x
    bf_round<kBF>(col);
    cs_apply<P1>(sB, col, t);
    bf_round<kBF>(t);
    store_line(t, S1 + v * P1 + u, P2);
    __syncthreads();
    load_line(col, S1 + v * P2 + u, P1);
    cs_apply<P1>(sB, col, t);
    bf_round<kBF>(t);
    store_line(t, S2 + v * P2 + u, P1);
    __syncthreads();
    V uq[P1];
    load_line(col, S2 + v * P2 + u * P1, 1);
    cs_apply<P1>(sB, col, uq);
    bf_round<kBF>(uq);
    store_line(uq, S1 + v * P2 + u * P1, 1);          // U (Gauss-point values)
    cs_apply<P1>(sK, uq, t);
#pragma unroll
    for (int q = 0; q < P1; ++q) {
      V r = vscale(vx[q], uq[q]);
      madd(r, fx, t[q]);
      t[q] = r;
    }
    store_line(t, S2 + v * P2 + u * P1, 1);           // R
    __syncthreads();
    // y-line (qx = u, qz = v): R += cy W W (Kq U)_y
    load_line(col, S1 + v * P2 + u, P1);
    cs_apply<P1>(sK, col, t);
#pragma unroll
    for (int q = 0; q < P1; ++q) {
      V r = S2[v * P2 + q * P1 + u];
      madd(r, fy, t[q]);
      S2[v * P2 + q * P1 + u] = r;
    }
    __syncthreads();
    // z-line (qx = u, qy = v): r = R + cz W W (Kq U)_z
    load_line(col, S1 + v * P1 + u, P2);
    cs_apply<P1>(sK, col, t);
    T apt = from_d<T>(0.0);
#pragma unroll
    for (int q = 0; q < P1; ++q) {
      V r = S2[q * P2 + v * P1 + u];
      madd(r, fz, t[q]);
      uq[q] = r;
      dot_acc(apt, col[q], r);
    }
    double apart;
    if constexpr (kF32) apart = f2d_bits(apt);
    else if constexpr (kDF) apart = f2d_bits(apt.hi) + f2d_bits(apt.lo);
    else apart = apt;
    __syncthreads();
    // backward z, y, x
    bf_round<kBF>(uq);
    cs_apply<P1>(sBT, uq, t);
    bf_round<kBF>(t);
    store_line(t, S1 + v * P1 + u, P2);
    __syncthreads();
    load_line(col, S1 + v * P2 + u, P1);
    cs_apply<P1>(sBT, col, t);
    bf_round<kBF>(t);
    store_line(t, S2 + v * P2 + u, P1);
    __syncthreads();
    load_line(col, S2 + v * P2 + u * P1, 1);
    cs_apply<P1>(sBT, col, t);
    if (valid) store_line(t, ev + ((long long)o * n_elem + eidx) * P3 + v * P2 + u * P1, 1);
    if (part) {
      const double s = block_sum(apart, red);
      if (threadIdx.x + blockDim.x * threadIdx.y == 0) part[(long long)o * part_stride + pslot] = s;
    }
    __syncthreads();
  }
}

// Shared-memory layout of one element's lines in the split body: entry (a, b, c) at
// c * PS + b * LS + a, the Gauss-space copy S2 at P1 * PS, the next element ES entries on.
// The strides are padded (chosen by counting shared-memory wavefronts of the x-, y- and
// z-line accesses of 32-thread warps that straddle elements, for 4- and 8-byte entries)
// so that the line loads and stores of a warp fall into distinct banks as far as the
// P1 x P1 thread planes allow: at p = 7 the wavefronts per request fall from 4.3 to 1.3,
// at p = 6 from 1.8 to 1.6.
template <int P1, typename T>
struct SplitLayout {
  static constexpr bool kF = sizeof(T) == 4;
  static constexpr int LS = P1 == 8 || P1 == 9 ? 9 : P1;
  static constexpr int PS = P1 == 5 ? 25 : P1 == 6 ? 39 : P1 == 7 ? (kF ? 56 : 52) : P1 == 8 ? 72
                          : P1 == 9 ? (kF ? 81 : 89) : P1 * P1;
  static constexpr int ES = P1 == 5 ? 253 : P1 == 6 ? (kF ? 484 : 468) : P1 == 7 ? (kF ? 785 : 737)
                          : P1 == 8 ? 1152 : P1 == 9 ? (kF ? 1465 : 1617) : 2 * P1 * P1 * P1;
  static_assert(PS >= P1 * LS && ES >= 2 * P1 * PS, "padded layout holds two element cubes");
};

// Split form of the element body for the double-float contractions: Hbar is real, so
// the real and imaginary parts pass through the element one after the other.  Each
// thread then holds real lines only, which halves the line registers and the shared
// memory per element: the double-float kernel fits in 128 registers (no spills up to
// p = 6, 8-56 bytes at p = 7, 8 against 190-540 in the complex form; 9 % faster at p = 6).
// The next orbital's input columns are prefetched into shared memory during the
// imaginary pass (7 % faster at p = 6: the loads no longer stall the two CTAs of an SM).
// FP32 (no gain measured) and FP64 (bound by the FP64 pipe) keep the complex lines.
// Per-stage precision study of the double-float body (diagnostics,
// tdks_set_f32_stages): a stage whose bit is set in `mask` runs in FP32 arithmetic
// with FP32 operator coefficients, its input rounded to FP32 and its output widened
// back.  Bits 0-2: interpolation to the Gauss points along z, y, x; 3-5: the kinetic
// contractions along x, y, z; 6-8: the transposed interpolation along z, y, x; 9: the
// pointwise potential and kinetic combination; 10: the gathered, scaled input;
// 11: the element results as stored for the assembly.
template <int P1, typename T, bool kStudy>
__device__ __forceinline__ void stage_apply(const T* __restrict__ t, const float* tf, const T (&in)[P1],
                                            T (&out)[P1], unsigned mask, int bit) {
  if constexpr (kStudy) {
    if ((mask >> bit) & 1u) {
      float fi[P1], fo[P1];
#pragma unroll
      for (int k = 0; k < P1; ++k) fi[k] = __fadd_rn(in[k].hi, in[k].lo);
      cs_apply<P1>(tf, fi, fo);
#pragma unroll
      for (int k = 0; k < P1; ++k) out[k] = Df{fo[k], 0.0f};
      return;
    }
  }
  cs_apply<P1>(t, in, out);
}
template <bool kStudy, typename T>
__device__ __forceinline__ void stage_round(T& x, unsigned mask, int bit) {
  if constexpr (kStudy) {
    if ((mask >> bit) & 1u) x = Df{__fadd_rn(x.hi, x.lo), 0.0f};
  }
}

template <int P1, typename T, class OrbFn, bool kStudy = false>
__device__ __forceinline__ void hbar_elem_body_split(const Geom& g, const T* sB, const T* sBT, const T* sK,
                                                     const T* sw, T* S1, T* S2, double* red,
                                               const double* __restrict__ vks, long long eidx,
                                               int o_begin, int o_end, OrbFn orb,
                                               Cx<T>* __restrict__ ev, double* part,
                                               int64_t part_stride, long long pslot,
                                                     double2* __restrict__ pfbuf,
                                                     long long ev_ostride = 0, unsigned smask = 0,
                                                     const float* ftab = nullptr) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3;
  constexpr int LS = SplitLayout<P1, T>::LS, PS = SplitLayout<P1, T>::PS;
  constexpr int CSn = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;   // folded operator size
  typedef Cx<T> V;
  const int u = threadIdx.x % P1, v = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const bool valid = plain_elem(g, eidx, ex, ey, ez);
  const long long n_elem = (long long)g.nx * g.ny * g.nz;
  // Set-up of the element factors: the few FP64 products (no division, no FP64
  // conversion: the FP64 unit of this part is 1/64 of the FP32 rate) rounded into T
  // on the integer pipe.
  T fx = from_d<T>(0.0), fy = from_d<T>(0.0), fz = from_d<T>(0.0);
  T vx[P1];
#pragma unroll
  for (int q = 0; q < P1; ++q) vx[q] = from_d<T>(0.0);
  if (valid) {
    const double hx = g.brk[0][ex + 1] - g.brk[0][ex];
    const double hy = g.brk[1][ey + 1] - g.brk[1][ey];
    const double hz = g.brk[2][ez + 1] - g.brk[2][ez];
    const double wl4 = 0.25 * g.wq[u] * g.wq[v];
    fx = d2t<T>(hy * hz * g.ih[0][ex] * wl4);
    fy = d2t<T>(hx * hz * g.ih[1][ey] * wl4);
    fz = d2t<T>(hx * hy * g.ih[2][ez] * wl4);
    const double jw = 0.5 * hx * hy * hz * wl4;          // J wl, J = hx hy hz / 8
    const long long e = ex + (long long)g.nx * (ey + (long long)g.ny * ez);
    const double* vp = vks + e * P3 + v * P2 + u * P1;      // x-line (qy = u, qz = v)
#pragma unroll
    for (int q = 0; q < P1; ++q) vx[q] = d2t<T>(vp[q] * (jw * g.wq[q]));
  }
  const long long plane = (long long)g.nix * g.niy;
  // gather: z-column (a = u, b = v); Loewdin scales of the column (once per CTA)
  constexpr bool kF32 = std::is_same<T, float>::value;
  const int Ig = ex * g.p + u, Jg = ey * g.p + v;
  const bool inG = valid && Ig >= 1 && Ig <= g.nix && Jg >= 1 && Jg <= g.niy;
  const long long baseG = inG ? (long long)(Ig - 1) + (long long)g.nix * (Jg - 1) : 0;
  const double sxy = inG ? g.s[0][Ig] * g.s[1][Jg] : 0.0;
  T gsc[P1];
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    const int K = ez * g.p + c;
    gsc[c] = d2t<T>((inG && K >= 1 && K <= g.niz) ? sxy * g.s[2][K] : 0.0);
  }

  // The z-columns of the next active orbital are copied into shared memory
  // (cp.async, 16 B per node, zero-filled outside the interior) while the current
  // orbital is computed; the buffer holds P1 double2 per thread, [c][thread].
  const int tid_pf = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr_pf = blockDim.x * blockDim.y;
  auto issue = [&](const double2* src_base) {
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      const int K = ez * g.p + c;
      const bool ok = inG && K >= 1 && K <= g.niz;
      const double2* src = ok ? src_base + baseG + plane * (K - 1) : src_base;
      const unsigned sa = (unsigned)__cvta_generic_to_shared(pfbuf + c * nthr_pf + tid_pf);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(ok ? 16 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  int o = o_begin;
  {
    const double2* in0 = nullptr;
    double sc0 = 1.0;
    while (o < o_end && !orb(o, in0, sc0)) ++o;
    if (o < o_end) issue(in0);
  }
  while (o < o_end) {
    const double2* in = nullptr;
    double sc = 1.0;
    orb(o, in, sc);
    int on = o_end;   // next active orbital, found when its prefetch is issued
    const T scT = d2t<T>(sc);
    T apt = from_d<T>(0.0);
    // element results of orbital o start ev_ostride entries apart (n_elem P1^3 by default)
    T* evr = reinterpret_cast<T*>(ev + (long long)o * (ev_ostride > 0 ? ev_ostride : n_elem * P3) +
                                  eidx * P3 + v * P2 + u * P1);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
#pragma unroll 1
    for (int comp = 0; comp < 2; ++comp) {   // real part, then imaginary part
      T col[P1], t[P1];
#pragma unroll
      for (int c = 0; c < P1; ++c) {
        const int K = ez * g.p + c;
        vzero(col[c]);
        if (inG && K >= 1 && K <= g.niz) {
          const double2 w2 = pfbuf[c * nthr_pf + tid_pf];
          const double x = comp ? w2.y : w2.x;
          if constexpr (kF32) {
            col[c] = d2f_bits(x) * (gsc[c] * scT);
          } else {
            col[c] = df_mul(d2df_bits(x), df_mul(gsc[c], scT));
            stage_round<kStudy>(col[c], smask, 10);
          }
        }
      }
      // forward z, y, x
      stage_apply<P1, T, kStudy>(sB, ftab, col, t, smask, 0);
      store_line(t, S1 + v * LS + u, PS);
      __syncthreads();
      // the buffer was last read before this barrier: refill it for the next orbital
      if (comp == 1) {
        const double2* in_n = nullptr;
        double sc_n = 1.0;
        on = o + 1;
        while (on < o_end && !orb(on, in_n, sc_n)) ++on;
        if (on < o_end) issue(in_n);
      }
      load_line(col, S1 + v * PS + u, LS);
      stage_apply<P1, T, kStudy>(sB, ftab, col, t, smask, 1);
      store_line(t, S2 + v * PS + u, LS);
      __syncthreads();
      T uq[P1];
      load_line(col, S2 + v * PS + u * LS, 1);
      stage_apply<P1, T, kStudy>(sB, ftab, col, uq, smask, 2);
      store_line(uq, S1 + v * PS + u * LS, 1);          // U (Gauss-point values)
      stage_apply<P1, T, kStudy>(sK, ftab ? ftab + 2 * CSn : nullptr, uq, t, smask, 3);
#pragma unroll
      for (int q = 0; q < P1; ++q) {
        T r = vscale(vx[q], uq[q]);
        madd(r, fx, t[q]);
        stage_round<kStudy>(r, smask, 9);
        t[q] = r;
      }
      store_line(t, S2 + v * PS + u * LS, 1);           // R
      __syncthreads();
      load_line(col, S1 + v * PS + u, LS);
      stage_apply<P1, T, kStudy>(sK, ftab ? ftab + 2 * CSn : nullptr, col, t, smask, 4);
#pragma unroll
      for (int q = 0; q < P1; ++q) {
        T r = S2[v * PS + q * LS + u];
        madd(r, fy, t[q]);
        stage_round<kStudy>(r, smask, 9);
        S2[v * PS + q * LS + u] = r;
      }
      __syncthreads();
      load_line(col, S1 + v * LS + u, PS);
      stage_apply<P1, T, kStudy>(sK, ftab ? ftab + 2 * CSn : nullptr, col, t, smask, 5);
#pragma unroll
      for (int q = 0; q < P1; ++q) {
        T r = S2[q * PS + v * LS + u];
        madd(r, fz, t[q]);
        stage_round<kStudy>(r, smask, 9);
        uq[q] = r;
        dot_acc(apt, col[q], r);
      }
      __syncthreads();
      // backward z, y, x
      stage_apply<P1, T, kStudy>(sBT, ftab ? ftab + CSn : nullptr, uq, t, smask, 6);
      store_line(t, S1 + v * LS + u, PS);
      __syncthreads();
      load_line(col, S1 + v * PS + u, LS);
      stage_apply<P1, T, kStudy>(sBT, ftab ? ftab + CSn : nullptr, col, t, smask, 7);
      store_line(t, S2 + v * PS + u, LS);
      __syncthreads();
      load_line(col, S2 + v * PS + u * LS, 1);
      stage_apply<P1, T, kStudy>(sBT, ftab ? ftab + CSn : nullptr, col, t, smask, 8);
      if (valid) {
#pragma unroll
        for (int a2 = 0; a2 < P1; ++a2) {
          stage_round<kStudy>(t[a2], smask, 11);
          evr[2 * a2 + comp] = t[a2];
        }
      }
      __syncthreads();
    }
    if (part) {
      // the CTA's alpha partial summed in T (on the FP32 pipe), to FP64 once
      const T s = block_sum_t(apt, reinterpret_cast<T*>(red));
      if (threadIdx.x + blockDim.x * threadIdx.y == 0) part[(long long)o * part_stride + pslot] = t2d(s);
    }
    o = on;
  }
}

// Register budget of the element kernels: at most 128 registers, so that two CTAs
// (16 warps) share an SM.
template <int P1, typename T, bool kBF = false>
__global__ void __launch_bounds__(256, 2) k_hbar(Geom g, const T* __restrict__ tab,
                                              const double* __restrict__ vks, ApplyArgs a,
                                              int orb_per_cta, Cx<T>* __restrict__ ev) {
  constexpr int P3 = Cfg<P1>::P3;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  typedef Cx<T> V;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[8];
  T* sB = reinterpret_cast<T*>(smem);
  T* sBT = sB + CS;
  T* sK = sBT + CS;
  T* sw = sK + CS;
  const size_t off = ((3 * CS + P1) * sizeof(T) + 15) & ~size_t(15);
  V* S1 = reinterpret_cast<V*>(smem + off) + (size_t)threadIdx.y * 2 * P3;
  V* S2 = S1 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < 3 * CS; i += nthr) sB[i] = tab[tab_off_csB(P1) + i];
  for (int i = tid; i < P1; i += nthr) sw[i] = tab[tab_off_w(P1) + i];
  __syncthreads();
  const long long eidx = (long long)blockIdx.x * blockDim.y + threadIdx.y;
  const int o0 = blockIdx.y * orb_per_cta;
  const int o1 = min(o0 + orb_per_cta, a.n_orb);
  auto orb = [&](int o, const double2*& in, double& sc) -> bool {
    if (a.kry) {
      if (a.kry[o].status != KRY_ACTIVE) return false;
      sc = a.kry[o].s[a.kj];
    }
    in = a.in_base + (long long)o * a.in_stride;
    return true;
  };
  if (a.kry) {   // a CTA whose orbitals have all left the recurrence skips the element set-up
    bool any = false;
    for (int o = o0; o < o1 && !any; ++o) any = a.kry[o].status == KRY_ACTIVE;
    if (!any) return;
  }
  hbar_elem_body<P1, T, decltype(orb), kBF>(g, sB, sBT, sK, sw, S1, S2, red, vks, eidx, o0, o1, orb, ev,
                                            a.part, a.part_stride, blockIdx.x);
}

// split element body (real lines): double-float without register spills at two CTAs
// per SM; FP32 in 64 registers, four CTAs (32 warps) per SM to hide the latency of its
// light arithmetic (three, 85 registers, for p >= 7, whose longer lines spill at 64)
template <int P1, typename T>
struct SplitOcc {
  static constexpr int value = std::is_same<T, float>::value ? (P1 >= 8 ? 3 : 4) : 2;
};
template <int P1, typename T, bool kStudy = false>
__global__ void __launch_bounds__(256, SplitOcc<P1, T>::value) k_hbar_split(Geom g, const T* __restrict__ tab,
                                              const double* __restrict__ vks, ApplyArgs a,
                                              int orb_per_cta, Cx<T>* __restrict__ ev,
                                              unsigned smask) {
  constexpr int P3 = Cfg<P1>::P3;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[8];
  T* sB = reinterpret_cast<T*>(smem);
  T* sBT = sB + CS;
  T* sK = sBT + CS;
  T* sw = sK + CS;
  const size_t off = ((3 * CS + P1) * sizeof(T) + 15) & ~size_t(15);
  T* S1 = reinterpret_cast<T*>(smem + off) + (size_t)threadIdx.y * SplitLayout<P1, T>::ES;
  T* S2 = S1 + P1 * SplitLayout<P1, T>::PS;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < 3 * CS; i += nthr) sB[i] = tab[tab_off_csB(P1) + i];
  for (int i = tid; i < P1; i += nthr) sw[i] = tab[tab_off_w(P1) + i];
  __syncthreads();
  const float* ftab = nullptr;
  if constexpr (kStudy) {   // FP32 copies of the folded operators for the stage study
    __shared__ float fst[3 * CS];
    for (int i = tid; i < 3 * CS; i += nthr) fst[i] = __fadd_rn(sB[i].hi, sB[i].lo);
    __syncthreads();
    ftab = fst;
  }
  const long long eidx = (long long)blockIdx.x * blockDim.y + threadIdx.y;
  const int o0 = blockIdx.y * orb_per_cta;
  const int o1 = min(o0 + orb_per_cta, a.n_orb);
  auto orb = [&](int o, const double2*& in, double& sc) -> bool {
    if (a.kry) {
      if (a.kry[o].status != KRY_ACTIVE) return false;
      sc = a.kry[o].s[a.kj];
    }
    in = a.in_base + (long long)o * a.in_stride;
    return true;
  };
  if (a.kry) {   // a CTA whose orbitals have all left the recurrence skips the element set-up
    bool any = false;
    for (int o = o0; o < o1 && !any; ++o) any = a.kry[o].status == KRY_ACTIVE;
    if (!any) return;
  }
  hbar_elem_body_split<P1, T, decltype(orb), kStudy>(
      g, sB, sBT, sK, sw, S1, S2, red, vks, eidx, o0, o1, orb, ev, a.part, a.part_stride, blockIdx.x,
      reinterpret_cast<double2*>(smem + pf_offset(off + (size_t)blockDim.y * SplitLayout<P1, T>::ES * sizeof(T))),
      0, smask, ftab);
}

// alpha_j = sum of the element partials (fixed order), for the active orbitals
__global__ void k_alpha(KryOrb* kry, const double* part, int64_t pstride, int nparts, int j) {
  __shared__ double red[8];
  const int o = blockIdx.x;
  if (kry[o].status != KRY_ACTIVE) return;
  double v = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) v += part[(long long)o * pstride + k];
  const double s = block_sum(v, red);
  if (threadIdx.x == 0) kry[o].alpha[j] = s;
}

// Elements whose closure holds node I along one axis: 1 (inside an element) or 2
// (on a shared face), with the node's local index in each.
__device__ __forceinline__ int node_elems(int I, int p, int n, int* e, int* loc) {
  const int eh = I / p, l = I - eh * p;
  if (l != 0) {
    e[0] = eh;
    loc[0] = l;
    return 1;
  }
  int k = 0;
  if (eh - 1 >= 0) {
    e[k] = eh - 1;
    loc[k] = p;
    ++k;
  }
  if (eh < n) {
    e[k] = eh;
    loc[k] = 0;
    ++k;
  }
  return k;
}

// Assembly by gathering: every interior node sums its (at most 8) element-local
// contributions in a fixed order and applies the Loewdin scale.  With `lanczos`
// the three-term update w = Hbar q_j - alpha_j q_j - beta_{j-1} q_{j-1} is fused
// (ca = alpha_j s_j, cb = beta_{j-1} s_{j-1}) and the sum of |w|^2 over the rows
// r0, r0 + rstride, ... handled here is returned.  The degree is a compile-time
// constant: the node -> (element, local index) split is a multiply-shift.
template <int P1, typename T>
__device__ __forceinline__ double assemble_rows(const Geom& g, const Cx<T>* __restrict__ evo,
                                                const double2* qj, const double2* qm,
                                                double2* out, double ca, double cb, int lanczos,
                                                int accumulate, int r0, int rstride) {
  constexpr int p = P1 - 1, P2 = P1 * P1, P3 = P2 * P1;
  constexpr bool kF32 = std::is_same<T, float>::value;
  constexpr bool kDF = std::is_same<T, Df>::value;
  const int rows = g.niy * g.niz;
  // short rows (fewer nodes than threads) are processed several at a time
  const int nix = g.nix, nt = (int)blockDim.x;
  const int rpb = nix >= nt ? 1 : nt / nix;                 // rows in flight per block
  const int tr = nix >= nt ? 0 : (int)threadIdx.x / nix;    // this thread's row slot
  const int tI = nix >= nt ? (int)threadIdx.x : (int)threadIdx.x % nix;
  const int tstep = nix >= nt ? nt : nix;
  double acc = 0.0;
  if (tr >= rpb) return acc;
  const long long xstride = P3;                             // next element along x
  for (int r = r0 + tr * rstride; r < rows; r += rpb * rstride) {
    const int J = r % g.niy + 1, K = r / g.niy + 1;
    int ey[2], by[2], ez[2], bz[2];
    const int ny = node_elems(J, p, g.ny, ey, by);
    const int nz = node_elems(K, p, g.nz, ez, bz);
    // element rows (y, z) holding this node row, in the order z then y
    long long base[4] = {0, 0, 0, 0};
    const int nb = ny * nz;
#pragma unroll
    for (int kz = 0; kz < 2; ++kz)
#pragma unroll
      for (int ky = 0; ky < 2; ++ky)
        if (kz < nz && ky < ny)
          base[kz * ny + ky] = (long long)g.nx * (ey[ky] + (long long)g.ny * ez[kz]) * P3 + bz[kz] * P2 + by[ky] * P1;
    const double syz = g.s[1][J] * g.s[2][K];
    const float syzf = g.sf[1][J] * g.sf[2][K];
    const long long rowbase = (long long)g.nix * (r);
    for (int I = tI + 1; I <= g.nix; I += tstep) {
      // x: one element inside, two on a shared face (left element first)
      const int eh = I / p, l = I - eh * p;
      long long xo[2] = {0, 0};
      int nxc;
      if (l != 0) {
        xo[0] = eh * xstride + l;
        nxc = 1;
      } else {
        nxc = 0;
        if (eh - 1 >= 0) xo[nxc++] = (eh - 1) * xstride + p;
        if (eh < g.nx) xo[nxc++] = eh * xstride;
      }
      double re = 0.0, im = 0.0;
      float fre = 0.f, fim = 0.f;
      Df dre{0.f, 0.f}, dim{0.f, 0.f};
      // exactly nb * nxc additions in the fixed order (z, y, then x); the offsets are
      // picked by selects so that base[] and xo[] stay in registers (an unrolled loop
      // with predicates would turn into 16 unconditional FP64 additions per node)
      const int ncon = nb * nxc;
      for (int tcon = 0; tcon < ncon; ++tcon) {
          const int k = nxc == 2 ? (tcon >> 1) : tcon;
          const long long bk = k == 0 ? base[0] : (k == 1 ? base[1] : (k == 2 ? base[2] : base[3]));
          const long long xk = (nxc == 2 && (tcon & 1)) ? xo[1] : xo[0];
          const Cx<T> c = evo[bk + xk];
          if constexpr (kF32) {
            fre += c.re;
            fim += c.im;
          } else if constexpr (kDF) {
            dre = df_add(dre, c.re);
            dim = df_add(dim, c.im);
          } else {
            re += c.re;
            im += c.im;
          }
        }
      if constexpr (kDF) {
        re = f2d_bits(dre.hi) + f2d_bits(dre.lo);
        im = f2d_bits(dim.hi) + f2d_bits(dim.lo);
      }
      const long long idx = rowbase + (I - 1);
      double2 w;
      if constexpr (kF32) {   // sum, scale and convert without the FP64 pipe
        const float f = g.sf[0][I] * syzf;
        w = make_double2(f2d_bits(f * fre), f2d_bits(f * fim));
      } else {
        const double f = g.s[0][I] * syz;
        w = make_double2(f * re, f * im);
      }
      if (lanczos) {
        const double2 x = qj[idx];
        w.x = fma(-ca, x.x, w.x);
        w.y = fma(-ca, x.y, w.y);
        if (qm) {
          const double2 y = qm[idx];
          w.x = fma(-cb, y.x, w.x);
          w.y = fma(-cb, y.y, w.y);
        }
        acc = fma(w.x, w.x, fma(w.y, w.y, acc));
      }
      if (accumulate) {
        const double2 o2 = out[idx];
        w.x += o2.x;
        w.y += o2.y;
      }
      out[idx] = w;
    }
  }
  return acc;
}

template <int P1, typename T>
__global__ void __launch_bounds__(128) k_assemble(Geom g, const Cx<T>* __restrict__ ev, ApplyArgs a) {
  __shared__ double red[4];
  const int o = blockIdx.y;
  double ca = 0.0, cb = 0.0;
  if (a.kry) {
    const KryOrb& K = a.kry[o];
    if (K.status != KRY_ACTIVE) return;
    if (a.lanczos) {
      ca = K.alpha[a.kj] * K.s[a.kj];
      cb = a.kj > 0 ? K.beta[a.kj - 1] * K.s[a.kj - 1] : 0.0;
    }
  }
  const long long n_elem = (long long)g.nx * g.ny * g.nz;
  const Cx<T>* evo = ev + (long long)o * n_elem * P1 * P1 * P1;
  const double2* qj = a.in_base + (long long)o * a.in_stride;
  const double2* qm = a.vm_base ? a.vm_base + (long long)o * a.vm_stride : nullptr;
  double2* out = a.out_base + (long long)o * a.out_stride;
  const double acc = assemble_rows<P1, T>(g, evo, qj, qm, out, ca, cb, a.lanczos, a.accumulate,
                                          blockIdx.x, gridDim.x);
  if (a.npart) {
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) a.npart[(long long)o * a.npart_stride + blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// GLL-collocation variant: every integral of H by the GLL rule on the element nodes.
// Kinetic: sum_d c_d (K1 along d) x W_l x W_l (W_l: GLL weights; K1 = D^T W D is the
// exact 1-D stiffness, so only the transverse mass is lumped); the potential is the
// diagonal V(x_j) in the Loewdin basis and is added after the assembly.  Three
// one-dimensional contractions per element and component (folded K1).
// ---------------------------------------------------------------------------
template <int P1>
__global__ void __launch_bounds__(256, 2) k_hbar_gll(Geom g, const double* __restrict__ tab,
                                                  const double2* __restrict__ in, int64_t stride,
                                                  int n_orb, int orb_per_cta, Cx<double>* __restrict__ ev) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  typedef Cx<double> V;
  extern __shared__ __align__(16) unsigned char smem[];
  double* sK = reinterpret_cast<double*>(smem);
  double* swl = sK + CS;
  const size_t off = ((CS + P1) * sizeof(double) + 15) & ~size_t(15);
  V* S1 = reinterpret_cast<V*>(smem + off) + (size_t)threadIdx.y * 2 * P3;
  V* S2 = S1 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < CS; i += nthr) sK[i] = tab[tab_off_csK1(P1) + i];
  for (int i = tid; i < P1; i += nthr) swl[i] = tab[tab_off_wl(P1) + i];
  __syncthreads();
  const int u = threadIdx.x % P1, v = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const long long eidx = (long long)blockIdx.x * blockDim.y + threadIdx.y;
  const bool valid = plain_elem(g, eidx, ex, ey, ez);
  const long long n_elem = (long long)g.nx * g.ny * g.nz;
  double cx = 0.0, cy = 0.0, cz = 0.0;
  if (valid) {
    const double hx = g.brk[0][ex + 1] - g.brk[0][ex];
    const double hy = g.brk[1][ey + 1] - g.brk[1][ey];
    const double hz = g.brk[2][ez + 1] - g.brk[2][ez];
    cx = hy * hz / (4.0 * hx);
    cy = hx * hz / (4.0 * hy);
    cz = hx * hy / (4.0 * hz);
  }
  const long long plane = (long long)g.nix * g.niy;
  const int Ig = ex * g.p + u, Jg = ey * g.p + v;
  const bool inG = valid && Ig >= 1 && Ig <= g.nix && Jg >= 1 && Jg <= g.niy;
  const long long baseG = inG ? (long long)(Ig - 1) + (long long)g.nix * (Jg - 1) : 0;
  double gsc[P1];
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    const int K = ez * g.p + c;
    gsc[c] = (inG && K >= 1 && K <= g.niz) ? g.s[0][Ig] * g.s[1][Jg] * g.s[2][K] : 0.0;
  }
  const int o0 = blockIdx.y * orb_per_cta;
  const int o1 = min(o0 + orb_per_cta, n_orb);
  for (int o = o0; o < o1; ++o) {
    const double2* x = in + (long long)o * stride;
    V col[P1], t[P1];
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      const int K = ez * g.p + c;
      vzero(col[c]);
      if (inG && K >= 1 && K <= g.niz) {
        const double2 w2 = x[baseG + plane * (K - 1)];
        col[c].re = w2.x * gsc[c];
        col[c].im = w2.y * gsc[c];
      }
    }
    // z: r = cz Wl_x Wl_y (K1 u)_z  (thread owns the z-line at (x = u, y = v))
    store_line(col, S1 + v * P1 + u, P2);
    cs_apply<P1>(sK, col, t);
    const double fz = cz * swl[u] * swl[v];
#pragma unroll
    for (int c = 0; c < P1; ++c) t[c] = vscale(fz, t[c]);
    store_line(t, S2 + v * P1 + u, P2);
    __syncthreads();
    // y: r += cy Wl_x Wl_z (K1 u)_y  (y-line at (x = u, z = v))
    load_line(col, S1 + v * P2 + u, P1);
    cs_apply<P1>(sK, col, t);
    const double fy = cy * swl[u] * swl[v];
#pragma unroll
    for (int b = 0; b < P1; ++b) {
      V r = S2[v * P2 + b * P1 + u];
      madd(r, fy, t[b]);
      S2[v * P2 + b * P1 + u] = r;
    }
    __syncthreads();
    // x: r += cx Wl_y Wl_z (K1 u)_x  (x-line at (y = u, z = v)); element result
    load_line(col, S1 + v * P2 + u * P1, 1);
    cs_apply<P1>(sK, col, t);
    const double fx = cx * swl[u] * swl[v];
#pragma unroll
    for (int a2 = 0; a2 < P1; ++a2) {
      V r = S2[v * P2 + u * P1 + a2];
      madd(r, fx, t[a2]);
      t[a2] = r;
    }
    if (valid) store_line(t, ev + ((long long)o * n_elem + eidx) * P3 + v * P2 + u * P1, 1);
    __syncthreads();
  }
}

// out += v psi (the collocated potential, diagonal in the Loewdin basis)
__global__ void k_diag_add(long long n, int n_orb, const double* __restrict__ vn,
                           const double2* __restrict__ in, double2* __restrict__ out) {
  const long long tot = n * n_orb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const double f = vn[i % n];
    const double2 x = in[i];
    double2 y = out[i];
    y.x = fma(f, x.x, y.x);
    y.y = fma(f, x.y, y.y);
    out[i] = y;
  }
}

// ---------------------------------------------------------------------------
// Batched apply: a persistent grid walks the work list of one degree class.
// Item (sys, eblk, o0, o1): elements [eblk E, eblk E + E) of system sys for the
// orbitals o0..o1-1 that are in the Lanczos recurrence; each orbital reads its own
// current basis vector V_j (j = K.k): the exponential's start vector for j = 0
// (input or, after a sub-step, output), the workspace otherwise.
// ---------------------------------------------------------------------------
__device__ __forceinline__ const double2* bvec(const BSys& S, const KryOrb& K, int o, int j) {
  if (j == 0) return (K.nsub == 0 ? S.in : S.out) + (long long)o * S.n_int;
  return S.Vw + ((long long)o * S.kmax + (j - 1)) * S.n_int;
}

template <int P1, typename T>
__global__ void __launch_bounds__(256, 2) k_hbar_batch(const BSys* __restrict__ sys,
                                                    const BItem* __restrict__ items, int n_items,
                                                    const T* __restrict__ tab, int* __restrict__ qctr) {
  constexpr int P3 = Cfg<P1>::P3;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  typedef Cx<T> V;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[8];
  T* sB = reinterpret_cast<T*>(smem);
  T* sBT = sB + CS;
  T* sK = sBT + CS;
  T* sw = sK + CS;
  const size_t off = ((3 * CS + P1) * sizeof(T) + 15) & ~size_t(15);
  V* S1 = reinterpret_cast<V*>(smem + off) + (size_t)threadIdx.y * 2 * P3;
  V* S2 = S1 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < 3 * CS; i += nthr) sB[i] = tab[tab_off_csB(P1) + i];
  for (int i = tid; i < P1; i += nthr) sw[i] = tab[tab_off_w(P1) + i];
  __syncthreads();
  // the current item's system descriptor is staged in shared memory: its fields are
  // re-read where used instead of occupying registers across the element body
  // items are taken from a shared ticket counter (zeroed before every launch), so
  // CTAs that draw items of finished orbitals move on at once and the grid stays
  // balanced whatever the mix of active orbitals
  __shared__ BSys sS;
  __shared__ BItem sW;
  __shared__ int sIt;
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      const int it = atomicAdd(qctr, 1);
      sIt = it;
      if (it < n_items) sW = items[it];
    }
    __syncthreads();
    if (sIt >= n_items) break;
    for (int i = tid; i < (int)(sizeof(BSys) / 8); i += nthr)
      reinterpret_cast<long long*>(&sS)[i] = reinterpret_cast<const long long*>(&sys[sW.sys])[i];
    __syncthreads();
    const BItem w = sW;
    const BSys& S = sS;
    const Geom& g = S.g;
    const long long eidx = (long long)w.eblk * blockDim.y + threadIdx.y;
    auto orb = [&](int o, const double2*& in, double& sc) -> bool {
      const KryOrb& K = S.kry[o];
      if (K.status != KRY_ACTIVE) return false;
      const int j = K.k;
      in = bvec(S, K, o, j);
      sc = K.s[j];
      return true;
    };
    {   // an item none of whose orbitals is active is skipped before the element set-up
      bool any = false;
      for (int o = w.o0; o < w.o1 && !any; ++o) {
        const double2* in_o;
        double sc_o;
        any = orb(o, in_o, sc_o);
      }
      if (!any) continue;
    }
    hbar_elem_body<P1, T>(g, sB, sBT, sK, sw, S1, S2, red, S.vks, eidx, w.o0, w.o1, orb,
                          static_cast<Cx<T>*>(S.ev), S.apart, S.n_eblk, w.eblk);
  }
}

// Batched element results are kept at the orbital stride of 16-byte entries for every
// contraction type, so that under TDKS_MIXED FP32 and double-float orbitals share the
// buffer: entries of Cx<T> per orbital = n_elem P1^3 * omul<T>.
template <typename T>
__host__ __device__ constexpr int batch_omul() { return (int)(sizeof(double2) / sizeof(Cx<T>)); }

template <int P1, typename T>
__global__ void __launch_bounds__(256, SplitOcc<P1, T>::value) k_hbar_batch_split(const BSys* __restrict__ sys,
                                                    const BItem* __restrict__ items, int n_items,
                                                    const T* __restrict__ tab, int* __restrict__ qctr) {
  constexpr int P3 = Cfg<P1>::P3;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[8];
  T* sB = reinterpret_cast<T*>(smem);
  T* sBT = sB + CS;
  T* sK = sBT + CS;
  T* sw = sK + CS;
  const size_t off = ((3 * CS + P1) * sizeof(T) + 15) & ~size_t(15);
  T* S1 = reinterpret_cast<T*>(smem + off) + (size_t)threadIdx.y * SplitLayout<P1, T>::ES;
  T* S2 = S1 + P1 * SplitLayout<P1, T>::PS;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < 3 * CS; i += nthr) sB[i] = tab[tab_off_csB(P1) + i];
  for (int i = tid; i < P1; i += nthr) sw[i] = tab[tab_off_w(P1) + i];
  __syncthreads();
  // the current item's system descriptor is staged in shared memory: its fields are
  // re-read where used instead of occupying registers across the element body
  // items are taken from a shared ticket counter (zeroed before every launch), so
  // CTAs that draw items of finished orbitals move on at once and the grid stays
  // balanced whatever the mix of active orbitals
  __shared__ BSys sS;
  __shared__ BItem sW;
  __shared__ int sIt;
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      const int it = atomicAdd(qctr, 1);
      sIt = it;
      if (it < n_items) sW = items[it];
    }
    __syncthreads();
    if (sIt >= n_items) break;
    for (int i = tid; i < (int)(sizeof(BSys) / 8); i += nthr)
      reinterpret_cast<long long*>(&sS)[i] = reinterpret_cast<const long long*>(&sys[sW.sys])[i];
    __syncthreads();
    const BItem w = sW;
    const BSys& S = sS;
    const Geom& g = S.g;
    const long long eidx = (long long)w.eblk * blockDim.y + threadIdx.y;
    auto orb = [&](int o, const double2*& in, double& sc) -> bool {
      const KryOrb& K = S.kry[o];
      if (K.status != KRY_ACTIVE) return false;
      // relaxed schedule: this launch takes the orbitals whose next product is of type T
      if (S.mixed && K.f32 != (std::is_same<T, float>::value ? 1 : 0)) return false;
      const int j = K.k;
      in = bvec(S, K, o, j);
      sc = K.s[j];
      return true;
    };
    {   // an item none of whose orbitals takes a product of type T now is skipped before
        // the element set-up
      bool any = false;
      for (int o = w.o0; o < w.o1 && !any; ++o) {
        const double2* in_o;
        double sc_o;
        any = orb(o, in_o, sc_o);
      }
      if (!any) continue;
    }
    hbar_elem_body_split<P1, T>(g, sB, sBT, sK, sw, S1, S2, red, S.vks, eidx, w.o0, w.o1, orb,
                                static_cast<Cx<T>*>(S.ev), S.apart, S.n_eblk, w.eblk,
                                reinterpret_cast<double2*>(smem + pf_offset(off + (size_t)blockDim.y * SplitLayout<P1, T>::ES * sizeof(T))),
                                S.n_elem * P3 * batch_omul<T>());
  }
}

// alpha_j from the element partials (fixed order), one block per orbital
__global__ void k_balpha(const BSys* __restrict__ sys, const BOrb* __restrict__ orbs) {
  __shared__ double red[8];
  const BOrb b = orbs[blockIdx.x];
  const BSys& S = sys[b.sys];
  KryOrb& K = S.kry[b.o];
  if (K.status != KRY_ACTIVE) return;
  const double* part = S.apart + (long long)b.o * S.n_eblk;
  double v = 0.0;
  for (int k = threadIdx.x; k < S.n_eblk; k += blockDim.x) v += part[k];
  const double s = block_sum(v, red);
  if (threadIdx.x == 0) K.alpha[K.k] = s;
}

// gather assembly with the three-term update, one block per (system, orbital, row block)
// of one degree class (the degree as a compile-time constant, as in k_assemble)
template <int P1, typename T>
__global__ void __launch_bounds__(128) k_bassemble(const BSys* __restrict__ sys,
                                                   const BRow* __restrict__ rows) {
  __shared__ double red[4];
  const BRow w = rows[blockIdx.x];
  const BSys& S = sys[w.sys];
  const KryOrb& K = S.kry[w.o];
  if (K.status != KRY_ACTIVE) return;
  if (S.mixed && K.f32 != (std::is_same<T, float>::value ? 1 : 0)) return;
  const int j = K.k;
  const double ca = K.alpha[j] * K.s[j];
  const double cb = j > 0 ? K.beta[j - 1] * K.s[j - 1] : 0.0;
  const double2* qj = bvec(S, K, w.o, j);
  const double2* qm = j > 0 ? bvec(S, K, w.o, j - 1) : nullptr;
  double2* out = S.Vw + ((long long)w.o * S.kmax + j) * S.n_int;
  const Cx<T>* evo = static_cast<const Cx<T>*>(S.ev) +
                     (long long)w.o * S.n_elem * (P1 * P1 * P1) * batch_omul<T>();
  const double acc = assemble_rows<P1, T>(S.g, evo, qj, qm, out, ca, cb, 1, 0, w.rblk, S.n_rblk);
  const double sum = block_sum(acc, red);
  if (threadIdx.x == 0) S.npart[(long long)w.o * S.n_rblk + w.rblk] = sum;
}

// ---------------------------------------------------------------------------
// Poisson stiffness K u (real, FP64), nodal 7-contraction form
// ---------------------------------------------------------------------------
template <int P1>
__global__ void __launch_bounds__(256) k_stiff(Geom g, const double* __restrict__ tab,
                                               const double* __restrict__ in,
                                               double* __restrict__ out, double* part,
                                               int part_off, const CgState* cg, int color) {
  if (cg && cg->done) return;
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[8];
  double* sK1 = reinterpret_cast<double*>(smem);
  double* sMg = sK1 + P2;
  double* S1 = sMg + P2 + (size_t)threadIdx.y * 4 * P3;
  double* S2 = S1 + P3;
  double* S3 = S2 + P3;
  double* S4 = S3 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < P2; i += nthr) {
    sK1[i] = tab[tab_off_K1(P1) + i];
    sMg[i] = tab[tab_off_Mg(P1) + i];
  }
  const int ta = threadIdx.x % P1, tb = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const bool valid = color_elem(g, color, (long long)blockIdx.x * blockDim.y + threadIdx.y, ex, ey, ez);
  __syncthreads();
  double cx = 0, cy = 0, cz = 0;
  if (valid) {
    const double hx = g.brk[0][ex + 1] - g.brk[0][ex];
    const double hy = g.brk[1][ey + 1] - g.brk[1][ey];
    const double hz = g.brk[2][ez + 1] - g.brk[2][ez];
    cx = hy * hz / (2.0 * hx);
    cy = hx * hz / (2.0 * hy);
    cz = hx * hy / (2.0 * hz);
  }
  const int I = ex * g.p + ta, Jn = ey * g.p + tb;
  const bool inIJ = valid && I >= 1 && I <= g.nix && Jn >= 1 && Jn <= g.niy;
  const long long base = inIJ ? (long long)(I - 1) + (long long)g.nix * (Jn - 1) : 0;
  const long long plane = (long long)g.nix * g.niy;
  double u[P1];
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    const int K = ez * g.p + c;
    u[c] = (inIJ && K >= 1 && K <= g.niz) ? in[base + plane * (K - 1)] : 0.0;
  }
  // z: Mg_z u and K1_z u
  {
    double m1[P1], k1[P1];
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      m1[c] = 0.0;
      k1[c] = 0.0;
    }
#pragma unroll
    for (int c = 0; c < P1; ++c)
#pragma unroll
      for (int cc = 0; cc < P1; ++cc) {
        m1[cc] = fma(sMg[cc * P1 + c], u[c], m1[cc]);
        k1[cc] = fma(sK1[cc * P1 + c], u[c], k1[cc]);
      }
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      S1[c * P2 + tb * P1 + ta] = m1[c];
      S2[c * P2 + tb * P1 + ta] = k1[c];
    }
  }
  __syncthreads();
  // y: thread (a = ta, b' = tb)
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    double A = 0.0, Bv = 0.0, Cv = 0.0;
#pragma unroll
    for (int b = 0; b < P1; ++b) {
      const double s1 = S1[c * P2 + b * P1 + ta];
      A = fma(sMg[tb * P1 + b], s1, A);
      Bv = fma(sK1[tb * P1 + b], s1, Bv);
      Cv = fma(sMg[tb * P1 + b], S2[c * P2 + b * P1 + ta], Cv);
    }
    S3[c * P2 + tb * P1 + ta] = A;
    S4[c * P2 + tb * P1 + ta] = cy * Bv + cz * Cv;
  }
  __syncthreads();
  double ppart = 0.0;
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    double m = 0.0, k = 0.0;
#pragma unroll
    for (int a2 = 0; a2 < P1; ++a2) {
      m = fma(sMg[ta * P1 + a2], S4[c * P2 + tb * P1 + a2], m);
      k = fma(sK1[ta * P1 + a2], S3[c * P2 + tb * P1 + a2], k);
    }
    const double y = m + cx * k;
    const int K = ez * g.p + c;
    if (inIJ && K >= 1 && K <= g.niz) {
      const long long idx = base + plane * (K - 1);
      out[idx] += y;
      ppart = fma(u[c], y, ppart);
    }
  }
  if (part) {
    const double s = block_sum(ppart, red);
    if (tid == 0) part[part_off + blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// Load vector out += (B^T)^(x)3 (J W f_q) (real), Eq. 19 right-hand side:
// x-lines of the Gauss-point field, then y, then z, scatter of the z-column.
// ---------------------------------------------------------------------------
template <int P1>
__global__ void __launch_bounds__(256) k_load(Geom g, const double* __restrict__ tab,
                                              const double* __restrict__ fq,
                                              double* __restrict__ out, double scale, int color,
                                              int weighted) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  double* sBT = reinterpret_cast<double*>(smem);
  double* sw = sBT + CS;
  double* S1 = sw + P1 + (size_t)threadIdx.y * 2 * P3;
  double* S2 = S1 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < CS; i += nthr) sBT[i] = tab[tab_off_csBT(P1) + i];
  for (int i = tid; i < P1; i += nthr) sw[i] = tab[tab_off_w(P1) + i];
  const int u = threadIdx.x % P1, v = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const bool valid = color_elem(g, color, (long long)blockIdx.x * blockDim.y + threadIdx.y, ex, ey, ez);
  __syncthreads();
  double col[P1], t[P1];
#pragma unroll
  for (int q = 0; q < P1; ++q) col[q] = 0.0;
  if (valid) {
    const double hx = g.brk[0][ex + 1] - g.brk[0][ex];
    const double hy = g.brk[1][ey + 1] - g.brk[1][ey];
    const double hz = g.brk[2][ez + 1] - g.brk[2][ez];
    const double Jw = weighted ? 0.125 * hx * hy * hz * scale * sw[u] * sw[v] : scale;
    const long long e = ex + (long long)g.nx * (ey + (long long)g.ny * ez);
    const double* fp = fq + e * P3 + v * P2 + u * P1;      // x-line (qy = u, qz = v)
#pragma unroll
    for (int q = 0; q < P1; ++q) col[q] = fp[q] * Jw * (weighted ? sw[q] : 1.0);
  }
  cs_apply<P1>(sBT, col, t);
  store_line(t, S1 + v * P2 + u * P1, 1);                 // [qz][qy][a]
  __syncthreads();
  load_line(col, S1 + v * P2 + u, P1);                    // y-line (a = u, qz = v)
  cs_apply<P1>(sBT, col, t);
  store_line(t, S2 + v * P2 + u, P1);                     // [qz][b][a]
  __syncthreads();
  load_line(col, S2 + v * P1 + u, P2);                    // z-line (a = u, b = v)
  cs_apply<P1>(sBT, col, t);
  const int I = ex * g.p + u, Jn = ey * g.p + v;
  const bool inIJ = valid && I >= 1 && I <= g.nix && Jn >= 1 && Jn <= g.niy;
  const long long base = inIJ ? (long long)(I - 1) + (long long)g.nix * (Jn - 1) : 0;
  const long long plane = (long long)g.nix * g.niy;
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    const int K = ez * g.p + c;
    if (inIJ && K >= 1 && K <= g.niz) out[base + plane * (K - 1)] += t[c];
  }
}

// Forward pass of one element: gathered z-column -> Gauss values on the thread's
// x-line (qy = u, qz = v).  S1, S2 must be free on entry.
template <int P1, typename V, typename T>
__device__ __forceinline__ void forward_lines(V (&col)[P1], V (&uq)[P1], V* S1, V* S2,
                                              const T* sB, int u, int v) {
  constexpr int P2 = P1 * P1;
  V t[P1];
  cs_apply<P1>(sB, col, t);
  store_line(t, S1 + v * P1 + u, P2);
  __syncthreads();
  load_line(col, S1 + v * P2 + u, P1);
  cs_apply<P1>(sB, col, t);
  store_line(t, S2 + v * P2 + u, P1);
  __syncthreads();
  load_line(col, S2 + v * P2 + u * P1, 1);
  cs_apply<P1>(sB, col, uq);
}

// ---------------------------------------------------------------------------
// Interpolation of a real nodal field to the Gauss points: f_q = B^(x)3 u_e
// ---------------------------------------------------------------------------
template <int P1>
__global__ void __launch_bounds__(256) k_interp(Geom g, const double* __restrict__ tab,
                                                const double* __restrict__ nodal,
                                                double* __restrict__ fq, double scale,
                                                int weighted) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  double* sB = reinterpret_cast<double*>(smem);
  double* S1 = sB + CS + (size_t)threadIdx.y * 2 * P3;
  double* S2 = S1 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < CS; i += nthr) sB[i] = tab[tab_off_csB(P1) + i];
  const int u = threadIdx.x % P1, v = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const bool valid = plain_elem(g, (long long)blockIdx.x * blockDim.y + threadIdx.y, ex, ey, ez);
  __syncthreads();
  const int I = ex * g.p + u, Jn = ey * g.p + v;
  const bool inIJ = valid && I >= 1 && I <= g.nix && Jn >= 1 && Jn <= g.niy;
  const long long base = inIJ ? (long long)(I - 1) + (long long)g.nix * (Jn - 1) : 0;
  const long long plane = (long long)g.nix * g.niy;
  double col[P1], uq[P1];
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    const int K = ez * g.p + c;
    col[c] = (inIJ && K >= 1 && K <= g.niz) ? nodal[base + plane * (K - 1)] : 0.0;
  }
  forward_lines<P1, double, double>(col, uq, S1, S2, sB, u, v);
  if (valid) {
    const long long e = ex + (long long)g.nx * (ey + (long long)g.ny * ez);
    double f = scale;
    if (weighted) {
      const double* w = tab + tab_off_w(P1);
      f *= 0.125 * (g.brk[0][ex + 1] - g.brk[0][ex]) * (g.brk[1][ey + 1] - g.brk[1][ey]) *
           (g.brk[2][ez + 1] - g.brk[2][ez]) * w[u] * w[v];
#pragma unroll
      for (int q = 0; q < P1; ++q) uq[q] *= f * w[q];
    } else if (f != 1.0) {
#pragma unroll
      for (int q = 0; q < P1; ++q) uq[q] *= f;
    }
    store_line(uq, fq + e * P3 + v * P2 + u * P1, 1);
  }
}

// ---------------------------------------------------------------------------
// Density rho(x_q) = sum_a occ_a |(B^(x)3 M^-1/2 psibar_a)(x_q)|^2   (Eq. 2)
// ---------------------------------------------------------------------------
template <int P1>
__global__ void __launch_bounds__(256) k_density(Geom g, const double* __restrict__ tab,
                                                 const double2* __restrict__ psi, int64_t stride,
                                                 int n_orb, const double* __restrict__ occ,
                                                 double* __restrict__ rho) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  typedef Cx<double> V;
  extern __shared__ __align__(16) unsigned char smem[];
  double* sB = reinterpret_cast<double*>(smem);
  const size_t off = (CS * sizeof(double) + 15) & ~size_t(15);
  V* S1 = reinterpret_cast<V*>(smem + off) + (size_t)threadIdx.y * 2 * P3;
  V* S2 = S1 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < CS; i += nthr) sB[i] = tab[tab_off_csB(P1) + i];
  const int u = threadIdx.x % P1, v = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const bool valid = plain_elem(g, (long long)blockIdx.x * blockDim.y + threadIdx.y, ex, ey, ez);
  __syncthreads();
  const int I = ex * g.p + u, Jn = ey * g.p + v;
  const bool inIJ = valid && I >= 1 && I <= g.nix && Jn >= 1 && Jn <= g.niy;
  const double sxy = inIJ ? g.s[0][I] * g.s[1][Jn] : 0.0;
  const long long base = inIJ ? (long long)(I - 1) + (long long)g.nix * (Jn - 1) : 0;
  const long long plane = (long long)g.nix * g.niy;
  double acc[P1];
#pragma unroll
  for (int q = 0; q < P1; ++q) acc[q] = 0.0;
  for (int o = 0; o < n_orb; ++o) {
    const double2* in = psi + (long long)o * stride;
    V col[P1], uq[P1];
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      const int K = ez * g.p + c;
      vzero(col[c]);
      if (inIJ && K >= 1 && K <= g.niz) {
        const double f = sxy * g.s[2][K];
        const double2 w2 = in[base + plane * (K - 1)];
        col[c].re = w2.x * f;
        col[c].im = w2.y * f;
      }
    }
    forward_lines<P1, V, double>(col, uq, S1, S2, sB, u, v);
    const double f = occ[o];
#pragma unroll
    for (int q = 0; q < P1; ++q) acc[q] += f * (uq[q].re * uq[q].re + uq[q].im * uq[q].im);
    __syncthreads();
  }
  if (valid) {
    const long long e = ex + (long long)g.nx * (ey + (long long)g.ny * ez);
    store_line(acc, rho + e * P3 + v * P2 + u * P1, 1);
  }
}

// Density in the double-float runs: the interpolation to the Gauss points is a
// cell-level contraction and runs in double-float (real, then imaginary part, as
// in the split element kernel); |psi_q|^2 is formed in double-float, rounded once
// to FP64 and accumulated over the orbitals in FP64.
template <int P1>
__global__ void __launch_bounds__(256) k_density_df(Geom g, const Df* __restrict__ tab,
                                                    const double2* __restrict__ psi, int64_t stride,
                                                    int n_orb, const double* __restrict__ occ,
                                                    double* __restrict__ rho) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  Df* sB = reinterpret_cast<Df*>(smem);
  const size_t off = (CS * sizeof(Df) + 15) & ~size_t(15);
  Df* S1 = reinterpret_cast<Df*>(smem + off) + (size_t)threadIdx.y * 2 * P3;
  Df* S2 = S1 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < CS; i += nthr) sB[i] = tab[tab_off_csB(P1) + i];
  const int u = threadIdx.x % P1, v = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const bool valid = plain_elem(g, (long long)blockIdx.x * blockDim.y + threadIdx.y, ex, ey, ez);
  __syncthreads();
  const int I = ex * g.p + u, Jn = ey * g.p + v;
  const bool inIJ = valid && I >= 1 && I <= g.nix && Jn >= 1 && Jn <= g.niy;
  const long long base = inIJ ? (long long)(I - 1) + (long long)g.nix * (Jn - 1) : 0;
  const long long plane = (long long)g.nix * g.niy;
  Df gsc[P1];   // Loewdin scales of this thread's z-column
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    const int K = ez * g.p + c;
    gsc[c] = from_d<Df>((inIJ && K >= 1 && K <= g.niz) ? g.s[0][I] * g.s[1][Jn] * g.s[2][K] : 0.0);
  }
  double acc[P1];
#pragma unroll
  for (int q = 0; q < P1; ++q) acc[q] = 0.0;
  for (int o = 0; o < n_orb; ++o) {
    const double2* in = psi + (long long)o * stride;
    Df ur[P1];
#pragma unroll 1
    for (int comp = 0; comp < 2; ++comp) {
      Df col[P1], uq[P1];
#pragma unroll
      for (int c = 0; c < P1; ++c) {
        const int K = ez * g.p + c;
        col[c] = Df{0.f, 0.f};
        if (inIJ && K >= 1 && K <= g.niz) {
          const double2 w2 = in[base + plane * (K - 1)];
          col[c] = df_mul(d2df_bits(comp ? w2.y : w2.x), gsc[c]);
        }
      }
      forward_lines<P1, Df, Df>(col, uq, S1, S2, sB, u, v);
      if (comp == 0) {
#pragma unroll
        for (int q = 0; q < P1; ++q) ur[q] = uq[q];
      } else {
        const double f = occ[o];
#pragma unroll
        for (int q = 0; q < P1; ++q) {
          const Df m2 = df_add(df_mul(ur[q], ur[q]), df_mul(uq[q], uq[q]));
          acc[q] = fma(f, f2d_bits(m2.hi) + f2d_bits(m2.lo), acc[q]);
        }
      }
      __syncthreads();
    }
  }
  if (valid) {
    const long long e = ex + (long long)g.nx * (ey + (long long)g.ny * ez);
    store_line(acc, rho + e * P3 + v * P2 + u * P1, 1);
  }
}

// ---------------------------------------------------------------------------
// Density adjoint: element-local (B^T)^(x)3 [2 occ_a g_rho psi_a(x_q)] for every
// orbital (the assembly and the Loewdin scale follow in k_assemble).
// ---------------------------------------------------------------------------
template <int P1>
__global__ void __launch_bounds__(256) k_dens_adj(Geom g, const double* __restrict__ tab,
                                                  const double2* __restrict__ psi, int64_t stride,
                                                  int n_orb, const double* __restrict__ occ,
                                                  const double* __restrict__ grho,
                                                  Cx<double>* __restrict__ ev) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  typedef Cx<double> V;
  extern __shared__ __align__(16) unsigned char smem[];
  double* sB = reinterpret_cast<double*>(smem);
  double* sBT = sB + CS;
  const size_t off = (2 * CS * sizeof(double) + 15) & ~size_t(15);
  V* S1 = reinterpret_cast<V*>(smem + off) + (size_t)threadIdx.y * 2 * P3;
  V* S2 = S1 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < 2 * CS; i += nthr) sB[i] = tab[tab_off_csB(P1) + i];
  const int u = threadIdx.x % P1, v = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const long long eidx = (long long)blockIdx.x * blockDim.y + threadIdx.y;
  const bool valid = plain_elem(g, eidx, ex, ey, ez);
  const long long n_elem = (long long)g.nx * g.ny * g.nz;
  __syncthreads();
  const int I = ex * g.p + u, Jn = ey * g.p + v;
  const bool inIJ = valid && I >= 1 && I <= g.nix && Jn >= 1 && Jn <= g.niy;
  const double sxy = inIJ ? g.s[0][I] * g.s[1][Jn] : 0.0;
  const long long base = inIJ ? (long long)(I - 1) + (long long)g.nix * (Jn - 1) : 0;
  const long long plane = (long long)g.nix * g.niy;
  double gx[P1];
#pragma unroll
  for (int q = 0; q < P1; ++q) gx[q] = valid ? grho[eidx * P3 + v * P2 + u * P1 + q] : 0.0;
  for (int o = 0; o < n_orb; ++o) {
    const double2* in = psi + (long long)o * stride;
    V col[P1], uq[P1], t[P1];
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      const int K = ez * g.p + c;
      vzero(col[c]);
      if (inIJ && K >= 1 && K <= g.niz) {
        const double f = sxy * g.s[2][K];
        const double2 w2 = in[base + plane * (K - 1)];
        col[c].re = w2.x * f;
        col[c].im = w2.y * f;
      }
    }
    forward_lines<P1, V, double>(col, uq, S1, S2, sB, u, v);
    const double f2 = 2.0 * occ[o];
#pragma unroll
    for (int q = 0; q < P1; ++q) uq[q] = vscale(f2 * gx[q], uq[q]);
    __syncthreads();                                       // S1/S2 free again
    cs_apply<P1>(sBT, uq, t);                              // x-line -> B^T along x
    store_line(t, S1 + v * P2 + u * P1, 1);                // [qz][qy][a]
    __syncthreads();
    load_line(col, S1 + v * P2 + u, P1);                   // y-line (a = u, qz = v)
    cs_apply<P1>(sBT, col, t);
    store_line(t, S2 + v * P2 + u, P1);                    // [qz][b][a]
    __syncthreads();
    load_line(col, S2 + v * P1 + u, P2);                   // z-line (a = u, b = v)
    cs_apply<P1>(sBT, col, t);
    if (valid) store_line(t, ev + ((long long)o * n_elem + eidx) * P3 + v * P1 + u, P2);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// g_q += coef wJ_q sum_a Im(conj(mu_a(x_q)) phi_a(x_q))   (Frechet term of the
// exponential with respect to the potential at the Gauss points)
// ---------------------------------------------------------------------------
template <int P1>
__global__ void __launch_bounds__(256) k_cross(Geom g, const double* __restrict__ tab,
                                               const double2* __restrict__ mu,
                                               const double2* __restrict__ phi, int64_t stride,
                                               int n_orb, double coef, double* __restrict__ gq) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  typedef Cx<double> V;
  extern __shared__ __align__(16) unsigned char smem[];
  double* sB = reinterpret_cast<double*>(smem);
  double* sw = sB + CS;
  const size_t off = ((CS + P1) * sizeof(double) + 15) & ~size_t(15);
  V* S1 = reinterpret_cast<V*>(smem + off) + (size_t)threadIdx.y * 2 * P3;
  V* S2 = S1 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < CS; i += nthr) sB[i] = tab[tab_off_csB(P1) + i];
  for (int i = tid; i < P1; i += nthr) sw[i] = tab[tab_off_w(P1) + i];
  const int u = threadIdx.x % P1, v = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const long long eidx = (long long)blockIdx.x * blockDim.y + threadIdx.y;
  const bool valid = plain_elem(g, eidx, ex, ey, ez);
  __syncthreads();
  const int I = ex * g.p + u, Jn = ey * g.p + v;
  const bool inIJ = valid && I >= 1 && I <= g.nix && Jn >= 1 && Jn <= g.niy;
  const double sxy = inIJ ? g.s[0][I] * g.s[1][Jn] : 0.0;
  const long long base = inIJ ? (long long)(I - 1) + (long long)g.nix * (Jn - 1) : 0;
  const long long plane = (long long)g.nix * g.niy;
  double acc[P1];
#pragma unroll
  for (int q = 0; q < P1; ++q) acc[q] = 0.0;
  for (int o = 0; o < n_orb; ++o) {
    V cm[P1], cp[P1], mq[P1], pq[P1];
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      const int K = ez * g.p + c;
      vzero(cm[c]);
      vzero(cp[c]);
      if (inIJ && K >= 1 && K <= g.niz) {
        const double f = sxy * g.s[2][K];
        const long long idx = (long long)o * stride + base + plane * (K - 1);
        const double2 a = mu[idx], b = phi[idx];
        cm[c].re = a.x * f;
        cm[c].im = a.y * f;
        cp[c].re = b.x * f;
        cp[c].im = b.y * f;
      }
    }
    forward_lines<P1, V, double>(cm, mq, S1, S2, sB, u, v);
    __syncthreads();
    forward_lines<P1, V, double>(cp, pq, S1, S2, sB, u, v);
#pragma unroll
    for (int q = 0; q < P1; ++q) acc[q] += mq[q].re * pq[q].im - mq[q].im * pq[q].re;
    __syncthreads();
  }
  if (valid) {
    const double J = 0.125 * (g.brk[0][ex + 1] - g.brk[0][ex]) * (g.brk[1][ey + 1] - g.brk[1][ey]) *
                     (g.brk[2][ez + 1] - g.brk[2][ez]);
    double* gp = gq + eidx * P3 + v * P2 + u * P1;
#pragma unroll
    for (int q = 0; q < P1; ++q) gp[q] += coef * J * sw[u] * sw[v] * sw[q] * acc[q];
  }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
long long color_max(const tdks_ctx* c) {
  return (long long)((c->nx + 1) / 2) * ((c->ny + 1) / 2) * ((c->nz + 1) / 2);
}

template <int P1>
int blocks_per_color_t(const tdks_ctx* c) {
  return (int)((color_max(c) + Cfg<P1>::E - 1) / Cfg<P1>::E);
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int P1>
int elem_blocks_t(const tdks_ctx* c) {
  return (int)((c->n_elem + Cfg<P1>::E - 1) / Cfg<P1>::E);
}

template <int P1, typename T, bool kBF = false>
tdks_status hbar_t(tdks_ctx* c, const ApplyArgs& a) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3, E = Cfg<P1>::E;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  constexpr bool kSplit = std::is_same<T, Df>::value || (std::is_same<T, float>::value && !kBF);
  constexpr size_t elem = kSplit ? (size_t)SplitLayout<P1, T>::ES * sizeof(T) : 2 * P3 * sizeof(Cx<T>);
  const size_t lines_end = (((3 * CS + P1) * sizeof(T) + 15) & ~size_t(15)) + (size_t)E * elem;
  const size_t smem = kSplit ? pf_offset(lines_end) + (size_t)E * P2 * P1 * sizeof(double2)   // + prefetch buffer
                             : lines_end;
  // stage study (tdks_set_f32_stages): double-float applies at p = 4 and 6 only
  constexpr bool kStudyOk = std::is_same<T, Df>::value && (P1 == 5 || P1 == 7);
  const bool study = std::is_same<T, Df>::value && c->f32_stages != 0u;
  if (study && !kStudyOk)
    return tdks_fail(c, TDKS_ERR_ARG, "the per-stage precision study covers double-float applies at p = 4 and 6");
  if constexpr (kSplit) {
    TDKS_CU(c, cudaFuncSetAttribute(k_hbar_split<P1, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if constexpr (kStudyOk)
      if (study)
        TDKS_CU(c, cudaFuncSetAttribute(k_hbar_split<P1, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
  } else {
    TDKS_CU(c, set_smem(k_hbar<P1, T, kBF>, smem));
  }
  const size_t need = (size_t)a.n_orb * c->n_elem * P3 * sizeof(Cx<T>);
  if (need > c->evec_bytes) {
    cudaFree(c->d_evec);
    c->d_evec = nullptr;
    c->evec_bytes = 0;
    if (cudaMalloc(&c->d_evec, need) != cudaSuccess) {
      cudaGetLastError();
      return tdks_fail(c, TDKS_ERR_NOMEM, "element-result buffer");
    }
    c->evec_bytes = need;
  }
  Cx<T>* ev = static_cast<Cx<T>*>(c->d_evec);
  const int bpe = elem_blocks_t<P1>(c);
  // orbitals per CTA: V and geometry are reused across them; keep >= 8 CTAs per SM
  // (about four waves at two CTAs per SM, so the last partial wave costs little)
  int opc = 1;
  while (opc < a.n_orb && (long long)bpe * ((a.n_orb + 2 * opc - 1) / (2 * opc)) >= 8 * 152) opc *= 2;
  if (c->opc_force > 0) opc = c->opc_force < a.n_orb ? c->opc_force : a.n_orb;
  const int ochunks = (a.n_orb + opc - 1) / opc;
  const T* tab = std::is_same<T, double>::value ? (const T*)c->d_tab
                 : std::is_same<T, float>::value ? (const T*)(kBF ? c->d_tabbf : c->d_tabf)
                                                 : (const T*)c->d_tabdf;
  const Geom g = tdks_geom(c);
  if (c->kb) TDKS_TRY(kb_project(c, a));
  if constexpr (kStudyOk) {
    if (study)
      k_hbar_split<P1, T, true><<<dim3(bpe, ochunks), dim3(P2, E), smem, c->stream>>>(g, tab, c->d_vks, a, opc, ev,
                                                                                     c->f32_stages);
    else
      k_hbar_split<P1, T><<<dim3(bpe, ochunks), dim3(P2, E), smem, c->stream>>>(g, tab, c->d_vks, a, opc, ev, 0u);
  } else if constexpr (kSplit)
    k_hbar_split<P1, T><<<dim3(bpe, ochunks), dim3(P2, E), smem, c->stream>>>(g, tab, c->d_vks, a, opc, ev, 0u);
  else
    k_hbar<P1, T, kBF><<<dim3(bpe, ochunks), dim3(P2, E), smem, c->stream>>>(g, tab, c->d_vks, a, opc, ev);
  if (a.lanczos && a.kry && a.part) {
    k_alpha<<<a.n_orb, 256, 0, c->stream>>>(a.kry, a.part, a.part_stride, bpe, a.kj);
    if (c->kb) TDKS_TRY(kb_alpha(c, a));
  }
  const int gx = assemble_blocks(c, a.n_orb);
  k_assemble<P1, T><<<dim3(gx, a.n_orb), 128, 0, c->stream>>>(g, ev, a);
  if (c->kb) TDKS_TRY(kb_add(c, a));
  c->n_launch += (a.lanczos && a.kry && a.part) ? 3 : 2;
  c->n_apply_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

template <int P1>
tdks_status stiff_t(tdks_ctx* c, const double* in, double* out, double* part, const CgState* cg) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3, E = Cfg<P1>::E;
  const size_t smem = (2 * P2 + (size_t)E * 4 * P3) * sizeof(double);
  TDKS_CU(c, set_smem(k_stiff<P1>, smem));
  const int bpc = blocks_per_color_t<P1>(c);
  dim3 block(P2, E), grid(bpc);
  const Geom g = tdks_geom(c);
  for (int color = 0; color < 8; ++color)
    k_stiff<P1><<<grid, block, smem, c->stream>>>(g, c->d_tab, in, out, part, color * bpc, cg, color);
  c->n_launch += 8;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

template <int P1>
tdks_status load_t(tdks_ctx* c, const double* fq, double* out, double scale, int weighted) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3, E = Cfg<P1>::E;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  const size_t smem = (CS + P1 + (size_t)E * 2 * P3) * sizeof(double);
  TDKS_CU(c, set_smem(k_load<P1>, smem));
  dim3 block(P2, E), grid(blocks_per_color_t<P1>(c));
  const Geom g = tdks_geom(c);
  for (int color = 0; color < 8; ++color)
    k_load<P1><<<grid, block, smem, c->stream>>>(g, c->d_tab, fq, out, scale, color, weighted);
  c->n_launch += 8;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

template <int P1>
tdks_status interp_t(tdks_ctx* c, const double* nodal, double* fq, double scale, int weighted) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3, E = Cfg<P1>::E;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  const size_t smem = (CS + (size_t)E * 2 * P3) * sizeof(double);
  TDKS_CU(c, set_smem(k_interp<P1>, smem));
  dim3 block(P2, E), grid((unsigned)((c->n_elem + E - 1) / E));
  k_interp<P1><<<grid, block, smem, c->stream>>>(tdks_geom(c), c->d_tab, nodal, fq, scale, weighted);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

template <int P1>
tdks_status density_t(tdks_ctx* c, const double2* psi, int n_orb, double* rho, int prec) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3, E = Cfg<P1>::E;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  dim3 block(P2, E), grid((unsigned)((c->n_elem + E - 1) / E));
  if (prec == TDKS_DF64) {
    const size_t smem = ((CS * sizeof(Df) + 15) & ~size_t(15)) + (size_t)E * 2 * P3 * sizeof(Df);
    TDKS_CU(c, set_smem(k_density_df<P1>, smem));
    k_density_df<P1><<<grid, block, smem, c->stream>>>(tdks_geom(c), (const Df*)c->d_tabdf, psi, c->n_int,
                                                      n_orb, c->d_occ, rho);
  } else {
    const size_t smem = ((CS * sizeof(double) + 15) & ~size_t(15)) + (size_t)E * 2 * P3 * sizeof(Cx<double>);
    TDKS_CU(c, set_smem(k_density<P1>, smem));
    k_density<P1><<<grid, block, smem, c->stream>>>(tdks_geom(c), c->d_tab, psi, c->n_int, n_orb,
                                                   c->d_occ, rho);
  }
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

#define TDKS_DISPATCH(P1v, expr)                                   \
  switch (P1v) {                                                   \
    case 2: { constexpr int P1 = 2; return expr; }                 \
    case 3: { constexpr int P1 = 3; return expr; }                 \
    case 4: { constexpr int P1 = 4; return expr; }                 \
    case 5: { constexpr int P1 = 5; return expr; }                 \
    case 6: { constexpr int P1 = 6; return expr; }                 \
    case 7: { constexpr int P1 = 7; return expr; }                 \
    case 8: { constexpr int P1 = 8; return expr; }                 \
    case 9: { constexpr int P1 = 9; return expr; }                 \
    default: break;                                                \
  }

}  // namespace

template <int P1>
tdks_status dens_adj_t(tdks_ctx* c, const double2* psi, int n_orb, const double* grho, double2* lam,
                       int accumulate) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3, E = Cfg<P1>::E;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  const size_t smem = ((2 * CS * sizeof(double) + 15) & ~size_t(15)) + (size_t)E * 2 * P3 * sizeof(Cx<double>);
  TDKS_CU(c, set_smem(k_dens_adj<P1>, smem));
  const size_t need = (size_t)n_orb * c->n_elem * P3 * sizeof(Cx<double>);
  if (need > c->evec_bytes) {
    cudaFree(c->d_evec);
    c->d_evec = nullptr;
    c->evec_bytes = 0;
    if (cudaMalloc(&c->d_evec, need) != cudaSuccess) {
      cudaGetLastError();
      return tdks_fail(c, TDKS_ERR_NOMEM, "element-result buffer");
    }
    c->evec_bytes = need;
  }
  Cx<double>* ev = static_cast<Cx<double>*>(c->d_evec);
  const Geom g = tdks_geom(c);
  k_dens_adj<P1><<<dim3(elem_blocks_t<P1>(c)), dim3(P2, E), smem, c->stream>>>(
      g, c->d_tab, psi, c->n_int, n_orb, c->d_occ, grho, ev);
  ApplyArgs a{psi, c->n_int, lam, c->n_int, n_orb, nullptr, 0, nullptr, 0, 0, nullptr, 0, nullptr, 0,
              accumulate};
  k_assemble<P1, double><<<dim3(assemble_blocks(c, n_orb), n_orb), 128, 0, c->stream>>>(g, ev, a);
  c->n_launch += 2;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

template <int P1>
tdks_status cross_t(tdks_ctx* c, const double2* mu, const double2* phi, int n_orb, double coef,
                    double* gq) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3, E = Cfg<P1>::E;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  const size_t smem = (((CS + P1) * sizeof(double) + 15) & ~size_t(15)) + (size_t)E * 2 * P3 * sizeof(Cx<double>);
  TDKS_CU(c, set_smem(k_cross<P1>, smem));
  k_cross<P1><<<dim3(elem_blocks_t<P1>(c)), dim3(P2, E), smem, c->stream>>>(
      tdks_geom(c), c->d_tab, mu, phi, c->n_int, n_orb, coef, gq);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

tdks_status ensure_evec(tdks_ctx* c, int n_orb) {
  const size_t need = (size_t)n_orb * c->n_elem * c->P1 * c->P1 * c->P1 * sizeof(Cx<double>);
  if (need <= c->evec_bytes) return TDKS_OK;
  cudaFree(c->d_evec);
  c->d_evec = nullptr;
  c->evec_bytes = 0;
  if (cudaMalloc(&c->d_evec, need) != cudaSuccess) {
    cudaGetLastError();
    return tdks_fail(c, TDKS_ERR_NOMEM, "element-result buffer");
  }
  c->evec_bytes = need;
  return TDKS_OK;
}

int hbar_blocks_per_color(const tdks_ctx* c) {
  int b = 0;
  switch (c->P1) {
    case 2: b = elem_blocks_t<2>(c); break;
    case 3: b = elem_blocks_t<3>(c); break;
    case 4: b = elem_blocks_t<4>(c); break;
    case 5: b = elem_blocks_t<5>(c); break;
    case 6: b = elem_blocks_t<6>(c); break;
    case 7: b = elem_blocks_t<7>(c); break;
    case 8: b = elem_blocks_t<8>(c); break;
    case 9: b = elem_blocks_t<9>(c); break;
    default: break;
  }
  const int bs = stiff_blocks_per_color(c);
  return b > bs ? b : bs;
}

int stiff_blocks_per_color(const tdks_ctx* c) {
  TDKS_DISPATCH(c->P1, blocks_per_color_t<P1>(c));
  return 0;
}

int assemble_blocks(const tdks_ctx* c, int n_orb) {
  const int rows = c->Ni[1] * c->Ni[2];
  // several waves of 128-thread blocks over all orbitals, so the last partial wave is
  // a small share of the launch (at most 2048 partials per orbital)
  int gx = 8192 / (n_orb > 0 ? n_orb : 1);
  if (gx < 128) gx = 128;
  if (gx > 2048) gx = 2048;
  return rows < gx ? rows : gx;
}

tdks_status launch_hbar_apply(tdks_ctx* c, const ApplyArgs& a, int prec) {
  if (prec == TDKS_FP32) {
    TDKS_DISPATCH(c->P1, (hbar_t<P1, float>(c, a)));
  } else if (prec == TDKS_BF16) {
    TDKS_DISPATCH(c->P1, (hbar_t<P1, float, true>(c, a)));
  } else if (prec == TDKS_DF64) {
    TDKS_DISPATCH(c->P1, (hbar_t<P1, Df>(c, a)));
  } else {
    TDKS_DISPATCH(c->P1, (hbar_t<P1, double>(c, a)));
  }
  return tdks_fail(c, TDKS_ERR_ARG, "unsupported degree");
}

tdks_status launch_stiffness(tdks_ctx* c, const double* in, double* out, double* part,
                             const CgState* cg) {
  TDKS_DISPATCH(c->P1, (stiff_t<P1>(c, in, out, part, cg)));
  return tdks_fail(c, TDKS_ERR_ARG, "unsupported degree");
}

tdks_status launch_load_vector(tdks_ctx* c, const double* f_q, double* out, double scale,
                               int weighted) {
  TDKS_DISPATCH(c->P1, (load_t<P1>(c, f_q, out, scale, weighted)));
  return tdks_fail(c, TDKS_ERR_ARG, "unsupported degree");
}

tdks_status launch_interp(tdks_ctx* c, const double* nodal, double* f_q, double scale,
                          int weighted) {
  TDKS_DISPATCH(c->P1, (interp_t<P1>(c, nodal, f_q, scale, weighted)));
  return tdks_fail(c, TDKS_ERR_ARG, "unsupported degree");
}

tdks_status launch_density_adjoint(tdks_ctx* c, const double2* psi, int n_orb, const double* g_rho,
                                   double2* lam, int accumulate) {
  TDKS_DISPATCH(c->P1, (dens_adj_t<P1>(c, psi, n_orb, g_rho, lam, accumulate)));
  return tdks_fail(c, TDKS_ERR_ARG, "unsupported degree");
}

tdks_status launch_cross(tdks_ctx* c, const double2* mu, const double2* phi, int n_orb, double coef,
                         double* g_q) {
  TDKS_DISPATCH(c->P1, (cross_t<P1>(c, mu, phi, n_orb, coef, g_q)));
  return tdks_fail(c, TDKS_ERR_ARG, "unsupported degree");
}

tdks_status launch_density(tdks_ctx* c, const double2* psi, int n_orb, double* rho_q, int prec) {
  TDKS_DISPATCH(c->P1, (density_t<P1>(c, psi, n_orb, rho_q, prec)));
  return tdks_fail(c, TDKS_ERR_ARG, "unsupported degree");
}

// ---- batched apply launchers ------------------------------------------------
template <int P1, typename T>
static size_t hbar_batch_smem_t(int E) {
  constexpr int P3 = Cfg<P1>::P3;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  constexpr bool kSplit = !std::is_same<T, double>::value;
  constexpr size_t elem = kSplit ? (size_t)SplitLayout<P1, T>::ES * sizeof(T) : 2 * P3 * sizeof(Cx<T>);
  const size_t lines_end = (((3 * CS + P1) * sizeof(T) + 15) & ~size_t(15)) + (size_t)E * elem;
  return kSplit ? pf_offset(lines_end) + (size_t)E * Cfg<P1>::P2 * P1 * sizeof(double2)   // + prefetch buffer
                : lines_end;
}

template <int P1>
static size_t hbar_batch_smem_p(int prec, int E) {
  if (prec == TDKS_FP32) return hbar_batch_smem_t<P1, float>(E);
  if (prec == TDKS_DF64) return hbar_batch_smem_t<P1, Df>(E);
  return hbar_batch_smem_t<P1, double>(E);
}

size_t hbar_batch_smem(int P1, int prec, int E) {
  switch (P1) {
    case 2: return hbar_batch_smem_p<2>(prec, E);
    case 3: return hbar_batch_smem_p<3>(prec, E);
    case 4: return hbar_batch_smem_p<4>(prec, E);
    case 5: return hbar_batch_smem_p<5>(prec, E);
    case 6: return hbar_batch_smem_p<6>(prec, E);
    case 7: return hbar_batch_smem_p<7>(prec, E);
    case 8: return hbar_batch_smem_p<8>(prec, E);
    case 9: return hbar_batch_smem_p<9>(prec, E);
    default: return 0;
  }
}

template <int P1, typename T>
static cudaError_t hbar_batch_launch_t(const BSys* sys, const BItem* items, int n_items, int E,
                                       int grid, const void* tab, int* qctr, cudaStream_t st, int* occ) {
  const size_t smem = hbar_batch_smem_t<P1, T>(E);
  // split body for double-float (see k_hbar_split), complex body otherwise
  void (*kern)(const BSys*, const BItem*, int, const T*, int*);
  if constexpr (!std::is_same<T, double>::value) kern = k_hbar_batch_split<P1, T>;
  else kern = k_hbar_batch<P1, T>;
  // the kernel also holds ~330 B of static shared memory: opt in for any large size
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, Cfg<P1>::P2 * E, smem);
  if (n_items <= 0) return cudaSuccess;
  kern<<<grid, dim3(Cfg<P1>::P2, E), smem, st>>>(sys, items, n_items, static_cast<const T*>(tab), qctr);
  return cudaGetLastError();
}

template <int P1>
static cudaError_t hbar_batch_p(int prec, const BSys* sys, const BItem* items, int n_items, int E,
                                int grid, const void* tab, int* qctr, cudaStream_t st, int* occ) {
  if (E < 1 || Cfg<P1>::P2 * E > 256) return cudaErrorInvalidValue;
  if (prec == TDKS_FP32) return hbar_batch_launch_t<P1, float>(sys, items, n_items, E, grid, tab, qctr, st, occ);
  if (prec == TDKS_DF64) return hbar_batch_launch_t<P1, Df>(sys, items, n_items, E, grid, tab, qctr, st, occ);
  return hbar_batch_launch_t<P1, double>(sys, items, n_items, E, grid, tab, qctr, st, occ);
}

static cudaError_t hbar_batch_dispatch(int P1, int prec, const BSys* sys, const BItem* items,
                                       int n_items, int E, int grid, const void* tab, int* qctr,
                                       cudaStream_t st, int* occ) {
  switch (P1) {
    case 2: return hbar_batch_p<2>(prec, sys, items, n_items, E, grid, tab, qctr, st, occ);
    case 3: return hbar_batch_p<3>(prec, sys, items, n_items, E, grid, tab, qctr, st, occ);
    case 4: return hbar_batch_p<4>(prec, sys, items, n_items, E, grid, tab, qctr, st, occ);
    case 5: return hbar_batch_p<5>(prec, sys, items, n_items, E, grid, tab, qctr, st, occ);
    case 6: return hbar_batch_p<6>(prec, sys, items, n_items, E, grid, tab, qctr, st, occ);
    case 7: return hbar_batch_p<7>(prec, sys, items, n_items, E, grid, tab, qctr, st, occ);
    case 8: return hbar_batch_p<8>(prec, sys, items, n_items, E, grid, tab, qctr, st, occ);
    case 9: return hbar_batch_p<9>(prec, sys, items, n_items, E, grid, tab, qctr, st, occ);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t hbar_batch_occupancy(int P1, int prec, int E, int* blocks_per_sm) {
  *blocks_per_sm = 0;
  return hbar_batch_dispatch(P1, prec, nullptr, nullptr, 0, E, 0, nullptr, nullptr, nullptr, blocks_per_sm);
}

cudaError_t launch_hbar_batch(int P1, int prec, const BSys* sys, const BItem* items, int n_items,
                              int E, int grid, const void* tab, int* qctr, cudaStream_t st) {
  return hbar_batch_dispatch(P1, prec, sys, items, n_items, E, grid, tab, qctr, st, nullptr);
}

cudaError_t launch_balpha(const BSys* sys, const BOrb* orbs, int n_orbs, cudaStream_t st) {
  if (n_orbs <= 0) return cudaSuccess;
  k_balpha<<<n_orbs, 256, 0, st>>>(sys, orbs);
  return cudaGetLastError();
}

template <int P1>
static cudaError_t bassemble_p(int prec, const BSys* sys, const BRow* rows, int n_rows, cudaStream_t st) {
  if (prec == TDKS_FP32) k_bassemble<P1, float><<<n_rows, 128, 0, st>>>(sys, rows);
  else if (prec == TDKS_DF64) k_bassemble<P1, Df><<<n_rows, 128, 0, st>>>(sys, rows);
  else if (prec == TDKS_MIXED) {   // each orbital's rows in the type of its last product
    k_bassemble<P1, Df><<<n_rows, 128, 0, st>>>(sys, rows);
    k_bassemble<P1, float><<<n_rows, 128, 0, st>>>(sys, rows);
  } else k_bassemble<P1, double><<<n_rows, 128, 0, st>>>(sys, rows);
  return cudaGetLastError();
}

cudaError_t launch_bassemble(int P1, int prec, const BSys* sys, const BRow* rows, int n_rows, cudaStream_t st) {
  if (n_rows <= 0) return cudaSuccess;
  switch (P1) {
    case 2: return bassemble_p<2>(prec, sys, rows, n_rows, st);
    case 3: return bassemble_p<3>(prec, sys, rows, n_rows, st);
    case 4: return bassemble_p<4>(prec, sys, rows, n_rows, st);
    case 5: return bassemble_p<5>(prec, sys, rows, n_rows, st);
    case 6: return bassemble_p<6>(prec, sys, rows, n_rows, st);
    case 7: return bassemble_p<7>(prec, sys, rows, n_rows, st);
    case 8: return bassemble_p<8>(prec, sys, rows, n_rows, st);
    case 9: return bassemble_p<9>(prec, sys, rows, n_rows, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int P1>
static tdks_status hbar_gll_t(tdks_ctx* c, const double2* psi, const double* vn, double2* out, int n_orb) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3, E = Cfg<P1>::E;
  constexpr int CS = 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1;
  const size_t smem = (((CS + P1) * sizeof(double) + 15) & ~size_t(15)) + (size_t)E * 2 * P3 * sizeof(Cx<double>);
  TDKS_CU(c, cudaFuncSetAttribute(k_hbar_gll<P1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const size_t need = (size_t)n_orb * c->n_elem * P3 * sizeof(Cx<double>);
  if (need > c->evec_bytes) {
    cudaFree(c->d_evec);
    c->d_evec = nullptr;
    c->evec_bytes = 0;
    if (cudaMalloc(&c->d_evec, need) != cudaSuccess) {
      cudaGetLastError();
      return tdks_fail(c, TDKS_ERR_NOMEM, "element-result buffer");
    }
    c->evec_bytes = need;
  }
  Cx<double>* ev = static_cast<Cx<double>*>(c->d_evec);
  const int bpe = elem_blocks_t<P1>(c);
  int opc = 1;
  while (opc < n_orb && (long long)bpe * ((n_orb + 2 * opc - 1) / (2 * opc)) >= 8 * 152) opc *= 2;
  const Geom g = tdks_geom(c);
  k_hbar_gll<P1><<<dim3(bpe, (n_orb + opc - 1) / opc), dim3(P2, E), smem, c->stream>>>(g, c->d_tab, psi, c->n_int,
                                                                                   n_orb, opc, ev);
  ApplyArgs a{psi, c->n_int, out, c->n_int, n_orb, nullptr, 0, nullptr, 0, 0, nullptr, 0, nullptr, 0, 0};
  k_assemble<P1, double><<<dim3(assemble_blocks(c, n_orb), n_orb), 128, 0, c->stream>>>(g, ev, a);
  k_diag_add<<<608, 256, 0, c->stream>>>(c->n_int, n_orb, vn, psi, out);
  c->n_launch += 3;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

tdks_status launch_hbar_gll(tdks_ctx* c, const double2* psi, const double* v_nodes, double2* out,
                            int n_orb) {
  TDKS_DISPATCH(c->P1, (hbar_gll_t<P1>(c, psi, v_nodes, out, n_orb)));
  return tdks_fail(c, TDKS_ERR_ARG, "unsupported degree");
}
