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

// ---------------------------------------------------------------------------
// Hbar psibar, complex, contraction type T (double or float)
// ---------------------------------------------------------------------------
template <int P1, typename T>
__global__ void __launch_bounds__(256) k_hbar(Geom g, const T* __restrict__ tab,
                                              const double* __restrict__ vks, ApplyArgs a,
                                              int color, int orb_per_cta, int part_off) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3;
  typedef Cx<T> V;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[8];
  T* sB = reinterpret_cast<T*>(smem);
  T* sK = sB + P2;
  T* sw = sK + P2;
  const size_t off = ((2 * P2 + P1) * sizeof(T) + 15) & ~size_t(15);
  V* S1 = reinterpret_cast<V*>(smem + off) + (size_t)threadIdx.y * 2 * P3;
  V* S2 = S1 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < 2 * P2 + P1; i += nthr) sB[i] = tab[i];
  const int ta = threadIdx.x % P1, tb = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const bool valid = color_elem(g, color, (long long)blockIdx.x * blockDim.y + threadIdx.y, ex, ey, ez);
  __syncthreads();

  T ckx = T(0), cky = T(0), ckz = T(0);
  T vcol[P1];
#pragma unroll
  for (int q = 0; q < P1; ++q) vcol[q] = T(0);
  if (valid) {
    const double hx = g.brk[0][ex + 1] - g.brk[0][ex];
    const double hy = g.brk[1][ey + 1] - g.brk[1][ey];
    const double hz = g.brk[2][ez + 1] - g.brk[2][ez];
    const double J = 0.125 * hx * hy * hz;
    ckx = T(hy * hz / (4.0 * hx));
    cky = T(hx * hz / (4.0 * hy));
    ckz = T(hx * hy / (4.0 * hz));
    const long long e = ex + (long long)g.nx * (ey + (long long)g.ny * ez);
    const double* vp = vks + e * P3 + tb * P1 + ta;
    const double wab = J * (double)sw[ta] * (double)sw[tb];
#pragma unroll
    for (int q = 0; q < P1; ++q) vcol[q] = T(vp[q * P2] * wab * (double)sw[q]);
  }
  const int I = ex * g.p + ta, Jn = ey * g.p + tb;
  const bool inIJ = valid && I >= 1 && I <= g.nix && Jn >= 1 && Jn <= g.niy;
  const double sxy = inIJ ? g.s[0][I] * g.s[1][Jn] : 0.0;
  const long long base = inIJ ? (long long)(I - 1) + (long long)g.nix * (Jn - 1) : 0;
  const long long plane = (long long)g.nix * g.niy;
  const T wa = sw[ta], wb = sw[tb];

  for (int oo = 0; oo < orb_per_cta; ++oo) {
    const int o = blockIdx.y * orb_per_cta + oo;
    if (o >= a.n_orb) break;
    double sc = 1.0;
    if (a.kry) {
      if (a.kry[o].status != KRY_ACTIVE) continue;
      sc = a.kry[o].s[a.kj];
    }
    const double2* in = a.in_base + (long long)o * a.in_stride;
    V u[P1];
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      const int K = ez * g.p + c;
      vzero(u[c]);
      if (inIJ && K >= 1 && K <= g.niz) {
        const double f = sxy * g.s[2][K] * sc;
        const double2 v = in[base + plane * (K - 1)];
        u[c].re = T(v.x * f);
        u[c].im = T(v.y * f);
      }
    }
    V uq[P1];
    forward3<P1, V, T>(u, uq, S1, S2, sB, ta, tb);
#pragma unroll
    for (int q = 0; q < P1; ++q) S1[q * P2 + tb * P1 + ta] = uq[q];
    __syncthreads();
    V r[P1];
    double apart = 0.0;
#pragma unroll
    for (int qz = 0; qz < P1; ++qz) {
      V kz, kx, ky;
      vzero(kz);
      vzero(kx);
      vzero(ky);
#pragma unroll
      for (int q = 0; q < P1; ++q) {
        madd(kz, sK[qz * P1 + q], uq[q]);
        madd(kx, sK[ta * P1 + q], S1[qz * P2 + tb * P1 + q]);
        madd(ky, sK[tb * P1 + q], S1[qz * P2 + q * P1 + ta]);
      }
      const T wz = sw[qz];
      const T fz = ckz * wa * wb, fx = ckx * wb * wz, fy = cky * wa * wz;
      V rr = vscale(vcol[qz], uq[qz]);
      madd(rr, fz, kz);
      madd(rr, fx, kx);
      madd(rr, fy, ky);
      r[qz] = rr;
      apart += (double)uq[qz].re * (double)rr.re + (double)uq[qz].im * (double)rr.im;
    }
    V y[P1];
    backward3<P1, V, T>(r, y, S1, S2, sB, ta, tb);
    double2* out = a.out_base + (long long)o * a.out_stride;
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      const int K = ez * g.p + c;
      if (inIJ && K >= 1 && K <= g.niz) {
        const double f = sxy * g.s[2][K];
        const long long idx = base + plane * (K - 1);
        double2 old = out[idx];
        old.x = fma(f, (double)y[c].re, old.x);
        old.y = fma(f, (double)y[c].im, old.y);
        out[idx] = old;
      }
    }
    if (a.part) {
      const double s = block_sum(apart, red);
      if (tid == 0) a.part[(long long)o * a.part_stride + part_off + blockIdx.x] = s;
    }
    __syncthreads();
  }
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
// Load vector out += (B^T)^(x)3 (J W f_q) (real), Eq. 19 right-hand side
// ---------------------------------------------------------------------------
template <int P1>
__global__ void __launch_bounds__(256) k_load(Geom g, const double* __restrict__ tab,
                                              const double* __restrict__ fq,
                                              double* __restrict__ out, double scale, int color) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3;
  extern __shared__ __align__(16) unsigned char smem[];
  double* sB = reinterpret_cast<double*>(smem);
  double* sw = sB + P2;
  double* S1 = sw + P1 + (size_t)threadIdx.y * 2 * P3;
  double* S2 = S1 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < P2; i += nthr) sB[i] = tab[i];
  for (int i = tid; i < P1; i += nthr) sw[i] = tab[tab_off_w(P1) + i];
  const int ta = threadIdx.x % P1, tb = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const bool valid = color_elem(g, color, (long long)blockIdx.x * blockDim.y + threadIdx.y, ex, ey, ez);
  __syncthreads();
  double r[P1];
#pragma unroll
  for (int q = 0; q < P1; ++q) r[q] = 0.0;
  if (valid) {
    const double hx = g.brk[0][ex + 1] - g.brk[0][ex];
    const double hy = g.brk[1][ey + 1] - g.brk[1][ey];
    const double hz = g.brk[2][ez + 1] - g.brk[2][ez];
    const double J = 0.125 * hx * hy * hz * scale;
    const long long e = ex + (long long)g.nx * (ey + (long long)g.ny * ez);
    const double* fp = fq + e * P3 + tb * P1 + ta;
#pragma unroll
    for (int q = 0; q < P1; ++q) r[q] = fp[q * P2] * J * sw[ta] * sw[tb] * sw[q];
  }
  double y[P1];
  backward3<P1, double, double>(r, y, S1, S2, sB, ta, tb);
  const int I = ex * g.p + ta, Jn = ey * g.p + tb;
  const bool inIJ = valid && I >= 1 && I <= g.nix && Jn >= 1 && Jn <= g.niy;
  const long long base = inIJ ? (long long)(I - 1) + (long long)g.nix * (Jn - 1) : 0;
  const long long plane = (long long)g.nix * g.niy;
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    const int K = ez * g.p + c;
    if (inIJ && K >= 1 && K <= g.niz) out[base + plane * (K - 1)] += y[c];
  }
}

// ---------------------------------------------------------------------------
// Interpolation of a real nodal field to the Gauss points: f_q = B^(x)3 u_e
// ---------------------------------------------------------------------------
template <int P1>
__global__ void __launch_bounds__(256) k_interp(Geom g, const double* __restrict__ tab,
                                                const double* __restrict__ nodal,
                                                double* __restrict__ fq) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3;
  extern __shared__ __align__(16) unsigned char smem[];
  double* sB = reinterpret_cast<double*>(smem);
  double* S1 = sB + P2 + (size_t)threadIdx.y * 2 * P3;
  double* S2 = S1 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < P2; i += nthr) sB[i] = tab[i];
  const int ta = threadIdx.x % P1, tb = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const bool valid = plain_elem(g, (long long)blockIdx.x * blockDim.y + threadIdx.y, ex, ey, ez);
  __syncthreads();
  const int I = ex * g.p + ta, Jn = ey * g.p + tb;
  const bool inIJ = valid && I >= 1 && I <= g.nix && Jn >= 1 && Jn <= g.niy;
  const long long base = inIJ ? (long long)(I - 1) + (long long)g.nix * (Jn - 1) : 0;
  const long long plane = (long long)g.nix * g.niy;
  double u[P1];
#pragma unroll
  for (int c = 0; c < P1; ++c) {
    const int K = ez * g.p + c;
    u[c] = (inIJ && K >= 1 && K <= g.niz) ? nodal[base + plane * (K - 1)] : 0.0;
  }
  double uq[P1];
  forward3<P1, double, double>(u, uq, S1, S2, sB, ta, tb);
  if (valid) {
    const long long e = ex + (long long)g.nx * (ey + (long long)g.ny * ez);
#pragma unroll
    for (int q = 0; q < P1; ++q) fq[e * P3 + q * P2 + tb * P1 + ta] = uq[q];
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
  typedef Cx<double> V;
  extern __shared__ __align__(16) unsigned char smem[];
  double* sB = reinterpret_cast<double*>(smem);
  V* S1 = reinterpret_cast<V*>(sB + P2) + (size_t)threadIdx.y * 2 * P3;
  V* S2 = S1 + P3;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  for (int i = tid; i < P2; i += nthr) sB[i] = tab[i];
  const int ta = threadIdx.x % P1, tb = threadIdx.x / P1;
  int ex = 0, ey = 0, ez = 0;
  const bool valid = plain_elem(g, (long long)blockIdx.x * blockDim.y + threadIdx.y, ex, ey, ez);
  __syncthreads();
  const int I = ex * g.p + ta, Jn = ey * g.p + tb;
  const bool inIJ = valid && I >= 1 && I <= g.nix && Jn >= 1 && Jn <= g.niy;
  const double sxy = inIJ ? g.s[0][I] * g.s[1][Jn] : 0.0;
  const long long base = inIJ ? (long long)(I - 1) + (long long)g.nix * (Jn - 1) : 0;
  const long long plane = (long long)g.nix * g.niy;
  double acc[P1];
#pragma unroll
  for (int q = 0; q < P1; ++q) acc[q] = 0.0;
  for (int o = 0; o < n_orb; ++o) {
    const double2* in = psi + (long long)o * stride;
    V u[P1];
#pragma unroll
    for (int c = 0; c < P1; ++c) {
      const int K = ez * g.p + c;
      vzero(u[c]);
      if (inIJ && K >= 1 && K <= g.niz) {
        const double f = sxy * g.s[2][K];
        const double2 v = in[base + plane * (K - 1)];
        u[c].re = v.x * f;
        u[c].im = v.y * f;
      }
    }
    V uq[P1];
    forward3<P1, V, double>(u, uq, S1, S2, sB, ta, tb);
    const double f = occ[o];
#pragma unroll
    for (int q = 0; q < P1; ++q) acc[q] += f * (uq[q].re * uq[q].re + uq[q].im * uq[q].im);
    __syncthreads();
  }
  if (valid) {
    const long long e = ex + (long long)g.nx * (ey + (long long)g.ny * ez);
#pragma unroll
    for (int q = 0; q < P1; ++q) rho[e * P3 + q * P2 + tb * P1 + ta] = acc[q];
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

template <int P1, typename T>
tdks_status hbar_t(tdks_ctx* c, const ApplyArgs& a) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3, E = Cfg<P1>::E;
  const size_t smem = (((2 * P2 + P1) * sizeof(T) + 15) & ~size_t(15)) + (size_t)E * 2 * P3 * sizeof(Cx<T>);
  TDKS_CU(c, set_smem(k_hbar<P1, T>, smem));
  const int bpc = blocks_per_color_t<P1>(c);
  // orbitals per CTA: enough CTAs to fill the GPU, V and geometry reused across orbitals
  int opc = 1;
  while (opc < a.n_orb && (long long)bpc * ((a.n_orb + 2 * opc - 1) / (2 * opc)) >= 4 * 152) opc *= 2;
  const int ochunks = (a.n_orb + opc - 1) / opc;
  dim3 block(P2, E), grid(bpc, ochunks);
  const T* tab = std::is_same<T, double>::value ? (const T*)c->d_tab : (const T*)c->d_tabf;
  const Geom g = tdks_geom(c);
  for (int color = 0; color < 8; ++color) {
    k_hbar<P1, T><<<grid, block, smem, c->stream>>>(g, tab, c->d_vks, a, color, opc, color * bpc);
  }
  c->n_launch += 8;
  c->n_apply_launch += 8;
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
tdks_status load_t(tdks_ctx* c, const double* fq, double* out, double scale) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3, E = Cfg<P1>::E;
  const size_t smem = (P2 + P1 + (size_t)E * 2 * P3) * sizeof(double);
  TDKS_CU(c, set_smem(k_load<P1>, smem));
  dim3 block(P2, E), grid(blocks_per_color_t<P1>(c));
  const Geom g = tdks_geom(c);
  for (int color = 0; color < 8; ++color)
    k_load<P1><<<grid, block, smem, c->stream>>>(g, c->d_tab, fq, out, scale, color);
  c->n_launch += 8;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

template <int P1>
tdks_status interp_t(tdks_ctx* c, const double* nodal, double* fq) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3, E = Cfg<P1>::E;
  const size_t smem = (P2 + (size_t)E * 2 * P3) * sizeof(double);
  TDKS_CU(c, set_smem(k_interp<P1>, smem));
  dim3 block(P2, E), grid((unsigned)((c->n_elem + E - 1) / E));
  k_interp<P1><<<grid, block, smem, c->stream>>>(tdks_geom(c), c->d_tab, nodal, fq);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

template <int P1>
tdks_status density_t(tdks_ctx* c, const double2* psi, int n_orb, double* rho) {
  constexpr int P2 = Cfg<P1>::P2, P3 = Cfg<P1>::P3, E = Cfg<P1>::E;
  const size_t smem = P2 * sizeof(double) + (size_t)E * 2 * P3 * sizeof(Cx<double>);
  TDKS_CU(c, set_smem(k_density<P1>, smem));
  dim3 block(P2, E), grid((unsigned)((c->n_elem + E - 1) / E));
  k_density<P1><<<grid, block, smem, c->stream>>>(tdks_geom(c), c->d_tab, psi, c->n_int, n_orb,
                                                 c->d_occ, rho);
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

int hbar_blocks_per_color(const tdks_ctx* c) {
  TDKS_DISPATCH(c->P1, blocks_per_color_t<P1>(c));
  return 0;
}
int stiff_blocks_per_color(const tdks_ctx* c) { return hbar_blocks_per_color(c); }

tdks_status launch_hbar_apply(tdks_ctx* c, const ApplyArgs& a, int prec) {
  if (prec == TDKS_FP32) {
    TDKS_DISPATCH(c->P1, (hbar_t<P1, float>(c, a)));
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

tdks_status launch_load_vector(tdks_ctx* c, const double* f_q, double* out, double scale) {
  TDKS_DISPATCH(c->P1, (load_t<P1>(c, f_q, out, scale)));
  return tdks_fail(c, TDKS_ERR_ARG, "unsupported degree");
}

tdks_status launch_interp(tdks_ctx* c, const double* nodal, double* f_q) {
  TDKS_DISPATCH(c->P1, (interp_t<P1>(c, nodal, f_q)));
  return tdks_fail(c, TDKS_ERR_ARG, "unsupported degree");
}

tdks_status launch_density(tdks_ctx* c, const double2* psi, int n_orb, double* rho_q) {
  TDKS_DISPATCH(c->P1, (density_t<P1>(c, psi, n_orb, rho_q)));
  return tdks_fail(c, TDKS_ERR_ARG, "unsupported degree");
}
