// Hartree potential from the discrete Poisson problem (Eqs. 8a, 19):
//   K phi = 4 pi c,  K_jk = int grad N_j . grad N_k,  c_j = int rho N_j,
// zero Dirichlet values on the boundary, then V_H(x_q) = sum_j N_j(x_q) phi_j.
//
// Preconditioned conjugate gradients, warm-started from the previous phi,
// stopping at ||r|| <= tol ||b||.  Preconditioners:
//   * fast diagonalization (default): the stiffness of an axis-aligned tensor
//     mesh is separable (see fdm.cpp), so K^-1 = S D^-1 S^T with S = Sx (x) Sy (x) Sz,
//     applied as six strided matrix products along the three axes and a diagonal
//     scaling; for these meshes it is the exact inverse up to rounding and CG stops
//     after one or two iterations.  The products are FP64, or double-float for the
//     double-float runs (a preconditioner exact to ~1e-14; the CG stays FP64);
//   * Jacobi (diagonal of K from 1-D sums).
// Convergence is decided on the device: once converged every later kernel of the
// iteration returns at once, and the host polls the flag after iterations
// 1, 2, 4, 8, 16, 32, ... so results do not depend on the polling schedule.
#include <cmath>
#include <vector>

#include "df64.cuh"
#include "tdks_internal.h"

using tdks::Df;

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 608;

__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = a;
    red[kThreads / 32 + (threadIdx.x >> 5)] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) {
      sa += red[k];
      sb += red[kThreads / 32 + k];
    }
    a = sa;
    b = sb;
  }
}

// every caller sums the same partials in the same order
__device__ __forceinline__ double sum_fixed(const double* part, int n) {
  __shared__ double red[kThreads / 32];
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) v += part[k];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < kThreads / 32; ++k) s += red[k];
  __syncthreads();
  return s;
}

// 1 / diag(K) from 1-D sums: diag = 1/2 (kx my mz + mx ky mz + mx my kz)
__global__ void k_invdiag(long long n, int nix, int niy, const double* kx, const double* ky,
                          const double* kz, const double* mx, const double* my, const double* mz,
                          double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(i % nix) + 1;
    const int J = (int)((i / nix) % niy) + 1;
    const int K = (int)(i / ((long long)nix * niy)) + 1;
    out[i] = 2.0 / (kx[I] * my[J] * mz[K] + mx[I] * ky[J] * mz[K] + mx[I] * my[J] * kz[K]);
  }
}

// r = b - Ap; partials of b.b and r.r
__global__ void k_cg_init(long long n, const double* b, const double* Ap, double* r, double* part) {
  __shared__ double red[2 * kThreads / 32];
  double bb = 0.0, rr = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double ri = b[i] - Ap[i];
    r[i] = ri;
    bb = fma(b[i], b[i], bb);
    rr = fma(ri, ri, rr);
  }
  block_sum2(bb, rr, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = bb;
    part[gridDim.x + blockIdx.x] = rr;
  }
}

__global__ void k_cg_init_fin(const double* part, int nb, double tol, CgState* cg) {
  const double bb = sum_fixed(part, nb);
  const double rr = sum_fixed(part + nb, nb);
  if (threadIdx.x == 0) {
    cg->bb = bb;
    cg->rr = rr;
    cg->rz = 0.0;
    cg->alpha = 0.0;
    cg->iters = 0;
    cg->first = 1;
    cg->failed = (isfinite(bb) && isfinite(rr)) ? 0 : 1;
    if (!cg->failed && bb == 0.0) cg->failed = 3;   // zero right-hand side: phi = 0
    cg->done = (cg->failed || rr <= tol * tol * bb) ? 1 : 0;
  }
}

// z = r * invdiag (Jacobi)
__global__ void k_jacobi(long long n, const double* r, const double* invd, double* z,
                         const CgState* cg) {
  if (cg->done) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    z[i] = r[i] * invd[i];
}

// partial r.z
__global__ void k_dot_part(long long n, const double* r, const double* z, double* part,
                           const CgState* cg) {
  if (cg->done) return;
  __shared__ double red[2 * kThreads / 32];
  double a = 0.0, dummy = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    a = fma(r[i], z[i], a);
  block_sum2(a, dummy, red);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// rz_new = r.z; beta = rz_new / rz (unused for the first direction)
__global__ void k_cg_fin_rz(const double* part, int nb, CgState* cg) {
  if (cg->done) return;
  const double rz = sum_fixed(part, nb);
  if (threadIdx.x == 0) {
    cg->alpha = cg->first ? 0.0 : rz / cg->rz;
    cg->rz = rz;
  }
}

// p = z + beta p  (p = z for the first direction)
__global__ void k_cg_dir(long long n, const double* z, double* p, const CgState* cg) {
  if (cg->done) return;
  const double beta = cg->alpha;
  const bool first = cg->first != 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = first ? z[i] : fma(beta, p[i], z[i]);
}

__global__ void k_cg_clear_first(CgState* cg) {
  if (!cg->done) cg->first = 0;
}

// alpha = rz / p.Kp;  x += alpha p;  r -= alpha Ap;  partial r.r
__global__ void k_cg_update(long long n, const double* pAp_part, int npart, double* x, double* r,
                            const double* p, const double* Ap, double* part, const CgState* cg) {
  if (cg->done) return;
  __shared__ double red[2 * kThreads / 32];
  const double pAp = sum_fixed(pAp_part, npart);
  const double alpha = cg->rz / pAp;
  double rr = 0.0, dummy = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, Ap[i], r[i]);
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  block_sum2(rr, dummy, red);
  if (threadIdx.x == 0) part[blockIdx.x] = rr;
}

__global__ void k_cg_fin_rr(const double* part, int nb, double tol, int maxit, CgState* cg) {
  if (cg->done) return;
  const double rr = sum_fixed(part, nb);
  if (threadIdx.x == 0) {
    cg->rr = rr;
    cg->iters += 1;
    if (!isfinite(rr)) {
      cg->failed = 1;
      cg->done = 1;
    } else if (rr <= tol * tol * cg->bb) {
      cg->done = 1;
    } else if (cg->iters >= maxit) {
      cg->failed = 2;
      cg->done = 1;
    }
  }
}

// ---- strided batched FP64 matrix product: C[b] = A[b] B[b] -------------------
struct Gemm {
  const double* A;
  long long sAb, sAm, sAk;
  const double* B;
  long long sBb, sBk, sBn;
  double* C;
  long long sCb, sCm, sCn;
  int M, N, K;
};

constexpr int GT = 64;   // output tile
constexpr int GK = 16;   // depth tile

__global__ void __launch_bounds__(256) k_gemm(Gemm g, const CgState* cg) {
  if (cg && cg->done) return;
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const long long b = blockIdx.z;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const double* A = g.A + b * g.sAb;
  const double* B = g.B + b * g.sBb;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const bool a_k_fast = (g.sAk == 1);
  const bool b_n_fast = (g.sBn == 1);
  for (int k0 = 0; k0 < g.K; k0 += GK) {
#pragma unroll
    for (int r = 0; r < (GT * GK) / 256; ++r) {
      const int e = tid + 256 * r;
      int kk, mm;
      if (a_k_fast) {
        kk = e % GK;
        mm = e / GK;
      } else {
        mm = e % GT;
        kk = e / GT;
      }
      const long long gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < g.M && gk < g.K) ? A[gm * g.sAm + gk * g.sAk] : 0.0;
      int nn, kb;
      if (b_n_fast) {
        nn = e % GT;
        kb = e / GT;
      } else {
        kb = e % GK;
        nn = e / GK;
      }
      const long long gn = n0 + nn, gk2 = k0 + kb;
      Bs[kb][nn] = (gn < g.N && gk2 < g.K) ? B[gk2 * g.sBk + gn * g.sBn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* C = g.C + b * g.sCb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long gm = m0 + ty * 4 + i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long gn = n0 + tx * 4 + j;
      if (gn < g.N) C[gm * g.sCm + gn * g.sCn] = acc[i][j];
    }
  }
}

// The same product in double-float arithmetic on the FP32 pipe (FP64 in and out):
// operands split into float pairs on the integer pipe, every output an accumulator
// (hi, err) -- hi grows by exact two-sums, the product tails and rounding errors of
// the sums collect in err -- renormalized once at the end.  Relative error ~1e-14:
// used for the preconditioner of the double-float runs, whose CG stays FP64.
__device__ __forceinline__ void gemm_dfa(float& hi, float& err, Df a, Df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  const float s = __fadd_rn(hi, p);
  const float v = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(p, v));
  err = __fadd_rn(err, __fadd_rn(e, pe));
  hi = s;
}

__global__ void __launch_bounds__(256) k_gemm_df(Gemm g, const CgState* cg) {
  if (cg && cg->done) return;
  __shared__ Df As[GK][GT + 1];
  __shared__ Df Bs[GK][GT + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const long long b = blockIdx.z;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const double* A = g.A + b * g.sAb;
  const double* B = g.B + b * g.sBb;
  float hi[4][4], er[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      hi[i][j] = 0.0f;
      er[i][j] = 0.0f;
    }
  const bool a_k_fast = (g.sAk == 1);
  const bool b_n_fast = (g.sBn == 1);
  for (int k0 = 0; k0 < g.K; k0 += GK) {
#pragma unroll
    for (int r = 0; r < (GT * GK) / 256; ++r) {
      const int e = tid + 256 * r;
      int kk, mm;
      if (a_k_fast) {
        kk = e % GK;
        mm = e / GK;
      } else {
        mm = e % GT;
        kk = e / GT;
      }
      const long long gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = tdks::d2df_bits((gm < g.M && gk < g.K) ? A[gm * g.sAm + gk * g.sAk] : 0.0);
      int nn, kb;
      if (b_n_fast) {
        nn = e % GT;
        kb = e / GT;
      } else {
        kb = e % GK;
        nn = e / GK;
      }
      const long long gn = n0 + nn, gk2 = k0 + kb;
      Bs[kb][nn] = tdks::d2df_bits((gn < g.N && gk2 < g.K) ? B[gk2 * g.sBk + gn * g.sBn] : 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      Df a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) gemm_dfa(hi[i][j], er[i][j], a[i], bb[j]);
    }
    __syncthreads();
  }
  double* C = g.C + b * g.sCb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long gm = m0 + ty * 4 + i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long gn = n0 + tx * 4 + j;
      if (gn < g.N) {
        const Df r = tdks::df_norm(hi[i][j], er[i][j]);
        C[gm * g.sCm + gn * g.sCn] = (double)r.hi + (double)r.lo;
      }
    }
  }
}

// t[i,j,k] /= lx[i] + ly[j] + lz[k]
__global__ void k_fdm_scale(long long n, int nix, int niy, const double* lx, const double* ly,
                            const double* lz, double* t, const CgState* cg) {
  if (cg && cg->done) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(i % nix);
    const int J = (int)((i / nix) % niy);
    const int K = (int)(i / ((long long)nix * niy));
    t[i] /= (lx[I] + ly[J] + lz[K]);
  }
}

int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  return (int)(b < kBlocks ? (b < 1 ? 1 : b) : kBlocks);
}

// out = transform of `in` along `axis` with S (n_a x n_a, row-major [i][mode]):
// forward out[.., mode, ..] = sum_i S[i][mode] in[.., i, ..]; backward uses S^T.
void axis_gemm(tdks_ctx* c, int axis, bool forward, const double* in, double* out,
               const CgState* cg, bool df) {
  const long long nx = c->Ni[0], ny = c->Ni[1], nz = c->Ni[2];
  const double* S = c->d_fdmS[axis];
  const long long na = c->Ni[axis];
  Gemm g{};
  dim3 grid;
  if (axis == 0) {
    // rows (j,k): C[row][mode] = sum_i V[row][i] S[i][mode]
    g.A = in;
    g.sAb = 0;
    g.sAm = nx;
    g.sAk = 1;
    g.B = S;
    g.sBb = 0;
    g.sBk = forward ? na : 1;
    g.sBn = forward ? 1 : na;
    g.C = out;
    g.sCb = 0;
    g.sCm = nx;
    g.sCn = 1;
    g.M = (int)(ny * nz);
    g.N = (int)nx;
    g.K = (int)nx;
    grid = dim3((g.N + GT - 1) / GT, (g.M + GT - 1) / GT, 1);
  } else if (axis == 1) {
    // per z-slab: C[mode][i] = sum_j S[j][mode] V[j][i]
    g.A = S;
    g.sAb = 0;
    g.sAm = forward ? 1 : na;
    g.sAk = forward ? na : 1;
    g.B = in;
    g.sBb = nx * ny;
    g.sBk = nx;
    g.sBn = 1;
    g.C = out;
    g.sCb = nx * ny;
    g.sCm = nx;
    g.sCn = 1;
    g.M = (int)ny;
    g.N = (int)nx;
    g.K = (int)ny;
    grid = dim3((g.N + GT - 1) / GT, (g.M + GT - 1) / GT, (unsigned)nz);
  } else {
    // C[mode][(i,j)] = sum_k S[k][mode] V[k][(i,j)]
    g.A = S;
    g.sAb = 0;
    g.sAm = forward ? 1 : na;
    g.sAk = forward ? na : 1;
    g.B = in;
    g.sBb = 0;
    g.sBk = nx * ny;
    g.sBn = 1;
    g.C = out;
    g.sCb = 0;
    g.sCm = nx * ny;
    g.sCn = 1;
    g.M = (int)nz;
    g.N = (int)(nx * ny);
    g.K = (int)nz;
    grid = dim3((g.N + GT - 1) / GT, (g.M + GT - 1) / GT, 1);
  }
  if (df)
    k_gemm_df<<<grid, 256, 0, c->stream>>>(g, cg);
  else
    k_gemm<<<grid, 256, 0, c->stream>>>(g, cg);
}

// z = S D^-1 S^T r  (exact inverse of the separable stiffness)
// End of a fixed-length CG: zero right-hand side -> x = 0; not converged or
// non-finite -> error bits (4: iteration cap, 8: non-finite).
__global__ void k_cg_graph_end(long long n, double* x, const CgState* cg, int* err) {
  const int failed = cg->failed;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (failed == 1) atomicOr(err, 8);
    else if (failed != 3 && !cg->done) atomicOr(err, 4);
  }
  if (failed != 3) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = 0.0;
}

void fdm_apply(tdks_ctx* c, const double* r, double* z, const CgState* cg, bool df) {
  const long long n = c->n_int;
  axis_gemm(c, 0, true, r, c->d_t1, cg, df);
  axis_gemm(c, 1, true, c->d_t1, c->d_t2, cg, df);
  axis_gemm(c, 2, true, c->d_t2, c->d_t1, cg, df);
  k_fdm_scale<<<grid_for(n), kThreads, 0, c->stream>>>(n, c->Ni[0], c->Ni[1], c->d_fdmL[0],
                                                      c->d_fdmL[1], c->d_fdmL[2], c->d_t1, cg);
  axis_gemm(c, 2, false, c->d_t1, c->d_t2, cg, df);
  axis_gemm(c, 1, false, c->d_t2, c->d_t1, cg, df);
  axis_gemm(c, 0, false, c->d_t1, z, cg, df);
  c->n_launch += 7;
}

}  // namespace

tdks_status poisson_setup(tdks_ctx* c, const Tables1D& t) {
  const size_t n = (size_t)c->n_int;
  double** vecs[] = {&c->d_z, &c->d_t1, &c->d_t2, &c->d_invdiag};
  for (double** v : vecs) {
    if (cudaMalloc(v, n * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return tdks_fail(c, TDKS_ERR_NOMEM, "Poisson work vectors");
    }
  }
  k_invdiag<<<grid_for((long long)n), kThreads, 0, c->stream>>>(
      (long long)n, c->Ni[0], c->Ni[1], c->d_kd[0], c->d_kd[1], c->d_kd[2], c->d_md[0], c->d_md[1],
      c->d_md[2], c->d_invdiag);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  // fast diagonalization: per-axis generalized eigenpairs on the host (dense;
  // axes longer than 1024 interior nodes use the Jacobi preconditioner instead)
  c->fdm_ok = false;
  const int nn[3] = {c->nx, c->ny, c->nz};
  bool small = true;
  for (int d = 0; d < 3; ++d) small = small && (c->Ni[d] <= 1024);
  if (small) {
    try {
      for (int d = 0; d < 3; ++d) {
        std::vector<double> S, lam;
        tdks_fdm_axis(t, c->p, c->brk[d].data(), nn[d], S, lam);
        if (cudaMalloc(&c->d_fdmS[d], S.size() * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&c->d_fdmL[d], lam.size() * sizeof(double)) != cudaSuccess) {
          cudaGetLastError();
          return tdks_fail(c, TDKS_ERR_NOMEM, "FDM tables");
        }
        TDKS_CU(c, cudaMemcpy(c->d_fdmS[d], S.data(), S.size() * sizeof(double),
                              cudaMemcpyHostToDevice));
        TDKS_CU(c, cudaMemcpy(c->d_fdmL[d], lam.data(), lam.size() * sizeof(double),
                              cudaMemcpyHostToDevice));
      }
      c->fdm_ok = true;
    } catch (const std::exception&) {
      c->fdm_ok = false;
    }
  }
  if (!c->fdm_ok) c->cg_precond = 1;
  return TDKS_OK;
}

// Solve K x = b by the preconditioned CG above; x holds the initial guess.
tdks_status run_cg_solve(tdks_ctx* c, const double* b, double* x, int* iters, bool df) {
  const long long n = c->n_int;
  const int nb = grid_for(n);
  const int sbpc = stiff_blocks_per_color(c);
  const bool fdm = (c->cg_precond == 0 && c->fdm_ok);
  double* part_pAp = c->d_part;                       // 8 * sbpc
  double* part_vec = c->d_part + 8 * (int64_t)sbpc;   // 2 * nb
  CgState* cg = c->d_cg;
  // r = b - K x0
  TDKS_CU(c, cudaMemsetAsync(c->d_Ap, 0, n * sizeof(double), c->stream));
  TDKS_TRY(launch_stiffness(c, x, c->d_Ap, nullptr, nullptr));
  k_cg_init<<<nb, kThreads, 0, c->stream>>>(n, b, c->d_Ap, c->d_r, part_vec);
  k_cg_init_fin<<<1, kThreads, 0, c->stream>>>(part_vec, nb, c->cg_tol, cg);
  c->n_launch += 2;
  // z = P^-1 r; rz = r.z; p = z (first direction) or z + beta p
  auto precondition = [&]() {
    if (fdm) {
      fdm_apply(c, c->d_r, c->d_z, cg, df);
    } else {
      k_jacobi<<<nb, kThreads, 0, c->stream>>>(n, c->d_r, c->d_invdiag, c->d_z, cg);
      c->n_launch += 1;
    }
    k_dot_part<<<nb, kThreads, 0, c->stream>>>(n, c->d_r, c->d_z, part_vec, cg);
    k_cg_fin_rz<<<1, kThreads, 0, c->stream>>>(part_vec, nb, cg);
    k_cg_dir<<<nb, kThreads, 0, c->stream>>>(n, c->d_z, c->d_pv, cg);
    k_cg_clear_first<<<1, 1, 0, c->stream>>>(cg);
    c->n_launch += 4;
  };
  precondition();
  TDKS_CU(c, cudaGetLastError());
  int it = 0, next_poll = 1;
  CgState host{};
  while (true) {
    while (it < next_poll) {
      TDKS_CU(c, cudaMemsetAsync(c->d_Ap, 0, n * sizeof(double), c->stream));
      TDKS_TRY(launch_stiffness(c, c->d_pv, c->d_Ap, part_pAp, cg));
      k_cg_update<<<nb, kThreads, 0, c->stream>>>(n, part_pAp, 8 * sbpc, x, c->d_r, c->d_pv,
                                                  c->d_Ap, part_vec, cg);
      k_cg_fin_rr<<<1, kThreads, 0, c->stream>>>(part_vec, nb, c->cg_tol, c->cg_maxit, cg);
      c->n_launch += 2;
      precondition();
      ++it;
    }
    TDKS_CU(c, cudaGetLastError());
    TDKS_CU(c, cudaMemcpyAsync(&host, cg, sizeof(CgState), cudaMemcpyDeviceToHost, c->stream));
    TDKS_CU(c, cudaStreamSynchronize(c->stream));
    if (host.done) break;
    if (it > c->cg_maxit + 32) break;
    next_poll = next_poll < 32 ? 2 * next_poll : next_poll + 32;
  }
  if (iters) *iters = host.iters;
  c->n_cg += host.iters;
  if (host.failed == 3) {
    TDKS_CU(c, cudaMemsetAsync(x, 0, n * sizeof(double), c->stream));
    host.failed = 0;
  }
  if (host.failed == 1) return tdks_fail(c, TDKS_ERR_NAN, "non-finite residual in Poisson CG");
  if (host.failed == 2 || !host.done)
    return tdks_fail(c, TDKS_ERR_NOT_CONVERGED, "Poisson CG reached its iteration cap");
  return TDKS_OK;
}

tdks_status run_hartree(tdks_ctx* c, const double* rho_q, double* vh_q, int* iters, bool df) {
  const long long n = c->n_int;
  // b = 4 pi c
  TDKS_CU(c, cudaMemsetAsync(c->d_b, 0, n * sizeof(double), c->stream));
  TDKS_TRY(launch_load_vector(c, rho_q, c->d_b, 4.0 * M_PI));
  TDKS_TRY(run_cg_solve(c, c->d_b, c->d_phi, iters, df));
  TDKS_TRY(launch_interp(c, c->d_phi, vh_q));
  return TDKS_OK;
}

// The CG of run_cg_solve with a fixed number of iterations and no host
// synchronization, for stream capture: every kernel of an iteration returns at
// once after convergence, so extra iterations cost launches only.  Needs the
// fast-diagonalization preconditioner (one or two iterations); an unconverged
// solve sets bit 4 of *err.
tdks_status cg_solve_graph(tdks_ctx* c, const double* b, double* x, int n_iter, int* err, bool df) {
  if (!(c->cg_precond == 0 && c->fdm_ok))
    return tdks_fail(c, TDKS_ERR_ARG, "graph CG needs the fast-diagonalization preconditioner");
  const long long n = c->n_int;
  const int nb = grid_for(n);
  const int sbpc = stiff_blocks_per_color(c);
  double* part_pAp = c->d_part;
  double* part_vec = c->d_part + 8 * (int64_t)sbpc;
  CgState* cg = c->d_cg;
  TDKS_CU(c, cudaMemsetAsync(c->d_Ap, 0, n * sizeof(double), c->stream));
  TDKS_TRY(launch_stiffness(c, x, c->d_Ap, nullptr, nullptr));
  k_cg_init<<<nb, kThreads, 0, c->stream>>>(n, b, c->d_Ap, c->d_r, part_vec);
  k_cg_init_fin<<<1, kThreads, 0, c->stream>>>(part_vec, nb, c->cg_tol, cg);
  auto precondition = [&]() {
    fdm_apply(c, c->d_r, c->d_z, cg, df);
    k_dot_part<<<nb, kThreads, 0, c->stream>>>(n, c->d_r, c->d_z, part_vec, cg);
    k_cg_fin_rz<<<1, kThreads, 0, c->stream>>>(part_vec, nb, cg);
    k_cg_dir<<<nb, kThreads, 0, c->stream>>>(n, c->d_z, c->d_pv, cg);
    k_cg_clear_first<<<1, 1, 0, c->stream>>>(cg);
  };
  precondition();
  for (int it = 0; it < n_iter; ++it) {
    TDKS_CU(c, cudaMemsetAsync(c->d_Ap, 0, n * sizeof(double), c->stream));
    TDKS_TRY(launch_stiffness(c, c->d_pv, c->d_Ap, part_pAp, cg));
    k_cg_update<<<nb, kThreads, 0, c->stream>>>(n, part_pAp, 8 * sbpc, x, c->d_r, c->d_pv, c->d_Ap,
                                                part_vec, cg);
    k_cg_fin_rr<<<1, kThreads, 0, c->stream>>>(part_vec, nb, c->cg_tol, c->cg_maxit, cg);
    precondition();
  }
  k_cg_graph_end<<<nb, kThreads, 0, c->stream>>>(n, x, cg, err);
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

tdks_status hartree_graph(tdks_ctx* c, const double* rho_q, double* vh_q, int n_iter, int* err, bool df) {
  const long long n = c->n_int;
  TDKS_CU(c, cudaMemsetAsync(c->d_b, 0, n * sizeof(double), c->stream));
  TDKS_TRY(launch_load_vector(c, rho_q, c->d_b, 4.0 * M_PI));
  TDKS_TRY(cg_solve_graph(c, c->d_b, c->d_phi, n_iter, err, df));
  TDKS_TRY(launch_interp(c, c->d_phi, vh_q));
  return TDKS_OK;
}
