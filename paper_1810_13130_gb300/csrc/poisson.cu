// Hartree potential from the discrete Poisson problem (Eqs. 8a, 19):
//   K phi = 4 pi c,  K_jk = int grad N_j . grad N_k,  c_j = int rho N_j,
// zero Dirichlet values on the boundary, then V_H(x_q) = sum_j N_j(x_q) phi_j.
// Jacobi-preconditioned conjugate gradients, warm-started from the previous
// phi, stopping at ||r|| <= tol ||b||.  Convergence is decided on the device:
// once converged every later kernel of the iteration returns at once, and the
// host polls the flag every few iterations, so iteration counts and results do
// not depend on the polling interval.
#include <cmath>

#include "tdks_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 608;
constexpr int kPoll = 16;

// Jacobi diagonal of K from 1-D sums: diag = 1/2 (kx my mz + mx ky mz + mx my kz)
// with k_d[I] = sum_e K1_aa / h_e and m_d[I] = sum_e h_e Mg_aa over elements at node I.
struct Diag {
  const double *kx, *ky, *kz, *mx, *my, *mz;
  int nix, niy;
  __device__ __forceinline__ double at(long long i) const {
    const int I = (int)(i % nix) + 1;
    const int J = (int)((i / nix) % niy) + 1;
    const int K = (int)(i / ((long long)nix * niy)) + 1;
    return 0.5 * (kx[I] * my[J] * mz[K] + mx[I] * ky[J] * mz[K] + mx[I] * my[J] * kz[K]);
  }
};

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

__device__ __forceinline__ double sum_fixed(const double* part, int n) {
  // every caller sums the same partials in the same order
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

// r = b - Ap (Ap holds K x), z = r / diag, p = z; partials of b.b, r.z, r.r
__global__ void k_cg_init(long long n, const double* b, const double* Ap, double* r, double* p,
                          Diag dg, double* part) {
  __shared__ double red[2 * kThreads / 32];
  __shared__ double red2[2 * kThreads / 32];
  double bb = 0.0, rz = 0.0, rr = 0.0, dummy = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double ri = b[i] - Ap[i];
    const double zi = ri / dg.at(i);
    r[i] = ri;
    p[i] = zi;
    bb += b[i] * b[i];
    rz += ri * zi;
    rr += ri * ri;
  }
  block_sum2(bb, rz, red);
  block_sum2(rr, dummy, red2);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = bb;
    part[gridDim.x + blockIdx.x] = rz;
    part[2 * gridDim.x + blockIdx.x] = rr;
  }
}

__global__ void k_cg_init_fin(const double* part, int nb, double tol, CgState* cg) {
  const double bb = sum_fixed(part, nb);
  const double rz = sum_fixed(part + nb, nb);
  const double rr = sum_fixed(part + 2 * nb, nb);
  if (threadIdx.x == 0) {
    cg->bb = bb;
    cg->rz = rz;
    cg->rr = rr;
    cg->iters = 0;
    cg->failed = (isfinite(bb) && isfinite(rr)) ? 0 : 1;
    if (!cg->failed && bb == 0.0) cg->failed = 3;   // zero right-hand side: phi = 0
    cg->done = (cg->failed || rr <= tol * tol * bb) ? 1 : 0;
  }
}

// alpha = rz / p.Kp;  x += alpha p;  r -= alpha Ap;  partials of r.r and r.z
__global__ void k_cg_update(long long n, const double* pAp_part, int npart, double* x, double* r,
                            const double* p, const double* Ap, Diag dg, double* part,
                            CgState* cg) {
  if (cg->done) return;
  __shared__ double red[2 * kThreads / 32];
  const double pAp = sum_fixed(pAp_part, npart);
  const double alpha = cg->rz / pAp;
  double rr = 0.0, rz = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, Ap[i], r[i]);
    r[i] = ri;
    rr += ri * ri;
    rz += ri * ri / dg.at(i);
  }
  block_sum2(rr, rz, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = rr;
    part[gridDim.x + blockIdx.x] = rz;
  }
}

__global__ void k_cg_fin(const double* part, int nb, double tol, int maxit, CgState* cg) {
  if (cg->done) return;
  const double rr = sum_fixed(part, nb);
  const double rz = sum_fixed(part + nb, nb);
  if (threadIdx.x == 0) {
    const double beta = rz / cg->rz;
    cg->alpha = beta;                 // carries beta to the direction update
    cg->rz = rz;
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

// p = z + beta p, z = r / diag (skipped once converged)
__global__ void k_cg_dir(long long n, const double* r, double* p, Diag dg, const CgState* cg) {
  if (cg->done) return;
  const double beta = cg->alpha;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], r[i] / dg.at(i));
}

int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  return (int)(b < kBlocks ? (b < 1 ? 1 : b) : kBlocks);
}

}  // namespace

tdks_status run_hartree(tdks_ctx* c, const double* rho_q, double* vh_q, int* iters) {
  const long long n = c->n_int;
  const int nb = grid_for(n);
  const int sbpc = stiff_blocks_per_color(c);
  Diag dg{c->d_kd[0], c->d_kd[1], c->d_kd[2], c->d_md[0], c->d_md[1], c->d_md[2], c->Ni[0], c->Ni[1]};
  double* part_pAp = c->d_part;                       // 8 * sbpc
  double* part_vec = c->d_part + 8 * (int64_t)sbpc;   // 3 * nb
  // b = 4 pi c
  TDKS_CU(c, cudaMemsetAsync(c->d_b, 0, n * sizeof(double), c->stream));
  TDKS_TRY(launch_load_vector(c, rho_q, c->d_b, 4.0 * M_PI));
  // r = b - K x0
  TDKS_CU(c, cudaMemsetAsync(c->d_Ap, 0, n * sizeof(double), c->stream));
  TDKS_TRY(launch_stiffness(c, c->d_phi, c->d_Ap, nullptr, nullptr));
  k_cg_init<<<nb, kThreads, 0, c->stream>>>(n, c->d_b, c->d_Ap, c->d_r, c->d_pv, dg, part_vec);
  k_cg_init_fin<<<1, kThreads, 0, c->stream>>>(part_vec, nb, c->cg_tol, c->d_cg);
  c->n_launch += 2;
  TDKS_CU(c, cudaGetLastError());
  int it = 0;
  CgState host{};
  while (true) {
    for (int k = 0; k < kPoll; ++k) {
      TDKS_CU(c, cudaMemsetAsync(c->d_Ap, 0, n * sizeof(double), c->stream));
      TDKS_TRY(launch_stiffness(c, c->d_pv, c->d_Ap, part_pAp, c->d_cg));
      k_cg_update<<<nb, kThreads, 0, c->stream>>>(n, part_pAp, 8 * sbpc, c->d_phi, c->d_r, c->d_pv,
                                                  c->d_Ap, dg, part_vec, c->d_cg);
      k_cg_fin<<<1, kThreads, 0, c->stream>>>(part_vec, nb, c->cg_tol, c->cg_maxit, c->d_cg);
      k_cg_dir<<<nb, kThreads, 0, c->stream>>>(n, c->d_r, c->d_pv, dg, c->d_cg);
      c->n_launch += 3;
    }
    TDKS_CU(c, cudaGetLastError());
    it += kPoll;
    TDKS_CU(c, cudaMemcpyAsync(&host, c->d_cg, sizeof(CgState), cudaMemcpyDeviceToHost, c->stream));
    TDKS_CU(c, cudaStreamSynchronize(c->stream));
    if (host.done) break;
    if (it > c->cg_maxit + kPoll) break;
  }
  if (iters) *iters = host.iters;
  c->n_cg += host.iters;
  if (host.failed == 3) {
    TDKS_CU(c, cudaMemsetAsync(c->d_phi, 0, n * sizeof(double), c->stream));
    host.failed = 0;
  }
  if (host.failed == 1) return tdks_fail(c, TDKS_ERR_NAN, "non-finite residual in Poisson CG");
  if (host.failed == 2 || !host.done)
    return tdks_fail(c, TDKS_ERR_NOT_CONVERGED, "Poisson CG reached its iteration cap");
  TDKS_TRY(launch_interp(c, c->d_phi, vh_q));
  return TDKS_OK;
}
