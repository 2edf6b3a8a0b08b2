// Dipole-response objective and its adjoint gradient with respect to the field.
//
// Objective: J = sum_{n=0}^{N} w_n (e . mu(t_n))^2 over the dipoles after each
// Magnus step (Sec. V), as a function of the field samples E(t_{n-1} + dt/4) and
// E(t_{n-1} + dt/2) of V_field = -E . r (Eq. 7) used by the predictor and the
// corrector (Sec. VI.B).
//
// Forward: the ordinary propagation, with the state (psi, V_HXC^{n-1},
// V_HXC^{n-2}, Poisson warm start) stored every `ckpt_every` steps.
// Backward: per segment, restore the checkpoint, recompute the segment keeping
// psi^{n-1}, psi^{n-1/2}, V_pred, V_mid, then sweep it in reverse:
//   * exact adjoint of each unitary exponential: lambda <- exp(+i tau Hbar) lambda,
//     a Lanczos exponential with negative time;
//   * potential term: dJ/dv(x_q) = tau wJ_q int_0^1 sum_a Im[conj(mu_s) phi_s](x_q) ds,
//     phi_s = e^{-i tau s Hbar} psi and mu_s = e^{+i tau (1-s) Hbar} lambda, from one
//     Krylov basis each (recombinations only), s by Gauss-Legendre;
//   * Hartree adjoint through the symmetric K solve, LDA kernel, density adjoint.
// The exponentials are taken as exact (their Krylov error is below the tolerance).
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "tdks_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 608;

int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  return (int)(b < kBlocks ? (b < 1 ? 1 : b) : kBlocks);
}

// out[o] = sum_j coef[o][j] V_j[o], V_0 = base vector, V_j (j >= 1) in the workspace
__global__ void k_combine_basis(long long n, double2* out, const double2* V0, const double2* Vw,
                                int64_t wsorb, const double2* coef, int kcap, const int* kk) {
  const int o = blockIdx.y;
  const int m = kk[o];
  const double2* c = coef + (long long)o * kcap;
  const double2* v0 = V0 + (long long)o * n;
  const double2* vw = Vw + (long long)o * wsorb;
  double2* dst = out + (long long)o * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
#pragma unroll 4
    for (int j = 0; j < m; ++j) {
      const double2 v = (j == 0) ? v0[i] : vw[(long long)(j - 1) * n + i];
      const double2 cj = c[j];
      re = fma(cj.x, v.x, fma(-cj.y, v.y, re));
      im = fma(cj.x, v.y, fma(cj.y, v.x, im));
    }
    dst[i] = make_double2(re, im);
  }
}

__global__ void k_axpy_c(long long n, double a, const double2* x, double2* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 u = x[i];
    double2 v = y[i];
    v.x = fma(a, u.x, v.x);
    v.y = fma(a, u.y, v.y);
    y[i] = v;
  }
}

__global__ void k_axpby(long long n, double a, const double* x, double b, double* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

struct Seg {
  double2* psi_prev = nullptr;   // psi^{n-1} for each step of a segment
  double2* psi_half = nullptr;
  double* v_pred = nullptr;
  double* v_mid = nullptr;
};

}  // namespace

struct AdjState {
  int n_steps = 0, n_orb = 0, ckpt = 1, kmax = 64, prec = 0;
  double dt = 0, tol = 1e-10;
  std::vector<double> E, w, dip;
  double e[3] = {0, 0, 1};
  // checkpoints
  std::vector<double2*> ck_psi;
  std::vector<double*> ck_h1, ck_h2, ck_phi;
  // segment storage (ckpt steps) and work vectors
  double2 *psi = nullptr, *seg_psi = nullptr, *seg_half = nullptr, *psi_end = nullptr;
  double *seg_vpred = nullptr, *seg_vmid = nullptr;
  double2 *lam = nullptr, *lam_prev = nullptr, *lam_h = nullptr, *lam_tmp = nullptr, *phis = nullptr,
          *mus = nullptr;
  double *gh1 = nullptr, *gh2 = nullptr, *gh1n = nullptr, *grho = nullptr, *gvmid = nullptr,
         *gvpred = nullptr, *ny = nullptr, *nz = nullptr;
  double2* d_coef = nullptr;
  int* d_k = nullptr;
  bool ready = false;
};

namespace {

void free_adj(AdjState* a) {
  for (auto p : a->ck_psi) cudaFree(p);
  for (auto p : a->ck_h1) cudaFree(p);
  for (auto p : a->ck_h2) cudaFree(p);
  for (auto p : a->ck_phi) cudaFree(p);
  void* ptrs[] = {a->psi, a->seg_psi, a->seg_half, a->psi_end, a->seg_vpred, a->seg_vmid, a->lam,
                  a->lam_prev, a->lam_h, a->lam_tmp, a->phis, a->mus, a->gh1, a->gh2, a->gh1n,
                  a->grho, a->gvmid, a->gvpred, a->ny, a->nz, a->d_coef, a->d_k};
  for (void* p : ptrs) cudaFree(p);
  delete a;
}

template <typename T>
tdks_status amalloc(tdks_ctx* c, T** p, size_t count) {
  if (cudaMalloc((void**)p, (count ? count : 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return tdks_fail(c, TDKS_ERR_NOMEM, "adjoint buffers");
  }
  return TDKS_OK;
}

// Eigen-decomposition of the real symmetric tridiagonal T (diag alpha, off-diagonal beta):
// ev[j][k] component j of eigenvector k, lam[k] (host, small).
struct TriEig {
  int m = 0;
  std::vector<double> ev, lam;
};

void tri_eig(const double* alpha, const double* beta, int m, TriEig& E) {
  std::vector<double> C((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) {
    C[(size_t)i * m + i] = alpha[i];
    if (i + 1 < m) C[(size_t)i * m + i + 1] = C[(size_t)(i + 1) * m + i] = beta[i];
  }
  E.m = m;
  tdks_sym_eigen(C, m, E.ev, E.lam);
}

// y = exp(-i t T) e_1 from the decomposition
void tri_exp(const TriEig& E, double t, std::vector<std::complex<double>>& y) {
  const int m = E.m;
  y.assign(m, 0.0);
  for (int k = 0; k < m; ++k) {
    const std::complex<double> ph = std::exp(std::complex<double>(0.0, -t * E.lam[k])) * E.ev[k];
    for (int j = 0; j < m; ++j) y[j] += E.ev[(size_t)j * m + k] * ph;
  }
}

// g_out += dJ/dv of Re<lam, exp(-i tau Hbar) psi>; lam_out = exp(+i tau Hbar) lam.
// Hbar acts with the potential currently in the context.
tdks_status frechet(tdks_ctx* c, AdjState* A, const double2* psi, const double2* lam, double tau,
                    int n_s, double* g_out, double2* lam_out) {
  const int n_orb = A->n_orb;
  const long long n = c->n_int;
  int ns1 = 0, ns2 = 0;
  TDKS_TRY(run_expm_ws(c, 0, psi, A->phis, n_orb, tau, A->tol, A->kmax, TDKS_FP64, nullptr,
                       nullptr, nullptr, &ns1));
  TDKS_TRY(run_expm_ws(c, 1, lam, lam_out, n_orb, -tau, A->tol, A->kmax, TDKS_FP64, nullptr,
                       nullptr, nullptr, &ns2));
  if (ns1 || ns2)
    return tdks_fail(c, TDKS_ERR_NOT_CONVERGED,
                     "adjoint needs one Krylov basis per exponential: raise k_max");
  std::vector<KryOrb> kp(n_orb), kl(n_orb);
  TDKS_CU(c, cudaMemcpyAsync(kp.data(), c->d_kryw[0], n_orb * sizeof(KryOrb), cudaMemcpyDeviceToHost,
                             c->stream));
  TDKS_CU(c, cudaMemcpyAsync(kl.data(), c->d_kryw[1], n_orb * sizeof(KryOrb), cudaMemcpyDeviceToHost,
                             c->stream));
  TDKS_CU(c, cudaStreamSynchronize(c->stream));
  // Gauss-Legendre nodes on [0, 1]
  std::vector<double> sx(n_s), sw(n_s);
  for (int i = 0; i < n_s; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (n_s + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 1; k < n_s; ++k) {
        const double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      const double dp = n_s * (p0 - x * p1) / (1.0 - x * x);
      const double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double p0 = 1.0, p1 = x;
    for (int k = 1; k < n_s; ++k) {
      const double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
      p0 = p1;
      p1 = p2;
    }
    const double dp = n_s * (p0 - x * p1) / (1.0 - x * x);
    sx[i] = 0.5 * (x + 1.0);
    sw[i] = 1.0 / ((1.0 - x * x) * dp * dp);      // (2 / ((1-x^2) P'^2)) / 2
  }
  const int kcap = TDKS_KMAX;
  std::vector<double2> cp((size_t)n_orb * kcap), cl((size_t)n_orb * kcap);
  std::vector<int> kk(2 * n_orb);
  for (int o = 0; o < n_orb; ++o) {
    kk[o] = kp[o].k;
    kk[n_orb + o] = kl[o].k;
  }
  TDKS_CU(c, cudaMemcpyAsync(A->d_k, kk.data(), 2 * n_orb * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  const int nb = grid_for(n);
  std::vector<TriEig> ep(n_orb), el(n_orb);
  for (int o = 0; o < n_orb; ++o) {
    tri_eig(kp[o].alpha, kp[o].beta, kp[o].k, ep[o]);
    tri_eig(kl[o].alpha, kl[o].beta, kl[o].k, el[o]);
  }
  std::vector<std::complex<double>> y;
  for (int i = 0; i < n_s; ++i) {
    for (int o = 0; o < n_orb; ++o) {
      const KryOrb& P = kp[o];
      tri_exp(ep[o], tau * sx[i], y);
      for (int j = 0; j < P.k; ++j) {
        const std::complex<double> v = P.nrm * P.s[j] * y[j];
        cp[(size_t)o * kcap + j] = make_double2(v.real(), v.imag());
      }
      const KryOrb& L = kl[o];
      tri_exp(el[o], -tau * (1.0 - sx[i]), y);
      for (int j = 0; j < L.k; ++j) {
        const std::complex<double> v = L.nrm * L.s[j] * y[j];
        cl[(size_t)o * kcap + j] = make_double2(v.real(), v.imag());
      }
    }
    TDKS_CU(c, cudaMemcpyAsync(A->d_coef, cp.data(), cp.size() * sizeof(double2), cudaMemcpyHostToDevice,
                               c->stream));
    k_combine_basis<<<dim3(nb, n_orb), kThreads, 0, c->stream>>>(
        n, A->phis, psi, c->d_Vw[0], (int64_t)c->Vw_kmax[0] * n, A->d_coef, kcap, A->d_k);
    TDKS_CU(c, cudaMemcpyAsync(A->d_coef + (size_t)n_orb * kcap, cl.data(), cl.size() * sizeof(double2),
                               cudaMemcpyHostToDevice, c->stream));
    k_combine_basis<<<dim3(nb, n_orb), kThreads, 0, c->stream>>>(
        n, A->mus, lam, c->d_Vw[1], (int64_t)c->Vw_kmax[1] * n, A->d_coef + (size_t)n_orb * kcap, kcap,
        A->d_k + n_orb);
    c->n_launch += 2;
    TDKS_TRY(launch_cross(c, A->mus, A->phis, n_orb, sw[i] * tau, g_out));
    // the host coefficient arrays are reused: wait for the copies of this node
    TDKS_CU(c, cudaStreamSynchronize(c->stream));
  }
  return TDKS_OK;
}

// g_rho = dJ/drho from g_h = dJ/dV_HXC (at the Gauss points)
tdks_status hxc_adjoint(tdks_ctx* c, AdjState* A, const double* rho, const double* g_h, double* g_rho) {
  const size_t nf = (size_t)(c->n_elem * c->nq3);
  const long long n = c->n_int;
  if (c->hartree) {
    TDKS_CU(c, cudaMemsetAsync(A->ny, 0, n * sizeof(double), c->stream));
    TDKS_TRY(launch_load_vector(c, g_h, A->ny, 1.0, 0));     // (B^T)^(x)3 g_h, assembled
    TDKS_CU(c, cudaMemsetAsync(A->nz, 0, n * sizeof(double), c->stream));
    TDKS_TRY(run_cg_solve(c, A->ny, A->nz, nullptr));
    TDKS_TRY(launch_interp(c, A->nz, g_rho, 4.0 * M_PI, 1));  // 4 pi wJ interp
  } else {
    TDKS_CU(c, cudaMemsetAsync(g_rho, 0, nf * sizeof(double), c->stream));
  }
  if (c->xc) TDKS_TRY(launch_fxc_add(c, rho, g_h, g_rho));
  return TDKS_OK;
}

}  // namespace

void adjoint_free(tdks_ctx* c) {
  if (c && c->adj) {
    free_adj(static_cast<AdjState*>(c->adj));
    c->adj = nullptr;
  }
}

extern "C" {

tdks_status tdks_objective_forward(tdks_ctx* c, const double* psi0, int n_orb, int n_steps, double dt,
                                   const double* E_host, const double* w_host, const double e[3],
                                   int ckpt_every, double tol, int k_max, int prec, double* J_host,
                                   double* dip_host) {
  if (!c || !psi0 || !E_host || !w_host || !e || !J_host) return TDKS_ERR_ARG;
  if (n_orb < 1 || n_orb > c->n_orb || n_steps < 1 || ckpt_every < 1 || !(dt > 0))
    return tdks_fail(c, TDKS_ERR_ARG, "objective: bad sizes");
  adjoint_free(c);
  AdjState* A = new AdjState();
  c->adj = A;
  A->n_steps = n_steps;
  A->n_orb = n_orb;
  A->ckpt = ckpt_every;
  A->kmax = k_max;
  A->prec = prec;
  A->dt = dt;
  A->tol = tol;
  A->E.assign(E_host, E_host + 6 * (size_t)n_steps);
  A->w.assign(w_host, w_host + n_steps + 1);
  std::memcpy(A->e, e, 3 * sizeof(double));
  A->dip.assign(3 * (size_t)(n_steps + 1), 0.0);
  const size_t nv = (size_t)n_orb * c->n_int, nf = (size_t)(c->n_elem * c->nq3), nn = (size_t)c->n_int;
  TDKS_TRY(amalloc(c, &A->psi, nv));
  TDKS_CU(c, cudaMemcpyAsync(A->psi, psi0, nv * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  double d[3];
  TDKS_TRY(tdks_init_propagation(c, (const double*)A->psi, n_orb, d));
  std::memcpy(&A->dip[0], d, sizeof(d));
  double J = A->w[0] * std::pow(e[0] * d[0] + e[1] * d[1] + e[2] * d[2], 2);
  for (int s = 0; s < n_steps; ++s) {
    if (s % ckpt_every == 0) {
      double2* cp;
      double *h1, *h2, *ph;
      TDKS_TRY(amalloc(c, &cp, nv));
      TDKS_TRY(amalloc(c, &h1, nf));
      TDKS_TRY(amalloc(c, &h2, nf));
      TDKS_TRY(amalloc(c, &ph, nn));
      A->ck_psi.push_back(cp);
      A->ck_h1.push_back(h1);
      A->ck_h2.push_back(h2);
      A->ck_phi.push_back(ph);
      TDKS_CU(c, cudaMemcpyAsync(cp, A->psi, nv * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
      TDKS_CU(c, cudaMemcpyAsync(h1, c->d_vhxc1, nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      TDKS_CU(c, cudaMemcpyAsync(h2, c->d_vhxc2, nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      TDKS_CU(c, cudaMemcpyAsync(ph, c->d_phi, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    }
    tdks_stats st;
    TDKS_TRY(magnus_step_impl(c, A->psi, n_orb, dt, &A->E[6 * s], &A->E[6 * s + 3], tol, k_max, prec,
                              &st, nullptr, nullptr, nullptr));
    std::memcpy(&A->dip[3 * (s + 1)], st.dipole, 3 * sizeof(double));
    J += A->w[s + 1] * std::pow(e[0] * st.dipole[0] + e[1] * st.dipole[1] + e[2] * st.dipole[2], 2);
  }
  *J_host = J;
  if (dip_host) std::memcpy(dip_host, A->dip.data(), A->dip.size() * sizeof(double));
  A->ready = true;
  return TDKS_OK;
}

tdks_status tdks_objective_backward(tdks_ctx* c, int n_s, double* dJdE_host) {
  if (!c || !dJdE_host) return TDKS_ERR_ARG;
  AdjState* A = static_cast<AdjState*>(c->adj);
  if (!A || !A->ready) return tdks_fail(c, TDKS_ERR_ARG, "call tdks_objective_forward first");
  if (n_s < 1 || n_s > 64) return tdks_fail(c, TDKS_ERR_ARG, "n_s in [1, 64]");
  const int n_orb = A->n_orb, K = A->ckpt, N = A->n_steps;
  const size_t nv = (size_t)n_orb * c->n_int, nf = (size_t)(c->n_elem * c->nq3), nn = (size_t)c->n_int;
  const long long nvl = (long long)nv;
  if (!A->seg_psi) {
    TDKS_TRY(amalloc(c, &A->seg_psi, nv * K));
    TDKS_TRY(amalloc(c, &A->seg_half, nv * K));
    TDKS_TRY(amalloc(c, &A->psi_end, nv));
    TDKS_TRY(amalloc(c, &A->seg_vpred, nf * K));
    TDKS_TRY(amalloc(c, &A->seg_vmid, nf * K));
    double2** vs[] = {&A->lam, &A->lam_prev, &A->lam_h, &A->lam_tmp, &A->phis, &A->mus};
    for (auto v : vs) TDKS_TRY(amalloc(c, v, nv));
    double** fs[] = {&A->gh1, &A->gh2, &A->gh1n, &A->grho, &A->gvmid, &A->gvpred};
    for (auto f : fs) TDKS_TRY(amalloc(c, f, nf));
    TDKS_TRY(amalloc(c, &A->ny, nn));
    TDKS_TRY(amalloc(c, &A->nz, nn));
    TDKS_TRY(amalloc(c, &A->d_coef, 2 * (size_t)n_orb * TDKS_KMAX));
    TDKS_TRY(amalloc(c, &A->d_k, 2 * (size_t)n_orb));
  }
  TDKS_CU(c, cudaMemsetAsync(A->lam, 0, nv * sizeof(double2), c->stream));
  TDKS_CU(c, cudaMemsetAsync(A->gh1, 0, nf * sizeof(double), c->stream));
  TDKS_CU(c, cudaMemsetAsync(A->gh2, 0, nf * sizeof(double), c->stream));
  std::vector<double> dJdE(6 * (size_t)N, 0.0);
  const int nseg = (N + K - 1) / K;
  const double* e = A->e;
  const int ngrid = grid_for(nvl);
  const int fgrid = grid_for((long long)nf);
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int s0 = sg * K, s1 = std::min(N, s0 + K);
    // restore the checkpoint and recompute the segment, keeping its intermediates
    TDKS_CU(c, cudaMemcpyAsync(A->psi, A->ck_psi[sg], nv * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    TDKS_CU(c, cudaMemcpyAsync(c->d_vhxc1, A->ck_h1[sg], nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    TDKS_CU(c, cudaMemcpyAsync(c->d_vhxc2, A->ck_h2[sg], nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    TDKS_CU(c, cudaMemcpyAsync(c->d_phi, A->ck_phi[sg], nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    for (int s = s0; s < s1; ++s) {
      const int j = s - s0;
      TDKS_CU(c, cudaMemcpyAsync(A->seg_psi + j * nv, A->psi, nv * sizeof(double2), cudaMemcpyDeviceToDevice,
                                 c->stream));
      tdks_stats st;
      TDKS_TRY(magnus_step_impl(c, A->psi, n_orb, A->dt, &A->E[6 * s], &A->E[6 * s + 3], A->tol, A->kmax,
                                A->prec, &st, A->seg_half + j * nv, A->seg_vpred + j * nf,
                                A->seg_vmid + j * nf));
    }
    TDKS_CU(c, cudaMemcpyAsync(A->psi_end, A->psi, nv * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    for (int s = s1 - 1; s >= s0; --s) {
      const int j = s - s0;
      const double2* psi_prev = A->seg_psi + j * nv;
      const double2* psi_half = A->seg_half + j * nv;
      const double2* psi_new = (s + 1 < s1) ? A->seg_psi + (j + 1) * nv : A->psi_end;
      const double* dn = &A->dip[3 * (s + 1)];
      // a. objective and V_HXC^n terms at psi^n
      TDKS_TRY(launch_density(c, psi_new, n_orb, c->d_rho));
      TDKS_TRY(hxc_adjoint(c, A, c->d_rho, A->gh1, A->grho));
      const double ed = e[0] * dn[0] + e[1] * dn[1] + e[2] * dn[2];
      TDKS_TRY(launch_dipole_sens(c, 2.0 * A->w[s + 1] * ed, e, A->grho));
      TDKS_TRY(launch_density_adjoint(c, psi_new, n_orb, A->grho, A->lam, 1));
      // b. V_HXC^{n-1} sits in the second history slot of state n
      TDKS_CU(c, cudaMemcpyAsync(A->gh1n, A->gh2, nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      // c. full exponential under V_mid
      TDKS_CU(c, cudaMemcpyAsync(c->d_vks, A->seg_vmid + j * nf, nf * sizeof(double), cudaMemcpyDeviceToDevice,
                                 c->stream));
      TDKS_CU(c, cudaMemsetAsync(A->gvmid, 0, nf * sizeof(double), c->stream));
      TDKS_TRY(frechet(c, A, psi_prev, A->lam, A->dt, n_s, A->gvmid, A->lam_prev));
      double g3[3];
      TDKS_TRY(run_dipole(c, A->gvmid, g3, 0));
      for (int k = 0; k < 3; ++k) dJdE[6 * s + 3 + k] = -g3[k];
      // e. V_mid's V_HXC from psi^{n-1/2}
      TDKS_TRY(launch_density(c, psi_half, n_orb, c->d_rho));
      TDKS_TRY(hxc_adjoint(c, A, c->d_rho, A->gvmid, A->grho));
      TDKS_TRY(launch_density_adjoint(c, psi_half, n_orb, A->grho, A->lam_h, 0));
      // f. half exponential under V_pred
      TDKS_CU(c, cudaMemcpyAsync(c->d_vks, A->seg_vpred + j * nf, nf * sizeof(double), cudaMemcpyDeviceToDevice,
                                 c->stream));
      TDKS_CU(c, cudaMemsetAsync(A->gvpred, 0, nf * sizeof(double), c->stream));
      TDKS_TRY(frechet(c, A, psi_prev, A->lam_h, 0.5 * A->dt, n_s, A->gvpred, A->lam_tmp));
      k_axpy_c<<<ngrid, kThreads, 0, c->stream>>>(nvl, 1.0, A->lam_tmp, A->lam_prev);
      TDKS_TRY(run_dipole(c, A->gvpred, g3, 0));
      for (int k = 0; k < 3; ++k) dJdE[6 * s + k] = -g3[k];
      // g. predictor: V_pred = V_N + 1.25 V_HXC^{n-1} - 0.25 V_HXC^{n-2} - E . r
      k_axpby<<<fgrid, kThreads, 0, c->stream>>>((long long)nf, 1.25, A->gvpred, 1.0, A->gh1n);
      k_axpby<<<fgrid, kThreads, 0, c->stream>>>((long long)nf, -0.25, A->gvpred, 0.0, A->gh2);
      c->n_launch += 3;
      std::swap(A->gh1, A->gh1n);
      std::swap(A->lam, A->lam_prev);
      TDKS_CU(c, cudaGetLastError());
    }
  }
  TDKS_CU(c, cudaStreamSynchronize(c->stream));
  std::memcpy(dJdE_host, dJdE.data(), dJdE.size() * sizeof(double));
  return TDKS_OK;
}

}  // extern "C"
