// Variants of the propagation step and the spectrum post-processing.
//
// * Self-consistent midpoint step (Sec. VI.B, the approach the predictor-corrector
//   replaces): V_mid = 1.5 V_HXC^{n-1} - 0.5 V_HXC^{n-2}; then repeatedly
//   psibar^n = exp(-i dt Hbar[V_N + V_mid - E(t + dt/2).r]) psibar^{n-1},
//   V_HXC^n from its density, V_mid <- (V_HXC^{n-1} + V_HXC^n) / 2, until the largest change
//   of V_mid is at most sc_tol.
// * Absorption spectrum (Sec. VII): alpha_aa(omega) = -(1/kappa) int_0^T e^{i omega t}
//   g(t) (d_a(t) - d_a(0)) dt with g(t) = exp(-window t^2) (trapezoid rule on the
//   steps; the minus sign is the impulse of the kick psi(0) = exp(-i kappa r.d) psi_GS),
//   and S(omega) = (2 omega / 3 pi) Im alpha_aa(omega) per kick direction.
#include <cmath>
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

__global__ void k_lin2(long long n, double* out, double a, const double* x, double b, const double* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = a * x[i] + b * y[i];
}

// per-block max |x - y|
__global__ void k_maxdiff(long long n, const double* x, const double* y, double* part) {
  __shared__ double red[kThreads / 32];
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i] - y[i]));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) s = fmax(s, red[k]);
    part[blockIdx.x] = s;
  }
}

// alpha(omega_k) for one kick direction: one thread per frequency, the sum over the
// steps in ascending order
__global__ void k_spectrum(int n_t, const double* resp, double dt, double kappa, double window,
                           int n_om, const double* om, double2* alpha) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_om) return;
  double re = 0.0, im = 0.0;
  for (int n = 0; n < n_t; ++n) {
    const double t = dt * n;
    const double w = (n == 0 || n == n_t - 1) ? 0.5 * dt : dt;
    const double f = w * exp(-window * t * t) * resp[n];
    double s, c;
    sincos(om[k] * t, &s, &c);
    re = fma(f, c, re);
    im = fma(f, s, im);
  }
  alpha[k] = make_double2(-re / kappa, -im / kappa);
}

}  // namespace

extern "C" {

tdks_status tdks_magnus_step_sc(tdks_ctx* c, double* psi_d, int n_orb, double dt, const double Eh[3],
                                double tol, int k_max, int prec, double sc_tol, int sc_maxit,
                                tdks_stats* stats, int* iters) {
  if (!c || !psi_d || !Eh) return TDKS_ERR_ARG;
  if (n_orb < 1 || n_orb > c->n_orb) return tdks_fail(c, TDKS_ERR_ARG, "n_orb out of range");
  if (!c->propagation_ready) return tdks_fail(c, TDKS_ERR_ARG, "call tdks_init_propagation first");
  if (!(dt > 0) || !(tol > 0) || !(sc_tol > 0) || sc_maxit < 1)
    return tdks_fail(c, TDKS_ERR_ARG, "dt, tol, sc_tol > 0 and sc_maxit >= 1");
  double2* psi = reinterpret_cast<double2*>(psi_d);
  const long long nf = c->n_elem * c->nq3;
  const size_t vb = (size_t)n_orb * c->n_int * sizeof(double2);
  if (!c->d_psi_half) {
    if (cudaMalloc(&c->d_psi_half, (size_t)c->n_orb * c->n_int * sizeof(double2)) != cudaSuccess) {
      cudaGetLastError();
      return tdks_fail(c, TDKS_ERR_NOMEM, "orbital buffer");
    }
  }
  double *vmid = nullptr, *vnext = nullptr, *part = nullptr;
  const int nb = grid_for(nf);
  if (cudaMalloc(&vmid, nf * sizeof(double)) != cudaSuccess || cudaMalloc(&vnext, nf * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&part, nb * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(vmid);
    cudaFree(vnext);
    return tdks_fail(c, TDKS_ERR_NOMEM, "self-consistent step buffers");
  }
  auto done = [&](tdks_status s) {
    cudaFree(vmid);
    cudaFree(vnext);
    cudaFree(part);
    return s;
  };
  tdks_stats st{};
  std::vector<double> hp(nb);
  k_lin2<<<nb, kThreads, 0, c->stream>>>(nf, vmid, 1.5, c->d_vhxc1, -0.5, c->d_vhxc2);
  c->n_launch += 1;
  int it = 0;
  bool conv = false;
  while (it < sc_maxit) {
    ++it;
    tdks_status s = launch_combine(c, c->d_vks, c->d_vnuc, 1.0, vmid, 0.0, nullptr, nullptr, Eh);
    int kseen = 0, nsub = 0;
    int64_t app = 0;
    if (s == TDKS_OK)
      s = run_expm(c, psi, c->d_psi_half, n_orb, dt, tol, k_max, prec, nullptr, &kseen, &app, &nsub);
    if (s == TDKS_OK) s = vhxc_of(c, c->d_psi_half, n_orb, c->d_vtmp, &st.cg_iters[1], prec);
    if (s != TDKS_OK) return done(s);
    st.k_full_max = kseen > st.k_full_max ? kseen : st.k_full_max;
    st.applies += app;
    st.substeps += nsub;
    k_lin2<<<nb, kThreads, 0, c->stream>>>(nf, vnext, 0.5, c->d_vhxc1, 0.5, c->d_vtmp);
    k_maxdiff<<<nb, kThreads, 0, c->stream>>>(nf, vnext, vmid, part);
    c->n_launch += 2;
    if (cudaMemcpyAsync(hp.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      cudaGetLastError();
      return done(tdks_fail(c, TDKS_ERR_CUDA, "self-consistent step"));
    }
    double delta = 0.0;
    for (double v : hp) delta = delta > v ? delta : v;
    std::swap(vmid, vnext);
    if (!std::isfinite(delta)) return done(tdks_fail(c, TDKS_ERR_NAN, "non-finite midpoint potential"));
    if (delta <= sc_tol) {
      conv = true;
      break;
    }
  }
  if (iters) *iters = it;
  if (!conv) return done(tdks_fail(c, TDKS_ERR_NOT_CONVERGED, "self-consistent midpoint iteration cap"));
  // history V_HXC^{n-2} <- V_HXC^{n-1}, V_HXC^{n-1} <- V_HXC^n; orbitals; dipole of rho(psi^n)
  std::swap(c->d_vhxc1, c->d_vhxc2);
  if (cudaMemcpyAsync(c->d_vhxc1, c->d_vtmp, nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(psi, c->d_psi_half, vb, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return done(tdks_fail(c, TDKS_ERR_CUDA, "self-consistent step"));
  }
  tdks_status s = run_dipole(c, c->d_rho, st.dipole);
  if (stats) *stats = st;
  return done(s);
}

tdks_status tdks_spectrum(const double* dip_host, int n_t, double dt, double kappa, const double dir[3],
                          double window, const double* omega_host, int n_om, double* alpha_host,
                          double* S_host) {
  if (!dip_host || !dir || !omega_host || n_t < 2 || n_om < 1 || !(dt > 0) || kappa == 0.0 || window < 0)
    return TDKS_ERR_ARG;
  const double nrm = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  if (!(nrm > 0)) return TDKS_ERR_ARG;
  std::vector<double> resp(n_t);
  for (int n = 0; n < n_t; ++n) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += (dip_host[3 * n + k] - dip_host[k]) * dir[k] / nrm;
    resp[n] = s;
  }
  double *d_resp = nullptr, *d_om = nullptr;
  double2* d_alpha = nullptr;
  if (cudaMalloc(&d_resp, n_t * sizeof(double)) != cudaSuccess || cudaMalloc(&d_om, n_om * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_alpha, n_om * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_resp);
    cudaFree(d_om);
    return TDKS_ERR_NOMEM;
  }
  std::vector<double2> a(n_om);
  cudaError_t e = cudaMemcpy(d_resp, resp.data(), n_t * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_om, omega_host, n_om * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_spectrum<<<(n_om + 127) / 128, 128>>>(n_t, d_resp, dt, kappa, window, n_om, d_om, d_alpha);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(a.data(), d_alpha, n_om * sizeof(double2), cudaMemcpyDeviceToHost);
  cudaFree(d_resp);
  cudaFree(d_om);
  cudaFree(d_alpha);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TDKS_ERR_CUDA;
  }
  for (int k = 0; k < n_om; ++k) {
    if (alpha_host) {
      alpha_host[2 * k] = a[k].x;
      alpha_host[2 * k + 1] = a[k].y;
    }
    if (S_host) S_host[k] = 2.0 * omega_host[k] / (3.0 * M_PI) * a[k].y;
  }
  return TDKS_OK;
}

}  // extern "C"
