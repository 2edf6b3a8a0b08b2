// Pointwise fields at the Gauss points: nuclear potential, LDA exchange-
// correlation, potential assembly (Eqs. 3, 7, 16), dipole (Sec. V) and the
// delta kick (Sec. VII.A).
#include <cmath>

#include "tdks_internal.h"

namespace {

constexpr int kVecBlocks = 608;     // 4 x 152 SMs
constexpr int kVecThreads = 256;

// Coordinates of Gauss point q of element e.
__device__ __forceinline__ void quad_xyz(const Geom& g, const double* eta, int P1, long long idx,
                                         double* x) {
  const int P2 = P1 * P1, P3 = P2 * P1;
  const long long e = idx / P3;
  const int q = (int)(idx - e * P3);
  const int qx = q % P1, qy = (q / P1) % P1, qz = q / P2;
  const int ex = (int)(e % g.nx);
  const int ey = (int)((e / g.nx) % g.ny);
  const int ez = (int)(e / ((long long)g.nx * g.ny));
  const int ii[3] = {ex, ey, ez};
  const int qq[3] = {qx, qy, qz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double lo = g.brk[d][ii[d]], hi = g.brk[d][ii[d] + 1];
    x[d] = lo + 0.5 * (eta[qq[d]] + 1.0) * (hi - lo);
  }
}

// V_N at the point x for the nuclear-potential kinds of tdks_nuc_kind
__device__ __forceinline__ double nuc_at(const double* x, int kind, double param, int n_nuc,
                                         const double* R, const double* Z) {
  double acc = 0.0;
  if (kind == TDKS_NUC_HARMONIC) {
    const double dx = x[0] - R[0], dy = x[1] - R[1], dz = x[2] - R[2];
    acc = 0.5 * param * param * (dx * dx + dy * dy + dz * dz);
  } else if (kind != TDKS_NUC_NONE) {
    for (int I = 0; I < n_nuc; ++I) {
      const double dx = x[0] - R[3 * I], dy = x[1] - R[3 * I + 1], dz = x[2] - R[3 * I + 2];
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double r = sqrt(r2);
      if (kind == TDKS_NUC_SOFT) {
        acc -= Z[I] / sqrt(r2 + param);
      } else if (kind == TDKS_NUC_BARE) {
        acc -= Z[I] / r;
      } else {  // erf: -Z erf(r/rc)/r, limit 2 Z / (sqrt(pi) rc) at r = 0
        acc -= (r > 0.0) ? Z[I] * erf(r / param) / r : Z[I] * 2.0 / (sqrt(M_PI) * param);
      }
    }
  }
  return acc;
}

__global__ void k_nuclear(Geom g, const double* eta, int P1, long long n, int kind, double param,
                          int n_nuc, const double* R, const double* Z, double* v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double x[3];
    quad_xyz(g, eta, P1, i, x);
    v[i] = nuc_at(x, kind, param, n_nuc, R, Z);
  }
}

// V_N at the interior nodes (collocated potential of the GLL variant)
__global__ void k_nuclear_nodes(const double* cx, const double* cy, const double* cz, int nix, int niy,
                                long long n, int kind, double param, int n_nuc, const double* R,
                                const double* Z, double* v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(i % nix) + 1;
    const int J = (int)((i / nix) % niy) + 1;
    const int K = (int)(i / ((long long)nix * niy)) + 1;
    const double x[3] = {cx[I], cy[J], cz[K]};
    v[i] = nuc_at(x, kind, param, n_nuc, R, Z);
  }
}

// Perdew-Zunger (1981) fit to the Ceperley-Alder data, spin-unpolarized:
//   r_s = (3 / (4 pi rho))^(1/3);  v_x = -(3 rho / pi)^(1/3)
//   r_s >= 1: e_c = g/(1 + b1 sqrt(rs) + b2 rs),
//             v_c = e_c (1 + 7/6 b1 sqrt(rs) + 4/3 b2 rs)/(1 + b1 sqrt(rs) + b2 rs)
//   r_s <  1: v_c = A ln rs + (B - A/3) + 2/3 C rs ln rs + (2D - C)/3 rs
//   g = -0.1423, b1 = 1.0529, b2 = 0.3334, A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116
__device__ __forceinline__ double pz81_vxc(double rho) {
  if (!(rho >= 1e-14)) return 0.0;
  const double rs = cbrt(3.0 / (4.0 * M_PI * rho));
  const double vx = -cbrt(3.0 * rho / M_PI);
  double vc;
  if (rs >= 1.0) {
    const double sq = sqrt(rs);
    const double den = 1.0 + 1.0529 * sq + 0.3334 * rs;
    vc = (-0.1423 / den) * (1.0 + (7.0 / 6.0) * 1.0529 * sq + (4.0 / 3.0) * 0.3334 * rs) / den;
  } else {
    const double lr = log(rs);
    vc = 0.0311 * lr + (-0.048 - 0.0311 / 3.0) + (2.0 / 3.0) * 0.0020 * rs * lr +
         (2.0 * -0.0116 - 0.0020) / 3.0 * rs;
  }
  return vx + vc;
}

// d v_xc / d rho of the same fit (for the adjoint): with x = rho^(1/3) terms
//   dv_x/drho = -(1/3)(3/pi)^(1/3) rho^(-2/3),  dv_c/drho = dv_c/dr_s * (-r_s / (3 rho))
//   r_s >= 1: v_c = g N / D^2, dv_c/dr_s = g (N' D - 2 N D') / D^3,
//             D = 1 + b1 sqrt(rs) + b2 rs, N = 1 + 7/6 b1 sqrt(rs) + 4/3 b2 rs
//   r_s <  1: dv_c/dr_s = A / rs + 2/3 C (ln rs + 1) + (2D - C)/3
__device__ __forceinline__ double pz81_fxc(double rho) {
  if (!(rho >= 1e-14)) return 0.0;
  const double rs = cbrt(3.0 / (4.0 * M_PI * rho));
  const double dvx = -(1.0 / 3.0) * cbrt(3.0 / M_PI) / cbrt(rho * rho);
  double dvc;
  if (rs >= 1.0) {
    const double sq = sqrt(rs);
    const double D = 1.0 + 1.0529 * sq + 0.3334 * rs;
    const double N = 1.0 + (7.0 / 6.0) * 1.0529 * sq + (4.0 / 3.0) * 0.3334 * rs;
    const double dD = 0.5 * 1.0529 / sq + 0.3334;
    const double dN = (7.0 / 12.0) * 1.0529 / sq + (4.0 / 3.0) * 0.3334;
    dvc = -0.1423 * (dN * D - 2.0 * N * dD) / (D * D * D);
  } else {
    dvc = 0.0311 / rs + (2.0 / 3.0) * 0.0020 * (log(rs) + 1.0) + (2.0 * -0.0116 - 0.0020) / 3.0;
  }
  return dvx + dvc * (-rs / (3.0 * rho));
}

__global__ void k_fxc_add(const double* rho, const double* gh, double* grho, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    grho[i] += pz81_fxc(rho[i]) * gh[i];
}

// g[q] += coef wJ_q (e . x_q): sensitivity of e . mu to rho at the Gauss points
__global__ void k_dipole_sens(Geom g, const double* eta, const double* w, int P1, long long n,
                              double coef, double ex, double ey, double ez, double* out) {
  const int P2 = P1 * P1, P3 = P2 * P1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double x[3];
    quad_xyz(g, eta, P1, i, x);
    const long long e = i / P3;
    const int q = (int)(i - e * P3);
    const int ix = (int)(e % g.nx), iy = (int)((e / g.nx) % g.ny), iz = (int)(e / ((long long)g.nx * g.ny));
    const double J = 0.125 * (g.brk[0][ix + 1] - g.brk[0][ix]) * (g.brk[1][iy + 1] - g.brk[1][iy]) *
                     (g.brk[2][iz + 1] - g.brk[2][iz]);
    out[i] += coef * J * w[q % P1] * w[(q / P1) % P1] * w[q / P2] * (ex * x[0] + ey * x[1] + ez * x[2]);
  }
}

__global__ void k_xc(const double* rho, double* vxc, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    vxc[i] = pz81_vxc(rho[i]);
}

__global__ void k_combine(Geom g, const double* eta, int P1, long long n, double* v,
                          const double* vn, double a1, const double* h1, double a2,
                          const double* h2, const double* h3, double Ex, double Ey, double Ez) {
  const bool field = (Ex != 0.0 || Ey != 0.0 || Ez != 0.0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double acc = vn[i];
    if (h1) acc += a1 * h1[i];
    if (h2) acc += a2 * h2[i];
    if (h3) acc += h3[i];
    if (field) {
      double x[3];
      quad_xyz(g, eta, P1, i, x);
      acc -= Ex * x[0] + Ey * x[1] + Ez * x[2];
    }
    v[i] = acc;
  }
}

// Per-block partial sums of J w_qx w_qy w_qz x_q rho_q (3 components).
__global__ void k_dipole_part(Geom g, const double* eta, const double* w, int P1, long long n,
                              const double* rho, double* part, int weighted) {
  __shared__ double red[3][kVecThreads / 32];
  double acc[3] = {0.0, 0.0, 0.0};
  const int P2 = P1 * P1, P3 = P2 * P1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double x[3];
    quad_xyz(g, eta, P1, i, x);
    const long long e = i / P3;
    const int q = (int)(i - e * P3);
    const int ex = (int)(e % g.nx), ey = (int)((e / g.nx) % g.ny), ez = (int)(e / ((long long)g.nx * g.ny));
    const double J = 0.125 * (g.brk[0][ex + 1] - g.brk[0][ex]) * (g.brk[1][ey + 1] - g.brk[1][ey]) *
                     (g.brk[2][ez + 1] - g.brk[2][ez]);
    const double m = weighted ? J * w[q % P1] * w[(q / P1) % P1] * w[q / P2] * rho[i] : rho[i];
    acc[0] += m * x[0];
    acc[1] += m * x[1];
    acc[2] += m * x[2];
  }
  for (int d = 0; d < 3; ++d) {
    double v = acc[d];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[d][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int k = 0; k < kVecThreads / 32; ++k) s += red[threadIdx.x][k];
    part[threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_sum_parts3(const double* part, int nb, double* out) {
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += part[threadIdx.x * nb + k];
    out[threadIdx.x] = s;
  }
}

// d = sum of the partials, written to base + (*step) * stride (step counter on the device)
__global__ void k_sum_parts3_at(const double* part, int nb, double* base, const int* step,
                                int64_t stride) {
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += part[threadIdx.x * nb + k];
    base[(long long)(*step) * stride + threadIdx.x] = s;
  }
}

__global__ void k_counter_add(int* counter, int inc) {
  if (threadIdx.x == 0) *counter += inc;
}

__global__ void k_kick(const double* cx, const double* cy, const double* cz, int nix, int niy,
                       long long n, int n_orb, double2* psi, double kappa, double dx, double dy,
                       double dz) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(i % nix) + 1;
    const int J = (int)((i / nix) % niy) + 1;
    const int K = (int)(i / ((long long)nix * niy)) + 1;
    const double s = dx * cx[I] + dy * cy[J] + dz * cz[K];
    double sn, cs;
    sincos(-kappa * s, &sn, &cs);
    for (int o = 0; o < n_orb; ++o) {
      double2 v = psi[(long long)o * n + i];
      psi[(long long)o * n + i] = make_double2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
    }
  }
}

int vec_grid(long long n) {
  long long b = (n + kVecThreads - 1) / kVecThreads;
  return (int)(b < kVecBlocks ? (b < 1 ? 1 : b) : kVecBlocks);
}

}  // namespace

tdks_status launch_nuclear(tdks_ctx* c) {
  const long long n = c->n_elem * c->nq3;
  k_nuclear<<<vec_grid(n), kVecThreads, 0, c->stream>>>(
      tdks_geom(c), c->d_tab + tab_off_eta(c->P1), c->P1, n, c->nuc_kind, c->nuc_param, c->n_nuc,
      c->d_R, c->d_Z, c->d_vnuc);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

tdks_status launch_fxc_add(tdks_ctx* c, const double* rho, const double* g_h, double* g_rho) {
  const long long n = c->n_elem * c->nq3;
  k_fxc_add<<<vec_grid(n), kVecThreads, 0, c->stream>>>(rho, g_h, g_rho, n);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

tdks_status launch_dipole_sens(tdks_ctx* c, double coef, const double e[3], double* g_rho) {
  const long long n = c->n_elem * c->nq3;
  k_dipole_sens<<<vec_grid(n), kVecThreads, 0, c->stream>>>(
      tdks_geom(c), c->d_tab + tab_off_eta(c->P1), c->d_tab + tab_off_w(c->P1), c->P1, n, coef,
      e[0], e[1], e[2], g_rho);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

tdks_status launch_xc(tdks_ctx* c, const double* rho, double* vxc) {
  const long long n = c->n_elem * c->nq3;
  k_xc<<<vec_grid(n), kVecThreads, 0, c->stream>>>(rho, vxc, n);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

tdks_status launch_combine(tdks_ctx* c, double* v_out, const double* vn, double a1,
                           const double* h1, double a2, const double* h2, const double* h3,
                           const double E[3]) {
  const long long n = c->n_elem * c->nq3;
  const double z[3] = {0, 0, 0};
  const double* e = E ? E : z;
  k_combine<<<vec_grid(n), kVecThreads, 0, c->stream>>>(tdks_geom(c), c->d_tab + tab_off_eta(c->P1),
                                                        c->P1, n, v_out, vn, a1, h1, a2, h2, h3,
                                                        e[0], e[1], e[2]);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

tdks_status run_dipole(tdks_ctx* c, const double* rho, double d[3], int weighted) {
  const long long n = c->n_elem * c->nq3;
  const int nb = vec_grid(n);
  double* part = c->d_part;                 // 3 * nb doubles
  double* out = c->d_part + 3 * kVecBlocks;
  k_dipole_part<<<nb, kVecThreads, 0, c->stream>>>(tdks_geom(c), c->d_tab + tab_off_eta(c->P1),
                                                   c->d_tab + tab_off_w(c->P1), c->P1, n, rho, part,
                                                   weighted);
  k_sum_parts3<<<1, 32, 0, c->stream>>>(part, nb, out);
  c->n_launch += 2;
  TDKS_CU(c, cudaGetLastError());
  TDKS_CU(c, cudaMemcpyAsync(c->h_red, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TDKS_CU(c, cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 3; ++k) d[k] = c->h_red[k];
  return TDKS_OK;
}

tdks_status launch_kick(tdks_ctx* c, double2* psi, int n_orb, double kappa, const double dir[3]) {
  k_kick<<<vec_grid(c->n_int), kVecThreads, 0, c->stream>>>(
      c->d_coord[0], c->d_coord[1], c->d_coord[2], c->Ni[0], c->Ni[1], c->n_int, n_orb, psi, kappa,
      dir[0], dir[1], dir[2]);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

// run_dipole without the host read, for stream capture
tdks_status dipole_graph(tdks_ctx* c, const double* rho, double* base, const int* step,
                         int64_t step_stride) {
  const long long n = c->n_elem * c->nq3;
  const int nb = vec_grid(n);
  double* part = c->d_part;
  k_dipole_part<<<nb, kVecThreads, 0, c->stream>>>(tdks_geom(c), c->d_tab + tab_off_eta(c->P1),
                                                   c->d_tab + tab_off_w(c->P1), c->P1, n, rho, part, 1);
  k_sum_parts3_at<<<1, 32, 0, c->stream>>>(part, nb, base, step, step_stride);
  c->n_launch += 2;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

cudaError_t launch_counter_add(int* counter, int inc, cudaStream_t st) {
  k_counter_add<<<1, 32, 0, st>>>(counter, inc);
  return cudaGetLastError();
}

tdks_status launch_nuclear_nodes(tdks_ctx* c, double* v) {
  k_nuclear_nodes<<<vec_grid(c->n_int), kVecThreads, 0, c->stream>>>(
      c->d_coord[0], c->d_coord[1], c->d_coord[2], c->Ni[0], c->Ni[1], c->n_int, c->nuc_kind, c->nuc_param,
      c->n_nuc, c->d_R, c->d_Z, v);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}
