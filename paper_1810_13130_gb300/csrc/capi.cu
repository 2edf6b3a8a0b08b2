// C ABI: context set-up and the public entry points of include/tdks.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <string>
#include <vector>

#include "tdks_internal.h"

tdks_status tdks_fail(tdks_ctx* c, tdks_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

tdks_status tdks_cuda_check(tdks_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return tdks_fail(c, TDKS_ERR_NOMEM, m);
  return tdks_fail(c, TDKS_ERR_CUDA, m);
}

Geom tdks_geom(const tdks_ctx* c) {
  Geom g;
  g.nx = c->nx;
  g.ny = c->ny;
  g.nz = c->nz;
  g.p = c->p;
  g.nix = c->Ni[0];
  g.niy = c->Ni[1];
  g.niz = c->Ni[2];
  for (int d = 0; d < 3; ++d) {
    g.brk[d] = c->d_brk[d];
    g.s[d] = c->d_s[d];
    g.sf[d] = c->d_sf[d];
  }
  g.gauss = c->d_tab + tab_off_eta(c->P1);
  for (int d = 0; d < 3; ++d) g.ih[d] = c->d_ih[d];
  g.wq = c->d_tab + tab_off_w(c->P1);
  return g;
}

namespace {

template <typename T>
tdks_status dalloc(tdks_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return tdks_fail(c, TDKS_ERR_NOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes");
  }
  return TDKS_OK;
}

template <typename T>
tdks_status upload(tdks_ctx* c, T** p, const std::vector<T>& h) {
  TDKS_TRY(dalloc(c, p, h.size()));
  TDKS_CU(c, cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return TDKS_OK;
}

void free_ctx(tdks_ctx* c) {
  kb_free(c);
  if (c) kgraph_free(c);
  if (c) {
    cudaFree(c->d_ro_part);
    cudaFree(c->d_ro_h);
  }
  if (!c) return;
  for (int d = 0; d < 3; ++d) {
    cudaFree(c->d_brk[d]);
    cudaFree(c->d_s[d]);
    cudaFree(c->d_sf[d]);
    cudaFree(c->d_coord[d]);
    cudaFree(c->d_kd[d]);
    cudaFree(c->d_md[d]);
    cudaFree(c->d_ih[d]);
  }
  cudaFree(c->d_tab);
  cudaFree(c->d_tabf);
  cudaFree(c->d_tabdf);
  cudaFree(c->d_tabbf);
  cudaFree(c->d_occ);
  cudaFree(c->d_R);
  cudaFree(c->d_Z);
  cudaFree(c->d_vks);
  cudaFree(c->d_vnuc);
  cudaFree(c->d_vhxc1);
  cudaFree(c->d_vhxc2);
  cudaFree(c->d_vtmp);
  cudaFree(c->d_rho);
  cudaFree(c->d_vh);
  cudaFree(c->d_phi);
  cudaFree(c->d_b);
  cudaFree(c->d_r);
  cudaFree(c->d_pv);
  cudaFree(c->d_Ap);
  cudaFree(c->d_cg);
  for (int w = 0; w < 2; ++w) {
    cudaFree(c->d_Vw[w]);
    cudaFree(c->d_kryw[w]);
  }
  cudaFree(c->d_psi_half);
  cudaFree(c->d_evec);
  cudaFree(c->d_psi_e2e);
  cudaFree(c->d_part);
  cudaFree(c->d_z);
  cudaFree(c->d_t1);
  cudaFree(c->d_t2);
  cudaFree(c->d_invdiag);
  for (int d = 0; d < 3; ++d) {
    cudaFree(c->d_fdmS[d]);
    cudaFree(c->d_fdmL[d]);
  }
  if (c->h_red) cudaFreeHost(c->h_red);
  adjoint_free(c);
  if (c->ev[0]) cudaEventDestroy(c->ev[0]);
  if (c->ev[1]) cudaEventDestroy(c->ev[1]);
  delete c;
}

// float -> nearest bfloat16 (ties to even), returned as a float; finite inputs only
float round_bf16(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// Folded storage of a centrosymmetric n x n matrix (layout in tdks_internal.h).
void fold_centrosymmetric(const double* M, int n, double* out) {
  const int h = n / 2;
  for (int q = 0; q < h; ++q)
    for (int i = 0; i < h; ++i) {
      out[q * h + i] = 0.5 * (M[q * n + i] + M[q * n + (n - 1 - i)]);
      out[h * h + q * h + i] = 0.5 * (M[q * n + i] - M[q * n + (n - 1 - i)]);
    }
  double* mc = out + 2 * h * h;
  double* mr = mc + h;
  for (int q = 0; q < h; ++q) mc[q] = (n & 1) ? M[q * n + h] : 0.0;
  for (int i = 0; i < h; ++i) mr[i] = (n & 1) ? M[h * n + i] : 0.0;
  mr[h] = (n & 1) ? M[h * n + h] : 0.0;
}

tdks_status check_orb(tdks_ctx* c, int n_orb) {
  if (n_orb < 1 || n_orb > c->n_orb)
    return tdks_fail(c, TDKS_ERR_ARG, "n_orb must be in [1, system n_orb]");
  return TDKS_OK;
}

}  // namespace

bool valid_prec(int prec) {
  return prec == TDKS_FP64 || prec == TDKS_FP32 || prec == TDKS_DF64 || prec == TDKS_BF16 ||
         prec == TDKS_MIXED;
}

// V_HXC = V_H[rho] + V_XC[rho] of the orbitals psi; rho left in c->d_rho.
tdks_status vhxc_of(tdks_ctx* c, const double2* psi, int n_orb, double* out, int* cg_iters, int prec) {
  const size_t nf = (size_t)(c->n_elem * c->nq3);
  TDKS_TRY(launch_density(c, psi, n_orb, c->d_rho, prec == TDKS_MIXED ? TDKS_DF64 : prec));
  if (c->hartree) {
    TDKS_TRY(run_hartree(c, c->d_rho, c->d_vh, cg_iters, prec == TDKS_DF64 || prec == TDKS_MIXED));
  } else {
    TDKS_CU(c, cudaMemsetAsync(c->d_vh, 0, nf * sizeof(double), c->stream));
    if (cg_iters) *cg_iters = 0;
  }
  if (c->xc) {
    TDKS_TRY(launch_xc(c, c->d_rho, c->d_vtmp));
    TDKS_TRY(launch_combine(c, out, c->d_vh, 1.0, c->d_vtmp, 0.0, nullptr, nullptr, nullptr));
  } else {
    TDKS_CU(c, cudaMemcpyAsync(out, c->d_vh, nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  }
  return TDKS_OK;
}


// vhxc_of for stream capture (fixed-length Poisson CG, no host reads)
tdks_status vhxc_graph(tdks_ctx* c, const double2* psi, int n_orb, double* out, int n_iter, int* err,
                       int prec) {
  const size_t nf = (size_t)(c->n_elem * c->nq3);
  TDKS_TRY(launch_density(c, psi, n_orb, c->d_rho, prec));
  if (c->hartree) {
    TDKS_TRY(hartree_graph(c, c->d_rho, c->d_vh, n_iter, err, prec == TDKS_DF64 || prec == TDKS_MIXED));
  } else {
    TDKS_CU(c, cudaMemsetAsync(c->d_vh, 0, nf * sizeof(double), c->stream));
  }
  if (c->xc) {
    TDKS_TRY(launch_xc(c, c->d_rho, c->d_vtmp));
    TDKS_TRY(launch_combine(c, out, c->d_vh, 1.0, c->d_vtmp, 0.0, nullptr, nullptr, nullptr));
  } else {
    TDKS_CU(c, cudaMemcpyAsync(out, c->d_vh, nf * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  }
  return TDKS_OK;
}


extern "C" {

const char* tdks_status_string(int s) {
  switch (s) {
    case TDKS_OK: return "ok";
    case TDKS_ERR_ARG: return "invalid argument";
    case TDKS_ERR_CUDA: return "CUDA error";
    case TDKS_ERR_NOMEM: return "out of device memory";
    case TDKS_ERR_NOT_CONVERGED: return "not converged";
    case TDKS_ERR_TIMEOUT: return "timeout";
    case TDKS_ERR_NAN: return "non-finite value";
    default: return "unknown status";
  }
}

const char* tdks_last_error(const tdks_ctx* c) { return c ? c->err.c_str() : "null context"; }

tdks_status tdks_create(const tdks_mesh_desc* m, const tdks_system_desc* s, void* stream,
                        tdks_ctx** out) {
  if (!out) return TDKS_ERR_ARG;
  *out = nullptr;
  if (!m || !s) return TDKS_ERR_ARG;
  if (m->nx < 1 || m->ny < 1 || m->nz < 1 || !m->X || !m->Y || !m->Z) return TDKS_ERR_ARG;
  if (m->p < 1 || m->p > TDKS_MAX_P1 - 1) return TDKS_ERR_ARG;
  if (m->nq != 0 && m->nq != m->p + 1) return TDKS_ERR_ARG;
  if (s->n_orb < 1 || !s->occ || s->n_nuc < 0 || (s->n_nuc > 0 && (!s->R || !s->Z))) return TDKS_ERR_ARG;
  if (s->nuc_kind < TDKS_NUC_NONE || s->nuc_kind > TDKS_NUC_HARMONIC) return TDKS_ERR_ARG;
  if ((s->nuc_kind == TDKS_NUC_ERF && !(s->nuc_param > 0)) ||
      (s->nuc_kind == TDKS_NUC_SOFT && !(s->nuc_param > 0)))
    return TDKS_ERR_ARG;
  const int nn[3] = {m->nx, m->ny, m->nz};
  const double* br[3] = {m->X, m->Y, m->Z};
  for (int d = 0; d < 3; ++d) {
    if (nn[d] * m->p < 2) return TDKS_ERR_ARG;   // at least one interior node per axis
    for (int i = 0; i < nn[d]; ++i)
      if (!(br[d][i + 1] > br[d][i])) return TDKS_ERR_ARG;
  }
  tdks_ctx* c = new tdks_ctx();
  c->nx = m->nx;
  c->ny = m->ny;
  c->nz = m->nz;
  c->p = m->p;
  c->P1 = m->p + 1;
  c->nq = m->p + 1;
  c->nq3 = (int64_t)c->nq * c->nq * c->nq;
  c->stream = (cudaStream_t)stream;
  c->n_orb = s->n_orb;
  c->occ.assign(s->occ, s->occ + s->n_orb);
  c->n_nuc = s->n_nuc;
  c->R.assign(3 * std::max(s->n_nuc, 1), 0.0);
  c->Z.assign(std::max(s->n_nuc, 1), 0.0);
  if (s->n_nuc > 0) {
    std::memcpy(c->R.data(), s->R, 3 * s->n_nuc * sizeof(double));
    std::memcpy(c->Z.data(), s->Z, s->n_nuc * sizeof(double));
  }
  c->nuc_kind = s->nuc_kind;
  c->nuc_param = s->nuc_param;
  c->hartree = s->hartree ? 1 : 0;
  c->xc = s->xc ? 1 : 0;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return TDKS_ERR_CUDA;
  }
  Tables1D t;
  try {
    t = tdks_build_tables(c->p, c->nq);
  } catch (const std::exception&) {
    delete c;
    return TDKS_ERR_ARG;
  }
  const int P1 = c->P1;
  tdks_status st = TDKS_OK;
  auto fail = [&](tdks_status e) {
    free_ctx(c);
    return e;
  };
  // 1-D arrays per axis
  for (int d = 0; d < 3; ++d) {
    c->brk[d].assign(br[d], br[d] + nn[d] + 1);
    c->Nn[d] = nn[d] * c->p + 1;
    c->Ni[d] = c->Nn[d] - 2;
    std::vector<double> coord(c->Nn[d]), mass(c->Nn[d], 0.0), kd(c->Nn[d], 0.0),
        md(c->Nn[d], 0.0), sv(c->Nn[d], 0.0);
    for (int e = 0; e < nn[d]; ++e) {
      const double h = br[d][e + 1] - br[d][e];
      for (int a = 0; a < P1; ++a) {
        const int I = e * c->p + a;
        coord[I] = br[d][e] + 0.5 * (t.xi[a] + 1.0) * h;
        mass[I] += 0.5 * h * t.w[a];
        kd[I] += t.K1[a * P1 + a] / h;
        md[I] += h * t.Mg[a * P1 + a];
      }
    }
    coord[c->Nn[d] - 1] = br[d][nn[d]];
    for (int I = 0; I < c->Nn[d]; ++I) sv[I] = 1.0 / std::sqrt(mass[I]);
    if ((st = upload(c, &c->d_brk[d], c->brk[d])) != TDKS_OK) return fail(st);
    if ((st = upload(c, &c->d_coord[d], coord)) != TDKS_OK) return fail(st);
    if ((st = upload(c, &c->d_s[d], sv)) != TDKS_OK) return fail(st);
    std::vector<float> svf(sv.begin(), sv.end());
    if ((st = upload(c, &c->d_sf[d], svf)) != TDKS_OK) return fail(st);
    if ((st = upload(c, &c->d_kd[d], kd)) != TDKS_OK) return fail(st);
    if ((st = upload(c, &c->d_md[d], md)) != TDKS_OK) return fail(st);
    std::vector<double> ih(nn[d]);
    for (int e = 0; e < nn[d]; ++e) ih[e] = 1.0 / (br[d][e + 1] - br[d][e]);
    if ((st = upload(c, &c->d_ih[d], ih)) != TDKS_OK) return fail(st);
  }
  c->n_int = (int64_t)c->Ni[0] * c->Ni[1] * c->Ni[2];
  c->n_elem = (int64_t)c->nx * c->ny * c->nz;
  // tables (double and float copies)
  std::vector<double> tab(tab_size(P1), 0.0);
  std::memcpy(&tab[tab_off_B(P1)], t.B.data(), P1 * P1 * sizeof(double));
  std::memcpy(&tab[tab_off_Kq(P1)], t.Kq.data(), P1 * P1 * sizeof(double));
  std::memcpy(&tab[tab_off_w(P1)], t.omega.data(), P1 * sizeof(double));
  std::memcpy(&tab[tab_off_K1(P1)], t.K1.data(), P1 * P1 * sizeof(double));
  std::memcpy(&tab[tab_off_Mg(P1)], t.Mg.data(), P1 * P1 * sizeof(double));
  std::memcpy(&tab[tab_off_eta(P1)], t.eta.data(), P1 * sizeof(double));
  {
    // folded (even-odd) forms of B (q <- i), B^T (i <- q) and Kq
    std::vector<double> Bt(P1 * P1);
    for (int q = 0; q < P1; ++q)
      for (int i = 0; i < P1; ++i) Bt[i * P1 + q] = t.B[q * P1 + i];
    fold_centrosymmetric(t.B.data(), P1, &tab[tab_off_csB(P1)]);
    fold_centrosymmetric(Bt.data(), P1, &tab[tab_off_csBT(P1)]);
    fold_centrosymmetric(t.Kq.data(), P1, &tab[tab_off_csK(P1)]);
    // GLL-collocation variant: GLL weights and the folded 1-D stiffness K1 = D^T W D
    std::memcpy(&tab[tab_off_wl(P1)], t.w.data(), P1 * sizeof(double));
    fold_centrosymmetric(t.K1.data(), P1, &tab[tab_off_csK1(P1)]);
  }
  std::vector<float> tabf(tab.begin(), tab.end());
  std::vector<float> tabdf(2 * tab.size());
  for (size_t k = 0; k < tab.size(); ++k) {
    const float hi = (float)tab[k];
    tabdf[2 * k] = hi;
    tabdf[2 * k + 1] = (float)(tab[k] - (double)hi);
  }
  if ((st = upload(c, &c->d_tabdf, tabdf)) != TDKS_OK) return fail(st);
  if ((st = upload(c, &c->d_tab, tab)) != TDKS_OK) return fail(st);
  if ((st = upload(c, &c->d_tabf, tabf)) != TDKS_OK) return fail(st);
  std::vector<float> tabbf(tab.size());
  for (size_t k = 0; k < tab.size(); ++k) tabbf[k] = round_bf16(tabf[k]);
  if ((st = upload(c, &c->d_tabbf, tabbf)) != TDKS_OK) return fail(st);
  if ((st = upload(c, &c->d_occ, c->occ)) != TDKS_OK) return fail(st);
  if ((st = upload(c, &c->d_R, c->R)) != TDKS_OK) return fail(st);
  if ((st = upload(c, &c->d_Z, c->Z)) != TDKS_OK) return fail(st);
  const size_t nf = (size_t)(c->n_elem * c->nq3);
  double** fields[] = {&c->d_vks, &c->d_vnuc, &c->d_vhxc1, &c->d_vhxc2, &c->d_vtmp, &c->d_rho, &c->d_vh};
  for (double** f : fields) {
    if ((st = dalloc(c, f, nf)) != TDKS_OK) return fail(st);
    if (cudaMemset(*f, 0, nf * sizeof(double)) != cudaSuccess) return fail(TDKS_ERR_CUDA);
  }
  double** vecs[] = {&c->d_phi, &c->d_b, &c->d_r, &c->d_pv, &c->d_Ap};
  for (double** f : vecs) {
    if ((st = dalloc(c, f, (size_t)c->n_int)) != TDKS_OK) return fail(st);
    if (cudaMemset(*f, 0, c->n_int * sizeof(double)) != cudaSuccess) return fail(TDKS_ERR_CUDA);
  }
  if ((st = dalloc(c, &c->d_cg, 1)) != TDKS_OK) return fail(st);
  const int bpc = hbar_blocks_per_color(c);
  c->part_stride = std::max<int64_t>(2048, 8 * (int64_t)bpc);
  if ((st = dalloc(c, &c->d_part, (size_t)(2 * (c->n_orb + 2) * c->part_stride + 8192))) != TDKS_OK)
    return fail(st);
  if (cudaMallocHost((void**)&c->h_red, 64 * sizeof(double)) != cudaSuccess) return fail(TDKS_ERR_NOMEM);
  if ((st = poisson_setup(c, t)) != TDKS_OK) return fail(st);
  if ((st = launch_nuclear(c)) != TDKS_OK) return fail(st);
  if (cudaMemcpyAsync(c->d_vks, c->d_vnuc, nf * sizeof(double), cudaMemcpyDeviceToDevice,
                      c->stream) != cudaSuccess)
    return fail(TDKS_ERR_CUDA);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(TDKS_ERR_CUDA);
  *out = c;
  return TDKS_OK;
}

tdks_status tdks_destroy(tdks_ctx* c) {
  if (!c) return TDKS_ERR_ARG;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
  return TDKS_OK;
}

tdks_status tdks_set_stream(tdks_ctx* c, void* stream) {
  if (!c) return TDKS_ERR_ARG;
  c->stream = (cudaStream_t)stream;
  return TDKS_OK;
}

tdks_status tdks_sizes(const tdks_ctx* c, int64_t* n_int, int64_t* n_elem, int* nq3) {
  if (!c) return TDKS_ERR_ARG;
  if (n_int) *n_int = c->n_int;
  if (n_elem) *n_elem = c->n_elem;
  if (nq3) *nq3 = (int)c->nq3;
  return TDKS_OK;
}

tdks_status tdks_set_cg(tdks_ctx* c, double tol, int maxit, int precond) {
  if (!c) return TDKS_ERR_ARG;
  if (!(tol > 0) || maxit < 1) return tdks_fail(c, TDKS_ERR_ARG, "cg tol > 0, maxit >= 1");
  if (precond != TDKS_PRECOND_FDM && precond != TDKS_PRECOND_JACOBI)
    return tdks_fail(c, TDKS_ERR_ARG, "unknown preconditioner");
  if (precond == TDKS_PRECOND_FDM && !c->fdm_ok)
    return tdks_fail(c, TDKS_ERR_ARG, "fast diagonalization unavailable for this mesh");
  c->cg_tol = tol;
  c->cg_maxit = maxit;
  c->cg_precond = precond;
  return TDKS_OK;
}

tdks_status tdks_set_potential(tdks_ctx* c, const double* v) {
  if (!c || !v) return TDKS_ERR_ARG;
  TDKS_CU(c, cudaMemcpyAsync(c->d_vks, v, c->n_elem * c->nq3 * sizeof(double),
                             cudaMemcpyDeviceToDevice, c->stream));
  return TDKS_OK;
}

tdks_status tdks_nuclear_potential(tdks_ctx* c, double* v) {
  if (!c || !v) return TDKS_ERR_ARG;
  TDKS_CU(c, cudaMemcpyAsync(v, c->d_vnuc, c->n_elem * c->nq3 * sizeof(double),
                             cudaMemcpyDeviceToDevice, c->stream));
  return TDKS_OK;
}

tdks_status tdks_apply_H(tdks_ctx* c, const double* psi, double* out, int n_orb, int prec) {
  if (!c || !psi || !out) return TDKS_ERR_ARG;
  if (n_orb < 1) return tdks_fail(c, TDKS_ERR_ARG, "n_orb >= 1");
  if (!valid_prec(prec)) return tdks_fail(c, TDKS_ERR_ARG, "precision");
  ApplyArgs a{(const double2*)psi, c->n_int, (double2*)out, c->n_int, n_orb, nullptr, 0, nullptr, 0,
              0, nullptr, 0, nullptr, 0, 0};
  c->n_apply_units += (int64_t)n_orb * c->n_elem;
  return launch_hbar_apply(c, a, prec == TDKS_MIXED ? TDKS_DF64 : prec);
}

tdks_status tdks_nuclear_potential_nodes(tdks_ctx* c, double* v_nodes) {
  if (!c || !v_nodes) return TDKS_ERR_ARG;
  return launch_nuclear_nodes(c, v_nodes);
}

tdks_status tdks_apply_H_gll(tdks_ctx* c, const double* psi, const double* v_nodes, double* out,
                             int n_orb) {
  if (!c || !psi || !v_nodes || !out) return TDKS_ERR_ARG;
  if (n_orb < 1) return tdks_fail(c, TDKS_ERR_ARG, "n_orb >= 1");
  return launch_hbar_gll(c, (const double2*)psi, v_nodes, (double2*)out, n_orb);
}

tdks_status tdks_density(tdks_ctx* c, const double* psi, int n_orb, double* rho) {
  if (!c || !psi || !rho) return TDKS_ERR_ARG;
  TDKS_TRY(check_orb(c, n_orb));
  return launch_density(c, (const double2*)psi, n_orb, rho);
}

tdks_status tdks_dipole(tdks_ctx* c, const double* rho, double d[3]) {
  if (!c || !rho || !d) return TDKS_ERR_ARG;
  return run_dipole(c, rho, d);
}

tdks_status tdks_hartree(tdks_ctx* c, const double* rho, double* vh, int* iters) {
  if (!c || !rho || !vh) return TDKS_ERR_ARG;
  return run_hartree(c, rho, vh, iters);
}

tdks_status tdks_xc(tdks_ctx* c, const double* rho, double* vxc) {
  if (!c || !rho || !vxc) return TDKS_ERR_ARG;
  return launch_xc(c, rho, vxc);
}

tdks_status tdks_expm(tdks_ctx* c, const double* in, double* out, int n_orb, double tau,
                      double tol, int k_max, int prec, int* k_used) {
  if (!c || !in || !out) return TDKS_ERR_ARG;
  TDKS_TRY(check_orb(c, n_orb));
  if (!(tol > 0) || !std::isfinite(tau)) return tdks_fail(c, TDKS_ERR_ARG, "tol > 0, finite tau");
  if (!valid_prec(prec)) return tdks_fail(c, TDKS_ERR_ARG, "precision");
  if (in != out)
    TDKS_CU(c, cudaMemcpyAsync(out, in, (size_t)n_orb * c->n_int * sizeof(double2),
                               cudaMemcpyDeviceToDevice, c->stream));
  // the recurrence starts from `out` so that `in` is never written
  return run_expm(c, (const double2*)out, (double2*)out, n_orb, tau, tol, k_max, prec, k_used,
                  nullptr, nullptr, nullptr);
}

tdks_status tdks_kick(tdks_ctx* c, double* psi, int n_orb, double kappa, const double dir[3]) {
  if (!c || !psi || !dir || n_orb < 1) return TDKS_ERR_ARG;
  return launch_kick(c, (double2*)psi, n_orb, kappa, dir);
}

tdks_status tdks_init_propagation(tdks_ctx* c, const double* psi, int n_orb, double d[3]) {
  if (!c || !psi) return TDKS_ERR_ARG;
  TDKS_TRY(check_orb(c, n_orb));
  const size_t nf = (size_t)(c->n_elem * c->nq3);
  TDKS_CU(c, cudaMemsetAsync(c->d_phi, 0, c->n_int * sizeof(double), c->stream));
  TDKS_TRY(vhxc_of(c, (const double2*)psi, n_orb, c->d_vhxc1, nullptr));
  TDKS_CU(c, cudaMemcpyAsync(c->d_vhxc2, c->d_vhxc1, nf * sizeof(double), cudaMemcpyDeviceToDevice,
                             c->stream));
  c->propagation_ready = true;
  if (d) return run_dipole(c, c->d_rho, d);
  TDKS_CU(c, cudaStreamSynchronize(c->stream));
  return TDKS_OK;
}

tdks_status tdks_magnus_step(tdks_ctx* c, double* psi_d, int n_orb, double dt, const double Eq[3],
                             const double Eh[3], double tol, int k_max, int prec, tdks_stats* stats) {
  if (!c || !psi_d) return TDKS_ERR_ARG;
  return magnus_step_impl(c, (double2*)psi_d, n_orb, dt, Eq, Eh, tol, k_max, prec, stats, nullptr,
                          nullptr, nullptr);
}

tdks_status tdks_propagate_host(tdks_ctx* c, const double* psi_in, double* psi_out, int n_orb,
                                int init, int n_steps, double dt, const double* E, double tol,
                                int k_max, int prec, double* dip) {
  if (!c || !psi_in || !psi_out || n_steps < 0) return TDKS_ERR_ARG;
  TDKS_TRY(check_orb(c, n_orb));
  const size_t vb = (size_t)n_orb * c->n_int * sizeof(double2);
  if (!c->d_psi_e2e) {
    TDKS_TRY(dalloc(c, &c->d_psi_e2e, (size_t)c->n_orb * c->n_int));
  }
  TDKS_CU(c, cudaMemcpyAsync(c->d_psi_e2e, psi_in, vb, cudaMemcpyHostToDevice, c->stream));
  if (init) TDKS_TRY(tdks_init_propagation(c, (const double*)c->d_psi_e2e, n_orb, nullptr));
  const double zero[6] = {0, 0, 0, 0, 0, 0};
  for (int s = 0; s < n_steps; ++s) {
    const double* e = E ? E + 6 * s : zero;
    tdks_stats st;
    TDKS_TRY(tdks_magnus_step(c, (double*)c->d_psi_e2e, n_orb, dt, e, e + 3, tol, k_max, prec, &st));
    if (dip) std::memcpy(dip + 3 * s, st.dipole, 3 * sizeof(double));
  }
  TDKS_CU(c, cudaMemcpyAsync(psi_out, c->d_psi_e2e, vb, cudaMemcpyDeviceToHost, c->stream));
  TDKS_CU(c, cudaStreamSynchronize(c->stream));
  return TDKS_OK;
}

tdks_status tdks_set_lanczos(tdks_ctx* c, int reorth) {
  if (!c || (reorth != 0 && reorth != 1)) return TDKS_ERR_ARG;
  c->lanczos_reorth = reorth;
  return TDKS_OK;
}

tdks_status tdks_set_device_loop(tdks_ctx* c, int on) {
  if (!c || (on != 0 && on != 1)) return TDKS_ERR_ARG;
  c->device_loop = on;
  return TDKS_OK;
}

tdks_status tdks_set_mixed(tdks_ctx* c, double relax) {
  if (!c || !(relax >= 0) || !std::isfinite(relax)) return TDKS_ERR_ARG;
  c->mixed_relax = relax;
  return TDKS_OK;
}

tdks_status tdks_set_f32_stages(tdks_ctx* c, unsigned mask) {
  if (!c || mask >= (1u << 12)) return TDKS_ERR_ARG;
  c->f32_stages = mask;
  return TDKS_OK;
}

tdks_status tdks_set_apply_tile(tdks_ctx* c, int orbs_per_cta) {
  if (!c || orbs_per_cta < 0 || orbs_per_cta > 1024) return TDKS_ERR_ARG;
  c->opc_force = orbs_per_cta;
  return TDKS_OK;
}

tdks_status tdks_set_timing(tdks_ctx* c, int on) {
  if (!c) return TDKS_ERR_ARG;
  c->timing = on != 0;
  return TDKS_OK;
}

tdks_status tdks_get_counters(tdks_ctx* c, tdks_counters* out, int reset) {
  if (!c) return TDKS_ERR_ARG;
  if (out) {
    out->launches = c->n_launch;
    out->apply_launches = c->n_apply_launch;
    out->apply_elem_orb = c->n_apply_units;
    out->apply_ms = c->apply_ms;
    out->cg_iters = c->n_cg;
    out->apply_launches_fp32 = c->n_apply_fp32;
    out->state_reads = c->n_state_reads;
  }
  if (reset) {
    c->n_launch = c->n_apply_launch = c->n_apply_units = c->n_cg = c->n_apply_fp32 = 0;
    c->n_state_reads = 0;
    c->apply_ms = 0.0;
  }
  return TDKS_OK;
}

}  // extern "C"

tdks_status magnus_step_impl(tdks_ctx* c, double2* psi, int n_orb, double dt, const double Eq[3],
                             const double Eh[3], double tol, int k_max, int prec, tdks_stats* stats,
                             double2* keep_half, double* keep_vpred, double* keep_vmid) {
  TDKS_TRY(check_orb(c, n_orb));
  if (!c->propagation_ready) return tdks_fail(c, TDKS_ERR_ARG, "call tdks_init_propagation first");
  if (!(dt > 0) || !(tol > 0)) return tdks_fail(c, TDKS_ERR_ARG, "dt > 0 and tol > 0");
  if (!valid_prec(prec)) return tdks_fail(c, TDKS_ERR_ARG, "precision");
  const size_t vb = (size_t)n_orb * c->n_int * sizeof(double2);
  const size_t fb = (size_t)(c->n_elem * c->nq3) * sizeof(double);
  if (!c->d_psi_half) {
    TDKS_TRY(dalloc(c, &c->d_psi_half, (size_t)c->n_orb * c->n_int));
  }
  tdks_stats st{};
  int kseen = 0, nsub = 0;
  int64_t app = 0;
  // predictor: V(t + dt/4) = V_N + 1.25 V_HXC^{n-1} - 0.25 V_HXC^{n-2} - E(t + dt/4).r
  TDKS_TRY(launch_combine(c, c->d_vks, c->d_vnuc, 1.25, c->d_vhxc1, -0.25, c->d_vhxc2, nullptr, Eq));
  if (keep_vpred) TDKS_CU(c, cudaMemcpyAsync(keep_vpred, c->d_vks, fb, cudaMemcpyDeviceToDevice, c->stream));
  TDKS_CU(c, cudaMemcpyAsync(c->d_psi_half, psi, vb, cudaMemcpyDeviceToDevice, c->stream));
  TDKS_TRY(run_expm(c, c->d_psi_half, c->d_psi_half, n_orb, 0.5 * dt, tol, k_max, prec, nullptr,
                    &kseen, &app, &nsub));
  if (keep_half) TDKS_CU(c, cudaMemcpyAsync(keep_half, c->d_psi_half, vb, cudaMemcpyDeviceToDevice, c->stream));
  st.k_half_max = kseen;
  st.applies += app;
  st.substeps += nsub;
  // corrector: V(t + dt/2) from the density of psi^{n-1/2}
  TDKS_TRY(vhxc_of(c, c->d_psi_half, n_orb, c->d_vtmp, &st.cg_iters[0], prec));
  // d_vtmp now holds V_HXC(t + dt/2) (vhxc_of used d_vtmp as scratch before writing it)
  TDKS_TRY(launch_combine(c, c->d_vks, c->d_vnuc, 1.0, c->d_vtmp, 0.0, nullptr, nullptr, Eh));
  if (keep_vmid) TDKS_CU(c, cudaMemcpyAsync(keep_vmid, c->d_vks, fb, cudaMemcpyDeviceToDevice, c->stream));
  TDKS_TRY(run_expm(c, psi, psi, n_orb, dt, tol, k_max, prec, nullptr, &kseen, &app, &nsub));
  st.k_full_max = kseen;
  st.applies += app;
  st.substeps += nsub;
  // history: V_HXC^{n-2} <- V_HXC^{n-1}, V_HXC^{n-1} <- V_HXC[rho(psi^n)]
  std::swap(c->d_vhxc1, c->d_vhxc2);
  TDKS_TRY(vhxc_of(c, psi, n_orb, c->d_vhxc1, &st.cg_iters[1], prec));
  TDKS_TRY(run_dipole(c, c->d_rho, st.dipole));
  if (stats) *stats = st;
  return TDKS_OK;
}

