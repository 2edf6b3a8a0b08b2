// Nonlocal pseudopotential term in the Kleinman-Bylander form (Eq. 6):
//   V_nl phi = sum_p [int chi_p phi / h_p] chi_p,  chi_p = dV_l u_lm,  h_p = int u_lm dV_l u_lm,
// Galerkin (Eq. 15) and Loewdin (Eq. 21) form
//   Hbar_nl = M^-1/2 P D P^T M^-1/2,  P[j, p] = int chi_p N_j,  D = diag(1 / h_p),
// every integral by the tensor Gauss rule (Sec. VI.A).
//
// Synthetic projectors on every atom (d = r - R): u_lm = exp(-d^2/(2 a^2)) Y_lm(d) with
// Y_00 = 1, Y_1m = d_x, d_y, d_z, and dV_l = c_l exp(-d^2/(2 b^2)).
//
// Set-up: chi_p and u dV u at the Gauss points on the device, h_p by the Gauss rule,
// column p of Pbar = M^-1/2 P by the load-vector kernel.  The columns of one atom are
// kept on the box of interior nodes outside which every entry is below 1e-16 of the
// column's largest (the projectors are Gaussian; the dropped part is far below the
// Lanczos tolerance), dense inside the box.
//
// Apply: C[o][p] = Pbar_p^T psi_o (one block per projector and orbital, fixed-order
// reduction), then a gather over the nodes covered by any box:
//   y_j = sum over the boxes holding j of sum_p Pbar_p[j] C[o][p] / h_p.
// In a Lanczos step alpha_j gains sum_p |C[o][p]|^2 / h_p, and the gather adds y to the
// updated vector w and writes the partials of |w + y|^2 - |w|^2, which the Krylov
// decision adds to the assembly's partials of |w|^2.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tdks_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr double kDropRel = 1e-16;

struct KbGroup {          // one atom: box of interior nodes and its projector columns
  int I0, J0, K0, nI, nJ, nK;
  int n_pg;               // projectors of the atom
  int p0;                 // first projector index
  long long val_off;      // values [n_pg][box] start in the value array
};

struct KbEntry {          // one (group, local box index) that covers a node
  int g;
  int l;
};

__device__ __forceinline__ void gauss_xyz(const Geom& g, const double* eta, int P1, long long idx,
                                          double* x) {
  const int P2 = P1 * P1, P3 = P2 * P1;
  const long long e = idx / P3;
  const int q = (int)(idx - e * P3);
  const int qq[3] = {q % P1, (q / P1) % P1, q / P2};
  const int ii[3] = {(int)(e % g.nx), (int)((e / g.nx) % g.ny), (int)(e / ((long long)g.nx * g.ny))};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double lo = g.brk[d][ii[d]], hi = g.brk[d][ii[d] + 1];
    x[d] = lo + 0.5 * (eta[qq[d]] + 1.0) * (hi - lo);
  }
}

// chi_p and u dV u of projector (l, m) of the atom at R, at every Gauss point
__global__ void k_kb_fields(Geom g, const double* eta, int P1, long long n, double Rx, double Ry,
                            double Rz, int harm, double a, double b, double cl, double* chi,
                            double* udu) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double x[3];
    gauss_xyz(g, eta, P1, i, x);
    const double dx = x[0] - Rx, dy = x[1] - Ry, dz = x[2] - Rz;
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double Y = harm == 0 ? 1.0 : (harm == 1 ? dx : (harm == 2 ? dy : dz));
    const double u = exp(-r2 / (2.0 * a * a)) * Y;
    const double dV = cl * exp(-r2 / (2.0 * b * b));
    chi[i] = dV * u;
    udu[i] = u * dV * u;
  }
}

// per-block partials of sum_q w_q J_e f_q
__global__ void k_kb_wsum(Geom g, const double* w, int P1, long long n, const double* f, double* part) {
  __shared__ double red[kThreads / 32];
  const int P2 = P1 * P1, P3 = P2 * P1;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / P3;
    const int q = (int)(i - e * P3);
    const int ex = (int)(e % g.nx), ey = (int)((e / g.nx) % g.ny), ez = (int)(e / ((long long)g.nx * g.ny));
    const double J = 0.125 * (g.brk[0][ex + 1] - g.brk[0][ex]) * (g.brk[1][ey + 1] - g.brk[1][ey]) *
                     (g.brk[2][ez + 1] - g.brk[2][ez]);
    acc = fma(J * w[q % P1] * w[(q / P1) % P1] * w[q / P2], f[i], acc);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) s += red[k];
    part[blockIdx.x] = s;
  }
}

// v_j *= M^-1/2_jj
__global__ void k_kb_lowdin(Geom g, long long n, double* v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(i % g.nix) + 1;
    const int J = (int)((i / g.nix) % g.niy) + 1;
    const int K = (int)(i / ((long long)g.nix * g.niy)) + 1;
    v[i] *= g.s[0][I] * g.s[1][J] * g.s[2][K];
  }
}

__device__ __forceinline__ long long box_global(const KbGroup& G, int nix, int niy, long long l) {
  const int i = (int)(l % G.nI);
  const int j = (int)((l / G.nI) % G.nJ);
  const int k = (int)(l / ((long long)G.nI * G.nJ));
  return (long long)(G.I0 + i) + (long long)nix * ((G.J0 + j) + (long long)niy * (G.K0 + k));
}

// sc * sum_box Pbar_p[l] x[j(l)] by one block (fixed-order reduction), written by thread 0
__device__ __forceinline__ void kb_project_block(const KbGroup* __restrict__ grp, const int* __restrict__ pg,
                                                 const double* __restrict__ vals, int nix, int niy,
                                                 const double2* x, double sc, int p, double2* dst) {
  __shared__ double red[2][kThreads / 32];
  const KbGroup G = grp[pg[p]];
  const int slot = p - G.p0;
  const long long box = (long long)G.nI * G.nJ * G.nK;
  const double* v = vals + G.val_off + slot * box;
  double re = 0.0, im = 0.0;
  for (long long l = threadIdx.x; l < box; l += blockDim.x) {
    const double2 a = x[box_global(G, nix, niy, l)];
    re = fma(v[l], a.x, re);
    im = fma(v[l], a.y, im);
  }
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, off);
    im += __shfl_down_sync(0xffffffffu, im, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = re;
    red[1][threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) {
      sr += red[0][k];
      si += red[1][k];
    }
    *dst = make_double2(sc * sr, sc * si);
  }
}

// C[o][p] = sc_o sum_box Pbar_p[l] in_o[j(l)]; sc_o = s_kj of the orbital's Lanczos
// state (0 and no work for orbitals out of the recurrence) or 1
__global__ void k_kb_project(const KbGroup* __restrict__ grp, const int* __restrict__ pg,
                             const double* __restrict__ vals, int nix, int niy, const double2* in,
                             int64_t in_stride, const KryOrb* kry, int kj, double2* C, int n_proj) {
  const int p = blockIdx.x, o = blockIdx.y;
  double sc = 1.0;
  if (kry) {
    if (kry[o].status != KRY_ACTIVE) {
      if (threadIdx.x == 0) C[(long long)o * n_proj + p] = make_double2(0.0, 0.0);
      return;
    }
    sc = kry[o].s[kj];
  }
  kb_project_block(grp, pg, vals, nix, niy, in + (long long)o * in_stride, sc, p, &C[(long long)o * n_proj + p]);
}

// alpha_j += sum_p |C[o][p]|^2 / h_p (after the element partials were summed)
__global__ void k_kb_alpha(KryOrb* kry, int kj, const double2* C, const double* invh, int n_proj,
                           int n_orb) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_orb) return;
  if (kry[o].status != KRY_ACTIVE) return;
  double s = 0.0;
  for (int p = 0; p < n_proj; ++p) {
    const double2 c = C[(long long)o * n_proj + p];
    s = fma(invh[p], c.x * c.x + c.y * c.y, s);
  }
  kry[o].alpha[kj] += s;
}

// w_j += y_j = sum_entries sum_slots Pbar C / h over the covered nodes t = t0, t0 + dt, ...;
// returns the sum of |w + y|^2 - |w|^2 over them
__device__ __forceinline__ double kb_add_nodes(const KbGroup* __restrict__ grp, const double* __restrict__ vals,
                                               const long long* __restrict__ tnode, const int* __restrict__ toff,
                                               const KbEntry* __restrict__ tent, long long n_t, const double2* Co,
                                               const double* __restrict__ invh, double2* w, long long t0,
                                               long long dt) {
  double acc = 0.0;
  for (long long t = t0; t < n_t; t += dt) {
    double yr = 0.0, yi = 0.0;
    for (int e = toff[t]; e < toff[t + 1]; ++e) {
      const KbEntry E = tent[e];
      const KbGroup G = grp[E.g];
      const long long box = (long long)G.nI * G.nJ * G.nK;
      for (int s = 0; s < G.n_pg; ++s) {
        const int p = G.p0 + s;
        const double f = vals[G.val_off + s * box + E.l] * invh[p];
        yr = fma(f, Co[p].x, yr);
        yi = fma(f, Co[p].y, yi);
      }
    }
    const long long j = tnode[t];
    double2 v = w[j];
    acc += 2.0 * (v.x * yr + v.y * yi) + yr * yr + yi * yi;
    v.x += yr;
    v.y += yi;
    w[j] = v;
  }
  return acc;
}

// block sum of acc written by thread 0 to *dst
__device__ __forceinline__ void kb_block_sum(double acc, double* dst) {
  __shared__ double red[kThreads / 32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) s += red[k];
    *dst = s;
  }
}

// out_j (+)= y_j over the covered nodes; in a Lanczos step the partials of
// |w + y|^2 - |w|^2 go to part[o][block]
__global__ void k_kb_add(const KbGroup* __restrict__ grp, const double* __restrict__ vals,
                         const long long* __restrict__ tnode, const int* __restrict__ toff,
                         const KbEntry* __restrict__ tent, long long n_t, const double2* C,
                         const double* __restrict__ invh, int n_proj, double2* out,
                         int64_t out_stride, const KryOrb* kry, double* part, int64_t part_stride) {
  const int o = blockIdx.y;
  if (kry && kry[o].status != KRY_ACTIVE) return;
  const double acc = kb_add_nodes(grp, vals, tnode, toff, tent, n_t, C + (long long)o * n_proj, invh,
                                  out + (long long)o * out_stride,
                                  blockIdx.x * (long long)blockDim.x + threadIdx.x,
                                  (long long)gridDim.x * blockDim.x);
  if (part) kb_block_sum(acc, &part[(long long)o * part_stride + blockIdx.x]);
}

}  // namespace

// Device view of one context's projectors for the batched engine.
struct KbView {
  const KbGroup* grp;
  const int* pg;
  const double* vals;
  const double* invh;
  const long long* tnode;
  const int* toff;
  const KbEntry* tent;
  double2* C;             // [n_orb][n_proj]
  long long n_t;
  int n_proj, n_blocks, nix, niy;
};

namespace {

// the orbital's current Krylov vector V_j (j = K.k), as the batched apply reads it:
// the exponential's start vector for j = 0 (input, or output after a sub-step),
// the workspace otherwise
__device__ __forceinline__ const double2* kb_bcur(const BSys& S, const KryOrb& K, int o) {
  if (K.k == 0) return (K.nsub == 0 ? S.in : S.out) + (long long)o * S.n_int;
  return S.Vw + ((long long)o * S.kmax + (K.k - 1)) * S.n_int;
}

__global__ void k_bkb_project(const BSys* __restrict__ sys, const BKbItem* __restrict__ items) {
  const BKbItem it = items[blockIdx.x];
  const BSys& S = sys[it.sys];
  const KbView& V = *S.kb;
  const KryOrb& K = S.kry[it.o];
  double2* dst = &V.C[(long long)it.o * V.n_proj + it.p];
  if (K.status != KRY_ACTIVE) {
    if (threadIdx.x == 0) *dst = make_double2(0.0, 0.0);
    return;
  }
  kb_project_block(V.grp, V.pg, V.vals, V.nix, V.niy, kb_bcur(S, K, it.o), K.s[K.k], it.p, dst);
}

__global__ void k_bkb_alpha(const BSys* __restrict__ sys, const BOrb* __restrict__ orbs, int n) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const BOrb b = orbs[g];
  const BSys& S = sys[b.sys];
  KryOrb& K = S.kry[b.o];
  if (K.status != KRY_ACTIVE) return;
  const KbView& V = *S.kb;
  double s = 0.0;
  for (int p = 0; p < V.n_proj; ++p) {
    const double2 c = V.C[(long long)b.o * V.n_proj + p];
    s = fma(V.invh[p], c.x * c.x + c.y * c.y, s);
  }
  K.alpha[K.k] += s;
}

// one block per (system, orbital, node block): y into the assembly's output V_{j+1}
__global__ void k_bkb_add(const BSys* __restrict__ sys, const BRow* __restrict__ rows) {
  const BRow r = rows[blockIdx.x];
  const BSys& S = sys[r.sys];
  const KryOrb& K = S.kry[r.o];
  if (K.status != KRY_ACTIVE) return;
  const KbView& V = *S.kb;
  double2* w = S.Vw + ((long long)r.o * S.kmax + K.k) * S.n_int;
  const double acc = kb_add_nodes(V.grp, V.vals, V.tnode, V.toff, V.tent, V.n_t, V.C + (long long)r.o * V.n_proj,
                                  V.invh, w, r.rblk * (long long)blockDim.x + threadIdx.x,
                                  (long long)S.kb_nblk * blockDim.x);
  kb_block_sum(acc, &S.kb_part[(long long)r.o * S.kb_nblk + r.rblk]);
}

int grid_for(long long n, int cap) {
  long long b = (n + kThreads - 1) / kThreads;
  return (int)std::max<long long>(1, std::min<long long>(b, cap));
}

}  // namespace

struct KbState {
  int n_proj = 0, n_grp = 0, n_blocks = 0;
  long long n_t = 0, n_vals = 0;
  KbGroup* d_grp = nullptr;
  int* d_pg = nullptr;
  double* d_vals = nullptr;
  double* d_invh = nullptr;
  long long* d_tnode = nullptr;
  int* d_toff = nullptr;
  KbEntry* d_tent = nullptr;
  double2* d_C = nullptr;
  double* d_part = nullptr;     // [n_orb][n_blocks] partials of the Lanczos correction
  KbView* d_view = nullptr;     // device view for the batched engine (made on first use)
  std::vector<double> h;
};

void kb_free(tdks_ctx* c) {
  if (!c || !c->kb) return;
  KbState* k = static_cast<KbState*>(c->kb);
  void* ptrs[] = {k->d_grp, k->d_pg, k->d_vals, k->d_invh, k->d_tnode, k->d_toff, k->d_tent, k->d_C, k->d_part,
                  k->d_view};
  for (void* p : ptrs) cudaFree(p);
  delete k;
  c->kb = nullptr;
}

int kb_norm_blocks(const tdks_ctx* c) {
  const KbState* k = static_cast<const KbState*>(c->kb);
  return (k && k->n_t > 0) ? k->n_blocks : 0;   // kb_add writes the partials only when it runs
}
const double* kb_norm_parts(const tdks_ctx* c) {
  return c->kb ? static_cast<const KbState*>(c->kb)->d_part : nullptr;
}

const KbView* kb_view(tdks_ctx* c, double** part, int* n_blocks, int* n_proj) {
  KbState* k = c ? static_cast<KbState*>(c->kb) : nullptr;
  if (!k) return nullptr;
  if (!k->d_view) {
    const KbView v{k->d_grp, k->d_pg, k->d_vals, k->d_invh, k->d_tnode, k->d_toff, k->d_tent, k->d_C,
                   k->n_t, k->n_proj, k->n_blocks, c->Ni[0], c->Ni[1]};
    if (cudaMalloc((void**)&k->d_view, sizeof(KbView)) != cudaSuccess ||
        cudaMemcpy(k->d_view, &v, sizeof(v), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(k->d_view);
      k->d_view = nullptr;
      return nullptr;
    }
  }
  if (part) *part = k->d_part;
  if (n_blocks) *n_blocks = k->n_t > 0 ? k->n_blocks : 0;
  if (n_proj) *n_proj = k->n_proj;
  return k->d_view;
}

cudaError_t launch_bkb_project(const BSys* sys, const BKbItem* items, int n_items, cudaStream_t st) {
  if (n_items < 1) return cudaSuccess;
  k_bkb_project<<<n_items, kThreads, 0, st>>>(sys, items);
  return cudaGetLastError();
}

cudaError_t launch_bkb_alpha(const BSys* sys, const BOrb* orbs, int n_orbs, cudaStream_t st) {
  if (n_orbs < 1) return cudaSuccess;
  k_bkb_alpha<<<(n_orbs + 63) / 64, 64, 0, st>>>(sys, orbs, n_orbs);
  return cudaGetLastError();
}

cudaError_t launch_bkb_add(const BSys* sys, const BRow* rows, int n_rows, cudaStream_t st) {
  if (n_rows < 1) return cudaSuccess;
  k_bkb_add<<<n_rows, kThreads, 0, st>>>(sys, rows);
  return cudaGetLastError();
}

tdks_status kb_project(tdks_ctx* c, const ApplyArgs& a) {
  KbState* k = static_cast<KbState*>(c->kb);
  if (!k) return TDKS_OK;
  k_kb_project<<<dim3(k->n_proj, a.n_orb), kThreads, 0, c->stream>>>(
      k->d_grp, k->d_pg, k->d_vals, c->Ni[0], c->Ni[1], a.in_base, a.in_stride, a.kry, a.kj, k->d_C,
      k->n_proj);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

tdks_status kb_alpha(tdks_ctx* c, const ApplyArgs& a) {
  KbState* k = static_cast<KbState*>(c->kb);
  if (!k || !a.kry) return TDKS_OK;
  k_kb_alpha<<<(a.n_orb + 63) / 64, 64, 0, c->stream>>>(a.kry, a.kj, k->d_C, k->d_invh, k->n_proj, a.n_orb);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

tdks_status kb_add(tdks_ctx* c, const ApplyArgs& a) {
  KbState* k = static_cast<KbState*>(c->kb);
  if (!k || k->n_t == 0) return TDKS_OK;
  const bool lz = a.lanczos && a.kry;
  k_kb_add<<<dim3(k->n_blocks, a.n_orb), kThreads, 0, c->stream>>>(
      k->d_grp, k->d_vals, k->d_tnode, k->d_toff, k->d_tent, k->n_t, k->d_C, k->d_invh, k->n_proj,
      a.out_base, a.out_stride, a.kry, lz ? k->d_part : nullptr, k->n_blocks);
  c->n_launch += 1;
  TDKS_CU(c, cudaGetLastError());
  return TDKS_OK;
}

extern "C" tdks_status tdks_set_kb(tdks_ctx* c, int n_atoms, const double* R, double a, double b,
                                   const double cl[2], int lmax) {
  if (!c) return TDKS_ERR_ARG;
  kb_free(c);
  if (n_atoms == 0) return TDKS_OK;
  if (n_atoms < 0 || !R || !cl || lmax < 0 || lmax > 1 || !(a > 0) || !(b > 0))
    return tdks_fail(c, TDKS_ERR_ARG, "tdks_set_kb: n_atoms >= 0, R, c, lmax in {0, 1}, a, b > 0");
  const int npa = lmax == 0 ? 1 : 4;
  const int n_proj = n_atoms * npa;
  const long long nq = c->n_elem * c->nq3, n = c->n_int;
  const int nix = c->Ni[0], niy = c->Ni[1], niz = c->Ni[2];
  double *chi = nullptr, *udu = nullptr, *col = nullptr, *part = nullptr;
  auto cleanup = [&]() {
    cudaFree(chi);
    cudaFree(udu);
    cudaFree(col);
    cudaFree(part);
  };
  const int nbq = grid_for(nq, 1024);
  if (cudaMalloc(&chi, nq * sizeof(double)) != cudaSuccess || cudaMalloc(&udu, nq * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&col, n * sizeof(double)) != cudaSuccess || cudaMalloc(&part, nbq * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return tdks_fail(c, TDKS_ERR_NOMEM, "projector set-up");
  }
  const Geom g = tdks_geom(c);
  const double* eta = c->d_tab + tab_off_eta(c->P1);
  const double* w = c->d_tab + tab_off_w(c->P1);
  std::vector<double> hcol(n), hpart(nbq), h(n_proj);
  std::vector<std::vector<double>> cols(n_proj);
  for (int I = 0; I < n_atoms; ++I) {
    for (int m = 0; m < npa; ++m) {
      const int p = I * npa + m;
      const int l = m == 0 ? 0 : 1;
      k_kb_fields<<<nbq, kThreads, 0, c->stream>>>(g, eta, c->P1, nq, R[3 * I], R[3 * I + 1], R[3 * I + 2], m,
                                                   a, b, cl[l], chi, udu);
      k_kb_wsum<<<nbq, kThreads, 0, c->stream>>>(g, w, c->P1, nq, udu, part);
      cudaMemsetAsync(col, 0, n * sizeof(double), c->stream);
      tdks_status st = launch_load_vector(c, chi, col, 1.0, 1);
      if (st != TDKS_OK) {
        cleanup();
        return st;
      }
      k_kb_lowdin<<<grid_for(n, 1024), kThreads, 0, c->stream>>>(g, n, col);
      if (cudaMemcpyAsync(hpart.data(), part, nbq * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
          cudaMemcpyAsync(hcol.data(), col, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return tdks_fail(c, TDKS_ERR_CUDA, "projector set-up");
      }
      double hs = 0.0;
      for (int k = 0; k < nbq; ++k) hs += hpart[k];
      if (!(std::fabs(hs) > 0) || !std::isfinite(hs)) {
        cleanup();
        return tdks_fail(c, TDKS_ERR_ARG, "a projector has a zero or non-finite denominator");
      }
      h[p] = hs;
      cols[p] = hcol;
    }
  }
  cleanup();
  // boxes: per atom, the interior-index box outside which every entry of its columns
  // is below kDropRel of that column's largest magnitude
  std::vector<KbGroup> grp(n_atoms);
  std::vector<int> pg(n_proj);
  std::vector<double> vals;
  for (int I = 0; I < n_atoms; ++I) {
    int lo[3] = {nix, niy, niz}, hi[3] = {-1, -1, -1};
    for (int m = 0; m < npa; ++m) {
      const std::vector<double>& v = cols[I * npa + m];
      double mx = 0.0;
      for (double x : v) mx = std::max(mx, std::fabs(x));
      const double thr = kDropRel * mx;
      for (long long j = 0; j < n; ++j) {
        if (!(std::fabs(v[j]) > thr)) continue;
        const int ii = (int)(j % nix), jj = (int)((j / nix) % niy), kk = (int)(j / ((long long)nix * niy));
        lo[0] = std::min(lo[0], ii);
        lo[1] = std::min(lo[1], jj);
        lo[2] = std::min(lo[2], kk);
        hi[0] = std::max(hi[0], ii);
        hi[1] = std::max(hi[1], jj);
        hi[2] = std::max(hi[2], kk);
      }
    }
    if (hi[0] < 0) {   // projector entirely negligible on this mesh: empty box
      lo[0] = lo[1] = lo[2] = 0;
      hi[0] = hi[1] = hi[2] = -1;
    }
    KbGroup G;
    G.I0 = lo[0];
    G.J0 = lo[1];
    G.K0 = lo[2];
    G.nI = hi[0] - lo[0] + 1;
    G.nJ = hi[1] - lo[1] + 1;
    G.nK = hi[2] - lo[2] + 1;
    G.n_pg = npa;
    G.p0 = I * npa;
    G.val_off = (long long)vals.size();
    const long long box = (long long)G.nI * G.nJ * G.nK;
    for (int m = 0; m < npa; ++m) {
      pg[I * npa + m] = I;
      const std::vector<double>& v = cols[I * npa + m];
      for (long long l = 0; l < box; ++l) {
        const int i = (int)(l % G.nI), jj = (int)((l / G.nI) % G.nJ), kk = (int)(l / ((long long)G.nI * G.nJ));
        vals.push_back(v[(G.I0 + i) + (long long)nix * ((G.J0 + jj) + (long long)niy * (G.K0 + kk))]);
      }
    }
    grp[I] = G;
  }
  // covered nodes (ascending) and the (atom, local index) entries of each
  std::vector<int> cnt(n, 0);
  for (const KbGroup& G : grp)
    for (int kk = 0; kk < G.nK; ++kk)
      for (int jj = 0; jj < G.nJ; ++jj)
        for (int i = 0; i < G.nI; ++i)
          ++cnt[(G.I0 + i) + (long long)nix * ((G.J0 + jj) + (long long)niy * (G.K0 + kk))];
  std::vector<long long> tnode;
  std::vector<int> toff(1, 0);
  std::vector<long long> slot_of(n, -1);
  for (long long j = 0; j < n; ++j)
    if (cnt[j]) {
      slot_of[j] = (long long)tnode.size();
      tnode.push_back(j);
      toff.push_back(toff.back() + cnt[j]);
    }
  std::vector<KbEntry> tent(toff.back());
  std::vector<int> fill(tnode.size(), 0);
  for (int gi = 0; gi < n_atoms; ++gi) {   // entries of a node in atom order
    const KbGroup& G = grp[gi];
    for (int kk = 0; kk < G.nK; ++kk)
      for (int jj = 0; jj < G.nJ; ++jj)
        for (int i = 0; i < G.nI; ++i) {
          const long long j = (G.I0 + i) + (long long)nix * ((G.J0 + jj) + (long long)niy * (G.K0 + kk));
          const long long t = slot_of[j];
          tent[toff[t] + fill[t]++] = KbEntry{gi, i + G.nI * (jj + G.nJ * kk)};
        }
  }
  KbState* k = new KbState();
  k->n_proj = n_proj;
  k->n_grp = n_atoms;
  k->n_t = (long long)tnode.size();
  k->n_vals = (long long)vals.size();
  k->n_blocks = grid_for(std::max<long long>(k->n_t, 1), 512);
  k->h = h;
  std::vector<double> invh(n_proj);
  for (int p = 0; p < n_proj; ++p) invh[p] = 1.0 / h[p];
  c->kb = k;
  auto up = [&](auto** dst, const auto& src) -> bool {
    const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(src[0]);
    if (cudaMalloc((void**)dst, bytes) != cudaSuccess) return false;
    return src.empty() || cudaMemcpy(*dst, src.data(), src.size() * sizeof(src[0]), cudaMemcpyHostToDevice) == cudaSuccess;
  };
  if (!up(&k->d_grp, grp) || !up(&k->d_pg, pg) || !up(&k->d_vals, vals) || !up(&k->d_invh, invh) ||
      !up(&k->d_tnode, tnode) || !up(&k->d_toff, toff) || !up(&k->d_tent, tent) ||
      cudaMalloc(&k->d_C, (size_t)c->n_orb * n_proj * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&k->d_part, (size_t)c->n_orb * k->n_blocks * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    kb_free(c);
    return tdks_fail(c, TDKS_ERR_NOMEM, "projector storage");
  }
  return TDKS_OK;
}

extern "C" tdks_status tdks_kb_info(const tdks_ctx* c, int* n_proj, double* h_host, int64_t* n_covered,
                                    int64_t* n_values) {
  if (!c) return TDKS_ERR_ARG;
  const KbState* k = static_cast<const KbState*>(c->kb);
  if (n_proj) *n_proj = k ? k->n_proj : 0;
  if (h_host && k) std::memcpy(h_host, k->h.data(), k->h.size() * sizeof(double));
  if (n_covered) *n_covered = k ? k->n_t : 0;
  if (n_values) *n_values = k ? k->n_vals : 0;
  return TDKS_OK;
}
