// Internal declarations of the TDKS library (context, tables, launch helpers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tdks.h"

#define TDKS_KMAX 128          // hard cap on the Krylov dimension per sub-step
#define TDKS_MAX_P1 9          // p <= 8
#define TDKS_MAX_SUBSTEPS 1000

// Per-orbital Lanczos state, resident in device memory.
constexpr int kChebCache = 511;   // largest cached Chebyshev expansion order

struct KryOrb {
  double nrm;                  // ||psi|| at the start of the current sub-step
  double t_rem;                // time still to propagate
  double tau_sub;              // time covered by the current sub-step's result
  int k;                       // Krylov vectors built in the current sub-step
  int status;                  // KRY_* below
  int k_total;                 // sum of Krylov dimensions over sub-steps
  int nsub;                    // sub-steps taken
  int applies;                 // Hbar applications on this orbital
  int pad;
  double err;                  // last a-posteriori estimate of Eq. 38 (INFINITY before the first)
  int f32;                     // batched TDKS_MIXED: the next product of this orbital in FP32
  int pad2;
  double alpha[TDKS_KMAX];
  double beta[TDKS_KMAX];
  double s[TDKS_KMAX + 1];     // basis vector j is q_j = s[j] * V_j
  double yre[TDKS_KMAX];
  double yim[TDKS_KMAX];
  // small-exponential cache of the current exponential: the Chebyshev interval
  // [clo, chi] and time ctau of the last expansion and its (normalized, doubled) Bessel
  // coefficients cJ[0..cN]; valid for any later T whose Gershgorin interval lies inside
  // [clo, chi] (cv = 0: empty)
  double clo, chi, ctau;
  int cN, cv;
  double cJ[kChebCache + 1];
};

enum { KRY_ACTIVE = 0, KRY_CONVERGED = 1, KRY_SUBSTEP = 2, KRY_DONE = 3, KRY_FAILED = -1 };

// CG state, resident in device memory.
struct CgState {
  double bb;        // ||b||^2
  double rz;        // r.z of the current iterate
  double rr;        // ||r||^2
  double alpha;     // CG step length; carries beta between the last two kernels
  int iters;
  int done;         // 1 when converged
  int failed;
  int first;        // 1 until the first search direction is set
};

// Geometry passed by value to the element kernels.
struct Geom {
  int nx, ny, nz, p;
  int nix, niy, niz;           // interior nodes per axis
  const double* brk[3];        // breakpoints per axis (n+1)
  const double* s[3];          // 1-D factors of M^-1/2 per full node index
  const float* sf[3];          // the same factors rounded to float
  const double* gauss;         // Gauss points on [-1, 1] (P1)
  const double* ih[3];         // 1 / element width per element, per axis (n)
  const double* wq;            // Gauss weights on [-1, 1] (P1)
};

struct tdks_ctx {
  // mesh
  int nx = 0, ny = 0, nz = 0, p = 0, P1 = 0, nq = 0;
  int Nn[3] = {0, 0, 0}, Ni[3] = {0, 0, 0};
  int64_t n_int = 0, n_elem = 0, nq3 = 0;
  std::vector<double> brk[3];
  cudaStream_t stream = nullptr;
  int device = 0;
  // system
  int n_orb = 0;
  std::vector<double> occ, R, Z;
  int n_nuc = 0, nuc_kind = 0, hartree = 1, xc = 1;
  double nuc_param = 0.0;
  // device mesh data
  double* d_brk[3] = {nullptr, nullptr, nullptr};
  double* d_s[3] = {nullptr, nullptr, nullptr};          // M^-1/2 1-D factors
  float* d_sf[3] = {nullptr, nullptr, nullptr};          // float copies
  double* d_coord[3] = {nullptr, nullptr, nullptr};      // node coordinates
  double* d_kd[3] = {nullptr, nullptr, nullptr};         // sum K1_aa / h  (Jacobi diagonal)
  double* d_md[3] = {nullptr, nullptr, nullptr};         // sum h Mg_aa
  double* d_ih[3] = {nullptr, nullptr, nullptr};         // 1 / element width per element
  double* d_tab = nullptr;     // double tables (layout in tables.cpp)
  float* d_tabf = nullptr;     // float copy
  float* d_tabdf = nullptr;    // double-float copy (hi, lo pairs)
  float* d_tabbf = nullptr;    // float copy rounded to bfloat16 (BF16-operand mode)
  double* d_occ = nullptr;
  double* d_R = nullptr;
  double* d_Z = nullptr;
  // fields at the Gauss points
  double *d_vks = nullptr, *d_vnuc = nullptr, *d_vhxc1 = nullptr, *d_vhxc2 = nullptr;
  double *d_vtmp = nullptr, *d_rho = nullptr, *d_vh = nullptr;
  // Poisson
  double *d_phi = nullptr, *d_b = nullptr, *d_r = nullptr, *d_pv = nullptr, *d_Ap = nullptr;
  CgState* d_cg = nullptr;
  double cg_tol = 1e-12;
  int cg_maxit = 5000;
  int cg_precond = 0;          // 0: fast diagonalization (exact for these meshes), 1: Jacobi
  bool fdm_ok = false;
  double* d_fdmS[3] = {nullptr, nullptr, nullptr};    // per-axis eigenvectors [i][mode]
  double* d_fdmL[3] = {nullptr, nullptr, nullptr};    // per-axis eigenvalues
  double *d_z = nullptr, *d_t1 = nullptr, *d_t2 = nullptr, *d_invdiag = nullptr;
  // Krylov
  double2* d_Vw[2] = {nullptr, nullptr};      // Krylov bases [n_orb][kmax][n_int]
  int Vw_orb[2] = {0, 0}, Vw_kmax[2] = {0, 0};
  KryOrb* d_kryw[2] = {nullptr, nullptr};     // per-orbital Lanczos state of each basis
  double2* d_psi_half = nullptr;
  void* d_evec = nullptr;      // element-local Hbar results [n_orb][n_elem][P1^3] (complex)
  size_t evec_bytes = 0;
  double2* d_psi_e2e = nullptr;
  // reductions
  double* d_part = nullptr;    // partial sums
  int64_t part_stride = 0;     // per orbital
  double* h_red = nullptr;     // pinned small host buffer
  int* h_int = nullptr;
  bool propagation_ready = false;
  void* adj = nullptr;          // objective / adjoint state (adjoint.cu)
  void* kb = nullptr;           // nonlocal Kleinman-Bylander projectors (kb.cu)
  int lanczos_reorth = 0;       // 1: CGS2 re-orthogonalization of every new Lanczos vector
  int opc_force = 0;            // orbitals per CTA of the Hbar element kernel (0: chosen per launch)
  int device_loop = 1;          // Lanczos iterations of a sub-step as one CUDA graph (krylov.cu)
  void* kgraph = nullptr;       // its cached graphs
  double mixed_relax = 1e8;     // TDKS_MIXED: FP32 contractions once every estimate <= relax * tol
  unsigned f32_stages = 0;      // per-stage precision study of the double-float apply (diagnostics)
  double2* d_ro_part = nullptr; // its partial dots [n_orb][TDKS_KMAX][chunks]
  double2* d_ro_h = nullptr;    // its projections [n_orb][TDKS_KMAX]
  // counters
  int64_t n_launch = 0, n_apply_launch = 0, n_apply_units = 0, n_cg = 0, n_apply_fp32 = 0;
  int64_t n_state_reads = 0;
  double apply_ms = 0.0;
  bool timing = false;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::string err;
};

// ---------------------------------------------------------------- helpers
tdks_status tdks_fail(tdks_ctx* c, tdks_status s, const std::string& msg);
tdks_status tdks_cuda_check(tdks_ctx* c, cudaError_t e, const char* what);
#define TDKS_CU(ctx, call)                                              \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return tdks_cuda_check((ctx), e_, #call);    \
  } while (0)
#define TDKS_TRY(call)                     \
  do {                                     \
    tdks_status s_ = (call);               \
    if (s_ != TDKS_OK) return s_;          \
  } while (0)

Geom tdks_geom(const tdks_ctx* c);

// tables.cpp: host construction of the 1-D tables (long double)
struct Tables1D {
  std::vector<double> xi, w;       // GLL nodes and weights (P1)
  std::vector<double> eta, omega;  // Gauss points and weights (nq)
  std::vector<double> B, D;        // [nq][P1] Lagrange values / derivatives at Gauss points
  std::vector<double> Kq;          // [nq][nq] Dg^T diag(omega) Dg on Gauss-point Lagrange basis
  std::vector<double> K1, Mg;      // [P1][P1] D^T W D and B^T W B
};
Tables1D tdks_build_tables(int p, int nq);
// fdm.cpp: generalized eigenpairs (1-D stiffness, 1-D Gauss mass) of one axis
void tdks_fdm_axis(const Tables1D& t, int p, const double* br, int n_el, std::vector<double>& S,
                   std::vector<double>& lam);

#ifdef __CUDACC__
#define TDKS_HD __host__ __device__
#else
#define TDKS_HD
#endif

// Device table layout (both double and float copies), offsets in elements.
//   B [P1*P1] | Kq [P1*P1] | w [P1] | K1 [P1*P1] | Mg [P1*P1] | eta [P1]
//   | csB | csBT | csKq      (even-odd folded forms, see cs_apply in elements.cuh)
// A centrosymmetric n x n matrix M (M[n-1-i][n-1-j] = M[i][j]) is stored folded as
// Me[h][h] = (M[q][i] + M[q][n-1-i])/2, Mo[h][h] = (M[q][i] - M[q][n-1-i])/2 for
// q, i < h = n/2, then (odd n) the middle column M[q][h], the middle row M[h][i]
// and M[h][h].  B, B^T and Kq are centrosymmetric because the GLL nodes and the
// Gauss points are symmetric about 0.
TDKS_HD inline int cs_size(int P1) { return 2 * (P1 / 2) * (P1 / 2) + 2 * (P1 / 2) + 1; }
TDKS_HD inline int tab_off_B(int) { return 0; }
TDKS_HD inline int tab_off_Kq(int P1) { return P1 * P1; }
TDKS_HD inline int tab_off_w(int P1) { return 2 * P1 * P1; }
TDKS_HD inline int tab_off_K1(int P1) { return 2 * P1 * P1 + P1; }
TDKS_HD inline int tab_off_Mg(int P1) { return 3 * P1 * P1 + P1; }
TDKS_HD inline int tab_off_eta(int P1) { return 4 * P1 * P1 + P1; }
TDKS_HD inline int tab_off_csB(int P1) { return 4 * P1 * P1 + 2 * P1; }
TDKS_HD inline int tab_off_csBT(int P1) { return tab_off_csB(P1) + cs_size(P1); }
TDKS_HD inline int tab_off_csK(int P1) { return tab_off_csBT(P1) + cs_size(P1); }
TDKS_HD inline int tab_off_wl(int P1) { return tab_off_csK(P1) + cs_size(P1); }   // GLL weights
TDKS_HD inline int tab_off_csK1(int P1) { return tab_off_wl(P1) + P1; }            // folded K1
TDKS_HD inline int tab_size(int P1) { return tab_off_csK1(P1) + cs_size(P1); }

// ---------------------------------------------------------------- launchers
// element kernels (elements.cu)
struct ApplyArgs {
  const double2* in_base;     // q_j = s[kj] * V_j (V_j when kry is null)
  int64_t in_stride;
  double2* out_base;          // Hbar q_j, or the Lanczos residual when `lanczos`
  int64_t out_stride;
  int n_orb;
  KryOrb* kry;                // optional: scale s[kj], skip non-active orbitals
  int kj;
  double* part;               // optional: per-block partials of Re(u^H H u) per orbital
  int64_t part_stride;
  // fused Lanczos update: out = Hbar q_j - alpha_j s_j V_j - beta_{j-1} s_{j-1} V_{j-1}
  int lanczos;
  const double2* vm_base;     // V_{j-1} (null when kj == 0)
  int64_t vm_stride;
  double* npart;              // per-block partials of ||out||^2 per orbital
  int64_t npart_stride;
  int accumulate;             // out += result instead of out = result (plain apply only)
};
tdks_status launch_hbar_apply(tdks_ctx* c, const ApplyArgs& a, int prec);
tdks_status launch_stiffness(tdks_ctx* c, const double* in, double* out, double* part,
                             const CgState* cg);
tdks_status launch_load_vector(tdks_ctx* c, const double* f_q, double* out, double scale,
                               int weighted = 1);
tdks_status launch_interp(tdks_ctx* c, const double* nodal, double* f_q, double scale = 1.0,
                          int weighted = 0);
// adjoint kernels (elements.cu)
// lam_a (+)= 2 occ_a M^-1/2 (B^T)^(x)3 (g_rho psi_a(x_q))
tdks_status launch_density_adjoint(tdks_ctx* c, const double2* psi, int n_orb, const double* g_rho,
                                   double2* lam, int accumulate);
// g_q += coef wJ_q sum_a Im(conj(mu_a(x_q)) phi_a(x_q))
tdks_status launch_cross(tdks_ctx* c, const double2* mu, const double2* phi, int n_orb, double coef,
                         double* g_q);
// prec TDKS_DF64: interpolation in double-float, |psi|^2 summed over orbitals in FP64;
// any other value: FP64 throughout
tdks_status launch_density(tdks_ctx* c, const double2* psi, int n_orb, double* rho_q,
                           int prec = TDKS_FP64);
int hbar_blocks_per_color(const tdks_ctx* c);
int assemble_blocks(const tdks_ctx* c, int n_orb);   // partial-sum count of the fused update
int stiff_blocks_per_color(const tdks_ctx* c);

// magnus step with optional recording of the intermediates (capi.cu)
tdks_status magnus_step_impl(tdks_ctx* c, double2* psi, int n_orb, double dt, const double Eq[3],
                             const double Eh[3], double tol, int k_max, int prec, tdks_stats* st,
                             double2* keep_half, double* keep_vpred, double* keep_vmid);
void adjoint_free(tdks_ctx* c);
void tdks_sym_eigen(std::vector<double>& C, int n, std::vector<double>& V, std::vector<double>& lam);

// fields.cu
tdks_status launch_fxc_add(tdks_ctx* c, const double* rho, const double* g_h, double* g_rho);
tdks_status launch_dipole_sens(tdks_ctx* c, double coef, const double e[3], double* g_rho);
tdks_status launch_nuclear(tdks_ctx* c);
tdks_status launch_nuclear_nodes(tdks_ctx* c, double* v);   // V_N at the interior nodes
tdks_status launch_xc(tdks_ctx* c, const double* rho, double* vxc);
tdks_status run_dipole(tdks_ctx* c, const double* rho, double d[3], int weighted = 1);
tdks_status launch_kick(tdks_ctx* c, double2* psi, int n_orb, double kappa, const double dir[3]);
// v_out = vn + a1*h1 + a2*h2 + h3 - E.x_q   (h2/h3 may be null)
tdks_status launch_combine(tdks_ctx* c, double* v_out, const double* vn, double a1,
                           const double* h1, double a2, const double* h2,
                           const double* h3, const double E[3]);

// poisson.cu
// df: the fast-diagonalization preconditioner in double-float (the CG stays FP64)
tdks_status run_hartree(tdks_ctx* c, const double* rho_q, double* vh_q, int* iters, bool df = false);
tdks_status run_cg_solve(tdks_ctx* c, const double* b, double* x, int* iters, bool df = false);
tdks_status poisson_setup(tdks_ctx* c, const Tables1D& t);

// krylov.cu
tdks_status run_expm(tdks_ctx* c, const double2* in, double2* out, int n_orb, double tau,
                     double tol, int kmax, int prec, int* k_used, int* kmax_seen,
                     int64_t* applies, int* nsub);
tdks_status run_expm_ws(tdks_ctx* c, int w, const double2* in, double2* out, int n_orb, double tau,
                        double tol, int kmax, int prec, int* k_used, int* kmax_seen,
                        int64_t* applies, int* nsub);

// TDKS_FP64 .. TDKS_MIXED (capi.cu)
bool valid_prec(int prec);

// krylov.cu: cached graphs of the device-driven Lanczos loop
void kgraph_free(tdks_ctx* c);
// elements.cu: the element-result buffer sized for n_orb orbitals of any contraction type
tdks_status ensure_evec(tdks_ctx* c, int n_orb);

// reduction helper used by several files
tdks_status ensure_part(tdks_ctx* c, int n_orb, int64_t per_orb);

// ---------------------------------------------------------------------------
// Batched engine: many independent systems advanced by the same launches.
// Every orbital keeps its own Lanczos state (KryOrb); its current Krylov index is
// K.k, so systems and orbitals progress independently inside one device loop.
// ---------------------------------------------------------------------------
enum { KRY_RESTART = 4 };      // ||v|| needed before the recurrence (re)starts

struct KbView;                 // device view of a context's nonlocal projectors (kb.cu)

struct BSys {
  Geom g;
  int P1, n_orb, kmax;
  int n_eblk;                  // element blocks of the apply (alpha partials per orbital)
  int n_rblk;                  // row blocks of assembly / norms / recombination
  int mixed;                   // TDKS_MIXED batch: each orbital's product type follows KryOrb::f32
  long long n_int, n_elem;
  const double2* in;           // exponential input [n_orb][n_int]
  double2* out;                // output [n_orb][n_int] (may equal in)
  const double* vks;           // V_KS at the Gauss points
  double2* Vw;                 // Krylov vectors V_1 .. V_kmax [n_orb][kmax][n_int]
  KryOrb* kry;                 // [n_orb]
  void* ev;                    // element results [n_orb][n_elem][P1^3] (contraction type)
  double* apart;               // alpha partials [n_orb][n_eblk]
  double* npart;               // norm partials [n_orb][n_rblk]
  double dt;
  const KbView* kb;            // nonlocal projectors of the system, or nullptr
  double* kb_part;             // partials of |w + y|^2 - |w|^2 of the nonlocal term [n_orb][kb_nblk]
  int kb_nblk;                 // 0 without projectors
  int pad1;
};
static_assert(sizeof(BSys) % 8 == 0, "BSys is copied as 64-bit words");
struct BItem { int sys, eblk, o0, o1; };   // apply: E elements of block eblk, orbitals [o0, o1)
struct BRow { int sys, o, rblk, pad; };    // one row block of one orbital
struct BOrb { int sys, o; };               // one orbital of one system
struct BKbItem { int sys, o, p, pad; };    // nonlocal projection: projector p of orbital o

// elements.cu
size_t hbar_batch_smem(int P1, int prec, int E);
cudaError_t hbar_batch_occupancy(int P1, int prec, int E, int* blocks_per_sm);
// qctr: the launch's work ticket counter, zero at launch
cudaError_t launch_hbar_batch(int P1, int prec, const BSys* sys, const BItem* items, int n_items,
                              int E, int grid, const void* tab, int* qctr, cudaStream_t st);
cudaError_t launch_balpha(const BSys* sys, const BOrb* orbs, int n_orbs, cudaStream_t st);
// rows: (system, orbital, row block) items of systems of degree P1 - 1 only
cudaError_t launch_bassemble(int P1, int prec, const BSys* sys, const BRow* rows, int n_rows,
                             cudaStream_t st);
// krylov.cu
cudaError_t launch_bkry_init(const BSys* sys, const BOrb* orbs, int n_orbs, double factor,
                             cudaStream_t st);
cudaError_t launch_bkry_prepare(const BSys* sys, const BOrb* orbs, int n_orbs, const BRow* rows,
                                int n_rows, cudaStream_t st);
// theta >= 0 (TDKS_MIXED): an orbital whose estimate is <= theta takes FP32 products next
cudaError_t launch_bkry_exp(const BSys* sys, const BOrb* orbs, int n_orbs, double tol, double theta,
                            cudaStream_t st);
cudaError_t launch_bkry_finish(const BSys* sys, const BOrb* orbs, int n_orbs, const BRow* rows,
                               int n_rows, int prec, cudaStream_t st);
// the loop kernels also zero the n_q work ticket counters qctr for the next pass
cudaError_t launch_bloop_begin(cudaGraphConditionalHandle h, int* iter, int* qctr, int n_q,
                               cudaStream_t st);
cudaError_t launch_bloop_control(cudaGraphConditionalHandle h, const BSys* sys, const BOrb* orbs,
                                 int n_orbs, int* iter, int cap, int* err, int* qctr, int n_q,
                                 cudaStream_t st);
// kb.cu, batched nonlocal term: the device view of c's projectors (nullptr without
// them; owned by the context), its partial buffer [n_orb][*n_blocks] and projector count
const KbView* kb_view(tdks_ctx* c, double** part, int* n_blocks, int* n_proj);
// C of every item's (orbital, projector) from the orbital's current Krylov vector
cudaError_t launch_bkb_project(const BSys* sys, const BKbItem* items, int n_items, cudaStream_t st);
// alpha_j += sum_p |C_p|^2 / h_p of every listed orbital (after launch_balpha)
cudaError_t launch_bkb_alpha(const BSys* sys, const BOrb* orbs, int n_orbs, cudaStream_t st);
// w += y over the covered nodes of block rows[i].rblk, partials to kb_part (after the assembly)
cudaError_t launch_bkb_add(const BSys* sys, const BRow* rows, int n_rows, cudaStream_t st);
// sys_sub[2 s] = largest sub-step count of system s, sys_sub[2 s + 1] = its
// orbital-vector Hbar applications (both accumulated until the host clears them)
cudaError_t launch_bkry_stats(const BSys* sys, const BOrb* orbs, int n_orbs,
                              unsigned long long* dof_applies, int* kseen, unsigned long long* sys_sub,
                              cudaStream_t st);
// V_HXC of an orbital block (density, Hartree by the polling CG, LDA) into out (capi.cu)
tdks_status vhxc_of(tdks_ctx* c, const double2* psi, int n_orb, double* out, int* cg_iters,
                    int prec = TDKS_FP64);
// capturable forms of the per-system field work (no host synchronization)
tdks_status cg_solve_graph(tdks_ctx* c, const double* b, double* x, int n_iter, int* err, bool df = false);
tdks_status hartree_graph(tdks_ctx* c, const double* rho_q, double* vh_q, int n_iter, int* err,
                          bool df = false);
tdks_status vhxc_graph(tdks_ctx* c, const double2* psi, int n_orb, double* out, int n_iter,
                       int* err,
                       int prec = TDKS_FP64);
tdks_status dipole_graph(tdks_ctx* c, const double* rho, double* base, const int* step,
                         int64_t step_stride);
cudaError_t launch_counter_add(int* counter, int inc, cudaStream_t st);

// kb.cu: nonlocal Kleinman-Bylander term, hooked into the Hbar application
void kb_free(tdks_ctx* c);
tdks_status kb_project(tdks_ctx* c, const ApplyArgs& a);   // C = Pbar^T (s_j) in
tdks_status kb_alpha(tdks_ctx* c, const ApplyArgs& a);     // alpha_j += sum |C|^2 / h
tdks_status kb_add(tdks_ctx* c, const ApplyArgs& a);       // out += Pbar D C (+ norm partials)
int kb_norm_blocks(const tdks_ctx* c);                      // partials of the Lanczos correction
const double* kb_norm_parts(const tdks_ctx* c);             // [n_orb][kb_norm_blocks]

// GLL-collocation variant of Hbar (elements.cu): out = M^-1/2 K_gll M^-1/2 psi + v_nodes psi
tdks_status launch_hbar_gll(tdks_ctx* c, const double2* psi, const double* v_nodes, double2* out,
                            int n_orb);
