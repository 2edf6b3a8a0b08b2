/*
 * tdks.h -- C ABI of the GB300 (sm_103a) library for real-time TDKS propagation
 * with higher-order spectral finite elements (Kanungo & Gavini, arXiv 1810.13130).
 *
 * The method (paper Sec. III-VI):
 *   * orbitals are expanded in C0 Lagrange elements on hexahedra whose nodes are
 *     the Gauss-Lobatto-Legendre (GLL) points (Eq. 13, Sec. VI.A), with zero
 *     Dirichlet values on the domain boundary;
 *   * the overlap M is integrated with the GLL rule on those nodes, so it is
 *     diagonal; every other integral uses the Gauss rule with nq = p+1 points per
 *     direction (Sec. VI.A);
 *   * the semi-discrete system i M psi' = H psi (Eqs. 14-15) is written in the
 *     Loewdin basis psibar = M^1/2 psi, i psibar' = Hbar psibar,
 *     Hbar = M^-1/2 H M^-1/2 (Eq. 21);
 *   * one time step is the second-order Magnus propagator with the midpoint rule,
 *     psibar^n = exp(-i dt Hbar[rho(t_{n-1} + dt/2)]) psibar^{n-1} (Eqs. 25-26),
 *     the midpoint Hamiltonian coming from a predictor-corrector (Sec. VI.B);
 *   * the exponential acts through adaptive Lanczos (Eqs. 36-38).
 *
 * Conventions for every entry point:
 *   * Buffers suffixed _dev are device pointers owned by the caller; _host are host
 *     pointers.  Complex vectors are interleaved (re, im) doubles.
 *   * An orbital block psi is [n_orb][n_int] complex values: the Loewdin
 *     coefficients psibar at the interior nodes, ordered x fastest, then y, then z.
 *     Interior node (I, J, K), 1 <= I <= nx*p - 1 etc., has index
 *     (I-1) + (nx*p-1) * ((J-1) + (ny*p-1) * (K-1)).
 *   * Quadrature-point fields (potentials, densities) are [n_elem][nq^3] doubles,
 *     element e = ex + nx*(ey + ny*ez), point q = qx + nq*(qy + nq*qz), Gauss
 *     points ascending within each element.
 *   * All work is ordered on the context's CUDA stream.  Calls that return host
 *     values synchronize that stream; the others are asynchronous.
 *   * Every call returns a tdks_status; nothing aborts or traps.  On failure,
 *     tdks_last_error() describes the cause.  Device-side loops (Krylov, CG) are
 *     bounded by iteration caps and report TDKS_ERR_NOT_CONVERGED.
 */
#ifndef TDKS_H
#define TDKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdks_ctx tdks_ctx;

typedef enum {
  TDKS_OK = 0,
  TDKS_ERR_ARG = -1,            /* invalid argument or descriptor            */
  TDKS_ERR_CUDA = -2,           /* a CUDA runtime call failed                */
  TDKS_ERR_NOMEM = -3,          /* device allocation failed                  */
  TDKS_ERR_NOT_CONVERGED = -4,  /* Krylov sub-step or CG cap reached          */
  TDKS_ERR_TIMEOUT = -5,        /* reserved for bounded device-side waits    */
  TDKS_ERR_NAN = -6             /* a non-finite value reached a reduction     */
} tdks_status;

/* Arithmetic of the cell-level contractions in apply_H.  Stored vectors, the
 * Lanczos recurrence, the small exponential, Poisson and the density and dipole
 * sums are always FP64; with TDKS_DF64 the Krylov recombination (tdks_expm,
 * tdks_magnus_step) and the density interpolation of a Magnus step are
 * double-float as well. */
typedef enum {
  TDKS_FP64 = 0,   /* double contractions                                  */
  TDKS_FP32 = 1,   /* float contractions with float accumulation, FP64 I/O  */
  TDKS_DF64 = 2,   /* double-float (compensated float-pair) contractions:
                      ~48-bit accurate products and sums on the FP32 pipe   */
  TDKS_BF16 = 3,   /* accuracy study: every contraction operand (input, 1-D
                      operator coefficients, each contraction result feeding
                      the next) rounded to bfloat16, FP32 products and sums,
                      i.e. the arithmetic of a BF16 tensor-core contraction,
                      run on the CUDA cores (no speed claim).  Single-system
                      calls only: tdks_batch_create rejects it.             */
  TDKS_MIXED = 4   /* relaxed precision inside each Lanczos exponential: the
                      Hbar applications of iteration j use double-float
                      contractions while some orbital's a-posteriori estimate
                      of Eq. 38 from iteration j-1 exceeds relax * tol, FP32
                      contractions after (see tdks_set_mixed); recombination
                      and density as TDKS_DF64.  tdks_apply_H treats it as
                      TDKS_DF64.  Single-system calls only.                 */
} tdks_prec;

typedef enum {
  TDKS_NUC_NONE = 0,
  TDKS_NUC_SOFT = 1,       /* -Z / sqrt(r^2 + a2),  nuc_param = a2          */
  TDKS_NUC_ERF = 2,        /* -Z erf(r / rc) / r,    nuc_param = rc          */
  TDKS_NUC_BARE = 3,       /* -Z / r                                          */
  TDKS_NUC_HARMONIC = 4    /* omega^2 |r - R_0|^2 / 2, nuc_param = omega      */
} tdks_nuc_kind;

/* Tensor-product hexahedral mesh: element breakpoints per axis (host arrays of
 * length n+1, strictly increasing), polynomial degree 1 <= p <= 8, nq Gauss
 * points per direction (0 selects p+1, the only value the GPU path accepts). */
typedef struct {
  int nx, ny, nz;
  const double* X;
  const double* Y;
  const double* Z;
  int p;
  int nq;
} tdks_mesh_desc;

/* The electronic system: n_orb orbitals with occupations occ (host, length n_orb;
 * 2.0 for doubly occupied), n_nuc nuclei at R (host, [n_nuc][3]) with charges Z,
 * the nuclear potential form, and switches for the Hartree and LDA terms. */
typedef struct {
  int n_orb;
  const double* occ;
  int n_nuc;
  const double* R;
  const double* Z;
  int nuc_kind;
  double nuc_param;
  int hartree;
  int xc;
} tdks_system_desc;

/* Per-step statistics returned by tdks_magnus_step. */
typedef struct {
  int k_half_max;      /* largest Krylov dimension in the dt/2 predictor exp   */
  int k_full_max;      /* largest Krylov dimension in the dt corrector exp     */
  int64_t applies;     /* orbital-vector Hbar applications in this step        */
  int substeps;        /* extra Krylov sub-steps taken (0 when none needed)    */
  int cg_iters[3];     /* Poisson CG iterations: half-step, full-step, unused  */
  double dipole[3];    /* dipole int r rho(t_n) dr                             */
} tdks_stats;

/* Create a context: builds the GLL/Gauss tables, the diagonal overlap (as 1-D
 * factors), the nuclear potential at the Gauss points and the work buffers.
 * stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: TDKS_ERR_ARG for a malformed descriptor, TDKS_ERR_NOMEM, TDKS_ERR_CUDA. */
tdks_status tdks_create(const tdks_mesh_desc* mesh, const tdks_system_desc* sys,
                        void* stream, tdks_ctx** out);
tdks_status tdks_destroy(tdks_ctx* ctx);
tdks_status tdks_set_stream(tdks_ctx* ctx, void* stream);

/* Sizes: interior nodes, elements, Gauss points per element. */
tdks_status tdks_sizes(const tdks_ctx* ctx, int64_t* n_int, int64_t* n_elem, int* nq3);

/* Poisson CG: stopping rule ||r|| <= tol ||b|| (at most maxit iterations) and
 * preconditioner.  TDKS_PRECOND_FDM (default) is the fast-diagonalization inverse
 * of the separable stiffness of an axis-aligned tensor mesh (exact up to rounding:
 * CG stops after one or two iterations); it is unavailable when an axis has more
 * than 1024 interior nodes (TDKS_ERR_ARG), where Jacobi is the default. */
typedef enum { TDKS_PRECOND_FDM = 0, TDKS_PRECOND_JACOBI = 1 } tdks_precond;
tdks_status tdks_set_cg(tdks_ctx* ctx, double tol, int maxit, int precond);

/* Copy the total Kohn-Sham potential V_KS at the Gauss points ([n_elem][nq^3],
 * device) into the context; tdks_apply_H and tdks_expm act with it. */
tdks_status tdks_set_potential(tdks_ctx* ctx, const double* v_q_dev);

/* Copy the nuclear potential V_N at the Gauss points into v_q_dev. */
tdks_status tdks_nuclear_potential(tdks_ctx* ctx, double* v_q_dev);

/* out = Hbar psi for n_orb orbitals (Eqs. 15, 21): matrix-free, element by
 * element: Loewdin scale and gather, interpolation to the Gauss points, the
 * kinetic form 1/2 int grad N . grad N and the potential form int V N N, and the
 * scatter-add with the Loewdin scale.  psi_dev and out_dev must not overlap.
 * n_orb >= 1 vectors of n_int complex values each; the system's orbital count
 * does not bound it (the element-result buffer grows to fit). */
tdks_status tdks_apply_H(tdks_ctx* ctx, const double* psi_dev, double* out_dev,
                         int n_orb, int prec);

/* rho(x_q) = sum_a occ_a |psi_a(x_q)|^2 with psi = M^-1/2 psibar (Eq. 2). */
tdks_status tdks_density(tdks_ctx* ctx, const double* psi_dev, int n_orb, double* rho_q_dev);

/* Dipole int r rho(r) dr by the Gauss rule (Sec. V, Eq. 30); synchronizes. */
tdks_status tdks_dipole(tdks_ctx* ctx, const double* rho_q_dev, double d_host[3]);

/* Hartree potential at the Gauss points: K phi = 4 pi c (Eq. 19), zero Dirichlet
 * boundary, preconditioned CG (see tdks_set_cg) warm-started from the previous
 * solution kept in the context.  iters_host receives the iteration count (may be
 * NULL); synchronizes. */
tdks_status tdks_hartree(tdks_ctx* ctx, const double* rho_q_dev, double* vh_q_dev,
                         int* iters_host);

/* LDA exchange-correlation potential v_xc(rho) at the Gauss points (Sec. II:
 * Ceperley-Alder data, Perdew-Zunger 1981 unpolarized fit; 0 below rho = 1e-14). */
tdks_status tdks_xc(tdks_ctx* ctx, const double* rho_q_dev, double* vxc_q_dev);

/* psi_out = exp(-i tau Hbar) psi_in by adaptive Lanczos (Eqs. 36-38) with the
 * potential last set by tdks_set_potential.  Stops each orbital when
 * tau beta_k ||psi|| |[exp(-i tau T_k) e_1]_k| <= tol; at k_max (<= 128) without
 * convergence it takes exact sub-steps tau_rem / 2^m.  psi_out may equal psi_in.
 * k_used_host (may be NULL): [n_orb] sum of Krylov dimensions over sub-steps.
 * Synchronizes. */
tdks_status tdks_expm(tdks_ctx* ctx, const double* psi_in_dev, double* psi_out_dev,
                      int n_orb, double tau, double tol, int k_max, int prec,
                      int* k_used_host);

/* Delta kick psibar_j <- exp(-i kappa dir . x_j) psibar_j at every interior node. */
tdks_status tdks_kick(tdks_ctx* ctx, double* psi_dev, int n_orb, double kappa,
                      const double dir[3]);

/* Start a propagation from psi: V_HXC(t_0) from its density, history
 * V_HXC(t_{-1}) := V_HXC(t_0).  d_host (may be NULL) receives the dipole. */
tdks_status tdks_init_propagation(tdks_ctx* ctx, const double* psi_dev, int n_orb,
                                  double d_host[3]);

/* One predictor-corrector Magnus step (Eqs. 25-26, Sec. VI.B) in place:
 *   V_pred = V_N + 1.25 V_HXC^{n-1} - 0.25 V_HXC^{n-2} - E_quarter . r
 *   psi_half = exp(-i dt/2 Hbar[V_pred]) psi
 *   V_mid = V_N + V_HXC[rho(psi_half)] - E_half . r
 *   psi <- exp(-i dt Hbar[V_mid]) psi;  V_HXC^n from rho(psi)
 * E_quarter, E_half: host 3-vectors, the field at t_{n-1} + dt/4 and + dt/2.
 * prec selects the contraction arithmetic of every Hbar application; with
 * TDKS_DF64 the Krylov recombination and the interpolation of the density to the
 * Gauss points are double-float as well (sums over orbitals stay FP64).
 * stats (may be NULL) is filled; synchronizes. */
tdks_status tdks_magnus_step(tdks_ctx* ctx, double* psi_dev, int n_orb, double dt,
                             const double E_quarter[3], const double E_half[3],
                             double tol, int k_max, int prec, tdks_stats* stats);

/* End-to-end call with host buffers: copies psi_host_in to the device, runs
 * tdks_init_propagation when init != 0, then n_steps Magnus steps with the field
 * samples E_host ([n_steps][6]: E at t+dt/4 then at t+dt/2), writes the dipoles
 * ([n_steps][3]) and copies the final orbitals to psi_host_out.  Uses a device
 * orbital buffer owned by the context. */
tdks_status tdks_propagate_host(tdks_ctx* ctx, const double* psi_host_in,
                                double* psi_host_out, int n_orb, int init, int n_steps,
                                double dt, const double* E_host, double tol, int k_max,
                                int prec, double* dipole_host);

/* Nonlocal pseudopotential term in the Kleinman-Bylander form (Eq. 6):
 *   V_nl phi = sum_p [int chi_p phi / h_p] chi_p,  chi_p = dV_l u_lm,  h_p = int u_lm dV_l u_lm,
 * discretized as Hbar_nl = M^-1/2 P D P^T M^-1/2 with P[j][p] = int chi_p N_j and
 * D = diag(1/h_p), all integrals by the Gauss rule (Sec. VI.A).  Synthetic projectors on
 * n_atoms atoms at R_host ([n_atoms][3], bohr), with d = r - R:
 *   u_lm = exp(-|d|^2 / (2 a^2)) Y_lm(d),  Y_00 = 1, Y_1m = d_x, d_y, d_z  (l <= lmax),
 *   dV_l = c[l] exp(-|d|^2 / (2 b^2)),
 * projectors ordered atom by atom, l = 0 then d_x, d_y, d_z.  After the call every
 * Hbar application of the context (tdks_apply_H, tdks_expm, tdks_magnus_step, the
 * objective and its adjoint) includes Hbar_nl; n_atoms = 0 removes it.  Each atom's
 * projector columns are stored on the box of nodes where some entry exceeds 1e-16 of
 * the column maximum.  lmax in {0, 1}; a, b > 0.  Synchronizes.  tdks_batch_set_kb
 * gives one system of a batch the same term.
 * tdks_kb_info: projector count, the denominators h_p (h_host, n_proj doubles, may be
 * NULL), the number of nodes covered by some box and the stored values. */
tdks_status tdks_set_kb(tdks_ctx* ctx, int n_atoms, const double* R_host, double a, double b,
                        const double c[2], int lmax);
tdks_status tdks_kb_info(const tdks_ctx* ctx, int* n_proj, double* h_host, int64_t* n_covered,
                         int64_t* n_values);

/* GLL-collocation variant of Hbar (not the paper's operator: every integral of H by
 * the GLL rule on the element nodes instead of the Gauss rule of Sec. VI.A):
 *   out = M^-1/2 K_gll M^-1/2 psi + v_nodes .* psi,
 * K_gll per element = sum_d c_d (K1 along d) (x) W_l (x) W_l with the exact 1-D stiffness
 * K1 and the GLL weights W_l (transverse mass lumped); the potential is diagonal in
 * the Loewdin basis.  v_nodes_dev: V at the interior nodes ([n_int], device, e.g. from
 * tdks_nuclear_potential_nodes).  FP64.  psi_dev and out_dev must not overlap. */
tdks_status tdks_apply_H_gll(tdks_ctx* ctx, const double* psi_dev, const double* v_nodes_dev,
                             double* out_dev, int n_orb);
/* V_N at the interior nodes ([n_int], device). */
tdks_status tdks_nuclear_potential_nodes(tdks_ctx* ctx, double* v_nodes_dev);

/* Self-consistent midpoint step (Sec. VI.B, the fully consistent approach that the
 * predictor-corrector of tdks_magnus_step replaces): starting from
 * V_mid = 1.5 V_HXC^{n-1} - 0.5 V_HXC^{n-2}, repeat
 *   psi^n = exp(-i dt Hbar[V_N + V_mid - E_half . r]) psi^{n-1}, V_HXC^n from rho(psi^n),
 *   V_mid <- (V_HXC^{n-1} + V_HXC^n) / 2
 * until the largest change of V_mid is <= sc_tol (at most sc_maxit exponentials, else
 * TDKS_ERR_NOT_CONVERGED).  E_half: field at t + dt/2 (host).  *iters = exponentials
 * taken.  Needs tdks_init_propagation; updates the history like tdks_magnus_step.
 * Synchronizes once per iteration. */
tdks_status tdks_magnus_step_sc(tdks_ctx* ctx, double* psi_dev, int n_orb, double dt,
                                const double E_half[3], double tol, int k_max, int prec,
                                double sc_tol, int sc_maxit, tdks_stats* stats, int* iters);

/* Absorption spectrum (Sec. VII): for a dipole series dip_host ([n_t][3], d(t_n),
 * t_n = n dt) after a kick psi(0) = exp(-i kappa r.dir) psi_GS,
 *   alpha(omega) = -(1/kappa) sum_n w_n exp(i omega t_n) g(t_n) (d(t_n) - d(0)) . dir/|dir|
 * (trapezoid weights w_n, window g(t) = exp(-window t^2)) into alpha_host ([n_om] complex
 * (re, im), may be NULL) and S(omega) = (2 omega / 3 pi) Im alpha(omega) into S_host
 * ([n_om], may be NULL); summing S over kicks along x, y, z gives the trace.  All
 * arrays are host memory; computed on the current device.  Synchronizes. */
tdks_status tdks_spectrum(const double* dip_host, int n_t, double dt, double kappa,
                          const double dir[3], double window, const double* omega_host, int n_om,
                          double* alpha_host, double* S_host);

/* Dipole-response objective and its gradient with respect to the field (the
 * adjoint of Secs. VI.B and V; the paper optimizes nothing, this is the reverse
 * mode of its propagation).
 *
 * J = sum_{n=0}^{n_steps} w_host[n] (e . mu_n)^2, mu_0 the dipole of psi0 and mu_n
 * the dipole after Magnus step n with field samples E_host[n-1] ([n_steps][6]:
 * E(t+dt/4) for the predictor, then E(t+dt/2) for the corrector).
 *
 * tdks_objective_forward: psi0 is device memory ([n_orb][n_int] complex, left
 * unchanged); re-initializes the propagation (as tdks_init_propagation) and
 * propagates n_steps steps with precision prec, storing a checkpoint of the
 * state every ckpt_every steps in device memory owned by the context
 * (ceil(n_steps / ckpt_every) x (orbitals + 2 potentials + Poisson solution)).
 * Writes J to *J_host and, if dip_host is not NULL, the n_steps + 1 dipoles
 * ([n_steps+1][3]).  Replaces the state of an earlier forward call.
 *
 * tdks_objective_backward: after a forward call, writes dJ/dE to dJdE_host
 * ([n_steps][6], same layout as E_host).  Each segment of ckpt_every steps is
 * recomputed from its checkpoint (extra device memory: ckpt_every x (2 orbital
 * sets + 2 potentials)), then swept in reverse: the exact adjoint of every
 * exponential (a Lanczos exponential with time -tau), the Frechet derivative of
 * exp(-i tau Hbar[v]) with respect to v by n_s-point Gauss-Legendre quadrature
 * in the splitting parameter (1 <= n_s <= 64), and the adjoints of the Hartree
 * solve (Eq. 19), the LDA potential and the density.  Each adjoint exponential
 * must converge within one Krylov basis of dimension k_max (else
 * TDKS_ERR_NOT_CONVERGED).  Leaves the context's propagation state undefined:
 * call tdks_init_propagation before propagating again.  Synchronizes. */
tdks_status tdks_objective_forward(tdks_ctx* ctx, const double* psi0, int n_orb, int n_steps,
                                   double dt, const double* E_host, const double* w_host,
                                   const double e[3], int ckpt_every, double tol, int k_max,
                                   int prec, double* J_host, double* dip_host);
tdks_status tdks_objective_backward(tdks_ctx* ctx, int n_s, double* dJdE_host);

/* Batched propagation of many independent systems (no counterpart in the paper,
 * which propagates one system at a time: a throughput form of the same step).
 *
 * Each system has its own mesh, degree, orbitals, nuclei and time step; all
 * advance together by the predictor-corrector Magnus step of Sec. VI.B with no
 * external field.  One step of all systems is one CUDA graph replay; the Krylov
 * loops run on the device (conditional graph nodes) and the Poisson CG of every
 * system takes a fixed number of fast-diagonalization-preconditioned iterations
 * (each system's axes must have <= 1024 interior nodes, else TDKS_ERR_ARG).
 *
 * tdks_batch_create: n_sys systems; meshes/systems as for tdks_create, dt[n_sys]
 *   (> 0), contraction precision prec (TDKS_FP64/FP32/DF64/MIXED), Lanczos tolerance
 *   and k_max (2..128).  TDKS_MIXED chooses per orbital: an orbital's products are
 *   double-float until its own a-posteriori estimate (Eq. 38) is <= 1e8 * tol, FP32
 *   after (each persistent apply launch takes the orbitals of its type); recombination
 *   and density double-float.  The batch owns one CUDA stream (tdks_batch_stream) on
 *   which all its work runs, the orbitals of every system and all workspaces
 *   (Krylov basis: n_orb x k_max x n_int complex per system).
 * tdks_batch_set_orbitals / get_orbitals: device copies of one system's block
 *   [n_orb][n_int] complex128 (tdks_batch_sizes gives the sizes).
 * tdks_batch_kick: psi_s <- exp(-i kappa[s] r . dir[s]) psi_s (Sec. VII.A).
 * tdks_batch_init: V_HXC history and the dipoles ([n_sys][3]) of the current
 *   orbitals (as tdks_init_propagation for every system).
 * tdks_batch_tune: chooses the elements per CTA of every degree and the orbitals
 *   per work item of every (degree, orbital count) class by timing `reps`
 *   (1..32) launches of each candidate; writes up to cap choices (tile table)
 *   to out.
 *   Optional; without it the largest tile and one orbital per item are used.
 * tdks_batch_tune_kmax: per-system Krylov caps.  The Lanczos loop of a system whose
 *   a-posteriori estimate (Eq. 38) has not met the tolerance at its cap restarts
 *   from the vector reached (sub-steps), which costs Hbar applications; a larger
 *   basis for that system avoids them at the price of memory.  After at least one
 *   tdks_batch_steps call, every system that took more than one sub-step in an
 *   exponential (since creation, or since its cap was last raised) gets the cap
 *   k_cap (above its current cap, <= 128), the systems with the most Hbar work
 *   first, as long as the added Krylov basis
 *   (n_orb x (k_cap - cap) x n_int complex128 per system) fits in mem_budget bytes
 *   (< 0: half of the device's free memory); the others keep theirs.  A system
 *   whose larger basis cannot be allocated keeps its cap.  Writes the caps
 *   [n_sys] to kmax_out (may be NULL).  The orbitals are unchanged; later steps
 *   take at most as many sub-steps as before and reach the same tolerance.
 *   The step graph is rebuilt on the next tdks_batch_steps call.  TDKS_ERR_ARG for
 *   k_cap outside 2..128 or before any step.
 * tdks_batch_set_kb: the nonlocal Kleinman-Bylander term of tdks_set_kb (same
 *   arguments, same projectors and storage) for system sys of the batch; every later
 *   step of that system applies Hbar + Hbar_nl in its Lanczos iterations (projection
 *   with each orbital's own Krylov vector, alpha and the norm of the new vector
 *   corrected as in the single-system path; Eq. 6).  n_atoms = 0 removes it.
 *   Synchronizes; the step graph is rebuilt on the next tdks_batch_steps call.
 *   TDKS_ERR_ARG for sys outside 0..n_sys-1 or the argument errors of tdks_set_kb;
 *   TDKS_ERR_NOMEM if the projector storage cannot be allocated.
 * tdks_batch_steps: n_steps steps of every system; dipoles [n_steps][n_sys][3].
 *   Synchronizes.  TDKS_ERR_NOT_CONVERGED if a Lanczos loop failed or hit its
 *   pass cap (16 x the largest k_max passes) or a Poisson solve did not converge.
 * tdks_batch_stats: sum over orbital-vector Hbar applications of the system's
 *   interior DoF count, and the largest Krylov dimension seen. */
typedef struct tdks_batch tdks_batch;
typedef struct {
  int p;                /* degree of the class                                  */
  int n_orb;            /* orbital count of the class                           */
  int elems_per_cta;    /* tile: elements per CTA chosen for the degree          */
  int orbs_per_item;    /* tile: orbitals per work item chosen for the class     */
  double ms;            /* measured apply time of the class with that tile       */
} tdks_tile_choice;
tdks_status tdks_batch_create(int n_sys, const tdks_mesh_desc* meshes,
                              const tdks_system_desc* systems, const double* dt, int prec,
                              double tol, int k_max, tdks_batch** out);
tdks_status tdks_batch_destroy(tdks_batch* b);
void* tdks_batch_stream(tdks_batch* b);
tdks_status tdks_batch_sizes(const tdks_batch* b, int sys, int64_t* n_int, int64_t* n_elem,
                             int* nq3, int* n_orb);
tdks_status tdks_batch_set_orbitals(tdks_batch* b, int sys, const double* psi_dev);
tdks_status tdks_batch_get_orbitals(tdks_batch* b, int sys, double* psi_dev);
tdks_status tdks_batch_kick(tdks_batch* b, const double* kappa, const double* dir);
tdks_status tdks_batch_init(tdks_batch* b, double* dip_host);
tdks_status tdks_batch_tune(tdks_batch* b, int reps, tdks_tile_choice* out, int cap, int* n_out);
tdks_status tdks_batch_tune_kmax(tdks_batch* b, int k_cap, int64_t mem_budget, int* kmax_out);
tdks_status tdks_batch_set_kb(tdks_batch* b, int sys, int n_atoms, const double* R_host, double a,
                              double b_, const double c[2], int lmax);
tdks_status tdks_batch_steps(tdks_batch* b, int n_steps, double* dip_host);
tdks_status tdks_batch_stats(tdks_batch* b, int64_t* dof_applies, int* k_max_seen, int reset);
/* Phase timing of the step graph (diagnostics): with timing on, the graph records
 * CUDA events at the phase boundaries; tdks_batch_phase_ms gives the device time
 * of the last step's phases [predictor, half-step exponential, corrector
 * fields, full-step exponential, history + dipole] and the loop passes of the two
 * exponentials.  Turning timing on or off rebuilds the graph. */
tdks_status tdks_batch_set_timing(tdks_batch* b, int on);
tdks_status tdks_batch_phase_ms(tdks_batch* b, double ms[5], int passes[2]);
/* The half-step exponential of the current state once more, outside the graph,
 * kernel group by kernel group (as many passes as the last step's half-step
 * loop): ms = device time of [norms, apply, alpha, assembly, small exponentials,
 * recombination].  Overwrites only internal scratch; the state is unchanged. */
tdks_status tdks_batch_profile_pass(tdks_batch* b, double ms[6]);
const char* tdks_batch_last_error(const tdks_batch* b);

/* Lanczos variant of every exponential of the context (tdks_expm, the Magnus steps,
 * the adjoint).  reorth = 0 (default): the plain three-term recurrence (Sec. VI.B
 * names no re-orthogonalization).  reorth = 1: after the three-term update the new
 * vector is orthogonalized against every basis vector so far by classical
 * Gram-Schmidt applied twice (CGS2), and beta_j is its norm after the two passes;
 * alpha_j keeps its three-term value.  Costs about 4 (j + 1) vector reads at step j.
 * The batched engine does not take this option. */
tdks_status tdks_set_lanczos(tdks_ctx* ctx, int reorth);

/* Lanczos loop of every exponential of the context (tdks_expm, the Magnus steps, the
 * objective and its adjoint; Eqs. 36-38 -- an execution choice, not part of the method).
 * on = 1 (default): the iterations of a sub-step are one CUDA graph launch, each
 * iteration after the first a conditional node whose condition a one-block kernel sets
 * from the Lanczos state of the previous iteration (some orbital still active; under
 * TDKS_MIXED also the contraction arithmetic), so the host reads that state once per
 * sub-step.  The graph is captured on first use for a given starting vector and
 * settings and kept with the context.  on = 0: the host launches every iteration and
 * reads the state after each.  Both run the same kernels in the same order, so the
 * results are identical. */
tdks_status tdks_set_device_loop(tdks_ctx* ctx, int on);

/* Switch level of TDKS_MIXED (no counterpart in the paper; a precision schedule for
 * the Lanczos exponential of Eqs. 36-38).  With inexact matrix-vector products the
 * error that the product of iteration j adds to exp(-i tau Hbar) psi is about
 * |tau| ||psi|| |y_j| ||delta_j||, y = exp(-i tau T) e_1 and delta_j the product's
 * error; the a-posteriori estimate eps_j = |tau| beta_j ||psi|| |y_j| measures that
 * weight.  Products after the iteration whose estimate fell to relax * tol (for every
 * active orbital) therefore use FP32 contractions (relative error ~1e-7 of
 * ||Hbar||), the earlier ones double-float.  relax >= 0; default 1e8; 0 gives
 * double-float throughout.  The stopping rule is unchanged. */
tdks_status tdks_set_mixed(tdks_ctx* ctx, double relax);

/* Orbitals per CTA of the element kernel of every Hbar application of the context
 * (the kernel of Eqs. 15, 21; a launch-shape setting, not part of the method).  The
 * CTAs of the kernel form a grid of element blocks x orbital chunks; each CTA
 * applies Hbar to its elements for orbs_per_cta orbitals in turn, reusing the
 * potential, geometry and Loewdin scales of its elements.  0 (default): chosen per
 * launch (the largest power of two that keeps at least 8 CTAs per SM); n > 0: n
 * (at most the orbital count of the call).  Results do not depend on it. */
tdks_status tdks_set_apply_tile(tdks_ctx* ctx, int orbs_per_cta);

/* Per-stage precision study of the double-float Hbar application (diagnostics, no
 * counterpart in the paper).  The element kernel of Eqs. 15, 21 applies the
 * sum-factorized operator as nine one-dimensional contractions in Gauss-point space
 * (Sec. VI.A): bits 0-2 the interpolation to the Gauss points along z, y, x; bits 3-5
 * the kinetic contractions along x, y, z; bits 6-8 the transposed interpolation along
 * z, y, x; bit 9 the pointwise combination of the potential and kinetic terms; bit 10
 * the gathered, Loewdin-scaled input; bit 11 the element results handed to the
 * assembly.  Every later double-float application of the context (TDKS_DF64 and the
 * double-float products of TDKS_MIXED) runs the stages whose bit is set in mask in
 * FP32 arithmetic with FP32 operator coefficients and the others in double-float, so
 * that the error each stage contributes can be measured on its own.  mask = 0
 * (default) restores the ordinary kernel.  Degrees p = 4 and 6 only: a double-float
 * application at another degree with a nonzero mask fails with TDKS_ERR_ARG.
 * mask < 2^12. */
tdks_status tdks_set_f32_stages(tdks_ctx* ctx, unsigned mask);

/* Work counters of a context (for benchmarking): kernel launches issued, Hbar
 * colour launches, element-orbital applications, and -- when timing is on --
 * the summed device time of the Hbar applications inside tdks_expm measured
 * with CUDA events on the context's stream.  reset != 0 zeroes them after
 * reading.  out may be NULL (reset only). */
typedef struct {
  int64_t launches;
  int64_t apply_launches;
  int64_t apply_elem_orb;
  double apply_ms;
  int64_t cg_iters;
  int64_t apply_launches_fp32;   /* TDKS_MIXED: applications run with FP32 contractions */
  int64_t state_reads;           /* synchronizing reads of the Lanczos state by the host */
} tdks_counters;
tdks_status tdks_set_timing(tdks_ctx* ctx, int on);
tdks_status tdks_get_counters(tdks_ctx* ctx, tdks_counters* out, int reset);

/* One-dimensional contraction stage of the element kernels in four arithmetic forms (a
 * measurement utility, no counterpart in the paper): y = M^reps x for n_lines lines of
 * P1 values (x_dev, y_dev: [n_lines][P1] doubles, device; n_lines a multiple of 512),
 * M the P1 x P1 operator op_host (row-major M[q][i], host; 2 <= P1 <= 8), every power
 * applied in shared memory after one load, so the time is that of the stage's arithmetic
 * and shared-memory traffic.  variant 0: FP32 FMAs on the CUDA cores; 1: double-float
 * on the CUDA cores; 2: tensor cores with BF16 operands and FP32 accumulation
 * (mma m16n8k16, lines as the M dimension, K and N padded to 16 and 8); 3: tensor cores,
 * three TF32 products per product (mma m16n8k8, FP32-level products).  ms_host: device
 * time of one launch after an untimed one (CUDA events).  Synchronizes. */
tdks_status tdks_contraction_probe(int variant, int P1, const double* op_host, const double* x_dev,
                                   double* y_dev, int64_t n_lines, int reps, void* stream,
                                   double* ms_host);

/* Arithmetic peak of the current device for the roofline of the contraction
 * kernels (no counterpart in the paper: a measurement utility).  prec TDKS_FP64 or
 * TDKS_FP32: reps launches of ctas_per_sm (1..32) CTAs per SM x 256 threads, each
 * thread running 8 independent chains of iters fused multiply-adds in that type,
 * timed with CUDA events on stream (a cudaStream_t) after one untimed launch.
 * tflops_host: 2 x FMAs / time in TFLOP/s; ms_host: time per launch (either may be
 * NULL).  Allocates and frees a small output buffer; synchronizes. */
tdks_status tdks_fma_probe(int prec, int ctas_per_sm, int iters, int reps, void* stream,
                           double* tflops_host, double* ms_host);

/* Allocation-free dipole (no counterpart in the paper; a service for callers that
 * cannot allocate device memory -- programs whose device memory belongs to another
 * allocator with a fixed budget, or code that must not allocate once it is running,
 * e.g. a real-time propagation loop after its start-up).
 * Computes the same int r rho dr as tdks_dipole without a context: rho_q_dev is
 * [nx*ny*nz][(p+1)^3] at the Gauss points (layout as above; the call reads exactly
 * that many doubles and cannot check the length itself), X/Y/Z the host
 * breakpoints, 1 <= p <= 8, stream a cudaStream_t of the current device (rho_q_dev
 * must be memory of that device).  Allocates nothing: its scratch (partial sums,
 * results, copies of the breakpoints and Gauss rule) is a fixed 16384-double array
 * in the library's device image, held by every GPU that loads the library until the
 * process exits; meshes with nx + ny + nz + 2(p+1) > 14549 are rejected with
 * TDKS_ERR_ARG.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process, so make the
 * first call on each device before any stream capture, and do not call it on a
 * device after cudaDeviceReset (the kept address would be stale).  All calls share
 * the array: calls that overlap on the GPU race; serialize them.  Every call
 * synchronizes the stream (it copies the three results to d_host); returns
 * TDKS_ERR_CUDA if a CUDA call fails. */
tdks_status tdks_dipole_noalloc(const double* rho_q_dev, int nx, int ny, int nz,
                                const double* X, const double* Y, const double* Z, int p,
                                void* stream, double d_host[3]);

const char* tdks_last_error(const tdks_ctx* ctx);
const char* tdks_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* TDKS_H */
