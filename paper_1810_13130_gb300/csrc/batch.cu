// Batched propagation of many independent systems (uneven meshes, degrees and
// orbital counts) by the same launches.
//
// One Magnus predictor-corrector step (Sec. VI.B, Eqs. 25-26) of every system is
// one CUDA graph:
//   V_pred of every system                       (per-system kernels)
//   WHILE (some orbital active): one pass of the batched Lanczos exponential
//     exp(-i dt/2 Hbar) psi -> psi_half           (conditional graph node)
//   density, Hartree (fixed-length CG), LDA, V_mid of every system
//   WHILE: exp(-i dt Hbar) psi -> psi               (conditional graph node)
//   V_HXC history, dipole of every system
// A pass of the loop body is a handful of launches covering all systems: the
// apply is a persistent kernel per degree class walking a work list of
// (system, element block, orbital block) tiles; norms, assembly with the fused
// three-term update, the small exponentials and the recombination are one launch
// each over all (system, orbital) pairs.  Every orbital carries its own Lanczos
// state, so systems with different Krylov dimensions, time steps and sub-steps
// progress independently; the loop ends on the device when all are done (or at
// a pass cap, reported as an error).  The host reads nothing inside a step.
//
// Tiles: the elements per CTA (E) of each degree and the orbitals per work item
// of each (degree, orbital count) class are chosen by timing the candidates on
// the batch itself (tdks_batch_tune).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "tdks_internal.h"

namespace {

constexpr int kMaxSubPasses = 16;   // loop cap = kMaxSubPasses * (largest k_max) passes
constexpr int kFieldStreams = 16;   // parallel branches of the per-system field work
constexpr int kDegStreams = 9;      // parallel branches of the per-degree applies
std::string g_create_err;           // message of the last failed tdks_batch_create

struct Deg {
  int P1 = 0, E = 1, grid = 1, n_items = 0;
  BItem* d_items = nullptr;
  const void* tab = nullptr;
  int grid32 = 1;                 // TDKS_MIXED: the FP32 launch over the same work list
  const void* tab32 = nullptr;
  BRow* d_rows_asm = nullptr;     // gather items of the class's systems (larger rows first)
  int n_rows_asm = 0;
};

}  // namespace

struct tdks_batch {
  int n_sys = 0, prec = 0, cg_iters = 4, n_sm = 152;
  int kmax = 64;                    // largest per-system Krylov cap (BSys::kmax)
  double tol = 1e-10;
  double theta = -1.0;              // TDKS_MIXED: FP32 products once an estimate is <= theta
  cudaStream_t st = nullptr, st_body = nullptr;
  cudaStream_t fs[kFieldStreams] = {};   // capture-only fork streams (field work)
  cudaStream_t ds[kDegStreams] = {};     // capture-only fork streams (loop body)
  cudaEvent_t fork_ev = nullptr, body_fork_ev = nullptr;
  cudaEvent_t join_ev[kFieldStreams] = {}, body_join_ev[kDegStreams] = {};
  std::vector<int> field_order;          // systems by decreasing size
  std::vector<tdks_ctx*> ctx;
  std::vector<int> n_orb, n_eblk, n_rblk, opb;
  std::vector<double> dt;
  std::vector<double2*> psi, psi_half, Vw;
  std::vector<KryOrb*> kry;
  std::vector<void*> ev;
  std::vector<double*> apart, npart;
  std::vector<BSys> h_half, h_full;
  BSys *d_half = nullptr, *d_full = nullptr;
  BOrb* d_orbs = nullptr;
  int n_gorb = 0;
  BRow* d_rows = nullptr;
  int n_rows = 0;
  // nonlocal term of the systems that have projectors: projection items, orbitals,
  // node blocks of the gather
  BKbItem* d_kb_items = nullptr;
  BOrb* d_kb_orbs = nullptr;
  BRow* d_kb_rows = nullptr;
  int n_kb_items = 0, n_kb_orbs = 0, n_kb_rows = 0;
  std::vector<Deg> degs;
  int* d_ctrl = nullptr;            // [0], [1]: pass counters, [2]: error bits, [3]: step, [4]: k seen
  int* d_qctr = nullptr;            // work ticket counters of the apply launches (one per degree)
  unsigned long long* d_dof = nullptr;
  unsigned long long* d_sub = nullptr;   // per system: largest sub-step count, Hbar applies
  double* d_dip = nullptr;
  int dip_cap = 256;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool orbitals_set = false, ready = false;
  bool timing = false;              // event nodes at the phase boundaries of the step graph
  cudaEvent_t tev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  std::vector<tdks_tile_choice> tiles;
  std::string err;
};

namespace {

tdks_status bfail(tdks_batch* b, tdks_status s, const std::string& m) {
  b->err = m;
  return s;
}

#define B_CU(b, call)                                                             \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      cudaGetLastError();                                                         \
      return bfail(b, TDKS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                             \
  } while (0)

#define B_TRY(b, call, who)                                                       \
  do {                                                                            \
    tdks_status s_ = (call);                                                      \
    if (s_ != TDKS_OK) return bfail(b, s_, std::string(who) + ": " + (b)->err);   \
  } while (0)

template <typename T>
tdks_status balloc(tdks_batch* b, T** p, size_t count) {
  if (cudaMalloc((void**)p, (count ? count : 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, TDKS_ERR_NOMEM, "batch buffers");
  }
  return TDKS_OK;
}

tdks_status ctx_try(tdks_batch* b, tdks_ctx* c, tdks_status s) {
  if (s != TDKS_OK) b->err = c ? c->err : std::string("context");
  return s;
}

// contraction type of the apply launches (TDKS_MIXED: double-float, plus an FP32 launch)
int apply_prec(const tdks_batch* b) { return b->prec == TDKS_MIXED ? TDKS_DF64 : b->prec; }
// arithmetic of the density interpolation
int field_prec(const tdks_batch* b) { return b->prec == TDKS_MIXED ? TDKS_DF64 : b->prec; }
// ticket counters zeroed per pass: one per degree, two under TDKS_MIXED
int n_tickets(const tdks_batch* b) { return b->prec == TDKS_MIXED ? 2 * kDegStreams : kDegStreams; }

// the apply of degree class i on `sys` (both launches under TDKS_MIXED)
cudaError_t apply_degree(const tdks_batch* b, int i, const BSys* sys, cudaStream_t st) {
  const Deg& d = b->degs[i];
  cudaError_t e = launch_hbar_batch(d.P1, apply_prec(b), sys, d.d_items, d.n_items, d.E, d.grid, d.tab,
                                    b->d_qctr + i, st);
  if (e == cudaSuccess && b->prec == TDKS_MIXED)
    e = launch_hbar_batch(d.P1, TDKS_FP32, sys, d.d_items, d.n_items, d.E, d.grid32, d.tab32,
                          b->d_qctr + kDegStreams + i, st);
  return e;
}

void free_batch(tdks_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto* p : b->psi) cudaFree(p);
  for (auto* p : b->psi_half) cudaFree(p);
  for (auto* p : b->Vw) cudaFree(p);
  for (auto* p : b->kry) cudaFree(p);
  for (auto* p : b->ev) cudaFree(p);
  for (auto* p : b->apart) cudaFree(p);
  for (auto* p : b->npart) cudaFree(p);
  for (auto& d : b->degs) {
    cudaFree(d.d_items);
    cudaFree(d.d_rows_asm);
  }
  void* ptrs[] = {b->d_half, b->d_full, b->d_orbs, b->d_rows, b->d_ctrl, b->d_qctr,
                  b->d_dof, b->d_sub, b->d_dip, b->d_kb_items, b->d_kb_orbs, b->d_kb_rows};
  for (void* p : ptrs) cudaFree(p);
  for (auto* c : b->ctx) tdks_destroy(c);
  for (auto& e : b->tev)
    if (e) cudaEventDestroy(e);
  for (auto& x : b->fs)
    if (x) cudaStreamDestroy(x);
  for (auto& x : b->ds)
    if (x) cudaStreamDestroy(x);
  for (auto& e : b->join_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : b->body_join_ev)
    if (e) cudaEventDestroy(e);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->body_fork_ev) cudaEventDestroy(b->body_fork_ev);
  if (b->st_body) cudaStreamDestroy(b->st_body);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

void invalidate_graph(tdks_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

int emax_of(int P1) { return std::max(1, 256 / (P1 * P1)); }

// Work list of one degree class with E elements per tile and opb[s] orbitals per item,
// larger items first (static striding of the persistent grid then balances better).
std::vector<BItem> make_items(const tdks_batch* b, int P1, int E, const std::vector<int>& opb,
                              const std::vector<int>* only) {
  std::vector<BItem> items;
  for (int s = 0; s < b->n_sys; ++s) {
    if (b->ctx[s]->P1 != P1) continue;
    if (only && std::find(only->begin(), only->end(), s) == only->end()) continue;
    const long long ne = b->ctx[s]->n_elem;
    const int nb = (int)((ne + E - 1) / E);
    const int ob = std::max(1, opb[s]);
    for (int eb = 0; eb < nb; ++eb)
      for (int o0 = 0; o0 < b->n_orb[s]; o0 += ob)
        items.push_back(BItem{s, eb, o0, std::min(o0 + ob, b->n_orb[s])});
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const BItem& x, const BItem& y) { return (x.o1 - x.o0) > (y.o1 - y.o0); });
  return items;
}

tdks_status upload_descriptors(tdks_batch* b) {
  for (int s = 0; s < b->n_sys; ++s) {
    b->h_half[s].n_eblk = b->n_eblk[s];
    b->h_full[s].n_eblk = b->n_eblk[s];
  }
  B_CU(b, cudaMemcpyAsync(b->d_half, b->h_half.data(), b->n_sys * sizeof(BSys), cudaMemcpyHostToDevice, b->st));
  B_CU(b, cudaMemcpyAsync(b->d_full, b->h_full.data(), b->n_sys * sizeof(BSys), cudaMemcpyHostToDevice, b->st));
  B_CU(b, cudaStreamSynchronize(b->st));
  return TDKS_OK;
}

// Work lists of the nonlocal term over the systems whose descriptors carry projectors.
tdks_status build_kb_lists(tdks_batch* b) {
  std::vector<BKbItem> items;
  std::vector<BOrb> orbs;
  std::vector<BRow> rows;
  for (int s = 0; s < b->n_sys; ++s) {
    if (!b->h_full[s].kb) continue;
    int nblk = 0, nproj = 0;
    kb_view(b->ctx[s], nullptr, &nblk, &nproj);
    for (int o = 0; o < b->n_orb[s]; ++o) {
      orbs.push_back(BOrb{s, o});
      for (int p = 0; p < nproj; ++p) items.push_back(BKbItem{s, o, p, 0});
      for (int r = 0; r < nblk; ++r) rows.push_back(BRow{s, o, r, 0});
    }
  }
  auto put = [&](auto** dst, int* n, const auto& src) -> tdks_status {
    cudaFree(*dst);
    *dst = nullptr;
    *n = (int)src.size();
    if (src.empty()) return TDKS_OK;
    B_TRY(b, balloc(b, dst, src.size()), "nonlocal work lists");
    B_CU(b, cudaMemcpy(*dst, src.data(), src.size() * sizeof(src[0]), cudaMemcpyHostToDevice));
    return TDKS_OK;
  };
  B_TRY(b, put(&b->d_kb_items, &b->n_kb_items, items), "nonlocal work lists");
  B_TRY(b, put(&b->d_kb_orbs, &b->n_kb_orbs, orbs), "nonlocal work lists");
  B_TRY(b, put(&b->d_kb_rows, &b->n_kb_rows, rows), "nonlocal work lists");
  return TDKS_OK;
}

// (Re)build the work list of degree class d with elements-per-tile E and the
// current per-system orbital blocks.
tdks_status build_degree(tdks_batch* b, Deg& d, int E) {
  d.E = E;
  for (int s = 0; s < b->n_sys; ++s)
    if (b->ctx[s]->P1 == d.P1) b->n_eblk[s] = (int)((b->ctx[s]->n_elem + E - 1) / E);
  std::vector<BItem> items = make_items(b, d.P1, E, b->opb, nullptr);
  cudaFree(d.d_items);
  d.d_items = nullptr;
  B_TRY(b, balloc(b, &d.d_items, items.size()), "work list");
  B_CU(b, cudaMemcpy(d.d_items, items.data(), items.size() * sizeof(BItem), cudaMemcpyHostToDevice));
  d.n_items = (int)items.size();
  for (int k = 0; k < (b->prec == TDKS_MIXED ? 2 : 1); ++k) {
    const int pr = k == 0 ? apply_prec(b) : TDKS_FP32;
    int occ = 0;
    const cudaError_t ce = hbar_batch_occupancy(d.P1, pr, E, &occ);
    if (ce != cudaSuccess || occ < 1) {
      cudaGetLastError();
      return bfail(b, TDKS_ERR_CUDA, "occupancy query of the batched apply (p = " + std::to_string(d.P1 - 1) +
                                         ", E = " + std::to_string(E) + "): " + cudaGetErrorString(ce) +
                                         ", blocks/SM " + std::to_string(occ));
    }
    (k == 0 ? d.grid : d.grid32) = std::max(1, std::min(d.n_items, occ * b->n_sm));
  }
  return TDKS_OK;
}

// Capture of one pass of the batched exponential loop body (on the body stream).
tdks_status capture_body(tdks_batch* b, const BSys* sys, int* iter, cudaGraphConditionalHandle h) {
  cudaStream_t s = b->st_body;
  B_CU(b, launch_bkry_prepare(sys, b->d_orbs, b->n_gorb, b->d_rows, b->n_rows, s));
  B_CU(b, launch_bkb_project(sys, b->d_kb_items, b->n_kb_items, s));
  // the degree classes touch disjoint systems: concurrent branches, so that the
  // tail of one persistent grid overlaps the next
  const int nd = (int)b->degs.size();
  B_CU(b, cudaEventRecord(b->body_fork_ev, s));
  for (int i = 0; i < nd; ++i) {
    const Deg& d = b->degs[i];
    B_CU(b, cudaStreamWaitEvent(b->ds[i], b->body_fork_ev, 0));
    B_CU(b, apply_degree(b, i, sys, b->ds[i]));
    B_CU(b, cudaEventRecord(b->body_join_ev[i], b->ds[i]));
  }
  for (int i = 0; i < nd; ++i) B_CU(b, cudaStreamWaitEvent(s, b->body_join_ev[i], 0));
  B_CU(b, launch_balpha(sys, b->d_orbs, b->n_gorb, s));
  B_CU(b, launch_bkb_alpha(sys, b->d_kb_orbs, b->n_kb_orbs, s));
  // gather of each degree class on its branch (the kernel takes the degree as a constant)
  B_CU(b, cudaEventRecord(b->body_fork_ev, s));
  for (int i = 0; i < nd; ++i) {
    const Deg& d = b->degs[i];
    B_CU(b, cudaStreamWaitEvent(b->ds[i], b->body_fork_ev, 0));
    B_CU(b, launch_bassemble(d.P1, b->prec, sys, d.d_rows_asm, d.n_rows_asm, b->ds[i]));
    B_CU(b, cudaEventRecord(b->body_join_ev[i], b->ds[i]));
  }
  for (int i = 0; i < nd; ++i) B_CU(b, cudaStreamWaitEvent(s, b->body_join_ev[i], 0));
  B_CU(b, launch_bkb_add(sys, b->d_kb_rows, b->n_kb_rows, s));
  B_CU(b, launch_bkry_exp(sys, b->d_orbs, b->n_gorb, b->tol, b->theta, s));
  B_CU(b, launch_bkry_finish(sys, b->d_orbs, b->n_gorb, b->d_rows, b->n_rows, b->prec, s));
  B_CU(b, launch_bloop_control(h, sys, b->d_orbs, b->n_gorb, iter, kMaxSubPasses * b->kmax,
                               b->d_ctrl + 2, b->d_qctr, n_tickets(b), s));
  return TDKS_OK;
}

// Inside an active capture of b->st: append a WHILE node on handle h whose body is
// one pass of the batched exponential over `sys`.
tdks_status add_loop(tdks_batch* b, const BSys* sys, int* iter, cudaGraphConditionalHandle h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  B_CU(b, cudaStreamGetCaptureInfo(b->st, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return bfail(b, TDKS_ERR_CUDA, "stream is not capturing");
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  B_CU(b, cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  B_CU(b, cudaStreamUpdateCaptureDependencies(b->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  B_CU(b, cudaStreamBeginCaptureToGraph(b->st_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  tdks_status s = capture_body(b, sys, iter, h);
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->st_body, &out);
  if (s != TDKS_OK) return s;
  if (e != cudaSuccess) return bfail(b, TDKS_ERR_CUDA, std::string("loop body capture: ") + cudaGetErrorString(e));
  return TDKS_OK;
}

// Per-system field work on parallel capture branches: system field_order[k] runs on
// fork stream k % kFieldStreams (its context's stream is pointed there); the join
// returns every context to the batch stream.
tdks_status fork_fields(tdks_batch* b) {
  B_CU(b, cudaEventRecord(b->fork_ev, b->st));
  for (int i = 0; i < kFieldStreams; ++i) B_CU(b, cudaStreamWaitEvent(b->fs[i], b->fork_ev, 0));
  for (int k = 0; k < b->n_sys; ++k) b->ctx[b->field_order[k]]->stream = b->fs[k % kFieldStreams];
  return TDKS_OK;
}

tdks_status join_fields(tdks_batch* b) {
  for (int i = 0; i < kFieldStreams; ++i) {
    B_CU(b, cudaEventRecord(b->join_ev[i], b->fs[i]));
    B_CU(b, cudaStreamWaitEvent(b->st, b->join_ev[i], 0));
  }
  for (auto* c : b->ctx) c->stream = b->st;
  return TDKS_OK;
}

tdks_status capture_step(tdks_batch* b, cudaGraphConditionalHandle h1, cudaGraphConditionalHandle h2) {
  const double zero[3] = {0.0, 0.0, 0.0};
  int* err = b->d_ctrl + 2;
  auto mark = [&](int i) -> cudaError_t { return b->timing ? cudaEventRecordWithFlags(b->tev[i], b->st, cudaEventRecordExternal) : cudaSuccess; };
  B_CU(b, mark(0));
  // predictor potential V_N + 1.25 V_HXC^{n-1} - 0.25 V_HXC^{n-2} (no external field)
  for (int s = 0; s < b->n_sys; ++s) {
    tdks_ctx* c = b->ctx[s];
    B_TRY(b, ctx_try(b, c, launch_combine(c, c->d_vks, c->d_vnuc, 1.25, c->d_vhxc1, -0.25, c->d_vhxc2,
                                          nullptr, zero)), "predictor");
  }
  B_CU(b, mark(1));
  B_CU(b, launch_bkry_init(b->d_half, b->d_orbs, b->n_gorb, 0.5, b->st));
  B_CU(b, launch_bloop_begin(h1, b->d_ctrl + 0, b->d_qctr, n_tickets(b), b->st));
  B_TRY(b, add_loop(b, b->d_half, b->d_ctrl + 0, h1), "half step");
  B_CU(b, launch_bkry_stats(b->d_half, b->d_orbs, b->n_gorb, b->d_dof, b->d_ctrl + 4, b->d_sub, b->st));
  B_CU(b, mark(2));
  // corrector potential from the density of psi^{n-1/2}
  B_TRY(b, fork_fields(b), "fork");
  for (int s = 0; s < b->n_sys; ++s) {
    tdks_ctx* c = b->ctx[s];
    B_TRY(b, ctx_try(b, c, vhxc_graph(c, b->psi_half[s], b->n_orb[s], c->d_vtmp, b->cg_iters, err, field_prec(b))),
          "corrector");
    B_TRY(b, ctx_try(b, c, launch_combine(c, c->d_vks, c->d_vnuc, 1.0, c->d_vtmp, 0.0, nullptr, nullptr,
                                          zero)), "corrector");
  }
  B_TRY(b, join_fields(b), "join");
  B_CU(b, mark(3));
  B_CU(b, launch_bkry_init(b->d_full, b->d_orbs, b->n_gorb, 1.0, b->st));
  B_CU(b, launch_bloop_begin(h2, b->d_ctrl + 1, b->d_qctr, n_tickets(b), b->st));
  B_TRY(b, add_loop(b, b->d_full, b->d_ctrl + 1, h2), "full step");
  B_CU(b, launch_bkry_stats(b->d_full, b->d_orbs, b->n_gorb, b->d_dof, b->d_ctrl + 4, b->d_sub, b->st));
  B_CU(b, mark(4));
  // history and dipole of every system
  B_TRY(b, fork_fields(b), "fork");
  for (int s = 0; s < b->n_sys; ++s) {
    tdks_ctx* c = b->ctx[s];
    const size_t fb = (size_t)(c->n_elem * c->nq3) * sizeof(double);
    B_CU(b, cudaMemcpyAsync(c->d_vhxc2, c->d_vhxc1, fb, cudaMemcpyDeviceToDevice, c->stream));
    B_TRY(b, ctx_try(b, c, vhxc_graph(c, b->psi[s], b->n_orb[s], c->d_vhxc1, b->cg_iters, err, field_prec(b))), "history");
    B_TRY(b, ctx_try(b, c, dipole_graph(c, c->d_rho, b->d_dip + 3 * (size_t)s, b->d_ctrl + 3,
                                        3 * (int64_t)b->n_sys)), "dipole");
  }
  B_TRY(b, join_fields(b), "join");
  B_CU(b, launch_counter_add(b->d_ctrl + 3, 1, b->st));
  B_CU(b, mark(5));
  return TDKS_OK;
}

tdks_status build_graph(tdks_batch* b) {
  invalidate_graph(b);
  B_CU(b, cudaGraphCreate(&b->graph, 0));
  cudaGraphConditionalHandle h1, h2;
  // default 0: a loop runs only after its begin kernel set the condition to 1
  B_CU(b, cudaGraphConditionalHandleCreate(&h1, b->graph, 0, cudaGraphCondAssignDefault));
  B_CU(b, cudaGraphConditionalHandleCreate(&h2, b->graph, 0, cudaGraphCondAssignDefault));
  B_CU(b, cudaStreamBeginCaptureToGraph(b->st, b->graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  tdks_status s = capture_step(b, h1, h2);
  for (auto* c : b->ctx) c->stream = b->st;
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->st, &out);
  if (s != TDKS_OK) {
    invalidate_graph(b);
    return s;
  }
  if (e != cudaSuccess) {
    invalidate_graph(b);
    return bfail(b, TDKS_ERR_CUDA, std::string("step capture: ") + cudaGetErrorString(e));
  }
  B_CU(b, cudaGraphInstantiate(&b->exec, b->graph, 0));
  return TDKS_OK;
}

// time `reps` launches of one degree class's apply with the given work list
tdks_status time_apply(tdks_batch* b, const Deg& d, const std::vector<BItem>& items, int E, int reps,
                       double* ms) {
  BItem* di = nullptr;
  B_TRY(b, balloc(b, &di, items.size()), "tuning");
  cudaMemcpy(di, items.data(), items.size() * sizeof(BItem), cudaMemcpyHostToDevice);
  int occ = 0;
  hbar_batch_occupancy(d.P1, apply_prec(b), E, &occ);
  const int grid = std::max(1, std::min((int)items.size(), std::max(occ, 1) * b->n_sm));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int* q = b->d_qctr;
  cudaMemsetAsync(q, 0, sizeof(int) * (reps + 1), b->st);
  cudaError_t ce = launch_hbar_batch(d.P1, apply_prec(b), b->d_full, di, (int)items.size(), E, grid, d.tab, q, b->st);
  cudaEventRecord(e0, b->st);
  for (int r = 0; r < reps && ce == cudaSuccess; ++r)
    ce = launch_hbar_batch(d.P1, apply_prec(b), b->d_full, di, (int)items.size(), E, grid, d.tab, q + 1 + r, b->st);
  cudaEventRecord(e1, b->st);
  cudaError_t se = cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(di);
  if (ce != cudaSuccess || se != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, TDKS_ERR_CUDA, std::string("tuning launch: ") + cudaGetErrorString(ce != cudaSuccess ? ce : se));
  }
  *ms = t / std::max(reps, 1);
  return TDKS_OK;
}

}  // namespace

extern "C" {

tdks_status tdks_batch_create(int n_sys, const tdks_mesh_desc* meshes, const tdks_system_desc* systems,
                              const double* dt, int prec, double tol, int k_max, tdks_batch** out) {
  if (!out) return TDKS_ERR_ARG;
  *out = nullptr;
  if (n_sys < 1 || !meshes || !systems || !dt) return TDKS_ERR_ARG;
  if (prec != TDKS_FP64 && prec != TDKS_FP32 && prec != TDKS_DF64 && prec != TDKS_MIXED) return TDKS_ERR_ARG;
  if (k_max < 2 || k_max > TDKS_KMAX || !(tol > 0)) return TDKS_ERR_ARG;
  tdks_batch* b = new tdks_batch();
  b->n_sys = n_sys;
  b->prec = prec;
  b->tol = tol;
  b->kmax = k_max;
  auto fail = [&](tdks_status s) {
    // the batch is freed: its message moves to the global slot (tdks_batch_last_error(NULL))
    g_create_err = b->err.empty() ? std::string(tdks_status_string(s)) : b->err;
    free_batch(b);
    return s;
  };
  if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->st_body, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    b->err = "stream creation";
    return fail(TDKS_ERR_CUDA);
  }
  for (int i = 0; i < kFieldStreams; ++i)
    if (cudaStreamCreateWithFlags(&b->fs[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join_ev[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      b->err = "stream creation";
      return fail(TDKS_ERR_CUDA);
    }
  for (int i = 0; i < kDegStreams; ++i)
    if (cudaStreamCreateWithFlags(&b->ds[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->body_join_ev[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      b->err = "stream creation";
      return fail(TDKS_ERR_CUDA);
    }
  if (cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->body_fork_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    b->err = "event creation";
    return fail(TDKS_ERR_CUDA);
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev);
  b->ctx.assign(n_sys, nullptr);
  for (int s = 0; s < n_sys; ++s) {
    if (!(dt[s] > 0)) {
      b->err = "system " + std::to_string(s) + ": dt must be > 0";
      return fail(TDKS_ERR_ARG);
    }
    tdks_status st = tdks_create(&meshes[s], &systems[s], (void*)b->st, &b->ctx[s]);
    if (st != TDKS_OK) {
      b->err = "system " + std::to_string(s) + ": tdks_create failed";
      return fail(st);
    }
    tdks_ctx* c = b->ctx[s];
    if (!c->fdm_ok) {   // the in-graph Poisson CG needs the exact preconditioner
      b->err = "system " + std::to_string(s) + ": an axis has more than 1024 interior nodes";
      return fail(TDKS_ERR_ARG);
    }
  }
  b->n_orb.resize(n_sys);
  b->n_eblk.resize(n_sys);
  b->n_rblk.resize(n_sys);
  b->opb.assign(n_sys, 1);
  b->dt.assign(dt, dt + n_sys);
  b->psi.assign(n_sys, nullptr);
  b->psi_half.assign(n_sys, nullptr);
  b->Vw.assign(n_sys, nullptr);
  b->kry.assign(n_sys, nullptr);
  b->ev.assign(n_sys, nullptr);
  b->apart.assign(n_sys, nullptr);
  b->npart.assign(n_sys, nullptr);
  b->h_half.resize(n_sys);
  b->h_full.resize(n_sys);
  std::vector<BOrb> orbs;
  std::vector<BRow> rows;
  std::map<int, int> deg_index;
  for (int s = 0; s < n_sys; ++s) {
    tdks_ctx* c = b->ctx[s];
    const int no = c->n_orb;
    b->n_orb[s] = no;
    const size_t nv = (size_t)no * c->n_int;
    const int nrows = c->Ni[1] * c->Ni[2];
    b->n_rblk[s] = (int)std::max<long long>(1, std::min<long long>(nrows, (c->n_int + 4095) / 4096));
    b->n_eblk[s] = (int)((c->n_elem + emax_of(c->P1) - 1) / emax_of(c->P1));
    if (balloc(b, &b->psi[s], nv) || balloc(b, &b->psi_half[s], nv) ||
        balloc(b, &b->Vw[s], nv * k_max) || balloc(b, &b->kry[s], (size_t)no) ||
        balloc(b, (double2**)&b->ev[s], (size_t)no * c->n_elem * c->P1 * c->P1 * c->P1) ||
        balloc(b, &b->apart[s], (size_t)no * c->n_elem) || balloc(b, &b->npart[s], (size_t)no * b->n_rblk[s]))
      return fail(TDKS_ERR_NOMEM);
    cudaMemset(b->psi[s], 0, nv * sizeof(double2));
    BSys S;
    std::memset(&S, 0, sizeof(S));
    S.g = tdks_geom(c);
    S.P1 = c->P1;
    S.n_orb = no;
    S.kmax = k_max;
    S.n_eblk = b->n_eblk[s];
    S.n_rblk = b->n_rblk[s];
    S.n_int = c->n_int;
    S.n_elem = c->n_elem;
    S.in = b->psi[s];
    S.vks = c->d_vks;
    S.Vw = b->Vw[s];
    S.kry = b->kry[s];
    S.ev = b->ev[s];
    S.apart = b->apart[s];
    S.npart = b->npart[s];
    S.dt = dt[s];
    S.mixed = prec == TDKS_MIXED ? 1 : 0;
    if (prec == TDKS_MIXED) b->theta = c->mixed_relax * tol;   // the context default, 1e8 x tol
    b->h_half[s] = S;
    b->h_half[s].out = b->psi_half[s];
    b->h_full[s] = S;
    b->h_full[s].out = b->psi[s];
    for (int o = 0; o < no; ++o) {
      orbs.push_back(BOrb{s, o});
      for (int r = 0; r < b->n_rblk[s]; ++r) rows.push_back(BRow{s, o, r, 0});
    }
    if (!deg_index.count(c->P1)) {
      deg_index[c->P1] = (int)b->degs.size();
      Deg d;
      d.P1 = c->P1;
      d.tab = prec == TDKS_FP32 ? (const void*)c->d_tabf
              : (prec == TDKS_DF64 || prec == TDKS_MIXED) ? (const void*)c->d_tabdf
                                                          : (const void*)c->d_tab;
      d.tab32 = c->d_tabf;
      b->degs.push_back(d);
    }
  }
  b->field_order.resize(n_sys);
  for (int s = 0; s < n_sys; ++s) b->field_order[s] = s;
  std::stable_sort(b->field_order.begin(), b->field_order.end(), [&](int x, int y) {
    return b->ctx[x]->n_int * b->n_orb[x] > b->ctx[y]->n_int * b->n_orb[y];
  });
  b->n_gorb = (int)orbs.size();
  b->n_rows = (int)rows.size();
  if (balloc(b, &b->d_half, n_sys) || balloc(b, &b->d_full, n_sys) || balloc(b, &b->d_orbs, orbs.size()) ||
      balloc(b, &b->d_rows, rows.size()) ||
      balloc(b, &b->d_ctrl, 8) || balloc(b, &b->d_qctr, 64) || balloc(b, &b->d_dof, 1) ||
      balloc(b, &b->d_sub, 2 * (size_t)n_sys) ||
      balloc(b, &b->d_dip, (size_t)b->dip_cap * n_sys * 3))
    return fail(TDKS_ERR_NOMEM);
  // assembly items: larger systems first, so their many row blocks start early
  std::vector<BRow> rows_asm = rows;
  std::stable_sort(rows_asm.begin(), rows_asm.end(), [&](const BRow& x, const BRow& y) {
    return b->ctx[x.sys]->n_int / b->n_rblk[x.sys] > b->ctx[y.sys]->n_int / b->n_rblk[y.sys];
  });
  cudaMemcpy(b->d_orbs, orbs.data(), orbs.size() * sizeof(BOrb), cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_rows, rows.data(), rows.size() * sizeof(BRow), cudaMemcpyHostToDevice);
  for (Deg& d : b->degs) {
    std::vector<BRow> dr;
    for (const BRow& r : rows_asm)
      if (b->ctx[r.sys]->P1 == d.P1) dr.push_back(r);
    d.n_rows_asm = (int)dr.size();
    if (balloc(b, &d.d_rows_asm, dr.size())) return fail(TDKS_ERR_NOMEM);
    cudaMemcpy(d.d_rows_asm, dr.data(), dr.size() * sizeof(BRow), cudaMemcpyHostToDevice);
  }
  cudaMemset(b->d_ctrl, 0, 8 * sizeof(int));
  cudaMemset(b->d_qctr, 0, 64 * sizeof(int));
  cudaMemset(b->d_dof, 0, sizeof(unsigned long long));
  cudaMemset(b->d_sub, 0, 2 * n_sys * sizeof(unsigned long long));
  for (Deg& d : b->degs)
    if (build_degree(b, d, emax_of(d.P1)) != TDKS_OK) return fail(TDKS_ERR_CUDA);
  if (upload_descriptors(b) != TDKS_OK) return fail(TDKS_ERR_CUDA);
  const cudaError_t se = cudaDeviceSynchronize();
  if (se != cudaSuccess) {
    cudaGetLastError();
    b->err = std::string("setup: ") + cudaGetErrorString(se);
    return fail(TDKS_ERR_CUDA);
  }
  *out = b;
  return TDKS_OK;
}

tdks_status tdks_batch_destroy(tdks_batch* b) {
  if (!b) return TDKS_ERR_ARG;
  cudaStreamSynchronize(b->st);
  free_batch(b);
  return TDKS_OK;
}

void* tdks_batch_stream(tdks_batch* b) { return b ? (void*)b->st : nullptr; }

const char* tdks_batch_last_error(const tdks_batch* b) { return b ? b->err.c_str() : g_create_err.c_str(); }

tdks_status tdks_batch_sizes(const tdks_batch* b, int sys, int64_t* n_int, int64_t* n_elem, int* nq3,
                             int* n_orb) {
  if (!b || sys < 0 || sys >= b->n_sys) return TDKS_ERR_ARG;
  const tdks_ctx* c = b->ctx[sys];
  if (n_int) *n_int = c->n_int;
  if (n_elem) *n_elem = c->n_elem;
  if (nq3) *nq3 = (int)c->nq3;
  if (n_orb) *n_orb = c->n_orb;
  return TDKS_OK;
}

tdks_status tdks_batch_set_orbitals(tdks_batch* b, int sys, const double* psi_dev) {
  if (!b || !psi_dev || sys < 0 || sys >= b->n_sys) return TDKS_ERR_ARG;
  const size_t vb = (size_t)b->n_orb[sys] * b->ctx[sys]->n_int * sizeof(double2);
  B_CU(b, cudaMemcpyAsync(b->psi[sys], psi_dev, vb, cudaMemcpyDeviceToDevice, b->st));
  B_CU(b, cudaStreamSynchronize(b->st));
  b->ready = false;
  return TDKS_OK;
}

tdks_status tdks_batch_get_orbitals(tdks_batch* b, int sys, double* psi_dev) {
  if (!b || !psi_dev || sys < 0 || sys >= b->n_sys) return TDKS_ERR_ARG;
  const size_t vb = (size_t)b->n_orb[sys] * b->ctx[sys]->n_int * sizeof(double2);
  B_CU(b, cudaMemcpyAsync(psi_dev, b->psi[sys], vb, cudaMemcpyDeviceToDevice, b->st));
  B_CU(b, cudaStreamSynchronize(b->st));
  return TDKS_OK;
}

tdks_status tdks_batch_kick(tdks_batch* b, const double* kappa, const double* dir) {
  if (!b || !kappa || !dir) return TDKS_ERR_ARG;
  for (int s = 0; s < b->n_sys; ++s)
    B_TRY(b, ctx_try(b, b->ctx[s], launch_kick(b->ctx[s], b->psi[s], b->n_orb[s], kappa[s], dir + 3 * s)),
          "kick");
  B_CU(b, cudaStreamSynchronize(b->st));
  return TDKS_OK;
}

tdks_status tdks_batch_init(tdks_batch* b, double* dip_host) {
  if (!b) return TDKS_ERR_ARG;
  for (int s = 0; s < b->n_sys; ++s) {
    double d[3];
    B_TRY(b, ctx_try(b, b->ctx[s], tdks_init_propagation(b->ctx[s], (const double*)b->psi[s], b->n_orb[s], d)),
          "init");
    if (dip_host) std::memcpy(dip_host + 3 * s, d, sizeof(d));
  }
  b->orbitals_set = true;
  return TDKS_OK;
}

tdks_status tdks_batch_tune(tdks_batch* b, int reps, tdks_tile_choice* out, int cap, int* n_out) {
  if (!b || reps < 1 || reps > 32) return TDKS_ERR_ARG;
  if (!b->orbitals_set) return bfail(b, TDKS_ERR_ARG, "tune after tdks_batch_init (needs the orbitals)");
  invalidate_graph(b);
  // every orbital active at j = 0: the apply reads the orbitals themselves
  B_CU(b, launch_bkry_init(b->d_full, b->d_orbs, b->n_gorb, 1.0, b->st));
  B_CU(b, launch_bkry_prepare(b->d_full, b->d_orbs, b->n_gorb, b->d_rows, b->n_rows, b->st));
  b->tiles.clear();
  for (Deg& d : b->degs) {
    // classes of this degree by orbital count
    std::map<int, std::vector<int>> cls;
    for (int s = 0; s < b->n_sys; ++s)
      if (b->ctx[s]->P1 == d.P1) cls[b->n_orb[s]].push_back(s);
    // 1. elements per tile, one orbital per item
    const int em = emax_of(d.P1);
    std::vector<int> Es = {em, em - 1, (em + 1) / 2};
    std::sort(Es.begin(), Es.end());
    Es.erase(std::unique(Es.begin(), Es.end()), Es.end());
    std::vector<int> one(b->n_sys, 1);
    int bestE = em;
    double bestT = 1e300;
    for (int E : Es) {
      if (E < 1) continue;
      std::vector<BItem> items = make_items(b, d.P1, E, one, nullptr);
      for (int s = 0; s < b->n_sys; ++s)
        if (b->ctx[s]->P1 == d.P1) b->n_eblk[s] = (int)((b->ctx[s]->n_elem + E - 1) / E);
      B_TRY(b, upload_descriptors(b), "tuning");
      double t = 0;
      B_TRY(b, time_apply(b, d, items, E, reps, &t), "tuning");
      if (t < bestT) {
        bestT = t;
        bestE = E;
      }
    }
    for (int s = 0; s < b->n_sys; ++s)
      if (b->ctx[s]->P1 == d.P1) b->n_eblk[s] = (int)((b->ctx[s]->n_elem + bestE - 1) / bestE);
    B_TRY(b, upload_descriptors(b), "tuning");
    // 2. orbitals per item for each orbital-count class
    for (auto& kv : cls) {
      const int no = kv.first;
      int bestB = 1;
      double bT = 1e300;
      for (int ob : {1, 2, 4, 8}) {
        if (ob > no) break;
        std::vector<int> opb(b->n_sys, ob);
        std::vector<BItem> items = make_items(b, d.P1, bestE, opb, &kv.second);
        double t = 0;
        B_TRY(b, time_apply(b, d, items, bestE, reps, &t), "tuning");
        if (t < bT) {
          bT = t;
          bestB = ob;
        }
      }
      for (int s : kv.second) b->opb[s] = bestB;
      b->tiles.push_back(tdks_tile_choice{d.P1 - 1, no, bestE, bestB, bT});
    }
    B_TRY(b, build_degree(b, d, bestE), "tuning");
  }
  B_TRY(b, upload_descriptors(b), "tuning");
  if (out && n_out) {
    const int n = std::min<int>(cap, (int)b->tiles.size());
    for (int i = 0; i < n; ++i) out[i] = b->tiles[i];
    *n_out = n;
  } else if (n_out) {
    *n_out = (int)b->tiles.size();
  }
  return TDKS_OK;
}

tdks_status tdks_batch_set_kb(tdks_batch* b, int sys, int n_atoms, const double* R, double a, double bb,
                              const double c[2], int lmax) {
  if (!b || sys < 0 || sys >= b->n_sys) return TDKS_ERR_ARG;
  tdks_ctx* cx = b->ctx[sys];
  B_CU(b, cudaStreamSynchronize(b->st));
  B_TRY(b, ctx_try(b, cx, tdks_set_kb(cx, n_atoms, R, a, bb, c, lmax)), "tdks_set_kb");
  double* part = nullptr;
  int nblk = 0;
  const KbView* v = kb_view(cx, &part, &nblk, nullptr);
  if (cx->kb && !v) return bfail(b, TDKS_ERR_NOMEM, "projector view");
  for (BSys* S : {&b->h_half[sys], &b->h_full[sys]}) {
    S->kb = v;
    S->kb_part = v ? part : nullptr;
    S->kb_nblk = v ? nblk : 0;
  }
  invalidate_graph(b);
  B_TRY(b, build_kb_lists(b), "projectors");
  B_TRY(b, upload_descriptors(b), "projectors");
  return TDKS_OK;
}

tdks_status tdks_batch_tune_kmax(tdks_batch* b, int k_cap, int64_t mem_budget, int* kmax_out) {
  if (!b || k_cap < 2 || k_cap > TDKS_KMAX) return TDKS_ERR_ARG;
  // per system, over its exponentials since creation or since its cap was last
  // raised: the largest sub-step count and the Hbar applications
  std::vector<unsigned long long> sub(2 * (size_t)b->n_sys);
  B_CU(b, cudaStreamSynchronize(b->st));
  B_CU(b, cudaMemcpy(sub.data(), b->d_sub, sub.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  bool stepped = false;
  for (int s = 0; s < b->n_sys; ++s) stepped = stepped || sub[2 * s + 1] > 0;
  if (!stepped) return bfail(b, TDKS_ERR_ARG, "run a step first (the caps follow its sub-steps)");
  // systems whose exponentials restarted at their cap, by Hbar work
  std::vector<std::pair<double, int>> cand;
  for (int s = 0; s < b->n_sys; ++s) {
    if (b->h_full[s].kmax >= k_cap || sub[2 * s] <= 1) continue;
    const double P1 = b->ctx[s]->P1;
    cand.emplace_back((double)sub[2 * s + 1] * (double)b->ctx[s]->n_elem * P1 * P1 * P1 * P1, s);
  }
  std::stable_sort(cand.begin(), cand.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
    return x.first > y.first;
  });
  if (mem_budget < 0) {
    size_t fr = 0, tot = 0;
    B_CU(b, cudaMemGetInfo(&fr, &tot));
    mem_budget = (int64_t)(fr / 2);
  }
  for (const auto& cs : cand) {
    const int s = cs.second;
    const size_t nv = (size_t)b->n_orb[s] * b->ctx[s]->n_int;
    const int64_t add = (int64_t)(nv * (size_t)(k_cap - b->h_full[s].kmax) * sizeof(double2));
    if (add > mem_budget) continue;
    double2* nw = nullptr;
    if (cudaMalloc((void**)&nw, nv * (size_t)k_cap * sizeof(double2)) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    invalidate_graph(b);
    cudaFree(b->Vw[s]);
    b->Vw[s] = nw;
    for (BSys* S : {&b->h_half[s], &b->h_full[s]}) {
      S->Vw = nw;
      S->kmax = k_cap;
    }
    B_CU(b, cudaMemset(b->d_sub + 2 * s, 0, 2 * sizeof(unsigned long long)));   // statistics of the new cap
    mem_budget -= add;
  }
  b->kmax = 0;
  for (int s = 0; s < b->n_sys; ++s) b->kmax = std::max(b->kmax, b->h_full[s].kmax);
  B_TRY(b, upload_descriptors(b), "Krylov caps");
  if (kmax_out)
    for (int s = 0; s < b->n_sys; ++s) kmax_out[s] = b->h_full[s].kmax;
  return TDKS_OK;
}

tdks_status tdks_batch_steps(tdks_batch* b, int n_steps, double* dip_host) {
  if (!b || n_steps < 0) return TDKS_ERR_ARG;
  if (!b->orbitals_set) return bfail(b, TDKS_ERR_ARG, "call tdks_batch_init first");
  if (!b->exec) B_TRY(b, build_graph(b), "graph");
  std::vector<double> buf;
  int done = 0;
  while (done < n_steps) {
    const int chunk = std::min(b->dip_cap, n_steps - done);
    B_CU(b, cudaMemsetAsync(b->d_ctrl + 3, 0, sizeof(int), b->st));
    for (int k = 0; k < chunk; ++k) B_CU(b, cudaGraphLaunch(b->exec, b->st));
    int ctrl[8];
    B_CU(b, cudaMemcpyAsync(ctrl, b->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost, b->st));
    if (dip_host) {
      buf.resize((size_t)chunk * b->n_sys * 3);
      B_CU(b, cudaMemcpyAsync(buf.data(), b->d_dip, buf.size() * sizeof(double), cudaMemcpyDeviceToHost, b->st));
    }
    B_CU(b, cudaStreamSynchronize(b->st));
    if (ctrl[2]) {
      std::string m = "batched step failed:";
      if (ctrl[2] & 1) m += " Lanczos failure (sub-step cap or non-finite);";
      if (ctrl[2] & 2) m += " exponential loop reached its pass cap;";
      if (ctrl[2] & 4) m += " Poisson CG not converged in the fixed iteration count;";
      if (ctrl[2] & 8) m += " non-finite Poisson residual;";
      return bfail(b, TDKS_ERR_NOT_CONVERGED, m);
    }
    if (dip_host) std::memcpy(dip_host + (size_t)done * b->n_sys * 3, buf.data(), buf.size() * sizeof(double));
    done += chunk;
  }
  return TDKS_OK;
}

tdks_status tdks_batch_set_timing(tdks_batch* b, int on) {
  if (!b) return TDKS_ERR_ARG;
  if ((bool)on == b->timing) return TDKS_OK;
  for (auto& e : b->tev)
    if (!e) B_CU(b, cudaEventCreate(&e));
  b->timing = on != 0;
  invalidate_graph(b);
  return TDKS_OK;
}

tdks_status tdks_batch_phase_ms(tdks_batch* b, double ms[5], int passes[2]) {
  if (!b || !ms) return TDKS_ERR_ARG;
  if (!b->timing || !b->exec) return bfail(b, TDKS_ERR_ARG, "enable timing and run a step first");
  B_CU(b, cudaStreamSynchronize(b->st));
  for (int i = 0; i < 5; ++i) {
    float t = 0.f;
    B_CU(b, cudaEventElapsedTime(&t, b->tev[i], b->tev[i + 1]));
    ms[i] = t;
  }
  if (passes) B_CU(b, cudaMemcpy(passes, b->d_ctrl, 2 * sizeof(int), cudaMemcpyDeviceToHost));
  return TDKS_OK;
}

// Diagnostics: the half-step exponential of the current state run once more outside
// the graph, kernel group by kernel group, with the pass count of the last step's
// half-step loop; ms = device time of [norms/start, apply, alpha, assembly,
// small exponentials, recombination].  Writes only the scratch output psi_half.
tdks_status tdks_batch_profile_pass(tdks_batch* b, double ms[6]) {
  if (!b || !ms) return TDKS_ERR_ARG;
  int ctrl[8];
  B_CU(b, cudaMemcpy(ctrl, b->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost));
  const int passes = ctrl[0];
  if (passes < 1) return bfail(b, TDKS_ERR_ARG, "run a step first");
  cudaEvent_t ev[7];
  for (auto& e : ev) B_CU(b, cudaEventCreate(&e));
  for (int i = 0; i < 6; ++i) ms[i] = 0.0;
  const BSys* sys = b->d_half;
  B_CU(b, launch_bkry_init(sys, b->d_orbs, b->n_gorb, 0.5, b->st));
  for (int it = 0; it < passes; ++it) {
    B_CU(b, cudaMemsetAsync(b->d_qctr, 0, 64 * sizeof(int), b->st));
    B_CU(b, cudaEventRecord(ev[0], b->st));
    B_CU(b, launch_bkry_prepare(sys, b->d_orbs, b->n_gorb, b->d_rows, b->n_rows, b->st));
    B_CU(b, cudaEventRecord(ev[1], b->st));
    B_CU(b, launch_bkb_project(sys, b->d_kb_items, b->n_kb_items, b->st));
    for (size_t i = 0; i < b->degs.size(); ++i) B_CU(b, apply_degree(b, (int)i, sys, b->st));
    B_CU(b, cudaEventRecord(ev[2], b->st));
    B_CU(b, launch_balpha(sys, b->d_orbs, b->n_gorb, b->st));
    B_CU(b, launch_bkb_alpha(sys, b->d_kb_orbs, b->n_kb_orbs, b->st));
    B_CU(b, cudaEventRecord(ev[3], b->st));
    for (const Deg& d : b->degs)
      B_CU(b, launch_bassemble(d.P1, b->prec, sys, d.d_rows_asm, d.n_rows_asm, b->st));
    B_CU(b, launch_bkb_add(sys, b->d_kb_rows, b->n_kb_rows, b->st));
    B_CU(b, cudaEventRecord(ev[4], b->st));
    B_CU(b, launch_bkry_exp(sys, b->d_orbs, b->n_gorb, b->tol, b->theta, b->st));
    B_CU(b, cudaEventRecord(ev[5], b->st));
    B_CU(b, launch_bkry_finish(sys, b->d_orbs, b->n_gorb, b->d_rows, b->n_rows, b->prec, b->st));
    B_CU(b, cudaEventRecord(ev[6], b->st));
    B_CU(b, cudaEventSynchronize(ev[6]));
    for (int i = 0; i < 6; ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      ms[i] += t;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return TDKS_OK;
}

tdks_status tdks_batch_stats(tdks_batch* b, int64_t* dof_applies, int* k_max_seen, int reset) {
  if (!b) return TDKS_ERR_ARG;
  unsigned long long dof = 0;
  int ctrl[8];
  B_CU(b, cudaMemcpyAsync(&dof, b->d_dof, sizeof(dof), cudaMemcpyDeviceToHost, b->st));
  B_CU(b, cudaMemcpyAsync(ctrl, b->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost, b->st));
  B_CU(b, cudaStreamSynchronize(b->st));
  if (dof_applies) *dof_applies = (int64_t)dof;
  if (k_max_seen) *k_max_seen = ctrl[4];
  if (reset) {
    B_CU(b, cudaMemsetAsync(b->d_dof, 0, sizeof(unsigned long long), b->st));
    B_CU(b, cudaMemsetAsync(b->d_ctrl + 4, 0, sizeof(int), b->st));
    B_CU(b, cudaStreamSynchronize(b->st));
  }
  return TDKS_OK;
}

}  // extern "C"
