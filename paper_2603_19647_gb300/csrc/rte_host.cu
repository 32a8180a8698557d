// Host driver and C ABI of librte.so.
//
// The host side only sequences device work: it builds the angular rule and the direction
// layout, owns the device buffers, and runs the control flow of Algorithm 1 (SI-SA) and
// Algorithm 2 (on-the-fly ROM phases) of Liu & Peng.  Every arithmetic step on a cell
// vector or on the angular flux is a CUDA kernel (sweep.cu, vec.cu, cg.cu, rom.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "rte_internal.h"

namespace rte {
thread_local long long g_launches = 0;
}

using namespace rte;

struct rte_s {
  std::string err;
  int device = 0;
  cudaStream_t st = nullptr, own_st = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, kev0 = nullptr, kev1 = nullptr;
  // event pool and recorded spans of the device-time statistics
  std::vector<cudaEvent_t> evpool;
  int evnext = 0;
  struct Span {
    int kind, a, b, iter;   // iter > 0: work of SI iteration iter, dropped if it never ran
  };
  std::vector<Span> spans;
  // options.graph: SI iteration l (DSA of l, sweep and residual of l + 1) as a CUDA graph,
  // indexed by l, with the kernels each replay launches
  struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
  };
  std::vector<IterGraph> graphs;
  // options.graph = 2: the remaining SI iterations from iteration l on as one graph with a
  // while node, indexed by l (kernels: of one pass of the loop body)
  std::vector<IterGraph> loops;
  unsigned* d_loop = nullptr;             // the loop's iteration counter
  unsigned* h_loop = nullptr;             // pinned copy
  bool capturing = false;                 // no timing events while a graph is captured
  unsigned* d_conv = nullptr;             // skip word of the speculative SI-SA loop
  unsigned* res_ticket = nullptr;         // arrival counter of the fused residual + norms kernel
  const unsigned* skip_now = nullptr;     // skip word the sweep helpers pass on (or none)
  cudaEvent_t ev_norm[2] = {nullptr, nullptr};     // spin-wait
  cudaEvent_t ev_norm_b[2] = {nullptr, nullptr};   // blocking-sync (batched instances)
  // second stream: the ROM update overlaps the fused f sweep
  cudaStream_t st2 = nullptr, st3 = nullptr;   // st3: the PC-ROM's part of the update
  cudaEvent_t ev_rho = nullptr, ev_r0 = nullptr, ev_r1 = nullptr, ev_gate = nullptr,
              ev_pc = nullptr;
  Norms* h_norms = nullptr;   // pinned
  int* h_cg = nullptr;        // pinned, CG counts of one SI-SA solve
  int cg_slots = 0;
  bool blocking = false;             // wait on ev_wait (sleeping) instead of spinning
  bool dsa_f32 = false;              // the DSA solve in FP32 (FP32 modes, single handles)
  cudaEvent_t ev_wait = nullptr;     // blocking-sync event
  unsigned* h_err = nullptr;         // pinned copy of the sweeps' error word
  // ROM update queued on the device, finished on the host after the step's last wait
  struct RomPending {
    bool queued = false, ig = false, ig_building = false, ig_err = false;
    bool pc[RTE_MAX_PC_LEVELS] = {}, pc_building[RTE_MAX_PC_LEVELS] = {},
         pc_err[RTE_MAX_PC_LEVELS] = {};
  } rom_pend;
  double* rom_dv = nullptr;        // [2 + levels] device scalars of the indicators
  double* h_rom_dv = nullptr;      // pinned copy
  int* rom_gate = nullptr;         // [1 + levels] device gates (IG, PC of each iteration)
  double* rom_partials = nullptr;  // dot partials of the ROM streams, [1 + levels][3 * 1024]
  // problem
  int dim = 2, nx = 0, ny = 0;
  long ncell = 0;
  // DG degree (options.degree): nb unknowns per cell and direction (Q0: 1, Q1: 4), ndof =
  // nb ncell per direction and in every rho-like vector (mode-major for Q1)
  int deg = 0, nb = 1;
  long ndof = 0;
  double hx = 1, hy = 1, c_dt = 1, tau = 1;
  rte_options opt{};
  std::vector<double> mu_user, eta_user, w_user;  // library direction order
  Layout L;
  // 2D sweep tiles: [0] for the SI sweep and the y sweep, [1] for the fused f sweep
  struct Tile {
    int kind = 1;   // 1: strip chain (sweep.cu, R rows per lane group), 2: tile sequence
                    // (sweep_tile.cu, FP32 modes, R = TH rows per lane group), 3: Q1 strip
                    // chain (sweep_q1.cu, one warp per CTA)
    int R = 1, W = 8, rpb = 32, nblk = 1;
  } tile[2];
  int nblk_max = 1;   // edge buffers and control flags are sized for the larger tile count
  bool tuned = false;
  // device: problem data
  double *sig_t = nullptr, *sig_s = nullptr, *src = nullptr;
  double *ca = nullptr, *cb = nullptr, *cw = nullptr;
  int *fam_quad = nullptr, *dir_sign = nullptr;
  double* inv_d = nullptr;
  // device: angular flux and sweep scratch
  double* f = nullptr;
  double *pm = nullptr, *pm_a = nullptr, *edge = nullptr;
  SweepCtrl* ctrl = nullptr;
  double *psi_w = nullptr, *psi_w_a = nullptr;
  // FP32 mode (RTE_FP32): sweep data in float; FP64 refinement state
  bool fp32 = false;
  bool bf16 = false;     // RTE_FP32_BF16F: f stored as BF16 remainders about fref[fcur]
  __nv_bfloat16 *fb = nullptr, *fb_init = nullptr;
  float* fref[2] = {nullptr, nullptr};
  float* fref_init = nullptr;
  int fcur = 0;
  unsigned bf_seed = 0;  // counter of BF16 write launches (stochastic-rounding seed)
  float *sig_t_f = nullptr, *src_f = nullptr, *ca_f = nullptr, *cb_f = nullptr, *cw_f = nullptr;
  float *f_f = nullptr, *pm_f = nullptr, *edge_f = nullptr, *psi_w_f = nullptr, *q_f = nullptr;
  float *cth_f = nullptr, *ctl_f = nullptr;   // tau + a + b per slot as an exact hi / lo pair
  float* sig_tl_f = nullptr;                   // sigma_t - sig_t_f (low part of the pair)
  float *f_init_f = nullptr;
  double *y_ir = nullptr, *rho_ref = nullptr;   // y_ir = T Sigma_s rho_ref, accumulated in FP64
  // device: cell vectors
  double *rho = nullptr, *rho_prev = nullptr, *rho_half = nullptr, *rho_half1 = nullptr;
  // preconditioner ROMs of iterations l = 2 .. pc_levels (index l - 1; l = 1 uses rho_half1,
  // rho0, delta_pc1, tmp2, tmp3 and delta): rho^{n,(l-1/2)}, rho^{n,(l-1)}, the ROM correction,
  // the snapshot pair and the indicator's difference
  double* lv_half[RTE_MAX_PC_LEVELS] = {};
  double* lv_prev[RTE_MAX_PC_LEVELS] = {};
  double* lv_delta[RTE_MAX_PC_LEVELS] = {};
  double* lv_x[RTE_MAX_PC_LEVELS] = {};
  double* lv_b[RTE_MAX_PC_LEVELS] = {};
  double* lv_diff[RTE_MAX_PC_LEVELS] = {};
  double *rho0 = nullptr, *y = nullptr, *btilde = nullptr, *q = nullptr, *delta = nullptr;
  double *tmp = nullptr, *tmp2 = nullptr, *tmp3 = nullptr, *delta_pc1 = nullptr;
  double* resp[4] = {nullptr, nullptr, nullptr, nullptr};
  double *rho_init = nullptr, *f_init = nullptr;  // state of the last rte_set_initial
  int init_kind = 0;                              // 0 none, 1 isotropic rho0, 2 explicit f0
  double *partials = nullptr, *dotbuf = nullptr;
  Norms* norms = nullptr;
  int* cg_iters = nullptr;
  DsaOp dsa{};
  RomDev ig{};
  RomDev pcs[RTE_MAX_PC_LEVELS]{};   // preconditioner ROM of SI iteration l at index l - 1
  RomDev& pc = pcs[0];
  int levels = 1;                    // options.pc_levels
  // DMD-across-iterations SA steps (options.sa_kind): the cycle's model of I - T Sigma_s, the
  // last two residuals, their difference and a zero vector (the plain SI step)
  RomDev mh{};
  double *mh_r[2] = {nullptr, nullptr}, *mh_b = nullptr, *mh_zero = nullptr;
  // FNV-1a digest of the host cross sections and source given to rte_create (checked by
  // rte_load together with c_dt, so a blob of another problem on the same mesh is refused)
  uint64_t problem_digest = 0;
  std::vector<double> sig_t_host, sig_s_host;   // for the DSA operator when tau changes
  // BDF2 (options.time_scheme): f^{n-1} in the storage of f (f itself holds the history
  // h^{n+1} = (4 f^n - f^{n-1}) / 3 between steps)
  bool bdf2 = false;
  double* f_prev = nullptr;
  float* f_prev_f = nullptr;
  // state
  double g[4] = {0, 0, 0, 0};
  bool resp_ready = false;
  bool y_valid = false;
  bool flag_ig = false;
  bool flags_pc[RTE_MAX_PC_LEVELS] = {};   // Flag_PC of each iteration's ROM
  bool pending_rom = false;  // RTE_ROM_MANUAL: a step is waiting for rte_rom_update
  // per-step record kept for the ROM update
  bool ig_applied = false;
  bool pc_applied[RTE_MAX_PC_LEVELS] = {};
  int last_iters = 0;
  rte_stats stats{};
};

namespace {

thread_local std::string g_create_error;

rte_status fail(rte_handle h, rte_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

rte_status cuda_fail(rte_handle h, cudaError_t e, const char* what) {
  std::string m = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  return fail(h, RTE_ECUDA, m);
}

#define CK(call)                                               \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);     \
  } while (0)

#define TRY(call)                    \
  do {                               \
    rte_status s_ = (call);          \
    if (s_ != RTE_OK) return s_;     \
  } while (0)

rte_status set_tau(rte_handle h, double tau);   // the step's tau (backward Euler / BDF2)

// ---------------------------------------------------------------------------------------
// Angular rules (Sec. 2.1, App. A).  Gauss-Legendre nodes by Newton's method on the
// Legendre polynomial P_n (three-term recurrence), weights 2 / ((1 - x^2) P_n'(x)^2).
// ---------------------------------------------------------------------------------------
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // final derivative at the converged node
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = z;  // ascending
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Build the library direction order (user view) for GL1D and CL_HEMI rules.
rte_status make_rule(rte_handle h, const rte_quadrature* q, int dim) {
  h->mu_user.clear();
  h->eta_user.clear();
  h->w_user.clear();
  if (q->kind == RTE_Q_GL1D) {
    if (dim != 1) return fail(h, RTE_EINVAL, "RTE_Q_GL1D needs dim = 1");
    if (q->n_gl < 2 || q->n_gl % 2) return fail(h, RTE_EINVAL, "n_gl must be even and >= 2");
    std::vector<double> x, w;
    gauss_legendre(q->n_gl, x, w);
    for (int i = 0; i < q->n_gl; ++i) {
      h->mu_user.push_back(x[i]);
      h->eta_user.push_back(0.0);
      h->w_user.push_back(w[i] / 2.0);
    }
  } else if (q->kind == RTE_Q_CL_HEMI) {
    if (dim != 2) return fail(h, RTE_EINVAL, "RTE_Q_CL_HEMI needs dim = 2");
    if (q->n_gl < 2 || q->n_gl % 2 || q->n_phi < 4 || q->n_phi % 4)
      return fail(h, RTE_EINVAL, "CL rule needs even n_gl >= 2 and n_phi a multiple of 4");
    std::vector<double> x, w;
    gauss_legendre(q->n_gl, x, w);
    for (int j2 = 0; j2 < q->n_gl; ++j2) {
      if (!(x[j2] > 0.0)) continue;
      const double s = std::sqrt(1.0 - x[j2] * x[j2]);
      for (int j1 = 1; j1 <= q->n_phi; ++j1) {
        const double phi = (2.0 * j1 - 1.0) * M_PI / q->n_phi;
        h->mu_user.push_back(std::cos(phi) * s);
        h->eta_user.push_back(std::sin(phi) * s);
        h->w_user.push_back(w[j2] / q->n_phi);  // (w/2) * (1/n_phi) doubled for the hemisphere
      }
    }
  } else if (q->kind == RTE_Q_EXPLICIT) {
    if (q->n_dirs < 2 || !q->mu || !q->w || (dim == 2 && !q->eta))
      return fail(h, RTE_EINVAL, "explicit quadrature needs n_dirs >= 2 and mu, eta, w");
    for (int i = 0; i < q->n_dirs; ++i) {
      h->mu_user.push_back(q->mu[i]);
      h->eta_user.push_back(dim == 2 ? q->eta[i] : 0.0);
      h->w_user.push_back(q->w[i]);
    }
  } else {
    return fail(h, RTE_EINVAL, "unknown quadrature kind");
  }
  double ws = 0.0;
  for (size_t i = 0; i < h->w_user.size(); ++i) {
    if (!std::isfinite(h->mu_user[i]) || !std::isfinite(h->eta_user[i]) ||
        !std::isfinite(h->w_user[i]) || h->w_user[i] < 0.0)
      return fail(h, RTE_EINVAL, "quadrature has a non-finite direction or a negative weight");
    ws += h->w_user[i];
  }
  if (std::fabs(ws - 1.0) > 1e-12) return fail(h, RTE_EINVAL, "quadrature weights must sum to 1");
  return RTE_OK;
}

// Angular flux layout on the device: [family][cell][lane], slot = family * dl + lane.
size_t f_index(const Layout& L, long ncell, long c, int slot) {
  return ((size_t)(slot / L.dl) * ncell + c) * L.dl + slot % L.dl;
}
int slot_of_f_index(const Layout& L, long ncell, long i) {
  return (int)((i / (ncell * L.dl)) * L.dl + i % L.dl);
}

// The 2D FP64 sweeps carry w psi per direction (their table holds w / (tau + sigma_t + a + b)),
// so the stored angular flux there is w f: the per-slot weights to apply, else nullptr.
const double* f_weights(rte_handle h) {
  return (h->dim == 2 && !h->fp32 && h->deg == 0) ? h->cw : nullptr;
}

int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Group the directions into families of one quadrant (2D) or half-range (1D).
rte_status make_layout(rte_handle h, int dl_force) {
  Layout& L = h->L;
  L = Layout{};
  L.dim = h->dim;
  const int nv = (int)h->mu_user.size();
  L.nv = nv;
  L.slot_of_dir.assign(nv, -1);
  const int nq = h->dim == 2 ? 4 : 2;
  std::vector<std::vector<int>> byq(nq);
  for (int d = 0; d < nv; ++d) {
    const double mu = h->mu_user[d], eta = h->eta_user[d];
    if (mu == 0.0 || (h->dim == 2 && eta == 0.0))
      return fail(h, RTE_EINVAL, "a direction lies on a coordinate axis");
    int qd = mu > 0 ? 0 : 1;
    if (h->dim == 2 && eta < 0) qd += 2;
    byq[qd].push_back(d);
  }
  const int dq = (int)byq[0].size();
  for (int qd = 1; qd < nq; ++qd)
    if ((int)byq[qd].size() != dq)
      return fail(h, RTE_EINVAL, "every quadrant (half-range in 1D) needs the same number of directions");
  if (h->dim == 1) {
    L.dl = dq;
    L.nfam = 2;
    L.nslot = nv;
  } else {
    L.dl = dq >= 32 ? 32 : std::max(8, next_pow2(dq));
    if (h->opt.sweep_lanes) L.dl = h->opt.sweep_lanes;
    if (dl_force) L.dl = dl_force;
    const int gpq = (dq + L.dl - 1) / L.dl;
    L.nfam = 4 * gpq;
    L.nslot = L.nfam * L.dl;
  }
  L.mu.assign(L.nslot, 0.0);
  L.eta.assign(L.nslot, 0.0);
  L.w.assign(L.nslot, 0.0);
  L.fam_quadrant.assign(L.nfam, 0);
  const int gpq = L.nfam / nq;
  for (int qd = 0; qd < nq; ++qd) {
    for (int g = 0; g < gpq; ++g) L.fam_quadrant[qd * gpq + g] = qd;
    for (int k = 0; k < dq; ++k) {
      const int slot = (h->dim == 1) ? qd * dq + k : (qd * gpq + k / L.dl) * L.dl + k % L.dl;
      const int d = byq[qd][k];
      L.slot_of_dir[d] = slot;
      L.mu[slot] = h->mu_user[d];
      L.eta[slot] = h->eta_user[d];
      L.w[slot] = h->w_user[d];
    }
  }
  return RTE_OK;
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, sizeof(T) * count);
}

// The captured SI iterations hold the device pointers and the time step constant of the
// launches they replay: dropped whenever either changes.
void drop_graphs(rte_handle h) {
  for (auto* v : {&h->graphs, &h->loops}) {
    for (auto& g : *v)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    v->clear();
  }
}

void free_all(rte_handle h) {
  void* ptrs[] = {h->sig_t, h->sig_s, h->src, h->ca, h->cb, h->cw, h->fam_quad, h->dir_sign,
                  h->inv_d, h->f, h->pm, h->pm_a, h->edge, h->ctrl, h->psi_w, h->psi_w_a,
                  h->rho, h->rho_prev, h->rho_half, h->rho_half1, h->rho0, h->y, h->btilde,
                  h->q, h->delta, h->tmp, h->tmp2, h->tmp3, h->delta_pc1, h->resp[0],
                  h->resp[1], h->resp[2], h->resp[3], h->partials, h->dotbuf, h->norms,
                  h->cg_iters, h->rho_init, h->f_init, h->sig_t_f, h->src_f, h->ca_f,
                  h->cb_f, h->cw_f, h->f_f, h->pm_f, h->edge_f, h->psi_w_f, h->q_f, h->f_init_f,
                  h->y_ir, h->rho_ref, h->cth_f, h->ctl_f, h->fb, h->fb_init, h->fref[0],
                  h->fref[1], h->fref_init, h->sig_tl_f, h->f_prev, h->f_prev_f};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  dsa_free(h->dsa);
  rom_free(h->ig);
  for (auto& R : h->pcs) rom_free(R);
  rom_free(h->mh);
  for (double* q : {h->mh_r[0], h->mh_r[1], h->mh_b, h->mh_zero})
    if (q) cudaFree(q);
  for (int k = 0; k < RTE_MAX_PC_LEVELS; ++k) {
    double* lv[] = {h->lv_half[k], h->lv_prev[k], h->lv_delta[k], h->lv_x[k], h->lv_b[k],
                    h->lv_diff[k]};
    for (double* q : lv)
      if (q) cudaFree(q);
  }
  cudaEvent_t evs[] = {h->ev0,    h->ev1,    h->kev0,    h->kev1, h->ev_rho,
                       h->ev_r0, h->ev_r1, h->ev_gate, h->ev_pc};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
  drop_graphs(h);
  if (h->st2) cudaStreamDestroy(h->st2);
  if (h->st3) cudaStreamDestroy(h->st3);
  if (h->h_norms) cudaFreeHost(h->h_norms);
  if (h->h_cg) cudaFreeHost(h->h_cg);
  if (h->h_err) cudaFreeHost(h->h_err);
  if (h->h_loop) cudaFreeHost(h->h_loop);
  if (h->d_loop) cudaFree(h->d_loop);
  if (h->d_conv) cudaFree(h->d_conv);
  if (h->res_ticket) cudaFree(h->res_ticket);
  for (cudaEvent_t e : h->ev_norm)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_norm_b)
    if (e) cudaEventDestroy(e);
  if (h->ev_wait) cudaEventDestroy(h->ev_wait);
  if (h->h_rom_dv) cudaFreeHost(h->h_rom_dv);
  if (h->rom_dv) cudaFree(h->rom_dv);
  if (h->rom_gate) cudaFree(h->rom_gate);
  if (h->rom_partials) cudaFree(h->rom_partials);
  if (h->own_st) cudaStreamDestroy(h->own_st);
}

// ---------------------------------------------------------------------------------------
// Sweeps
// ---------------------------------------------------------------------------------------

// Device data of the sweeps in one precision.
template <class Real>
struct SV {
  const Real *sig_t, *sig_tl, *src, *ca, *cb, *cw, *inv_d, *cth, *ctl;
  Real *f, *pm, *edge, *psi_w, *q;
};
SV<double> sv64(rte_handle h) {
  return {h->sig_t, nullptr, h->src, h->ca, h->cb, h->cw, h->inv_d, nullptr, nullptr,
          h->f, h->pm, h->edge, h->psi_w, h->q};
}
SV<float> sv32(rte_handle h) {
  return {h->sig_t_f, h->sig_tl_f, h->src_f, h->ca_f, h->cb_f, h->cw_f, nullptr, h->cth_f,
          h->ctl_f, h->f_f, h->pm_f, h->edge_f, h->psi_w_f, h->q_f};
}

template <class Real>
Sweep2DArgs<Real> args2d(rte_handle h, const SV<Real>& v, int mode) {
  const auto& tl = h->tile[mode == 1 ? 1 : 0];
  Sweep2DArgs<Real> a{};
  a.nx = h->nx;
  a.ny = h->ny;
  a.nfam = h->L.nfam;
  a.nslot = h->L.nslot;
  a.nblk = tl.nblk;
  a.rows_per_blk = tl.rpb;
  a.tau = (Real)h->tau;
  a.tau_lo = (Real)(h->tau - (double)a.tau);
  a.a = v.ca;
  a.b = v.cb;
  a.w = v.cw;
  a.skip = h->skip_now;
  a.fam_quad = h->fam_quad;
  a.sig_t = v.sig_t;
  a.sig_tl = v.sig_tl;
  a.inv_d = v.inv_d;
  a.cth = v.cth;
  a.ctl = v.ctl;
  a.edge = v.edge;
  a.ctrl = h->ctrl;
  return a;
}

template <class Real>
Sweep1DArgs<Real> args1d(rte_handle h, const SV<Real>& v) {
  Sweep1DArgs<Real> a{};
  a.nx = h->nx;
  a.nslot = h->L.nslot;
  a.tau = (Real)h->tau;
  a.a = v.ca;
  a.w = v.cw;
  a.dir_sign = h->dir_sign;
  a.skip = h->skip_now;
  a.cth = v.cth;
  a.ctl = v.ctl;
  a.sig_t = v.sig_t;
  a.sig_tl = v.sig_tl;
  a.psi_w = v.psi_w;
  return a;
}

template <class Real>
void ghosts(const double g[4], Real gx[4], Real gy[4]) {
  for (int qd = 0; qd < 4; ++qd) {
    gx[qd] = (Real)((qd & 1) == 0 ? g[0] : g[1]);
    gy[qd] = (Real)(qd < 2 ? g[2] : g[3]);
  }
}

// Launch a 2D sweep with the tile of its kind (tl).
template <class Real>
cudaError_t launch2d(rte_handle h, const Sweep2DArgs<Real>& a, int mode, const rte_s::Tile& tl) {
  if (tl.kind == 3) return launch_sweep_q1(a, mode, h->L.dl, tl.R, h->st);
  if (tl.kind == 2) return launch_sweep2d_tile(a, mode, tl.R, tl.W, h->st);
  return launch_sweep2d<Real>(a, mode, tl.R, h->st);
}

// Partial moments (pm) of sum_j w_j L_j^{-1} q for the isotropic source in v.q, inflow g
// (nullptr: vacuum): per family in 2D, the full moment in 1D.
template <class Real>
rte_status k1(rte_handle h, const SV<Real>& v, const double* g) {
  const double zero[4] = {0, 0, 0, 0};
  if (!g) g = zero;
  if (h->dim == 2) {
    Sweep2DArgs<Real> a = args2d(h, v, 0);
    a.q = v.q;
    a.pm = v.pm;
    ghosts(g, a.gx, a.gy);
    CK(launch2d<Real>(h, a, 0, h->tile[0]));
  } else {
    Sweep1DArgs<Real> a = args1d(h, v);
    a.q = v.q;
    a.g_lo = (Real)g[0];
    a.g_hi = (Real)g[1];
    CK(launch_sweep1d<Real>(a, 0, h->st));
    CK(launch_moment1d<Real>(v.psi_w, h->L.nslot, (int)h->ncell, v.pm, h->st, h->skip_now));
  }
  return RTE_OK;
}

// Fused end-of-step sweep with the pass-A source already in v.q (sigma_s rho + G):
// f <- L^-1(q + tau f + g^bc) in place; pm <- partial moments of L^-1(G + tau f^n), zero inflow.
template <class Real>
rte_status k2(rte_handle h, const SV<Real>& v) {
  if (h->dim == 2) {
    Sweep2DArgs<Real> a = args2d(h, v, 1);
    a.q = v.q;
    a.g2 = v.src;
    a.f = v.f;
    a.pm = v.pm;
    ghosts(h->g, a.gx, a.gy);
    int mode = 1;
    if (h->bf16) {   // reads f^{n-1} about fref[fcur], writes f^n about fref[1 - fcur]
      a.fb = h->fb;
      a.fro = h->fref[h->fcur];
      a.frn = h->fref[1 - h->fcur];
      a.seed = h->bf_seed++;
      mode = 3;
    }
    CK(launch2d<Real>(h, a, mode, h->tile[1]));
    if (h->bf16) h->fcur = 1 - h->fcur;
  } else {
    Sweep1DArgs<Real> a = args1d(h, v);
    a.q = v.q;
    a.g2 = v.src;
    a.f = v.f;
    a.psi_w_a = nullptr;
    a.g_lo = (Real)h->g[0];
    a.g_hi = (Real)h->g[1];
    CK(launch_sweep1d<Real>(a, 1, h->st));
    CK(launch_moment1d<Real>(v.psi_w, h->L.nslot, (int)h->ncell, v.pm, h->st));
  }
  return RTE_OK;
}

// pm <- partial moments of L^-1(G + tau f) from the stored f, zero inflow.
template <class Real>
rte_status ky(rte_handle h, const SV<Real>& v) {
  if (h->dim == 2) {
    Sweep2DArgs<Real> a = args2d(h, v, 2);
    a.g2 = v.src;
    a.f = v.f;
    a.pm = v.pm;
    int mode = 2;
    if (h->bf16) {
      a.fb = h->fb;
      a.fro = a.frn = h->fref[h->fcur];
      mode = 4;
    }
    CK(launch2d<Real>(h, a, mode, h->tile[0]));
  } else {
    Sweep1DArgs<Real> a = args1d(h, v);
    a.g2 = v.src;
    a.f = v.f;
    CK(launch_sweep1d<Real>(a, 2, h->st));
    CK(launch_moment1d<Real>(v.psi_w, h->L.nslot, (int)h->ncell, v.pm, h->st));
  }
  return RTE_OK;
}

int nparts(rte_handle h) { return h->dim == 2 ? h->L.nfam : 1; }

// The sweep source q of the current precision: sigma_s (x - xref) (xref may be nullptr).
rte_status set_q(rte_handle h, const double* x, const double* xref) {
  if (h->fp32)
    CK(launch_scaled_diff<float>(x, xref, h->sig_s, (int)h->ndof, h->q_f, h->st, h->skip_now));
  else
    CK(launch_scaled_diff<double>(x, xref, h->sig_s, (int)h->ndof, h->q, h->st, h->skip_now));
  return RTE_OK;
}
// Pass-A source sigma_s rho + G of the fused sweep.
rte_status set_qa(rte_handle h, const double* rho) {
  if (h->fp32) CK(launch_scaled_plus<float>(rho, h->sig_s, h->src, (int)h->ndof, h->q_f, h->st));
  else CK(launch_scaled_plus<double>(rho, h->sig_s, h->src, (int)h->ndof, h->q, h->st));
  return RTE_OK;
}
// out (+)= sum of the partial moments, in FP64.
rte_status sum_pm(rte_handle h, double* out, int accumulate) {
  if (h->fp32)
    CK(launch_sum_pm<float>(h->pm_f, nparts(h), (int)h->ndof, out, accumulate, h->st,
                            h->skip_now));
  else
    CK(launch_sum_pm<double>(h->pm, nparts(h), (int)h->ndof, out, accumulate, h->st,
                             h->skip_now));
  return RTE_OK;
}
rte_status sweep_q(rte_handle h, const double* g) {
  return h->fp32 ? k1<float>(h, sv32(h), g) : k1<double>(h, sv64(h), g);
}

// out = sum_j w_j L_j^{-1} (sigma_s rho) with inflow g, FP64 out, in the handle's precision.
rte_status sweep_si(rte_handle h, const double* rho_or_null, const double* g, double* out) {
  if (rho_or_null) TRY(set_q(h, rho_or_null, nullptr));
  else {
    if (h->fp32) CK(cudaMemsetAsync(h->q_f, 0, sizeof(float) * h->ndof, h->st));
    else CK(cudaMemsetAsync(h->q, 0, sizeof(double) * h->ndof, h->st));
  }
  TRY(sweep_q(h, g));
  TRY(sum_pm(h, out, 0));
  return RTE_OK;
}

// Fused end-of-step sweep: f <- L^-1(sigma_s rho + tau f + G + g^bc) in place and
// y = sum_j w_j L_j^-1(G + tau f^n) with zero inflow.
rte_status sweep_f(rte_handle h, const double* rho, double* y_out) {
  TRY(set_qa(h, rho));
  if (h->bf16) CK(launch_to_float(rho, h->ncell, h->fref[1 - h->fcur], h->st));
  if (h->fp32) TRY(k2<float>(h, sv32(h)));
  else TRY(k2<double>(h, sv64(h)));
  TRY(sum_pm(h, y_out, 0));
  return RTE_OK;
}

// y = sum_j w_j L_j^-1(G + tau f) from the stored f, zero inflow.
rte_status sweep_y(rte_handle h, double* y_out) {
  if (h->fp32) TRY(ky<float>(h, sv32(h)));
  else TRY(ky<double>(h, sv64(h)));
  TRY(sum_pm(h, y_out, 0));
  return RTE_OK;
}

// Wait for the handle's stream.  Batched instances (each stepped by its own host thread)
// wait on a blocking-sync event so that the thread sleeps instead of spinning.
rte_status host_wait(rte_handle h) {
  if (h->blocking) {
    CK(cudaEventRecord(h->ev_wait, h->st));
    CK(cudaEventSynchronize(h->ev_wait));
  } else {
    CK(cudaStreamSynchronize(h->st));
  }
  return RTE_OK;
}

// The sweeps' error word (a bounded wait that ran out), copied to pinned memory with the
// step's other results; check_sweep_error_after reads it once the stream has been waited for.
// The same for the CG's grid barrier (word 2 of its barrier block).
rte_status queue_sweep_error(rte_handle h) {
  if (h->dim == 2)
    CK(cudaMemcpyAsync(h->h_err, &h->ctrl->err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(h->h_err + 1, reinterpret_cast<unsigned*>(h->dsa.scal) + 2, sizeof(unsigned),
                     cudaMemcpyDeviceToHost, h->st));
  return RTE_OK;
}
rte_status check_sweep_error_after(rte_handle h) {
  if (h->dim == 2 && h->h_err[0]) {
    h->h_err[0] = 0;
    const size_t bytes = sizeof(SweepCtrl) + sizeof(unsigned) * h->L.nfam * h->nblk_max;
    CK(cudaMemsetAsync(h->ctrl, 0, bytes, h->st));
    CK(cudaStreamSynchronize(h->st));
    return fail(h, RTE_ETIMEOUT, "a bounded wait in the sweep ran out");
  }
  if (h->h_err[1]) {
    h->h_err[1] = 0;
    CK(cudaMemsetAsync(h->dsa.scal, 0, 4 * sizeof(unsigned), h->st));
    CK(cudaStreamSynchronize(h->st));
    return fail(h, RTE_ETIMEOUT, "a bounded grid-barrier wait in the DSA solve ran out");
  }
  return RTE_OK;
}

rte_status check_sweep_error(rte_handle h) {
  unsigned err = 0;
  if (h->dim == 2) {
    CK(cudaMemcpyAsync(&err, &h->ctrl->err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (err) {
      const size_t bytes = sizeof(SweepCtrl) + sizeof(unsigned) * h->L.nfam * h->nblk_max;
      CK(cudaMemsetAsync(h->ctrl, 0, bytes, h->st));
      CK(cudaStreamSynchronize(h->st));
      return fail(h, RTE_ETIMEOUT, "a bounded wait in the sweep ran out");
    }
  }
  return RTE_OK;
}

// Responses to unit isotropic inflow on each side: b~ is linear in g, so
// b~ = y + sum_s g_s resp_s (Eq. (implicit_linear_system_rho) with g_j^bc split off).
rte_status ensure_responses(rte_handle h) {
  if (h->resp_ready) return RTE_OK;
  const int sides = h->dim == 2 ? 4 : 2;
  for (int s = 0; s < sides; ++s) {
    if (!h->resp[s]) CK(dalloc(&h->resp[s], h->ndof));
    double g[4] = {0, 0, 0, 0};
    g[s] = 1.0;
    TRY(sweep_si(h, nullptr, g, h->resp[s]));
  }
  h->resp_ready = true;
  return RTE_OK;
}

rte_status make_btilde(rte_handle h) {
  if (!h->y_valid) {
    TRY(sweep_y(h, h->y));
    h->y_valid = true;
  }
  CK(cudaMemcpyAsync(h->btilde, h->y, sizeof(double) * h->ndof, cudaMemcpyDeviceToDevice, h->st));
  const int sides = h->dim == 2 ? 4 : 2;
  bool any = false;
  for (int s = 0; s < sides; ++s) any = any || h->g[s] != 0.0;
  if (any) {
    TRY(ensure_responses(h));
    for (int s = 0; s < sides; ++s)
      if (h->g[s] != 0.0)
        CK(launch_axpby(1.0, h->btilde, h->g[s], h->resp[s], (int)h->ndof, h->btilde, h->st));
  }
  return RTE_OK;
}

// ---------------------------------------------------------------------------------------
// Device-time accounting without host waits: events are recorded into a per-handle pool as
// the work is queued, and the spans between them are read once the step's work is done.
// ---------------------------------------------------------------------------------------
enum SpanKind { SPAN_SWEEP = 0, SPAN_DSA, SPAN_ROM, SPAN_K1, SPAN_K2 };

int rec(rte_handle h) {
  if (h->capturing) return -1;
  if (h->evnext == (int)h->evpool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    h->evpool.push_back(e);
  }
  const int i = h->evnext++;
  cudaEventRecord(h->evpool[i], h->st);
  return i;
}

void span(rte_handle h, int kind, int a, int b, int iter = 0) {
  if (a >= 0 && b >= 0) h->spans.push_back({kind, a, b, iter});
}

// Adds the recorded spans to the statistics; the caller has synchronised the stream.
void resolve_spans(rte_handle h) {
  for (const auto& sp : h->spans) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->evpool[sp.a], h->evpool[sp.b]) != cudaSuccess) continue;
    switch (sp.kind) {
      case SPAN_SWEEP: h->stats.time_sweep_ms += ms; break;
      case SPAN_DSA: h->stats.time_dsa_ms += ms; break;
      case SPAN_ROM: h->stats.time_rom_ms += ms; break;
      case SPAN_K1:
        h->stats.si_sweep_kernel_ms += ms;
        h->stats.si_sweep_launches += 1;
        break;
      default:
        h->stats.f_sweep_kernel_ms += ms;
        h->stats.f_sweep_launches += 1;
        break;
    }
  }
  h->spans.clear();
  h->evnext = 0;
}

// ---------------------------------------------------------------------------------------
// Algorithm 1 on the current b~ from initial guess rho0.  Leaves rho^n in h->rho.
//
// With options.lookahead the loop runs one iteration ahead of the host: while the host waits
// for the norms of iteration l, the DSA step of l and the sweep and residual of l + 1 are
// already queued.  They carry a device skip word that the residual of l sets when l meets the
// stopping test, so past convergence they return at once and leave every result untouched.
// The l = 1 step of Phase 3 (the ROM preconditioner) is queued only after the host has seen
// l = 1 fail.  Measured on GB300 the host's turnaround between iterations (spin wait) is a
// few microseconds, less than the skipped launches cost, so lookahead is off by default.
// ---------------------------------------------------------------------------------------
// init_src: the initial guess when it is not in rho0 yet (it is then copied to rho0 too).
// pc_active: the SA steps of iterations 1 .. pc_active use the preconditioner ROMs of those
// iterations (Eq. (dmd-sa)); every other SA step is DSA.
rte_status si_sa(rte_handle h, int pc_active, int* iters_out, bool* converged_out,
                 const double* init_src) {
  const int n = (int)h->ndof;
  const int nb = vec_blocks(n);
  const int absmode = h->opt.residual_norm == RTE_ABS_INF ? 1 : 0;
  // rho^{l-1} = rho^{(0)}, skip word and CG iteration slots cleared, in one launch
  if (init_src)
    CK(launch_si_begin(init_src, h->rho0, h->rho_prev, n, h->d_conv, h->cg_iters,
                       h->opt.max_iter + 2, h->st));
  else
    CK(launch_si_begin(h->rho0, h->rho_prev, nullptr, n, h->d_conv, h->cg_iters,
                       h->opt.max_iter + 2, h->st));
  h->skip_now = h->d_conv;
  // FP64: each iteration sweeps sigma_s rho^{l-1}.  FP32 (iterative refinement): the sweeps
  // act on the increments rho^{l-1} - rho_ref in FP32 and their results accumulate into the
  // FP64 y_ir = T Sigma_s rho_ref, so rho^{l-1/2} = y_ir + b~ carries FP64 accuracy in the
  // residual; the first increment is measured from the last swept iterate of the previous step.
  auto sweep_increment = [&](int iter) -> rte_status {
    // rho^{n,(iter-1)} for the snapshot pair of the preconditioner ROM of iteration iter >= 2
    if (iter >= 2 && iter <= h->levels)
      CK(cudaMemcpyAsync(h->lv_prev[iter - 1], h->rho_prev, sizeof(double) * n,
                         cudaMemcpyDeviceToDevice, h->st));
    const int k0 = rec(h);
    if (h->fp32) {
      CK(launch_scaled_diff_update<float>(h->rho_prev, h->rho_ref, h->sig_s, n, h->q_f, h->st,
                                          h->d_conv));
      TRY(sweep_q(h, nullptr));
      span(h, SPAN_K1, k0, rec(h), iter);
      TRY(sum_pm(h, h->y_ir, 1));
    } else {
      // after a DSA solve (its kernel) or the PC (the update kernel), q = sigma_s rho^{l-1} is
      // in place already; the first sweep of a solve forms it from the initial guess
      if (iter == 1) TRY(set_q(h, h->rho_prev, nullptr));
      TRY(sweep_q(h, nullptr));
      span(h, SPAN_K1, k0, rec(h), iter);
    }
    return RTE_OK;
  };
  // rho^{l-1/2}, its norms (pinned copy, parity l & 1) and the device stopping test; the
  // kernel also writes rho^{l-1/2} to rho (the iterate the step returns once converged, work
  // past convergence skips itself) and, for l = 1, to rho^{n,1/2}
  // loop (optional): the while loop of a graph around the iteration (options.graph = 2), whose
  // residual leaves its norms on the device
  auto residual = [&](int l, const ResidualLoop* loop = nullptr) -> rte_status {
    const int p = l & 1;
    const int r0 = rec(h);
    const ResidualLoop lc = loop ? *loop : ResidualLoop{0, nullptr, 0, nullptr, nullptr};
    // rho^{n,(l-1/2)} kept for the snapshot pairs of the preconditioner ROM of iteration l
    double* half1 = l == 1 ? h->rho_half1 : (l <= h->levels ? h->lv_half[l - 1] : nullptr);
    if (h->fp32)
      CK(launch_combine_residual(h->y_ir, 1, h->btilde, h->rho_prev, n, h->rho_half, h->partials,
                                 nb, h->norms + p, h->st, h->d_conv, h->opt.eps_sisa, absmode,
                                 h->rho, half1, h->res_ticket, lc));
    else
      CK(launch_combine_residual(h->pm, nparts(h), h->btilde, h->rho_prev, n, h->rho_half,
                                 h->partials, nb, h->norms + p, h->st, h->d_conv, h->opt.eps_sisa,
                                 absmode, h->rho, half1, h->res_ticket, lc));
    if (!loop)
      CK(cudaMemcpyAsync(h->h_norms + p, h->norms + p, sizeof(Norms), cudaMemcpyDeviceToHost,
                         h->st));
    span(h, SPAN_SWEEP, r0, rec(h), l);
    return RTE_OK;
  };
  // the host waits for the norms of iteration l on this event
  auto norms_ready = [&](int l) -> rte_status {
    CK(cudaEventRecord(h->blocking ? h->ev_norm_b[l & 1] : h->ev_norm[l & 1], h->st));
    return RTE_OK;
  };
  // DSA, Eq. (rho_residual); the CG kernel also forms rho^l = rho^{l-1/2} + delta.  Its
  // iteration count stays on the device until the step ends.
  auto dsa_step = [&](int l, int iters_add = 0) -> rte_status {
    const int d0 = rec(h);
    CK(dsa_solve(h->dsa, h->sig_s, h->rho_half, h->rho_prev, h->opt.cg_rtol, h->opt.cg_max_iter,
                 h->delta, h->rho_half, h->rho_prev, h->q, h->cg_iters + l, h->st, h->d_conv,
                 iters_add));
    span(h, SPAN_DSA, d0, rec(h), l + 1);
    return RTE_OK;
  };
  // DMD-across-iterations SA step (options.sa_kind): a plain SI step that collects the
  // residual r_l = rho^{l-1/2} - rho^{l-1}; after mh_window residuals the iterate jumps to
  // rho^{l-1} + C_r^{-1} r_l, C_r the DMD model of I - T Sigma_s from the pairs
  // (r_i, r_i - r_{i+1}) of the cycle (appended as they come, with one host wait each).
  int cyc = 0;
  auto mh_step = [&](int l) -> rte_status {
    const int d0 = rec(h);
    double* r = h->mh_r[cyc & 1];
    CK(launch_axpby(1.0, h->rho_half, -1.0, h->rho_prev, n, r, h->st));
    if (cyc > 0) {
      double* rp = h->mh_r[(cyc - 1) & 1];
      CK(launch_axpby(1.0, rp, -1.0, r, n, h->mh_b, h->st));
      CK(rom_append(h->mh, rp, h->mh_b, -1.0, nullptr, nullptr, h->st));
    }
    if (++cyc == h->opt.mh_window) {
      cyc = 0;
      if (h->mh.rank > 0 && h->mh.lu_ok) {
        CK(rom_apply(h->mh, r, h->tmp, h->st));
        CK(launch_update_rho(h->rho_prev, h->tmp, h->sig_s, n, h->rho_prev, h->q, h->st));
        h->stats.total_mh_jumps += 1;
      } else {
        CK(launch_update_rho(h->rho_half, h->mh_zero, h->sig_s, n, h->rho_prev, h->q, h->st));
      }
      rom_reset(h->mh);
    } else {
      CK(launch_update_rho(h->rho_half, h->mh_zero, h->sig_s, n, h->rho_prev, h->q, h->st));
    }
    span(h, SPAN_DSA, d0, rec(h), l + 1);
    return RTE_OK;
  };
  const bool mh = h->opt.sa_kind == RTE_SA_DMD_ITER;
  if (mh) rom_reset(h->mh);
  auto sa_step = [&](int l) -> rte_status { return mh ? mh_step(l) : dsa_step(l); };
  // The SA step of iteration l, the sweep and the residual of l + 1.  With options.graph (DSA
  // steps only) they run as one CUDA graph, captured from the stream the first time l is
  // reached; every pointer and value they take is fixed for the handle until drop_graphs.
  auto iteration = [&](int l) -> rte_status {
    if (!h->opt.graph || mh) {
      TRY(sa_step(l));
      TRY(sweep_increment(l + 1));
      TRY(residual(l + 1));
      return norms_ready(l + 1);
    }
    if ((int)h->graphs.size() <= l) h->graphs.resize(l + 1);
    rte_s::IterGraph& g = h->graphs[l];
    if (!g.exec) {
      const long long k0 = g_launches;
      CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
      h->capturing = true;
      rte_status st = dsa_step(l);
      if (st == RTE_OK) st = sweep_increment(l + 1);
      if (st == RTE_OK) st = residual(l + 1);
      h->capturing = false;
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(h->st, &graph);
      g.kernels = g_launches - k0;
      g_launches = k0;
      if (st != RTE_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (st != RTE_OK) return st;
        return cuda_fail(h, e, "capturing an SI iteration as a CUDA graph");
      }
      const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) {
        g.exec = nullptr;
        return cuda_fail(h, ei, "instantiating the SI iteration's CUDA graph");
      }
    }
    CK(cudaGraphLaunch(g.exec, h->st));
    g_launches += g.kernels;
    return norms_ready(l + 1);
  };
  // options.graph = 2: once iteration l has failed its stopping test, and every iteration from
  // l on is a DSA step whose launches do not depend on its index (l >= the preconditioner ROM
  // levels), the iterations l, l + 1, ... run inside one CUDA graph: a while node whose body
  // is the SA step of l, the sweep and the residual of l + 1, and whose condition the residual
  // kernel sets from the stopping test and the iteration cap.  The CG counts of the loop add
  // up in slot l.  The host waits once, for the end of the loop; *l_out = the last iteration.
  const bool use_loop = h->opt.graph == 2 && !mh && !h->opt.lookahead;
  auto run_loop = [&](int l0, int* l_out) -> rte_status {
    if (!h->d_loop) {
      CK(cudaMalloc(&h->d_loop, sizeof(unsigned)));
      CK(cudaMallocHost(&h->h_loop, sizeof(unsigned)));
    }
    if ((int)h->loops.size() <= l0) h->loops.resize(l0 + 1);
    rte_s::IterGraph& g = h->loops[l0];
    if (!g.exec) {
      cudaGraph_t graph = nullptr;
      CK(cudaGraphCreate(&graph, 0));
      cudaGraphConditionalHandle cond = 0;
      cudaGraphNodeParams cp{};
      cudaGraphNode_t node = nullptr;
      cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
      if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
      }
      if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(h->st, cp.conditional.phGraph_out[0], nullptr, nullptr,
                                          0, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(h, e, "building the SI loop's CUDA graph");
      }
      const long long k0 = g_launches;
      const ResidualLoop lc{cond, h->d_loop, (unsigned)(h->opt.max_iter - l0),
                            h->dim == 2 ? &h->ctrl->err : nullptr,
                            reinterpret_cast<const unsigned*>(h->dsa.scal) + 2};
      h->capturing = true;
      rte_status st = dsa_step(l0, 1);
      if (st == RTE_OK) st = sweep_increment(l0 + 1);
      if (st == RTE_OK) st = residual(l0 + 1, &lc);
      h->capturing = false;
      cudaGraph_t body = nullptr;
      e = cudaStreamEndCapture(h->st, &body);
      g.kernels = g_launches - k0;
      g_launches = k0;
      if (st == RTE_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (st != RTE_OK) return st;
      if (e != cudaSuccess) {
        g.exec = nullptr;
        return cuda_fail(h, e, "capturing the SI loop as a CUDA graph");
      }
    }
    const int p = (l0 + 1) & 1;
    CK(cudaMemsetAsync(h->d_loop, 0, sizeof(unsigned), h->st));
    CK(cudaGraphLaunch(g.exec, h->st));
    CK(cudaMemcpyAsync(h->h_norms + p, h->norms + p, sizeof(Norms), cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(h->h_loop, h->d_loop, sizeof(unsigned), cudaMemcpyDeviceToHost, h->st));
    CK(cudaEventRecord(h->blocking ? h->ev_norm_b[p] : h->ev_norm[p], h->st));
    CK(cudaEventSynchronize(h->blocking ? h->ev_norm_b[p] : h->ev_norm[p]));
    const unsigned c = *h->h_loop;
    g_launches += g.kernels * (long long)c;
    *l_out = l0 + (int)c;
    return RTE_OK;
  };
  bool conv = false;
  int l = 1;
  for (bool& a : h->pc_applied) a = false;
  TRY(sweep_increment(1));
  TRY(residual(1));
  TRY(norms_ready(1));
  for (l = 1;; ++l) {
    const bool pc_now = l <= pc_active;
    if (h->opt.lookahead && !mh && l < h->opt.max_iter && !pc_now)   // l + 1, queued ahead
      TRY(iteration(l));
    CK(cudaEventSynchronize(h->blocking ? h->ev_norm_b[l & 1] : h->ev_norm[l & 1]));
    const Norms nm = h->h_norms[l & 1];
    const double res = absmode ? nm.diff_inf
                               : (nm.half_inf > 0 ? nm.diff_inf / nm.half_inf : nm.diff_inf);
    conv = absmode ? nm.diff_inf <= h->opt.eps_sisa : nm.diff_inf <= h->opt.eps_sisa * nm.half_inf;
    h->stats.last_residual = res;
    if (conv || l == h->opt.max_iter) break;
    if (use_loop && !pc_now && l >= h->levels) {
      const int p = (l + 1) & 1;
      TRY(run_loop(l, &l));
      const Norms nl = h->h_norms[p];
      h->stats.last_residual =
          absmode ? nl.diff_inf : (nl.half_inf > 0 ? nl.diff_inf / nl.half_inf : nl.diff_inf);
      conv = absmode ? nl.diff_inf <= h->opt.eps_sisa
                     : nl.diff_inf <= h->opt.eps_sisa * nl.half_inf;
      break;
    }
    if ((!h->opt.lookahead || mh) && !pc_now) TRY(iteration(l));
    if (pc_now) {
      // ROM preconditioner of iteration l, Eq. (dmd-sa):
      // delta = dU C_r^{-1} dU^T (rho^{l-1/2} - rho^{l-1})  (rho^{0} = the initial guess)
      const int k = l - 1;
      double* dpc = k == 0 ? h->delta_pc1 : h->lv_delta[k];
      const int r0 = rec(h);
      CK(launch_axpby(1.0, h->rho_half, -1.0, h->rho_prev, n, h->tmp, h->st));
      CK(rom_apply(h->pcs[k], h->tmp, dpc, h->st));
      CK(launch_update_rho(h->rho_half, dpc, h->sig_s, n, h->rho_prev, h->q, h->st));
      span(h, SPAN_ROM, r0, rec(h), l + 1);
      h->pc_applied[k] = true;
      TRY(sweep_increment(l + 1));
      TRY(residual(l + 1));
      TRY(norms_ready(l + 1));
    }
  }
  h->skip_now = nullptr;
  // drop the statistics of the speculative work that skipped itself
  h->spans.erase(std::remove_if(h->spans.begin(), h->spans.end(),
                                [&](const rte_s::Span& s) { return s.iter > l; }),
                 h->spans.end());
  // CG counts of this solve: slots 1 .. l-1 written by the DSA calls (the PC step and skipped
  // solves leave their slots at zero)
  CK(cudaMemcpyAsync(h->h_cg, h->cg_iters, sizeof(int) * (l + 2), cudaMemcpyDeviceToHost, h->st));
  h->cg_slots = l + 2;
  *iters_out = l;
  *converged_out = conv;
  return RTE_OK;
}

// Sums the CG counts copied at the end of si_sa (after the stream is synchronised); the next
// solve's first launch clears the device slots.
rte_status finish_cg_counts(rte_handle h) {
  int cg = 0;
  for (int i = 0; i < h->cg_slots; ++i) cg += h->h_cg[i];
  h->stats.last_cg_iterations = cg;
  h->stats.total_cg_iterations += cg;
  h->cg_slots = 0;
  return RTE_OK;
}

// ROM construction / adaptive update for the step just taken (Algorithm 2, Sec. 3.2), in
// two halves.  rom_update_enqueue queues every product, indicator and append on h->st
// without waiting: the indicator tests of Phase 3 become device gates that leave a ROM
// unchanged when closed.  rom_update_finish runs after the stream has passed that work and
// folds the outcome into the host view (ranks, Flag_IG / Flag_PC, statistics).  one_step
// runs the first half on a second stream beside the fused f sweep, which neither reads nor
// writes what it uses.
rte_status rom_update_enqueue(rte_handle h) {
  const int n = (int)h->ndof;
  const int nb = vec_blocks(n);
  auto& pd = h->rom_pend;
  pd = rte_s::RomPending{};
  double* dv = h->rom_dv;   // [0] ||rho^n||^2  [1] IG indicator^2  [2 + k] PC indicator^2 of
                            // iteration k + 1
  CK(launch_dot(h->rho, h->rho, n, h->rom_partials, nb, dv + 0, h->st));
  if (!h->flag_ig) {
    // Phase 1: the IG-ROM takes every snapshot pair (rho^n, b~^{n-1}), untruncated
    CK(rom_append_async(h->ig, h->rho, h->btilde, -1.0, nullptr, h->st));
    pd.ig = pd.ig_building = true;
  } else {
    if (h->ig_applied) {
      CK(launch_axpby(1.0, h->rho0, -1.0, h->rho, n, h->tmp, h->st));
      CK(launch_dot(h->tmp, h->tmp, n, h->rom_partials, nb, dv + 1, h->st));
    }
    CK(launch_rom_gate(dv + 1, dv + 0, h->opt.eps_up, h->opt.up_rel, !h->ig_applied, nullptr,
                       h->rom_gate + 0, h->st));
    // The PC-ROM's work depends on the IG gate only: it runs on a third stream beside the
    // IG append (its own scratch: tmp2, tmp3, delta, the second partials block).
    CK(cudaEventRecord(h->ev_gate, h->st));
    CK(cudaStreamWaitEvent(h->st3, h->ev_gate, 0));
    CK(rom_append_async(h->ig, h->rho, h->btilde, h->opt.eps_ig, h->rom_gate + 0, h->st));
    pd.ig = true;
    pd.ig_err = h->ig_applied;
    cudaStream_t s3 = h->st3;
    bool built_before[RTE_MAX_PC_LEVELS];
    for (int k = 0; k < RTE_MAX_PC_LEVELS; ++k) built_before[k] = h->flags_pc[k];
    const int* also = h->rom_gate + 0;   // an update of the IG-ROM forces one of the PC-ROMs
    for (int k = 0; k < h->levels; ++k) {
      // sequential construction: the ROM of iteration k+1 takes snapshots only from steps that
      // applied the ROMs of iterations 1 .. k; and only from steps that took a correction at
      // iteration k+1
      if (k > 0 && !built_before[k - 1]) break;
      if (!(h->last_iters > k + 1)) break;
      double* half = k == 0 ? h->rho_half1 : h->lv_half[k];
      const double* prev = k == 0 ? h->rho0 : h->lv_prev[k];
      double* x = k == 0 ? h->tmp2 : h->lv_x[k];
      double* b = k == 0 ? h->tmp3 : h->lv_b[k];
      // d_rho = rho^n - rho^{n,(k+1/2)} (x), d_b = rho^{n,(k+1/2)} - rho^{n,(k)} (b)
      CK(launch_axpby(1.0, h->rho, -1.0, half, n, x, s3));
      CK(launch_axpby(1.0, half, -1.0, prev, n, b, s3));
      if (!h->flags_pc[k]) {   // construction: every correction pair, untruncated
        CK(rom_append_async(h->pcs[k], x, b, -1.0, nullptr, s3));
        pd.pc[k] = pd.pc_building[k] = true;
      } else {
        double* diff = k == 0 ? h->delta : h->lv_diff[k];
        const double* dpc = k == 0 ? h->delta_pc1 : h->lv_delta[k];
        double* part = h->rom_partials + (size_t)(1 + k) * 3 * 1024;
        if (h->pc_applied[k]) {
          CK(launch_axpby(1.0, dpc, -1.0, x, n, diff, s3));
          CK(launch_dot(diff, diff, n, part, nb, dv + 2 + k, s3));
        }
        CK(launch_rom_gate(dv + 2 + k, dv + 0, h->opt.eps_up, h->opt.up_rel, !h->pc_applied[k],
                           also, h->rom_gate + 1 + k, s3));
        CK(rom_append_async(h->pcs[k], x, b, h->opt.eps_pc, h->rom_gate + 1 + k, s3));
        pd.pc[k] = true;
        pd.pc_err[k] = h->pc_applied[k];
        also = h->rom_gate + 1 + k;
      }
    }
    CK(cudaEventRecord(h->ev_pc, s3));
    CK(cudaStreamWaitEvent(h->st, h->ev_pc, 0));
  }
  CK(cudaMemcpyAsync(h->h_rom_dv, dv, sizeof(double) * (2 + h->levels), cudaMemcpyDeviceToHost,
                     h->st));
  pd.queued = true;
  return RTE_OK;
}

rte_status rom_update_finish(rte_handle h) {
  auto& pd = h->rom_pend;
  if (!pd.queued) return RTE_OK;
  pd.queued = false;
  int ig_ran = 0;
  int pc_ran[RTE_MAX_PC_LEVELS] = {};
  double ratio = 0.0;
  if (pd.ig) {
    CK(rom_commit(h->ig, &ig_ran, nullptr, &ratio, h->st));
    if (pd.ig_building && (ratio <= h->opt.eps_ig || h->ig.rank >= h->opt.r_max)) h->flag_ig = true;
  }
  for (int k = 0; k < h->levels; ++k) {
    if (!pd.pc[k]) continue;
    CK(rom_commit(h->pcs[k], &pc_ran[k], nullptr, &ratio, h->st));
    if (pd.pc_building[k] && (ratio <= h->opt.eps_pc || h->pcs[k].rank >= h->opt.r_max))
      h->flags_pc[k] = true;
  }
  h->stats.last_ig_error = pd.ig_err ? std::sqrt(h->h_rom_dv[1]) : NAN;
  h->stats.last_pc_error = pd.pc_err[0] ? std::sqrt(h->h_rom_dv[2]) : NAN;
  h->stats.ig_updated = ig_ran;
  h->stats.pc_updated = pc_ran[0];
  h->stats.ig_rank = h->ig.rank;
  h->stats.pc_rank = h->pc.rank;
  for (int k = 0; k < RTE_MAX_PC_LEVELS; ++k) {
    h->stats.pc_level_rank[k] = h->pcs[k].rank;
    h->stats.pc_level_updated[k] = pc_ran[k];
  }
  return RTE_OK;
}

// All preconditioner ROMs built: Phase 3.
bool all_pc_built(rte_handle h) {
  for (int k = 0; k < h->levels; ++k)
    if (!h->flags_pc[k]) return false;
  return true;
}

rte_status one_step(rte_handle h) {
  const bool rom_on = h->opt.rom != RTE_ROM_OFF;
  auto t0 = std::chrono::steady_clock::now();
  if (!h->spans.empty()) {   // left over by a failed call
    CK(cudaStreamSynchronize(h->st));
    resolve_spans(h);
  }
  int mark = rec(h);
  TRY(make_btilde(h));
  int m = rec(h);
  span(h, SPAN_SWEEP, mark, m);
  mark = m;
  h->ig_applied = false;
  if (rom_on && h->flag_ig && h->ig.lu_ok) {
    CK(rom_apply(h->ig, h->btilde, h->rho0, h->st));   // Eq. (dmd-ig)
    h->ig_applied = true;
    m = rec(h);
    span(h, SPAN_ROM, mark, m);
  }
  // the ROM of iteration l applies once it and the ROMs of iterations 1 .. l-1 are built
  int pc_active = 0;
  while (rom_on && pc_active < h->levels && h->flags_pc[pc_active] && h->pcs[pc_active].lu_ok)
    ++pc_active;
  int iters = 0;
  bool conv = false;
  // without the IG the initial guess is rho^{n-1} itself
  TRY(si_sa(h, pc_active, &iters, &conv, h->ig_applied ? nullptr : h->rho));
  h->last_iters = iters;
  // the phase this step ran in (the ROM update below may end it)
  const int phase = !rom_on ? 0 : (!h->flag_ig ? 1 : (!all_pc_built(h) ? 2 : 3));
  // rho^n is final: the ROM update may start beside the fused sweep
  CK(cudaEventRecord(h->ev_rho, h->st));
  // BDF2: the first step is a backward-Euler step; f^0 is kept for the first history
  const bool bdf2_start = h->bdf2 && h->stats.steps == 0;
  const size_t fcount = (size_t)h->ndof * h->L.nslot;
  if (bdf2_start) {
    if (h->fp32)
      CK(cudaMemcpyAsync(h->f_prev_f, h->f_f, sizeof(float) * fcount, cudaMemcpyDeviceToDevice, h->st));
    else
      CK(cudaMemcpyAsync(h->f_prev, h->f, sizeof(double) * fcount, cudaMemcpyDeviceToDevice, h->st));
  }
  // f^n and the next step's b~ (without inflow): Eq. (sweep_to_obtain_f), Eq. (implicit_linear_system_rho)
  mark = rec(h);
  TRY(sweep_f(h, h->rho, h->y));
  m = rec(h);
  span(h, SPAN_K2, mark, m);
  span(h, SPAN_SWEEP, mark, m);
  h->y_valid = true;
  if (h->bdf2) {
    // the buffer of f now holds the next step's history (4 f^n - f^{n-1}) / 3, that of f^{n-1}
    // holds f^n; the next step sweeps its b~ from the history (pass B above used f^n)
    if (h->fp32) CK(launch_bdf2_history<float>(h->f_f, h->f_prev_f, (long)fcount, h->st));
    else CK(launch_bdf2_history<double>(h->f, h->f_prev, (long)fcount, h->st));
    h->y_valid = false;
  }
  bool rom_ran = false;
  rte_status rom_status = RTE_OK;
  // BDF2's backward-Euler first step gives the ROMs no snapshot
  if (rom_on && conv && h->opt.rom == RTE_ROM_AUTO && !bdf2_start) {
    CK(cudaStreamWaitEvent(h->st2, h->ev_rho, 0));
    cudaStream_t main = h->st;
    h->st = h->st2;
    cudaEventRecord(h->ev_r0, h->st2);
    rom_status = rom_update_enqueue(h);
    cudaEventRecord(h->ev_r1, h->st2);
    h->st = main;
    CK(cudaStreamWaitEvent(h->st, h->ev_r1, 0));   // the next step applies the updated ROMs
    rom_ran = true;
  }
  TRY(queue_sweep_error(h));
  TRY(host_wait(h));
  resolve_spans(h);
  TRY(finish_cg_counts(h));
  TRY(rom_status);
  if (rom_ran) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_r0, h->ev_r1) == cudaSuccess) h->stats.time_rom_ms += ms;
    TRY(rom_update_finish(h));
  }
  TRY(check_sweep_error_after(h));
  h->stats.phase = phase;
  h->stats.steps += 1;
  h->stats.last_iterations = iters;
  h->stats.total_iterations += iters;
  // BDF2: one sweep more per step (the next step's b~ from the history)
  const int sweeps = iters + 2 + (h->bdf2 ? 1 : 0);
  h->stats.total_sweeps += sweeps;
  h->stats.cell_direction_updates += (long long)sweeps * h->ncell * h->L.nv;
  if (bdf2_start) TRY(set_tau(h, 1.5 / h->c_dt));   // BDF2 from the second step on
  if (!conv) return fail(h, RTE_ENOCONV, "SI-SA reached max_iter without meeting eps_sisa");
  if (rom_on && h->opt.rom == RTE_ROM_MANUAL && !bdf2_start) h->pending_rom = true;
  auto t1 = std::chrono::steady_clock::now();
  h->stats.time_total_ms += std::chrono::duration<double, std::milli>(t1 - t0).count();
  return RTE_OK;
}

// IEEE binary32 -> bfloat16 with round-to-nearest-even (NaN kept quiet), and back.
uint16_t bf16_bits(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float x;
  std::memcpy(&x, &u, 4);
  return x;
}

bool finite_all(const double* v, long n) {
  for (long i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

rte_status upload(rte_handle h, double* dst, const double* src, long n) {
  CK(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return RTE_OK;
}

// FP32 tau + a + b of each slot as an exact hi / lo pair (tau and a, b rounded to FP32 once).
void fp32_ct_pairs(rte_handle h, std::vector<float>& cth, std::vector<float>& ctl) {
  const Layout& L = h->L;
  const double tau32 = (double)(float)h->tau;
  cth.resize(L.nslot);
  ctl.resize(L.nslot);
  for (int s = 0; s < L.nslot; ++s) {
    const double a = (double)(float)(std::fabs(L.mu[s]) / h->hx);
    const double b = h->dim == 2 ? (double)(float)(std::fabs(L.eta[s]) / h->hy) : 0.0;
    const double ct = tau32 + a + b;
    cth[s] = (float)ct;
    ctl[s] = (float)(ct - (double)cth[s]);
  }
}

// The step's tau = 1 / (c dt) (backward Euler) or 3 / (2 c dt) (BDF2): the FP64 inverse table,
// the FP32 tau + a + b pairs, the DSA operator and the inflow responses follow it.
rte_status set_tau(rte_handle h, double tau) {
  if (h->tau == tau) return RTE_OK;
  h->tau = tau;
  drop_graphs(h);   // the sweeps take tau by value and the DSA operator is rebuilt
  const Layout& L = h->L;
  if (!h->fp32 && h->dim == 2 && h->inv_d) {
    if (h->deg == 0)
      CK(launch_inv_d<double>(h->sig_t, h->ca, h->cb, h->cw, h->tau, (int)h->ncell, L.nslot,
                              L.dl, h->inv_d, h->st));
    else
      CK(launch_q1_table(h->sig_t, h->ca, h->cb, h->tau, (int)h->ncell, L.nslot, L.dl, h->inv_d,
                         h->st));
  }
  if (h->fp32 && h->cth_f) {
    std::vector<float> cth, ctl;
    fp32_ct_pairs(h, cth, ctl);
    CK(cudaMemcpyAsync(h->cth_f, cth.data(), sizeof(float) * L.nslot, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->ctl_f, ctl.data(), sizeof(float) * L.nslot, cudaMemcpyHostToDevice, h->st));
  }
  if (h->fp32) {   // the refinement pair y_ir = T Sigma_s rho_ref belongs to the old tau
    CK(cudaMemsetAsync(h->y_ir, 0, sizeof(double) * h->ndof, h->st));
    CK(cudaMemsetAsync(h->rho_ref, 0, sizeof(double) * h->ndof, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  dsa_free(h->dsa);
  CK(dsa_setup(h->dsa, h->dim, h->nx, h->ny, h->hx, h->hy, h->tau, h->sig_t_host.data(),
               h->sig_s_host.data(), h->st, h->opt.cg_blocks, h->deg, h->dsa_f32,
               h->opt.dsa_cluster != 0));
  h->resp_ready = false;
  h->y_valid = false;
  return RTE_OK;
}

rte_status reset_state(rte_handle h) {
  // BDF2 starts with a backward-Euler step
  if (h->bdf2) TRY(set_tau(h, 1.0 / h->c_dt));
  if (h->fp32) {
    // refinement state: y_ir = T Sigma_s rho_ref with rho_ref = 0
    CK(cudaMemsetAsync(h->y_ir, 0, sizeof(double) * h->ndof, h->st));
    CK(cudaMemsetAsync(h->rho_ref, 0, sizeof(double) * h->ndof, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  h->stats = rte_stats{};
  h->rom_pend = rte_s::RomPending{};
  h->bf_seed = 0;
  h->flag_ig = false;
  for (bool& f : h->flags_pc) f = false;
  h->y_valid = false;
  h->pending_rom = false;
  rom_reset(h->ig);
  for (int k = 0; k < h->levels; ++k) rom_reset(h->pcs[k]);
  return RTE_OK;
}

// Nudge FP32 weights by whole units in the last place, largest first, until their exact
// (FP64) sum is as close to 1 as the grid of the smallest weight allows.
void balance_weights(std::vector<float>& w) {
  std::vector<int> order(w.size());
  for (size_t i = 0; i < w.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return w[x] > w[y]; });
  auto deficit = [&]() {
    double s = 0.0;
    for (float v : w) s += (double)v;
    return 1.0 - s;
  };
  for (int k : order) {
    if (w[k] <= 0.0f) continue;
    const double ulp = (double)std::nextafter(w[k], 2.0f * w[k] + 1.0f) - (double)w[k];
    const double steps = std::nearbyint(deficit() / ulp);
    if (steps != 0.0) w[k] = (float)((double)w[k] + steps * ulp);
  }
}

// Per-slot direction data of the current layout: a = |mu|/hx, b = |eta|/hy, the weights, the
// quadrant of each family and the sign of mu; in FP32 mode also their FP32 forms.
rte_status setup_slots(rte_handle h) {
  const Layout& L = h->L;
  std::vector<double> a(L.nslot), b(L.nslot);
  std::vector<int> sign(L.nslot);
  for (int s = 0; s < L.nslot; ++s) {
    a[s] = std::fabs(L.mu[s]) / h->hx;
    b[s] = h->dim == 2 ? std::fabs(L.eta[s]) / h->hy : 0.0;
    sign[s] = L.mu[s] > 0 ? 1 : -1;
  }
  CK(dalloc(&h->ca, L.nslot));
  CK(dalloc(&h->cb, L.nslot));
  CK(dalloc(&h->cw, L.nslot));
  CK(dalloc(&h->fam_quad, L.nfam));
  CK(dalloc(&h->dir_sign, L.nslot));
  TRY(upload(h, h->ca, a.data(), L.nslot));
  TRY(upload(h, h->cb, b.data(), L.nslot));
  TRY(upload(h, h->cw, L.w.data(), L.nslot));
  CK(cudaMemcpy(h->fam_quad, L.fam_quadrant.data(), sizeof(int) * L.nfam, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->dir_sign, sign.data(), sizeof(int) * L.nslot, cudaMemcpyHostToDevice));
  if (h->fp32) {
    // FP32 coefficients: a, b, tau and sigma_t rounded once; tau + a + b of each slot kept
    // exactly as a hi / lo pair, and the weights nudged by whole ulps so that their exact
    // sum is 1 again.  The FP32 sweeps then apply the exact Q0 operator of these rounded
    // coefficients, which conserves particles like the FP64 one.
    std::vector<float> a32(L.nslot), b32(L.nslot), cth, ctl, w32(L.nslot);
    for (int s = 0; s < L.nslot; ++s) {
      a32[s] = (float)a[s];
      b32[s] = (float)b[s];
      w32[s] = (float)L.w[s];
    }
    fp32_ct_pairs(h, cth, ctl);
    balance_weights(w32);
    CK(dalloc(&h->ca_f, L.nslot));
    CK(dalloc(&h->cb_f, L.nslot));
    CK(dalloc(&h->cw_f, L.nslot));
    CK(dalloc(&h->cth_f, L.nslot));
    CK(dalloc(&h->ctl_f, L.nslot));
    float* hv[] = {a32.data(), b32.data(), w32.data(), cth.data(), ctl.data()};
    float* dv[] = {h->ca_f, h->cb_f, h->cw_f, h->cth_f, h->ctl_f};
    for (int i = 0; i < 5; ++i)
      CK(cudaMemcpy(dv[i], hv[i], sizeof(float) * L.nslot, cudaMemcpyHostToDevice));
  }
  return RTE_OK;
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_slots(rte_handle h) {
  dfree(h->ca), dfree(h->cb), dfree(h->cw), dfree(h->fam_quad), dfree(h->dir_sign);
  dfree(h->ca_f), dfree(h->cb_f), dfree(h->cw_f), dfree(h->cth_f), dfree(h->ctl_f);
}

// Angular flux, partial-moment, face (edge) and control buffers of the sweeps, for the
// current layout; the edge buffers and flags are sized for nblk_max row blocks.
rte_status alloc_sweep(rte_handle h) {
  const Layout& L = h->L;
  const long n = h->ncell, nd = h->ndof;
  if (!h->fp32) {
    CK(dalloc(&h->f, (size_t)nd * L.nslot));
    CK(cudaMemsetAsync(h->f, 0, sizeof(double) * nd * L.nslot, h->st));
  } else if (!h->bf16) {
    CK(dalloc(&h->f_f, (size_t)nd * L.nslot));
    CK(cudaMemsetAsync(h->f_f, 0, sizeof(float) * nd * L.nslot, h->st));
  } else {
    CK(dalloc(&h->fb, (size_t)n * L.nslot));
    CK(cudaMemsetAsync(h->fb, 0, sizeof(__nv_bfloat16) * n * L.nslot, h->st));
    for (auto& r : h->fref) {
      CK(dalloc(&r, n));
      CK(cudaMemsetAsync(r, 0, sizeof(float) * n, h->st));
    }
    h->fcur = 0;
  }
  if (h->dim == 2) {
    // two passes (the fused sweep), times the face modes a row hands on (Q1: two)
    const size_t edge = (size_t)2 * L.nfam * h->nblk_max * h->nx * L.dl * (h->deg == 1 ? 2 : 1);
    if (!h->fp32) {
      if (h->deg == 0) {
        CK(dalloc(&h->inv_d, (size_t)n * L.nslot));
        CK(launch_inv_d<double>(h->sig_t, h->ca, h->cb, h->cw, h->tau, (int)n, L.nslot, L.dl,
                                h->inv_d, h->st));
      } else {   // Q1: four factors of the cell solve per cell and direction
        CK(dalloc(&h->inv_d, (size_t)4 * n * L.nslot));
        CK(launch_q1_table(h->sig_t, h->ca, h->cb, h->tau, (int)n, L.nslot, L.dl, h->inv_d,
                           h->st));
      }
      CK(dalloc(&h->pm, (size_t)L.nfam * nd));
      CK(dalloc(&h->edge, edge));
    } else {
      CK(dalloc(&h->pm_f, (size_t)L.nfam * nd));
      CK(dalloc(&h->edge_f, edge));
    }
    const size_t cb_bytes = sizeof(SweepCtrl) + sizeof(unsigned) * L.nfam * h->nblk_max;
    CK(cudaMalloc((void**)&h->ctrl, cb_bytes));
    CK(cudaMemsetAsync(h->ctrl, 0, cb_bytes, h->st));
  } else {
    if (!h->fp32) {
      CK(dalloc(&h->pm, n));
      CK(dalloc(&h->psi_w, (size_t)n * L.nslot));
    } else {
      CK(dalloc(&h->pm_f, n));
      CK(dalloc(&h->psi_w_f, (size_t)n * L.nslot));
    }
  }
  return RTE_OK;
}

void free_sweep(rte_handle h) {
  dfree(h->fb), dfree(h->fref[0]), dfree(h->fref[1]);
  dfree(h->f), dfree(h->f_f), dfree(h->inv_d), dfree(h->pm), dfree(h->pm_f), dfree(h->edge);
  dfree(h->edge_f), dfree(h->ctrl), dfree(h->psi_w), dfree(h->psi_w_f);
}

void set_tile(rte_handle h, rte_s::Tile& tl, int kind, int R, int W) {
  tl.kind = kind;
  tl.R = R;
  tl.W = W;
  tl.rpb = W * (32 / h->L.dl) * R;
  tl.nblk = (h->ny + tl.rpb - 1) / tl.rpb;
}

// A tile is usable when its kind applies (the tile sequence takes TH = 4 or 8, and 2 in the
// FP32 modes; the strip chain R <= dl) and every sweep mode's staging fits the 200 KiB the
// launchers allow.
bool tile_fits(rte_handle h, int dl, int kind, int R, int W) {
  if (h->deg == 1) return kind == 3 && W == 1 && (R == 1 || R == 2 || R == 4);
  if (kind == 3) return false;
  const int modes_plain[3] = {0, 1, 2}, modes_bf[3] = {0, 3, 4};
  const size_t real = h->fp32 ? sizeof(float) : sizeof(double);
  if (kind == 2) {
    if (dl < 8) return false;   // the tile sequence takes 8, 16 or 32 lanes
    if (R != 4 && R != 8 && !(R == 2 && h->fp32)) return false;
    for (int mode : h->bf16 ? modes_bf : modes_plain)
      if (sweep2d_tile_smem_bytes(real, dl, R, W, mode) > 200 * 1024) return false;
    return true;
  }
  if (R > dl) return false;
  // strip chain: 2 lanes in FP64 only, 4 lanes in FP64 and FP32 (a BF16 family of 4 lanes or
  // an FP32 family of 2 is less than one 16-byte piece of a cell)
  if (dl == 2 && h->fp32) return false;
  if (dl == 4 && h->bf16) return false;
  for (int mode : h->bf16 ? modes_bf : modes_plain)
    if (sweep2d_smem_bytes(real, dl, R, W, mode, !h->fp32) > 200 * 1024) return false;
  return true;
}

// Device time of one launch of one sweep mode (0: SI sweep, 1: fused f sweep) after one
// warm-up launch.
rte_status time_sweeps(rte_handle h, int kind, float* ms) {
  auto run = [&]() -> rte_status {
    return kind == 0 ? sweep_q(h, nullptr) : sweep_f(h, h->rho, h->y);
  };
  TRY(run());
  CK(cudaEventRecord(h->kev0, h->st));
  TRY(run());
  CK(cudaEventRecord(h->kev1, h->st));
  CK(cudaEventSynchronize(h->kev1));
  TRY(check_sweep_error(h));
  CK(cudaEventElapsedTime(ms, h->kev0, h->kev1));
  return RTE_OK;
}

struct TuneKey {
  int device, nx, ny, nv, precision, degree;
  bool operator<(const TuneKey& o) const {
    return std::tie(device, nx, ny, nv, precision, degree) <
           std::tie(o.device, o.nx, o.ny, o.nv, o.precision, o.degree);
  }
};
struct TuneVal {
  int dl;
  rte_s::Tile t0, t1;   // kind, R, W of the SI sweep and of the fused sweep
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

// Direction lanes per family (dl), and for each of the two sweep modes the kernel (strip
// chain, or for FP32 also the tile sequence) with its tile (R rows per lane group, W warps per
// CTA).  With options.tune every usable combination is timed on this problem's own data (zero
// flux; the kernels' work does not depend on the values) and the choice with the least
// 3 t_SI + t_f is kept, once per (device, grid, direction count, precision) and process.
// Explicit sweep_* options, or tune = 0, give the fixed choice instead.
rte_status choose_tiles(rte_handle h, int* dl_out) {
  const int dq = (int)h->mu_user.size() / 4;
  const int dl_max = dq >= 32 ? 32 : std::max(8, next_pow2(dq));
  const bool fixed = h->opt.sweep_lanes || h->opt.sweep_rows || h->opt.sweep_warps ||
                     h->opt.sweep_kernel || !h->opt.tune;
  if (fixed && h->deg == 1) {   // the Q1 strip chain: one warp per CTA
    const int dl = h->opt.sweep_lanes ? h->opt.sweep_lanes : std::min(dl_max, 8);
    const int R = h->opt.sweep_rows ? h->opt.sweep_rows : 2;
    if (!tile_fits(h, dl, 3, R, 1)) return fail(h, RTE_EINVAL, "the Q1 sweep takes sweep_rows 1, 2 or 4");
    for (auto& tl : h->tile) {
      tl.kind = 3;
      tl.R = R;
      tl.W = 1;
    }
    *dl_out = dl;
    return RTE_OK;
  }
  if (fixed) {
    int dl = h->opt.sweep_lanes ? h->opt.sweep_lanes
                                : std::min(dl_max, (!h->fp32 && h->ncell >= 512L * 512) ? 32 : 8);
    const int kind = h->opt.sweep_kernel == 2 ? 2 : 1;
    int R = h->opt.sweep_rows ? h->opt.sweep_rows : (kind == 2 ? 4 : (h->fp32 ? 2 : 1));
    if (kind == 1) R = std::min(R, dl);
    int W = h->opt.sweep_warps ? h->opt.sweep_warps : 8;
    while (W > 1 && !tile_fits(h, dl, kind, R, W)) --W;
    if (!tile_fits(h, dl, kind, R, W)) return fail(h, RTE_EINVAL, "the sweep tile does not fit");
    for (auto& tl : h->tile) {
      tl.kind = kind;
      tl.R = R;
      tl.W = W;
    }
    *dl_out = dl;
    return RTE_OK;
  }
  const TuneKey key{h->device, h->nx, h->ny, (int)h->mu_user.size(), h->opt.precision, h->deg};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      h->tile[0] = it->second.t0;
      h->tile[1] = it->second.t1;
      *dl_out = it->second.dl;
      h->tuned = true;
      return RTE_OK;
    }
  }
  float best = INFINITY;
  TuneVal bv{};
  // 2 and 4 lanes: the Q1 sweep and the FP64 Q0 strip chain, where narrow lane groups stack
  // more rows in a warp and halve the hand-offs between CTAs (measured at 256^2 x 128, SI
  // sweep with 8 / 4 / 2 lanes: Q1 FP64 2.89 / 2.58 / 2.42 ms, Q0 FP64 0.320 / 0.284 / 0.260 ms;
  // at 1024^2 the tuner keeps wider groups: Q1 FP32 5.6 ms with 2 lanes against 4.6 with 4)
  const int dls[5] = {2, 4, 8, 16, 32};
  struct Cand {
    int kind, R, W;
  };
  for (int dl : dls) {
    if (dl > dl_max || (dl == 2 && h->deg != 1 && h->fp32) || (dl == 4 && h->bf16)) continue;
    TRY(make_layout(h, dl));
    std::vector<Cand> cand;
    const int rs[3] = {1, 2, 4}, ws[3] = {2, 4, 8}, ths[3] = {2, 4, 8};
    for (int R : rs) {
      if (tile_fits(h, dl, 3, R, 1)) cand.push_back({3, R, 1});
      for (int W : ws)
        if (tile_fits(h, dl, 1, R, W)) cand.push_back({1, R, W});
    }
    // The FP64 tile sequence is left out of the search: on 256^2 and 1024^2 grids with 128
    // directions it measured 1.6-1.8x slower than the strip chain in both sweep modes (the
    // FP64 pipe, not the hand-offs, bounds those sweeps); it stays selectable by sweep_kernel.
    if (h->fp32)
      for (int th : ths)
        for (int W : ws)
          if (tile_fits(h, dl, 2, th, W)) cand.push_back({2, th, W});
    if (cand.empty()) continue;
    int nb = 1;
    for (auto& c : cand) {
      rte_s::Tile tl;
      set_tile(h, tl, c.kind, c.R, c.W);
      nb = std::max(nb, tl.nblk);
    }
    h->nblk_max = nb;
    TRY(setup_slots(h));
    TRY(alloc_sweep(h));
    TRY(set_q(h, h->src, nullptr));
    float t1b = INFINITY, t2b = INFINITY;
    Cand c1 = cand[0], c2 = cand[0];
    for (auto& c : cand) {
      set_tile(h, h->tile[0], c.kind, c.R, c.W);
      set_tile(h, h->tile[1], c.kind, c.R, c.W);
      float t1 = 0.f, t2 = 0.f;
      TRY(time_sweeps(h, 0, &t1));
      TRY(time_sweeps(h, 1, &t2));
      if (t1 < t1b) t1b = t1, c1 = c;
      if (t2 < t2b) t2b = t2, c2 = c;
    }
    CK(cudaStreamSynchronize(h->st));
    free_sweep(h);
    free_slots(h);
    const float score = 3.f * t1b + t2b;
    if (score < best) {
      best = score;
      bv.dl = dl;
      bv.t0.kind = c1.kind, bv.t0.R = c1.R, bv.t0.W = c1.W;
      bv.t1.kind = c2.kind, bv.t1.R = c2.R, bv.t1.W = c2.W;
    }
  }
  if (bv.dl == 0) return fail(h, RTE_EINVAL, "no sweep tile fits in shared memory");
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = bv;
  }
  h->tile[0] = bv.t0;
  h->tile[1] = bv.t1;
  *dl_out = bv.dl;
  h->tuned = true;
  return RTE_OK;
}

// Host-side checks of rte_create (no device work): options, mesh, cross sections, rule.
rte_status validate_impl(rte_handle h, const rte_mesh* mesh, const rte_quadrature* quad,
                         const double* sigma_t, const double* sigma_s, const double* source,
                         double c_dt, const rte_options* opt) {
  if (!mesh || !quad || !sigma_t || !sigma_s || !source)
    return fail(h, RTE_EINVAL, "mesh, quadrature and cross-section arrays are required");
  h->opt = opt ? *opt : rte_options{};
  if (!opt) rte_default_options(&h->opt);
  if (mesh->dim != 1 && mesh->dim != 2) return fail(h, RTE_EINVAL, "dim must be 1 or 2");
  if (mesh->nx < 1 || mesh->ny < 1 || (mesh->dim == 1 && mesh->ny != 1))
    return fail(h, RTE_EINVAL, "bad cell counts");
  if (!(mesh->x1 > mesh->x0) || (mesh->dim == 2 && !(mesh->y1 > mesh->y0)))
    return fail(h, RTE_EINVAL, "empty domain");
  if (!(c_dt > 0.0) || !std::isfinite(c_dt)) return fail(h, RTE_EINVAL, "c_dt must be > 0");
  if (h->opt.precision != RTE_FP64 && h->opt.precision != RTE_FP32 &&
      h->opt.precision != RTE_FP32_BF16F)
    return fail(h, RTE_EINVAL, "precision must be RTE_FP64, RTE_FP32 or RTE_FP32_BF16F");
  if (h->opt.precision == RTE_FP32_BF16F && mesh->dim != 2)
    return fail(h, RTE_EINVAL, "RTE_FP32_BF16F is available for 2D problems");
  h->fp32 = h->opt.precision != RTE_FP64;
  h->bf16 = h->opt.precision == RTE_FP32_BF16F;
  if (h->opt.r_max < 1 || h->opt.r_max > 64) return fail(h, RTE_EINVAL, "r_max must be in [1, 64]");
  if (h->opt.pc_levels == 0) h->opt.pc_levels = 1;   // options zeroed by hand: the default
  if (h->opt.pc_levels < 1 || h->opt.pc_levels > RTE_MAX_PC_LEVELS)
    return fail(h, RTE_EINVAL, "pc_levels must be in [1, RTE_MAX_PC_LEVELS]");
  h->levels = h->opt.pc_levels;
  if (h->opt.cg_blocks < 0) return fail(h, RTE_EINVAL, "cg_blocks must be >= 0");
  if (h->opt.dsa_cluster != 0 && h->opt.dsa_cluster != 1)
    return fail(h, RTE_EINVAL, "dsa_cluster must be 0 or 1");
  if (h->opt.time_scheme != RTE_BE && h->opt.time_scheme != RTE_BDF2)
    return fail(h, RTE_EINVAL, "time_scheme must be RTE_BE or RTE_BDF2");
  if (h->opt.time_scheme == RTE_BDF2 && h->opt.precision == RTE_FP32_BF16F)
    return fail(h, RTE_EINVAL, "RTE_BDF2 is not available with RTE_FP32_BF16F");
  h->bdf2 = h->opt.time_scheme == RTE_BDF2;
  if (h->opt.sa_kind != RTE_SA_DSA && h->opt.sa_kind != RTE_SA_DMD_ITER)
    return fail(h, RTE_EINVAL, "sa_kind must be RTE_SA_DSA or RTE_SA_DMD_ITER");
  if (h->opt.mh_window == 0) h->opt.mh_window = 4;   // options zeroed by hand: the default
  if (h->opt.mh_window < 2 || h->opt.mh_window > 16)
    return fail(h, RTE_EINVAL, "mh_window must be in [2, 16]");
  if (h->opt.max_iter < 1 || h->opt.cg_max_iter < 0) return fail(h, RTE_EINVAL, "bad iteration caps");
  if (h->opt.graph < 0 || h->opt.graph > 2) return fail(h, RTE_EINVAL, "graph must be 0, 1 or 2");
  if (h->opt.sweep_lanes != 0 && h->opt.sweep_lanes != 8 && h->opt.sweep_lanes != 16 &&
      h->opt.sweep_lanes != 32 &&
      !((h->opt.sweep_lanes == 2 || h->opt.sweep_lanes == 4) &&
        (h->opt.degree == 1 || h->opt.precision == RTE_FP64)) &&
      !(h->opt.sweep_lanes == 4 && h->opt.precision == RTE_FP32))
    return fail(h, RTE_EINVAL,
                "sweep_lanes must be 0, 8, 16 or 32 (2 also in RTE_FP64 and with degree 1, "
                "4 also in RTE_FP64 and RTE_FP32)");
  if (h->opt.sweep_rows != 0 && h->opt.sweep_rows != 1 && h->opt.sweep_rows != 2 &&
      h->opt.sweep_rows != 4 && h->opt.sweep_rows != 8)
    return fail(h, RTE_EINVAL, "sweep_rows must be 0, 1, 2, 4 or 8");
  if (h->opt.sweep_warps < 0 || h->opt.sweep_warps > 8)
    return fail(h, RTE_EINVAL, "sweep_warps must be in [0, 8]");
  if (h->opt.sweep_kernel < 0 || h->opt.sweep_kernel > 2)
    return fail(h, RTE_EINVAL, "sweep_kernel must be 0, 1 or 2");
  if (!(h->opt.eps_sisa >= 0.0)) return fail(h, RTE_EINVAL, "eps_sisa must be >= 0");
  if (h->opt.degree != 0 && h->opt.degree != 1) return fail(h, RTE_EINVAL, "degree must be 0 or 1");
  if (h->opt.degree == 1 && (mesh->dim != 2 || h->opt.precision == RTE_FP32_BF16F))
    return fail(h, RTE_EINVAL, "degree 1 (Q1) is available for 2D problems in RTE_FP64 or RTE_FP32");
  h->deg = h->opt.degree;
  h->nb = h->deg == 1 ? 4 : 1;
  h->dim = mesh->dim;
  h->nx = mesh->nx;
  h->ny = mesh->ny;
  h->ncell = (long)mesh->nx * mesh->ny;
  h->ndof = h->nb * h->ncell;
  if (h->ndof > (1L << 31) / 2) return fail(h, RTE_EINVAL, "too many cells");
  h->hx = (mesh->x1 - mesh->x0) / mesh->nx;
  h->hy = mesh->dim == 2 ? (mesh->y1 - mesh->y0) / mesh->ny : 1.0;
  h->c_dt = c_dt;
  h->tau = 1.0 / c_dt;
  const long n = h->ncell;
  if (!finite_all(sigma_t, n) || !finite_all(sigma_s, n) || !finite_all(source, h->ndof))
    return fail(h, RTE_EINVAL, "non-finite cross section or source");
  for (long i = 0; i < n; ++i)
    if (sigma_s[i] < 0.0 || sigma_t[i] < sigma_s[i])
      return fail(h, RTE_EINVAL, "need sigma_t >= sigma_s >= 0 in every cell");
  TRY(make_rule(h, quad, h->dim));
  TRY(make_layout(h, 0));   // validates the directions before any device work
  return RTE_OK;
}

rte_status create_impl(rte_handle h, const rte_mesh* mesh, const rte_quadrature* quad,
                       const double* sigma_t, const double* sigma_s, const double* source,
                       double c_dt, const rte_options* opt) {
  TRY(validate_impl(h, mesh, quad, sigma_t, sigma_s, source, c_dt, opt));
  const long n = h->ncell, nd = h->ndof;
  CK(cudaGetDevice(&h->device));
  // The step's own stream runs at the highest priority and the two ROM-update streams at the
  // lowest, so that the block scheduler hands freed SMs to the critical path (the fused f
  // sweep) before the ROM appends queued beside it.
  int prio_least = 0, prio_greatest = 0;
  CK(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
  CK(cudaStreamCreateWithPriority(&h->own_st, cudaStreamNonBlocking, prio_greatest));
  h->st = h->own_st;
  CK(cudaEventCreate(&h->ev0));
  CK(cudaEventCreate(&h->ev1));
  CK(cudaEventCreate(&h->kev0));
  CK(cudaEventCreate(&h->kev1));
  CK(cudaStreamCreateWithPriority(&h->st2, cudaStreamNonBlocking, prio_least));
  CK(cudaStreamCreateWithPriority(&h->st3, cudaStreamNonBlocking, prio_least));
  CK(cudaEventCreateWithFlags(&h->ev_gate, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_pc, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_rho, cudaEventDisableTiming));
  CK(cudaEventCreate(&h->ev_r0));
  CK(cudaEventCreate(&h->ev_r1));
  CK(cudaMallocHost((void**)&h->h_norms, 2 * sizeof(Norms)));
  CK(cudaMallocHost((void**)&h->h_cg, sizeof(int) * (h->opt.max_iter + 2)));
  CK(cudaMallocHost((void**)&h->h_rom_dv, sizeof(double) * (2 + RTE_MAX_PC_LEVELS)));
  CK(cudaMallocHost((void**)&h->h_err, 2 * sizeof(unsigned)));
  h->h_err[0] = h->h_err[1] = 0;
  CK(cudaEventCreateWithFlags(&h->ev_wait, cudaEventBlockingSync | cudaEventDisableTiming));
  CK(cudaMalloc((void**)&h->rom_dv, sizeof(double) * (2 + RTE_MAX_PC_LEVELS)));
  CK(cudaMemset(h->rom_dv, 0, sizeof(double) * (2 + RTE_MAX_PC_LEVELS)));
  CK(cudaMalloc((void**)&h->rom_gate, sizeof(int) * (1 + RTE_MAX_PC_LEVELS)));
  CK(dalloc(&h->rom_partials, (size_t)(1 + RTE_MAX_PC_LEVELS) * 3 * 1024));
  // data that does not depend on the direction layout
  CK(dalloc(&h->sig_t, n));
  CK(dalloc(&h->sig_s, nd));
  CK(dalloc(&h->src, nd));
  TRY(upload(h, h->sig_t, sigma_t, n));
  // sigma_s on every unknown of a cell (mode-major: the same value for each Q1 mode), so that
  // the vector kernels scale rho-like vectors by it elementwise
  for (int k = 0; k < h->nb; ++k) TRY(upload(h, h->sig_s + k * n, sigma_s, n));
  TRY(upload(h, h->src, source, nd));
  {
    uint64_t d = 1469598103934665603ull;   // FNV-1a, 64 bit, over the bytes of the three arrays
    const long lens[3] = {n, n, nd};
    int ai = 0;
    for (const double* a : {sigma_t, sigma_s, source}) {
      const unsigned char* b = reinterpret_cast<const unsigned char*>(a);
      for (size_t i = 0; i < sizeof(double) * (size_t)lens[ai]; ++i) d = (d ^ b[i]) * 1099511628211ull;
      ++ai;
    }
    h->problem_digest = d;
  }
  if (h->fp32) {
    CK(dalloc(&h->sig_t_f, n));
    CK(dalloc(&h->sig_tl_f, n));
    CK(dalloc(&h->src_f, nd));
    {   // sigma_t as an exact pair hi + lo of FP32 numbers
      std::vector<float> hi(n), lo(n);
      for (long c = 0; c < n; ++c) {
        hi[c] = (float)sigma_t[c];
        lo[c] = (float)(sigma_t[c] - (double)hi[c]);
      }
      CK(cudaMemcpy(h->sig_t_f, hi.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->sig_tl_f, lo.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    }
    CK(launch_to_float(h->src, nd, h->src_f, h->st));
    CK(dalloc(&h->q_f, nd));
    CK(dalloc(&h->y_ir, nd));
    CK(dalloc(&h->rho_ref, nd));
  }
  double** vecs[] = {&h->rho, &h->rho_prev, &h->rho_half, &h->rho_half1, &h->rho0, &h->y,
                     &h->btilde, &h->q, &h->delta, &h->tmp, &h->tmp2, &h->tmp3, &h->delta_pc1};
  for (double** v : vecs) {
    CK(dalloc(v, nd));
    CK(cudaMemsetAsync(*v, 0, sizeof(double) * nd, h->st));
  }
  CK(dalloc(&h->partials, 3 * 1024));
  CK(dalloc(&h->dotbuf, 4));
  CK(dalloc(&h->norms, 2));
  CK(cudaMalloc((void**)&h->d_conv, sizeof(unsigned)));
  CK(cudaMemset(h->d_conv, 0, sizeof(unsigned)));
  CK(cudaMalloc((void**)&h->res_ticket, sizeof(unsigned)));
  CK(cudaMemset(h->res_ticket, 0, sizeof(unsigned)));
  for (auto& e : h->ev_norm) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  for (auto& e : h->ev_norm_b)
    CK(cudaEventCreateWithFlags(&e, cudaEventBlockingSync | cudaEventDisableTiming));
  CK(dalloc(&h->cg_iters, (size_t)h->opt.max_iter + 2));
  CK(cudaMemsetAsync(h->cg_iters, 0, sizeof(int) * (h->opt.max_iter + 2), h->st));
  // direction layout and sweep tiles: measured (tune), else the fixed choice
  int dl = 0;
  if (h->dim == 2) TRY(choose_tiles(h, &dl));
  TRY(make_layout(h, dl));
  if (h->dim == 2) {
    for (auto& tl : h->tile) set_tile(h, tl, tl.kind, tl.R, tl.W);
    h->nblk_max = std::max(h->tile[0].nblk, h->tile[1].nblk);
  }
  TRY(setup_slots(h));
  TRY(alloc_sweep(h));
  h->sig_t_host.assign(sigma_t, sigma_t + n);
  h->sig_s_host.assign(sigma_s, sigma_s + n);
  if (h->bdf2) {
    const size_t fc = (size_t)nd * h->L.nslot;
    if (h->fp32) {
      CK(dalloc(&h->f_prev_f, fc));
      CK(cudaMemsetAsync(h->f_prev_f, 0, sizeof(float) * fc, h->st));
    } else {
      CK(dalloc(&h->f_prev, fc));
      CK(cudaMemsetAsync(h->f_prev, 0, sizeof(double) * fc, h->st));
    }
  }
  // The FP32 modes solve the DSA system in FP32 as well (dots and CG scalars in FP64) unless
  // options.dsa_fp64: it only preconditions the SI iteration, whose residual stays FP64, so
  // its precision moves the iteration count at most, never the fixed point.
  h->dsa_f32 = h->fp32 && !h->opt.dsa_fp64;
  CK(dsa_setup(h->dsa, h->dim, h->nx, h->ny, h->hx, h->hy, h->tau, sigma_t, sigma_s, h->st,
               h->opt.cg_blocks, h->deg, h->dsa_f32, h->opt.dsa_cluster != 0));
  CK(rom_alloc(h->ig, (int)nd, h->opt.r_max));
  if (h->opt.sa_kind == RTE_SA_DMD_ITER) {
    CK(rom_alloc(h->mh, (int)nd, h->opt.mh_window));
    for (double** q : {&h->mh_r[0], &h->mh_r[1], &h->mh_b, &h->mh_zero}) {
      CK(dalloc(q, nd));
      CK(cudaMemsetAsync(*q, 0, sizeof(double) * nd, h->st));
    }
  }
  for (int k = 0; k < h->levels; ++k) {
    CK(rom_alloc(h->pcs[k], (int)nd, h->opt.r_max));
    if (k == 0) continue;
    double** lv[] = {&h->lv_half[k], &h->lv_prev[k], &h->lv_delta[k], &h->lv_x[k], &h->lv_b[k],
                     &h->lv_diff[k]};
    for (double** q : lv) {
      CK(dalloc(q, nd));
      CK(cudaMemsetAsync(*q, 0, sizeof(double) * nd, h->st));
    }
  }
  CK(cudaStreamSynchronize(h->st));
  return reset_state(h);
}

// ---------------------------------------------------------------------------------------
// Checkpoint blob (rte_save / rte_load): a header with the problem's sizes, the direction
// layout and the host-side state, the handle's device state arrays in a fixed order, then
// the IG-ROM and the PC-ROM.
// ---------------------------------------------------------------------------------------
struct CkptHead {
  char magic[8];
  uint32_t version;
  int32_t dim, nx, ny, nslot, dl, nfam, precision, r_max;
  uint64_t bytes;   // whole blob
  double g[4];
  int32_t y_valid, flag_ig, flag_pc, fcur;
  uint32_t bf_seed, reserved;
  double c_dt;
  uint64_t problem_digest;   // of sigma_t, sigma_s and the source
  rte_stats stats;
};
const char kCkptMagic[8] = {'R', 'T', 'E', 'C', 'K', 'P', 'T', '\0'};
constexpr uint32_t kCkptVersion = 2;

struct StatePart {
  void* dev;
  size_t bytes;
};
// What a step reads from the previous one: f^n (in the precision's storage), rho^n, the next
// b~ without inflow (y) and, with FP32 sweeps, the refinement pair (rho_ref, y_ir).
std::vector<StatePart> state_parts(rte_handle h) {
  const size_t n = (size_t)h->ncell, nd = (size_t)h->ndof, ns = (size_t)h->L.nslot;
  std::vector<StatePart> v;
  if (!h->fp32) {
    v.push_back({h->f, sizeof(double) * nd * ns});
  } else if (!h->bf16) {
    v.push_back({h->f_f, sizeof(float) * nd * ns});
  } else {
    v.push_back({h->fb, sizeof(__nv_bfloat16) * n * ns});
    v.push_back({h->fref[0], sizeof(float) * n});
    v.push_back({h->fref[1], sizeof(float) * n});
  }
  if (h->bdf2) {
    if (h->fp32) v.push_back({h->f_prev_f, sizeof(float) * n * ns});
    else v.push_back({h->f_prev, sizeof(double) * nd * ns});
  }
  v.push_back({h->rho, sizeof(double) * nd});
  v.push_back({h->y, sizeof(double) * nd});
  if (h->fp32) {
    v.push_back({h->rho_ref, sizeof(double) * nd});
    v.push_back({h->y_ir, sizeof(double) * nd});
  }
  return v;
}

size_t state_fixed_bytes(rte_handle h) {
  size_t b = 0;
  for (const auto& p : state_parts(h)) b += p.bytes;
  return b;
}

size_t rom_state_bytes_pcs(rte_handle h) {
  size_t b = 0;
  for (int k = 0; k < h->levels; ++k) b += rom_state_bytes(h->pcs[k]);
  return b;
}

// rte_set_initial for the Q1 scheme: rho0 [ndof] copied to every direction, or f0
// [n_dirs][ndof] in the device layout [fam][cell][k][dl] with rho = sum_j w_j f0_j.
rte_status set_initial_q1(rte_handle h, const double* rho0, const double* f0) {
  const Layout& L = h->L;
  const long n = h->ncell, nd = h->ndof;
  if (f0) {
    if (!finite_all(f0, nd * L.nv)) return fail(h, RTE_EINVAL, "non-finite f0");
    std::vector<double> fl((size_t)nd * L.nslot, 0.0), rho(nd, 0.0);
    for (int d = 0; d < L.nv; ++d) {
      const int sl = L.slot_of_dir[d];
      for (int k = 0; k < 4; ++k)
        for (long c = 0; c < n; ++c) fl[f_index(L, 4 * n, 4 * c + k, sl)] = f0[(size_t)d * nd + k * n + c];
    }
    for (int d = 0; d < L.nv; ++d)
      for (long i = 0; i < nd; ++i) rho[i] += h->w_user[d] * f0[(size_t)d * nd + i];
    TRY(upload(h, h->rho, rho.data(), nd));
    if (!h->fp32) {
      TRY(upload(h, h->f, fl.data(), (long)fl.size()));
      if (!h->f_init) CK(dalloc(&h->f_init, fl.size()));
      CK(cudaMemcpyAsync(h->f_init, h->f, sizeof(double) * fl.size(), cudaMemcpyDeviceToDevice,
                         h->st));
    } else {
      std::vector<float> ff(fl.begin(), fl.end());
      CK(cudaMemcpyAsync(h->f_f, ff.data(), sizeof(float) * ff.size(), cudaMemcpyHostToDevice,
                         h->st));
      if (!h->f_init_f) CK(dalloc(&h->f_init_f, ff.size()));
      CK(cudaMemcpyAsync(h->f_init_f, h->f_f, sizeof(float) * ff.size(), cudaMemcpyDeviceToDevice,
                         h->st));
      CK(cudaStreamSynchronize(h->st));
    }
    h->init_kind = 2;
  } else {
    if (!rho0) return fail(h, RTE_EINVAL, "rho0 or f0 is required");
    if (!finite_all(rho0, nd)) return fail(h, RTE_EINVAL, "non-finite rho0");
    TRY(upload(h, h->rho, rho0, nd));
    if (!h->fp32) CK(launch_isotropic_f_q1(h->rho, (int)n, L.nslot, L.dl, h->f, h->st));
    else CK(launch_isotropic_f32_q1(h->rho, (int)n, L.nslot, L.dl, h->f_f, h->st));
    h->init_kind = 1;
  }
  return RTE_OK;
}

rte_status sync_streams(rte_handle h) {
  CK(cudaStreamSynchronize(h->st));
  if (h->st2) CK(cudaStreamSynchronize(h->st2));
  if (h->st3) CK(cudaStreamSynchronize(h->st3));
  return RTE_OK;
}

}  // namespace

// =========================================================================================
// C ABI
// =========================================================================================
extern "C" {

void rte_default_options(rte_options* o) {
  if (!o) return;
  *o = rte_options{};
  o->eps_sisa = 1e-8;
  o->eps_ig = 1e-6;
  o->eps_pc = 1e-6;
  o->eps_up = 1e-6;
  o->max_iter = 500;
  o->r_max = 40;
  o->precision = RTE_FP64;
  o->rom = RTE_ROM_AUTO;
  o->residual_norm = RTE_REL_INF;
  o->up_rel = 1;
  o->cg_rtol = 1e-6;
  o->cg_max_iter = 500;
  o->tune = 1;
  o->lookahead = 0;
  o->pc_levels = 1;
  o->sa_kind = RTE_SA_DSA;
  o->mh_window = 4;
}

rte_status rte_create(rte_handle* out, const rte_mesh* mesh, const rte_quadrature* quad,
                      const double* sigma_t, const double* sigma_s, const double* source,
                      double c_dt, const rte_options* opt) {
  if (!out) return RTE_EINVAL;
  *out = nullptr;
  rte_handle h = new (std::nothrow) rte_s();
  if (!h) return RTE_ENOMEM;
  rte_status s = create_impl(h, mesh, quad, sigma_t, sigma_s, source, c_dt, opt);
  if (s != RTE_OK) {
    g_create_error = h->err;   // the handle is gone; rte_last_error(NULL) reports it
    free_all(h);
    delete h;
    return s;
  }
  *out = h;
  return RTE_OK;
}

rte_status rte_set_initial(rte_handle h, const double* rho0, const double* f0) {
  if (!h) return RTE_EINVAL;
  const long n = h->ncell;
  const Layout& L = h->L;
  if (h->deg == 1) TRY(set_initial_q1(h, rho0, f0));
  else if (f0) {
    if (!finite_all(f0, n * L.nv)) return fail(h, RTE_EINVAL, "non-finite f0");
    std::vector<double> fl((size_t)n * L.nslot, 0.0), rho(n, 0.0);
    for (int d = 0; d < L.nv; ++d) {
      const int s = L.slot_of_dir[d];
      for (long c = 0; c < n; ++c) fl[f_index(L, n, c, s)] = f0[(size_t)d * n + c];
    }
    for (int d = 0; d < L.nv; ++d)
      for (long c = 0; c < n; ++c) rho[c] += h->w_user[d] * f0[(size_t)d * n + c];
    TRY(upload(h, h->rho, rho.data(), n));
    if (!h->fp32) {
      if (f_weights(h))
        for (size_t i = 0; i < fl.size(); ++i) fl[i] *= L.w[slot_of_f_index(L, n, (long)i)];
      TRY(upload(h, h->f, fl.data(), (long)fl.size()));
      if (!h->f_init) CK(dalloc(&h->f_init, (size_t)n * L.nslot));
      CK(cudaMemcpyAsync(h->f_init, h->f, sizeof(double) * n * L.nslot, cudaMemcpyDeviceToDevice,
                         h->st));
    } else if (!h->bf16) {
      std::vector<float> ff(fl.begin(), fl.end());
      CK(cudaMemcpyAsync(h->f_f, ff.data(), sizeof(float) * ff.size(), cudaMemcpyHostToDevice, h->st));
      if (!h->f_init_f) CK(dalloc(&h->f_init_f, (size_t)n * L.nslot));
      CK(cudaMemcpyAsync(h->f_init_f, h->f_f, sizeof(float) * n * L.nslot, cudaMemcpyDeviceToDevice,
                         h->st));
      CK(cudaStreamSynchronize(h->st));
    } else {
      // reference = the FP32 scalar flux of f0, remainders in BF16
      std::vector<float> ref(n);
      for (long c = 0; c < n; ++c) ref[c] = (float)rho[c];
      std::vector<uint16_t> rb(fl.size());
      for (size_t i = 0; i < fl.size(); ++i) {
        const long c = (long)((i / L.dl) % n);
        rb[i] = bf16_bits((float)(fl[i] - (double)ref[c]));
      }
      h->fcur = 0;
      CK(cudaMemcpy(h->fb, rb.data(), sizeof(uint16_t) * rb.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->fref[0], ref.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
      if (!h->fb_init) CK(dalloc(&h->fb_init, (size_t)n * L.nslot));
      if (!h->fref_init) CK(dalloc(&h->fref_init, n));
      CK(cudaMemcpy(h->fb_init, rb.data(), sizeof(uint16_t) * rb.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->fref_init, ref.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    }
    h->init_kind = 2;
  } else {
    if (!rho0) return fail(h, RTE_EINVAL, "rho0 or f0 is required");
    if (!finite_all(rho0, n)) return fail(h, RTE_EINVAL, "non-finite rho0");
    TRY(upload(h, h->rho, rho0, n));
    if (!h->fp32) {
      CK(launch_isotropic_f(h->rho, (int)n, L.nslot, L.dl, f_weights(h), h->f, h->st));
    } else if (!h->bf16) {
      CK(launch_isotropic_f32(h->rho, (int)n, L.nslot, L.dl, h->f_f, h->st));
    } else {   // isotropic: zero remainders about the reference rho0
      h->fcur = 0;
      CK(cudaMemsetAsync(h->fb, 0, sizeof(__nv_bfloat16) * n * L.nslot, h->st));
      CK(launch_to_float(h->rho, n, h->fref[0], h->st));
    }
    h->init_kind = 1;
  }
  if (!h->rho_init) CK(dalloc(&h->rho_init, h->ndof));
  CK(cudaMemcpyAsync(h->rho_init, h->rho, sizeof(double) * h->ndof, cudaMemcpyDeviceToDevice,
                     h->st));
  CK(cudaStreamSynchronize(h->st));
  return reset_state(h);
}

rte_status rte_set_stream(rte_handle h, void* cuda_stream) {
  if (!h) return RTE_EINVAL;
  CK(cudaStreamSynchronize(h->st));
  h->st = cuda_stream ? (cudaStream_t)cuda_stream : h->own_st;
  return RTE_OK;
}

rte_status rte_restart(rte_handle h) {
  if (!h) return RTE_EINVAL;
  if (h->init_kind == 0) return fail(h, RTE_ESTATE, "rte_set_initial has not been called");
  const long n = h->ncell;
  CK(cudaMemcpyAsync(h->rho, h->rho_init, sizeof(double) * h->ndof, cudaMemcpyDeviceToDevice,
                     h->st));
  if (h->deg == 1) {
    const size_t fc = (size_t)h->ndof * h->L.nslot;
    if (h->init_kind == 2 && !h->fp32)
      CK(cudaMemcpyAsync(h->f, h->f_init, sizeof(double) * fc, cudaMemcpyDeviceToDevice, h->st));
    else if (h->init_kind == 2)
      CK(cudaMemcpyAsync(h->f_f, h->f_init_f, sizeof(float) * fc, cudaMemcpyDeviceToDevice, h->st));
    else if (!h->fp32)
      CK(launch_isotropic_f_q1(h->rho, (int)n, h->L.nslot, h->L.dl, h->f, h->st));
    else
      CK(launch_isotropic_f32_q1(h->rho, (int)n, h->L.nslot, h->L.dl, h->f_f, h->st));
  } else if (h->bf16) {
    h->fcur = 0;
    if (h->init_kind == 2) {
      CK(cudaMemcpyAsync(h->fb, h->fb_init, sizeof(__nv_bfloat16) * n * h->L.nslot,
                         cudaMemcpyDeviceToDevice, h->st));
      CK(cudaMemcpyAsync(h->fref[0], h->fref_init, sizeof(float) * n, cudaMemcpyDeviceToDevice,
                         h->st));
    } else {
      CK(cudaMemsetAsync(h->fb, 0, sizeof(__nv_bfloat16) * n * h->L.nslot, h->st));
      CK(launch_to_float(h->rho, n, h->fref[0], h->st));
    }
  } else if (h->init_kind == 2 && !h->fp32)
    CK(cudaMemcpyAsync(h->f, h->f_init, sizeof(double) * n * h->L.nslot, cudaMemcpyDeviceToDevice,
                       h->st));
  else if (h->init_kind == 2)
    CK(cudaMemcpyAsync(h->f_f, h->f_init_f, sizeof(float) * n * h->L.nslot,
                       cudaMemcpyDeviceToDevice, h->st));
  else if (!h->fp32)
    CK(launch_isotropic_f(h->rho, (int)n, h->L.nslot, h->L.dl, f_weights(h), h->f, h->st));
  else
    CK(launch_isotropic_f32(h->rho, (int)n, h->L.nslot, h->L.dl, h->f_f, h->st));
  CK(cudaStreamSynchronize(h->st));
  return reset_state(h);
}

rte_status rte_set_inflow(rte_handle h, const double g[4]) {
  if (!h || !g) return RTE_EINVAL;
  for (int s = 0; s < 4; ++s)
    if (!std::isfinite(g[s])) return fail(h, RTE_EINVAL, "non-finite inflow");
  for (int s = 0; s < 4; ++s) h->g[s] = (h->dim == 1 && s >= 2) ? 0.0 : g[s];
  return RTE_OK;
}

rte_status rte_step(rte_handle h, int nsteps) {
  if (!h) return RTE_EINVAL;
  if (nsteps < 0) return fail(h, RTE_EINVAL, "nsteps must be >= 0");
  if (h->pending_rom) return fail(h, RTE_ESTATE, "RTE_ROM_MANUAL: call rte_rom_update first");
  const long long l0 = g_launches;
  rte_status s = RTE_OK;
  for (int k = 0; k < nsteps && s == RTE_OK; ++k) s = one_step(h);
  h->stats.kernel_launches += g_launches - l0;
  return s;
}

rte_status rte_rom_update(rte_handle h) {
  if (!h) return RTE_EINVAL;
  if (h->opt.rom != RTE_ROM_MANUAL || !h->pending_rom)
    return fail(h, RTE_ESTATE, "no manual ROM update is pending");
  h->pending_rom = false;
  const long long l0 = g_launches;
  cudaEventRecord(h->ev_r0, h->st);
  rte_status s = rom_update_enqueue(h);
  cudaEventRecord(h->ev_r1, h->st);
  h->stats.kernel_launches += g_launches - l0;
  if (s != RTE_OK) return s;
  CK(cudaStreamSynchronize(h->st));
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, h->ev_r0, h->ev_r1) == cudaSuccess) h->stats.time_rom_ms += ms;
  TRY(rom_update_finish(h));
  CK(cudaStreamSynchronize(h->st));   // a compaction queued by the commit
  return RTE_OK;
}

rte_status rte_get_scalar_flux(rte_handle h, double* rho) {
  if (!h || !rho) return RTE_EINVAL;
  CK(cudaMemcpyAsync(rho, h->rho, sizeof(double) * h->ndof, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return RTE_OK;
}

rte_status rte_get_angular_flux(rte_handle h, double* f) {
  if (!h || !f) return RTE_EINVAL;
  const Layout& L = h->L;
  const long n = h->ncell;
  if (h->deg == 1) {
    // device [fam][cell][k][dl] -> caller [dir][k ncell + cell]
    std::vector<double> fl((size_t)h->ndof * L.nslot);
    const bool prev = h->bdf2 && h->stats.steps > 0;
    if (!h->fp32) {
      CK(cudaMemcpyAsync(fl.data(), prev ? h->f_prev : h->f, sizeof(double) * fl.size(),
                         cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
    } else {
      std::vector<float> ff(fl.size());
      CK(cudaMemcpyAsync(ff.data(), prev ? h->f_prev_f : h->f_f, sizeof(float) * ff.size(),
                         cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
      for (size_t i = 0; i < ff.size(); ++i) fl[i] = ff[i];
    }
    for (int d = 0; d < L.nv; ++d) {
      const int sl = L.slot_of_dir[d];
      for (int k = 0; k < 4; ++k)
        for (long c = 0; c < n; ++c)
          f[(size_t)d * h->ndof + k * n + c] = fl[f_index(L, 4 * n, 4 * c + k, sl)];
    }
    return RTE_OK;
  }
  std::vector<double> fl((size_t)n * L.nslot);
  // BDF2 after a step: f^n sits in the buffer of f^{n-1} (that of f holds the history)
  const bool prev = h->bdf2 && h->stats.steps > 0;
  if (!h->fp32) {
    CK(cudaMemcpyAsync(fl.data(), prev ? h->f_prev : h->f, sizeof(double) * fl.size(),
                       cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (f_weights(h))
      for (size_t i = 0; i < fl.size(); ++i) {
        const double w = L.w[slot_of_f_index(L, n, (long)i)];
        fl[i] = w != 0.0 ? fl[i] / w : 0.0;
      }
  } else if (!h->bf16) {
    std::vector<float> ff(fl.size());
    CK(cudaMemcpyAsync(ff.data(), prev ? h->f_prev_f : h->f_f, sizeof(float) * ff.size(),
                       cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    for (size_t i = 0; i < ff.size(); ++i) fl[i] = ff[i];
  } else {
    std::vector<uint16_t> rb(fl.size());
    std::vector<float> ref(n);
    CK(cudaMemcpyAsync(rb.data(), h->fb, sizeof(uint16_t) * rb.size(), cudaMemcpyDeviceToHost,
                       h->st));
    CK(cudaMemcpyAsync(ref.data(), h->fref[h->fcur], sizeof(float) * n, cudaMemcpyDeviceToHost,
                       h->st));
    CK(cudaStreamSynchronize(h->st));
    for (size_t i = 0; i < rb.size(); ++i)
      fl[i] = (double)(ref[(i / L.dl) % n] + bf16_value(rb[i]));
  }
  for (int d = 0; d < L.nv; ++d) {
    const int s = L.slot_of_dir[d];
    for (long c = 0; c < n; ++c) f[(size_t)d * n + c] = fl[f_index(L, n, c, s)];
  }
  return RTE_OK;
}

rte_status rte_quadrature_rule(const rte_quadrature* quad, int dim, int* n_dirs, double* mu,
                               double* eta, double* w) {
  if (!quad || !n_dirs || (dim != 1 && dim != 2)) {
    g_create_error = "rte_quadrature_rule: NULL argument or dim not 1 or 2";
    return RTE_EINVAL;
  }
  rte_s tmp;   // host fields only: nothing here touches a device
  const rte_status st = make_rule(&tmp, quad, dim);
  if (st != RTE_OK) {
    g_create_error = tmp.err;
    return st;
  }
  *n_dirs = (int)tmp.w_user.size();
  for (int d = 0; d < *n_dirs; ++d) {
    if (mu) mu[d] = tmp.mu_user[d];
    if (eta) eta[d] = tmp.eta_user[d];
    if (w) w[d] = tmp.w_user[d];
  }
  return RTE_OK;
}

rte_status rte_get_quadrature(rte_handle h, int* n_dirs, double* mu, double* eta, double* w) {
  if (!h) return RTE_EINVAL;
  if (n_dirs) *n_dirs = h->L.nv;
  for (int d = 0; d < h->L.nv; ++d) {
    if (mu) mu[d] = h->mu_user[d];
    if (eta) eta[d] = h->eta_user[d];
    if (w) w[d] = h->w_user[d];
  }
  return RTE_OK;
}

rte_status rte_save_size(rte_handle h, size_t* bytes) {
  if (!h || !bytes) return RTE_EINVAL;
  *bytes = sizeof(CkptHead) + state_fixed_bytes(h) + rom_state_bytes(h->ig) +
           rom_state_bytes_pcs(h);
  return RTE_OK;
}

rte_status rte_save(rte_handle h, void* buf, size_t bytes) {
  if (!h || !buf) return RTE_EINVAL;
  if (h->pending_rom)
    return fail(h, RTE_ESTATE, "RTE_ROM_MANUAL: call rte_rom_update before rte_save");
  size_t need = 0;
  TRY(rte_save_size(h, &need));
  if (bytes < need) return fail(h, RTE_EINVAL, "checkpoint buffer smaller than rte_save_size");
  TRY(sync_streams(h));
  CkptHead hd{};
  std::memcpy(hd.magic, kCkptMagic, sizeof(hd.magic));
  hd.version = kCkptVersion;
  hd.dim = h->dim;
  hd.nx = h->nx;
  hd.ny = h->ny;
  hd.nslot = h->L.nslot;
  hd.dl = h->L.dl;
  hd.nfam = h->L.nfam;
  hd.precision = h->opt.precision;
  hd.r_max = h->opt.r_max;
  hd.bytes = need;
  for (int s = 0; s < 4; ++s) hd.g[s] = h->g[s];
  hd.y_valid = h->y_valid ? 1 : 0;
  hd.flag_ig = h->flag_ig ? 1 : 0;
  hd.flag_pc = 0;
  for (int k = 0; k < h->levels; ++k) hd.flag_pc |= h->flags_pc[k] ? 1 << k : 0;
  hd.reserved = (uint32_t)(h->levels | (h->deg << 8));   // pc_levels and the DG degree
  hd.fcur = h->fcur;
  hd.bf_seed = h->bf_seed;
  hd.c_dt = h->c_dt;
  hd.problem_digest = h->problem_digest;
  hd.stats = h->stats;
  unsigned char* out = static_cast<unsigned char*>(buf);
  std::memcpy(out, &hd, sizeof(hd));
  out += sizeof(hd);
  for (const auto& p : state_parts(h)) {
    CK(cudaMemcpyAsync(out, p.dev, p.bytes, cudaMemcpyDeviceToHost, h->st));
    out += p.bytes;
  }
  CK(cudaStreamSynchronize(h->st));
  CK(rom_save(h->ig, out, h->st));
  out += rom_state_bytes(h->ig);
  for (int k = 0; k < h->levels; ++k) {
    CK(rom_save(h->pcs[k], out, h->st));
    out += rom_state_bytes(h->pcs[k]);
  }
  return RTE_OK;
}

rte_status rte_load(rte_handle h, const void* buf, size_t bytes) {
  if (!h || !buf) return RTE_EINVAL;
  CkptHead hd;
  if (bytes < sizeof(hd)) return fail(h, RTE_EINVAL, "checkpoint shorter than its header");
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, kCkptMagic, sizeof(hd.magic)) != 0 || hd.version != kCkptVersion)
    return fail(h, RTE_EINVAL, "not a checkpoint of this library version");
  if (hd.dim != h->dim || hd.nx != h->nx || hd.ny != h->ny || hd.nslot != h->L.nslot ||
      hd.dl != h->L.dl || hd.nfam != h->L.nfam || hd.precision != h->opt.precision ||
      hd.r_max != h->opt.r_max || hd.reserved != (uint32_t)(h->levels | (h->deg << 8)))
    return fail(h, RTE_EINVAL,
                "checkpoint of another mesh, direction layout, precision, r_max, pc_levels or degree");
  if (hd.c_dt != h->c_dt || hd.problem_digest != h->problem_digest)
    return fail(h, RTE_EINVAL, "checkpoint of another time step, cross sections or source");
  if (hd.bytes != bytes) return fail(h, RTE_EINVAL, "checkpoint length differs from its header");
  if (hd.fcur != 0 && hd.fcur != 1) return fail(h, RTE_EINVAL, "malformed checkpoint");
  // sizes first, so that a malformed blob changes nothing
  const unsigned char* in = static_cast<const unsigned char*>(buf) + sizeof(hd);
  const size_t left = bytes - sizeof(hd);
  const size_t fixed = state_fixed_bytes(h);
  if (left < fixed) return fail(h, RTE_EINVAL, "checkpoint truncated");
  const size_t b_ig = rom_checked_bytes(h->ig, in + fixed, left - fixed);
  size_t b_pc[RTE_MAX_PC_LEVELS] = {};
  size_t used = fixed + b_ig;
  bool ok = b_ig != 0;
  for (int k = 0; k < h->levels && ok; ++k) {
    b_pc[k] = rom_checked_bytes(h->pcs[k], in + used, left - used);
    ok = b_pc[k] != 0;
    used += b_pc[k];
  }
  if (!ok || used != left) return fail(h, RTE_EINVAL, "malformed ROM part of the checkpoint");
  TRY(sync_streams(h));
  // BDF2: the step's tau is backward Euler's before the first step, BDF2's after it (set
  // before the state is copied: a change of tau clears the FP32 refinement pair)
  if (h->bdf2) TRY(set_tau(h, hd.stats.steps > 0 ? 1.5 / h->c_dt : 1.0 / h->c_dt));
  for (const auto& p : state_parts(h)) {
    CK(cudaMemcpyAsync(p.dev, in, p.bytes, cudaMemcpyHostToDevice, h->st));
    in += p.bytes;
  }
  CK(cudaStreamSynchronize(h->st));
  CK(rom_load(h->ig, in, h->st));
  in += b_ig;
  for (int k = 0; k < h->levels; ++k) {
    CK(rom_load(h->pcs[k], in, h->st));
    in += b_pc[k];
  }
  for (int s = 0; s < 4; ++s) h->g[s] = hd.g[s];
  h->y_valid = hd.y_valid != 0;
  h->flag_ig = hd.flag_ig != 0;
  for (int k = 0; k < RTE_MAX_PC_LEVELS; ++k)
    h->flags_pc[k] = k < h->levels && (hd.flag_pc & (1 << k)) != 0;
  h->fcur = hd.fcur;
  h->bf_seed = hd.bf_seed;
  h->stats = hd.stats;
  h->pending_rom = false;
  h->rom_pend = rte_s::RomPending{};
  return RTE_OK;
}

rte_status rte_get_stats(rte_handle h, rte_stats* st) {
  if (!h || !st) return RTE_EINVAL;
  *st = h->stats;
  st->ig_rank = h->ig.rank;
  st->pc_rank = h->pc.rank;
  for (int k = 0; k < RTE_MAX_PC_LEVELS; ++k) st->pc_level_rank[k] = h->pcs[k].rank;
  if (h->dim == 2) {
    st->sweep_lanes = h->L.dl;
    st->sweep_si_rows = h->tile[0].R;
    st->sweep_si_warps = h->tile[0].W;
    st->sweep_f_rows = h->tile[1].R;
    st->sweep_f_warps = h->tile[1].W;
    st->sweep_tuned = h->tuned ? 1 : 0;
    st->sweep_si_kernel = h->tile[0].kind;
    st->sweep_f_kernel = h->tile[1].kind;
  }
  return RTE_OK;
}

const char* rte_last_error(rte_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void rte_destroy(rte_handle h) {
  if (!h) return;
  free_all(h);
  delete h;
}

// ------------------------------- operator-level calls -------------------------------

rte_status rte_op_sweep(rte_handle h, const double* rho, double* out) {
  if (!h || !rho || !out) return RTE_EINVAL;
  const int n = (int)h->ndof;
  TRY(upload(h, h->tmp, rho, n));
  TRY(set_q(h, h->tmp, nullptr));
  cudaEventRecord(h->kev0, h->st);
  TRY(sweep_q(h, nullptr));
  cudaEventRecord(h->kev1, h->st);
  TRY(sum_pm(h, h->tmp2, 0));
  TRY(check_sweep_error(h));
  {
    float kms = 0.f;
    cudaEventElapsedTime(&kms, h->kev0, h->kev1);
    h->stats.si_sweep_kernel_ms += kms;
    h->stats.si_sweep_launches += 1;
  }
  CK(cudaMemcpyAsync(out, h->tmp2, sizeof(double) * n, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return RTE_OK;
}

rte_status rte_op_fsweep(rte_handle h, const double* rho, double* btilde) {
  if (!h || !rho) return RTE_EINVAL;
  const int n = (int)h->ndof;
  TRY(upload(h, h->tmp, rho, n));
  cudaEventRecord(h->kev0, h->st);
  TRY(sweep_f(h, h->tmp, h->y));
  cudaEventRecord(h->kev1, h->st);
  h->y_valid = true;
  TRY(check_sweep_error(h));
  {
    float kms = 0.f;
    cudaEventElapsedTime(&kms, h->kev0, h->kev1);
    h->stats.f_sweep_kernel_ms += kms;
    h->stats.f_sweep_launches += 1;
  }
  if (btilde) {
    TRY(make_btilde(h));
    CK(cudaMemcpyAsync(btilde, h->btilde, sizeof(double) * n, cudaMemcpyDeviceToHost, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  return RTE_OK;
}

rte_status rte_op_dsa(rte_handle h, const double* residual, double* delta, int* iterations) {
  if (!h || !residual || !delta) return RTE_EINVAL;
  const int n = (int)h->ndof;
  TRY(upload(h, h->tmp, residual, n));
  CK(dsa_solve(h->dsa, h->sig_s, h->tmp, nullptr, h->opt.cg_rtol, h->opt.cg_max_iter, h->delta,
               nullptr, nullptr, nullptr, h->cg_iters, h->st));
  int its = 0;
  CK(cudaMemcpyAsync(&its, h->cg_iters, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(delta, h->delta, sizeof(double) * n, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (iterations) *iterations = its;
  return RTE_OK;
}

rte_status rte_op_rom_append(rte_handle h, int which, const double* x, const double* b,
                             double trunc_eps, int* grew) {
  if (!h || !x || !b || (which != RTE_ROM_IG && which != RTE_ROM_PC)) return RTE_EINVAL;
  const int n = (int)h->ndof;
  TRY(upload(h, h->tmp2, x, n));
  TRY(upload(h, h->tmp3, b, n));
  RomDev& R = which == RTE_ROM_IG ? h->ig : h->pc;
  int g = 0;
  double ratio = 0;
  CK(rom_append(R, h->tmp2, h->tmp3, trunc_eps, &g, &ratio, h->st));
  if (grew) *grew = g;
  return RTE_OK;
}

rte_status rte_op_rom_apply(rte_handle h, int which, const double* rhs, double* out) {
  if (!h || !rhs || !out || (which != RTE_ROM_IG && which != RTE_ROM_PC)) return RTE_EINVAL;
  RomDev& R = which == RTE_ROM_IG ? h->ig : h->pc;
  if (R.rank <= 0 || !R.lu_ok) return fail(h, RTE_ESTATE, "ROM is empty or its operator is singular");
  const int n = (int)h->ndof;
  TRY(upload(h, h->tmp2, rhs, n));
  CK(rom_apply(R, h->tmp2, h->tmp3, h->st));
  CK(cudaMemcpyAsync(out, h->tmp3, sizeof(double) * n, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return RTE_OK;
}

rte_status rte_op_rom_get(rte_handle h, int which, int* rank, double* S, double* U, double* Ar) {
  if (!h || (which != RTE_ROM_IG && which != RTE_ROM_PC)) return RTE_EINVAL;
  RomDev& R = which == RTE_ROM_IG ? h->ig : h->pc;
  if (rank) *rank = R.rank;
  CK(rom_get(R, S, U, Ar, h->st));
  return RTE_OK;
}

rte_status rte_dsa_solve_noalloc(int dim, int nx, int ny, double x0, double x1, double y0,
                                 double y1, double c_dt, const double* sigma_t_dev,
                                 const double* sigma_s_dev, const double* residual_dev,
                                 double cg_rtol, int cg_max_iter, double* delta_dev,
                                 int* iterations, void* stream) {
  std::string err;
  const rte_status s = dsa_solve_noalloc(dim, nx, ny, x0, x1, y0, y1, c_dt, sigma_t_dev,
                                         sigma_s_dev, residual_dev, cg_rtol, cg_max_iter,
                                         delta_dev, iterations, stream, &err);
  if (s != RTE_OK) g_create_error = err;
  return s;
}

rte_status rte_op_rom_reset(rte_handle h) {
  if (!h) return RTE_EINVAL;
  rom_reset(h->ig);
  for (int k = 0; k < h->levels; ++k) rom_reset(h->pcs[k]);
  h->flag_ig = false;
  for (bool& f : h->flags_pc) f = false;
  return RTE_OK;
}

}  // extern "C"

// =========================================================================================
// Batched instances: one full handle per problem, stepped by one host thread each.
// =========================================================================================
struct rte_batch_s {
  std::vector<rte_handle> h;
  std::vector<rte_status> status;
};

extern "C" {

rte_status rte_batch_create(rte_batch* out, int count, const rte_problem* problems,
                            const rte_options* opt) {
  if (!out) return RTE_EINVAL;
  *out = nullptr;
  if (count < 1 || count > 4096 || !problems) {
    g_create_error = "count must be in [1, 4096] and problems non-NULL";
    return RTE_EINVAL;
  }
  rte_batch b = new (std::nothrow) rte_batch_s();
  if (!b) return RTE_ENOMEM;
  b->h.assign(count, nullptr);
  b->status.assign(count, RTE_OK);
  for (int i = 0; i < count; ++i) {   // every instance's host-side checks first
    const rte_problem& p = problems[i];
    rte_s probe;
    const rte_status s = validate_impl(&probe, &p.mesh, &p.quad, p.sigma_t, p.sigma_s, p.source,
                                       p.c_dt, opt);
    if (s != RTE_OK) {
      g_create_error = "instance " + std::to_string(i) + ": " + probe.err;
      delete b;
      return s;
    }
  }
  // Sweep tiles of concurrent instances.  The per-instance tuner times each instance alone,
  // where the widest wavefront wins; beside 63 others the tile sequence with 32 directions per
  // lane group, 4-row tiles and 8 warps per CTA was measured faster for every instance on the
  // 64-instance FP32 workload (34.9 against 38.8 ms per step; 16 directions per group:
  // 45.9 ms; the strip chain: 65.4 ms).  It applies to the FP32 modes when the caller leaves
  // the sweep choice to the library; FP64 instances keep the tuner (the FP64 tile sequence is
  // slower than the strip chain).
  rte_options bopt;
  if (opt) bopt = *opt;
  else rte_default_options(&bopt);
  // The DSA solve in one thread-block cluster: with cooperative launches over every SM, an
  // instance of the 64-instance FP32 batch had a bounded grid-barrier wait run out
  // (RTE_ETIMEOUT) while the other instances' kernels, their solves among them, filled the GPU
  // (first with the FP32 solve, later with the FP64 one).  A cluster's CTAs are started
  // together by the hardware, so no solve waits on blocks that have not started.
  bopt.dsa_cluster = 1;
  bopt.dsa_fp64 = 1;
  if (bopt.precision != RTE_FP64 && bopt.tune && !bopt.sweep_kernel && !bopt.sweep_lanes &&
      !bopt.sweep_rows && !bopt.sweep_warps) {
    bopt.sweep_kernel = 2;
    bopt.sweep_lanes = 32;
    bopt.sweep_rows = 4;
    bopt.sweep_warps = 8;
  }
  for (int i = 0; i < count; ++i) {
    const rte_problem& p = problems[i];
    rte_status s = rte_create(&b->h[i], &p.mesh, &p.quad, p.sigma_t, p.sigma_s, p.source, p.c_dt,
                              &bopt);
    if (s == RTE_OK) {
      b->h[i]->blocking = true;
      if (p.rho0) {
        s = rte_set_initial(b->h[i], p.rho0, nullptr);
      } else {
        std::vector<double> z((size_t)b->h[i]->ndof, 0.0);
        s = rte_set_initial(b->h[i], z.data(), nullptr);
      }
      if (s != RTE_OK) g_create_error = b->h[i]->err;
    }
    if (s != RTE_OK) {
      g_create_error = "instance " + std::to_string(i) + ": " + g_create_error;
      rte_batch_destroy(b);
      return s;
    }
  }
  *out = b;
  return RTE_OK;
}

rte_status rte_batch_step(rte_batch b, int nsteps) {
  if (!b) return RTE_EINVAL;
  if (nsteps < 0) return RTE_EINVAL;
  const int count = (int)b->h.size();
  std::vector<std::thread> th;
  th.reserve(count);
  for (int i = 0; i < count; ++i) {
    th.emplace_back([b, i, nsteps]() {
      rte_handle h = b->h[i];
      if (cudaSetDevice(h->device) != cudaSuccess) {
        b->status[i] = RTE_ECUDA;
        return;
      }
      b->status[i] = rte_step(h, nsteps);
    });
  }
  for (auto& t : th) t.join();
  for (int i = 0; i < count; ++i)
    if (b->status[i] != RTE_OK) return b->status[i];
  return RTE_OK;
}

rte_status rte_batch_restart(rte_batch b) {
  if (!b) return RTE_EINVAL;
  for (rte_handle h : b->h) TRY(rte_restart(h));
  return RTE_OK;
}

int rte_batch_size(rte_batch b) { return b ? (int)b->h.size() : 0; }

rte_handle rte_batch_instance(rte_batch b, int i) {
  if (!b || i < 0 || i >= (int)b->h.size()) return nullptr;
  return b->h[i];
}

rte_status rte_batch_status(rte_batch b, int i) {
  if (!b || i < 0 || i >= (int)b->h.size()) return RTE_EINVAL;
  return b->status[i];
}

void rte_batch_destroy(rte_batch b) {
  if (!b) return;
  for (rte_handle h : b->h) rte_destroy(h);
  delete b;
}

}  // extern "C"
