// Internal declarations shared by the CUDA kernels and the host driver of librte.so.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rte.h"

namespace rte {

// Number of kernels launched by this library on the calling host thread (for reporting).
extern thread_local long long g_launches;

// ---------------------------------------------------------------------------------------
// Direction layout.  The directions of a 2D rule fall into four quadrants that share one
// upwind order each (Sec. 2.3: the sweep reorders cells along the upwind direction).  A
// "family" is a group of dl directions of one quadrant that one lane group of a warp
// sweeps together (lane = direction).  Slots are padded so every family has dl lanes; a
// padded slot has weight 0.  1D slabs have two half-ranges (mu > 0, mu < 0).
// ---------------------------------------------------------------------------------------
struct Layout {
  int dim = 2;
  int nv = 0;        // caller directions
  int dl = 32;       // lanes per family (power of two, <= 32)
  int nfam = 0;      // families
  int nslot = 0;     // nfam * dl
  std::vector<int> slot_of_dir;    // caller direction -> slot
  std::vector<int> fam_quadrant;   // family -> quadrant (2D: 0 (+,+) 1 (-,+) 2 (+,-) 3 (-,-); 1D: 0 (+) 1 (-))
  std::vector<double> mu, eta, w;  // per slot
};

// Control block of one strip-chain sweep launch (self-resetting: the last CTA zeroes it).
struct SweepCtrl {
  unsigned int ticket;
  unsigned int done;
  unsigned int err;      // 1: a bounded wait ran out
  unsigned int pad;
  unsigned int flags[1]; // [nfam * nblk] columns published by each row block
};

// Arguments of the 2D strip-chain sweep (Sec. 2.3 transport sweep, Q0 upwind cell solve).
template <class Real>
struct Sweep2DArgs {
  int nx, ny, nfam, nslot, nblk, rows_per_blk;
  Real tau;
  Real tau_lo;          // Q1 FP32: tau - (float)tau (the exact pair tau + tau_lo), else 0
  const Real* a;        // [nslot] |mu|/hx
  const Real* b;        // [nslot] |eta|/hy
  const Real* w;        // [nslot]
  const int* fam_quad;  // [nfam]
  const Real* sig_t;    // [ncell]
  const Real* sig_tl;   // [ncell] FP32: sigma_t - sig_t exactly (the low part), or nullptr
  const Real* inv_d;    // FP64: [nfam][ncell][dl] w / (tau + sigma_t + a + b) (Q1: the cell
                        // solve's factors, launch_q1_table); FP32: nullptr
  const unsigned* skip; // set: the launch does nothing (speculative SI-SA work past convergence)
  const Real* cth;      // [nslot] tau + a + b, high part, or nullptr (formed from tau, a, b)
  const Real* ctl;      // [nslot] its low part (FP32: the exact sum is cth + ctl)
  // K1: isotropic source q = Sigma_s rho; K2 pass A: q = Sigma_s rho + G.
  const Real* q;        // [ncell]
  const Real* g2;       // K2 pass B isotropic source G [ncell]
  Real* f;              // K2: [nfam][ncell][dl] in / out (f^{n-1} -> f^n)
  __nv_bfloat16* fb;    // BF16 mode (MODE 3 / 4): f - reference, [nfam][ncell][dl]
  const float* fro;     // BF16 mode: reference of the stored f^{n-1} [ncell]
  const float* frn;     // BF16 mode: reference of f^n [ncell] (MODE 4: = fro)
  unsigned seed;        // BF16 mode: per-launch seed of the stochastic rounding
  Real* pm;             // [nfam][ncell] partial moments (K1: of L^-1 q; K2: of pass B)
  Real gx[4], gy[4];    // per quadrant inflow ghost of pass A (K1: zero)
  Real* edge;           // [nfam][nblk][nx][dl] (K2: two planes, A then B)
  SweepCtrl* ctrl;
};

// Arguments of the 1D scan sweep (one CTA per slot).
template <class Real>
struct Sweep1DArgs {
  int nx, nslot;
  Real tau;
  const Real* a;
  const Real* w;
  const int* dir_sign;  // [nslot] +1 / -1
  const unsigned* skip; // as in Sweep2DArgs
  const Real* cth;      // [nslot] tau + a split as hi / lo (FP32), or nullptr
  const Real* ctl;
  const Real* sig_t;
  const Real* sig_tl;   // as in Sweep2DArgs
  const Real* q;        // [ncell]
  const Real* g2;       // K2 pass B source
  Real* f;              // [2][ncell][nslot/2]
  Real* psi_w;          // scratch [nslot][ncell] of w * psi (moment input)
  Real* psi_w_a;        // K2: scratch of w * f^n or nullptr
  Real g_lo, g_hi;      // inflow at x0 (for mu > 0) and x1 (for mu < 0), pass A
};

// Q1 sweeps (sweep_q1.cu), FP64 or FP32, mode 0 / 1 / 2 as in the Q0 strip chain; one warp per CTA,
// rows_per_blk = (32 / dl) R.  q, g2: [4][ncell]; f: [nfam][ncell][4][dl]; pm: [nfam][4][ncell];
// edge: per pass [nfam][nblk][nx][2][dl] (mode 1: two passes).
cudaError_t launch_sweep_q1(const Sweep2DArgs<double>& a, int mode, int dl, int R, cudaStream_t s);
cudaError_t launch_sweep_q1(const Sweep2DArgs<float>& a, int mode, int dl, int R, cudaStream_t s);
// The FP64 Q1 sweeps' table (their inv_d): the closed form's factors kS, kQ, s1, ps of every
// cell and direction slot, [nfam][ncell][4][dl] (nslot = nfam dl), for c = tau + sigma_t.
cudaError_t launch_q1_table(const double* sig_t, const double* a, const double* b, double tau,
                            int ncell, int nslot, int dl, double* out, cudaStream_t s);
// FP32: f[fam][cell][k][dl] = float(rho[k ncell + cell])
cudaError_t launch_isotropic_f32_q1(const double* rho, int ncell, int nslot, int dl, float* f,
                                    cudaStream_t s);
// f[fam][cell][k][dl] = rho[k ncell + cell] in every slot (isotropic Q1 angular flux)
cudaError_t launch_isotropic_f_q1(const double* rho, int ncell, int nslot, int dl, double* f,
                                  cudaStream_t s);

// Launchers (sweep.cu).
// Dynamic shared memory of one 2D sweep CTA (the launcher rejects more than 200 KiB).
size_t sweep2d_smem_bytes(size_t real, int dl, int R, int W, int mode, bool table);
template <class Real>
cudaError_t launch_sweep2d(const Sweep2DArgs<Real>& a, int mode, int R, cudaStream_t s);
// Tile-sequence sweep (sweep_tile.cu): TH rows per lane group, W warps per CTA,
// rows_per_blk = W (32 / dl) TH; FP32 modes 0-4, FP64 modes 0-2 (FP64 needs inv_d).
cudaError_t launch_sweep2d_tile(const Sweep2DArgs<float>& a, int mode, int th, int W,
                                cudaStream_t s);
cudaError_t launch_sweep2d_tile(const Sweep2DArgs<double>& a, int mode, int th, int W,
                                cudaStream_t s);
size_t sweep2d_tile_smem_bytes(size_t real, int dl, int th, int W, int mode);
template <class Real>
cudaError_t launch_sweep1d(const Sweep1DArgs<Real>& a, int mode, cudaStream_t s);
template <class Real>
cudaError_t launch_moment1d(const Real* psi_w, int nslot, int ncell, Real* out, cudaStream_t s,
                            const unsigned* skip = nullptr);
// inv_d = w / (tau + sigma_t + a + b) in the family layout [fam][cell][dl]
template <class Real>
cudaError_t launch_inv_d(const Real* sig_t, const Real* a, const Real* b, const Real* w, Real tau,
                         int ncell, int nslot, int dl, Real* inv_d, cudaStream_t s);

// Vector kernels (vec.cu).
struct Norms {             // device-side reduction results of one residual evaluation
  double diff_inf, half_inf, diff_l2sq, pad;
};
// conv (optional): skip word of a speculative SI-SA loop; the residual does nothing when it
// is set and otherwise sets it to the outcome of the stopping test (eps, absolute or relative).
// copy1 / copy2 (optional): further destinations of rho^{l-1/2}.
// loop.count (optional): iteration counter of a CUDA graph's while loop around the SI
// iteration; the residual adds one and sets loop.cond to 1 while the stopping test fails, the
// counter is below loop.limit and neither error word (optional: the sweep's and the CG's
// bounded waits) is set, else to 0.  A residual skipped on a set skip word sets it to 0.
struct ResidualLoop {
  cudaGraphConditionalHandle cond;
  unsigned* count;
  unsigned limit;
  const unsigned* err0;
  const unsigned* err1;
};
cudaError_t launch_combine_residual(const double* pm, int nfam, const double* btilde,
                                    const double* rho_prev, int ncell, double* rho_half,
                                    double* partials, int nblocks, Norms* out, cudaStream_t s,
                                    unsigned* conv = nullptr, double eps = 0.0, int absmode = 0,
                                    double* copy1 = nullptr, double* copy2 = nullptr,
                                    unsigned* ticket = nullptr,
                                    ResidualLoop loop = ResidualLoop{0, nullptr, 0, nullptr, nullptr});
// ticket: a zeroed device word; the residual kernel's last block forms the norms and the
// stopping test and zeroes it again.
// Start of an SI-SA solve: src -> dst1 (and dst2 when given), *conv = 0, slots[0..nslots) = 0.
cudaError_t launch_si_begin(const double* src, double* dst1, double* dst2, int ncell,
                            unsigned* conv, int* slots, int nslots, cudaStream_t s);
cudaError_t launch_update_rho(const double* rho_half, const double* delta, const double* sig_s,
                              int ncell, double* rho, double* q, cudaStream_t s);
cudaError_t launch_scale_copy(const double* x, const double* sig_s, int ncell, double* q,
                              cudaStream_t s);
cudaError_t launch_sum_partials(const double* pm, int nfam, int ncell, const double* add,
                                double* out, cudaStream_t s);
cudaError_t launch_axpby(double alpha, const double* x, double beta, const double* y, int n,
                         double* out, cudaStream_t s);
// f = rho in every slot, times w of the slot when w is given (the 2D FP64 storage w f)
cudaError_t launch_isotropic_f(const double* rho, int ncell, int nslot, int dl, const double* w,
                               double* f, cudaStream_t s);
cudaError_t launch_dot(const double* x, const double* y, int n, double* partials, int nblocks,
                       double* out, cudaStream_t s);
int vec_blocks(int n);
cudaError_t launch_rom_gate(const double* e2, const double* n2, double eps_up, int rel, int force,
                            const int* also, int* gate, cudaStream_t s);
// Sources of the sweeps in their precision (FP32 mode: float).
template <class Real>
// Real(sigma_s (x - xref)); skip: a set skip word makes the launch do nothing
cudaError_t launch_scaled_diff(const double* x, const double* xref, const double* sig_s, int n,
                               Real* out, cudaStream_t s, const unsigned* skip = nullptr);
template <class Real>
// the same, then xref <- x
cudaError_t launch_scaled_diff_update(const double* x, double* xref, const double* sig_s, int n,
                                      Real* out, cudaStream_t s, const unsigned* skip = nullptr);
template <class Real>
cudaError_t launch_scaled_plus(const double* rho, const double* sig_s, const double* src, int n,
                               Real* out, cudaStream_t s);        // Real(sigma_s rho + G)
template <class Real>
// out (+)= sum_f pm, in FP64
cudaError_t launch_sum_pm(const Real* pm, int nfam, int n, double* out, int accumulate,
                          cudaStream_t s, const unsigned* skip = nullptr);
cudaError_t launch_isotropic_f32(const double* rho, int n, int nslot, int dl, float* f,
                                 cudaStream_t s);
cudaError_t launch_to_float(const double* x, long n, float* y, cudaStream_t s);
// BDF2 (options.time_scheme): f <- (4 f - prev) / 3 and prev <- the old f, elementwise
template <class Real>
cudaError_t launch_bdf2_history(Real* f, Real* prev, long n, cudaStream_t s);

// DSA (cg.cu): 5-point (1D: 3-point) diffusion operator with Marshak vacuum faces.
struct DsaOp {
  int nx, ny, n;  // n: unknowns (Q0: cells; Q1: 4 modes per cell, mode-major)
  int ncell, deg;
  bool f32;       // vectors, coefficients and their arithmetic in FP32 (dots and scalars FP64)
  // coefficients and CG vectors, in FP64 or (f32) FP32 storage
  void* diag;     // Q0 [n]
  void* cx;       // Q0 [n] coupling of cell c with c+1 (0 at the east edge)
  void* cy;       // Q0 [n] coupling of cell c with c+nx (0 at the north edge / 1D)
  void* blk;      // Q1 [14][ncell] block coefficients
  void* dinv;     // Q1 [n] inverse diagonal (the Jacobi preconditioner)
  void *r, *p0, *p1, *ap, *x;
  void *r1, *w1, *s1;   // second buffers of the single-barrier CG (r, w = C r, s = C p)
  double* partial;   // [3 * blocks]
  double* scal;      // [8] device scalars
  int blocks;
  bool single_phase;   // cg1_kernel (one barrier per iteration) instead of cg_kernel
  bool cluster;        // cg_cluster_kernel: the solve in one thread-block cluster (Q0)
};
// max_blocks > 0 caps the blocks of the cooperative CG launch (default: one or two per SM).
// degree 1: the Q1 interior-penalty operator (2D) on mode-major vectors of 4 nx ny values.
// f32: the solve's vectors and operator arithmetic in FP32, dot products and CG scalars in
// FP64 (the FP32 modes; the solve's inputs and outputs stay FP64).
// cluster: the Q0 solve in one thread-block cluster instead of a cooperative launch over the
// GPU (max_blocks then has no effect; the Q1 solve ignores it).
cudaError_t dsa_setup(DsaOp& op, int dim, int nx, int ny, double hx, double hy, double tau,
                      const double* sig_t_host, const double* sig_s_host, cudaStream_t s,
                      int max_blocks = 0, int degree = 0, bool f32 = false, bool cluster = false);
void dsa_free(DsaOp& op);
// delta = C^{-1} (sig_s .* (residual - residual_b)) (residual_b may be nullptr);
// rho_out = rho_half + delta and q_out = sig_s .* rho_out when rho_out != nullptr.
// Iteration count to *iters_dev (device int).
cudaError_t dsa_solve(DsaOp& op, const double* sig_s, const double* residual,
                      const double* residual_b, double rtol, int max_iter, double* delta,
                      const double* rho_half, double* rho_out, double* q_out, int* iters_dev,
                      cudaStream_t s, const unsigned* skip = nullptr, int iters_add = 0);

// Allocation-free DSA solve behind rte_dsa_solve_noalloc (cg.cu); *err receives the message.
rte_status dsa_solve_noalloc(int dim, int nx, int ny, double x0, double x1, double y0, double y1,
                             double c_dt, const double* sigma_t_dev, const double* sigma_s_dev,
                             const double* residual_dev, double cg_rtol, int cg_max_iter,
                             double* delta_dev, int* iterations, void* stream, std::string* err);

// ROM (rom.cu).
struct RomDev {
  int n, r_max, rank;
  int wu, ww;     // columns in use of U0 and W0
  double* U;      // U0: [WCAP][n] column-major (column k at U + k*n); U = U0 Q
  double* W;      // W0: [WCAP][n]; W = W0 P (W = B V)
  double* Utmp;   // [WCAP][n]
  double* Wtmp;   // [WCAP][n]
  double *Q, *P, *Qtmp, *Ptmp;   // [WCAP][65] row-major small factors
  double* S;      // [r_max+1]
  double* core;   // small workspace
  double* lu;     // [r_max*r_max] A_r^{-1}, row-major
  int* piv;
  double* proj;   // [2*(r_max+1)] projections and reduced coordinates
  double* partial;
  double* sec;    // scratch of the core SVD
  double* dstate; // [8] outcome of the last append (device), see rom_append_async
  double* hstate; // [8] pinned host copy of it
  int lu_ok;
};
// SVD of the core [[diag(S), p], [0, alpha]] (csvd.cu); alpha^2 and ||x||^2 in sc[1], sc[0];
// writes U_c, V_c, the new singular values, and keep / grew / ratio into sc[3..6].
long secular_scratch_doubles();
cudaError_t core_svd_secular(const double* S, int r, const double* p, double* sc, double* Uc,
                             double* Vc, double* snew, double trunc_eps, int r_max,
                             double* scratch, cudaStream_t s);
cudaError_t rom_alloc(RomDev& R, int n, int r_max);
void rom_free(RomDev& R);
void rom_reset(RomDev& R);   // empty ROM (rank 0), keeps the allocation
// Incremental SVD append (App. B), synchronous: updates the host view (rank, columns in
// use, lu_ok) before returning, with the grew flag and the stop ratio s_last / sum s.
cudaError_t rom_append(RomDev& R, const double* x, const double* b, double trunc_eps,
                       int* grew, double* smallest_ratio, cudaStream_t s);
// The same append queued without any host wait.  gate: device int, 0 = leave the ROM as it
// is (the work still runs, into scratch), nullptr = always.  The host view is stale until
// rom_commit runs after the stream has passed the append.
cudaError_t rom_append_async(RomDev& R, const double* x, const double* b, double trunc_eps,
                             const int* gate, cudaStream_t s);
// Folds the outcome of the last rom_append_async into the host view (compacting the factored
// bases when full, queued on s); ran = the gate was open.
cudaError_t rom_commit(RomDev& R, int* ran, int* grew, double* smallest_ratio, cudaStream_t s);
// out = U A_r^{-1} U^T rhs.  Returns cudaErrorInvalidValue if the LU is not available.
cudaError_t rom_apply(RomDev& R, const double* rhs, double* out, cudaStream_t s);
cudaError_t rom_get(RomDev& R, double* S, double* U, double* Ar, cudaStream_t s);
// Checkpoint of one ROM's state (host counters and device arrays) in host memory.
// rom_checked_bytes: bytes of the checkpoint at `in`, 0 when it is malformed or longer than
// avail; rom_load reads a checkpoint that rom_checked_bytes accepted.
size_t rom_state_bytes(const RomDev& R);
cudaError_t rom_save(const RomDev& R, unsigned char* out, cudaStream_t s);
size_t rom_checked_bytes(const RomDev& R, const unsigned char* in, size_t avail);
cudaError_t rom_load(RomDev& R, const unsigned char* in, cudaStream_t s);

}  // namespace rte
