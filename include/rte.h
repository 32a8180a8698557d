/*
 * rte.h -- C ABI of the GB300-native ROM-accelerated SI-DSA library (librte.so).
 *
 * Method: N. Liu and Z. Peng, "On-the-fly ROM-based acceleration of SI-DSA for implicit
 * time marching of the radiative transfer equation".  The library solves the one-group
 * linear RTE with isotropic scattering and isotropic inflow (Sec. 2, Eq. (rte)) with
 *   - S_N directions (Sec. 2.1; Gauss-Legendre in 1D, Chebyshev-Legendre CL rule of App. A),
 *   - backward Euler in time (Sec. 2.1, Eq. (time_discrete)), tau = 1/(c dt),
 *   - upwind DG in space, Eq. (DG): the Q0 member of Eq. (dg_space) (one value per cell), or
 *     with options.degree = 1 the Q1 member the paper computes with (bilinear functions on
 *     each rectangle, 2D) and an interior-penalty DSA on the same space,
 *   - memory-efficient SI with DSA (Sec. 2.3, Algorithm 1),
 *   - on-the-fly DMD / incremental-SVD reduced models for the initial guess and the
 *     first-iteration preconditioner (Sec. 3, Algorithm 2, App. B).
 * Everything on the time-stepping path runs in CUDA kernels on one GPU (sm_103a); the host
 * side only sequences them.
 *
 * Conventions (all calls):
 *   - Every call returns rte_status; nothing throws or aborts across the ABI.  On failure
 *     rte_last_error(h) returns a NUL-terminated message owned by the handle; after a failed
 *     rte_create, rte_last_error(NULL) returns that call's message (per host thread).
 *   - Array arguments are HOST pointers unless the name ends in _dev.  Input arrays are
 *     copied during the call; the caller keeps ownership of every pointer it passes.
 *   - Cell arrays have ncell = nx*ny entries, cell index c = i + nx*j (x fastest), FP64,
 *     whatever the internal precision.
 *   - Arrays over the degrees of freedom (the source, rho0, scalar fluxes, residuals and ROM
 *     snapshots) have ndof entries: ndof = ncell for degree 0; for degree 1, ndof = 4 ncell,
 *     mode-major: mode k of cell c at k*ncell + c, where mode k = a + 2b is the coefficient of
 *     p_a(xi) p_b(zeta), p_0 = 1, p_1 = sqrt(3) t, in the cell's local coordinates
 *     xi, zeta in [-1, 1] (orthonormal under the cell average: mode 0 is the cell average).
 *     sigma_t and sigma_s are per cell in both.
 *   - Angular arrays are [n_dirs][ndof], direction order = the order rte_get_quadrature
 *     reports (for RTE_Q_EXPLICIT: the caller's order).
 *   - A handle is not thread-safe; use one handle per host thread.  All device work of a
 *     handle is issued on its own CUDA streams (or, after rte_set_stream, on the caller's
 *     stream and the handle's side streams) on the device that was current at create.
 */
#ifndef RTE_H
#define RTE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rte_s* rte_handle;

typedef enum {
  RTE_OK = 0,
  RTE_EINVAL = 1,   /* invalid argument (detail in rte_last_error) */
  RTE_ENOMEM = 2,   /* host or device allocation failed */
  RTE_ENOCONV = 3,  /* SI-SA reached max_iter; state = last iterate, still usable */
  RTE_ECUDA = 4,    /* a CUDA runtime call failed */
  RTE_ETIMEOUT = 5, /* a bounded device-side wait ran out (the kernel returned early) */
  RTE_ESTATE = 6    /* call not valid in the handle's current state */
} rte_status;

enum { RTE_Q_GL1D = 0, RTE_Q_CL_HEMI = 1, RTE_Q_EXPLICIT = 2 };
enum { RTE_FP64 = 0, RTE_FP32 = 1, RTE_FP32_BF16F = 2 };
enum { RTE_REL_INF = 0, RTE_ABS_INF = 1 };
enum { RTE_ROM_OFF = 0, RTE_ROM_AUTO = 1, RTE_ROM_MANUAL = 2 };
enum { RTE_ROM_IG = 0, RTE_ROM_PC = 1 };
#define RTE_MAX_PC_LEVELS 4   /* preconditioner ROMs: one per SI iteration l = 1 .. 4 at most */
enum { RTE_SA_DSA = 0, RTE_SA_DMD_ITER = 1 };
enum { RTE_BE = 0, RTE_BDF2 = 1 };

/* Uniform Cartesian mesh.  dim = 1: slab [x0,x1] with nx cells (ny must be 1);
 * dim = 2: [x0,x1] x [y0,y1] with nx*ny rectangles (Sec. 2.1). */
typedef struct {
  int dim;
  int nx, ny;
  double x0, x1, y0, y1;
} rte_mesh;

/* Angular quadrature (Sec. 2.1: weights sum to 1).
 *   RTE_Q_GL1D    n_gl-point Gauss-Legendre rule in mu, weights / 2 (dim = 1).
 *   RTE_Q_CL_HEMI CL(n_phi, n_gl) rule of App. A restricted to v_z > 0 with doubled
 *                 weights (X-Y geometry); n_gl even; n_dirs = n_phi * n_gl / 2 (dim = 2).
 *   RTE_Q_EXPLICIT n_dirs directions mu[], eta[] (eta ignored for dim = 1), weights w[].
 *                 2D rules need the same number of directions in each quadrant and no
 *                 direction on an axis; 1D rules the same number with mu > 0 and mu < 0. */
typedef struct {
  int kind;
  int n_gl;
  int n_phi;
  int n_dirs;
  const double* mu;
  const double* eta;
  const double* w;
} rte_quadrature;

typedef struct {
  double eps_sisa;   /* Algorithm 1 stopping tolerance (default 1e-8) */
  double eps_ig;     /* Phase 1 stop Eq. (ig_stop) and IG-ROM truncation (default 1e-6) */
  double eps_pc;     /* Phase 2 stop Eq. (pc_stop) and PC-ROM truncation (default 1e-6) */
  double eps_up;     /* Phase 3 update indicators, Sec. 3.2 (default 1e-6) */
  int max_iter;      /* N_iter of Algorithm 1 (default 500) */
  int r_max;         /* rank cap of each ROM, <= 64 (default 40) */
  int precision;     /* RTE_FP64 (default) | RTE_FP32: sweeps and f in FP32, the SI residual,
                        DSA and ROMs in FP64 (iterative refinement of the SI increments) |
                        RTE_FP32_BF16F (2D): as RTE_FP32 with f stored as a per-cell FP32
                        reference plus BF16 remainders (stochastic rounding) */
  int rom;           /* RTE_ROM_AUTO (default) | RTE_ROM_OFF | RTE_ROM_MANUAL */
  int residual_norm; /* RTE_REL_INF (default): ||.||_inf relative to ||rho^{l-1/2}||_inf;
                        RTE_ABS_INF: the paper's absolute test */
  int up_rel;        /* 1 (default): eps_up multiplies ||rho^n||_2; 0: absolute */
  double cg_rtol;    /* DSA conjugate-gradient tolerance ||r|| <= cg_rtol ||b|| (default 1e-6) */
  int cg_max_iter;   /* default 500 */
  int tune;          /* 1 (default): pick sweep tile shapes by timing at create; 0: heuristic */
  int sweep_rows;    /* 2D sweep: rows per lane group, 1, 2, 4 or 8 (0 = automatic); the tile
                        sequence takes 2 (FP32 modes), 4 or 8 */
  int sweep_lanes;   /* 2D sweep: directions per lane group, 8, 16 or 32; also 2 in RTE_FP64
                        and with degree 1, 4 in RTE_FP64, RTE_FP32 and with degree 1
                        (0 = automatic) */
  int sweep_warps;   /* 2D sweep: warps per CTA, 1..8 (0 = automatic); reduced to fit shared memory */
  int sweep_kernel;  /* 2D sweep kernel: 0 measured choice (with tune), 1 strip chain, 2 tile
                        sequence (sweep_rows then = rows per tile: 2 in the FP32 modes, 4 or 8) */
  int lookahead;     /* 1: queue SI iteration l+1 before reading the stopping test of l (work
                        past convergence skips itself on the device); 0 (default): wait first */
  int pc_levels;     /* preconditioner ROMs, one for each of the first pc_levels SI iterations
                        (1 .. RTE_MAX_PC_LEVELS; default 1, Algorithm 2 as printed).  The ROM of
                        iteration l maps the residual rho^{n,(l-1/2)} - rho^{n,(l-1)} to the
                        correction rho^n - rho^{n,(l-1/2)}; it is built only from steps that
                        already applied the ROMs of iterations 1 .. l-1 (Sec. 3.2, key feature
                        1), Phase 3 begins once all are built, and in Phase 3 each is updated
                        when the IG-ROM or an earlier iteration's ROM was updated in the same
                        step, or when its own indicator exceeds eps_up */
  int sa_kind;       /* the SA steps that are not ROM corrections: RTE_SA_DSA (default, Eq.
                        (rho_residual)) | RTE_SA_DMD_ITER: the DMD-across-iterations
                        acceleration the paper combines with its ROMs in place of DSA (Sec. 4,
                        compared in Sec. 3.3): plain SI steps collect mh_window residuals
                        r_l = rho^{l-1/2} - rho^{l-1}, then the iterate jumps to
                        rho^{l-1} + C_r^{-1} r_l with C_r the DMD reduced operator of
                        I - T Sigma_s from the pairs (r_l, r_l - r_{l+1}); lookahead is off */
  int mh_window;     /* residuals per DMD-across-iterations cycle, 2 .. 16 (default 4) */
  int cg_blocks;     /* blocks of the DSA solve's cooperative CG launch: 0 (default) one per SM
                        (two above 2^18 cells); a cap leaves the other SMs to concurrent work
                        at the price of a longer solve; no effect with dsa_cluster = 1 */
  int time_scheme;   /* RTE_BE (default): backward Euler, Sec. 2.1 | RTE_BDF2: the second-order
                        backward difference formula Sec. 2.1 names as an alternative: the step's
                        system is backward Euler's with tau' = 3 / (2 c dt) and the history
                        (4 f^{n-1} - f^{n-2}) / 3 in place of f^{n-1}; the first step (after
                        rte_set_initial, rte_restart) is a backward-Euler step of c_dt and gives
                        the ROMs no snapshot.  Each step sweeps once more (b~ of the next step
                        from the history).  Not with RTE_FP32_BF16F. */
  int degree;        /* K of the DG space Eq. (dg_space): 0 (default) one value per cell, or 1
                        (2D; RTE_FP64, or RTE_FP32 with FP32 sweeps and f refined by the FP64
                        residual as for degree 0): bilinear functions per rectangle with the upwind flux
                        of Eq. (DG), four unknowns per cell-direction solved together in the
                        sweeps, and a DSA by the symmetric interior-penalty discretisation of
                        the diffusion correction on the same space (penalty
                        max(2 (D_L + D_R) / h, 1/4) per face, Marshak condition taken weakly).
                        The paper's own fully consistent DSA is given by citation only. */
  int dsa_fp64;      /* 1: solve the DSA system in FP64 in the FP32 modes too; 0 (default): in
                        the FP32 modes its vectors and operator are FP32 (dot products and CG
                        scalars FP64).  Batched instances always take 1. */
  int graph;         /* 1: each SI iteration after its stopping test (the DSA solve of l, the
                        sweep and the residual of l + 1) runs as one CUDA graph, captured from
                        the handle's stream the first time iteration l is reached and replayed
                        in every later step (a new time step constant, as the first BDF2 step
                        after a restart sets, captures them again); the ROM-preconditioned
                        iterations and the steps of RTE_SA_DMD_ITER are launched one by one.
                        2: as 1, and once the iterations left are all DSA steps (from
                        iteration pc_levels on), they run as one graph whose while node
                        repeats the iteration until the stopping test of Algorithm 1 (or
                        max_iter) ends it on the device: one host wait for all of them
                        (with lookahead = 1, as 1).
                        The stream given to rte_set_stream must then be a created stream, not
                        the legacy default stream (RTE_ECUDA otherwise).  The statistics'
                        device times (time_sweep_ms, time_dsa_ms, si_sweep_kernel_ms) then
                        leave out the work inside the graphs.  0 (default): launch every kernel
                        one by one. */
  int dsa_cluster;   /* 1: the DSA solve (degree 0) runs in one thread-block cluster of 8 CTAs
                        instead of a cooperative launch over every SM: slower when the solve
                        has the GPU to itself (measured 3.9 against 0.7 ms at 512^2), but the
                        hardware starts the cluster's CTAs together, so a solve never waits at
                        its barrier on blocks that concurrent kernels keep off the SMs (two
                        cooperative solves running beside each other and other work can each
                        hold part of their blocks and wait on the rest until the bounded wait
                        runs out, RTE_ETIMEOUT).  The same CG iteration as the two-phase
                        cooperative solve; degree 1 keeps its cooperative solve.  Batched
                        instances always take 1.  0 (default): cooperative launch. */
} rte_options;

typedef struct {
  int steps;            /* time steps taken */
  int phase;            /* 1, 2 or 3 (Sec. 3.2); 0 with ROM off */
  int last_iterations;  /* SI-SA iterations of the last step */
  int last_cg_iterations;
  long long total_iterations;
  long long total_sweeps;   /* counted as in Sec. 4: 1 (b~) + iterations + 1 (f) per step */
  long long total_cg_iterations;
  int ig_rank, pc_rank;
  int ig_updated, pc_updated;  /* last step */
  double last_residual;        /* final ||rho^{l-1/2} - rho^{l-1}||_inf (relative if REL_INF) */
  double last_ig_error;        /* ||rho_DMD^{n,(0)} - rho^n||_2, NaN when not applied */
  double last_pc_error;        /* ||delta_rho_DMD^{n,(1)} - delta_rho^{n,(1)}||_2, NaN when not applied */
  long long cell_direction_updates; /* upwind cell solves done (Sec. 4 sweeps x N_x N_v) */
  double time_sweep_ms, time_dsa_ms, time_rom_ms, time_total_ms; /* device time by phase */
  long long si_sweep_launches;  /* SI sweep kernels (one application of T Sigma_s each) */
  double si_sweep_kernel_ms;    /* their summed duration, CUDA events around each launch */
  long long f_sweep_launches;   /* fused end-of-step sweeps (two cell solves per cell-direction) */
  double f_sweep_kernel_ms;
  long long kernel_launches;    /* CUDA kernels this library launched inside rte_step / rte_rom_update */
  /* 2D sweep tiling in use: directions per lane group, then rows per lane group and warps
   * per CTA of the SI sweep and of the fused f sweep; sweep_tuned = 1 when measured */
  int sweep_lanes, sweep_si_rows, sweep_si_warps, sweep_f_rows, sweep_f_warps, sweep_tuned;
  int sweep_si_kernel, sweep_f_kernel;   /* 1 strip chain, 2 tile sequence, 3 Q1 strip chain */
  /* rank of the preconditioner ROM of each SI iteration l (index l - 1) and whether it was
   * updated in the last step (the l = 1 entries repeat pc_rank and pc_updated) */
  int pc_level_rank[RTE_MAX_PC_LEVELS];
  int pc_level_updated[RTE_MAX_PC_LEVELS];
  long long total_mh_jumps;     /* DMD-across-iterations jumps (sa_kind = RTE_SA_DMD_ITER) */
} rte_stats;

/* Fill *opt with the defaults listed above. */
void rte_default_options(rte_options* opt);

/* Create a problem (Sec. 2 Eq. (rte), data of Eq. (kinetic_dg_discrete)).
 * sigma_t, sigma_s: host [ncell]; source: host [ndof] (its modes for degree 1); requires
 * finite values, sigma_s >= 0,
 * sigma_t >= sigma_s (Sec. 2), c_dt > 0, quadrature weights summing to 1 within 1e-12.
 * opt may be NULL (defaults).  Initial state: f^0 = 0, vacuum inflow.
 * On success *out owns all device memory; on failure *out = NULL. */
rte_status rte_create(rte_handle* out, const rte_mesh* mesh, const rte_quadrature* quad,
                      const double* sigma_t, const double* sigma_s, const double* source,
                      double c_dt, const rte_options* opt);

/* Initial state: f^0_j = rho0 for every direction j (isotropic) when f0 == NULL, else
 * f^0 = f0 [n_dirs][ndof] and rho0 [ndof] is ignored (may be NULL).  Resets the step counter,
 * statistics and both ROMs. */
rte_status rte_set_initial(rte_handle h, const double* rho0, const double* f0);

/* Isotropic inflow value per side, g = {west, east, south, north} (Eq. (boundary));
 * 1D uses west and east.  Applies from the next step on. */
rte_status rte_set_inflow(rte_handle h, const double g[4]);

/* Issue all further device work of h on the caller's CUDA stream (a cudaStream_t of the
 * handle's device, e.g. a torch stream); NULL returns to the handle's own stream.  The
 * handle does not take ownership; the stream must outlive its use by h.  The ROM update
 * runs beside the fused f sweep on two side streams of the lowest priority, and the handle's
 * own stream has the highest; give the caller's stream a high priority as well, or the ROM
 * work competes with the sweep for SMs on equal terms. */
rte_status rte_set_stream(rte_handle h, void* cuda_stream);

/* Return to the state given by the last rte_set_initial (kept on the device): step counter,
 * statistics and ROMs reset, no host-device copy.  RTE_ESTATE before any rte_set_initial. */
rte_status rte_restart(rte_handle h);

/* Advance nsteps implicit steps (Algorithm 2 per step).  With rom = RTE_ROM_AUTO the ROM
 * construction/update of each step runs inside; with RTE_ROM_MANUAL it runs only when the
 * caller calls rte_rom_update after a step.  RTE_ENOCONV leaves the last iterate as rho^n. */
rte_status rte_step(rte_handle h, int nsteps);

/* ROM construction / adaptive update for the step just taken (the ROM branch of
 * Algorithm 2).  RTE_ESTATE unless rom == RTE_ROM_MANUAL and a step has been taken
 * since the last call. */
rte_status rte_rom_update(rte_handle h);

/* Copy rho^n (host [ndof]). */
rte_status rte_get_scalar_flux(rte_handle h, double* rho);
/* Copy f^n (host [n_dirs][ndof]). */
rte_status rte_get_angular_flux(rte_handle h, double* f);
/* Copy the directions and weights in the library's direction order (host [n_dirs] each). */
rte_status rte_get_quadrature(rte_handle h, int* n_dirs, double* mu, double* eta, double* w);
/* The angular rule a quadrature description gives for dim (1 or 2), host-side only (no
 * device is needed): *n_dirs receives the direction count; mu, eta, w (host [n_dirs] each,
 * any may be NULL, e.g. to query the count first) the directions and weights in the order
 * rte_create and rte_get_quadrature use.  The layout conditions rte_create adds for explicit
 * rules (equal quadrant counts, no direction on an axis) are not checked here.
 * Errors: RTE_EINVAL, message from rte_last_error(NULL). */
rte_status rte_quadrature_rule(const rte_quadrature* quad, int dim, int* n_dirs, double* mu,
                               double* eta, double* w);
rte_status rte_get_stats(rte_handle h, rte_stats* st);
const char* rte_last_error(rte_handle h);
/* Free everything; NULL-safe. */
void rte_destroy(rte_handle h);

/* ---------------- checkpoint and resume ----------------
 * The paper has no counterpart: these calls let a long march stop and resume.  rte_save
 * writes what a step reads from the previous one into a caller-owned host buffer of
 * rte_save_size bytes: f^n in the handle's storage precision, rho^n, the next step's b~
 * without inflow, the FP32 refinement pair, both ROMs with their phase flags, the inflow
 * values and the statistics.  rte_load restores such a blob into a handle created with the
 * same mesh, quadrature, cross sections, source, c_dt and options; the mesh, the direction
 * layout, the precision, r_max, c_dt and a 64-bit digest (FNV-1a) of the cross sections and
 * the source are checked, the other options are the caller's to keep equal.
 *   - The loaded march repeats the saved one bit for bit when the sweep configuration is
 *     also the same.  rte_stats reports it in its sweep_* fields.  It is the same within one
 *     process, where the measured choice is cached.  Fix it with the sweep_* options to
 *     resume in another process.
 *   - rte_restart still returns to the handle's own last rte_set_initial.
 * Errors: RTE_EINVAL for a buffer smaller than rte_save_size, or for a blob that is of
 * another problem or layout, truncated or malformed (the handle is then left unchanged);
 * RTE_ESTATE for rte_save while an RTE_ROM_MANUAL update is pending; RTE_ECUDA. */
rte_status rte_save_size(rte_handle h, size_t* bytes);
rte_status rte_save(rte_handle h, void* buf, size_t bytes);
rte_status rte_load(rte_handle h, const void* buf, size_t bytes);   /* bytes: the blob's length */

/* ---------------- operator-level calls (one hot-path step each) ----------------
 * These run exactly one step of the method on the handle's problem with host arrays in
 * and out, so that each kernel can be checked on its own.  They do not advance time. */

/* out = T Sigma_s rho (Sec. 2.3 Eq. (SI_rho) without b~): one SI sweep with zero inflow and
 * the quadrature moment, in the handle's precision. */
rte_status rte_op_sweep(rte_handle h, const double* rho, double* out);

/* The fused sweep that ends a step (Eq. (sweep_to_obtain_f) then Eq.
 * (implicit_linear_system_rho)): with the handle's current f (= f^{n-1}) and the given rho
 * (= rho^n), f <- L^{-1}(Sigma_s rho + tau f + G + g^bc) in place, and
 * btilde = sum_j w_j L_j^{-1}(tau f_j + G + g_j^bc) with the updated f.  btilde may be NULL. */
rte_status rte_op_fsweep(rte_handle h, const double* rho, double* btilde);

/* delta = C^{-1} Sigma_s residual (Eq. (rho_residual)) by conjugate gradients;
 * *iterations (may be NULL) receives the CG count. */
rte_status rte_op_dsa(rte_handle h, const double* residual, double* delta, int* iterations);

/* Append the snapshot pair (x, b) to ROM `which` (RTE_ROM_IG / RTE_ROM_PC) by the
 * incremental SVD of App. B; trunc_eps < 0 means no truncation (rank cap r_max still holds).
 * *grew (may be NULL) = 1 when the rank grew. */
rte_status rte_op_rom_append(rte_handle h, int which, const double* x, const double* b,
                             double trunc_eps, int* grew);
/* out = U c with A_r c = U^T rhs (Eq. (dmd-ig) / Eq. (dmd-sa)) for ROM `which`. */
rte_status rte_op_rom_apply(rte_handle h, int which, const double* rhs, double* out);
/* Rank, singular values (descending, [rank]) and optionally U ([rank][ndof]) and the
 * reduced operator A_r = U^T W S^{-1} ([rank][rank], row-major); NULL skips an output. */
rte_status rte_op_rom_get(rte_handle h, int which, int* rank, double* S, double* U, double* Ar);
/* Drop both ROMs and the phase flags. */
rte_status rte_op_rom_reset(rte_handle h);

/* ---------------- allocation-free diffusion solve ----------------
 * The paper has no counterpart of this call: it is a service for callers that cannot
 * allocate device memory, such as code running inside another framework's fixed,
 * pre-reserved memory budget (where a cudaMalloc can fail) or latency-critical code that
 * must not trigger the device-wide synchronisation of cudaMalloc / cudaFree.
 *
 * It computes the same diffusion correction as rte_op_dsa: delta solves C delta =
 * sigma_s .* residual, where C is the handle's cell-centred diffusion operator for the mesh
 * [x0,x1] x [y0,y1] with nx * ny cells (dim = 1: ny = 1) and time step c_dt, by conjugate
 * gradients from zero until ||r|| <= cg_rtol ||b||, on the stream `stream` (a
 * cudaStream_t, NULL = the legacy default stream) of the current device.
 *   - sigma_t_dev, sigma_s_dev, residual_dev: device [nx*ny] inputs; delta_dev: device
 *     [nx*ny] output; all owned by the caller.  *iterations (host, may be NULL) = CG count.
 *   - All scratch (operator coefficients, CG vectors, reduction and barrier words) lives in
 *     one library-owned device array of fixed size, which every GPU that loads the library
 *     holds until the process exits.  nx * ny above 65536 is rejected with RTE_EINVAL.
 *   - Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.  Each call
 *     looks up the array's device address on the current device (cudaGetSymbolAddress).
 *   - Every call shares the one array and leaves the last call's contents in it; calls whose
 *     work overlaps on the GPU (other streams, other host threads) race on it.
 *   - The call blocks: it waits for its stream to finish the solve before returning.
 * Errors: RTE_EINVAL (sizes, NULL pointers), RTE_ECUDA, RTE_ETIMEOUT; the message is
 * available from rte_last_error(NULL) on the calling thread. */
rte_status rte_dsa_solve_noalloc(int dim, int nx, int ny, double x0, double x1, double y0,
                                 double y1, double c_dt, const double* sigma_t_dev,
                                 const double* sigma_s_dev, const double* residual_dev,
                                 double cg_rtol, int cg_max_iter, double* delta_dev,
                                 int* iterations, void* stream);

/* ---------------------------------------------------------------------------------------
 * Batched instances.  Many independent problems (their own grid, quadrature, cross
 * sections, c_dt and initial flux) marched side by side on one GPU: every instance is a
 * full rte_handle on its own CUDA streams, and rte_batch_step steps all of them
 * concurrently, one host thread per instance, so that their kernels overlap on the device
 * (small grids leave most SMs idle on their own).  Algorithm 2 runs per instance, exactly
 * as rte_step would run it.  Set CUDA_DEVICE_MAX_CONNECTIONS=32 in the environment before
 * the process creates its CUDA context: with the default 8 hardware queues the instances'
 * streams share queues and their kernels serialise (64 instances: 66 -> 39 ms per step).
 * ------------------------------------------------------------------------------------- */
typedef struct rte_batch_s* rte_batch;

typedef struct {
  rte_mesh mesh;
  rte_quadrature quad;
  const double* sigma_t;   /* host [ncell] */
  const double* sigma_s;   /* host [ncell] */
  const double* source;    /* host [ndof] */
  const double* rho0;      /* host [ndof]: isotropic initial flux f0 = rho0, or NULL (zero) */
  double c_dt;
} rte_problem;

/* Create `count` instances (1 .. 4096) with the same options (NULL = defaults).  In the FP32
 * modes, when the options leave the sweep choice to the library, every instance takes the
 * tile sequence with 32 directions per lane group, 4-row tiles and 8 warps per CTA (measured
 * faster beside other instances than each instance's own tuning, which times it alone).  Every
 * instance solves its DSA system in FP64 in one thread-block cluster (options dsa_fp64 = 1,
 * dsa_cluster = 1), whatever the options say.  Arrays are
 * copied.  On failure nothing is kept; rte_last_error(NULL) names the failing instance. */
rte_status rte_batch_create(rte_batch* out, int count, const rte_problem* problems,
                            const rte_options* opt);
/* nsteps implicit steps of every instance, concurrently.  Returns the first non-OK status
 * in instance order (RTE_ENOCONV, RTE_ECUDA, ...); each instance's own status and message
 * stay available through rte_batch_status and rte_last_error(rte_batch_instance(b, i)). */
rte_status rte_batch_step(rte_batch b, int nsteps);
/* Back to every instance's initial state (rte_restart on each). */
rte_status rte_batch_restart(rte_batch b);
int rte_batch_size(rte_batch b);
/* The handle of instance i (owned by the batch; valid until rte_batch_destroy) for the
 * per-instance calls (rte_get_scalar_flux, rte_get_stats, rte_set_inflow, ...) between
 * batch steps; NULL when i is out of range. */
rte_handle rte_batch_instance(rte_batch b, int i);
/* Status of instance i in the last rte_batch_step (RTE_EINVAL when i is out of range). */
rte_status rte_batch_status(rte_batch b, int i);
void rte_batch_destroy(rte_batch b);   /* NULL-safe */

#ifdef __cplusplus
}
#endif
#endif /* RTE_H */
