// Diffusion synthetic acceleration (Sec. 2.3 Eq. (rho_residual)):
//   C delta = Sigma_s (rho^{l-1/2} - rho^{l-1}),
// C the cell-centred diffusion discretisation of the correction equation Eq.
// (discrete_correction_f) (sigma_a~ = tau + sigma_a, D = 1/(3 (tau + sigma_t)), zero inflow):
// 5-point (1D: 3-point) stencil, harmonic-mean face coefficients 2 D_L D_R/((D_L+D_R) h^2) and
// Marshak vacuum faces 1/(h (2 + h/(2D))), each floored at 1/(4h) (the half-range current of
// the upwind sweep).  Solved by conjugate gradients (Sec. 4) in one cooperative launch, with
// grid-wide phases separated by a bounded software grid barrier; every block sums the block
// partials in the same fixed order, so the CG scalars are identical everywhere and bitwise
// reproducible.  The handle's solves on grids of up to 2^18 cells use cg1_kernel, one phase
// per iteration (the Chronopoulos-Gear arrangement); larger grids and the allocation-free
// solve use cg_kernel, two phases per iteration:
//   (1) p <- r + beta p (double-buffered, neighbours recomputed from r and the old p),
//       Ap = C p, and the block partials of p.Ap;
//   (2) x += alpha p, r -= alpha Ap and the block partials of r.r.
// With options.dsa_cluster (batched instances) the same two-phase solve runs in one
// thread-block cluster (cg_cluster_kernel): the hardware schedules the cluster's CTAs together
// and its barrier is the cluster barrier, so no solve waits on blocks that other kernels keep
// from starting.  A cooperative launch gives no such guarantee beside other work: two solves
// that each got only some of their blocks onto the SMs could wait on each other until their
// bounded barrier waits ran out.
//
// Q1 scheme (bilinear modes per cell, mode-major vectors): C is the symmetric interior-penalty
// DG discretisation of the same correction equation on the same bilinear space, with the
// penalty of the modified-interior-penalty DSA (Wang and Ragusa, 2010), the Marshak condition
// -D d(delta)/dn = delta / 2 taken weakly, and every term divided by the cell area:
//   a(u, v) = sum_T int_T (D grad u . grad v + sigma_a~ u v)
//           + sum_{interior F} int_F (kappa_F [u][v] - {D du/dn}[v] - [u]{D dv/dn})
//           + sum_{boundary F} int_F u v / 2,     kappa_F = max(2 (D_L + D_R) / h_perp, 1/4).
// On a tensor-product basis every term acts on the x modes or on the y modes alone, so the
// operator of a cell is Xd (x) I + I (x) Yd on its own modes plus one 2 x 2 block per
// neighbour: 14 coefficients per cell, set up on the host.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "rte_internal.h"

namespace rte {

struct DsaRow {
  double diag, cx, cy;
};

namespace {
constexpr int CT = 256;
constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned BARRIER_SPIN_LIMIT = 1u << 22;

// S: the storage and arithmetic type of the solve's vectors and operator coefficients (double,
// or float in the FP32 modes); the dot products, CG scalars and the FP64 inputs and outputs
// (residual, delta, rho) stay in double.
template <class S>
struct CgArgs {
  int nx, ny, n;
  const S* diag;
  const S* cx;
  const S* cy;
  const S* blk;   // Q1: [14][ncell] Xd00 Xd01 Xd11 Yd00 Yd01 Yd11 Ex00 Ex01 Ex10 Ex11 Ny..
  const S* dinv;  // Q1: [n] inverse diagonal of C (the Jacobi preconditioner)
  int ncell;           // Q1: cells (n = 4 ncell)
  const double* sig_s;
  const double* residual;
  const double* residual_b;   // optional: residual = residual - residual_b
  double rtol2;
  int max_iter;
  S *r, *p0, *p1, *ap, *x;
  S *r1, *w1, *s1;   // cg1_kernel: second buffers of r, w = A r (first: ap), s = A p (first: p1)
  double* partial;     // [2 * gridDim.x]
  unsigned* bar;       // [0] arrive count, [1] generation, [2] error
  double* delta;       // output (may alias x)
  const double* rho_half;
  double* rho_out;
  double* q_out;
  int* iters;
  int iters_add;       // 1: add the count to *iters (solves repeated by a device-side loop)
  const unsigned* skip;   // set: the whole solve is skipped (speculative SI-SA work)
};

__device__ __forceinline__ float fmaS(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaS(double a, double b, double c) { return __fma_rn(a, b, c); }
// whether a double output and an S vector are the same array (the solve may write delta into x)
template <class S>
__device__ __forceinline__ bool same_array(const double* d, const S* x) {
  return (const void*)d == (const void*)x;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Grid barrier for a cooperative launch (all blocks co-resident).  Bounded: after
// BARRIER_SPIN_LIMIT polls it records an error and returns true (for the whole block), and
// the caller leaves the solve; a wait that ended normally returns false.  A block that left
// no longer arrives at later barriers, so the other blocks' next waits run out as well and
// they leave too: a solve whose barrier timed out ends after at most two wait limits.
__device__ bool grid_barrier(unsigned* bar, unsigned& gen) {
  __shared__ int s_timeout;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_timeout = 0;
    __threadfence();
    const unsigned g = gen;
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      bar[0] = 0u;
      __threadfence();
      atomicExch(&bar[1], g + 1u);
    } else {
      unsigned spins = 0;
      while (ld_acquire(&bar[1]) == g) {
        if (++spins > BARRIER_SPIN_LIMIT) {
          atomicExch(&bar[2], 1u);
          s_timeout = 1;
          break;
        }
        if (spins > 1024) __nanosleep(32);
      }
    }
    __threadfence();
  }
  gen += 1u;
  __syncthreads();
  return s_timeout != 0;
}

__device__ double block_sum_store(double v, double* dst) {
  __shared__ double sh[CT / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < CT / 32 ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *dst = v;
  }
  __syncthreads();
  return v;
}

// Sum of gridDim.x partials in a fixed order; result broadcast to the block.
__device__ double grid_total(const double* part) {
  __shared__ double tot;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) s += __ldcg(part + b);
    s = warp_sum(s);
    if (threadIdx.x == 0) tot = s;
  }
  __syncthreads();
  const double v = tot;
  __syncthreads();
  return v;
}

// (C v) at cell index c of the 5-point (1D: 3-point) stencil, for v given at c (vc) and at the
// neighbours by a function of the index.
template <class S, class V>
__device__ __forceinline__ S op_apply(const CgArgs<S>& a, int c, S vc, V v) {
  const int i = c % a.nx;
  S s = a.diag[c] * vc;
  if (i + 1 < a.nx) s -= a.cx[c] * v(c + 1);
  if (i > 0) s -= a.cx[c - 1] * v(c - 1);
  if (a.ny > 1) {
    if (c + a.nx < a.n) s -= a.cy[c] * v(c + a.nx);
    if (c - a.nx >= 0) s -= a.cy[c - a.nx] * v(c - a.nx);
  }
  return s;
}

// Q1: (C v) for the four modes of one cell (mode k = a + 2b at index k ncell + cell), given
// the cell's own modes u and the neighbours' by a function of the vector index, each
// neighbour value taken once.  With U[a][b] = u[a + 2b]:
//   Y = Xd U + U Yd^T + Ex U_{+x} + Ex_{-x}^T U_{-x} + U_{+y} Ny^T + U_{-y} Ny_{-y}
// (Xd, Yd symmetric; Ex, Ny the cell's own blocks to its +x and +y neighbours, Ex_{-x} and
// Ny_{-y} those of the -x and -y neighbours, i.e. the transposes of the blocks seen from here).
template <class S, class V>
__device__ __forceinline__ void q1_apply_cell(const CgArgs<S>& a, int cell, const S u[4], V v,
                                              S y[4]) {
  const int nc = a.ncell, nx = a.nx;
  const int i = cell % nx, j = cell / nx;
  const S* B = a.blk;
  auto co = [&](int e, int cc) { return __ldg(B + (size_t)e * nc + cc); };
  const S x00 = co(0, cell), x01 = co(1, cell), x11 = co(2, cell);
  const S y00 = co(3, cell), y01 = co(4, cell), y11 = co(5, cell);
  // own block: y[a + 2b] = sum_c Xd[a][c] u[c + 2b] + sum_d Yd[b][d] u[a + 2d]
  y[0] = x00 * u[0] + x01 * u[1] + y00 * u[0] + y01 * u[2];
  y[1] = x01 * u[0] + x11 * u[1] + y00 * u[1] + y01 * u[3];
  y[2] = x00 * u[2] + x01 * u[3] + y01 * u[0] + y11 * u[2];
  y[3] = x01 * u[2] + x11 * u[3] + y01 * u[1] + y11 * u[3];
  if (i + 1 < nx) {   // sum_c Ex[a][c] v(c + 2b) of the +x neighbour
    const int nb = cell + 1;
    const S e00 = co(6, cell), e01 = co(7, cell), e10 = co(8, cell), e11 = co(9, cell);
    const S w0 = v(nb), w1 = v(nc + nb), w2 = v(2 * nc + nb), w3 = v(3 * nc + nb);
    y[0] += e00 * w0 + e01 * w1;
    y[1] += e10 * w0 + e11 * w1;
    y[2] += e00 * w2 + e01 * w3;
    y[3] += e10 * w2 + e11 * w3;
  }
  if (i > 0) {        // sum_c Ex_{-x}[c][a] v(c + 2b) of the -x neighbour
    const int nb = cell - 1;
    const S e00 = co(6, nb), e01 = co(7, nb), e10 = co(8, nb), e11 = co(9, nb);
    const S w0 = v(nb), w1 = v(nc + nb), w2 = v(2 * nc + nb), w3 = v(3 * nc + nb);
    y[0] += e00 * w0 + e10 * w1;
    y[1] += e01 * w0 + e11 * w1;
    y[2] += e00 * w2 + e10 * w3;
    y[3] += e01 * w2 + e11 * w3;
  }
  if (j + 1 < a.ny) { // sum_d Ny[b][d] v(a + 2d) of the +y neighbour
    const int nb = cell + nx;
    const S n00 = co(10, cell), n01 = co(11, cell), n10 = co(12, cell), n11 = co(13, cell);
    const S w0 = v(nb), w1 = v(nc + nb), w2 = v(2 * nc + nb), w3 = v(3 * nc + nb);
    y[0] += n00 * w0 + n01 * w2;
    y[1] += n00 * w1 + n01 * w3;
    y[2] += n10 * w0 + n11 * w2;
    y[3] += n10 * w1 + n11 * w3;
  }
  if (j > 0) {        // sum_d Ny_{-y}[d][b] v(a + 2d) of the -y neighbour
    const int nb = cell - nx;
    const S n00 = co(10, nb), n01 = co(11, nb), n10 = co(12, nb), n11 = co(13, nb);
    const S w0 = v(nb), w1 = v(nc + nb), w2 = v(2 * nc + nb), w3 = v(3 * nc + nb);
    y[0] += n00 * w0 + n10 * w2;
    y[1] += n00 * w1 + n10 * w3;
    y[2] += n01 * w0 + n11 * w2;
    y[3] += n01 * w1 + n11 * w3;
  }
}

template <class S>
__global__ void __launch_bounds__(CT) cg_kernel(const CgArgs<S> a) {
  if (a.skip && *a.skip) return;   // every block returns before the first barrier
  unsigned gen = ld_acquire(&a.bar[1]);
  const int tid = blockIdx.x * CT + threadIdx.x, nth = gridDim.x * CT;
  double* partA = a.partial;
  double* partB = a.partial + gridDim.x;
  // r = b = sig_s .* residual, x = 0, p = r
  double acc = 0.0;
  for (int c = tid; c < a.n; c += nth) {
    const double rc = a.residual_b ? a.residual[c] - a.residual_b[c] : a.residual[c];
    const S b = S(a.sig_s[c] * rc);
    a.r[c] = b;
    a.x[c] = S(0);
    a.p0[c] = b;
    acc += double(b) * double(b);
  }
  block_sum_store(acc, partB + blockIdx.x);
  bool dead = grid_barrier(a.bar, gen);   // a barrier wait ran out: leave the solve
  double rr = grid_total(partB);
  const double bb = rr;
  double beta = 0.0;
  int it = 0;
  S* pold = a.p0;
  S* pnew = a.p1;
  while (!dead && it < a.max_iter && rr > a.rtol2 * bb) {
    // (1) p <- r + beta p ; Ap = C p ; p.Ap
    acc = 0.0;
    const S bt = S(beta);
    for (int c = tid; c < a.n; c += nth) {
      // Neighbours belong to other blocks: read them through L2 (__ldcg), never a stale L1 line.
      auto pval = [&](int k) {
        return (it == 0) ? __ldcg(pold + k) : __ldcg(a.r + k) + bt * __ldcg(pold + k);
      };
      const S pc = pval(c);
      const S sc = op_apply(a, c, pc, pval);
      pnew[c] = pc;
      a.ap[c] = sc;
      acc += double(pc) * double(sc);
    }
    block_sum_store(acc, partA + blockIdx.x);
    if ((dead = grid_barrier(a.bar, gen))) break;
    const double alpha = rr / grid_total(partA);
    const S al = S(alpha);
    // (2) x += alpha p ; r -= alpha Ap ; r.r
    acc = 0.0;
    for (int c = tid; c < a.n; c += nth) {
      a.x[c] += al * pnew[c];
      const S rc = a.r[c] - al * a.ap[c];
      a.r[c] = rc;
      acc += double(rc) * double(rc);
    }
    block_sum_store(acc, partB + blockIdx.x);
    if ((dead = grid_barrier(a.bar, gen))) break;
    const double rr_new = grid_total(partB);
    beta = rr_new / rr;
    rr = rr_new;
    S* t = pold;
    pold = pnew;
    pnew = t;
    ++it;
  }
  for (int c = tid; c < a.n; c += nth) {
    const double d = double(a.x[c]);
    if (!same_array(a.delta, a.x)) a.delta[c] = d;
    if (a.rho_out) {
      const double r = a.rho_half[c] + d;
      a.rho_out[c] = r;
      a.q_out[c] = a.sig_s[c] * r;
    }
  }
  if (tid == 0) *a.iters = a.iters_add ? *a.iters + it : it;
}

// One thread-block cluster per solve: CL_CTAS CTAs of CL_CT threads.
constexpr int CL_CTAS = 8;   // the portable maximum cluster size
constexpr int CL_CT = 512;

// Sum of a CTA's CL_CT values into *slot (the CTA's own shared memory).  Every call is
// followed by a cluster barrier before the next one, which keeps the staging array's reuse
// ordered.
__device__ void cta_sum_to(double v, double* slot) {
  __shared__ double sh[CL_CT / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < CL_CT / 32 ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *slot = v;
  }
}

// The two-phase solve of cg_kernel inside one cluster.  The grid is the cluster; a phase ends
// with a fence and the cluster barrier (release / acquire at cluster scope); the CTA partials
// stay in each CTA's shared memory and every thread sums them over the distributed shared
// memory in CTA-rank order, so all CTAs hold the same CG scalars bit for bit and take the same
// branch.  Two partial slots: phase 1 writes slot 0 while a slower CTA may still be reading
// slot 1 of the previous phase, and the reverse.  No software wait: nothing here can time out.
template <class S>
__global__ void __launch_bounds__(CL_CT) cg_cluster_kernel(const CgArgs<S> a) {
  if (a.skip && *a.skip) return;   // every CTA returns before any shared-memory exchange
  namespace cgr = cooperative_groups;
  cgr::cluster_group cl = cgr::this_cluster();
  const unsigned ncta = cl.num_blocks();
  const int tid = (int)cl.block_rank() * CL_CT + (int)threadIdx.x;
  const int nth = (int)ncta * CL_CT;
  __shared__ double s_part[2];
  auto phase_end = [&]() {
    __threadfence();
    cl.sync();
  };
  auto total = [&](int k) {
    double t = 0.0;
    for (unsigned b = 0; b < ncta; ++b) t += *cl.map_shared_rank(&s_part[k], b);
    return t;
  };
  // r = b = sig_s .* residual, x = 0, p = r
  double acc = 0.0;
  for (int c = tid; c < a.n; c += nth) {
    const double rc = a.residual_b ? a.residual[c] - a.residual_b[c] : a.residual[c];
    const S b = S(a.sig_s[c] * rc);
    a.r[c] = b;
    a.x[c] = S(0);
    a.p0[c] = b;
    acc += double(b) * double(b);
  }
  cta_sum_to(acc, &s_part[1]);
  phase_end();
  double rr = total(1);
  const double bb = rr;
  double beta = 0.0;
  int it = 0;
  S* pold = a.p0;
  S* pnew = a.p1;
  while (it < a.max_iter && rr > a.rtol2 * bb) {
    // (1) p <- r + beta p ; Ap = C p ; p.Ap
    acc = 0.0;
    const S bt = S(beta);
    for (int c = tid; c < a.n; c += nth) {
      // neighbours belong to other CTAs: read them through L2 (__ldcg), never a stale L1 line
      auto pval = [&](int k) {
        return (it == 0) ? __ldcg(pold + k) : __ldcg(a.r + k) + bt * __ldcg(pold + k);
      };
      const S pc = pval(c);
      const S sc = op_apply(a, c, pc, pval);
      pnew[c] = pc;
      a.ap[c] = sc;
      acc += double(pc) * double(sc);
    }
    cta_sum_to(acc, &s_part[0]);
    phase_end();
    const double alpha = rr / total(0);
    const S al = S(alpha);
    // (2) x += alpha p ; r -= alpha Ap ; r.r
    acc = 0.0;
    for (int c = tid; c < a.n; c += nth) {
      a.x[c] += al * pnew[c];
      const S rc = a.r[c] - al * a.ap[c];
      a.r[c] = rc;
      acc += double(rc) * double(rc);
    }
    cta_sum_to(acc, &s_part[1]);
    phase_end();
    const double rr_new = total(1);
    beta = rr_new / rr;
    rr = rr_new;
    S* t = pold;
    pold = pnew;
    pnew = t;
    ++it;
  }
  for (int c = tid; c < a.n; c += nth) {
    const double d = double(a.x[c]);
    if (!same_array(a.delta, a.x)) a.delta[c] = d;
    if (a.rho_out) {
      const double r = a.rho_half[c] + d;
      a.rho_out[c] = r;
      a.q_out[c] = a.sig_s[c] * r;
    }
  }
  if (tid == 0) *a.iters = a.iters_add ? *a.iters + it : it;
  cl.sync();   // no CTA leaves while another may still read its partials
}

template <class S>
cudaError_t launch_cg_cluster(const CgArgs<S>& a, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(CL_CTAS);
  cfg.blockDim = dim3(CL_CT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL_CTAS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cg_cluster_kernel<S>, a);
}

// Forward declarations of the two-value block and grid sums (defined below).
__device__ void block_sum2_store(double u, double v, double* dst0, double* dst1);
__device__ void grid_total2(const double* part0, const double* part1, double& t0, double& t1);

// Q1 solves: conjugate gradients preconditioned by the diagonal of C (Jacobi; Sec. 4
// preconditions its DSA solves), two grid-wide phases per iteration as cg_kernel:
//   (1) p <- z + beta p with z = D^-1 r (neighbours' p recomputed from r and the old p),
//       Ap = C p and the block partials of p.Ap, one cell (four unknowns) per thread;
//   (2) x += alpha p, r -= alpha Ap and the block partials of r.r (the stopping test) and of
//       r.z (the next beta).
// Three partial arrays: phase 1 writes the first while every block may still be reading the
// second and third of the previous phase, and the reverse.
template <class S>
__global__ void __launch_bounds__(CT) pcg_q1_kernel(const CgArgs<S> a) {
  if (a.skip && *a.skip) return;   // every block returns before the first barrier
  unsigned gen = ld_acquire(&a.bar[1]);
  const int tid = blockIdx.x * CT + threadIdx.x, nth = gridDim.x * CT;
  double* partA = a.partial;
  double* partR = a.partial + gridDim.x;
  double* partZ = a.partial + 2 * gridDim.x;
  // r = b = sig_s .* residual, x = 0, p = z = D^-1 b; (b, b) and (b, z)
  double accr = 0.0, accz = 0.0;
  for (int c = tid; c < a.n; c += nth) {
    const double rc = a.residual_b ? a.residual[c] - a.residual_b[c] : a.residual[c];
    const S b = S(a.sig_s[c] * rc);
    const S z = b * a.dinv[c];
    a.r[c] = b;
    a.x[c] = S(0);
    a.p0[c] = z;
    accr += double(b) * double(b);
    accz += double(b) * double(z);
  }
  block_sum2_store(accr, accz, partR + blockIdx.x, partZ + blockIdx.x);
  bool dead = grid_barrier(a.bar, gen);
  double rr, rz;
  grid_total2(partR, partZ, rr, rz);
  const double bb = rr;
  double beta = 0.0;
  int it = 0;
  S* pold = a.p0;
  S* pnew = a.p1;
  while (!dead && it < a.max_iter && rr > a.rtol2 * bb) {
    double acc = 0.0;
    const int nc = a.ncell;
    const S bt = S(beta);
    for (int cell = tid; cell < nc; cell += nth) {   // one cell (its four modes) per thread
      auto pval = [&](int k) {
        return (it == 0) ? __ldcg(pold + k)
                         : fmaS(bt, __ldcg(pold + k), __ldcg(a.r + k) * __ldg(a.dinv + k));
      };
      S pc[4], y[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) pc[k] = pval(k * nc + cell);
      q1_apply_cell(a, cell, pc, pval, y);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        pnew[k * nc + cell] = pc[k];
        a.ap[k * nc + cell] = y[k];
        acc += double(pc[k]) * double(y[k]);
      }
    }
    block_sum_store(acc, partA + blockIdx.x);
    if ((dead = grid_barrier(a.bar, gen))) break;
    const double alpha = rz / grid_total(partA);
    const S al = S(alpha);
    accr = 0.0;
    accz = 0.0;
    for (int c = tid; c < a.n; c += nth) {
      a.x[c] += al * pnew[c];
      const S rc = a.r[c] - al * a.ap[c];
      a.r[c] = rc;
      accr += double(rc) * double(rc);
      accz += double(rc) * double(rc * a.dinv[c]);
    }
    block_sum2_store(accr, accz, partR + blockIdx.x, partZ + blockIdx.x);
    if ((dead = grid_barrier(a.bar, gen))) break;
    double rz_new;
    grid_total2(partR, partZ, rr, rz_new);
    beta = rz_new / rz;
    rz = rz_new;
    S* t = pold;
    pold = pnew;
    pnew = t;
    ++it;
  }
  for (int c = tid; c < a.n; c += nth) {
    const double d = double(a.x[c]);
    if (!same_array(a.delta, a.x)) a.delta[c] = d;
    if (a.rho_out) {
      const double r = a.rho_half[c] + d;
      a.rho_out[c] = r;
      a.q_out[c] = a.sig_s[c] * r;
    }
  }
  if (tid == 0) *a.iters = a.iters_add ? *a.iters + it : it;
}

// Block sums of two values, thread 0 storing them to dst0 / dst1.
__device__ void block_sum2_store(double u, double v, double* dst0, double* dst1) {
  __shared__ double sh[2][CT / 32];
  u = warp_sum(u);
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = u;
    sh[1][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    u = threadIdx.x < CT / 32 ? sh[0][threadIdx.x] : 0.0;
    v = threadIdx.x < CT / 32 ? sh[1][threadIdx.x] : 0.0;
    u = warp_sum(u);
    v = warp_sum(v);
    if (threadIdx.x == 0) {
      *dst0 = u;
      *dst1 = v;
    }
  }
  __syncthreads();
}

// Sums of two arrays of gridDim.x partials, read by the whole block in one pass and added in a
// fixed tree order, so every block obtains the same two values.
__device__ void grid_total2(const double* part0, const double* part1, double& t0, double& t1) {
  __shared__ double sh[2][CT / 32];
  __shared__ double tot[2];
  double u = 0.0, v = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += CT) {
    u += __ldcg(part0 + b);
    v += __ldcg(part1 + b);
  }
  u = warp_sum(u);
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = u;
    sh[1][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    u = threadIdx.x < CT / 32 ? sh[0][threadIdx.x] : 0.0;
    v = threadIdx.x < CT / 32 ? sh[1][threadIdx.x] : 0.0;
    u = warp_sum(u);
    v = warp_sum(v);
    if (threadIdx.x == 0) {
      tot[0] = u;
      tot[1] = v;
    }
  }
  __syncthreads();
  t0 = tot[0];
  t1 = tot[1];
  __syncthreads();
}

// The same CG solve in the Chronopoulos-Gear arrangement (s = A p and w = A r carried by
// recurrences, x, r, p as in the textbook method): in exact arithmetic the iterates, and with
// the stopping test (r, r) <= rtol^2 (b, b) on the directly summed (r, r) the iteration count,
// are those of the textbook recurrence, but the two inner products of an iteration, (r, r)
// and (w, r), come from one reduction, so an iteration is one grid-wide phase and one barrier:
//   p = r + beta p, s = w + beta s, x += alpha p, r' = r - alpha s, w' = A r', (r', r'), (w', r').
// A neighbour's r' is recomputed from its r, w and s of the previous phase (double-buffered),
// with the same fused operations as its owner uses, so every copy is bitwise the owner's.
// The setup forms only r = b and (b, b); the first step length needs (C r, r), which one more
// phase computes when the stopping test lets CG iterate at all (a solve of k >= 1 iterations
// takes k + 2 barriers, a solve that stops at once one).
template <class S>
__global__ void __launch_bounds__(CT) cg1_kernel(const CgArgs<S> a) {
  if (a.skip && *a.skip) return;   // every block returns before the first barrier
  unsigned gen = ld_acquire(&a.bar[1]);
  const int tid = blockIdx.x * CT + threadIdx.x, nth = gridDim.x * CT;
  const int n = a.n;
  double* partG = a.partial;
  double* partD = a.partial + gridDim.x;
  // (C v)_c for v given at c (vc) and elsewhere by a function of the vector index
  auto apply = [&](int c, S vc, auto v) { return op_apply(a, c, vc, v); };
  // r = b = sig_s .* residual and (b, b)
  double g = 0.0, d = 0.0;
  for (int c = tid; c < n; c += nth) {
    const double rc = a.residual_b ? a.residual[c] - a.residual_b[c] : a.residual[c];
    const S b = S(a.sig_s[c] * rc);
    a.r[c] = b;
    g += double(b) * double(b);
  }
  block_sum2_store(g, 0.0, partG + blockIdx.x, partD + blockIdx.x);
  bool dead = grid_barrier(a.bar, gen);   // a barrier wait ran out: leave the solve
  double gamma, delta;
  grid_total2(partG, partD, gamma, delta);
  const double bb = gamma;
  if (!dead && a.max_iter > 0 && gamma > a.rtol2 * bb) {
    // w = C r and (w, r) for the first step length (only when CG iterates at all)
    d = 0.0;
    for (int c = tid; c < n; c += nth) {
      const S rc = a.r[c];
      const S w = apply(c, rc, [&](int k) { return __ldcg(a.r + k); });
      a.ap[c] = w;
      d += double(w) * double(rc);
    }
    block_sum2_store(0.0, d, partG + blockIdx.x, partD + blockIdx.x);
    dead = grid_barrier(a.bar, gen);
    double unused;
    grid_total2(partG, partD, unused, delta);
  }
  double gamma_prev = 0.0, alpha_prev = 0.0;
  int it = 0;
  while (!dead && it < a.max_iter && gamma > a.rtol2 * bb) {
    const bool first = it == 0;   // p = r, s = w, x = alpha p (p, s, x start at zero)
    const double beta = first ? 0.0 : gamma / gamma_prev;
    const double alpha = first ? gamma / delta : gamma / (delta - beta * gamma / alpha_prev);
    const S bt = S(beta), al = S(alpha);
    const bool odd = (it & 1) != 0;
    const S* r_o = odd ? a.r1 : a.r;
    const S* w_o = odd ? a.w1 : a.ap;
    const S* s_o = odd ? a.s1 : a.p1;
    S* r_n = odd ? a.r : a.r1;
    S* w_n = odd ? a.ap : a.w1;
    S* s_n = odd ? a.p1 : a.s1;
    auto rnext = [&](int k) {
      const S sk = first ? __ldcg(w_o + k) : fmaS(bt, __ldcg(s_o + k), __ldcg(w_o + k));
      return fmaS(-al, sk, __ldcg(r_o + k));
    };
    g = 0.0;
    d = 0.0;
    for (int c = tid; c < n; c += nth) {
      const S rc0 = r_o[c];
      const S sc = first ? w_o[c] : fmaS(bt, s_o[c], w_o[c]);
      const S pc = first ? rc0 : fmaS(bt, a.p0[c], rc0);
      a.p0[c] = pc;
      s_n[c] = sc;
      a.x[c] = first ? al * pc : fmaS(al, pc, a.x[c]);
      const S rc = fmaS(-al, sc, rc0);
      const S wc = apply(c, rc, rnext);
      r_n[c] = rc;
      w_n[c] = wc;
      g += double(rc) * double(rc);
      d += double(wc) * double(rc);
    }
    block_sum2_store(g, d, partG + blockIdx.x, partD + blockIdx.x);
    if ((dead = grid_barrier(a.bar, gen))) break;
    gamma_prev = gamma;
    alpha_prev = alpha;
    grid_total2(partG, partD, gamma, delta);
    ++it;
  }
  for (int c = tid; c < n; c += nth) {
    const double dd = it > 0 ? double(a.x[c]) : 0.0;
    if (!same_array(a.delta, a.x) || it == 0) a.delta[c] = dd;
    if (a.rho_out) {
      const double r = a.rho_half[c] + dd;
      a.rho_out[c] = r;
      a.q_out[c] = a.sig_s[c] * r;
    }
  }
  if (tid == 0) *a.iters = a.iters_add ? *a.iters + it : it;
}

}  // namespace

// Row c of the diffusion operator C, shared by the handle's set-up (on the host) and the
// allocation-free solve (on the device) so that both build the same operator bit for bit:
// D = 1/(3 (sigma_t + tau)); interior face coupling max(2 D_L D_R / ((D_L + D_R) h), 1/4) / h;
// vacuum (Marshak) face max(1 / (2 + h / (2 D)), 1/4) / h; diagonal sigma_t - sigma_s + tau
// plus the couplings of the cell's faces, added in a fixed order (x: low face, high face;
// then y).  cx / cy: the coupling to the +x / +y neighbour (0 on the last column / row).
__host__ __device__ inline DsaRow dsa_row(int dim, int nx, int ny, int c, double hx, double hy,
                                          double tau, const double* sig_t, const double* sig_s) {
  const int i = c % nx, j = c / nx;
  auto D = [&](int k) { return 1.0 / (3.0 * (sig_t[k] + tau)); };
  auto face = [](double dl, double dr, double h) {
    return fmax(2.0 * dl * dr / ((dl + dr) * h), 0.25) / h;
  };
  auto marshak = [](double d, double h) { return fmax(1.0 / (2.0 + h / (2.0 * d)), 0.25) / h; };
  const double dc = D(c);
  DsaRow row{sig_t[c] - sig_s[c] + tau, 0.0, 0.0};
  row.diag += i > 0 ? face(D(c - 1), dc, hx) : marshak(dc, hx);
  if (i + 1 < nx) row.cx = face(dc, D(c + 1), hx);
  row.diag += i + 1 < nx ? row.cx : marshak(dc, hx);
  if (dim == 2) {
    row.diag += j > 0 ? face(D(c - nx), dc, hy) : marshak(dc, hy);
    if (j + 1 < ny) row.cy = face(dc, D(c + nx), hy);
    row.diag += j + 1 < ny ? row.cy : marshak(dc, hy);
  }
  return row;
}

namespace {
// Coefficients of the Q1 interior-penalty operator, [14][ncell] (see the file comment).  Per
// axis, on the reference interval with the orthonormal p_0 = 1, p_1 = sqrt(3) t: traces
// P(+1) = (1, sqrt 3) and P(-1) = (1, -sqrt 3), derivative (2/h) (0, sqrt 3), stiffness
// (4/h^2) diag(0, 3); a face term divided by the cell area carries 1/h.  For the face between
// L (trace P(+1)) and R (trace P(-1)), test function on the rows and trial on the columns:
//   LL = kappa P+ P+^T - D_L (P+ g^T + g P+^T) / 2
//   LR = -kappa P+ P-^T - D_R P+ g^T / 2 + D_L g P-^T / 2
//   RR = kappa P- P-^T + D_R (P- g^T + g P-^T) / 2
// and a boundary face adds P P^T / 2 with the cell's own trace there.
void dsa_q1_blocks(int nx, int ny, double hx, double hy, double tau, const double* sig_t,
                   const double* sig_s, std::vector<double>& blk) {
  const long nc = (long)nx * ny;
  blk.assign((size_t)14 * nc, 0.0);
  const double r3 = std::sqrt(3.0);
  const double tp[2] = {1.0, r3}, tm[2] = {1.0, -r3};
  auto D = [&](long k) { return 1.0 / (3.0 * (sig_t[k] + tau)); };
  using M2 = double[2][2];
  auto outer = [](const double* u, const double* v, double f, M2& out) {
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) out[a][b] += f * u[a] * v[b];
  };
  // the face's blocks, scaled by 1/h
  auto face = [&](double h, double dl, double dr, M2& LL, M2& LR, M2& RR) {
    const double g[2] = {0.0, 2.0 * r3 / h};
    const double kap = std::fmax(2.0 * (dl + dr) / h, 0.25);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) LL[a][b] = LR[a][b] = RR[a][b] = 0.0;
    outer(tp, tp, kap / h, LL);
    outer(tp, g, -0.5 * dl / h, LL);
    outer(g, tp, -0.5 * dl / h, LL);
    outer(tp, tm, -kap / h, LR);
    outer(tp, g, -0.5 * dr / h, LR);
    outer(g, tm, 0.5 * dl / h, LR);
    outer(tm, tm, kap / h, RR);
    outer(tm, g, 0.5 * dr / h, RR);
    outer(g, tm, 0.5 * dr / h, RR);
  };
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const long c = i + (long)nx * j;
      const double dc = D(c);
      for (int axis = 0; axis < 2; ++axis) {
        const double h = axis == 0 ? hx : hy;
        const bool lo_in = axis == 0 ? i > 0 : j > 0;
        const bool hi_in = axis == 0 ? i + 1 < nx : j + 1 < ny;
        const long lo = axis == 0 ? c - 1 : c - nx, hi = axis == 0 ? c + 1 : c + nx;
        M2 d = {{0.0, 0.0}, {0.0, 0.0}}, LL, LR, RR;
        d[1][1] = dc * 12.0 / (h * h);   // stiffness (4/h^2) diag(0, 3)
        if (lo_in) {   // the cell is R of the low face
          face(h, D(lo), dc, LL, LR, RR);
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) d[a][b] += RR[a][b];
        } else {
          outer(tm, tm, 0.5 / h, d);
        }
        if (hi_in) {   // the cell is L of the high face
          face(h, dc, D(hi), LL, LR, RR);
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) d[a][b] += LL[a][b];
          const int e0 = axis == 0 ? 6 : 10;
          blk[(size_t)(e0 + 0) * nc + c] = LR[0][0];
          blk[(size_t)(e0 + 1) * nc + c] = LR[0][1];
          blk[(size_t)(e0 + 2) * nc + c] = LR[1][0];
          blk[(size_t)(e0 + 3) * nc + c] = LR[1][1];
        } else {
          outer(tp, tp, 0.5 / h, d);
        }
        if (axis == 0) {
          d[0][0] += sig_t[c] - sig_s[c] + tau;
          d[1][1] += sig_t[c] - sig_s[c] + tau;
        }
        const int e0 = axis == 0 ? 0 : 3;
        blk[(size_t)(e0 + 0) * nc + c] = d[0][0];
        blk[(size_t)(e0 + 1) * nc + c] = d[0][1];
        blk[(size_t)(e0 + 2) * nc + c] = d[1][1];
      }
    }
}
}  // namespace

cudaError_t dsa_setup(DsaOp& op, int dim, int nx, int ny, double hx, double hy, double tau,
                      const double* sig_t, const double* sig_s, cudaStream_t s, int max_blocks,
                      int degree, bool f32, bool cluster) {
  const int ncell = nx * ny;
  const int n = degree == 1 ? 4 * ncell : ncell;
  op.nx = nx;
  op.ny = ny;
  op.n = n;
  op.ncell = ncell;
  op.deg = degree;
  op.f32 = f32;
  std::vector<double> diag, cx, cy, blk;
  if (degree == 1) {
    dsa_q1_blocks(nx, ny, hx, hy, tau, sig_t, sig_s, blk);
  } else {
    diag.resize(n), cx.resize(n), cy.resize(n);
    for (int c = 0; c < n; ++c) {
      const DsaRow row = dsa_row(dim, nx, ny, c, hx, hy, tau, sig_t, sig_s);
      diag[c] = row.diag;
      cx[c] = row.cx;
      cy[c] = row.cy;
    }
  }
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // Small grids, where a CG iteration costs its grid barriers rather than its memory traffic,
  // take the one-barrier arrangement (cg1_kernel, one block per SM: the barrier's cost grows
  // with the blocks that arrive); large grids the two-phase one (cg_kernel, up to two blocks
  // per SM), which moves fewer bytes in solves of few iterations (measured: 256^2 cells 16-20 %
  // faster per solve with cg1_kernel, 1024^2 cells 20-25 % slower).
  // Q1: the Jacobi-preconditioned two-phase solve (measured with plain CG at 256^2 cells, the
  // two-phase arrangement took 20 % less time per solve than the one-barrier one, whose
  // recomputation of a neighbour's r' costs three loads and the Q1 operator reads ten)
  // cluster: the Q0 solve in one thread-block cluster (cg_cluster_kernel), for solves that run
  // beside other work (batched instances); the Q1 solve keeps its cooperative launch.
  op.cluster = cluster && degree == 0;
  op.single_phase = degree == 0 && n <= (1 << 18) && !op.cluster;
  const void* kern =
      f32 ? (degree == 1 ? (const void*)pcg_q1_kernel<float>
                         : (op.single_phase ? (const void*)cg1_kernel<float> : (const void*)cg_kernel<float>))
          : (degree == 1 ? (const void*)pcg_q1_kernel<double>
                         : (op.single_phase ? (const void*)cg1_kernel<double> : (const void*)cg_kernel<double>));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CT, 0);
  if (per_sm < 1) per_sm = 1;
  const int want = (n + CT - 1) / CT;
  int cap = op.single_phase ? sms : 2 * sms;
  if (cap > per_sm * sms) cap = per_sm * sms;
  if (max_blocks > 0 && cap > max_blocks) cap = max_blocks;
  op.blocks = want < cap ? want : cap;
  if (op.blocks < 1) op.blocks = 1;
  if (op.cluster) op.blocks = CL_CTAS;
  cudaError_t e;
  const size_t real = f32 ? sizeof(float) : sizeof(double);
  const size_t bytes = real * (size_t)n;
  void** bufs[] = {&op.diag, &op.cx, &op.cy, &op.r, &op.p0, &op.p1, &op.ap, &op.x,
                   &op.r1, &op.w1, &op.s1};
  op.blk = nullptr;
  op.dinv = nullptr;
  for (void** b : bufs) {
    *b = nullptr;
    if (!op.single_phase && (b == &op.r1 || b == &op.w1 || b == &op.s1)) continue;
    if (degree == 1 && (b == &op.diag || b == &op.cx || b == &op.cy)) continue;
    if ((e = cudaMalloc(b, bytes)) != cudaSuccess) return e;
  }
  if ((e = cudaMalloc(&op.partial, sizeof(double) * 3 * op.blocks)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&op.scal, 64)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(op.scal, 0, 64, s)) != cudaSuccess) return e;
  // coefficient arrays in the solve's storage (FP32: rounded once from the FP64 set-up)
  auto upload = [&](void** dst, const std::vector<double>& v) -> cudaError_t {
    cudaError_t err;
    if (!*dst && (err = cudaMalloc(dst, real * v.size())) != cudaSuccess) return err;
    if (!f32) return cudaMemcpyAsync(*dst, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, s);
    std::vector<float> w(v.begin(), v.end());
    if ((err = cudaMemcpyAsync(*dst, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      return err;
    return cudaStreamSynchronize(s);   // w is a local
  };
  if (degree == 1) {
    // inverse diagonal of C: mode k = a + 2b of a cell has Xd[a][a] + Yd[b][b]
    std::vector<double> dinv(n);
    for (int k = 0; k < 4; ++k)
      for (int c = 0; c < ncell; ++c) {
        const double d = blk[(size_t)((k & 1) ? 2 : 0) * ncell + c] +
                         blk[(size_t)((k >> 1) ? 5 : 3) * ncell + c];
        dinv[(size_t)k * ncell + c] = 1.0 / d;
      }
    if ((e = upload(&op.blk, blk)) != cudaSuccess) return e;
    if ((e = upload(&op.dinv, dinv)) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
  }
  if ((e = upload(&op.diag, diag)) != cudaSuccess) return e;
  if ((e = upload(&op.cx, cx)) != cudaSuccess) return e;
  if ((e = upload(&op.cy, cy)) != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

void dsa_free(DsaOp& op) {
  void* bufs[] = {op.diag, op.cx, op.cy, op.r,       op.p0,      op.p1,  op.ap,
                  op.x,    op.r1, op.w1, op.s1, op.partial, op.scal, op.blk, op.dinv};
  for (void* b : bufs)
    if (b) cudaFree(b);
  op = DsaOp{};
}

namespace {
template <class S>
cudaError_t dsa_solve_impl(DsaOp& op, const double* sig_s, const double* residual,
                           const double* residual_b, double rtol, int max_iter, double* delta,
                           const double* rho_half, double* rho_out, double* q_out,
                           int* iters_dev, cudaStream_t s, const unsigned* skip, int iters_add) {
  CgArgs<S> a{};
  a.skip = skip;
  a.iters_add = iters_add;
  a.nx = op.nx;
  a.ny = op.ny;
  a.n = op.n;
  a.diag = static_cast<const S*>(op.diag);
  a.cx = static_cast<const S*>(op.cx);
  a.cy = static_cast<const S*>(op.cy);
  a.blk = static_cast<const S*>(op.blk);
  a.dinv = static_cast<const S*>(op.dinv);
  a.ncell = op.ncell;
  a.sig_s = sig_s;
  a.residual = residual;
  a.residual_b = residual_b;
  a.rtol2 = rtol * rtol;
  a.max_iter = max_iter;
  a.r = static_cast<S*>(op.r);
  a.p0 = static_cast<S*>(op.p0);
  a.p1 = static_cast<S*>(op.p1);
  a.ap = static_cast<S*>(op.ap);
  a.x = static_cast<S*>(op.x);
  a.r1 = static_cast<S*>(op.r1);
  a.w1 = static_cast<S*>(op.w1);
  a.s1 = static_cast<S*>(op.s1);
  a.partial = op.partial;
  a.bar = reinterpret_cast<unsigned*>(op.scal);
  a.delta = delta;
  a.rho_half = rho_half;
  a.rho_out = rho_out;
  a.q_out = q_out;
  a.iters = iters_dev;
  ++g_launches;
  if (op.cluster) return launch_cg_cluster<S>(a, s);
  void* args[] = {&a};
  const void* kern = op.deg == 1
                         ? (const void*)pcg_q1_kernel<S>
                         : (op.single_phase ? (const void*)cg1_kernel<S> : (const void*)cg_kernel<S>);
  return cudaLaunchCooperativeKernel(kern, dim3(op.blocks), dim3(CT), args, 0, s);
}
}  // namespace

cudaError_t dsa_solve(DsaOp& op, const double* sig_s, const double* residual,
                      const double* residual_b, double rtol, int max_iter, double* delta,
                      const double* rho_half, double* rho_out, double* q_out, int* iters_dev,
                      cudaStream_t s, const unsigned* skip, int iters_add) {
  if (op.f32) {
    if (!delta) return cudaErrorInvalidValue;   // the FP32 iterate cannot hold the FP64 output
    return dsa_solve_impl<float>(op, sig_s, residual, residual_b, rtol, max_iter, delta,
                                 rho_half, rho_out, q_out, iters_dev, s, skip, iters_add);
  }
  return dsa_solve_impl<double>(op, sig_s, residual, residual_b, rtol, max_iter,
                                delta ? delta : static_cast<double*>(op.x), rho_half, rho_out,
                                q_out, iters_dev, s, skip, iters_add);
}

}  // namespace rte

// =========================================================================================
// Allocation-free DSA solve: the same diffusion operator and conjugate gradients, with every
// scratch vector in one file-scope device array instead of memory allocated by the caller or
// by a handle.  The array exists on every GPU that loads the library, until the process exits.
// =========================================================================================
namespace rte {

namespace {
constexpr int NOALLOC_MAX_CELLS = 65536;   // 256 x 256 cells
constexpr int NOALLOC_MAX_BLOCKS = 512;
// diag, cx, cy, r, p0, p1, ap, x  (8 cell vectors) | partial sums | barrier + iteration words
constexpr long NOALLOC_DOUBLES = 8L * NOALLOC_MAX_CELLS + 2L * NOALLOC_MAX_BLOCKS + 8;
static __device__ __align__(256) double g_dsa_noalloc_scratch[NOALLOC_DOUBLES];

// The operator's coefficients on the device, one thread per cell (the row function of the
// handle's set-up).
__global__ void dsa_coeff_kernel(int dim, int nx, int ny, double hx, double hy, double tau,
                                 const double* sig_t, const double* sig_s, double* diag,
                                 double* cx, double* cy) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nx * ny) return;
  const DsaRow row = dsa_row(dim, nx, ny, c, hx, hy, tau, sig_t, sig_s);
  diag[c] = row.diag;
  cx[c] = row.cx;
  cy[c] = row.cy;
}

// Device address of the scratch array on the current device.  It is looked up on every call
// (cheap, and it allocates nothing): after a cudaDeviceReset the library's module is loaded
// again, possibly at another address, so a cached address could be stale.
cudaError_t noalloc_scratch(double** out) {
  double* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_dsa_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

}  // namespace

rte_status dsa_solve_noalloc(int dim, int nx, int ny, double x0, double x1, double y0, double y1,
                             double c_dt, const double* sigma_t_dev, const double* sigma_s_dev,
                             const double* residual_dev, double cg_rtol, int cg_max_iter,
                             double* delta_dev, int* iterations, void* stream, std::string* err) {
  if ((dim != 1 && dim != 2) || nx < 1 || ny < 1 || (dim == 1 && ny != 1)) {
    *err = "rte_dsa_solve_noalloc: bad mesh";
    return RTE_EINVAL;
  }
  if ((long)nx * ny > NOALLOC_MAX_CELLS) {
    *err = "rte_dsa_solve_noalloc: nx*ny exceeds the fixed scratch capacity of " +
           std::to_string(NOALLOC_MAX_CELLS) + " cells";
    return RTE_EINVAL;
  }
  if (!(x1 > x0) || (dim == 2 && !(y1 > y0)) || !(c_dt > 0.0) || !(cg_rtol >= 0.0) ||
      cg_max_iter < 0 || !sigma_t_dev || !sigma_s_dev || !residual_dev || !delta_dev) {
    *err = "rte_dsa_solve_noalloc: bad argument";
    return RTE_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* base = nullptr;
  cudaError_t e = noalloc_scratch(&base);
  if (e != cudaSuccess) {
    *err = std::string("rte_dsa_solve_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return RTE_ECUDA;
  }
  const int n = nx * ny;
  const long M = NOALLOC_MAX_CELLS;
  double* diag = base;
  double* cx = base + M;
  double* cy = base + 2 * M;
  double* partial = base + 8 * M;
  unsigned* words = reinterpret_cast<unsigned*>(base + 8 * M + 2 * NOALLOC_MAX_BLOCKS);
  int* iters_dev = reinterpret_cast<int*>(words + 4);
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_kernel<double>, CT, 0);
  int blocks = (n + CT - 1) / CT;
  int cap = (per_sm < 1 ? 1 : per_sm) * sms;
  if (cap > 2 * sms) cap = 2 * sms;
  if (cap > NOALLOC_MAX_BLOCKS) cap = NOALLOC_MAX_BLOCKS;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  // barrier count, generation, error flag and the iteration count start at zero
  if ((e = cudaMemsetAsync(words, 0, 8 * sizeof(unsigned), s)) != cudaSuccess) {
    *err = std::string("rte_dsa_solve_noalloc: ") + cudaGetErrorString(e);
    return RTE_ECUDA;
  }
  const double hx = (x1 - x0) / nx, hy = dim == 2 ? (y1 - y0) / ny : 1.0;
  ++g_launches;
  dsa_coeff_kernel<<<(n + 255) / 256, 256, 0, s>>>(dim, nx, ny, hx, hy, 1.0 / c_dt, sigma_t_dev,
                                                   sigma_s_dev, diag, cx, cy);
  if ((e = cudaGetLastError()) != cudaSuccess) {
    *err = std::string("rte_dsa_solve_noalloc: coefficient kernel: ") + cudaGetErrorString(e);
    return RTE_ECUDA;
  }
  CgArgs<double> a{};
  a.nx = nx;
  a.ny = ny;
  a.n = n;
  a.diag = diag;
  a.cx = cx;
  a.cy = cy;
  a.sig_s = sigma_s_dev;
  a.residual = residual_dev;
  a.residual_b = nullptr;
  a.rtol2 = cg_rtol * cg_rtol;
  a.max_iter = cg_max_iter;
  a.r = base + 3 * M;
  a.p0 = base + 4 * M;
  a.p1 = base + 5 * M;
  a.ap = base + 6 * M;
  a.x = base + 7 * M;
  a.partial = partial;
  a.bar = words;
  a.delta = delta_dev;
  a.rho_half = nullptr;
  a.rho_out = nullptr;
  a.q_out = nullptr;
  a.iters = iters_dev;
  void* args[] = {&a};
  ++g_launches;
  e = cudaLaunchCooperativeKernel((const void*)cg_kernel<double>, dim3(blocks), dim3(CT), args, 0, s);
  if (e != cudaSuccess) {
    *err = std::string("rte_dsa_solve_noalloc: ") + cudaGetErrorString(e);
    return RTE_ECUDA;
  }
  unsigned host_words[8];
  if ((e = cudaMemcpyAsync(host_words, words, sizeof(host_words), cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    *err = std::string("rte_dsa_solve_noalloc: ") + cudaGetErrorString(e);
    return RTE_ECUDA;
  }
  if (iterations) *iterations = (int)host_words[4];
  if (host_words[2] != 0u) {
    *err = "rte_dsa_solve_noalloc: a bounded grid-barrier wait ran out";
    return RTE_ETIMEOUT;
  }
  return RTE_OK;
}

}  // namespace rte
