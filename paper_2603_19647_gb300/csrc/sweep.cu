// Transport sweeps: the Q0 upwind cell solve of Sec. 2.1 Eq. (DG) (K = 0), applied for all
// directions in upwind order (Sec. 2.3, "transport sweep"), with the quadrature moment of
// Sec. 2.1 fused in.
//
//   psi_j[c] = (S[c] + a_j psi_j[upwind x] + b_j psi_j[upwind y]) / (tau + sigma_t[c] + a_j + b_j)
//   a_j = |mu_j|/hx, b_j = |eta_j|/hy, inflow ghosts carry g (Eq. (boundary)).
//
// 2D: strip-chain wavefront.  Lane = direction (dl lanes per family of one quadrant), a
// lane group owns R consecutive rows and runs them on a skewed anti-diagonal schedule
// (row m handles column t - m at step t), so its R cell solves per step are independent.
// The lane groups of a warp are stacked vertically and hand the bottom row to the group
// below through a shuffle; CTAs (one warp each) of the same family are stacked vertically
// and hand their bottom row to the next CTA through global memory, published in chunks
// of K columns behind a release flag.  CTAs take tickets in row-block-major order, so a
// CTA only waits for CTAs that already started: no deadlock whatever the scheduling.  All
// waits are bounded; on timeout the kernel records an error and stops waiting.
//
// 1D: each direction's sweep psi_i = alpha_i psi_{i-1} + beta_i is a linear recurrence,
// evaluated as a block-wide associative scan of affine maps.
#include <cuda_runtime.h>

#include "rte_internal.h"

namespace rte {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int KCHUNK = 8;            // columns per published edge chunk
constexpr unsigned SPIN_LIMIT = 1u << 20;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

template <class Real>
__device__ __forceinline__ Real ldcg(const Real* p) {
  return __ldcg(p);
}

// Transpose-reduce R values over the DL lanes of a lane group: after it, lane dl holds the
// group-wide sum of value index m = dl / (DL / R).
template <class Real, int N, int O>
struct TReduce {
  static __device__ __forceinline__ void run(Real* v, int dl) {
    if constexpr (O == 0) {
      return;
    } else if constexpr (N > 1) {
      const bool hi = (dl & O) != 0;
#pragma unroll
      for (int i = 0; i < N / 2; ++i) {
        const Real send = hi ? v[i] : v[i + N / 2];
        const Real keep = hi ? v[i + N / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL, send, O);
      }
      TReduce<Real, N / 2, O / 2>::run(v, dl);
    } else {
      v[0] += __shfl_xor_sync(FULL, v[0], O);
      TReduce<Real, 1, O / 2>::run(v, dl);
    }
  }
};

// MODE 0: SI sweep (K1): S = q with the given inflow ghosts (zero for SI), moment of psi.
// MODE 2: y = L^-1(g2 + tau f) from the stored f, zero inflow, moment of y.
// MODE 1: fused f sweep (K2): pass A  f^n = L^-1(q + tau f^{n-1}) with inflow ghosts,
//         pass B  y = L^-1(g2 + tau f^n) with zero inflow; moment of B (and of A).
template <class Real, int DL, int R, int MODE, bool TABLE>
__global__ void __launch_bounds__(32) sweep2d_kernel(const Sweep2DArgs<Real> A) {
  constexpr int NG = 32 / DL;
  static_assert(R <= DL, "rows per lane group must not exceed the lane count");
  const int lane = threadIdx.x;
  const int gi = lane / DL, dl = lane % DL;
  unsigned t0 = 0;
  if (lane == 0) t0 = atomicAdd(&A.ctrl->ticket, 1u);
  const unsigned ticket = __shfl_sync(FULL, t0, 0);
  const int blk = (int)(ticket / (unsigned)A.nfam);
  const int fam = (int)(ticket % (unsigned)A.nfam);
  const int quad = A.fam_quad[fam];
  const bool xpos = (quad & 1) == 0;
  const bool ypos = quad < 2;
  const int nx = A.nx, ny = A.ny;
  const long ncell = (long)nx * ny;
  const int slot = fam * DL + dl;
  const Real ca = A.a[slot], cb = A.b[slot], cw = A.w[slot];
  const Real ct = A.tau + ca + cb;
  const int row0 = blk * A.rows_per_blk + gi * R;
  const Real gx = A.gx[quad];
  const Real gy = A.gy[quad];

  Real psA[R], psB[R];
#pragma unroll
  for (int m = 0; m < R; ++m) {
    psA[m] = gx;
    psB[m] = Real(0);
  }
  const bool has_up = blk > 0;
  const bool has_down = blk + 1 < A.nblk;
  const size_t plane = (size_t)A.nfam * A.nblk * nx * DL;
  const Real* edge_in = A.edge + ((size_t)(fam * A.nblk + (has_up ? blk - 1 : 0)) * nx) * DL;
  Real* edge_out = A.edge + ((size_t)(fam * A.nblk + blk) * nx) * DL;
  unsigned* flag_in = &A.ctrl->flags[fam * A.nblk + (has_up ? blk - 1 : 0)];
  unsigned* flag_out = &A.ctrl->flags[fam * A.nblk + blk];
  const int nsteps = nx + NG * R - 1;
  bool abandon = false;

  for (int tb = 0; tb < nsteps; tb += KCHUNK) {
    // Top inflow of this row block: the previous block's bottom row, KCHUNK columns at once.
    Real ebA[KCHUNK], ebB[KCHUNK];
    if (has_up && tb < nx) {
      const unsigned need = (unsigned)min(tb + KCHUNK, nx);
      if (lane == 0 && !abandon) {
        unsigned spins = 0;
        while (ld_acquire(flag_in) < need) {
          if (++spins > SPIN_LIMIT || ld_acquire(&A.ctrl->err) != 0u) {
            atomicExch(&A.ctrl->err, 1u);
            abandon = true;
            break;
          }
          __nanosleep(64);
        }
      }
      abandon = __shfl_sync(FULL, abandon, 0);
      __syncwarp();
      __threadfence();
#pragma unroll
      for (int k = 0; k < KCHUNK; ++k) {
        const int x = tb + k;
        ebA[k] = (gi == 0 && x < nx) ? ldcg(edge_in + (size_t)x * DL + dl) : Real(0);
        if constexpr (MODE == 1)
          ebB[k] = (gi == 0 && x < nx) ? ldcg(edge_in + plane + (size_t)x * DL + dl) : Real(0);
      }
    } else {
#pragma unroll
      for (int k = 0; k < KCHUNK; ++k) {
        ebA[k] = gy;
        ebB[k] = Real(0);
      }
    }
#pragma unroll
    for (int k = 0; k < KCHUNK; ++k) {
      const int t = tb + k;
      if (t >= nsteps) break;
      Real upA = __shfl_up_sync(FULL, psA[R - 1], DL);
      Real upB = __shfl_up_sync(FULL, psB[R - 1], DL);
      if (gi == 0) {
        upA = ebA[k];
        upB = ebB[k];
      }
      Real mom[R], momA[R];
#pragma unroll
      for (int m = R - 1; m >= 0; --m) {
        const int x = t - m - gi * R;
        const int jj = row0 + m;
        mom[m] = Real(0);
        momA[m] = Real(0);
        if (x >= 0 && x < nx && jj < ny) {
          const int px = xpos ? x : nx - 1 - x;
          const int py = ypos ? jj : ny - 1 - jj;
          const long cell = (long)py * nx + px;
          const Real dinv = TABLE ? A.inv_d[cell * A.nslot + slot] : recip(ct + A.sig_t[cell]);
          const Real uA = (m == 0) ? upA : psA[m > 0 ? m - 1 : 0];
          if constexpr (MODE == 0) {
            const Real v = (A.q[cell] + ca * psA[m] + cb * uA) * dinv;
            psA[m] = v;
            mom[m] = cw * v;
          } else if constexpr (MODE == 2) {
            // y = L^-1 (g2 + tau f) with the stored f, zero inflow (the recurrence runs in psA)
            const Real v = (A.g2[cell] + A.tau * A.f[cell * A.nslot + slot] + ca * psA[m] +
                            cb * uA) * dinv;
            psA[m] = v;
            mom[m] = cw * v;
          } else {
            Real* fp = A.f + cell * A.nslot + slot;
            const Real sa = A.q[cell] + A.tau * (*fp);
            const Real va = (sa + ca * psA[m] + cb * uA) * dinv;
            psA[m] = va;
            *fp = va;
            momA[m] = cw * va;
            const Real uB = (m == 0) ? upB : psB[m > 0 ? m - 1 : 0];
            const Real vb = (A.g2[cell] + A.tau * va + ca * psB[m] + cb * uB) * dinv;
            psB[m] = vb;
            mom[m] = cw * vb;
          }
        }
      }
      // Quadrature moment over the lane group's directions, one partial per family.
      TReduce<Real, R, DL / 2>::run(mom, dl);
      if constexpr (MODE == 1) {
        if (A.pm_a) TReduce<Real, R, DL / 2>::run(momA, dl);
      }
      if ((dl & (DL / R - 1)) == 0) {
        const int m = dl / (DL / R);
        const int x = t - m - gi * R;
        const int jj = row0 + m;
        if (x >= 0 && x < nx && jj < ny) {
          const int px = xpos ? x : nx - 1 - x;
          const int py = ypos ? jj : ny - 1 - jj;
          const long cell = (long)py * nx + px;
          A.pm[fam * ncell + cell] = mom[0];
          if constexpr (MODE == 1) {
            if (A.pm_a) A.pm_a[fam * ncell + cell] = momA[0];
          }
        }
      }
      // Bottom row of the block goes to the next row block.
      const int xb = t - (R - 1) - (NG - 1) * R;
      if (has_down && xb >= 0 && xb < nx) {
        if (gi == NG - 1) {
          edge_out[(size_t)xb * DL + dl] = psA[R - 1];
          if constexpr (MODE == 1) edge_out[plane + (size_t)xb * DL + dl] = psB[R - 1];
        }
        if ((xb + 1) % KCHUNK == 0 || xb == nx - 1) {
          __threadfence();
          __syncwarp();
          if (lane == 0) st_release(flag_out, (unsigned)(xb + 1));
        }
      }
    }
  }
  // Self-reset of the control block by the last CTA to finish.
  if (lane == 0) {
    __threadfence();
    const unsigned total = (unsigned)(A.nfam * A.nblk);
    if (atomicAdd(&A.ctrl->done, 1u) == total - 1) {
      for (unsigned i = 0; i < total; ++i) A.ctrl->flags[i] = 0u;
      A.ctrl->ticket = 0u;
      A.ctrl->done = 0u;
      __threadfence();
    }
  }
}

template <class Real, int DL, int R, int MODE>
cudaError_t launch_dl_r(const Sweep2DArgs<Real>& a, cudaStream_t s) {
  const dim3 grid((unsigned)(a.nfam * a.nblk));
  ++g_launches;
  if (a.inv_d)
    sweep2d_kernel<Real, DL, R, MODE, true><<<grid, 32, 0, s>>>(a);
  else
    sweep2d_kernel<Real, DL, R, MODE, false><<<grid, 32, 0, s>>>(a);
  return cudaGetLastError();
}

template <class Real, int DL, int MODE>
cudaError_t launch_dl(const Sweep2DArgs<Real>& a, int R, cudaStream_t s) {
  switch (R) {
    case 1: return launch_dl_r<Real, DL, 1, MODE>(a, s);
    case 2: return launch_dl_r<Real, DL, 2, MODE>(a, s);
    case 4: return launch_dl_r<Real, DL, 4, MODE>(a, s);
    case 8: return launch_dl_r<Real, DL, 8, MODE>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <class Real, int MODE>
cudaError_t launch_mode_impl(const Sweep2DArgs<Real>& a, int dl, int R, cudaStream_t s) {
  switch (dl) {
    case 8: return launch_dl<Real, 8, MODE>(a, R, s);
    case 16: return launch_dl<Real, 16, MODE>(a, R, s);
    case 32: return launch_dl<Real, 32, MODE>(a, R, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------------------
// 1D slab: one CTA per slot, affine-map scan.
// ---------------------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;

template <class Real>
struct Aff {
  Real a, b;  // x -> a x + b
};
template <class Real>
__device__ __forceinline__ Aff<Real> compose(Aff<Real> first, Aff<Real> then) {
  return {then.a * first.a, then.a * first.b + then.b};
}

// Exclusive scan of per-thread affine maps; returns the value entering this thread's
// chunk when the recurrence starts from ghost value g.
template <class Real>
__device__ Real block_scan_entry(Aff<Real> mine, Real g, Aff<Real>* sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  Aff<Real> inc = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    Aff<Real> prev;
    prev.a = __shfl_up_sync(FULL, inc.a, o);
    prev.b = __shfl_up_sync(FULL, inc.b, o);
    if (lane >= o) inc = compose(prev, inc);
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    Aff<Real> w = (lane < SCAN_THREADS / 32) ? sh[lane] : Aff<Real>{Real(1), Real(0)};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      Aff<Real> prev;
      prev.a = __shfl_up_sync(FULL, w.a, o);
      prev.b = __shfl_up_sync(FULL, w.b, o);
      if (lane >= o) w = compose(prev, w);
    }
    if (lane < SCAN_THREADS / 32) sh[32 + lane] = w;  // inclusive per-warp prefix
  }
  __syncthreads();
  // exclusive prefix of this thread = (prefix of earlier warps) then (earlier lanes of this warp)
  Aff<Real> ex_lane;
  ex_lane.a = __shfl_up_sync(FULL, inc.a, 1);
  ex_lane.b = __shfl_up_sync(FULL, inc.b, 1);
  if (lane == 0) ex_lane = {Real(1), Real(0)};
  Aff<Real> ex = ex_lane;
  if (warp > 0) ex = compose(sh[32 + warp - 1], ex_lane);
  __syncthreads();
  return ex.a * g + ex.b;
}

template <class Real, int MODE>
__global__ void __launch_bounds__(SCAN_THREADS) sweep1d_kernel(const Sweep1DArgs<Real> A) {
  __shared__ Aff<Real> sh[64];
  const int slot = blockIdx.x;
  const int nx = A.nx;
  const int chunk = (nx + SCAN_THREADS - 1) / SCAN_THREADS;
  const int k0 = threadIdx.x * chunk;
  const int k1 = min(nx, k0 + chunk);
  const bool pos = A.dir_sign[slot] > 0;
  const Real ca = A.a[slot], cw = A.w[slot];
  const Real ct = A.tau + ca;
  // pass A (MODE 1) or the only pass (MODE 0)
  Aff<Real> mine{Real(1), Real(0)};
  for (int k = k0; k < k1; ++k) {
    const int c = pos ? k : nx - 1 - k;
    const Real dinv = Real(1) / (ct + A.sig_t[c]);
    Real s = (MODE == 2) ? A.g2[c] : A.q[c];
    if (MODE != 0) s += A.tau * A.f[(long)c * A.nslot + slot];
    mine = compose(mine, Aff<Real>{ca * dinv, s * dinv});
  }
  const Real gA = (MODE == 2) ? Real(0) : (pos ? A.g_lo : A.g_hi);
  Real psi = block_scan_entry(mine, gA, sh);
  for (int k = k0; k < k1; ++k) {
    const int c = pos ? k : nx - 1 - k;
    const Real dinv = Real(1) / (ct + A.sig_t[c]);
    Real s = (MODE == 2) ? A.g2[c] : A.q[c];
    if (MODE == 2) {
      s += A.tau * A.f[(long)c * A.nslot + slot];
      psi = (s + ca * psi) * dinv;
      A.psi_w[(long)slot * nx + c] = cw * psi;
    } else if (MODE == 1) {
      Real* fp = A.f + (long)c * A.nslot + slot;
      s += A.tau * (*fp);
      psi = (s + ca * psi) * dinv;
      *fp = psi;
      if (A.psi_w_a) A.psi_w_a[(long)slot * nx + c] = cw * psi;
    } else {
      psi = (s + ca * psi) * dinv;
      A.psi_w[(long)slot * nx + c] = cw * psi;
    }
  }
  if (MODE == 1) {
    // pass B: y = L^-1 (g2 + tau f^n), zero inflow; this thread reads back its own writes.
    Aff<Real> mb{Real(1), Real(0)};
    for (int k = k0; k < k1; ++k) {
      const int c = pos ? k : nx - 1 - k;
      const Real dinv = Real(1) / (ct + A.sig_t[c]);
      const Real s = A.g2[c] + A.tau * A.f[(long)c * A.nslot + slot];
      mb = compose(mb, Aff<Real>{ca * dinv, s * dinv});
    }
    Real y = block_scan_entry(mb, Real(0), sh);
    for (int k = k0; k < k1; ++k) {
      const int c = pos ? k : nx - 1 - k;
      const Real dinv = Real(1) / (ct + A.sig_t[c]);
      const Real s = A.g2[c] + A.tau * A.f[(long)c * A.nslot + slot];
      y = (s + ca * y) * dinv;
      A.psi_w[(long)slot * nx + c] = cw * y;
    }
  }
}

template <class Real>
__global__ void moment1d_kernel(const Real* psi_w, int nslot, int ncell, Real* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  Real s = Real(0);
  for (int k = 0; k < nslot; ++k) s += psi_w[(long)k * ncell + c];
  out[c] = s;
}

template <class Real>
__global__ void inv_d_kernel(const Real* sig_t, const Real* a, const Real* b, Real tau, int ncell,
                             int nslot, Real* inv_d) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)ncell * nslot) return;
  const long c = i / nslot;
  const int s = (int)(i % nslot);
  inv_d[i] = Real(1) / (tau + sig_t[c] + a[s] + b[s]);
}

}  // namespace

// The 2D kernels are instantiated in six translation units (precision x mode) so that the
// build compiles them in parallel: RTE_SWEEP_PART selects one, -1 builds everything.
#ifndef RTE_SWEEP_PART
#define RTE_SWEEP_PART -1
#endif

template <class Real, int MODE>
cudaError_t launch_sweep2d_mode(const Sweep2DArgs<Real>& a, int dl, int R, cudaStream_t s) {
  return launch_mode_impl<Real, MODE>(a, dl, R, s);
}

#define RTE_SWEEP_INST(PART, REAL, MODE)                                                        \
  template cudaError_t launch_sweep2d_mode<REAL, MODE>(const Sweep2DArgs<REAL>&, int, int,      \
                                                       cudaStream_t);
#define RTE_SWEEP_EXTERN(REAL, MODE)                                                           \
  extern template cudaError_t launch_sweep2d_mode<REAL, MODE>(const Sweep2DArgs<REAL>&, int,   \
                                                              int, cudaStream_t);

#if RTE_SWEEP_PART == -1 || RTE_SWEEP_PART == 0
RTE_SWEEP_INST(0, double, 0)
#endif
#if RTE_SWEEP_PART == -1 || RTE_SWEEP_PART == 1
RTE_SWEEP_INST(1, double, 1)
#endif
#if RTE_SWEEP_PART == -1 || RTE_SWEEP_PART == 2
RTE_SWEEP_INST(2, double, 2)
#endif
#if RTE_SWEEP_PART == -1 || RTE_SWEEP_PART == 3
RTE_SWEEP_INST(3, float, 0)
#endif
#if RTE_SWEEP_PART == -1 || RTE_SWEEP_PART == 4
RTE_SWEEP_INST(4, float, 1)
#endif
#if RTE_SWEEP_PART == -1 || RTE_SWEEP_PART == 5
RTE_SWEEP_INST(5, float, 2)
#endif

#if RTE_SWEEP_PART == -1 || RTE_SWEEP_PART == 6
#if RTE_SWEEP_PART == 6
RTE_SWEEP_EXTERN(double, 0)
RTE_SWEEP_EXTERN(double, 1)
RTE_SWEEP_EXTERN(double, 2)
RTE_SWEEP_EXTERN(float, 0)
RTE_SWEEP_EXTERN(float, 1)
RTE_SWEEP_EXTERN(float, 2)
#endif
template <class Real>
cudaError_t launch_sweep2d(const Sweep2DArgs<Real>& a, int mode, int R, cudaStream_t s) {
  const int dl = a.nslot / a.nfam;
  if (mode == 0) return launch_sweep2d_mode<Real, 0>(a, dl, R, s);
  if (mode == 2) return launch_sweep2d_mode<Real, 2>(a, dl, R, s);
  return launch_sweep2d_mode<Real, 1>(a, dl, R, s);
}

template <class Real>
cudaError_t launch_sweep1d(const Sweep1DArgs<Real>& a, int mode, cudaStream_t s) {
  ++g_launches;
  if (mode == 0)
    sweep1d_kernel<Real, 0><<<a.nslot, SCAN_THREADS, 0, s>>>(a);
  else if (mode == 2)
    sweep1d_kernel<Real, 2><<<a.nslot, SCAN_THREADS, 0, s>>>(a);
  else
    sweep1d_kernel<Real, 1><<<a.nslot, SCAN_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

template <class Real>
cudaError_t launch_moment1d(const Real* psi_w, int nslot, int ncell, Real* out, cudaStream_t s) {
  ++g_launches;
  moment1d_kernel<Real><<<(ncell + 255) / 256, 256, 0, s>>>(psi_w, nslot, ncell, out);
  return cudaGetLastError();
}

template <class Real>
cudaError_t launch_inv_d(const Real* sig_t, const Real* a, const Real* b, Real tau, int ncell,
                         int nslot, Real* inv_d, cudaStream_t s) {
  const long n = (long)ncell * nslot;
  ++g_launches;
  inv_d_kernel<Real><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sig_t, a, b, tau, ncell, nslot,
                                                                 inv_d);
  return cudaGetLastError();
}

template cudaError_t launch_sweep2d<double>(const Sweep2DArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_sweep2d<float>(const Sweep2DArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_sweep1d<double>(const Sweep1DArgs<double>&, int, cudaStream_t);
template cudaError_t launch_sweep1d<float>(const Sweep1DArgs<float>&, int, cudaStream_t);
template cudaError_t launch_moment1d<double>(const double*, int, int, double*, cudaStream_t);
template cudaError_t launch_moment1d<float>(const float*, int, int, float*, cudaStream_t);
template cudaError_t launch_inv_d<double>(const double*, const double*, const double*, double, int,
                                          int, double*, cudaStream_t);
template cudaError_t launch_inv_d<float>(const float*, const float*, const float*, float, int, int,
                                         float*, cudaStream_t);
#endif  // base part

}  // namespace rte
