// Cell-vector kernels of the SI-SA loop (Algorithm 1): the residual and convergence test of
// Sec. 2.3 (||rho^{l-1/2} - rho^{l-1}||_inf), the density update rho^l = rho^{l-1/2} + delta,
// and small reductions.  All FP64; reductions use a fixed block partition and a fixed
// summation order, so results are bitwise reproducible.
#include <cuda_runtime.h>

#include "rte_internal.h"

namespace rte {

namespace {
constexpr int VT = 256;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
  return v;
}

// rho_half = sum_f pm[f] + btilde; diff = rho_half - rho_prev; per-block max|diff|,
// max|rho_half|, sum diff^2.
__global__ void combine_residual_kernel(const double* __restrict__ pm, int nfam,
                                        const double* __restrict__ btilde,
                                        const double* __restrict__ rho_prev, int n,
                                        double* __restrict__ rho_half, double* __restrict__ copy1,
                                        double* __restrict__ copy2, double* partials,
                                        unsigned* skip, unsigned* ticket, Norms* out, double eps,
                                        int absmode, ResidualLoop loop) {
  if (skip && *skip) {   // the solve has converged: speculative work does nothing
    if (loop.count && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(loop.cond, 0u);
    return;
  }
  __shared__ double sh[3][VT / 32];
  double dinf = 0.0, hinf = 0.0, d2 = 0.0;
  for (int c = blockIdx.x * VT + threadIdx.x; c < n; c += gridDim.x * VT) {
    double s = 0.0;
    for (int f = 0; f < nfam; ++f) s += pm[(long)f * n + c];
    s += btilde[c];
    rho_half[c] = s;
    if (copy1) copy1[c] = s;
    if (copy2) copy2[c] = s;
    const double d = s - rho_prev[c];
    dinf = fmax(dinf, fabs(d));
    hinf = fmax(hinf, fabs(s));
    d2 += d * d;
  }
  dinf = warp_max(dinf);
  hinf = warp_max(hinf);
  d2 = warp_sum(d2);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sh[0][w] = dinf;
    sh[1][w] = hinf;
    sh[2][w] = d2;
  }
  __syncthreads();
  if (w == 0) {
    dinf = l < VT / 32 ? sh[0][l] : 0.0;
    hinf = l < VT / 32 ? sh[1][l] : 0.0;
    d2 = l < VT / 32 ? sh[2][l] : 0.0;
    dinf = warp_max(dinf);
    hinf = warp_max(hinf);
    d2 = warp_sum(d2);
    if (l == 0) {
      partials[3 * blockIdx.x + 0] = dinf;
      partials[3 * blockIdx.x + 1] = hinf;
      partials[3 * blockIdx.x + 2] = d2;
    }
  }
  {
    // the last block to finish forms the norms and the stopping test (the host makes the same
    // comparison; later speculative launches read it as their skip word) from every block's
    // partials in a fixed order, and re-arms the ticket
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last && w == 0) {
      __threadfence();
      double dmax = 0.0, hmax = 0.0, dsum = 0.0;
      for (int b = l; b < (int)gridDim.x; b += 32) {
        dmax = fmax(dmax, __ldcg(partials + 3 * b));
        hmax = fmax(hmax, __ldcg(partials + 3 * b + 1));
        dsum += __ldcg(partials + 3 * b + 2);
      }
      dmax = warp_max(dmax);
      hmax = warp_max(hmax);
      dsum = warp_sum(dsum);
      if (l == 0) {
        out->diff_inf = dmax;
        out->half_inf = hmax;
        out->diff_l2sq = dsum;
        const bool conv = absmode ? dmax <= eps : dmax <= eps * hmax;
        if (skip) *skip = conv ? 1u : 0u;
        if (loop.count) {   // one more iteration of the graph's loop unless this one converged,
                            // the cap is reached or a bounded wait of the iteration ran out
          const unsigned c = *loop.count + 1u;
          *loop.count = c;
          const bool failed = (loop.err0 && __ldcg(loop.err0)) || (loop.err1 && __ldcg(loop.err1));
          cudaGraphSetConditional(loop.cond, !conv && !failed && c < loop.limit ? 1u : 0u);
        }
        *ticket = 0u;
      }
    }
  }
}

__global__ void update_rho_kernel(const double* rho_half, const double* delta, const double* sig_s,
                                  int n, double* rho, double* q) {
  const int c = blockIdx.x * VT + threadIdx.x;
  if (c >= n) return;
  const double r = rho_half[c] + delta[c];
  rho[c] = r;
  q[c] = sig_s[c] * r;
}

__global__ void scale_copy_kernel(const double* x, const double* sig_s, int n, double* q) {
  const int c = blockIdx.x * VT + threadIdx.x;
  if (c >= n) return;
  q[c] = sig_s[c] * x[c];
}

__global__ void sum_partials_kernel(const double* pm, int nfam, int n, const double* add,
                                    double* out) {
  const int c = blockIdx.x * VT + threadIdx.x;
  if (c >= n) return;
  double s = 0.0;
  for (int f = 0; f < nfam; ++f) s += pm[(long)f * n + c];
  if (add) s += add[c];
  out[c] = s;
}

__global__ void axpby_kernel(double alpha, const double* x, double beta, const double* y, int n,
                             double* out) {
  const int c = blockIdx.x * VT + threadIdx.x;
  if (c >= n) return;
  out[c] = alpha * x[c] + beta * y[c];
}

// f = rho in every direction; f layout [family][cell][lane] with nslot / dl families.
__global__ void isotropic_f_kernel(const double* rho, int n, int nslot, int dl, const double* w,
                                   double* f) {
  const long i = (long)blockIdx.x * VT + threadIdx.x;
  if (i >= (long)n * nslot) return;
  const long c = (i / dl) % n;
  // family layout [fam][cell][dl]: slot = fam * dl + lane
  f[i] = w ? w[(i / ((long)n * dl)) * dl + i % dl] * rho[c] : rho[c];
}

// Q1: f[fam][cell][k][dl] = rho[k ncell + cell] (mode-major rho) in every slot.
__global__ void isotropic_f_q1_kernel(const double* rho, int ncell, int nslot, int dl, double* f) {
  const long i = (long)blockIdx.x * VT + threadIdx.x;
  if (i >= 4L * ncell * nslot) return;
  const long k = (i / dl) % 4, c = (i / (4L * dl)) % ncell;
  f[i] = rho[k * ncell + c];
}

__global__ void isotropic_f32_q1_kernel(const double* rho, int ncell, int nslot, int dl, float* f) {
  const long i = (long)blockIdx.x * VT + threadIdx.x;
  if (i >= 4L * ncell * nslot) return;
  const long k = (i / dl) % 4, c = (i / (4L * dl)) % ncell;
  f[i] = (float)rho[k * ncell + c];
}

__global__ void dot_partial_kernel(const double* x, const double* y, int n, double* partials) {
  __shared__ double sh[VT / 32];
  double s = 0.0;
  for (int c = blockIdx.x * VT + threadIdx.x; c < n; c += gridDim.x * VT) s += x[c] * y[c];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < VT / 32 ? sh[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

__global__ void dot_finish_kernel(const double* partials, int nblocks, double* out) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 32) s += partials[b];
  s = warp_sum(s);
  if (threadIdx.x == 0) *out = s;
}

// out = Real(sigma_s (x - xref)) (xref may be nullptr); with `update`, xref <- x afterwards.
template <class Real>
__global__ void scaled_diff_kernel(const double* x, double* xref, const double* sig_s, int n,
                                   Real* out, int update, const unsigned* skip) {
  const int c = blockIdx.x * VT + threadIdx.x;
  if (c >= n || (skip && *skip)) return;
  const double xv = x[c];
  const double d = xref ? xv - xref[c] : xv;
  out[c] = (Real)(sig_s[c] * d);
  if (update) xref[c] = xv;
}

// out = Real(sigma_s rho + G)
template <class Real>
__global__ void scaled_plus_kernel(const double* rho, const double* sig_s, const double* src,
                                   int n, Real* out) {
  const int c = blockIdx.x * VT + threadIdx.x;
  if (c >= n) return;
  out[c] = (Real)(sig_s[c] * rho[c] + src[c]);
}

// out (+)= sum over families of pm, accumulated in FP64 in family order
template <class Real>
__global__ void sum_pm_kernel(const Real* pm, int nfam, int n, double* out, int accumulate,
                              const unsigned* skip) {
  const int c = blockIdx.x * VT + threadIdx.x;
  if (c >= n || (skip && *skip)) return;
  double s = 0.0;
  for (int f = 0; f < nfam; ++f) s += (double)pm[(long)f * n + c];
  out[c] = accumulate ? out[c] + s : s;
}

__global__ void isotropic_f32_kernel(const double* rho, int n, int nslot, int dl, float* f) {
  const long i = (long)blockIdx.x * VT + threadIdx.x;
  if (i >= (long)n * nslot) return;
  f[i] = (float)rho[(i / dl) % n];
}

__global__ void to_float_kernel(const double* x, long n, float* y) {
  const long i = (long)blockIdx.x * VT + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

}  // namespace

template <class Real>
cudaError_t launch_scaled_diff(const double* x, const double* xref, const double* sig_s, int n,
                               Real* out, cudaStream_t s, const unsigned* skip) {
  ++g_launches;
  scaled_diff_kernel<Real><<<(n + VT - 1) / VT, VT, 0, s>>>(x, const_cast<double*>(xref), sig_s, n,
                                                            out, 0, skip);
  return cudaGetLastError();
}
template <class Real>
cudaError_t launch_scaled_diff_update(const double* x, double* xref, const double* sig_s, int n,
                                      Real* out, cudaStream_t s, const unsigned* skip) {
  ++g_launches;
  scaled_diff_kernel<Real><<<(n + VT - 1) / VT, VT, 0, s>>>(x, xref, sig_s, n, out, 1, skip);
  return cudaGetLastError();
}
template <class Real>
cudaError_t launch_scaled_plus(const double* rho, const double* sig_s, const double* src, int n,
                               Real* out, cudaStream_t s) {
  ++g_launches;
  scaled_plus_kernel<Real><<<(n + VT - 1) / VT, VT, 0, s>>>(rho, sig_s, src, n, out);
  return cudaGetLastError();
}
template <class Real>
cudaError_t launch_sum_pm(const Real* pm, int nfam, int n, double* out, int accumulate,
                          cudaStream_t s, const unsigned* skip) {
  ++g_launches;
  sum_pm_kernel<Real><<<(n + VT - 1) / VT, VT, 0, s>>>(pm, nfam, n, out, accumulate, skip);
  return cudaGetLastError();
}
cudaError_t launch_isotropic_f32(const double* rho, int n, int nslot, int dl, float* f,
                                 cudaStream_t s) {
  const long tot = (long)n * nslot;
  ++g_launches;
  isotropic_f32_kernel<<<(unsigned)((tot + VT - 1) / VT), VT, 0, s>>>(rho, n, nslot, dl, f);
  return cudaGetLastError();
}
namespace {
// BDF2 history after a step: f holds f^n, prev holds f^{n-1}; afterwards f holds the next
// step's history h^{n+1} = (4 f^n - f^{n-1}) / 3 and prev holds f^n.
template <class Real>
__global__ void bdf2_history_kernel(Real* f, Real* prev, long n) {
  const long i = (long)blockIdx.x * VT + threadIdx.x;
  if (i >= n) return;
  const Real t = f[i];
  f[i] = (Real(4) * t - prev[i]) * (Real(1) / Real(3));
  prev[i] = t;
}
}  // namespace

template <class Real>
cudaError_t launch_bdf2_history(Real* f, Real* prev, long n, cudaStream_t s) {
  ++g_launches;
  bdf2_history_kernel<Real><<<(unsigned)((n + VT - 1) / VT), VT, 0, s>>>(f, prev, n);
  return cudaGetLastError();
}
template cudaError_t launch_bdf2_history<double>(double*, double*, long, cudaStream_t);
template cudaError_t launch_bdf2_history<float>(float*, float*, long, cudaStream_t);

cudaError_t launch_to_float(const double* x, long n, float* y, cudaStream_t s) {
  ++g_launches;
  to_float_kernel<<<(unsigned)((n + VT - 1) / VT), VT, 0, s>>>(x, n, y);
  return cudaGetLastError();
}
template cudaError_t launch_scaled_diff<double>(const double*, const double*, const double*, int,
                                                double*, cudaStream_t, const unsigned*);
template cudaError_t launch_scaled_diff<float>(const double*, const double*, const double*, int,
                                               float*, cudaStream_t, const unsigned*);
template cudaError_t launch_scaled_diff_update<float>(const double*, double*, const double*, int,
                                                      float*, cudaStream_t, const unsigned*);
template cudaError_t launch_scaled_diff_update<double>(const double*, double*, const double*, int,
                                                       double*, cudaStream_t, const unsigned*);
template cudaError_t launch_scaled_plus<double>(const double*, const double*, const double*, int,
                                                double*, cudaStream_t);
template cudaError_t launch_scaled_plus<float>(const double*, const double*, const double*, int,
                                               float*, cudaStream_t);
template cudaError_t launch_sum_pm<double>(const double*, int, int, double*, int, cudaStream_t,
                                          const unsigned*);
template cudaError_t launch_sum_pm<float>(const float*, int, int, double*, int, cudaStream_t,
                                         const unsigned*);

int vec_blocks(int n) {
  int b = (n + VT - 1) / VT;
  return b < 1 ? 1 : (b > 1024 ? 1024 : b);
}

namespace {
// Start of an SI-SA solve: the initial guess copied into place (dst1, and dst2 when given),
// the skip word cleared and the CG iteration slots zeroed, in one launch.
__global__ void si_begin_kernel(const double* __restrict__ src, double* __restrict__ dst1,
                                double* __restrict__ dst2, int n, unsigned* conv, int* slots,
                                int nslots) {
  const int i = blockIdx.x * VT + threadIdx.x;
  if (i < n) {
    const double v = src[i];
    dst1[i] = v;
    if (dst2) dst2[i] = v;
  }
  if (blockIdx.x == 0) {
    for (int k = threadIdx.x; k < nslots; k += VT) slots[k] = 0;
    if (threadIdx.x == 0) *conv = 0u;
  }
}
}  // namespace

cudaError_t launch_si_begin(const double* src, double* dst1, double* dst2, int n, unsigned* conv,
                            int* slots, int nslots, cudaStream_t s) {
  ++g_launches;
  si_begin_kernel<<<(n + VT - 1) / VT, VT, 0, s>>>(src, dst1, dst2, n, conv, slots, nslots);
  return cudaGetLastError();
}

cudaError_t launch_combine_residual(const double* pm, int nfam, const double* btilde,
                                    const double* rho_prev, int n, double* rho_half,
                                    double* partials, int nblocks, Norms* out, cudaStream_t s,
                                    unsigned* conv, double eps, int absmode, double* copy1,
                                    double* copy2, unsigned* ticket, ResidualLoop loop) {
  if (!ticket) return cudaErrorInvalidValue;
  ++g_launches;
  combine_residual_kernel<<<nblocks, VT, 0, s>>>(pm, nfam, btilde, rho_prev, n, rho_half, copy1,
                                                 copy2, partials, conv, ticket, out, eps, absmode,
                                                 loop);
  return cudaGetLastError();
}

cudaError_t launch_update_rho(const double* rho_half, const double* delta, const double* sig_s,
                              int n, double* rho, double* q, cudaStream_t s) {
  ++g_launches;
  update_rho_kernel<<<(n + VT - 1) / VT, VT, 0, s>>>(rho_half, delta, sig_s, n, rho, q);
  return cudaGetLastError();
}

cudaError_t launch_scale_copy(const double* x, const double* sig_s, int n, double* q,
                              cudaStream_t s) {
  ++g_launches;
  scale_copy_kernel<<<(n + VT - 1) / VT, VT, 0, s>>>(x, sig_s, n, q);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* pm, int nfam, int n, const double* add, double* out,
                                cudaStream_t s) {
  ++g_launches;
  sum_partials_kernel<<<(n + VT - 1) / VT, VT, 0, s>>>(pm, nfam, n, add, out);
  return cudaGetLastError();
}

cudaError_t launch_axpby(double alpha, const double* x, double beta, const double* y, int n,
                         double* out, cudaStream_t s) {
  ++g_launches;
  axpby_kernel<<<(n + VT - 1) / VT, VT, 0, s>>>(alpha, x, beta, y, n, out);
  return cudaGetLastError();
}

cudaError_t launch_isotropic_f(const double* rho, int n, int nslot, int dl, const double* w,
                               double* f, cudaStream_t s) {
  const long tot = (long)n * nslot;
  ++g_launches;
  isotropic_f_kernel<<<(unsigned)((tot + VT - 1) / VT), VT, 0, s>>>(rho, n, nslot, dl, w, f);
  return cudaGetLastError();
}

cudaError_t launch_isotropic_f_q1(const double* rho, int ncell, int nslot, int dl, double* f,
                                  cudaStream_t s) {
  const long tot = 4L * ncell * nslot;
  ++g_launches;
  isotropic_f_q1_kernel<<<(unsigned)((tot + VT - 1) / VT), VT, 0, s>>>(rho, ncell, nslot, dl, f);
  return cudaGetLastError();
}

cudaError_t launch_isotropic_f32_q1(const double* rho, int ncell, int nslot, int dl, float* f,
                                    cudaStream_t s) {
  const long tot = 4L * ncell * nslot;
  ++g_launches;
  isotropic_f32_q1_kernel<<<(unsigned)((tot + VT - 1) / VT), VT, 0, s>>>(rho, ncell, nslot, dl, f);
  return cudaGetLastError();
}

namespace {
// ROM update gate of Algorithm 2: open when forced, when the gate it follows is open, or when
// the indicator sqrt(e2) exceeds eps_up (times ||rho|| = sqrt(n2) when relative).
__global__ void rom_gate_kernel(const double* e2, const double* n2, double eps_up, int rel,
                                int force, const int* also, int* gate) {
  if (threadIdx.x != 0) return;
  const double thr = eps_up * (rel ? sqrt(*n2) : 1.0);
  const bool open = force || (also && *also != 0) || !(sqrt(*e2) <= thr);
  *gate = open ? 1 : 0;
}
}  // namespace

cudaError_t launch_rom_gate(const double* e2, const double* n2, double eps_up, int rel, int force,
                            const int* also, int* gate, cudaStream_t s) {
  ++g_launches;
  rom_gate_kernel<<<1, 32, 0, s>>>(e2, n2, eps_up, rel, force, also, gate);
  return cudaGetLastError();
}

cudaError_t launch_dot(const double* x, const double* y, int n, double* partials, int nblocks,
                       double* out, cudaStream_t s) {
  ++g_launches;
  dot_partial_kernel<<<nblocks, VT, 0, s>>>(x, y, n, partials);
  ++g_launches;
  dot_finish_kernel<<<1, 32, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

}  // namespace rte
