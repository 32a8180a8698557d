// On-the-fly reduced-order models (Sec. 3.1, 3.2, App. B), FP64.
//
// A ROM keeps the thin SVD R ~ U S V^T of its solution snapshots and W = B V (B the
// right-hand-side snapshots), so that the DMD operator of Eq. (dmd-operator) is
// A_r = U^T W S^{-1}; V itself is never stored.
//
// Append (App. B, Eq. (svd_core)), one snapshot pair (x, b):
//   p = U^T x;  q~ = x - U p;  repeated once (classical Gram-Schmidt twice);
//   alpha = ||q~||; the rank grows iff alpha > 1e-12 ||x|| (else q is dropped);
//   K = [[S, p], [0, alpha]] = U_c S_c V_c^T  (secular equation of the broken-arrow form,
//   FP64, csvd.cu);
//   keep = r+1 (or r), truncated to s_k / sum s > eps when asked, capped at r_max;
//   U <- [U q] U_c(:, :keep);  W <- [W b] V_c(:, :keep);
//   G = U^T W <- U_c^T [[G, U^T b], [q^T W, q^T b]] V_c;  A_r = G S^{-1} and its inverse by
//   Gauss-Jordan elimination with partial pivoting (the paper solves the reduced system by LU;
//   the explicit inverse turns every later solve into a small matrix-vector product).
// Apply (Eq. (dmd-ig), Eq. (dmd-sa)): out = U A_r^{-1} U^T rhs.
//
// The bases are kept in the factored form of Brand's method: U = U0 Q and W = W0 P, where
// U0 and W0 (N_x x w) only ever gain columns (q when the rank grows, b always) and the
// small Q, P (w x r) absorb the rotations U_c, V_c.  An append therefore costs a few
// N_x x w matrix-vector products instead of two N_x x (r+1)^2 rotations; when w reaches
// its capacity the factors are multiplied out once (U0 <- U0 Q, Q <- I).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <utility>

#include "rte_internal.h"

namespace rte {

namespace {
constexpr unsigned FULL = 0xffffffffu;
constexpr int GT = 256;          // rows per GEMV block
constexpr int MAXR = 65;         // r_max + 1 <= 65
constexpr int WCAP = 96;         // columns of U0 / W0
constexpr int COMPACT_SLACK = 24;  // stored columns beyond the rank that trigger a compaction
constexpr int TALL_ROWS = 64;    // rows per tall x small product block

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Partial U^T x: warp (blockIdx.x, blockIdx.y) takes rows [256 bx, 256 bx + 256) and columns
// [8 by, 8 by + 8); each lane forms 8 column sums over its 8 rows, and a transpose-reduce over
// the warp leaves the tile's sum of column c in lane 4c.  partial[k * nb + bx].
constexpr int GV_ROWS = 256, GV_COLS = 8;
__global__ void __launch_bounds__(32) gemv_t_partial(const double* __restrict__ U, long n, int w,
                                                     const double* __restrict__ x,
                                                     double* __restrict__ partial) {
  const int lane = threadIdx.x;
  const long r0 = (long)blockIdx.x * GV_ROWS;
  const int c0 = blockIdx.y * GV_COLS;
  double xv[GV_ROWS / 32];
#pragma unroll
  for (int i = 0; i < GV_ROWS / 32; ++i) {
    const long row = r0 + lane + 32 * i;
    xv[i] = row < n ? x[row] : 0.0;
  }
  double v[GV_COLS];
#pragma unroll
  for (int c = 0; c < GV_COLS; ++c) {
    double s = 0.0;
    if (c0 + c < w) {
      const double* u = U + (long)(c0 + c) * n;
#pragma unroll
      for (int i = 0; i < GV_ROWS / 32; ++i) {
        const long row = r0 + lane + 32 * i;
        if (row < n) s += u[row] * xv[i];
      }
    }
    v[c] = s;
  }
  // transpose-reduce 8 values over 32 lanes: after 3 halving rounds and 2 butterflies the
  // sum of column c sits in lanes 4c .. 4c+3
#pragma unroll
  for (int o = 16, m = GV_COLS; o >= 4; o >>= 1, m >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < m / 2; ++i) {
      const double send = hi ? v[i] : v[i + m / 2];
      const double keep = hi ? v[i + m / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(FULL, send, o);
    }
  }
  v[0] += __shfl_xor_sync(FULL, v[0], 2);
  v[0] += __shfl_xor_sync(FULL, v[0], 1);
  const int c = lane >> 2;
  if ((lane & 3) == 0 && c0 + c < w) partial[(long)(c0 + c) * gridDim.x + blockIdx.x] = v[0];
}

// out[k] = sum_b partial[k * nb + b], fixed order.
__global__ void gemv_t_finish(const double* partial, int nb, int w, double* out) {
  const int k = blockIdx.x;
  if (k >= w) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) s += partial[(long)k * nb + b];
  s = warp_sum(s);
  if (threadIdx.x == 0) out[k] = s;
}

// out[i] = cx * x[i] - sign * sum_k U[k n + i] c[k]   (sign = +1: x - U c; sign = -1: U c)
__global__ void gemv_n(const double* __restrict__ U, long n, int w, const double* __restrict__ c,
                       double cx, const double* x, double sign, double* out) {
  __shared__ double cs[WCAP];
  if (threadIdx.x < w) cs[threadIdx.x] = c[threadIdx.x];
  __syncthreads();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int k = 0; k < w; ++k) s += U[(long)k * n + i] * cs[k];
  out[i] = (x ? cx * x[i] : 0.0) - sign * s;
}

__global__ void dot_partial(const double* x, const double* y, long n, double* partial) {
  __shared__ double sh[GT / 32];
  double s = 0.0;
  for (long i = (long)blockIdx.x * GT + threadIdx.x; i < n; i += (long)gridDim.x * GT)
    s += x[i] * y[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < GT / 32 ? sh[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

// y[j] = sum_{i<rows} M[i*MAXR + j] v[i] for j < cols  (M^T v; M row-major, ld MAXR);
// one warp per output.
__global__ void small_t_kernel(const double* M, int rows, int cols, const double* v, double* y) {
  const int lane = threadIdx.x & 31;
  for (int j = threadIdx.x >> 5; j < cols; j += blockDim.x >> 5) {
    double s = 0.0;
    for (int i = lane; i < rows; i += 32) s += M[i * MAXR + j] * v[i];
    s = warp_sum(s);
    if (lane == 0) y[j] = s;
  }
}

// y[i] = sum_{j<cols} M[i*MAXR + j] v[j] for i < rows  (M v); one warp per output.
__global__ void small_n_kernel(const double* M, int rows, int cols, const double* v, double* y) {
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x >> 5; i < rows; i += blockDim.x >> 5) {
    double s = 0.0;
    for (int j = lane; j < cols; j += 32) s += M[i * MAXR + j] * v[j];
    s = warp_sum(s);
    if (lane == 0) y[i] = s;
  }
}

__global__ void add_vec_kernel(double* a, const double* b, int r) {
  if ((int)threadIdx.x < r) a[threadIdx.x] += b[threadIdx.x];
}

// Scratch layout of one ROM (device doubles).
struct Scr {
  double* p;      // [MAXR]  U^T x (after CGS2)
  double* p2;     // [MAXR]  second-pass projection, then the new singular values
  double* ub;     // [MAXR]  U^T b
  double* wq;     // [MAXR]  W^T q
  double* sc;     // [16]    0: ||x||^2  1: alpha^2  2: q.b  3: 1/alpha (0 if no growth)
                  //         4: keep  5: grew  6: stop ratio  7: lu_ok
  double* Uc;     // [MAXR*MAXR] column-major (ld r+1), sorted
  double* Vc;     // [MAXR*MAXR]
  double* G;      // [MAXR*MAXR] row-major U^T W (rank x rank)
  double* Gx;     // [MAXR*MAXR] extended G, row-major (ld r+1)
  double* T;      // [MAXR*MAXR] Gx V_c, row-major (ld keep)
  double* w0;     // [WCAP] U0^T / W0^T projections
  double* c0;     // [WCAP] Q p
};

Scr scr_of(double* core) {
  Scr s;
  double* w = core;
  s.p = w; w += MAXR;
  s.p2 = w; w += MAXR;
  s.ub = w; w += MAXR;
  s.wq = w; w += MAXR;
  s.sc = w; w += 16;
  s.Uc = w; w += MAXR * MAXR;
  s.Vc = w; w += MAXR * MAXR;
  s.G = w; w += MAXR * MAXR;
  s.Gx = w; w += MAXR * MAXR;
  s.T = w; w += MAXR * MAXR;
  s.w0 = w; w += WCAP;
  s.c0 = w; w += WCAP;
  return s;
}
constexpr long SCR_DOUBLES = 4 * MAXR + 16 + 5 * MAXR * MAXR + 2 * WCAP;

// scaled copy q = q~ * (1/alpha) (0 when the rank does not grow)
__global__ void scale_q_kernel(double* q, long n, const double* sc) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] *= sc[3];
}

// Gx = [[G, U^T b], [q^T W, q^T b]]  ((r+1) x (r+1), row-major, ld r+1)
__global__ void build_gx_kernel(int r, Scr sc) {
  const int n = r + 1;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    double v;
    if (i < r && j < r) v = sc.G[i * MAXR + j];
    else if (i < r) v = sc.ub[i];
    else if (j < r) v = sc.wq[j];
    else v = sc.sc[2];
    sc.Gx[e] = v;
  }
}

// T = Gx V_c  (n x keep); one block per output column.
__global__ void gx_times_vc_kernel(int r, Scr sc) {
  const int n = r + 1, keep = (int)sc.sc[4], b = blockIdx.x;
  if (b >= keep) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += sc.Gx[i * n + j] * sc.Vc[b * n + j];
    sc.T[i * keep + b] = s;
  }
}

// G = U_c^T T  (keep x keep); one block per output column.  Skipped when the gate is 0.
__global__ void uct_times_t_kernel(int r, Scr sc, const int* gate) {
  const int n = r + 1, keep = (int)sc.sc[4], b = blockIdx.x;
  if (b >= keep || (gate && *gate == 0)) return;
  for (int a = threadIdx.x; a < keep; a += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += sc.Uc[a * n + i] * sc.T[i * keep + b];
    sc.G[a * MAXR + b] = s;
  }
}

// |x| as an ordered integer: the bits of a double without its sign compare like |x|
// (non-NaN values), so magnitude comparisons run on the integer ALU instead of the FP64 pipe.
__device__ __forceinline__ unsigned long long mag_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}

// S <- new singular values; A_r = G S^{-1}; its inverse by Gauss-Jordan elimination with
// partial pivoting (row-major, keep x keep) into inv.  Pivot search: warp-wide argmax on
// the magnitude bits.  lu_ok = 0 when a pivot falls below 1e-14 max |A_r|.  Skipped when
// the gate is 0 (the ROM keeps its state).
__global__ void __launch_bounds__(256) inverse_kernel(Scr sc, double* S, double* inv,
                                                      const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ double A[(MAXR - 1) * (MAXR - 1)];
  __shared__ double B[(MAXR - 1) * (MAXR - 1)];
  __shared__ int s_ok, s_piv;
  __shared__ unsigned long long s_wmax[8];
  const int keep = (int)sc.sc[4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long mx = 0ULL;
  for (int e = tid; e < keep * keep; e += blockDim.x) {
    const int a = e / keep, b = e % keep;
    const double v = sc.G[a * MAXR + b] / sc.p2[b];
    A[e] = v;
    B[e] = (a == b) ? 1.0 : 0.0;
    mx = max(mx, mag_bits(v));
  }
  for (int a = tid; a < keep; a += blockDim.x) S[a] = sc.p2[a];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL, mx, o));
  if (lane == 0) s_wmax[warp] = mx;
  if (tid == 0) s_ok = keep > 0 ? 1 : 0;
  __syncthreads();
  if (tid == 0) {
    unsigned long long m = 0ULL;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, s_wmax[w]);
    s_wmax[0] = m;
  }
  __syncthreads();
  const double amax = __longlong_as_double((long long)s_wmax[0]);
  for (int k = 0; k < keep; ++k) {
    if (warp == 0) {
      unsigned long long best = 0ULL;
      int p = k;
      for (int i = k + lane; i < keep; i += 32) {
        const unsigned long long m = mag_bits(A[i * keep + k]);
        if (m > best) {
          best = m;
          p = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(FULL, best, o);
        const int op = __shfl_xor_sync(FULL, p, o);
        if (ob > best || (ob == best && op < p)) {
          best = ob;
          p = op;
        }
      }
      if (lane == 0) {
        s_piv = p;
        if (!(__longlong_as_double((long long)best) > 1e-14 * amax)) s_ok = 0;
      }
    }
    __syncthreads();
    const int p = s_piv;
    if (p != k) {
      for (int j = tid; j < keep; j += blockDim.x) {
        double t = A[k * keep + j];
        A[k * keep + j] = A[p * keep + j];
        A[p * keep + j] = t;
        t = B[k * keep + j];
        B[k * keep + j] = B[p * keep + j];
        B[p * keep + j] = t;
      }
      __syncthreads();
    }
    const double dinv = 1.0 / A[k * keep + k];
    __syncthreads();
    for (int j = tid; j < keep; j += blockDim.x) {
      A[k * keep + j] *= dinv;
      B[k * keep + j] *= dinv;
    }
    __syncthreads();
    for (int e = tid; e < keep * keep; e += blockDim.x) {
      const int i = e / keep, j = e % keep;
      if (i == k) continue;
      const double f = A[i * keep + k];
      if (j != k) A[i * keep + j] -= f * A[k * keep + j];
      B[i * keep + j] -= f * B[k * keep + j];
    }
    __syncthreads();
    for (int i = tid; i < keep; i += blockDim.x)
      if (i != k) A[i * keep + k] = 0.0;
    __syncthreads();
  }
  for (int e = tid; e < keep * keep; e += blockDim.x) inv[e] = B[e];
  if (tid == 0) sc.sc[7] = s_ok;
}

// The small products of a ROM apply in one block: p = Q^T w0, c = A_r^{-1} p, c0 = Q c (Q
// row-major, ld MAXR; A_r^{-1} row-major r x r).  Each output is one warp's lane-strided sum,
// as in small_t_kernel and small_n_kernel.
__global__ void __launch_bounds__(1024) apply_core_kernel(const double* Q, int wu, int r,
                                                          const double* inv, const double* w0,
                                                          double* pc, double* c0) {
  __shared__ double p[MAXR], c[MAXR];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < r; j += nw) {
    double s = 0.0;
    for (int i = lane; i < wu; i += 32) s += Q[i * MAXR + j] * w0[i];
    s = warp_sum(s);
    if (lane == 0) p[j] = s;
  }
  __syncthreads();
  for (int i = warp; i < r; i += nw) {
    double s = 0.0;
    for (int j = lane; j < r; j += 32) s += inv[i * r + j] * p[j];
    s = warp_sum(s);
    if (lane == 0) c[i] = s;
  }
  __syncthreads();
  for (int k = warp; k < wu; k += nw) {
    double s = 0.0;
    for (int j = lane; j < r; j += 32) s += Q[k * MAXR + j] * c[j];
    s = warp_sum(s);
    if (lane == 0) c0[k] = s;
  }
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    pc[j] = p[j];
    pc[MAXR + j] = c[j];
  }
}

// Factor update M' = [[M, 0], [0, 1]] C(:, :keep) (ext = 1) or M C(0:inner0, :keep) (ext = 0),
// M row-major (rows0 x inner0, ld MAXR), C column-major (ld inner0 + 1).  ext = -1 reads the
// growth flag from sc[5].  One block per output column.
__global__ void factor_update_kernel(const double* M, int rows0, int inner0, const double* C,
                                     const double* sc, int ext, double* out) {
  const int keep = (int)sc[4], j = blockIdx.x;
  if (j >= keep) return;
  const bool grow = ext < 0 ? sc[5] != 0.0 : ext != 0;
  const int rows = rows0 + (grow ? 1 : 0);
  const int ldc = inner0 + 1;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    double s;
    if (i < rows0) {
      s = 0.0;
      for (int k = 0; k < inner0; ++k) s += M[i * MAXR + k] * C[j * ldc + k];
    } else {
      s = C[j * ldc + inner0];
    }
    out[i * MAXR + j] = s;
  }
}

// out[:, j] = sum_{k < kin} in[:, k] M[k*MAXR + j] for j < cols (tall x small, row tile in smem)
__global__ void __launch_bounds__(TALL_ROWS) tall_small_kernel(const double* __restrict__ in, long n,
                                                               int kin, const double* __restrict__ M,
                                                               int cols, double* __restrict__ out) {
  extern __shared__ double tsm[];
  double* Ms = tsm;                           // [kin][cols]
  double* tile = Ms + WCAP * (MAXR - 1);      // [TALL_ROWS][kin + 1]
  const int ld = kin + 1;
  for (int e = threadIdx.x; e < kin * cols; e += TALL_ROWS) Ms[e] = M[(e / cols) * MAXR + e % cols];
  const long i0 = (long)blockIdx.x * TALL_ROWS;
  for (int k = 0; k < kin; ++k) {
    const long i = i0 + threadIdx.x;
    tile[threadIdx.x * ld + k] = i < n ? in[(long)k * n + i] : 0.0;
  }
  __syncthreads();
  const long i = i0 + threadIdx.x;
  if (i >= n) return;
  const double* row = tile + threadIdx.x * ld;
  for (int j = 0; j < cols; ++j) {
    double s = 0.0;
    for (int k = 0; k < kin; ++k) s += row[k] * Ms[k * cols + j];
    out[(long)j * n + i] = s;
  }
}
constexpr int TALL_SMEM = (WCAP * (MAXR - 1) + TALL_ROWS * (WCAP + 1)) * (int)sizeof(double);

__global__ void identity_kernel(double* M, int k) {
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e % k;
    M[i * MAXR + j] = i == j ? 1.0 : 0.0;
  }
}

// Q <- Qtmp and P <- Ptmp (rows x keep of each, ld MAXR) when the gate is open.
__global__ void factor_commit_kernel(const double* Qtmp, double* Q, int qrows, const double* Ptmp,
                                     double* P, int prows, const double* sc, const int* gate) {
  if (gate && *gate == 0) return;
  const int keep = (int)sc[4];
  const bool grow = sc[5] != 0.0;
  const int qr = qrows + (grow ? 1 : 0);
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < (qr + prows + 1) * keep;
       e += blockDim.x * gridDim.x) {
    const int i = e / keep, j = e % keep;
    if (i < qr) Q[i * MAXR + j] = Qtmp[i * MAXR + j];
    else P[(i - qr) * MAXR + j] = Ptmp[(i - qr) * MAXR + j];
  }
}

// Outcome of one append in st[0..6]: rank, columns of U0, columns of W0, lu_ok, grew, ran,
// stop ratio (the state before the append when the gate is closed).
__global__ void append_finish_kernel(int r, int wu, int ww, const double* sc, const int* gate,
                                     double* st) {
  if (threadIdx.x != 0) return;
  const bool on = !gate || *gate != 0;
  const bool g = on && sc[5] != 0.0;
  st[0] = on ? sc[4] : r;
  st[1] = wu + (g ? 1 : 0);
  st[2] = ww + (on ? 1 : 0);
  st[3] = on ? sc[7] : -1.0;   // -1: unchanged
  st[4] = g ? 1.0 : 0.0;
  st[5] = on ? 1.0 : 0.0;
  st[6] = on ? sc[6] : 0.0;
}

int gemv_blocks(long n) {
  long b = (n + GT - 1) / GT;
  if (b > 256) b = 256;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t gemv_t(const double* U, long n, int w, const double* x, double* partial, double* out,
                   cudaStream_t s) {
  if (w <= 0) return cudaSuccess;
  const int nb = (int)((n + GV_ROWS - 1) / GV_ROWS);
  ++g_launches;
  gemv_t_partial<<<dim3(nb, (w + GV_COLS - 1) / GV_COLS), 32, 0, s>>>(U, n, w, x, partial);
  ++g_launches;
  gemv_t_finish<<<w, 32, 0, s>>>(partial, nb, w, out);
  return cudaGetLastError();
}

cudaError_t dot(const double* x, const double* y, long n, double* partial, double* out,
                cudaStream_t s) {
  const int nb = gemv_blocks(n);
  ++g_launches;
  dot_partial<<<nb, GT, 0, s>>>(x, y, n, partial);
  ++g_launches;
  gemv_t_finish<<<1, 32, 0, s>>>(partial, nb, 1, out);
  return cudaGetLastError();
}

// U^T v = Q^T (U0^T v) into out (r values)
cudaError_t proj_u(RomDev& R, const double* v, double* out, cudaStream_t s) {
  Scr sc = scr_of(R.core);
  cudaError_t e = gemv_t(R.U, R.n, R.wu, v, R.partial, sc.w0, s);
  if (e != cudaSuccess) return e;
  ++g_launches;
  small_t_kernel<<<1, 1024, 0, s>>>(R.Q, R.wu, R.rank, sc.w0, out);
  return cudaGetLastError();
}

// out = cx x - sign U0 (Q c)
cudaError_t expand_u(RomDev& R, const double* c, double cx, const double* x, double sign,
                     double* out, cudaStream_t s) {
  Scr sc = scr_of(R.core);
  ++g_launches;
  small_n_kernel<<<1, 1024, 0, s>>>(R.Q, R.wu, R.rank, c, sc.c0);
  ++g_launches;
  gemv_n<<<(unsigned)((R.n + 255) / 256), 256, 0, s>>>(R.U, R.n, R.wu, sc.c0, cx, x, sign, out);
  return cudaGetLastError();
}

// U0 <- U0 Q, Q <- I (and the same for W0, P): the factored bases multiplied out.
cudaError_t compact(RomDev& R, cudaStream_t s) {
  const unsigned rb = (unsigned)((R.n + TALL_ROWS - 1) / TALL_ROWS);
  if (R.rank > 0) {
    ++g_launches;
    tall_small_kernel<<<rb, TALL_ROWS, TALL_SMEM, s>>>(R.U, R.n, R.wu, R.Q, R.rank, R.Utmp);
    ++g_launches;
    tall_small_kernel<<<rb, TALL_ROWS, TALL_SMEM, s>>>(R.W, R.n, R.ww, R.P, R.rank, R.Wtmp);
    std::swap(R.U, R.Utmp);
    std::swap(R.W, R.Wtmp);
  }
  ++g_launches;
  identity_kernel<<<1, 256, 0, s>>>(R.Q, R.rank);
  ++g_launches;
  identity_kernel<<<1, 256, 0, s>>>(R.P, R.rank);
  R.wu = R.ww = R.rank;
  return cudaGetLastError();
}

}  // namespace

cudaError_t rom_append_async(RomDev& R, const double* x, const double* b, double trunc_eps,
                             const int* gate, cudaStream_t s) {
  const long n = R.n;
  const int r = R.rank;
  Scr sc = scr_of(R.core);
  double* q = R.U + (long)R.wu * n;   // next column of U0 holds q~, then q
  const unsigned vb = (unsigned)((n + 255) / 256);
  cudaError_t e;
  // Everything up to the commit writes scratch only (the new columns of U0 and W0 lie beyond
  // the columns in use), so a closed gate needs no test before it.
  if ((e = dot(x, x, n, R.partial, sc.sc + 0, s)) != cudaSuccess) return e;
  if (r > 0) {
    // classical Gram-Schmidt, twice: p = U^T x, q~ = x - U p; p2 = U^T q~, q~ -= U p2
    if ((e = proj_u(R, x, sc.p, s)) != cudaSuccess) return e;
    if ((e = expand_u(R, sc.p, 1.0, x, 1.0, q, s)) != cudaSuccess) return e;
    if ((e = proj_u(R, q, sc.p2, s)) != cudaSuccess) return e;
    if ((e = expand_u(R, sc.p2, 1.0, q, 1.0, q, s)) != cudaSuccess) return e;
    ++g_launches;
    add_vec_kernel<<<1, 64, 0, s>>>(sc.p, sc.p2, r);
    if ((e = proj_u(R, b, sc.ub, s)) != cudaSuccess) return e;
  } else {
    if ((e = cudaMemcpyAsync(q, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
  }
  if ((e = dot(q, q, n, R.partial, sc.sc + 1, s)) != cudaSuccess) return e;
  if ((e = core_svd_secular(R.S, r, sc.p, sc.sc, sc.Uc, sc.Vc, sc.p2, trunc_eps, R.r_max, R.sec,
                            s)) != cudaSuccess)
    return e;
  ++g_launches;
  scale_q_kernel<<<vb, 256, 0, s>>>(q, n, sc.sc);
  if (r > 0) {
    if ((e = gemv_t(R.W, n, R.ww, q, R.partial, sc.w0, s)) != cudaSuccess) return e;
    ++g_launches;
    small_t_kernel<<<1, 1024, 0, s>>>(R.P, R.ww, r, sc.w0, sc.wq);
  }
  if ((e = dot(q, b, n, R.partial, sc.sc + 2, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(R.W + (long)R.ww * n, b, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                           s)) != cudaSuccess)
    return e;
  // G, A_r and its inverse (committed only through an open gate)
  ++g_launches;
  build_gx_kernel<<<1, 256, 0, s>>>(r, sc);
  ++g_launches;
  gx_times_vc_kernel<<<r + 1, 64, 0, s>>>(r, sc);
  ++g_launches;
  uct_times_t_kernel<<<r + 1, 64, 0, s>>>(r, sc, gate);
  ++g_launches;
  inverse_kernel<<<1, 256, 0, s>>>(sc, R.S, R.lu, gate);
  // factors: Q' = [[Q,0],[0,1]] U_c or Q U_c(0:r) ; P' = [[P,0],[0,1]] V_c
  ++g_launches;
  factor_update_kernel<<<r + 1, 64, 0, s>>>(R.Q, R.wu, r, sc.Uc, sc.sc, -1, R.Qtmp);
  ++g_launches;
  factor_update_kernel<<<r + 1, 64, 0, s>>>(R.P, R.ww, r, sc.Vc, sc.sc, 1, R.Ptmp);
  ++g_launches;
  factor_commit_kernel<<<8, 256, 0, s>>>(R.Qtmp, R.Q, R.wu, R.Ptmp, R.P, R.ww, sc.sc, gate);
  ++g_launches;
  append_finish_kernel<<<1, 32, 0, s>>>(r, R.wu, R.ww, sc.sc, gate, R.dstate);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaMemcpyAsync(R.hstate, R.dstate, sizeof(double) * 8, cudaMemcpyDeviceToHost, s);
}

cudaError_t rom_commit(RomDev& R, int* ran, int* grew, double* ratio, cudaStream_t s) {
  const double* h = R.hstate;
  const bool on = h[5] != 0.0;
  if (ran) *ran = on;
  if (grew) *grew = h[4] != 0.0;
  if (ratio) *ratio = h[6];
  if (!on) return cudaSuccess;
  R.rank = (int)h[0];
  R.wu = (int)h[1];
  R.ww = (int)h[2];
  R.lu_ok = (h[3] != 0.0) ? 1 : 0;
  // Multiply the factored bases out when the stored columns run out, or once they exceed the
  // rank by COMPACT_SLACK: every projection and expansion reads all w stored columns, so a
  // basis whose rank has settled well below WCAP pays for its truncated columns on every use.
  if (R.wu >= WCAP - 1 || R.ww >= WCAP - 1 || R.wu - R.rank >= COMPACT_SLACK ||
      R.ww - R.rank >= COMPACT_SLACK)
    return compact(R, s);
  return cudaSuccess;
}

cudaError_t rom_append(RomDev& R, const double* x, const double* b, double trunc_eps, int* grew,
                       double* ratio, cudaStream_t s) {
  cudaError_t e = rom_append_async(R, x, b, trunc_eps, nullptr, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  return rom_commit(R, nullptr, grew, ratio, s);
}

cudaError_t rom_apply(RomDev& R, const double* rhs, double* out, cudaStream_t s) {
  if (R.rank <= 0 || !R.lu_ok) return cudaErrorInvalidValue;
  Scr sc = scr_of(R.core);
  cudaError_t e;
  // U0^T rhs, then Q^T, A_r^{-1} and Q in one block, then U0 c0
  if ((e = gemv_t(R.U, R.n, R.wu, rhs, R.partial, sc.w0, s)) != cudaSuccess) return e;
  ++g_launches;
  apply_core_kernel<<<1, 1024, 0, s>>>(R.Q, R.wu, R.rank, R.lu, sc.w0, R.proj, sc.c0);
  ++g_launches;
  gemv_n<<<(unsigned)((R.n + 255) / 256), 256, 0, s>>>(R.U, R.n, R.wu, sc.c0, 0.0, nullptr, -1.0,
                                                       out);
  return cudaGetLastError();
}

cudaError_t rom_get(RomDev& R, double* S, double* U, double* Ar, cudaStream_t s) {
  const int r = R.rank;
  cudaError_t e;
  if (S && r > 0 &&
      (e = cudaMemcpyAsync(S, R.S, sizeof(double) * r, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if (U && r > 0) {
    const unsigned rb = (unsigned)((R.n + TALL_ROWS - 1) / TALL_ROWS);
    ++g_launches;
    tall_small_kernel<<<rb, TALL_ROWS, TALL_SMEM, s>>>(R.U, R.n, R.wu, R.Q, r, R.Utmp);
    if ((e = cudaMemcpyAsync(U, R.Utmp, sizeof(double) * r * (size_t)R.n, cudaMemcpyDeviceToHost,
                             s)) != cudaSuccess)
      return e;
  }
  if (Ar && r > 0) {
    Scr sc = scr_of(R.core);
    double G[MAXR * MAXR], Sh[MAXR];
    if ((e = cudaMemcpyAsync(G, sc.G, sizeof(G), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(Sh, R.S, sizeof(double) * r, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < r; ++j) Ar[i * r + j] = G[i * MAXR + j] / Sh[j];
  }
  return cudaStreamSynchronize(s);
}

cudaError_t rom_alloc(RomDev& R, int n, int r_max) {
  R = RomDev{};
  R.n = n;
  R.r_max = r_max;
  const size_t col = sizeof(double) * (size_t)n * WCAP;
  const size_t small = sizeof(double) * WCAP * MAXR;
  cudaError_t e;
  if ((e = cudaMalloc(&R.U, col)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.W, col)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.Utmp, col)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.Wtmp, col)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.Q, small)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.P, small)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.Qtmp, small)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.Ptmp, small)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.S, sizeof(double) * MAXR)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.core, sizeof(double) * SCR_DOUBLES)) != cudaSuccess) return e;
  if ((e = cudaMemset(R.core, 0, sizeof(double) * SCR_DOUBLES)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.lu, sizeof(double) * MAXR * MAXR)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.piv, sizeof(int) * MAXR)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.proj, sizeof(double) * 2 * MAXR)) != cudaSuccess) return e;
  const long nbp = ((long)n + GV_ROWS - 1) / GV_ROWS;
  if ((e = cudaMalloc(&R.partial, sizeof(double) * WCAP * (nbp > 256 ? nbp : 256))) != cudaSuccess)
    return e;
  if ((e = cudaMalloc(&R.sec, sizeof(double) * secular_scratch_doubles())) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.dstate, sizeof(double) * 8)) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&R.hstate, sizeof(double) * 8)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(tall_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TALL_SMEM)) != cudaSuccess)
    return e;
  return cudaSuccess;
}

void rom_reset(RomDev& R) {
  R.rank = 0;
  R.wu = R.ww = 0;
  R.lu_ok = 0;
}

void rom_free(RomDev& R) {
  double* d[] = {R.U, R.W, R.Utmp, R.Wtmp, R.Q, R.P, R.Qtmp, R.Ptmp, R.S, R.core, R.lu,
                 R.proj, R.partial, R.sec, R.dstate};
  for (double* p : d)
    if (p) cudaFree(p);
  if (R.hstate) cudaFreeHost(R.hstate);
  if (R.piv) cudaFree(R.piv);
  R = RomDev{};
}

// Checkpoint of one ROM: its host counters (rank, stored columns of U0 and W0, lu_ok), then
// every device array that carries state from one append or apply to the next: the stored
// columns of U0 and W0, the small factors Q and P, the singular values, A_r^{-1} and the core
// workspace (which keeps U^T W for the next append).
namespace {
constexpr size_t ROM_SMALL_DOUBLES = 2 * (size_t)WCAP * MAXR + MAXR + (size_t)MAXR * MAXR + SCR_DOUBLES;
}

size_t rom_state_bytes(const RomDev& R) {
  return 4 * sizeof(int) + sizeof(double) * ((size_t)(R.wu + R.ww) * R.n + ROM_SMALL_DOUBLES);
}

cudaError_t rom_save(const RomDev& R, unsigned char* out, cudaStream_t s) {
  const int head[4] = {R.rank, R.wu, R.ww, R.lu_ok};
  std::memcpy(out, head, sizeof(head));
  out += sizeof(head);
  const std::pair<const double*, size_t> parts[] = {
      {R.U, (size_t)R.wu * R.n}, {R.W, (size_t)R.ww * R.n}, {R.Q, (size_t)WCAP * MAXR},
      {R.P, (size_t)WCAP * MAXR}, {R.S, (size_t)MAXR},      {R.lu, (size_t)MAXR * MAXR},
      {R.core, (size_t)SCR_DOUBLES}};
  for (const auto& pt : parts) {
    const size_t b = sizeof(double) * pt.second;
    cudaError_t e = cudaMemcpyAsync(out, pt.first, b, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    out += b;
  }
  return cudaStreamSynchronize(s);
}

size_t rom_checked_bytes(const RomDev& R, const unsigned char* in, size_t avail) {
  int head[4];
  if (avail < sizeof(head)) return 0;
  std::memcpy(head, in, sizeof(head));
  const int rank = head[0], wu = head[1], ww = head[2];
  if (rank < 0 || rank > R.r_max || wu < rank || ww < rank || wu > WCAP - 1 || ww > WCAP - 1)
    return 0;
  const size_t need =
      4 * sizeof(int) + sizeof(double) * ((size_t)(wu + ww) * R.n + ROM_SMALL_DOUBLES);
  return need <= avail ? need : 0;
}

cudaError_t rom_load(RomDev& R, const unsigned char* in, cudaStream_t s) {
  int head[4];
  std::memcpy(head, in, sizeof(head));
  in += sizeof(head);
  const int wu = head[1], ww = head[2];
  const std::pair<double*, size_t> parts[] = {
      {R.U, (size_t)wu * R.n}, {R.W, (size_t)ww * R.n}, {R.Q, (size_t)WCAP * MAXR},
      {R.P, (size_t)WCAP * MAXR}, {R.S, (size_t)MAXR},   {R.lu, (size_t)MAXR * MAXR},
      {R.core, (size_t)SCR_DOUBLES}};
  for (const auto& pt : parts) {
    const size_t b = sizeof(double) * pt.second;
    cudaError_t e = cudaMemcpyAsync(pt.first, in, b, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    in += b;
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  R.rank = head[0];
  R.wu = wu;
  R.ww = ww;
  R.lu_ok = head[3] != 0 ? 1 : 0;
  return cudaSuccess;
}

}  // namespace rte
