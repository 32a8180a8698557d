// On-the-fly reduced-order models (Sec. 3.1, 3.2, App. B), FP64.
//
// A ROM keeps the thin SVD R ~ U S V^T of its solution snapshots and W = B V (B the
// right-hand-side snapshots), so that the DMD operator of Eq. (dmd-operator) is
// A_r = U^T W S^{-1}; V itself is never stored.  G = U^T W (r x r) is kept and updated
// with the same small rotations as U and W, so A_r costs O(r^2) per update instead of a
// reduction over the N_x rows.
//
// Append (App. B, Eq. (svd_core)), one snapshot pair (x, b):
//   p = U^T x;  q~ = x - U p;  repeated once (classical Gram-Schmidt twice);
//   alpha = ||q~||; the rank grows iff alpha > 1e-12 ||x|| (else q is dropped);
//   K = [[S, p], [0, alpha]] = U_c S_c V_c^T  (secular equation of the broken-arrow form,
//   FP64, csvd.cu);
//   keep = r+1 (or r), truncated to s_k / sum s > eps when asked, capped at r_max;
//   U <- [U q] U_c(:, :keep);  W <- [W b] V_c(:, :keep);
//   G <- U_c^T [[G, U^T b], [q^T W, q^T b]] V_c;  A_r = G S^{-1}, LU with partial pivoting.
// Apply (Eq. (dmd-ig), Eq. (dmd-sa)): out = U A_r^{-1} U^T rhs.
#include <cuda_runtime.h>

#include <cmath>

#include "rte_internal.h"

namespace rte {

namespace {
constexpr unsigned FULL = 0xffffffffu;
constexpr int GT = 256;          // rows per GEMV block
constexpr int MAXR = 65;         // r_max + 1 <= 65
constexpr int ROT_ROWS = 64;     // rows per rotation block

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// partial[k * nb + blockIdx.x] = sum over this block's rows of U[:,k] . x   (grid: nb x r)
__global__ void gemv_t_partial(const double* __restrict__ U, long n, const double* __restrict__ x,
                               double* __restrict__ partial) {
  __shared__ double sh[GT / 32];
  const int k = blockIdx.y;
  const double* u = U + (long)k * n;
  double s = 0.0;
  for (long i = (long)blockIdx.x * GT + threadIdx.x; i < n; i += (long)gridDim.x * GT)
    s += u[i] * x[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < GT / 32 ? sh[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) partial[(long)k * gridDim.x + blockIdx.x] = s;
  }
}

// out[k] = (accumulate ? out[k] : 0) + sum_b partial[k * nb + b], fixed order.
__global__ void gemv_t_finish(const double* partial, int nb, int r, double* out, int accumulate) {
  const int k = blockIdx.x;
  if (k >= r) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) s += partial[(long)k * nb + b];
  s = warp_sum(s);
  if (threadIdx.x == 0) out[k] = (accumulate ? out[k] : 0.0) + s;
}

// out[i] = cx * x[i] - sign * sum_k U[k n + i] c[k]   (sign = +1: x - U c; sign = -1: U c)
__global__ void gemv_n(const double* __restrict__ U, long n, int r, const double* __restrict__ c,
                       double cx, const double* __restrict__ x, double sign, double* __restrict__ out) {
  __shared__ double cs[MAXR];
  if (threadIdx.x < r) cs[threadIdx.x] = c[threadIdx.x];
  __syncthreads();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int k = 0; k < r; ++k) s += U[(long)k * n + i] * cs[k];
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

// Scratch layout of one ROM (device doubles).
struct Scr {
  double* p;      // [MAXR]  U^T x (after CGS2)
  double* p2;     // [MAXR]
  double* ub;     // [MAXR]  U^T b
  double* wq;     // [MAXR]  W^T q
  double* sc;     // [16]    0: ||x||^2  1: alpha^2  2: q.b  3: 1/alpha (0 if no growth)
                  //         4: keep  5: grew  6: stop ratio  7: lu_ok
  double* Uc;     // [MAXR*MAXR] column-major, sorted
  double* Vc;     // [MAXR*MAXR]
  double* G;      // [MAXR*MAXR] row-major U^T W (rank x rank)
  double* Gx;     // [MAXR*MAXR]
};

Scr scr_of(double* core) {
  Scr s;
  s.p = core;
  s.p2 = s.p + MAXR;
  s.ub = s.p2 + MAXR;
  s.wq = s.ub + MAXR;
  s.sc = s.wq + MAXR;
  s.Uc = s.sc + 16;
  s.Vc = s.Uc + MAXR * MAXR;
  s.G = s.Vc + MAXR * MAXR;
  s.Gx = s.G + MAXR * MAXR;
  return s;
}
constexpr long SCR_DOUBLES = 4 * MAXR + 16 + 4 * MAXR * MAXR;

// scaled copy q = q~ * (1/alpha) (0 when the rank does not grow)
__global__ void scale_q_kernel(double* q, long n, const double* sc) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] *= sc[3];
}

// G <- U_c^T [[G, U^T b], [q^T W, q^T b]] V_c ; S <- new singular values ; A_r = G S^{-1} ;
// LU factorisation with partial pivoting of A_r (row-major) into lu / piv.
__global__ void __launch_bounds__(256) g_update_lu_kernel(int r, Scr sc, double* S, double* lu,
                                                         int* piv) {
  extern __shared__ double gsm[];
  double* Gx = gsm;
  double* T = Gx + MAXR * MAXR;
  double* A = T + MAXR * MAXR;
  __shared__ int s_ok;
  const int n = r + 1;
  const int keep = (int)sc.sc[4];
  const int tid = threadIdx.x;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    double v;
    if (i < r && j < r) v = sc.G[i * MAXR + j];
    else if (i < r) v = sc.ub[i];
    else if (j < r) v = sc.wq[j];
    else v = sc.sc[2];
    Gx[i * n + j] = v;
  }
  __syncthreads();
  // T = Gx V_c  (n x keep)
  for (int e = tid; e < n * keep; e += blockDim.x) {
    const int i = e / keep, b = e % keep;
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += Gx[i * n + j] * sc.Vc[b * n + j];
    T[i * keep + b] = s;
  }
  __syncthreads();
  // G = U_c^T T (keep x keep), A_r = G / S_new (column scaling)
  for (int e = tid; e < keep * keep; e += blockDim.x) {
    const int a = e / keep, b = e % keep;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += sc.Uc[a * n + i] * T[i * keep + b];
    sc.G[a * MAXR + b] = s;
    A[a * keep + b] = s / sc.p2[b];
  }
  __syncthreads();
  for (int a = tid; a < keep; a += blockDim.x) S[a] = sc.p2[a];
  // LU with partial pivoting (single thread does the pivot search; rows updated in parallel)
  double amax = 0.0;
  for (int e = 0; e < keep * keep; ++e) amax = fmax(amax, fabs(A[e]));
  if (tid == 0) s_ok = keep > 0 ? 1 : 0;
  __syncthreads();
  for (int k = 0; k < keep; ++k) {
    if (tid == 0) {
      int p = k;
      double best = fabs(A[k * keep + k]);
      for (int i = k + 1; i < keep; ++i)
        if (fabs(A[i * keep + k]) > best) {
          best = fabs(A[i * keep + k]);
          p = i;
        }
      piv[k] = p;
      if (!(best > 1e-14 * amax)) s_ok = 0;
      if (p != k)
        for (int j = 0; j < keep; ++j) {
          const double t = A[k * keep + j];
          A[k * keep + j] = A[p * keep + j];
          A[p * keep + j] = t;
        }
    }
    __syncthreads();
    const double d = A[k * keep + k];
    for (int e = tid; e < (keep - k - 1) * (keep - k); e += blockDim.x) {
      const int i = k + 1 + e / (keep - k);
      const int j = k + e % (keep - k);
      if (j == k) continue;
      A[i * keep + j] -= (A[i * keep + k] / d) * A[k * keep + j];
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < keep; i += blockDim.x) A[i * keep + k] /= d;
    __syncthreads();
  }
  for (int e = tid; e < keep * keep; e += blockDim.x) lu[e] = A[e];
  if (tid == 0) sc.sc[7] = s_ok;
}

// out_col[j] = sum_{k < kin} in_k[i] M[k][j] for j < keep, with in_k = base column k for
// k < r and in_r = extra (the new column); M column-major with leading dimension n = r+1.
__global__ void __launch_bounds__(ROT_ROWS) rotate_kernel(const double* __restrict__ base,
                                                          const double* __restrict__ extra, long n,
                                                          int r, const double* __restrict__ Mc,
                                                          const double* sc,
                                                          double* __restrict__ out) {
  extern __shared__ double rsm[];
  double* Ms = rsm;
  double* tile = Ms + MAXR * MAXR;
  const int kin = r + 1;
  const int keep = (int)sc[4];
  const int ld = kin + 1;
  for (int e = threadIdx.x; e < kin * keep; e += ROT_ROWS) Ms[e] = Mc[e];
  const long i0 = (long)blockIdx.x * ROT_ROWS;
  for (int k = 0; k < kin; ++k) {
    const long i = i0 + threadIdx.x;
    double v = 0.0;
    if (i < n) v = (k < r) ? base[(long)k * n + i] : (extra ? extra[i] : 0.0);
    tile[threadIdx.x * ld + k] = v;
  }
  __syncthreads();
  const long i = i0 + threadIdx.x;
  if (i >= n) return;
  const double* row = tile + threadIdx.x * ld;
  for (int j = 0; j < keep; ++j) {
    double s = 0.0;
    for (int k = 0; k < kin; ++k) s += row[k] * Ms[j * kin + k];
    out[(long)j * n + i] = s;
  }
}

// c = A_r^{-1} proj by the stored LU (one thread; r <= 64).
__global__ void lu_solve_kernel(const double* lu, const int* piv, int r, double* x) {
  if (threadIdx.x != 0) return;
  for (int k = 0; k < r; ++k) {
    const int p = piv[k];
    if (p != k) {
      const double t = x[k];
      x[k] = x[p];
      x[p] = t;
    }
  }
  for (int i = 0; i < r; ++i) {
    double s = x[i];
    for (int j = 0; j < i; ++j) s -= lu[i * r + j] * x[j];
    x[i] = s;
  }
  for (int i = r - 1; i >= 0; --i) {
    double s = x[i];
    for (int j = i + 1; j < r; ++j) s -= lu[i * r + j] * x[j];
    x[i] = s / lu[i * r + i];
  }
}

int gemv_blocks(long n) {
  long b = (n + GT - 1) / GT;
  if (b > 256) b = 256;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t gemv_t(const double* U, long n, int r, const double* x, double* partial, double* out,
                   int accumulate, cudaStream_t s) {
  if (r <= 0) return cudaSuccess;
  const int nb = gemv_blocks(n);
  ++g_launches;
  gemv_t_partial<<<dim3(nb, r), GT, 0, s>>>(U, n, x, partial);
  ++g_launches;
  gemv_t_finish<<<r, 32, 0, s>>>(partial, nb, r, out, accumulate);
  return cudaGetLastError();
}

cudaError_t dot(const double* x, const double* y, long n, double* partial, double* out,
                cudaStream_t s) {
  const int nb = gemv_blocks(n);
  ++g_launches;
  dot_partial<<<nb, GT, 0, s>>>(x, y, n, partial);
  ++g_launches;
  gemv_t_finish<<<1, 32, 0, s>>>(partial, nb, 1, out, 0);
  return cudaGetLastError();
}

}  // namespace

__global__ void add_vec_kernel(double* a, const double* b, int r) {
  if ((int)threadIdx.x < r) a[threadIdx.x] += b[threadIdx.x];
}

constexpr int GLU_SMEM = 3 * MAXR * MAXR * (int)sizeof(double);
constexpr int ROT_SMEM = (MAXR * MAXR + ROT_ROWS * (MAXR + 1)) * (int)sizeof(double);

cudaError_t rom_append(RomDev& R, const double* x, const double* b, double trunc_eps, int* grew,
                       double* ratio, cudaStream_t s) {
  const long n = R.n;
  const int r = R.rank;
  Scr sc = scr_of(R.core);
  double* q = R.U + (long)r * n;   // spare column r of U holds q~ then q
  const unsigned vb = (unsigned)((n + 255) / 256);
  cudaError_t e;
  if ((e = dot(x, x, n, R.partial, sc.sc + 0, s)) != cudaSuccess) return e;
  if (r > 0) {
    // classical Gram-Schmidt, twice
    if ((e = gemv_t(R.U, n, r, x, R.partial, sc.p, 0, s)) != cudaSuccess) return e;
    ++g_launches;
    gemv_n<<<vb, 256, 0, s>>>(R.U, n, r, sc.p, 1.0, x, 1.0, q);
    if ((e = gemv_t(R.U, n, r, q, R.partial, sc.p2, 0, s)) != cudaSuccess) return e;
    ++g_launches;
    gemv_n<<<vb, 256, 0, s>>>(R.U, n, r, sc.p2, 1.0, q, 1.0, q);
    ++g_launches;
    add_vec_kernel<<<1, 64, 0, s>>>(sc.p, sc.p2, r);
    if ((e = gemv_t(R.U, n, r, b, R.partial, sc.ub, 0, s)) != cudaSuccess) return e;
  } else {
    if ((e = cudaMemcpyAsync(q, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
  }
  if ((e = dot(q, q, n, R.partial, sc.sc + 1, s)) != cudaSuccess) return e;
  ++g_launches;
  if ((e = core_svd_secular(R.S, r, sc.p, sc.sc, sc.Uc, sc.Vc, sc.p2, trunc_eps, R.r_max, R.sec,
                            s)) != cudaSuccess)
    return e;
  ++g_launches;
  scale_q_kernel<<<vb, 256, 0, s>>>(q, n, sc.sc);
  if (r > 0 && (e = gemv_t(R.W, n, r, q, R.partial, sc.wq, 0, s)) != cudaSuccess) return e;
  if ((e = dot(q, b, n, R.partial, sc.sc + 2, s)) != cudaSuccess) return e;
  ++g_launches;
  g_update_lu_kernel<<<1, 256, GLU_SMEM, s>>>(r, sc, R.S, R.lu, R.piv);
  const unsigned rb = (unsigned)((n + ROT_ROWS - 1) / ROT_ROWS);
  ++g_launches;
  rotate_kernel<<<rb, ROT_ROWS, ROT_SMEM, s>>>(R.U, q, n, r, sc.Uc, sc.sc, R.Utmp);
  ++g_launches;
  rotate_kernel<<<rb, ROT_ROWS, ROT_SMEM, s>>>(R.W, b, n, r, sc.Vc, sc.sc, R.Wtmp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  double h[8];
  if ((e = cudaMemcpyAsync(h, sc.sc, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  double* t = R.U;
  R.U = R.Utmp;
  R.Utmp = t;
  t = R.W;
  R.W = R.Wtmp;
  R.Wtmp = t;
  R.rank = (int)h[4];
  R.lu_ok = (h[7] != 0.0) ? 1 : 0;
  if (grew) *grew = h[5] != 0.0;
  if (ratio) *ratio = h[6];
  return cudaSuccess;
}

cudaError_t rom_apply(RomDev& R, const double* rhs, double* out, cudaStream_t s) {
  if (R.rank <= 0 || !R.lu_ok) return cudaErrorInvalidValue;
  const long n = R.n;
  cudaError_t e;
  if ((e = gemv_t(R.U, n, R.rank, rhs, R.partial, R.proj, 0, s)) != cudaSuccess) return e;
  ++g_launches;
  lu_solve_kernel<<<1, 32, 0, s>>>(R.lu, R.piv, R.rank, R.proj);
  ++g_launches;
  gemv_n<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(R.U, n, R.rank, R.proj, 0.0, nullptr, -1.0, out);
  return cudaGetLastError();
}

cudaError_t rom_get(RomDev& R, double* S, double* U, double* Ar, cudaStream_t s) {
  const int r = R.rank;
  cudaError_t e;
  if (S && r > 0 &&
      (e = cudaMemcpyAsync(S, R.S, sizeof(double) * r, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if (U && r > 0 &&
      (e = cudaMemcpyAsync(U, R.U, sizeof(double) * r * (size_t)R.n, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess)
    return e;
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
  const size_t col = sizeof(double) * (size_t)n * (r_max + 1);
  cudaError_t e;
  if ((e = cudaMalloc(&R.U, col)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.W, col)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.Utmp, col)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.Wtmp, col)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.S, sizeof(double) * MAXR)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.core, sizeof(double) * SCR_DOUBLES)) != cudaSuccess) return e;
  if ((e = cudaMemset(R.core, 0, sizeof(double) * SCR_DOUBLES)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.lu, sizeof(double) * MAXR * MAXR)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.piv, sizeof(int) * MAXR)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.proj, sizeof(double) * MAXR)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.partial, sizeof(double) * MAXR * 256)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&R.sec, sizeof(double) * secular_scratch_doubles())) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(g_update_lu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                GLU_SMEM)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(rotate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                ROT_SMEM)) != cudaSuccess)
    return e;
  return cudaSuccess;
}

void rom_free(RomDev& R) {
  double* d[] = {R.U, R.W, R.Utmp, R.Wtmp, R.S, R.core, R.lu, R.proj, R.partial, R.sec};
  for (double* p : d)
    if (p) cudaFree(p);
  if (R.piv) cudaFree(R.piv);
  R = RomDev{};
}

}  // namespace rte
