// SVD of the incremental-SVD core matrix (App. B, Eq. (svd_core)),
//   K = [[diag(S), p], [0, alpha]]   ((r+1) x (r+1), S_1 >= ... >= S_r > 0),
// in FP64 by the secular equation of a broken-arrow matrix instead of a dense SVD.
//
// Moving the last row/column of K^T to the front and sorting S ascending gives
//   M = [[z_1, z_2, ..., z_n], [0, diag(d_2, ..., d_n)]],  d_1 = 0 < d_2 < ... < d_n,
// z = (alpha, p in the same order), n = r + 1, and K = P^T M^T P, so the left singular
// vectors of K are the (permuted) right singular vectors of M and vice versa.
// M^T M = diag(d^2) + z z^T, so the singular values solve
//   f(sigma^2) = 1 + sum_j z_j^2 / (d_j^2 - sigma^2) = 0,   d_k < sigma_k < d_{k+1},
// and the singular vectors are v_k ~ (z_j / (d_j^2 - sigma_k^2))_j,
// u_k ~ (-1, d_j z_j / (d_j^2 - sigma_k^2))_j.
// Each root is bracketed, written as sigma_k^2 = d_s^2 + mu (s the nearer pole, so that
// d_j^2 - sigma_k^2 = (d_j - d_s)(d_j + d_s) - mu is formed without cancellation), located
// by bisection on the ordered bit pattern of mu (which reaches any scale quickly) and
// finished by rational steps (pole term exact, the other terms linearised, as in the
// classical secular-equation solvers) kept inside the bisection bracket.
// For orthogonal vectors z is replaced by the z^ for which the computed roots are exact
// (Gu and Eisenstat's formula, the Loewner theorem):
//   z^_j^2 = (s_n^2 - d_j^2) prod_{i<j} (s_i^2 - d_j^2)/(d_i^2 - d_j^2)
//                            prod_{j<=i<n} (s_i^2 - d_j^2)/(d_{i+1}^2 - d_j^2).
// Deflation: |z_j| <= tol gives sigma = d_j with unit vectors; d_{j+1} - d_j <= tol is
// removed by a Givens rotation that zeroes z_j; a tiny z_1 (no rank growth) is raised to
// tol, which leaves a singular value of order tol that the caller drops.
//
// One warp per root, vector, and z^ entry, spread over many CTAs: the FP64 work is
// O(n^2) per core instead of the O(n^3) per sweep of a one-sided Jacobi on one SM.
#include <cuda_runtime.h>

#include <cmath>

#include "rte_internal.h"

namespace rte {

namespace {
constexpr unsigned FULL = 0xffffffffu;
constexpr int MAXN = 65;

// Secular scratch layout (doubles).
struct Sec {
  double* d;      // [MAXN] sorted d (M order)
  double* z;      // [MAXN]
  double* zh;     // [MAXN] z^
  double* mu;     // [MAXN] root offsets (active index order)
  double* sidx;   // [MAXN] pole index of each root (as double)
  double* sig;    // [MAXN] singular values, M column order
  double* info;   // [8]: 0 n, 1 n_active, 2 n_rot, 3 tol, 4 znorm
  double* act;    // [MAXN] active M-indices (ascending)
  double* defl;   // [MAXN] deflated M-indices
  double* rot;    // [3*MAXN] (j, c, s) Givens rotations in application order
  double* kidx;   // [MAXN] K-index of each M-index
  double* UM;     // [MAXN*MAXN] column-major, column = singular triple
  double* VM;     // [MAXN*MAXN]
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
__device__ __forceinline__ double warp_prod(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(FULL, v, o);
  return v;
}

// Build d, z, deflation and rotations (one thread; n <= 65).
__global__ void sec_setup_kernel(const double* S, int r, const double* p, const double* sc,
                                 Sec q) {
  if (threadIdx.x != 0) return;
  const int n = r + 1;
  const double xn = sqrt(sc[0]);
  const double alpha = sqrt(fmax(sc[1], 0.0));
  const bool grew = alpha > 1e-12 * xn;
  // M-index 0 <-> K-index r (the new column); M-index m >= 1 <-> K-index r - m.
  q.d[0] = 0.0;
  q.z[0] = grew ? alpha : 0.0;
  q.kidx[0] = r;
  for (int m = 1; m < n; ++m) {
    q.d[m] = S[r - m];
    q.z[m] = p[r - m];
    q.kidx[m] = r - m;
  }
  double zn = 0.0;
  for (int m = 0; m < n; ++m) zn += q.z[m] * q.z[m];
  zn = sqrt(zn);
  const double tol = 8.0 * 2.220446049250313e-16 * fmax(q.d[n - 1], zn);
  if (fabs(q.z[0]) < tol) q.z[0] = tol;
  int nrot = 0;
  // nearly equal d: rotate (z_j, z_{j+1}) -> (0, rho) and deflate j
  for (int j = 0; j + 1 < n; ++j) {
    if (q.d[j + 1] - q.d[j] <= tol && q.z[j] != 0.0) {
      const double a = q.z[j], b = q.z[j + 1];
      const double rho = hypot(a, b);
      const double c = b / rho, s = a / rho;
      q.z[j] = 0.0;
      q.z[j + 1] = rho;
      q.d[j] = q.d[j + 1];
      q.rot[3 * nrot + 0] = j;
      q.rot[3 * nrot + 1] = c;
      q.rot[3 * nrot + 2] = s;
      ++nrot;
    }
  }
  int na = 0, nd = 0;
  for (int m = 0; m < n; ++m) {
    if (m == 0 || fabs(q.z[m]) > tol)
      q.act[na++] = m;
    else
      q.defl[nd++] = m;
  }
  q.info[0] = n;
  q.info[1] = na;
  q.info[2] = nrot;
  q.info[3] = tol;
  q.info[4] = zn;
}

// g(mu) = 1 + sum_j z_j^2 / (delta_j - mu) over the active set, delta_j = (d_j - d_s)(d_j + d_s).
__device__ double sec_g(const Sec& q, int na, double ds, double mu, int lane) {
  double acc = 0.0;
  for (int a = lane; a < na; a += 32) {
    const int j = (int)q.act[a];
    const double dj = q.d[j];
    const double zj = q.z[j];
    acc += zj * zj / ((dj - ds) * (dj + ds) - mu);
  }
  return 1.0 + warp_sum(acc);
}

// Root k (active order) per CTA of one warp.
__global__ void __launch_bounds__(32) sec_root_kernel(Sec q) {
  const int k = blockIdx.x, lane = threadIdx.x;
  const int na = (int)q.info[1];
  if (k >= na) return;
  const double zn = q.info[4];
  const double dk = q.d[(int)q.act[k]];
  int s;
  double lo, hi;
  bool neg = false;
  if (k < na - 1) {
    const double dk1 = q.d[(int)q.act[k + 1]];
    const double mid = 0.5 * (dk1 - dk) * (dk1 + dk);
    const double fmid = sec_g(q, na, dk, mid, lane);
    if (fmid > 0.0) {
      s = k;
      lo = 0.0;
      hi = mid;
    } else {
      s = k + 1;
      lo = 0.0;
      hi = mid;
      neg = true;    // mu = -t, t in (0, mid]
    }
  } else {
    s = k;
    lo = 0.0;
    hi = zn * zn;
  }
  const double ds = q.d[(int)q.act[s]];
  // h(t) = +-g(+-t) is increasing on (0, hi] with h(0+) = -inf and h(hi) >= 0.  A few steps
  // of bisection on the bit pattern of t (which halves the exponent range first, so any scale
  // is bracketed quickly) are followed by Newton steps on h kept inside the bracket [a, b];
  // a Newton step that leaves the bracket or stalls is replaced by a bit-pattern bisection.
  long long a = __double_as_longlong(lo), b = __double_as_longlong(hi);
  for (int it = 0; it < 4 && b - a > 1; ++it) {
    const long long m = a + (b - a) / 2;
    const double t = __longlong_as_double(m);
    const double g = sec_g(q, na, ds, neg ? -t : t, lane);
    if ((neg ? -g : g) > 0.0) b = m; else a = m;
  }
  // Rational steps: with the pole term z_s^2 / (0 - mu) kept exact and the rest
  // R(mu) = sum_{j != s} z_j^2 / (delta_j - mu) linearised at the current mu, g = 0 becomes
  // R1 x^2 + (1 + R0 - R1 mu) x - z_s^2 = 0 for the new mu = x (one root of each sign).
  const int ps = (int)q.act[s];
  const double A2 = q.z[ps] * q.z[ps];
  double t = __longlong_as_double(a + (b - a) / 2);
  for (int it = 0; it < 60 && b - a > 1; ++it) {
    const double mu = neg ? -t : t;
    double r0 = 0.0, r1 = 0.0;
    for (int e = lane; e < na; e += 32) {
      const int j = (int)q.act[e];
      if (j == ps) continue;
      const double dj = q.d[j], zj = q.z[j];
      const double w = zj / ((dj - ds) * (dj + ds) - mu);
      r0 += zj * w;
      r1 += w * w;
    }
    r0 = warp_sum(r0);
    r1 = warp_sum(r1);
    const double g = 1.0 + r0 - A2 / mu;
    const double h = neg ? -g : g;
    const long long tbits = __double_as_longlong(t);
    if (h > 0.0) b = tbits; else a = tbits;
    if (b - a <= 1) break;
    const double bq = 1.0 + r0 - r1 * mu;
    double x;
    if (r1 > 0.0) {
      const double sq = sqrt(bq * bq + 4.0 * r1 * A2);
      if (!neg) x = bq >= 0.0 ? 2.0 * A2 / (bq + sq) : (sq - bq) / (2.0 * r1);
      else x = bq <= 0.0 ? 2.0 * A2 / (bq - sq) : (-bq - sq) / (2.0 * r1);
    } else {
      x = A2 / bq;
    }
    double tn = neg ? -x : x;
    if (tn > 0.0 && fabs(tn - t) <= 4.440892098500626e-16 * fabs(t)) {
      t = tn;   // converged to the resolution of t
      break;
    }
    const long long nbits = __double_as_longlong(tn);
    if (!(tn > 0.0) || nbits <= a || nbits >= b) tn = __longlong_as_double(a + (b - a) / 2);
    t = tn;
  }
  {
    const double ta = __longlong_as_double(a), tbv = __longlong_as_double(b);
    const double ga = a > 0 ? sec_g(q, na, ds, neg ? -ta : ta, lane) : -1e300;
    const double gb = sec_g(q, na, ds, neg ? -tbv : tbv, lane);
    const double gt = sec_g(q, na, ds, neg ? -t : t, lane);
    // the best of the bracket ends and the last iterate
    double best = tbv, bv = fabs(gb);
    if (a > 0 && fabs(ga) < bv) {
      best = ta;
      bv = fabs(ga);
    }
    if (t > 0.0 && fabs(gt) < bv) best = t;
    t = best;
  }
  if (lane == 0) {
    q.mu[k] = neg ? -t : t;
    q.sidx[k] = s;
  }
}

// s_i^2 - d_j^2 for root i (active order) and M-index j.
__device__ __forceinline__ double sdiff(const Sec& q, int i, double dj) {
  const double ds = q.d[(int)q.act[(int)q.sidx[i]]];
  return (ds - dj) * (ds + dj) + q.mu[i];
}

// z^_j for active entry a (one warp per entry).
__global__ void __launch_bounds__(32) sec_zhat_kernel(Sec q) {
  const int a = blockIdx.x, lane = threadIdx.x;
  const int na = (int)q.info[1];
  if (a >= na) return;
  const double dj = q.d[(int)q.act[a]];
  double prod = 1.0;
  for (int i = lane; i < na - 1; i += 32) {
    // factor i < a: (s_i^2 - d_j^2)/(d_i^2 - d_j^2); i >= a: (s_i^2 - d_j^2)/(d_{i+1}^2 - d_j^2)
    const double di = q.d[(int)q.act[i < a ? i : i + 1]];
    prod *= sdiff(q, i, dj) / ((di - dj) * (di + dj));
  }
  prod = warp_prod(prod);
  if (lane == 0) {
    const double full = prod * sdiff(q, na - 1, dj);
    const double zj = q.z[(int)q.act[a]];
    const double m = sqrt(fabs(full));
    q.zh[a] = zj >= 0.0 ? m : -m;
  }
}

// Singular triple i (M column i): roots first, deflated ones after.
__global__ void __launch_bounds__(32) sec_vec_kernel(Sec q) {
  const int i = blockIdx.x, lane = threadIdx.x;
  const int n = (int)q.info[0], na = (int)q.info[1];
  if (i >= n) return;
  double* u = q.UM + (size_t)i * MAXN;
  double* v = q.VM + (size_t)i * MAXN;
  for (int j = lane; j < n; j += 32) {
    u[j] = 0.0;
    v[j] = 0.0;
  }
  __syncwarp();
  if (i >= na) {
    const int m = (int)q.defl[i - na];
    if (lane == 0) {
      u[m] = 1.0;
      v[m] = 1.0;
      q.sig[i] = q.d[m];
    }
    return;
  }
  double su = 0.0, sv = 0.0;
  for (int a = lane; a < na; a += 32) {
    const int j = (int)q.act[a];
    const double dj = q.d[j];
    const double den = -sdiff(q, i, dj);          // d_j^2 - s_i^2
    const double vj = q.zh[a] / den;
    const double uj = (j == 0) ? -1.0 : dj * q.zh[a] / den;
    v[j] = vj;
    u[j] = uj;
    su += uj * uj;
    sv += vj * vj;
  }
  su = warp_sum(su);
  sv = warp_sum(sv);
  __syncwarp();
  const double iu = 1.0 / sqrt(su), iv = 1.0 / sqrt(sv);
  for (int a = lane; a < na; a += 32) {
    const int j = (int)q.act[a];
    u[j] *= iu;
    v[j] *= iv;
  }
  if (lane == 0) {
    const double ds = q.d[(int)q.act[(int)q.sidx[i]]];
    q.sig[i] = sqrt(ds * ds + q.mu[i]);
  }
}

// Undo the deflation rotations, map to K order, sort descending, decide rank growth and
// truncation, and write U_c, V_c (first `keep` columns) and the new singular values.
__global__ void __launch_bounds__(256) sec_finish_kernel(int r, Sec q, double* sc, double* Uc,
                                                         double* Vc, double* snew,
                                                         double trunc_eps, int r_max) {
  __shared__ int ord[MAXN];
  const int n = r + 1, tid = threadIdx.x;
  const int nrot = (int)q.info[2];
  // rotations act on M rows (j, j+1) of every column: x_j = c x'_j + s x'_{j+1},
  // x_{j+1} = -s x'_j + c x'_{j+1}; applied last-recorded first.
  for (int col = tid; col < n; col += blockDim.x) {
    double* u = q.UM + (size_t)col * MAXN;
    double* v = q.VM + (size_t)col * MAXN;
    for (int t = nrot - 1; t >= 0; --t) {
      const int j = (int)q.rot[3 * t];
      const double c = q.rot[3 * t + 1], s = q.rot[3 * t + 2];
      const double u0 = u[j], u1 = u[j + 1], v0 = v[j], v1 = v[j + 1];
      u[j] = c * u0 + s * u1;
      u[j + 1] = -s * u0 + c * u1;
      v[j] = c * v0 + s * v1;
      v[j + 1] = -s * v0 + c * v1;
    }
  }
  __syncthreads();
  const double xn = sqrt(sc[0]);
  const double alpha = sqrt(fmax(sc[1], 0.0));
  const bool grew = alpha > 1e-12 * xn;
  if (tid == 0) {
    for (int j = 0; j < n; ++j) ord[j] = j;
    // selection sort, descending, on the bit patterns (non-negative doubles order like integers)
    for (int a = 0; a < n; ++a) {
      int best = a;
      long long bb = __double_as_longlong(q.sig[ord[a]]);
      for (int b = a + 1; b < n; ++b) {
        const long long vb = __double_as_longlong(q.sig[ord[b]]);
        if (vb > bb) {
          best = b;
          bb = vb;
        }
      }
      const int t = ord[a];
      ord[a] = ord[best];
      ord[best] = t;
    }
    int keep = grew ? n : r;
    double ratio = 0.0;
    if (grew) {
      double tot = 0.0;
      for (int a = 0; a < n; ++a) tot += q.sig[ord[a]];
      ratio = tot > 0.0 ? q.sig[ord[n - 1]] / tot : 0.0;
    }
    if (trunc_eps >= 0.0 && keep > 0) {
      double tot = 0.0;
      for (int a = 0; a < keep; ++a) tot += q.sig[ord[a]];
      int k2 = 0;
      for (int a = 0; a < keep; ++a)
        if (q.sig[ord[a]] / tot > trunc_eps) ++k2;
      keep = k2;
    }
    if (keep > r_max) keep = r_max;
    sc[3] = grew ? 1.0 / alpha : 0.0;
    sc[4] = keep;
    sc[5] = grew ? 1.0 : 0.0;
    sc[6] = ratio;
  }
  __syncthreads();
  const int keep = (int)sc[4];
  // K = P^T M^T P: U_K(kidx[m], col) = V_M(m, col), V_K(kidx[m], col) = U_M(m, col)
  for (int e = tid; e < n * keep; e += blockDim.x) {
    const int a = e / n, m = e % n;
    const int col = ord[a];
    const int row = (int)q.kidx[m];
    Uc[a * n + row] = q.VM[(size_t)col * MAXN + m];
    Vc[a * n + row] = q.UM[(size_t)col * MAXN + m];
  }
  for (int a = tid; a < keep; a += blockDim.x) snew[a] = q.sig[ord[a]];
}

}  // namespace

long secular_scratch_doubles() { return 13L * MAXN + 3L * MAXN + 8 + 2L * MAXN * MAXN; }

cudaError_t core_svd_secular(const double* S, int r, const double* p, double* sc, double* Uc,
                             double* Vc, double* snew, double trunc_eps, int r_max,
                             double* scratch, cudaStream_t s) {
  Sec q;
  double* w = scratch;
  q.d = w; w += MAXN;
  q.z = w; w += MAXN;
  q.zh = w; w += MAXN;
  q.mu = w; w += MAXN;
  q.sidx = w; w += MAXN;
  q.sig = w; w += MAXN;
  q.info = w; w += 8;
  q.act = w; w += MAXN;
  q.defl = w; w += MAXN;
  q.rot = w; w += 3 * MAXN;
  q.kidx = w; w += MAXN;
  q.UM = w; w += MAXN * MAXN;
  q.VM = w; w += MAXN * MAXN;
  const int n = r + 1;
  ++g_launches;
  sec_setup_kernel<<<1, 32, 0, s>>>(S, r, p, sc, q);
  ++g_launches;
  sec_root_kernel<<<n, 32, 0, s>>>(q);
  ++g_launches;
  sec_zhat_kernel<<<n, 32, 0, s>>>(q);
  ++g_launches;
  sec_vec_kernel<<<n, 32, 0, s>>>(q);
  ++g_launches;
  sec_finish_kernel<<<1, 256, 0, s>>>(r, q, sc, Uc, Vc, snew, trunc_eps, r_max);
  return cudaGetLastError();
}

}  // namespace rte
