/*
 * Oracle transport sweep: plain FP64 loops, test infrastructure only.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm may load this library.  The GPU product path never links or calls it.
 *
 * What it computes (paper Sec. 2.1, Eq. (DG) with the K = 0 member of the DG
 * space Eq. (dg_space), i.e. one constant per rectangular cell, divided by the
 * cell area; backward Euler Eq. (time_discrete); matrix form Eq.
 * (kinetic_dg_discrete)):
 *
 *   for every direction k with Omega_k = (mu_k, eta_k), a_k = |mu_k|/hx,
 *   b_k = |eta_k|/hy, and every cell c visited in upwind order,
 *
 *     (tau + sigma_t[c] + a_k + b_k) psi[k][c]
 *         = S_iso[c] + scale * S_dir[k][c] + a_k psi_upx + b_k psi_upy
 *
 *   where psi_upx / psi_upy are psi of the upwind x / y neighbour, or the
 *   isotropic inflow value g of that side on the inflow boundary (the upwind
 *   flux of Eq. (DG); boundary term g_j^(bc) of Eq. (kinetic_dg_discrete)).
 *   The moment is rho[c] = sum_k w_k psi[k][c] (Sec. 2.1, S_N quadrature),
 *   summed in direction index order.
 *
 * Layout: cell c = i + nx*j, x fastest.  psi / S_dir are [nv][ncell].
 * A 1D slab is nx cells, ny = 1, eta_k = 0 (b_k = 0).
 * inflow = {west, east, south, north} or NULL for vacuum.
 */
#include <stdlib.h>
#include <string.h>
#include <math.h>

static void sweep_one_direction(int nx, int ny, double hx, double hy, double mu, double eta,
                                double tau, const double* sigma_t, const double* s_iso,
                                const double* s_dir, double scale, const double* inflow,
                                double* psi) {
  const double a = fabs(mu) / hx;
  const double b = (ny > 1 || eta != 0.0) ? fabs(eta) / hy : 0.0;
  /* x order: mu > 0 sweeps west -> east, inflow on the west side. */
  const int i0 = mu > 0 ? 0 : nx - 1, di = mu > 0 ? 1 : -1;
  const int j0 = eta >= 0 ? 0 : ny - 1, dj = eta >= 0 ? 1 : -1;
  const double gx = inflow ? (mu > 0 ? inflow[0] : inflow[1]) : 0.0;
  const double gy = inflow ? (eta >= 0 ? inflow[2] : inflow[3]) : 0.0;
  for (int jj = 0; jj < ny; ++jj) {
    const int j = j0 + dj * jj;
    for (int ii = 0; ii < nx; ++ii) {
      const int i = i0 + di * ii;
      const int c = i + nx * j;
      const double up_x = (ii == 0) ? gx : psi[c - di];
      const double up_y = (jj == 0) ? gy : psi[c - dj * nx];
      double rhs = a * up_x + b * up_y;
      if (s_iso) rhs += s_iso[c];
      if (s_dir) rhs += scale * s_dir[c];
      psi[c] = rhs / (tau + sigma_t[c] + a + b);
    }
  }
}

/* Returns 0 on success, 1 on allocation failure. */
int oracle_sweep(int nx, int ny, double hx, double hy, int nv, const double* mu, const double* eta,
                 const double* w, double tau, const double* sigma_t, const double* s_iso,
                 const double* s_dir, double s_dir_scale, const double* inflow, double* psi_out,
                 double* moment_out) {
  const long ncell = (long)nx * ny;
  double* psi = psi_out;
  if (!psi) {
    psi = (double*)malloc(sizeof(double) * ncell * nv);
    if (!psi) return 1;
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < nv; ++k)
    sweep_one_direction(nx, ny, hx, hy, mu[k], eta ? eta[k] : 0.0, tau, sigma_t, s_iso,
                        s_dir ? s_dir + (long)k * ncell : NULL, s_dir_scale, inflow,
                        psi + (long)k * ncell);
  if (moment_out) {
    for (long c = 0; c < ncell; ++c) moment_out[c] = 0.0;
    for (int k = 0; k < nv; ++k)
      for (long c = 0; c < ncell; ++c) moment_out[c] += w[k] * psi[(long)k * ncell + c];
  }
  if (!psi_out) free(psi);
  return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * Q1 upwind DG sweep (Sec. 2.1, Eq. (DG) with K = 1 in Eq. (dg_space): bilinear functions on
 * each rectangle), the paper's own discretisation.  Plain FP64 loops, test infrastructure.
 *
 * Basis of cell c: phi_{a,b}(x, y) = p_a(xi) p_b(zeta), p_0 = 1, p_1 = sqrt(3) xi, with
 * xi, zeta in [-1, 1] the cell's local coordinates; the four functions are orthonormal under
 * the cell average (1/|T|) int_T, so the mass matrix is the identity and every equation below
 * is Eq. (DG) tested with phi_{a,b} and divided by |T|.  Degree of freedom k = a + 2 b.
 *
 * Terms of Eq. (DG) for direction (mu, eta) on one cell, from the 1D pieces
 *   Dv[a][c] = (1/2) int p_a'(xi) p_c(xi) dxi     (derivative on the test function)
 *   P(s)[a]  = p_a(s)                              (trace at xi = s):
 *   (tau + sigma_t) f_k
 *   - (2 mu / hx) sum_c Dv[a][c] f_{c,b} - (2 eta / hy) sum_d Dv[b][d] f_{a,d}  (volume term)
 *   + (|mu| / hx) P(sx)[a] sum_c P(sx)[c] f_{c,b}                                (outflow x face)
 *   + (|eta| / hy) P(sy)[b] sum_d P(sy)[d] f_{a,d}                               (outflow y face)
 *   = S_k + (|mu| / hx) P(-sx)[a] tx_b + (|eta| / hy) P(-sy)[b] ty_a            (inflow faces)
 * where sx = sign(mu), sy = sign(eta) (eta = 0 counts as +), and tx_b / ty_a are the face
 * modes (face-average orthonormal: 1 and sqrt(3) times the face coordinate) of the upwind
 * value on the inflow faces: the upwind neighbour's outflow trace, or the boundary data g on
 * the inflow boundary (the upwind flux of Eq. (DG)).  The 4 x 4 system is solved by Gaussian
 * elimination with partial pivoting.
 *
 * Layout: psi / s_dir [nv][4][ncell] (mode-major per direction), s_iso / moment [4][ncell].
 * gx [2][ny][2]: face modes of the inflow on the west (0) and east (1) sides, row by row;
 * gy [2][nx][2]: south (0) and north (1), column by column; NULL means vacuum.
 */
static void solve4(double M[4][4], double r[4]) {
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int i = col + 1; i < 4; ++i)
      if (fabs(M[i][col]) > fabs(M[piv][col])) piv = i;
    if (piv != col) {
      for (int k = 0; k < 4; ++k) {
        const double t = M[col][k];
        M[col][k] = M[piv][k];
        M[piv][k] = t;
      }
      const double t = r[col];
      r[col] = r[piv];
      r[piv] = t;
    }
    for (int i = col + 1; i < 4; ++i) {
      const double m = M[i][col] / M[col][col];
      for (int k = col; k < 4; ++k) M[i][k] -= m * M[col][k];
      r[i] -= m * r[col];
    }
  }
  for (int i = 3; i >= 0; --i) {
    double s = r[i];
    for (int k = i + 1; k < 4; ++k) s -= M[i][k] * r[k];
    r[i] = s / M[i][i];
  }
}

static void sweep_q1_one_direction(int nx, int ny, double hx, double hy, double mu, double eta,
                                   double tau, const double* sigma_t, const double* s_iso,
                                   const double* s_dir, double scale, const double* gx,
                                   const double* gy, double* psi) {
  const long nc = (long)nx * ny;
  const double r3 = sqrt(3.0);
  const double Dv[2][2] = {{0.0, 0.0}, {r3, 0.0}};
  const int sx = mu > 0 ? 1 : -1, sy = eta >= 0 ? 1 : -1;
  const double Pout_x[2] = {1.0, sx * r3}, Pin_x[2] = {1.0, -sx * r3};
  const double Pout_y[2] = {1.0, sy * r3}, Pin_y[2] = {1.0, -sy * r3};
  const double ax = fabs(mu) / hx, ay = fabs(eta) / hy;
  const int i0 = mu > 0 ? 0 : nx - 1, di = mu > 0 ? 1 : -1;
  const int j0 = eta >= 0 ? 0 : ny - 1, dj = eta >= 0 ? 1 : -1;
  for (int jj = 0; jj < ny; ++jj) {
    const int j = j0 + dj * jj;
    for (int ii = 0; ii < nx; ++ii) {
      const int i = i0 + di * ii;
      const long c = i + (long)nx * j;
      /* face modes of the upwind value on the two inflow faces */
      double tx[2], ty[2];
      for (int m = 0; m < 2; ++m) {
        if (ii == 0) {
          tx[m] = gx ? gx[((sx > 0 ? 0 : 1) * ny + j) * 2 + m] : 0.0;
        } else {
          const long u = c - di;   /* upwind x neighbour, its outflow trace, y mode m */
          tx[m] = Pout_x[0] * psi[(0 + 2 * m) * nc + u] + Pout_x[1] * psi[(1 + 2 * m) * nc + u];
        }
        if (jj == 0) {
          ty[m] = gy ? gy[((sy > 0 ? 0 : 1) * nx + i) * 2 + m] : 0.0;
        } else {
          const long u = c - (long)dj * nx;   /* upwind y neighbour, x mode m */
          ty[m] = Pout_y[0] * psi[(m + 0) * nc + u] + Pout_y[1] * psi[(m + 2) * nc + u];
        }
      }
      double M[4][4], r[4];
      for (int k = 0; k < 4; ++k) {
        const int a = k & 1, b = k >> 1;
        for (int m = 0; m < 4; ++m) {
          const int cc = m & 1, d = m >> 1;
          double v = (k == m) ? tau + sigma_t[c] : 0.0;
          if (b == d) v += -(2.0 * mu / hx) * Dv[a][cc] + ax * Pout_x[a] * Pout_x[cc];
          if (a == cc) v += -(2.0 * eta / hy) * Dv[b][d] + ay * Pout_y[b] * Pout_y[d];
          M[k][m] = v;
        }
        double s = 0.0;
        if (s_iso) s += s_iso[k * nc + c];
        if (s_dir) s += scale * s_dir[k * nc + c];
        r[k] = s + ax * Pin_x[a] * tx[b] + ay * Pin_y[b] * ty[a];
      }
      solve4(M, r);
      for (int k = 0; k < 4; ++k) psi[k * nc + c] = r[k];
    }
  }
}

/* Returns 0 on success, 1 on allocation failure. */
int oracle_sweep_q1(int nx, int ny, double hx, double hy, int nv, const double* mu,
                    const double* eta, const double* w, double tau, const double* sigma_t,
                    const double* s_iso, const double* s_dir, double s_dir_scale,
                    const double* gx, const double* gy, double* psi_out, double* moment_out) {
  const long ndof = 4L * nx * ny;
  double* psi = psi_out;
  if (!psi) {
    psi = (double*)malloc(sizeof(double) * ndof * nv);
    if (!psi) return 1;
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < nv; ++k)
    sweep_q1_one_direction(nx, ny, hx, hy, mu[k], eta[k], tau, sigma_t, s_iso,
                           s_dir ? s_dir + (long)k * ndof : NULL, s_dir_scale, gx, gy,
                           psi + (long)k * ndof);
  if (moment_out) {
    for (long i = 0; i < ndof; ++i) moment_out[i] = 0.0;
    for (int k = 0; k < nv; ++k)
      for (long i = 0; i < ndof; ++i) moment_out[i] += w[k] * psi[(long)k * ndof + i];
  }
  if (!psi_out) free(psi);
  return 0;
}
