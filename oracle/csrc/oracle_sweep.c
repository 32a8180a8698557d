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
