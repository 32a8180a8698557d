// Q1 transport sweeps: the upwind DG cell solve of Sec. 2.1 Eq. (DG) with K = 1 (bilinear
// functions on each rectangle, the paper's own discretisation), applied for all directions in
// upwind order (Sec. 2.3, "transport sweep"), with the quadrature moment of Sec. 2.1 fused in.
//
// Unknowns of a cell: f_k, k = a + 2 b, the coefficients of p_a(xi) p_b(zeta) with p_0 = 1,
// p_1 = sqrt(3) t in the cell's local coordinates (orthonormal under the cell average, so the
// mass matrix is I).  As a 2 x 2 array F[a][b] (a: x mode, b: y mode) the cell equations of
// direction (mu, eta) are
//
//   (c I + ax Bx) F + F (ay By)^T = R,   c = tau + sigma_t,  ax = |mu|/hx,  ay = |eta|/hy,
//   Bx = [[1, ux], [-ux, 3]], ux = sign(mu) sqrt(3)   (By likewise with uy = sign(eta) sqrt(3)),
//
// from the volume term and the outflow faces of Eq. (DG); R holds the source and the upwind
// traces on the two inflow faces.  Column by column (b = 0, 1), with Q0 = (c + ay) I + ax Bx,
// Q1 = (c + 3 ay) I + ax Bx and beta = uy ay:
//   Q0 F0 + beta F1 = R0,   -beta F0 + Q1 F1 = R1,
// so F1 = S^-1 (Q0 R1 + beta R0), S = Q0 Q1 + beta^2 I, and F0 = Q0^-1 (R0 - beta F1).
// S and Q0 are both of the form s0 I + s1 Bx, and since Bx^2 = 4 Bx - 6 I the inverse of such a
// matrix is ((s0 + 4 s1) I - s1 Bx) / (s0^2 + 4 s0 s1 + 6 s1^2): one division per cell solve.
//
// The sweep schedule is the strip chain of the Q0 kernel in its simplest form: lane =
// direction (dl lanes per family of one quadrant), a lane group owns R consecutive rows and runs
// them on a skewed schedule (row m handles column t - m at step t), lane groups of a warp are
// stacked vertically and hand their bottom row to the group below through a shuffle, and a CTA
// is one warp that takes the top row of its strip from the CTA above through global memory,
// published in chunks of K columns behind a release flag.  CTAs take tickets in
// row-block-major order, so a CTA only waits for CTAs that already started.  A cell solve is
// about a hundred FP64 flops: the kernel is bound by the FP64 pipe, not by memory, and reads
// its per-cell data straight from global memory.  All waits are bounded.
#include <cuda_runtime.h>

#include <atomic>

#include "rte_internal.h"
#include "sweep_common.cuh"

namespace rte {

namespace {
using namespace sweep_detail;

constexpr int KQ1 = 4;   // columns per published edge chunk
constexpr double SQRT3 = 1.7320508075688772;

// One cell solve (see the file comment).  s: source modes; tx: face modes (y mode b) of the
// upwind value on the inflow x face; ty: face modes (x mode a) on the inflow y face.
// Returns the cell's modes in f and its outflow traces in ox (per y mode), oy (per x mode).
__device__ __forceinline__ void q1_cell(double c, double ax, double ay, double ux, double uy,
                                        const double s[4], const double tx[2],
                                        const double ty[2], double f[4], double ox[2],
                                        double oy[2]) {
  const double axt0 = ax * tx[0], axt1 = ax * tx[1], ayt0 = ay * ty[0], ayt1 = ay * ty[1];
  const double r00 = s[0] + axt0 + ayt0;
  const double r10 = fma(-ux, axt0, s[1] + ayt1);
  const double r01 = fma(-uy, ayt0, s[2] + axt1);
  const double r11 = fma(-uy, ayt1, fma(-ux, axt1, s[3]));
  const double q0 = c + ay, q1 = fma(2.0, ay, q0), beta = uy * ay;
  const double s1 = ax * (q0 + q1 + 4.0 * ax);
  const double s0 = fma(q0, q1, 3.0 * ay * ay - 6.0 * ax * ax);
  // t = Q0 R1 + beta R0
  const double b0 = fma(ux, r11, r01), b1 = fma(-ux, r01, 3.0 * r11);
  const double t0 = fma(q0, r01, fma(ax, b0, beta * r00));
  const double t1 = fma(q0, r11, fma(ax, b1, beta * r10));
  const double e0 = fma(ux, t1, t0), e1 = fma(-ux, t0, 3.0 * t1);
  const double dS = fma(s0, s0 + 4.0 * s1, 6.0 * s1 * s1);
  const double pq = q0 + 4.0 * ax;
  const double dQ = fma(q0, pq, 6.0 * ax * ax);
  const double inv = 1.0 / (dS * dQ);
  const double kS = dQ * inv, kQ = dS * inv;
  const double ps = s0 + 4.0 * s1;
  const double f01 = fma(ps, t0, -s1 * e0) * kS;
  const double f11 = fma(ps, t1, -s1 * e1) * kS;
  const double u0 = fma(-beta, f01, r00), u1 = fma(-beta, f11, r10);
  const double g0 = fma(ux, u1, u0), g1 = fma(-ux, u0, 3.0 * u1);
  const double f00 = fma(pq, u0, -ax * g0) * kQ;
  const double f10 = fma(pq, u1, -ax * g1) * kQ;
  f[0] = f00;
  f[1] = f10;
  f[2] = f01;
  f[3] = f11;
  ox[0] = fma(ux, f10, f00);
  ox[1] = fma(ux, f11, f01);
  oy[0] = fma(uy, f01, f00);
  oy[1] = fma(uy, f11, f10);
}

// MODE 0: SI sweep (K1): source q [4][ncell], inflow ghosts gx / gy (face mode 0), moment.
// MODE 1: fused f sweep (K2): pass A f^n = L^-1(q + tau f^{n-1}) with the inflow ghosts,
//         pass B y = L^-1(g2 + tau f^n) with zero inflow; moment of pass B.
// MODE 2: y = L^-1(g2 + tau f) from the stored f, zero inflow, moment of y.
// f: [nfam][ncell][4][dl]; pm: [nfam][4][ncell]; edge: per pass [nfam][nblk][nx][2][dl].
template <int DL, int R, int MODE>
__global__ void __launch_bounds__(32) sweep_q1_kernel(const Sweep2DArgs<double> A) {
  constexpr int NG = 32 / DL;
  constexpr int RW = NG * R;
  constexpr int K = KQ1;
  constexpr bool TWO = MODE == 1;
  constexpr int NV = 4 * R;   // moment values of one step: (mode, row)
  if (A.skip && *A.skip) return;   // before the ticket: the control block stays untouched
  const int lane = threadIdx.x;
  const int gi = lane / DL, dl = lane % DL;
  unsigned ticket = 0;
  if (lane == 0) ticket = atomicAdd(&A.ctrl->ticket, 1u);
  ticket = __shfl_sync(FULL, ticket, 0);
  const int blk = (int)(ticket / (unsigned)A.nfam);
  const int fam = (int)(ticket % (unsigned)A.nfam);
  const int quad = A.fam_quad[fam];
  const bool xpos = (quad & 1) == 0;
  const bool ypos = quad < 2;
  const int nx = A.nx, ny = A.ny;
  const long ncell = (long)nx * ny;
  const int slot = fam * DL + dl;
  const double ax = A.a[slot], ay = A.b[slot], cw = A.w[slot];
  const double ux = xpos ? SQRT3 : -SQRT3, uy = ypos ? SQRT3 : -SQRT3;
  const double tau = A.tau;
  const int row0 = blk * RW + gi * R;
  const double gxA = A.gx[quad], gyA = A.gy[quad];
  double* f_fam = (MODE != 0) ? A.f + (size_t)fam * ncell * 4 * DL : nullptr;

  // x traces carried along each row (the inflow ghost before the first column) and the y
  // traces each row passes to the row below, per pass
  double xA[R][2], yA[R][2], xB[R][2], yB[R][2];
#pragma unroll
  for (int m = 0; m < R; ++m) {
    xA[m][0] = MODE == 0 || MODE == 1 ? gxA : 0.0;
    xA[m][1] = 0.0;
    yA[m][0] = yA[m][1] = 0.0;
    xB[m][0] = xB[m][1] = yB[m][0] = yB[m][1] = 0.0;
  }
  const bool has_up = blk > 0;
  const bool has_down = blk + 1 < A.nblk;
  const size_t plane = (size_t)A.nfam * A.nblk * nx * 2 * DL;
  const double* edge_in = A.edge + ((size_t)(fam * A.nblk + (has_up ? blk - 1 : 0)) * nx) * 2 * DL;
  double* edge_out = A.edge + ((size_t)(fam * A.nblk + blk) * nx) * 2 * DL;
  unsigned* flag_in = &A.ctrl->flags[fam * A.nblk + (has_up ? blk - 1 : 0)];
  unsigned* flag_out = &A.ctrl->flags[fam * A.nblk + blk];
  const double gyTop = MODE == 2 ? 0.0 : gyA;
  const int T = nx + RW - 1;
  const int nchunk = (T + K - 1) / K;
  bool abandon = false;

  for (int c = 0; c < nchunk; ++c) {
    const int tb = c * K;
    // top input of lane group 0 for columns [tb, tb + K)
    double eA[K][2], eB[K][2];
    if (has_up && tb < nx) {
      const int need = min(tb + K, nx);
      if (!abandon) {
        unsigned spins = 0;
        while (ld_acquire(flag_in) < (unsigned)need) {
          if (++spins > SPIN_LIMIT || ld_acquire(&A.ctrl->err) != 0u) {
            if (lane == 0) atomicExch(&A.ctrl->err, 1u);
            abandon = true;
            break;
          }
          if (spins > 256) __nanosleep(64);
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int x = tb + k;
        const bool ok = gi == 0 && x < nx;
#pragma unroll
        for (int md = 0; md < 2; ++md) {
          eA[k][md] = ok ? ldcg(edge_in + ((size_t)x * 2 + md) * DL + dl) : 0.0;
          eB[k][md] = (TWO && ok) ? ldcg(edge_in + plane + ((size_t)x * 2 + md) * DL + dl) : 0.0;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        eA[k][0] = gyTop;
        eA[k][1] = 0.0;
        eB[k][0] = eB[k][1] = 0.0;
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int t = tb + k;
      double upA[2], upB[2];
#pragma unroll
      for (int md = 0; md < 2; ++md) {
        upA[md] = __shfl_up_sync(FULL, yA[R - 1][md], DL);
        upB[md] = TWO ? __shfl_up_sync(FULL, yB[R - 1][md], DL) : 0.0;
        if (gi == 0) {
          upA[md] = eA[k][md];
          upB[md] = eB[k][md];
        }
      }
      double mv[NV];
#pragma unroll
      for (int m = R - 1; m >= 0; --m) {
        const int x = t - m - gi * R;
        const int jj = row0 + m;
#pragma unroll
        for (int md = 0; md < 4; ++md) mv[md * R + m] = 0.0;
        if (x >= 0 && x < nx && jj < ny) {
          const int px = xpos ? x : nx - 1 - x;
          const int py = ypos ? jj : ny - 1 - jj;
          const long cell = (long)py * nx + px;
          const double cc = tau + A.sig_t[cell];
          const double tyA[2] = {m == 0 ? upA[0] : yA[m > 0 ? m - 1 : 0][0],
                                 m == 0 ? upA[1] : yA[m > 0 ? m - 1 : 0][1]};
          double fo[4] = {0.0, 0.0, 0.0, 0.0};
          if constexpr (MODE != 0) {
#pragma unroll
            for (int md = 0; md < 4; ++md) fo[md] = f_fam[(cell * 4 + md) * DL + dl];
          }
          double s[4], fA[4], ox[2], oy[2];
#pragma unroll
          for (int md = 0; md < 4; ++md) {
            if constexpr (MODE == 0) s[md] = A.q[md * ncell + cell];
            else if constexpr (MODE == 2) s[md] = fma(tau, fo[md], A.g2[md * ncell + cell]);
            else s[md] = fma(tau, fo[md], A.q[md * ncell + cell]);
          }
          q1_cell(cc, ax, ay, ux, uy, s, xA[m], tyA, fA, ox, oy);
          xA[m][0] = ox[0];
          xA[m][1] = ox[1];
          yA[m][0] = oy[0];
          yA[m][1] = oy[1];
          if constexpr (TWO) {
#pragma unroll
            for (int md = 0; md < 4; ++md) f_fam[(cell * 4 + md) * DL + dl] = fA[md];
            const double tyB[2] = {m == 0 ? upB[0] : yB[m > 0 ? m - 1 : 0][0],
                                   m == 0 ? upB[1] : yB[m > 0 ? m - 1 : 0][1]};
            double sB[4], fB[4];
#pragma unroll
            for (int md = 0; md < 4; ++md) sB[md] = fma(tau, fA[md], A.g2[md * ncell + cell]);
            q1_cell(cc, ax, ay, ux, uy, sB, xB[m], tyB, fB, ox, oy);
            xB[m][0] = ox[0];
            xB[m][1] = ox[1];
            yB[m][0] = oy[0];
            yB[m][1] = oy[1];
#pragma unroll
            for (int md = 0; md < 4; ++md) mv[md * R + m] = fB[md];
          } else {
#pragma unroll
            for (int md = 0; md < 4; ++md) mv[md * R + m] = fA[md];
          }
        }
      }
      // quadrature moment of the step's R cells, four modes each: one weighted
      // transpose-reduce over the lane group's directions
      TReduceW<double, NV, DL / 2>::run(mv, cw, dl);
      constexpr int PER = NV >= DL ? NV / DL : 1;
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        int idx;
        bool writer;
        if constexpr (NV >= DL) {
          idx = dl * PER + i;
          writer = true;
        } else {
          idx = dl / (DL / NV);
          writer = (dl & (DL / NV - 1)) == 0;
        }
        const int md = idx / R, m = idx % R;
        const int x = t - m - gi * R;
        const int jj = row0 + m;
        if (writer && x >= 0 && x < nx && jj < ny) {
          const int px = xpos ? x : nx - 1 - x;
          const int py = ypos ? jj : ny - 1 - jj;
          A.pm[((size_t)fam * 4 + md) * ncell + (long)py * nx + px] = mv[i];
        }
      }
      // bottom row of the strip: to the next CTA
      const int xb = t - (RW - 1);
      if (has_down && gi == NG - 1 && xb >= 0 && xb < nx) {
#pragma unroll
        for (int md = 0; md < 2; ++md) {
          edge_out[((size_t)xb * 2 + md) * DL + dl] = yA[R - 1][md];
          if constexpr (TWO) edge_out[plane + ((size_t)xb * 2 + md) * DL + dl] = yB[R - 1][md];
        }
      }
    }
    // publish the bottom-row columns finished in this chunk
    const int done = min(tb + K - (RW - 1), nx);
    if (done > 0 && has_down) {
      __syncwarp();
      if (lane == 0) st_release(flag_out, (unsigned)done);
    }
  }
  // Self-reset of the control block by the last CTA to finish.
  __syncwarp();
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

template <int DL, int R, int MODE>
cudaError_t launch_q1_dlr(const Sweep2DArgs<double>& a, cudaStream_t s) {
  constexpr int RW = (32 / DL) * R;
  if (a.rows_per_blk != RW || a.nblk != (a.ny + RW - 1) / RW) return cudaErrorInvalidValue;
  ++g_launches;
  sweep_q1_kernel<DL, R, MODE><<<(unsigned)(a.nfam * a.nblk), 32, 0, s>>>(a);
  return cudaGetLastError();
}

template <int DL, int MODE>
cudaError_t launch_q1_dl(const Sweep2DArgs<double>& a, int R, cudaStream_t s) {
  switch (R) {
    case 1: return launch_q1_dlr<DL, 1, MODE>(a, s);
    case 2: return launch_q1_dlr<DL, 2, MODE>(a, s);
    case 4: return launch_q1_dlr<DL, 4, MODE>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int MODE>
cudaError_t launch_q1_mode(const Sweep2DArgs<double>& a, int dl, int R, cudaStream_t s) {
  switch (dl) {
    case 8: return launch_q1_dl<8, MODE>(a, R, s);
    case 16: return launch_q1_dl<16, MODE>(a, R, s);
    case 32: return launch_q1_dl<32, MODE>(a, R, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_sweep_q1(const Sweep2DArgs<double>& a, int mode, int dl, int R,
                            cudaStream_t s) {
  if (a.nslot != a.nfam * dl) return cudaErrorInvalidValue;
  switch (mode) {
    case 0: return launch_q1_mode<0>(a, dl, R, s);
    case 1: return launch_q1_mode<1>(a, dl, R, s);
    case 2: return launch_q1_mode<2>(a, dl, R, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rte
