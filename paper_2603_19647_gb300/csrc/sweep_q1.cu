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
// about a hundred flops: in FP64 the kernel is bound by the FP64 pipe, not by memory, so four
// of the closed form's factors, the division among them, come from a table per cell and
// direction (built once per time step constant, 32 B per cell-direction).  Each row's
// per-cell data are read from global memory one step ahead of their use.  The FP32 instantiation (options.precision
// RTE_FP32) runs the same solve in FP32 arithmetic; the SI-SA loop's FP64 residual refines its
// increments.  All waits are bounded.
#include <cuda_runtime.h>

#include <atomic>

#include "rte_internal.h"
#include "sweep_common.cuh"

namespace rte {

namespace {
using namespace sweep_detail;

// Columns per published edge chunk: a CTA's strip starts K + RW steps after the strip above, so
// narrow chunks fill the wavefront sooner, and every chunk costs a flag poll.  Measured at
// 256^2 x 128 (SI / fused sweep): FP64 K = 2 against 4 2.88 / 5.09 against 3.30 / 5.62 ms,
// FP32 1.03 / 1.28 against 0.79 / 1.17 ms.
template <class Real>
constexpr int KQ1 = sizeof(Real) == 8 ? 2 : 4;
constexpr double SQRT3 = 1.7320508075688772;

// sqrt(3) in FP32 as an exact pair: SQRT3_HI + SQRT3_LO (to about 2^-48)
constexpr float SQRT3_HI = 1.73205077648162841796875f;
constexpr float SQRT3_LO = 3.1087250107475484e-08f;

// a * b + c rounded once, in the sweep's precision
__device__ __forceinline__ float mad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return __fma_rn(a, b, c); }

// The c-dependent factors of one cell solve (see the file comment): Q0 = q0 I + ax Bx, the
// second column's q1, beta = uy ay, S = s0 I + s1 Bx, and the inverses' scales kS, kQ.
template <class Real>
struct Q1Coef {
  Real q0, beta, s1, ps, pq, kS, kQ;
};
template <class Real>
__device__ __forceinline__ Q1Coef<Real> q1_coef(Real c, Real ax, Real ay) {
  Q1Coef<Real> k;
  k.q0 = c + ay;
  const Real q1 = mad(Real(2.0), ay, k.q0);
  k.beta = ay;   // times uy at the use
  k.s1 = ax * (k.q0 + q1 + Real(4.0) * ax);
  const Real s0 = mad(k.q0, q1, Real(3.0) * ay * ay - Real(6.0) * ax * ax);
  const Real dS = mad(s0, s0 + Real(4.0) * k.s1, Real(6.0) * k.s1 * k.s1);
  k.pq = k.q0 + Real(4.0) * ax;
  const Real dQ = mad(k.q0, k.pq, Real(6.0) * ax * ax);
  if constexpr (sizeof(Real) == 8) {   // one division: 1 / (dS dQ), both about c^4
    const Real inv = Real(1) / (dS * dQ);
    k.kS = dQ * inv;
    k.kQ = dS * inv;
  } else {                             // FP32: their product could leave the exponent range
    k.kS = Real(1) / dS;
    k.kQ = Real(1) / dQ;
  }
  k.ps = s0 + Real(4.0) * k.s1;
  return k;
}

// The same factors with the four that cost most (the division among them) read from the FP64
// table of q1_table_kernel: t = {kS, kQ, s1, ps} of the cell and direction.
template <class Real>
__device__ __forceinline__ Q1Coef<Real> q1_coef_from(Real c, Real ax, Real ay, const Real t[4]) {
  Q1Coef<Real> k;
  k.q0 = c + ay;
  k.beta = ay;
  k.pq = k.q0 + Real(4.0) * ax;
  k.kS = t[0];
  k.kQ = t[1];
  k.s1 = t[2];
  k.ps = t[3];
  return k;
}

// F = L^-1 R for the right side r (r[a + 2b] = R[a][b]) by the closed form of the file comment.
template <class Real>
__device__ __forceinline__ void q1_apply(const Q1Coef<Real>& k, Real ax, Real ux, Real uy,
                                         const Real r[4], Real f[4]) {
  const Real beta = uy * k.beta;
  // t = Q0 R1 + beta R0
  const Real b0 = mad(ux, r[3], r[2]), b1 = mad(-ux, r[2], Real(3.0) * r[3]);
  const Real t0 = mad(k.q0, r[2], mad(ax, b0, beta * r[0]));
  const Real t1 = mad(k.q0, r[3], mad(ax, b1, beta * r[1]));
  const Real e0 = mad(ux, t1, t0), e1 = mad(-ux, t0, Real(3.0) * t1);
  const Real f01 = mad(k.ps, t0, -k.s1 * e0) * k.kS;
  const Real f11 = mad(k.ps, t1, -k.s1 * e1) * k.kS;
  const Real u0 = mad(-beta, f01, r[0]), u1 = mad(-beta, f11, r[1]);
  const Real g0 = mad(ux, u1, u0), g1 = mad(-ux, u0, Real(3.0) * u1);
  f[0] = mad(k.pq, u0, -ax * g0) * k.kQ;
  f[1] = mad(k.pq, u1, -ax * g1) * k.kQ;
  f[2] = f01;
  f[3] = f11;
}

// One cell solve.  s: source modes; tx: face modes (y mode b) of the upwind value on the
// inflow x face; ty: face modes (x mode a) on the inflow y face; c = ch + cl (cl = 0 in FP64).
// Returns the cell's modes in f and its outflow traces in ox (per y mode), oy (per x mode).
// FP32: the closed form's factors carry FP32 roundings that are the same for every step and
// every solve of the cell and direction, and the rounding of c = tau + sigma_t is the same for
// all directions of the cell; left alone, they bias the operator (measured: the FP32 march
// drifting from the FP64 one by 2.3e-8 per step on the 256^2 checkerboard).  One step of
// refinement removes the bias: the residual R - L F is formed with the exact c = ch + cl and
// the cell's equations term by term, and the closed form solves for the correction.  What is
// left are the roundings of the residual, which change with the values from solve to solve.
// u x + y with u = uh + ul given as a pair (FP32; FP64 takes u = uh)
template <class Real>
__device__ __forceinline__ Real madp(Real uh, Real ul, Real x, Real y) {
  if constexpr (sizeof(Real) == 4) return mad(ul, x, mad(uh, x, y));
  else return mad(uh, x, y);
}

// kt (FP64, optional): the cell and direction's factors from the table, else computed here.
template <class Real>
__device__ __forceinline__ void q1_cell(Real ch, Real cl, Real ax, Real ay, Real ux, Real ul,
                                        Real uy, Real vl, const Real s[4], const Real tx[2],
                                        const Real ty[2], Real f[4], Real ox[2], Real oy[2],
                                        const Real* kt = nullptr) {
  // ux = ux + ul and uy = uy + vl (+-sqrt(3)) wherever they define the equations (the right
  // side's inflow terms, the residual, the outflow traces); the closed form takes ux, uy
  const Real axt0 = ax * tx[0], axt1 = ax * tx[1], ayt0 = ay * ty[0], ayt1 = ay * ty[1];
  Real r[4];
  r[0] = s[0] + axt0 + ayt0;
  r[1] = madp(-ux, -ul, axt0, s[1] + ayt1);
  r[2] = madp(-uy, -vl, ayt0, s[2] + axt1);
  r[3] = madp(-uy, -vl, ayt1, madp(-ux, -ul, axt1, s[3]));
  const Q1Coef<Real> k = kt ? q1_coef_from(ch, ax, ay, kt) : q1_coef(ch, ax, ay);
  q1_apply(k, ax, ux, uy, r, f);
  if constexpr (sizeof(Real) == 4) {
    // (L F)[a][b] = c F[a][b] + ax (Bx F)[a][b] + ay (F By^T)[a][b]
    Real bx[4], by[4], d[4], g[4];
    bx[0] = madp(ux, ul, f[1], f[0]);
    bx[1] = madp(-ux, -ul, f[0], Real(3.0) * f[1]);
    bx[2] = madp(ux, ul, f[3], f[2]);
    bx[3] = madp(-ux, -ul, f[2], Real(3.0) * f[3]);
    by[0] = madp(uy, vl, f[2], f[0]);
    by[1] = madp(uy, vl, f[3], f[1]);
    by[2] = madp(-uy, -vl, f[0], Real(3.0) * f[2]);
    by[3] = madp(-uy, -vl, f[1], Real(3.0) * f[3]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      Real e = mad(-ch, f[i], r[i]);
      e = mad(-cl, f[i], e);
      e = mad(-ax, bx[i], e);
      d[i] = mad(-ay, by[i], e);
    }
    q1_apply(k, ax, ux, uy, d, g);
#pragma unroll
    for (int i = 0; i < 4; ++i) f[i] += g[i];
  }
  ox[0] = madp(ux, ul, f[1], f[0]);
  ox[1] = madp(ux, ul, f[3], f[2]);
  oy[0] = madp(uy, vl, f[2], f[0]);
  oy[1] = madp(uy, vl, f[3], f[1]);
}

// MODE 0: SI sweep (K1): source q [4][ncell], inflow ghosts gx / gy (face mode 0), moment.
// MODE 1: fused f sweep (K2): pass A f^n = L^-1(q + tau f^{n-1}) with the inflow ghosts,
//         pass B y = L^-1(g2 + tau f^n) with zero inflow; moment of pass B.
// MODE 2: y = L^-1(g2 + tau f) from the stored f, zero inflow, moment of y.
// f: [nfam][ncell][4][dl]; pm: [nfam][4][ncell]; edge: per pass [nfam][nblk][nx][2][dl].
template <class Real, int DL, int R, int MODE>
__global__ void __launch_bounds__(32) sweep_q1_kernel(const Sweep2DArgs<Real> A) {
  constexpr int NG = 32 / DL;
  constexpr int RW = NG * R;
  constexpr int K = KQ1<Real>;
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
  const Real ax = A.a[slot], ay = A.b[slot], cw = A.w[slot];
  const Real ux = sizeof(Real) == 4 ? Real(xpos ? SQRT3_HI : -SQRT3_HI) : Real(xpos ? SQRT3 : -SQRT3);
  const Real uy = sizeof(Real) == 4 ? Real(ypos ? SQRT3_HI : -SQRT3_HI) : Real(ypos ? SQRT3 : -SQRT3);
  const Real ul = sizeof(Real) == 4 ? Real(xpos ? SQRT3_LO : -SQRT3_LO) : Real(0);
  const Real vl = sizeof(Real) == 4 ? Real(ypos ? SQRT3_LO : -SQRT3_LO) : Real(0);
  const Real tau = A.tau, tau_lo = A.tau_lo;
  const int row0 = blk * RW + gi * R;
  const Real gxA = A.gx[quad], gyA = A.gy[quad];
  Real* f_fam = (MODE != 0) ? A.f + (size_t)fam * ncell * 4 * DL : nullptr;

  // x traces carried along each row (the inflow ghost before the first column) and the y
  // traces each row passes to the row below, per pass
  Real xA[R][2], yA[R][2], xB[R][2], yB[R][2];
#pragma unroll
  for (int m = 0; m < R; ++m) {
    xA[m][0] = MODE == 0 || MODE == 1 ? gxA : Real(0);
    xA[m][1] = Real(0);
    yA[m][0] = yA[m][1] = Real(0);
    xB[m][0] = xB[m][1] = yB[m][0] = yB[m][1] = Real(0);
  }
  const bool has_up = blk > 0;
  const bool has_down = blk + 1 < A.nblk;
  const size_t plane = (size_t)A.nfam * A.nblk * nx * 2 * DL;
  const Real* edge_in = A.edge + ((size_t)(fam * A.nblk + (has_up ? blk - 1 : 0)) * nx) * 2 * DL;
  Real* edge_out = A.edge + ((size_t)(fam * A.nblk + blk) * nx) * 2 * DL;
  unsigned* flag_in = &A.ctrl->flags[fam * A.nblk + (has_up ? blk - 1 : 0)];
  unsigned* flag_out = &A.ctrl->flags[fam * A.nblk + blk];
  const Real gyTop = MODE == 2 ? Real(0) : gyA;
  const int T = nx + RW - 1;
  const int nchunk = (T + K - 1) / K;
  bool abandon = false;
  auto cell_of = [&](int x, int jj) {
    return (long)(ypos ? jj : ny - 1 - jj) * nx + (xpos ? x : nx - 1 - x);
  };
  // The per-cell inputs of each row (sigma_t, the source modes, the stored f) are loaded one
  // step ahead of their use, into the other half of a double buffer, so that the loads' latency
  // overlaps the current step's cell solves instead of stalling the wavefront (measured at
  // 256^2 x 128: FP32 SI sweep 0.79 -> 0.69 ms, fused sweep 1.38 -> 1.04-1.10 ms, FP64 fused
  // sweep 5.86 -> 5.76 ms; the FP64 SI sweep, once the table below took a third of its FP64
  // work, 1.99 -> 1.86 ms).
  struct In {
    Real st, stl, q[4], fo[4], g[4];
  };
  In buf[2][R];
  auto fetch = [&](int t, In (&d)[R]) {
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int x = t - m - gi * R;
      const int jj = row0 + m;
      if (x >= 0 && x < nx && jj < ny) {
        const long cell = cell_of(x, jj);
        d[m].st = A.sig_t[cell];
        if constexpr (sizeof(Real) == 4) d[m].stl = A.sig_tl[cell];
#pragma unroll
        for (int md = 0; md < 4; ++md) {
          if constexpr (MODE != 2) d[m].q[md] = A.q[md * ncell + cell];
          if constexpr (MODE != 0) {
            d[m].fo[md] = f_fam[(cell * 4 + md) * DL + dl];
            d[m].g[md] = A.g2[md * ncell + cell];
          }
        }
      }
    }
  };
  static_assert(K % 2 == 0, "the double buffer alternates within a chunk");
  fetch(0, buf[0]);
  // FP64: four of the closed form's factors per cell and direction (q1_table_kernel, family
  // layout [fam][cell][4][dl]), read one step ahead: the table is too large for L2, and the
  // factors take the division and about a third of the FP64 operations of a cell solve
  constexpr bool TABLE = sizeof(Real) == 8;
  Real kt[2][R][4];
  const Real* tab = TABLE ? A.inv_d + (size_t)fam * ncell * 4 * DL : nullptr;
  auto fetch_k = [&](int t, Real (&d)[R][4]) {
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int x = t - m - gi * R;
      const int jj = row0 + m;
      if (x >= 0 && x < nx && jj < ny) {
        const Real* p = tab + (size_t)cell_of(x, jj) * 4 * DL + dl;
#pragma unroll
        for (int i = 0; i < 4; ++i) d[m][i] = __ldcs(p + i * DL);
      }
    }
  };
  if constexpr (TABLE) fetch_k(0, kt[0]);

  for (int c = 0; c < nchunk; ++c) {
    const int tb = c * K;
    // top input of lane group 0 for columns [tb, tb + K)
    Real eA[K][2], eB[K][2];
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
          eA[k][md] = ok ? ldcg(edge_in + ((size_t)x * 2 + md) * DL + dl) : Real(0);
          eB[k][md] = (TWO && ok) ? ldcg(edge_in + plane + ((size_t)x * 2 + md) * DL + dl) : Real(0);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        eA[k][0] = gyTop;
        eA[k][1] = Real(0);
        eB[k][0] = eB[k][1] = Real(0);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int t = tb + k;
      Real upA[2], upB[2];
#pragma unroll
      for (int md = 0; md < 2; ++md) {
        upA[md] = __shfl_up_sync(FULL, yA[R - 1][md], DL);
        upB[md] = TWO ? __shfl_up_sync(FULL, yB[R - 1][md], DL) : Real(0);
        if (gi == 0) {
          upA[md] = eA[k][md];
          upB[md] = eB[k][md];
        }
      }
      fetch(t + 1, buf[(k + 1) & 1]);
      if constexpr (TABLE) fetch_k(t + 1, kt[(k + 1) & 1]);
      Real mv[NV];
#pragma unroll
      for (int m = R - 1; m >= 0; --m) {
        const int x = t - m - gi * R;
        const int jj = row0 + m;
#pragma unroll
        for (int md = 0; md < 4; ++md) mv[md * R + m] = Real(0);
        if (x >= 0 && x < nx && jj < ny) {
          const In& in = buf[k & 1][m];
          const long cell = cell_of(x, jj);
          // c = tau + sigma_t: in FP32 as an exact pair ch + cl (both given as exact pairs)
          Real ch, cl = Real(0);
          if constexpr (sizeof(Real) == 4) {
            const Real sum = tau + in.st, bb = sum - tau;
            const Real e = ((tau - (sum - bb)) + (in.st - bb)) + (tau_lo + in.stl);
            ch = sum + e;
            cl = e - (ch - sum);
          } else {
            ch = tau + in.st;
          }
          const Real tyA[2] = {m == 0 ? upA[0] : yA[m > 0 ? m - 1 : 0][0],
                                 m == 0 ? upA[1] : yA[m > 0 ? m - 1 : 0][1]};
          Real s[4], fA[4], ox[2], oy[2];
#pragma unroll
          for (int md = 0; md < 4; ++md) {
            if constexpr (MODE == 0) s[md] = in.q[md];
            else if constexpr (MODE == 2) s[md] = mad(tau, in.fo[md], in.g[md]);
            else s[md] = mad(tau, in.fo[md], in.q[md]);
          }
          const Real* kc = TABLE ? kt[k & 1][m] : nullptr;
          q1_cell(ch, cl, ax, ay, ux, ul, uy, vl, s, xA[m], tyA, fA, ox, oy, kc);
          xA[m][0] = ox[0];
          xA[m][1] = ox[1];
          yA[m][0] = oy[0];
          yA[m][1] = oy[1];
          if constexpr (TWO) {
#pragma unroll
            for (int md = 0; md < 4; ++md) f_fam[(cell * 4 + md) * DL + dl] = fA[md];
            const Real tyB[2] = {m == 0 ? upB[0] : yB[m > 0 ? m - 1 : 0][0],
                                   m == 0 ? upB[1] : yB[m > 0 ? m - 1 : 0][1]};
            Real sB[4], fB[4];
#pragma unroll
            for (int md = 0; md < 4; ++md) sB[md] = mad(tau, fA[md], in.g[md]);
            q1_cell(ch, cl, ax, ay, ux, ul, uy, vl, sB, xB[m], tyB, fB, ox, oy, kc);
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
      TReduceW<Real, NV, DL / 2>::run(mv, cw, dl);
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
        if (writer && x >= 0 && x < nx && jj < ny)
          A.pm[((size_t)fam * 4 + md) * ncell + cell_of(x, jj)] = mv[i];
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

template <class Real, int DL, int R, int MODE>
cudaError_t launch_q1_dlr(const Sweep2DArgs<Real>& a, cudaStream_t s) {
  constexpr int RW = (32 / DL) * R;
  if (a.rows_per_blk != RW || a.nblk != (a.ny + RW - 1) / RW) return cudaErrorInvalidValue;
  ++g_launches;
  sweep_q1_kernel<Real, DL, R, MODE><<<(unsigned)(a.nfam * a.nblk), 32, 0, s>>>(a);
  return cudaGetLastError();
}

template <class Real, int DL, int MODE>
cudaError_t launch_q1_dl(const Sweep2DArgs<Real>& a, int R, cudaStream_t s) {
  switch (R) {
    case 1: return launch_q1_dlr<Real, DL, 1, MODE>(a, s);
    case 2: return launch_q1_dlr<Real, DL, 2, MODE>(a, s);
    case 4: return launch_q1_dlr<Real, DL, 4, MODE>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// One (precision, mode) per translation unit: the build compiles the six parts in parallel
// (RTE_Q1_PART 0-5 = FP64 modes 0-2, FP32 modes 0-2; -1 builds all), and part 0 also holds
// the public entry points.
template <class Real, int MODE>
cudaError_t launch_q1_mode(const Sweep2DArgs<Real>& a, int dl, int R, cudaStream_t s) {
  switch (dl) {
    case 2: return launch_q1_dl<Real, 2, MODE>(a, R, s);
    case 4: return launch_q1_dl<Real, 4, MODE>(a, R, s);
    case 8: return launch_q1_dl<Real, 8, MODE>(a, R, s);
    case 16: return launch_q1_dl<Real, 16, MODE>(a, R, s);
    case 32: return launch_q1_dl<Real, 32, MODE>(a, R, s);
    default: return cudaErrorInvalidValue;
  }
}

#ifndef RTE_Q1_PART
#define RTE_Q1_PART -1
#endif
#define RTE_Q1_INST(REAL, MODE)                                                               \
  template cudaError_t launch_q1_mode<REAL, MODE>(const Sweep2DArgs<REAL>&, int, int,        \
                                                  cudaStream_t);
#define RTE_Q1_EXTERN(REAL, MODE)                                                            \
  extern template cudaError_t launch_q1_mode<REAL, MODE>(const Sweep2DArgs<REAL>&, int, int, \
                                                         cudaStream_t);
#if RTE_Q1_PART == -1 || RTE_Q1_PART == 0
RTE_Q1_INST(double, 0)
#else
RTE_Q1_EXTERN(double, 0)
#endif
#if RTE_Q1_PART == -1 || RTE_Q1_PART == 1
RTE_Q1_INST(double, 1)
#else
RTE_Q1_EXTERN(double, 1)
#endif
#if RTE_Q1_PART == -1 || RTE_Q1_PART == 2
RTE_Q1_INST(double, 2)
#else
RTE_Q1_EXTERN(double, 2)
#endif
#if RTE_Q1_PART == -1 || RTE_Q1_PART == 3
RTE_Q1_INST(float, 0)
#else
RTE_Q1_EXTERN(float, 0)
#endif
#if RTE_Q1_PART == -1 || RTE_Q1_PART == 4
RTE_Q1_INST(float, 1)
#else
RTE_Q1_EXTERN(float, 1)
#endif
#if RTE_Q1_PART == -1 || RTE_Q1_PART == 5
RTE_Q1_INST(float, 2)
#else
RTE_Q1_EXTERN(float, 2)
#endif

#if RTE_Q1_PART == -1 || RTE_Q1_PART == 0
namespace {
// {kS, kQ, s1, ps} of q1_coef for every cell and direction slot (slot = fam dl + d), in the
// family layout [fam][cell][4][dl]: one thread per (cell, slot).
__global__ void q1_table_kernel(const double* __restrict__ sig_t, const double* __restrict__ a,
                                const double* __restrict__ b, double tau, int ncell, int nslot,
                                int dl, double* __restrict__ out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)ncell * nslot) return;
  const int slot = (int)(i % nslot);
  const long cell = i / nslot;
  const Q1Coef<double> k = q1_coef(tau + sig_t[cell], a[slot], b[slot]);
  const int fam = slot / dl, d = slot % dl;
  double* o = out + ((size_t)fam * ncell + cell) * 4 * dl + d;
  o[0] = k.kS;
  o[(size_t)dl] = k.kQ;
  o[2 * (size_t)dl] = k.s1;
  o[3 * (size_t)dl] = k.ps;
}

template <class Real>
cudaError_t launch_sweep_q1_impl(const Sweep2DArgs<Real>& a, int mode, int dl, int R,
                                 cudaStream_t s) {
  if (a.nslot != a.nfam * dl) return cudaErrorInvalidValue;
  switch (mode) {
    case 0: return launch_q1_mode<Real, 0>(a, dl, R, s);
    case 1: return launch_q1_mode<Real, 1>(a, dl, R, s);
    case 2: return launch_q1_mode<Real, 2>(a, dl, R, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t launch_q1_table(const double* sig_t, const double* a, const double* b, double tau,
                            int ncell, int nslot, int dl, double* out, cudaStream_t s) {
  if (dl < 1 || nslot % dl != 0) return cudaErrorInvalidValue;
  const long n = (long)ncell * nslot;
  ++g_launches;
  q1_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sig_t, a, b, tau, ncell, nslot, dl,
                                                            out);
  return cudaGetLastError();
}

cudaError_t launch_sweep_q1(const Sweep2DArgs<double>& a, int mode, int dl, int R,
                            cudaStream_t s) {
  return launch_sweep_q1_impl(a, mode, dl, R, s);
}
cudaError_t launch_sweep_q1(const Sweep2DArgs<float>& a, int mode, int dl, int R, cudaStream_t s) {
  return launch_sweep_q1_impl(a, mode, dl, R, s);
}
#endif

}  // namespace rte
