// 2D transport sweep in tile sequence (Sec. 2.1 Eq. (DG) with K = 0, in upwind order,
// Sec. 2.3), with the quadrature moment fused in; FP32 (modes 0-4) and FP64 (modes 0-2).
//
// Lane = direction (dl lanes per family of one quadrant), as in the strip chain of sweep.cu,
// but a lane group owns a strip of TH rows and walks it one TW x TH tile at a time: inside a
// tile every lane solves all TW * TH cells of its direction by itself (the x-upwind value is
// the cell to the left, the y-upwind value the cell above, both in the lane's registers), so
// the per-cell work is the cell solve alone and the hand-offs happen once per tile:
//   * the bottom row of a tile goes to the lane group below by one warp shuffle per column,
//   * from the last group of a warp to the first group of the next warp through a ring of
//     RD tiles in shared memory (bounded spins on shared counters),
//   * from the last warp of a CTA to the first warp of the next CTA of the same family
//     through global memory behind a release flag per tile (bounded spins).
// At warp step T lane group g works on tile T - g, so a warp keeps NG = 32 / dl tiles in
// flight and the strips of a family form one pipeline down the grid.  Each group stages the
// per-cell data of its next tile (the sources, f for the fused sweep, and the diagonal: in
// FP32 sigma_t as an exact pair for the two-part reciprocal, in FP64 the per-direction table
// 1 / (tau + sigma_t + a + b) of the cells) into its own double buffer with cp.async while it
// computes the current one.
// Out-of-range cells of the last tiles are computed from zero-filled inputs and never
// stored; they lie downstream of every valid cell.
//
// Modes: 0 SI sweep (q, zero inflow unless given), 1 fused f sweep (pass A writes f^n, pass B
// the moment of L^-1(g2 + tau f^n)), 2 y from the stored f, 3 / 4 = 1 / 2 with f stored as a
// BF16 remainder about a per-cell FP32 reference (stochastic rounding on write).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>

#include "rte_internal.h"
#include "sweep_common.cuh"

namespace rte {

namespace {
using namespace sweep_detail;

constexpr int TW = 8;   // columns per tile
constexpr int RD = 4;   // tiles held by a ring between two warps

template <class Real, int DL, int TH, int MODE>
struct TileCfg {
  static constexpr bool TBL = sizeof(Real) == 8;   // FP64: diagonal from the inverse table
  static constexpr bool BF = MODE >= 3;
  static_assert(!(TBL && BF), "BF16 storage is an FP32 mode");
  static constexpr int MB = BF ? MODE - 2 : MODE;
  static constexpr int NG = 32 / DL;
  static constexpr int NP = MB == 1 ? 2 : 1;
  static constexpr int CELLS = TH * TW;
  static constexpr int RS = (int)sizeof(Real);
  // per-cell arrays: (FP32) sigma_t hi, lo, then q (modes 0, 1), g2 (modes 1, 2), BF16
  // references
  static constexpr int A_ST = 0, A_STL = 1, A_Q = TBL ? 0 : 2;
  static constexpr int A_G2 = A_Q + (MB != 2 ? 1 : 0);
  static constexpr int A_FRO = A_G2 + (MB != 0 ? 1 : 0);
  static constexpr int A_FRN = A_FRO + 1;
  static constexpr int NARR = (TBL ? 0 : 2) + (MB != 2 ? 1 : 0) + (MB != 0 ? 1 : 0) + (BF ? 2 : 0);
  static constexpr int ESZ = BF ? 2 : RS;                      // bytes of one stored f value
  static constexpr int F_BYTES = (MB != 0) ? CELLS * DL * ESZ : 0;
  static constexpr int T_BYTES = TBL ? CELLS * DL * RS : 0;    // inverse-diagonal table
  static constexpr int GROUP_BYTES = NARR * CELLS * RS + F_BYTES + T_BYTES;   // one buffer
  static constexpr int WARP_BYTES = 2 * NG * GROUP_BYTES;
  static constexpr int RING_REALS = NP * RD * TW * DL;
  static constexpr int FP = (MB != 0) ? DL * ESZ / 16 : 0;     // 16-byte pieces of f per cell
  static constexpr int TP = TBL ? DL * RS / 16 : 0;            // the same for the table
  static_assert((NARR * CELLS * RS) % 16 == 0 && F_BYTES % 16 == 0, "16-byte staging pieces");
};

// The diagonal 1 / (tau + sigma_t + a + b) of staged cell c for the lane's direction as h + l:
// FP32 from the exact sigma_t pair (arrays 0 and 1) by the two-part reciprocal, FP64 from the
// staged inverse table (l = 0).
template <bool TBL, class Real>
__device__ __forceinline__ void diag(Real ct, Real ctl, const Real* arr, const Real* tab, int c,
                                     int dl, int cells, int dln, Real& h, Real& l) {
  if constexpr (TBL) {
    h = tab[c * dln + dl];
    l = Real(0);
  } else {
    const Rcp2 rp = rcp_pair(ct, ctl, arr[c], arr[cells + c]);
    h = rp.h;
    l = rp.l;
  }
}

template <class Real, int DL, int TH, int MODE>
__global__ void __launch_bounds__(256) sweep2d_tile_kernel(const Sweep2DArgs<Real> A) {
  using C = TileCfg<Real, DL, TH, MODE>;
  constexpr bool TBL = C::TBL;
  constexpr int MB = C::MB;
  constexpr bool BF = C::BF;
  constexpr int NG = C::NG;
  if (A.skip && *A.skip) return;   // before the ticket: the control block stays untouched
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ unsigned s_ticket;
  __shared__ volatile int s_prod[8];    // tiles of its last group's bottom rows warp w has put in the ring
  __shared__ volatile int s_cons[8];    // tiles of the ring above warp w has read
  __shared__ volatile int s_abandon;

  const int W = blockDim.x >> 5;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane / DL, dl = lane % DL;
  if (tid == 0) {
    s_ticket = atomicAdd(&A.ctrl->ticket, 1u);
    s_abandon = 0;
  }
  if (tid < 8) {
    s_prod[tid] = 0;
    s_cons[tid] = 0;
  }
  __syncthreads();
  const unsigned ticket = s_ticket;
  const int blk = (int)(ticket / (unsigned)A.nfam);
  const int fam = (int)(ticket % (unsigned)A.nfam);
  const int quad = A.fam_quad[fam];
  const bool xpos = (quad & 1) == 0;
  const bool ypos = quad < 2;
  const int nx = A.nx, ny = A.ny;
  const long ncell = (long)nx * ny;
  const int slot = fam * DL + dl;
  // FP64 (table): the lane carries w psi of its direction, as in the strip chain: the table
  // holds w / (tau + sigma_t + a + b), the recurrence takes a / w, b / w, tau / w and ghosts
  // times w, and the moment is a plain sum (stored f is w f).
  const Real w0 = A.w[slot];
  const Real iw = TBL ? (w0 != Real(0) ? Real(1) / w0 : Real(0)) : Real(1);
  const Real ca = A.a[slot] * iw, cb = A.b[slot] * iw, cw = TBL ? Real(1) : w0;
  Real ct = Real(0), ctl = Real(0);   // FP32: tau + a + b as an exact pair
  if constexpr (!TBL) {
    ct = A.cth[slot];
    ctl = A.ctl[slot];
  }
  const Real tau = A.tau * iw;
  const int strip = warp * NG + g;
  const int row0 = blk * A.rows_per_blk + strip * TH;     // sweep-order first row of the strip
  const int ntile = (nx + TW - 1) / TW;
  const Real gx = TBL ? A.gx[quad] * w0 : A.gx[quad], gy = TBL ? A.gy[quad] * w0 : A.gy[quad];

  unsigned char* wbase = smraw + (size_t)warp * C::WARP_BYTES;
  Real* rings = reinterpret_cast<Real*>(smraw + (size_t)W * C::WARP_BYTES);
  const Real* ring_in = warp > 0 ? rings + (size_t)(warp - 1) * C::RING_REALS : nullptr;
  Real* ring_out = warp < W - 1 ? rings + (size_t)warp * C::RING_REALS : nullptr;
  Real* f_fam = (MB == 1 && !BF) ? A.f + (size_t)fam * ncell * DL : nullptr;
  const unsigned char* tab_fam =
      TBL ? reinterpret_cast<const unsigned char*>(A.inv_d + (size_t)fam * ncell * DL) : nullptr;
  __nv_bfloat16* fb_fam = (MB == 1 && BF) ? A.fb + (size_t)fam * ncell * DL : nullptr;
  const unsigned char* fsrc = nullptr;
  if constexpr (MB != 0) {
    fsrc = BF ? reinterpret_cast<const unsigned char*>(A.fb + (size_t)fam * ncell * DL)
              : reinterpret_cast<const unsigned char*>(A.f + (size_t)fam * ncell * DL);
  }
  const bool has_up = blk > 0;
  const bool has_down = blk + 1 < A.nblk;
  const size_t plane = (size_t)A.nfam * A.nblk * nx * DL;
  const Real* edge_in = A.edge + ((size_t)(fam * A.nblk + (has_up ? blk - 1 : 0)) * nx) * DL;
  Real* edge_out = A.edge + ((size_t)(fam * A.nblk + blk) * nx) * DL;
  unsigned* flag_in = &A.ctrl->flags[fam * A.nblk + (has_up ? blk - 1 : 0)];
  unsigned* flag_out = &A.ctrl->flags[fam * A.nblk + blk];

  auto phys = [&](int x, int y) -> long {
    return (long)(ypos ? y : ny - 1 - y) * nx + (xpos ? x : nx - 1 - x);
  };
  auto group_buf = [&](int buf) -> unsigned char* {
    return wbase + (size_t)(buf * NG + g) * C::GROUP_BYTES;
  };
  // cp.async the inputs of tile t of this group's strip into buffer buf.
  auto stage = [&](int t, int buf) {
    if (t >= 0 && t < ntile) {
      Real* arr = reinterpret_cast<Real*>(group_buf(buf));
      for (int e = dl; e < C::NARR * C::CELLS; e += DL) {
        const int a = e / C::CELLS, c = e % C::CELLS;
        const int x = t * TW + c % TW, y = row0 + c / TW;
        const bool ok = x < nx && y < ny;
        const long cell = ok ? phys(x, y) : 0;
        const Real* src;
        if constexpr (BF) {
          src = a == C::A_ST ? A.sig_t
              : a == C::A_STL ? A.sig_tl
              : (MB != 2 && a == C::A_Q) ? A.q
              : (MB != 0 && a == C::A_G2) ? A.g2
              : a == C::A_FRO ? A.fro
              : A.frn;
        } else if constexpr (TBL) {
          src = (MB != 2 && a == C::A_Q) ? A.q : A.g2;
        } else {
          src = a == C::A_ST ? A.sig_t
              : a == C::A_STL ? A.sig_tl
              : (MB != 2 && a == C::A_Q) ? A.q
              : A.g2;
        }
        cp_async(arr + e, src + cell, ok && src != nullptr);
      }
      if constexpr (TBL) {
        unsigned char* tdst = group_buf(buf) + C::NARR * C::CELLS * C::RS + C::F_BYTES;
        for (int e = dl; e < C::CELLS * C::TP; e += DL) {
          const int c = e / C::TP, v = e % C::TP;
          const int x = t * TW + c % TW, y = row0 + c / TW;
          const bool ok = x < nx && y < ny;
          const long cell = ok ? phys(x, y) : 0;
          cp_async_16(tdst + (size_t)e * 16, tab_fam + ((size_t)cell * DL * C::RS + v * 16), ok);
        }
      }
      if constexpr (MB != 0) {
        unsigned char* fdst = group_buf(buf) + C::NARR * C::CELLS * C::RS;
        for (int e = dl; e < C::CELLS * C::FP; e += DL) {
          const int c = e / C::FP, v = e % C::FP;
          const int x = t * TW + c % TW, y = row0 + c / TW;
          const bool ok = x < nx && y < ny;
          const long cell = ok ? phys(x, y) : 0;
          cp_async_16(fdst + (size_t)e * 16, fsrc + ((size_t)cell * DL * C::ESZ + v * 16), ok);
        }
      }
    }
    cp_async_commit();
  };

  Real yA[TW], yB[TW];   // row above the next row to solve (after a tile: its bottom row)
  Real xA[TH], xB[TH];   // left column of the next tile (after a tile: its right column)
#pragma unroll
  for (int i = 0; i < TW; ++i) yA[i] = yB[i] = Real(0);
#pragma unroll
  for (int j = 0; j < TH; ++j) {
    xA[j] = gx;
    xB[j] = Real(0);
  }

  const int nstep = ntile + NG - 1;
  stage(-g, 0);
  for (int T = 0; T < nstep; ++T) {
    const int t = T - g;
    const bool active = t >= 0 && t < ntile;
    const int buf = T & 1;
    cp_async_wait0();
    __syncwarp();
    stage(t + 1, buf ^ 1);
    // the row above this tile: from the group above (shuffle); group 0 from the warp above
    // (ring), the CTA above (global edge) or the inflow ghost
    Real upA[TW], upB[TW];
#pragma unroll
    for (int i = 0; i < TW; ++i) {
      upA[i] = __shfl_up_sync(FULL, yA[i], DL);
      upB[i] = (MB == 1) ? __shfl_up_sync(FULL, yB[i], DL) : Real(0);
    }
    if (warp > 0) {
      // group 0 works on tile T; wait until the warp above has put that tile in the ring
      if (T < ntile) {
        if (g == 0) {
          // every lane of group 0 polls (one broadcast read per poll) and fences for itself,
          // so no warp barrier hands the value on before the ring reads
          unsigned spins = 0;
          while (s_prod[warp - 1] <= T && !s_abandon) {
            if (++spins > SMEM_SPIN_LIMIT) {
              if (dl == 0) atomicExch(&A.ctrl->err, 1u);
              s_abandon = 1;
              break;
            }
          }
          __threadfence_block();
          const Real* rs = ring_in + (size_t)(T % RD) * TW * DL + dl;
#pragma unroll
          for (int i = 0; i < TW; ++i) {
            upA[i] = rs[i * DL];
            if constexpr (MB == 1) upB[i] = rs[(size_t)RD * TW * DL + i * DL];
          }
        }
        __syncwarp();
        if (lane == 0) s_cons[warp] = T + 1;   // ring slot of tile T may be reused
      }
    } else if (g == 0) {
      if (has_up) {
        if (T < ntile) {
          // every lane of the group acquires the flag itself, so its edge loads are ordered
          // after its own acquire (no group barrier or fence)
          if (!s_abandon) {
            unsigned spins = 0;
            while (ld_acquire(flag_in) < (unsigned)(T + 1)) {
              if (++spins > SPIN_LIMIT || ld_acquire(&A.ctrl->err) != 0u) {
                if (dl == 0) atomicExch(&A.ctrl->err, 1u);
                s_abandon = 1;
                break;
              }
              if (spins > 256) __nanosleep(64);
            }
          }
#pragma unroll
          for (int i = 0; i < TW; ++i) {
            const int x = T * TW + i;
            upA[i] = x < nx ? ldcg(edge_in + (size_t)x * DL + dl) : Real(0);
            if constexpr (MB == 1)
              upB[i] = x < nx ? ldcg(edge_in + plane + (size_t)x * DL + dl) : Real(0);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < TW; ++i) {
          upA[i] = gy;
          upB[i] = Real(0);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < TW; ++i) {
      yA[i] = upA[i];
      yB[i] = upB[i];
    }
    if (t == 0) {
#pragma unroll
      for (int j = 0; j < TH; ++j) {
        xA[j] = gx;
        xB[j] = Real(0);
      }
    }
    if constexpr (MB == 1) {
      // fused sweep: row by row (its two recurrences already give two independent chains,
      // and holding the whole tile of both passes would double the registers)
      const Real* arr = reinterpret_cast<const Real*>(group_buf(buf));
      const unsigned char* fb = group_buf(buf) + C::NARR * C::CELLS * C::RS;
      const Real* tab = reinterpret_cast<const Real*>(fb + C::F_BYTES);
  #pragma unroll
      for (int j = 0; j < TH; ++j) {
        const int y = row0 + j;
        Real mv[TW];
  #pragma unroll
        for (int i = 0; i < TW; ++i) {
          const int c = j * TW + i;
          Real dh, dlo;
          diag<TBL>(ct, ctl, arr, tab, c, dl, C::CELLS, DL, dh, dlo);
          const Real leftA = (i == 0) ? xA[j] : yA[i - 1];
          Real fo = Real(0);
          if constexpr (MB != 0) {
            if constexpr (BF)
              fo = arr[C::A_FRO * C::CELLS + c] +
                   __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(fb)[c * DL + dl]);
            else
              fo = reinterpret_cast<const Real*>(fb)[c * DL + dl];
          }
          Real srcA;
          if constexpr (MB == 0) srcA = arr[C::A_Q * C::CELLS + c];
          else if constexpr (MB == 2) srcA = arr[C::A_G2 * C::CELLS + c] + tau * fo;
          else srcA = arr[C::A_Q * C::CELLS + c] + tau * fo;
          // yA[i - 1] is already this row's value: the left neighbour; yA[i] is still the row above
          const Real va = scale2(srcA + ca * leftA + cb * yA[i], dh, dlo);
          if constexpr (MB == 1) {
            const int x = t * TW + i;
            const bool store = active && x < nx && y < ny;
            Real vst;
            if constexpr (BF) {
              const long cell = phys(x < nx ? x : 0, y < ny ? y : 0);
              const __nv_bfloat16 rb = bf16_stochastic(va - arr[C::A_FRN * C::CELLS + c],
                                                       (unsigned)(cell * A.nslot + slot), A.seed);
              if (store) fb_fam[(size_t)cell * DL + dl] = rb;
              vst = arr[C::A_FRN * C::CELLS + c] + __bfloat162float(rb);
            } else {
              if (store) f_fam[(size_t)phys(x, y) * DL + dl] = va;
              vst = va;
            }
            const Real leftB = (i == 0) ? xB[j] : yB[i - 1];
            const Real vb =
                scale2(arr[C::A_G2 * C::CELLS + c] + tau * vst + ca * leftB + cb * yB[i], dh, dlo);
            yB[i] = vb;
            mv[i] = cw * vb;
          } else {
            mv[i] = cw * va;
          }
          yA[i] = va;
        }
        xA[j] = yA[TW - 1];
        if constexpr (MB == 1) xB[j] = yB[TW - 1];
        // quadrature moment of row j over the group's directions: one partial per family and cell
        TReduce<Real, TW, DL / 2>::run(mv, dl);
        int idx;
        bool writer;
        if constexpr (TW >= DL) {
          idx = dl;
          writer = true;
        } else {
          idx = dl / (DL / TW);
          writer = (dl & (DL / TW - 1)) == 0;
        }
        const int x = t * TW + idx;
        if (writer && active && x < nx && y < ny) A.pm[fam * ncell + phys(x, y)] = mv[0];
      }
    } else {
      // single recurrence (SI sweep, y sweep): anti-diagonal by anti-diagonal, so that the up
      // to TH cells of a diagonal are independent and the dependent FMA chain of the recurrence
      // overlaps across them; the moment of the whole tile in one transpose-reduce at the end
      const Real* arr = reinterpret_cast<const Real*>(group_buf(buf));
      const unsigned char* fb = group_buf(buf) + C::NARR * C::CELLS * C::RS;
      const Real* tab = reinterpret_cast<const Real*>(fb + C::F_BYTES);
      Real vA[TH][TW];
  #pragma unroll
      for (int dg = 0; dg < TW + TH - 1; ++dg) {
  #pragma unroll
        for (int j = 0; j < TH; ++j) {
          const int i = dg - j;
          if (i < 0 || i >= TW) continue;
          const int c = j * TW + i;
          Real dh, dlo;
          diag<TBL>(ct, ctl, arr, tab, c, dl, C::CELLS, DL, dh, dlo);
          const Real left = (i == 0) ? xA[j] : vA[j][i > 0 ? i - 1 : 0];
          const Real up = (j == 0) ? yA[i] : vA[j > 0 ? j - 1 : 0][i];
          Real src;
          if constexpr (MB == 0) {
            src = arr[C::A_Q * C::CELLS + c];
          } else {
            Real fo;
            if constexpr (BF)
              fo = arr[C::A_FRO * C::CELLS + c] +
                   __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(fb)[c * DL + dl]);
            else
              fo = reinterpret_cast<const Real*>(fb)[c * DL + dl];
            src = arr[C::A_G2 * C::CELLS + c] + tau * fo;
          }
          vA[j][i] = scale2(src + ca * left + cb * up, dh, dlo);
        }
      }
  #pragma unroll
      for (int j = 0; j < TH; ++j) xA[j] = vA[j][TW - 1];
  #pragma unroll
      for (int i = 0; i < TW; ++i) yA[i] = vA[TH - 1][i];
      {
        constexpr int NV = TH * TW;
        Real mv[NV];
  #pragma unroll
        for (int c = 0; c < NV; ++c) mv[c] = cw * vA[c / TW][c % TW];
        TReduce<Real, NV, DL / 2>::run(mv, dl);
        constexpr int PER = NV >= DL ? NV / DL : 1;
  #pragma unroll
        for (int q = 0; q < PER; ++q) {
          int idx;
          bool writer;
          if constexpr (NV >= DL) {
            idx = dl * PER + q;
            writer = true;
          } else {
            idx = dl / (DL / NV);
            writer = (dl & (DL / NV - 1)) == 0;
          }
          const int x = t * TW + idx % TW, y = row0 + idx / TW;
          if (writer && active && x < nx && y < ny) A.pm[fam * ncell + phys(x, y)] = mv[q];
        }
      }
    }
    // the bottom row of this tile: to the warp below (ring) or the next CTA (edge)
    const int tl = T - (NG - 1);   // the last group's tile
    if (tl >= 0 && tl < ntile) {
      if (warp < W - 1) {
        if (tl - RD >= 0) {
          int kc = 0;
          if (lane == 0) {
            unsigned spins = 0;
            while ((kc = s_cons[warp + 1]) <= tl - RD && !s_abandon) {
              if (++spins > SMEM_SPIN_LIMIT) {
                atomicExch(&A.ctrl->err, 1u);
                s_abandon = 1;
                break;
              }
            }
          }
          __syncwarp();
        }
        if (g == NG - 1) {
          Real* rs = ring_out + (size_t)(tl % RD) * TW * DL + dl;
#pragma unroll
          for (int i = 0; i < TW; ++i) {
            rs[i * DL] = yA[i];
            if constexpr (MB == 1) rs[(size_t)RD * TW * DL + i * DL] = yB[i];
          }
        }
        __syncwarp();
        __threadfence_block();
        if (lane == 0) s_prod[warp] = tl + 1;
      } else if (has_down) {
        if (g == NG - 1) {
#pragma unroll
          for (int i = 0; i < TW; ++i) {
            const int x = tl * TW + i;
            if (x < nx) {
              edge_out[(size_t)x * DL + dl] = yA[i];
              if constexpr (MB == 1) edge_out[plane + (size_t)x * DL + dl] = yB[i];
            }
          }
        }
        // the warp barrier orders the group's edge stores before lane 0's release store
        __syncwarp();
        if (lane == 0) st_release(flag_out, (unsigned)(tl + 1));
      }
    }
  }
  cp_async_wait0();
  // Self-reset of the control block by the last CTA to finish.
  __syncthreads();
  if (tid == 0) {
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

template <class Real, int DL, int TH, int MODE>
size_t tile_smem(int W) {
  using C = TileCfg<Real, DL, TH, MODE>;
  return (size_t)W * C::WARP_BYTES + (size_t)(W > 1 ? W - 1 : 0) * C::RING_REALS * sizeof(Real);
}

template <class Real, int DL, int TH, int MODE>
cudaError_t launch_tile(const Sweep2DArgs<Real>& a, int W, cudaStream_t s) {
  constexpr int NG = 32 / DL;
  if (W < 1 || W > 8 || a.rows_per_blk != W * NG * TH) return cudaErrorInvalidValue;
  if (sizeof(Real) == 8 && a.inv_d == nullptr) return cudaErrorInvalidValue;
  const size_t smem = tile_smem<Real, DL, TH, MODE>(W);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  static std::atomic<bool> attr_set{false};   // host threads of a batch share it
  if (!attr_set.load()) {
    cudaError_t e = cudaFuncSetAttribute(sweep2d_tile_kernel<Real, DL, TH, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  ++g_launches;
  sweep2d_tile_kernel<Real, DL, TH, MODE><<<(unsigned)(a.nfam * a.nblk), 32 * W, smem, s>>>(a);
  return cudaGetLastError();
}

template <class Real, int MODE>
cudaError_t launch_tile_mode(const Sweep2DArgs<Real>& a, int dl, int th, int W, cudaStream_t s) {
  if constexpr (sizeof(Real) == 4) {   // two-row tiles: FP32 only
    if (th == 2) {
      if (dl == 8) return launch_tile<Real, 8, 2, MODE>(a, W, s);
      if (dl == 16) return launch_tile<Real, 16, 2, MODE>(a, W, s);
      if (dl == 32) return launch_tile<Real, 32, 2, MODE>(a, W, s);
    }
  }
  if (th == 4) {
    if (dl == 8) return launch_tile<Real, 8, 4, MODE>(a, W, s);
    if (dl == 16) return launch_tile<Real, 16, 4, MODE>(a, W, s);
    if (dl == 32) return launch_tile<Real, 32, 4, MODE>(a, W, s);
  } else if (th == 8) {
    if (dl == 8) return launch_tile<Real, 8, 8, MODE>(a, W, s);
    if (dl == 16) return launch_tile<Real, 16, 8, MODE>(a, W, s);
    if (dl == 32) return launch_tile<Real, 32, 8, MODE>(a, W, s);
  }
  return cudaErrorInvalidValue;
}

template <class Real, int MODE>
size_t tile_smem_mode(int dl, int th, int W) {
  if constexpr (sizeof(Real) == 4) {
    if (th == 2) {
      if (dl == 8) return tile_smem<Real, 8, 2, MODE>(W);
      if (dl == 16) return tile_smem<Real, 16, 2, MODE>(W);
      if (dl == 32) return tile_smem<Real, 32, 2, MODE>(W);
    }
  }
  if (th == 4) {
    if (dl == 8) return tile_smem<Real, 8, 4, MODE>(W);
    if (dl == 16) return tile_smem<Real, 16, 4, MODE>(W);
    if (dl == 32) return tile_smem<Real, 32, 4, MODE>(W);
  } else if (th == 8) {
    if (dl == 8) return tile_smem<Real, 8, 8, MODE>(W);
    if (dl == 16) return tile_smem<Real, 16, 8, MODE>(W);
    if (dl == 32) return tile_smem<Real, 32, 8, MODE>(W);
  }
  return ~(size_t)0;
}

}  // namespace

#ifndef RTE_TILE_PART
#define RTE_TILE_PART -1
#endif

// One translation unit per precision and mode, compiled in parallel (parts 0-4: FP32 modes
// 0-4, parts 5-7: FP64 modes 0-2); the dispatchers sit in part 0.
template <class Real, int MODE>
cudaError_t launch_tile_part(const Sweep2DArgs<Real>& a, int dl, int th, int W, cudaStream_t s);
template <class Real, int MODE>
size_t tile_smem_part(int dl, int th, int W);

#define RTE_TILE_INST(REAL, MODE)                                                            \
  template <>                                                                                \
  cudaError_t launch_tile_part<REAL, MODE>(const Sweep2DArgs<REAL>& a, int dl, int th, int W, \
                                           cudaStream_t s) {                                 \
    return launch_tile_mode<REAL, MODE>(a, dl, th, W, s);                                    \
  }                                                                                          \
  template <>                                                                                \
  size_t tile_smem_part<REAL, MODE>(int dl, int th, int W) {                                 \
    return tile_smem_mode<REAL, MODE>(dl, th, W);                                            \
  }
#define RTE_TILE_DECL(REAL, MODE)                                                            \
  template <>                                                                                \
  cudaError_t launch_tile_part<REAL, MODE>(const Sweep2DArgs<REAL>& a, int dl, int th, int W, \
                                           cudaStream_t s);                                  \
  template <>                                                                                \
  size_t tile_smem_part<REAL, MODE>(int dl, int th, int W);

#if RTE_TILE_PART == -1 || RTE_TILE_PART == 0
RTE_TILE_INST(float, 0)
#else
RTE_TILE_DECL(float, 0)
#endif
#if RTE_TILE_PART == -1 || RTE_TILE_PART == 1
RTE_TILE_INST(float, 1)
#else
RTE_TILE_DECL(float, 1)
#endif
#if RTE_TILE_PART == -1 || RTE_TILE_PART == 2
RTE_TILE_INST(float, 2)
#else
RTE_TILE_DECL(float, 2)
#endif
#if RTE_TILE_PART == -1 || RTE_TILE_PART == 3
RTE_TILE_INST(float, 3)
#else
RTE_TILE_DECL(float, 3)
#endif
#if RTE_TILE_PART == -1 || RTE_TILE_PART == 4
RTE_TILE_INST(float, 4)
#else
RTE_TILE_DECL(float, 4)
#endif
#if RTE_TILE_PART == -1 || RTE_TILE_PART == 5
RTE_TILE_INST(double, 0)
#else
RTE_TILE_DECL(double, 0)
#endif
#if RTE_TILE_PART == -1 || RTE_TILE_PART == 6
RTE_TILE_INST(double, 1)
#else
RTE_TILE_DECL(double, 1)
#endif
#if RTE_TILE_PART == -1 || RTE_TILE_PART == 7
RTE_TILE_INST(double, 2)
#else
RTE_TILE_DECL(double, 2)
#endif

#if RTE_TILE_PART == -1 || RTE_TILE_PART == 0
cudaError_t launch_sweep2d_tile(const Sweep2DArgs<float>& a, int mode, int th, int W,
                                cudaStream_t s) {
  const int dl = a.nslot / a.nfam;
  switch (mode) {
    case 0: return launch_tile_part<float, 0>(a, dl, th, W, s);
    case 1: return launch_tile_part<float, 1>(a, dl, th, W, s);
    case 2: return launch_tile_part<float, 2>(a, dl, th, W, s);
    case 3: return launch_tile_part<float, 3>(a, dl, th, W, s);
    case 4: return launch_tile_part<float, 4>(a, dl, th, W, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sweep2d_tile(const Sweep2DArgs<double>& a, int mode, int th, int W,
                                cudaStream_t s) {
  const int dl = a.nslot / a.nfam;
  switch (mode) {
    case 0: return launch_tile_part<double, 0>(a, dl, th, W, s);
    case 1: return launch_tile_part<double, 1>(a, dl, th, W, s);
    case 2: return launch_tile_part<double, 2>(a, dl, th, W, s);
    default: return cudaErrorInvalidValue;
  }
}

size_t sweep2d_tile_smem_bytes(size_t real, int dl, int th, int W, int mode) {
  if (real == sizeof(double)) {
    switch (mode) {
      case 0: return tile_smem_part<double, 0>(dl, th, W);
      case 1: return tile_smem_part<double, 1>(dl, th, W);
      case 2: return tile_smem_part<double, 2>(dl, th, W);
      default: return ~(size_t)0;
    }
  }
  switch (mode) {
    case 0: return tile_smem_part<float, 0>(dl, th, W);
    case 1: return tile_smem_part<float, 1>(dl, th, W);
    case 2: return tile_smem_part<float, 2>(dl, th, W);
    case 3: return tile_smem_part<float, 3>(dl, th, W);
    case 4: return tile_smem_part<float, 4>(dl, th, W);
    default: return ~(size_t)0;
  }
}
#endif

}  // namespace rte
