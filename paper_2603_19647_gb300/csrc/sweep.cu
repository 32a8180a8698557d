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
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>

#include "rte_internal.h"
#include "sweep_common.cuh"

namespace rte {

namespace {
using namespace sweep_detail;

constexpr int KCHUNK = 8;            // columns per published edge chunk

// MODE 0: SI sweep (K1): S = q with the given inflow ghosts (zero for SI), moment of psi.
// MODE 2: y = L^-1(g2 + tau f) from the stored f, zero inflow, moment of y.
// MODE 1: fused f sweep (K2): pass A  f^n = L^-1(q + tau f^{n-1}) with inflow ghosts,
//         pass B  y = L^-1(g2 + tau f^n) with zero inflow; moment of B (and of A).
//
// CTA = W warps stacked vertically, each a pipeline stage: warp w owns RW = NG R rows and
// works through the columns in chunks of K.  The bottom row of warp w-1 is handed to warp w
// step by step through a shared ring: the producer bumps a shared progress counter after
// every column, the consumer re-reads it (bounded spin) only when its cached copy says the
// column is not there yet, and reports how far it has read once per chunk so the producer
// may reuse ring slots.  Each warp stages the per-cell data of its next chunk into its own
// shared buffers with cp.async while it computes the current one.  Warp 0 takes its top row
// from the CTA above through global memory behind a release flag, a chunk at a time.  No
// CTA-wide barrier runs inside the column loop.
template <class Real, int DL, int R, int K, int MODE, bool TABLE>
__global__ void __launch_bounds__(256) sweep2d_kernel(const Sweep2DArgs<Real> A) {
  // MODE 3 / 4: MODE 1 / 2 with f stored as a BF16 remainder about a per-cell FP32 reference
  constexpr bool BF = MODE >= 3;
  constexpr int MB = BF ? MODE - 2 : MODE;
  static_assert(!BF || sizeof(Real) == 4, "BF16 storage of f goes with FP32 sweeps");
  constexpr int NG = 32 / DL;
  constexpr int RW = NG * R;
  constexpr int RING = 4 * K;
  constexpr int NP = (MB == 1) ? 2 : 1;              // planes (recurrences) carried
  constexpr bool STAGE_F = MB != 0;
  constexpr int V = DL * (int)sizeof(Real) / 16;     // 16-byte pieces per cell of a family
  constexpr int VB = DL * 2 / 16;                    // the same for BF16 values
  constexpr int PER_DL = (TABLE ? 1 : 0) + (STAGE_F ? 1 : 0);              // [RW][K][DL] arrays
  constexpr int PER_S =
      (TABLE ? 0 : 2) + (MB != 2 ? 1 : 0) + (MB != 0 ? 1 : 0) + (BF ? 2 : 0);  // [RW][K]
  constexpr int WARP_REALS = 2 * RW * K * (PER_DL * DL + PER_S);
  static_assert(R <= DL, "rows per lane group must not exceed the lane count");
  if (A.skip && *A.skip) return;   // before the ticket: the control block stays untouched
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ unsigned s_ticket;
  __shared__ volatile int s_prod[8];    // columns of its bottom row warp w has put in the ring
  __shared__ volatile int s_cons[8];    // columns of the ring above warp w has consumed
  __shared__ volatile int s_abandon;

  const int W = blockDim.x >> 5;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gi = lane / DL, dl = lane % DL;
  // per-warp staging buffers, then the W-1 rings
  Real* wbuf = reinterpret_cast<Real*>(smraw) + (size_t)warp * WARP_REALS;
  Real* tab_s = wbuf;                                            // [2][RW][K][DL]
  Real* f_s = tab_s + (TABLE ? 2 * RW * K * DL : 0);             // [2][RW][K][DL]
  Real* st_s = f_s + (STAGE_F ? 2 * RW * K * DL : 0);            // [2][RW][K]
  Real* stl_s = st_s + (TABLE ? 0 : 2 * RW * K);                  // [2][RW][K] its low part
  Real* qa_s = stl_s + (TABLE ? 0 : 2 * RW * K);
  Real* g2_s = qa_s + (MB != 2 ? 2 * RW * K : 0);
  Real* fro_s = g2_s + (MB != 0 ? 2 * RW * K : 0);   // BF16 mode: reference of f^{n-1}
  Real* frn_s = fro_s + (BF ? 2 * RW * K : 0);        // BF16 mode: reference of f^n
  __nv_bfloat16* bf_s = reinterpret_cast<__nv_bfloat16*>(f_s);
  Real* rings = reinterpret_cast<Real*>(smraw) + (size_t)W * WARP_REALS;  // [W-1][NP][RING][DL]
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
  const Real ca = A.a[slot], cb = A.b[slot], cw = A.w[slot];
  // tau + a + b of this direction: hi / lo pair in FP32 (exact), one value in FP64
  const Real ct = A.cth ? A.cth[slot] : A.tau + ca + cb;
  const Real ctl = A.ctl ? A.ctl[slot] : Real(0);
  // With the table (FP64) the lane carries w psi, its direction's weighted flux: the table
  // holds w / (tau + sigma_t + a + b), so the recurrence keeps its form with a / w, b / w,
  // tau / w in place of a, b, tau and with inflow ghosts times w, and the quadrature moment
  // is a plain sum over the directions.  Stored f is then w f.  (Padding slots have w = 0
  // and stay zero.)
  const Real iw = TABLE ? (cw != Real(0) ? Real(1) / cw : Real(0)) : Real(1);
  const Real ka = TABLE ? ca * iw : ca, kb = TABLE ? cb * iw : cb;
  const Real ktau = TABLE ? A.tau * iw : A.tau;
  const int wrow0 = blk * A.rows_per_blk + warp * RW;   // first sweep-order row of this warp
  const int row0 = wrow0 + gi * R;                       // lane group's row m = 0
  const Real gx = TABLE ? A.gx[quad] * cw : A.gx[quad];
  const Real gy = TABLE ? A.gy[quad] * cw : A.gy[quad];
  const Real* tab_fam = TABLE ? A.inv_d + (size_t)fam * ncell * DL : nullptr;
  Real* f_fam = (STAGE_F && !BF) ? A.f + (size_t)fam * ncell * DL : nullptr;
  __nv_bfloat16* fb_fam = BF ? A.fb + (size_t)fam * ncell * DL : nullptr;
  Real* ring_in = warp > 0 ? rings + (size_t)(warp - 1) * NP * RING * DL : nullptr;
  Real* ring_out = warp < W - 1 ? rings + (size_t)warp * NP * RING * DL : nullptr;

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
  const int T = nx + RW - 1;              // warp-local steps: row rr handles column t - rr
  const int nchunk = (T + K - 1) / K;

  // Copy this warp's data of chunk c into its buffer c & 1: row rr, step k -> column c K + k - rr.
  // Which pieces a lane copies does not depend on the chunk, so each lane's pieces are
  // described once: the row's first cell, the column offset k - rr, the shared-memory offset in
  // buffer 0 and the offset within the cell's DL values (16-byte pieces of the per-direction
  // arrays; single values of the per-cell arrays).
  struct Piece {
    long row;
    int kr, o, vv;
    bool on;
  };
  constexpr int SW = 16 / (int)sizeof(Real);   // values per 16-byte piece
  constexpr int NPD = (TABLE || (STAGE_F && !BF)) ? (RW * K * V + 31) / 32 : 0;
  constexpr int NPB = BF ? (RW * K * VB + 31) / 32 : 0;
  constexpr int NPS = (RW * K + 31) / 32;
  static_assert(NPD == 0 || (RW * K * V) % 32 == 0, "16-byte pieces fill whole warps");
  static_assert(NPB == 0 || (RW * K * VB) % 32 == 0, "16-byte pieces fill whole warps");
  // piece e of per_cell pieces per cell, unit values per piece; stride: values per (row, step)
  // slot in shared memory (DL for the per-direction arrays, 1 for the per-cell arrays)
  auto describe = [&](int e, int per_cell, int unit, int stride, int count) {
    Piece p;
    const int v = e % per_cell, rk = e / per_cell;
    const int rr = rk / K, k = rk % K;
    const int jj = wrow0 + rr;
    p.on = e < count && jj < ny;
    p.row = (long)(ypos ? jj : ny - 1 - jj) * nx;
    p.kr = k - rr;
    p.o = (rr * K + k) * stride + v * unit;
    p.vv = v * unit;
    return p;
  };
  Piece pd[NPD > 0 ? NPD : 1], pb[NPB > 0 ? NPB : 1], ps[NPS];
#pragma unroll
  for (int i = 0; i < NPD; ++i) pd[i] = describe(lane + 32 * i, V, SW, DL, RW * K * V);
#pragma unroll
  for (int i = 0; i < NPB; ++i) pb[i] = describe(lane + 32 * i, VB, 8, DL, RW * K * VB);
#pragma unroll
  for (int i = 0; i < NPS; ++i) ps[i] = describe(lane + 32 * i, 1, 1, 1, RW * K);
  auto stage = [&](int c) {
    const int buf = c & 1;
    const int cK = c * K;
    auto locate = [&](const Piece& p, bool& ok) -> long {
      const int x = cK + p.kr;
      ok = p.on && x >= 0 && x < nx;
      return ok ? p.row + (xpos ? x : nx - 1 - x) : 0;
    };
#pragma unroll
    for (int i = 0; i < NPD; ++i) {
      bool ok;
      const long cell = locate(pd[i], ok);
      const int o = buf * (RW * K * DL) + pd[i].o;
      const size_t g = (size_t)cell * DL + pd[i].vv;
      if constexpr (TABLE) cp_async_16(tab_s + o, tab_fam + g, ok);
      if constexpr (STAGE_F && !BF) cp_async_16(f_s + o, f_fam + g, ok);
    }
    if constexpr (BF) {
#pragma unroll
      for (int i = 0; i < NPB; ++i) {
        bool ok;
        const long cell = locate(pb[i], ok);
        const int o = buf * (RW * K * DL) + pb[i].o;
        cp_async_16(bf_s + o, fb_fam + (size_t)cell * DL + pb[i].vv, ok);
      }
    }
#pragma unroll
    for (int i = 0; i < NPS; ++i) {
      bool ok;
      const long cell = locate(ps[i], ok);
      if (lane + 32 * i >= RW * K) continue;
      const int o = buf * (RW * K) + ps[i].o;
      if constexpr (!TABLE) {
        cp_async(st_s + o, A.sig_t + cell, ok);
        cp_async(stl_s + o, A.sig_tl + cell, ok && A.sig_tl != nullptr);
      }
      if constexpr (MB != 2) cp_async(qa_s + o, A.q + cell, ok);
      if constexpr (MB != 0) cp_async(g2_s + o, A.g2 + cell, ok);
      if constexpr (BF) {
        cp_async(fro_s + o, A.fro + cell, ok);
        cp_async(frn_s + o, A.frn + cell, ok);
      }
    }
    cp_async_commit();
  };

  int known_prod = 0;   // lower bound of s_prod[warp - 1] seen by this warp
  int known_cons = 0;   // lower bound of s_cons[warp + 1] seen by this warp

  stage(0);
  for (int c = 0; c < nchunk; ++c) {
    cp_async_wait0();
    __syncwarp();                       // chunk c's staged data is visible to the warp
    if (c + 1 < nchunk) stage(c + 1);   // buffer (c+1)&1 was last read in chunk c-1
    const int buf = c & 1;
    const int tb = c * K;
    // Top row input for columns [tb, tb + K): lane group 0, row 0 handles column t at step t.
    Real ebA[K], ebB[K];
    Real mb[K * R];   // unweighted cell values of this chunk, reduced at its end
    const int need = min(tb + K, nx);
    if (warp == 0) {
      if (has_up && tb < nx) {
        // every lane acquires the flag itself (one broadcast read per poll), so its edge loads
        // are ordered after its own acquire: no warp barrier or fence on the CTA's head warp
        if (!s_abandon) {
          unsigned spins = 0;
          while (ld_acquire(flag_in) < (unsigned)need) {
            if (++spins > SPIN_LIMIT || ld_acquire(&A.ctrl->err) != 0u) {
              if (lane == 0) atomicExch(&A.ctrl->err, 1u);
              s_abandon = 1;
              break;
            }
            if (spins > 256) __nanosleep(64);
          }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int x = tb + k;
          ebA[k] = (gi == 0 && x < nx) ? ldcg(edge_in + (size_t)x * DL + dl) : Real(0);
          if constexpr (MB == 1)
            ebB[k] = (gi == 0 && x < nx) ? ldcg(edge_in + plane + (size_t)x * DL + dl) : Real(0);
          else
            ebB[k] = Real(0);
        }
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          ebA[k] = gy;
          ebB[k] = Real(0);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int t = tb + k;
      Real upA = __shfl_up_sync(FULL, psA[R - 1], DL);
      Real upB = Real(0);
      if constexpr (MB == 1) upB = __shfl_up_sync(FULL, psB[R - 1], DL);
      if (warp > 0 && t < nx) {
        // column t of the warp above's bottom row, handed over step by step
        if (known_prod <= t) {
          // every lane polls (one broadcast read per poll), so no shuffle hands the value on
          int kp;
          unsigned spins = 0;
          while ((kp = s_prod[warp - 1]) <= t && !s_abandon) {
            if (++spins > SMEM_SPIN_LIMIT) {
              if (lane == 0) atomicExch(&A.ctrl->err, 1u);
              s_abandon = 1;
              break;
            }
          }
          known_prod = kp;
          __threadfence_block();
        }
        const int rs = (t % RING) * DL + dl;
        ebA[k] = ring_in[rs];
        if constexpr (MB == 1) ebB[k] = ring_in[RING * DL + rs];
        if (k == K - 1 || t == nx - 1) {
          __syncwarp();
          if (lane == 0) s_cons[warp] = t + 1;   // ring slots of columns <= t may be reused
        }
      }
      if (gi == 0) {
        upA = ebA[k];
        upB = ebB[k];
      }
#pragma unroll
      for (int m = R - 1; m >= 0; --m) {
        const int x = t - m - gi * R;
        const int jj = row0 + m;
        mb[k * R + m] = Real(0);
        if (x >= 0 && x < nx && jj < ny) {
          const int rr = gi * R + m;
          const int o = (buf * RW + rr) * K + k;
          const int od = o * DL + dl;
          Real dinv, dinvl = Real(0);
          if constexpr (TABLE) {
            dinv = tab_s[od];
          } else if constexpr (sizeof(Real) == 4) {
            const Rcp2 rp = rcp_pair(ct, ctl, st_s[o], stl_s[o]);
            dinv = rp.h;
            dinvl = rp.l;
          } else {
            dinv = recip(ct + st_s[o]);
          }
          const Real uA = (m == 0) ? upA : psA[m > 0 ? m - 1 : 0];
          if constexpr (MB == 0) {
            const Real v = scale2(qa_s[o] + ka * psA[m] + kb * uA, dinv, dinvl);
            psA[m] = v;
            mb[k * R + m] = v;
          } else if constexpr (MB == 2) {
            Real fo;
            if constexpr (BF) fo = fro_s[o] + __bfloat162float(bf_s[od]);
            else fo = f_s[od];
            const Real v = scale2(g2_s[o] + ktau * fo + ka * psA[m] + kb * uA, dinv, dinvl);
            psA[m] = v;
            mb[k * R + m] = v;
          } else {
            Real fo;
            if constexpr (BF) fo = fro_s[o] + __bfloat162float(bf_s[od]);
            else fo = f_s[od];
            const Real va = scale2(qa_s[o] + ktau * fo + ka * psA[m] + kb * uA, dinv, dinvl);
            psA[m] = va;
            const int px = xpos ? x : nx - 1 - x;
            const int py = ypos ? jj : ny - 1 - jj;
            // f^n as stored: exactly in FP32 / FP64, as reference + BF16(f^n - reference) in
            // BF16 mode; pass B sweeps the stored value, so the next step's b~ matches f^n
            Real vst;
            if constexpr (BF) {
              const __nv_bfloat16 rb =
                  bf16_stochastic(va - frn_s[o], (unsigned)(((long)py * nx + px) * A.nslot + slot),
                                  A.seed);
              fb_fam[((long)py * nx + px) * DL + dl] = rb;
              vst = frn_s[o] + __bfloat162float(rb);
            } else {
              f_fam[((long)py * nx + px) * DL + dl] = va;
              vst = va;
            }
            const Real uB = (m == 0) ? upB : psB[m > 0 ? m - 1 : 0];
            const Real vb = scale2(g2_s[o] + ktau * vst + ka * psB[m] + kb * uB, dinv, dinvl);
            psB[m] = vb;
            mb[k * R + m] = vb;
          }
        }
      }
      // bottom row of this warp: to the warp below (shared ring) or the next CTA (global)
      const int xb = t - (RW - 1);
      if (xb >= 0 && xb < nx) {
        if (warp < W - 1) {
          // slot of column xb - RING must have been read by the warp below
          if (xb - RING >= known_cons) {
            int kc = 0;
            if (lane == 0) {
              unsigned spins = 0;
              while ((kc = s_cons[warp + 1]) <= xb - RING && !s_abandon) {
                if (++spins > SMEM_SPIN_LIMIT) {
                  atomicExch(&A.ctrl->err, 1u);
                  s_abandon = 1;
                  break;
                }
              }
            }
            known_cons = __shfl_sync(FULL, kc, 0);
          }
          if (gi == NG - 1) {
            const int rs = (xb % RING) * DL + dl;
            ring_out[rs] = psA[R - 1];
            if constexpr (MB == 1) ring_out[RING * DL + rs] = psB[R - 1];
          }
          __syncwarp();
          __threadfence_block();
          if (lane == 0) s_prod[warp] = xb + 1;
        } else if (has_down && gi == NG - 1) {
          edge_out[(size_t)xb * DL + dl] = psA[R - 1];
          if constexpr (MB == 1) edge_out[plane + (size_t)xb * DL + dl] = psB[R - 1];
        }
      }
    }
    // Quadrature moment of the chunk: one transpose-reduce over the lane group's directions
    // for all K x R cells (the values already weighted with the table, else the weights
    // applied in its first round); one partial per family and cell.
    {
      constexpr int NV = K * R;
      if constexpr (TABLE)
        TReduce<Real, NV, DL / 2>::run(mb, dl);
      else
        TReduceW<Real, NV, DL / 2>::run(mb, cw, dl);
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
        const int k = idx / R, m = idx % R;
        const int x = tb + k - m - gi * R;
        const int jj = row0 + m;
        if (writer && x >= 0 && x < nx && jj < ny) {
          const int px = xpos ? x : nx - 1 - x;
          const int py = ypos ? jj : ny - 1 - jj;
          A.pm[fam * ncell + (long)py * nx + px] = mb[i];
        }
      }
    }
    // publish the bottom-row columns finished in this chunk
    const int done = min(tb + K - (RW - 1), nx);
    if (done > 0 && warp == W - 1 && has_down) {
      // the warp barrier orders every lane's edge stores before lane 0's release store, whose
      // release semantics then publish them at GPU scope to the acquiring CTA
      __syncwarp();
      if (lane == 0) st_release(flag_out, (unsigned)done);
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

constexpr int KSTEP = 8;   // columns per chunk

}  // namespace

inline size_t sweep2d_smem_bytes_impl(size_t real, int dl, int R, int W, int mode, bool table) {
  const int K = 8;
  const bool bf = mode >= 3;
  const int mb = bf ? mode - 2 : mode;
  const int RW = (32 / dl) * R, np = mb == 1 ? 2 : 1;
  const int per_dl = (table ? 1 : 0) + (mb != 0 ? 1 : 0);
  const int per_s = (table ? 0 : 2) + (mb != 2 ? 1 : 0) + (mb != 0 ? 1 : 0) + (bf ? 2 : 0);
  const size_t warp_reals = (size_t)2 * RW * K * (per_dl * dl + per_s);
  return real * (W * warp_reals + (size_t)(W - 1) * np * 4 * K * dl);
}

namespace {

template <class Real, int DL, int R, int MODE>
cudaError_t launch_dl_r(const Sweep2DArgs<Real>& a, cudaStream_t s) {
  constexpr int NG = 32 / DL;
  constexpr int RW = NG * R;
  const int W = a.rows_per_blk / RW;
  if (W < 1 || W > 8 || W * RW != a.rows_per_blk) return cudaErrorInvalidValue;
  // FP64 takes the diagonal from the inverse table, FP32 forms it by the two-part reciprocal
  constexpr bool table = sizeof(Real) == 8;
  if (table != (a.inv_d != nullptr)) return cudaErrorInvalidValue;
  const size_t smem = sweep2d_smem_bytes_impl(sizeof(Real), DL, R, W, MODE, table);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  auto kern = sweep2d_kernel<Real, DL, R, KSTEP, MODE, table>;
  static std::atomic<bool> attr_set{false};   // host threads of a batch share it
  if (!attr_set.load()) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const dim3 grid((unsigned)(a.nfam * a.nblk));
  ++g_launches;
  kern<<<grid, 32 * W, smem, s>>>(a);
  return cudaGetLastError();
}

template <class Real, int DL, int MODE>
cudaError_t launch_dl(const Sweep2DArgs<Real>& a, int R, cudaStream_t s) {
  switch (R) {
    case 1: return launch_dl_r<Real, DL, 1, MODE>(a, s);
    case 2: return launch_dl_r<Real, DL, 2, MODE>(a, s);
    case 4:
      if constexpr (DL >= 4) return launch_dl_r<Real, DL, 4, MODE>(a, s);
      return cudaErrorInvalidValue;
    case 8:
      if constexpr (DL >= 8) return launch_dl_r<Real, DL, 8, MODE>(a, s);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template <class Real, int MODE>
cudaError_t launch_mode_impl(const Sweep2DArgs<Real>& a, int dl, int R, cudaStream_t s) {
  switch (dl) {
    case 2:   // 2 lanes: FP64 only, 4 lanes: FP64 and FP32 (an FP32 family of 2 lanes, or a
              // BF16 one of 4, is less than one 16-byte piece of a cell)
      if constexpr (sizeof(Real) == 8) return launch_dl<Real, 2, MODE>(a, R, s);
      return cudaErrorInvalidValue;
    case 4:
      if constexpr (sizeof(Real) == 8 || MODE < 3) return launch_dl<Real, 4, MODE>(a, R, s);
      return cudaErrorInvalidValue;
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

// Per-cell coefficient of the 1D recurrence psi_c = (s_c + a psi_{c-1}) / d_c: the reciprocal
// of d_c as a pair (FP32) or a value (FP64), and d_c itself in FP64 for the scan.
template <class Real>
struct Cell1D {
  Real h, l;
  double d;
};
template <class Real>
__device__ __forceinline__ Cell1D<Real> cell1d(Real ct, Real ctl, Real sig, Real sigl) {
  if constexpr (sizeof(Real) == 4) {
    const Rcp2 rp = rcp_pair(ct, ctl, sig, sigl);
    return {rp.h, rp.l, (double)ct + (double)ctl + (double)sig + (double)sigl};
  } else {
    const double d = ct + sig;
    return {Real(1) / d, Real(0), d};
  }
}

// The block scan composes the cells' affine maps in FP64 in both precisions (its products
// of a / d_c are per-direction coefficients, where an FP32 rounding would bias the
// operator); each thread then runs its cells' recurrence in the run precision.
template <class Real, int MODE>
__global__ void __launch_bounds__(SCAN_THREADS) sweep1d_kernel(const Sweep1DArgs<Real> A) {
  if (A.skip && *A.skip) return;
  __shared__ Aff<double> sh[64];
  const int slot = blockIdx.x;
  const int nx = A.nx;
  const int dlh = A.nslot / 2;   // f layout [half-range][cell][direction in half-range]
  const long fbase = (long)(slot / dlh) * nx * dlh + slot % dlh;
  const int chunk = (nx + SCAN_THREADS - 1) / SCAN_THREADS;
  const int k0 = threadIdx.x * chunk;
  const int k1 = min(nx, k0 + chunk);
  const bool pos = A.dir_sign[slot] > 0;
  const Real ca = A.a[slot], cw = A.w[slot];
  const Real ct = A.cth ? A.cth[slot] : A.tau + ca;
  const Real ctl = A.ctl ? A.ctl[slot] : Real(0);
  // pass A (MODE 1) or the only pass (MODE 0)
  Aff<double> mine{1.0, 0.0};
  for (int k = k0; k < k1; ++k) {
    const int c = pos ? k : nx - 1 - k;
    const Cell1D<Real> cc = cell1d(ct, ctl, A.sig_t[c], A.sig_tl ? A.sig_tl[c] : Real(0));
    Real s = (MODE == 2) ? A.g2[c] : A.q[c];
    if (MODE != 0) s += A.tau * A.f[fbase + (long)c * dlh];
    mine = compose(mine, Aff<double>{(double)ca / cc.d, (double)s / cc.d});
  }
  const Real gA = (MODE == 2) ? Real(0) : (pos ? A.g_lo : A.g_hi);
  Real psi = (Real)block_scan_entry(mine, (double)gA, sh);
  for (int k = k0; k < k1; ++k) {
    const int c = pos ? k : nx - 1 - k;
    const Cell1D<Real> cc = cell1d(ct, ctl, A.sig_t[c], A.sig_tl ? A.sig_tl[c] : Real(0));
    Real s = (MODE == 2) ? A.g2[c] : A.q[c];
    if (MODE == 2) {
      s += A.tau * A.f[fbase + (long)c * dlh];
      psi = scale2(s + ca * psi, cc.h, cc.l);
      A.psi_w[(long)slot * nx + c] = cw * psi;
    } else if (MODE == 1) {
      Real* fp = A.f + fbase + (long)c * dlh;
      s += A.tau * (*fp);
      psi = scale2(s + ca * psi, cc.h, cc.l);
      *fp = psi;
      if (A.psi_w_a) A.psi_w_a[(long)slot * nx + c] = cw * psi;
    } else {
      psi = scale2(s + ca * psi, cc.h, cc.l);
      A.psi_w[(long)slot * nx + c] = cw * psi;
    }
  }
  if (MODE == 1) {
    // pass B: y = L^-1 (g2 + tau f^n), zero inflow; this thread reads back its own writes.
    Aff<double> mb{1.0, 0.0};
    for (int k = k0; k < k1; ++k) {
      const int c = pos ? k : nx - 1 - k;
      const Cell1D<Real> cc = cell1d(ct, ctl, A.sig_t[c], A.sig_tl ? A.sig_tl[c] : Real(0));
      const Real s = A.g2[c] + A.tau * A.f[fbase + (long)c * dlh];
      mb = compose(mb, Aff<double>{(double)ca / cc.d, (double)s / cc.d});
    }
    Real y = (Real)block_scan_entry(mb, 0.0, sh);
    for (int k = k0; k < k1; ++k) {
      const int c = pos ? k : nx - 1 - k;
      const Cell1D<Real> cc = cell1d(ct, ctl, A.sig_t[c], A.sig_tl ? A.sig_tl[c] : Real(0));
      const Real s = A.g2[c] + A.tau * A.f[fbase + (long)c * dlh];
      y = scale2(s + ca * y, cc.h, cc.l);
      A.psi_w[(long)slot * nx + c] = cw * y;
    }
  }
}

template <class Real>
__global__ void moment1d_kernel(const Real* psi_w, int nslot, int ncell, Real* out,
                                const unsigned* skip) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell || (skip && *skip)) return;
  Real s = Real(0);
  for (int k = 0; k < nslot; ++k) s += psi_w[(long)k * ncell + c];
  out[c] = s;
}

template <class Real>
__global__ void inv_d_kernel(const Real* sig_t, const Real* a, const Real* b, const Real* w, Real tau,
                             int ncell, int nslot, int dl, Real* inv_d) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)ncell * nslot) return;
  // family layout [fam][cell][dl] with dl = 32 / 16 / 8 lanes: i = (fam * ncell + c) * dl + lane
  const long lanei = i % dl, rest = i / dl;
  const long c = rest % ncell, fam = rest / ncell;
  const int s = (int)(fam * dl + lanei);
  inv_d[i] = w[s] / (tau + sig_t[c] + a[s] + b[s]);
}

}  // namespace

// The 2D kernels are instantiated in eight translation units (precision x mode) so that the
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

#if RTE_SWEEP_PART == -1 || RTE_SWEEP_PART == 7
RTE_SWEEP_INST(7, float, 3)
#endif
#if RTE_SWEEP_PART == -1 || RTE_SWEEP_PART == 8
RTE_SWEEP_INST(8, float, 4)
#endif

#if RTE_SWEEP_PART == -1 || RTE_SWEEP_PART == 6
#if RTE_SWEEP_PART == 6
RTE_SWEEP_EXTERN(double, 0)
RTE_SWEEP_EXTERN(double, 1)
RTE_SWEEP_EXTERN(double, 2)
RTE_SWEEP_EXTERN(float, 0)
RTE_SWEEP_EXTERN(float, 1)
RTE_SWEEP_EXTERN(float, 2)
RTE_SWEEP_EXTERN(float, 3)
RTE_SWEEP_EXTERN(float, 4)
#endif
size_t sweep2d_smem_bytes(size_t real, int dl, int R, int W, int mode, bool table) {
  return sweep2d_smem_bytes_impl(real, dl, R, W, mode, table);
}

template <class Real>
cudaError_t launch_sweep2d(const Sweep2DArgs<Real>& a, int mode, int R, cudaStream_t s) {
  const int dl = a.nslot / a.nfam;
  if (mode == 0) return launch_sweep2d_mode<Real, 0>(a, dl, R, s);
  if (mode == 2) return launch_sweep2d_mode<Real, 2>(a, dl, R, s);
  if (mode == 1) return launch_sweep2d_mode<Real, 1>(a, dl, R, s);
  if constexpr (sizeof(Real) == 4) {
    if (mode == 3) return launch_sweep2d_mode<Real, 3>(a, dl, R, s);
    if (mode == 4) return launch_sweep2d_mode<Real, 4>(a, dl, R, s);
  }
  return cudaErrorInvalidValue;
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
cudaError_t launch_moment1d(const Real* psi_w, int nslot, int ncell, Real* out, cudaStream_t s,
                            const unsigned* skip) {
  ++g_launches;
  moment1d_kernel<Real><<<(ncell + 255) / 256, 256, 0, s>>>(psi_w, nslot, ncell, out, skip);
  return cudaGetLastError();
}

template <class Real>
cudaError_t launch_inv_d(const Real* sig_t, const Real* a, const Real* b, const Real* w, Real tau,
                         int ncell, int nslot, int dl, Real* inv_d, cudaStream_t s) {
  const long n = (long)ncell * nslot;
  ++g_launches;
  inv_d_kernel<Real><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sig_t, a, b, w, tau, ncell,
                                                                 nslot, dl, inv_d);
  return cudaGetLastError();
}

template cudaError_t launch_sweep2d<double>(const Sweep2DArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_sweep2d<float>(const Sweep2DArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_sweep1d<double>(const Sweep1DArgs<double>&, int, cudaStream_t);
template cudaError_t launch_sweep1d<float>(const Sweep1DArgs<float>&, int, cudaStream_t);
template cudaError_t launch_moment1d<double>(const double*, int, int, double*, cudaStream_t,
                                             const unsigned*);
template cudaError_t launch_moment1d<float>(const float*, int, int, float*, cudaStream_t,
                                            const unsigned*);
template cudaError_t launch_inv_d<double>(const double*, const double*, const double*,
                                          const double*, double, int, int, int, double*,
                                          cudaStream_t);
#endif  // base part

}  // namespace rte
