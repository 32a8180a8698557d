// Device helpers shared by the 2D sweep kernels (sweep.cu: strip chain; sweep_tile.cu:
// tile sequence): memory-order primitives for the inter-CTA hand-off, the compensated FP32
// reciprocal, stochastic BF16 rounding, the warp transpose-reduce of the quadrature moment
// and cp.async staging.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace rte {
namespace sweep_detail {

constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned SPIN_LIMIT = 1u << 20;        // global-flag polls (sleeping after the first 256)
constexpr unsigned SMEM_SPIN_LIMIT = 1u << 26;   // shared-counter polls (about a second)

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// 1 / (ch + cl + s + sl) as an unevaluated pair h + l, to about 2^-46 relative, in FP32.
// ch + cl is tau + a + b of the direction and s + sl is sigma_t of the cell, both split
// exactly on the host: the sum is formed exactly (Knuth's TwoSum, then a renormalisation),
// the reciprocal by one Newton correction whose residual 1 - d_h g_h is exact under FMA.
// With it the FP32 sweeps are the exact Q0 operator of the problem up to the FP32 rounding
// of the streaming coefficients a, b (conservative, no per-step bias), not an operator whose
// division is off by an ulp or whose absorption sigma_t - sigma_s is off by an ulp of
// sigma_t (which in a strongly scattering cell is a large error in the absorption).
struct Rcp2 {
  float h, l;
};
__device__ __forceinline__ Rcp2 rcp_pair(float ch, float cl, float s, float sl) {
  const float sum = ch + s;
  const float bb = sum - ch;
  float e = (ch - (sum - bb)) + (s - bb);
  e += cl + sl;
  const float dh = sum + e;
  const float dl = e - (dh - sum);
  const float gh = recip(dh);
  float r = fmaf(-dh, gh, 1.0f);
  r = fmaf(-dl, gh, r);
  return {gh, r * gh};
}
// Unbiased (stochastic) rounding of x to BF16: a uniform 16-bit integer is added below the
// kept bits before truncation, so E[result] = x; it keeps increments far below one BF16 ulp
// from being lost step after step.  The random bits come from a counter-based integer hash
// (the "lowbias32" mixer) of the cell-direction index and a per-launch seed.
__device__ __forceinline__ unsigned hash32(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}
__device__ __forceinline__ __nv_bfloat16 bf16_stochastic(float x, unsigned idx, unsigned seed) {
  unsigned u = __float_as_uint(x);
  if ((u & 0x7f800000u) != 0x7f800000u) u += hash32(idx ^ hash32(seed)) & 0xffffu;
  return __ushort_as_bfloat16((unsigned short)(u >> 16));
}

// t * (h + l): the low part only in FP32 (l = 0 in FP64).
__device__ __forceinline__ float scale2(float t, float h, float l) { return fmaf(t, h, t * l); }
__device__ __forceinline__ double scale2(double t, double h, double) { return t * h; }

template <class Real>
__device__ __forceinline__ Real ldcg(const Real* p) {
  return __ldcg(p);
}

// Transpose-reduce N values over the DL lanes of a lane group.  Each round with offset O
// halves the values a lane keeps (the lane with bit O set keeps the upper half) and adds the
// partner's copy; once one value is left the remaining rounds are plain butterflies.  After
// it, for N >= DL lane dl holds in v[i] (i < N/DL) the group sum of value index
// dl * (N/DL) + i; for N < DL it holds in v[0] the sum of value index dl / (DL/N).
template <class Real, int N, int O>
struct TReduce {
  static __device__ __forceinline__ void run(Real* v, int dl) {
    if constexpr (O == 0) {
      return;
    } else if constexpr (N > 1) {
      const bool hi = (dl & O) != 0;
#pragma unroll
      for (int i = 0; i < N / 2; ++i) {
        const Real send = hi ? v[i] : v[i + N / 2];
        const Real keep = hi ? v[i + N / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL, send, O);
      }
      TReduce<Real, N / 2, O / 2>::run(v, dl);
    } else {
      v[0] += __shfl_xor_sync(FULL, v[0], O);
      TReduce<Real, 1, O / 2>::run(v, dl);
    }
  }
};

// TReduce whose first halving round also applies the weight w of the lane's own direction:
// each lane scales what it sends and what it keeps, so the weights cost N / 2 multiplies and
// N / 2 fused multiply-adds instead of N multiplies before an unweighted reduce.
template <class Real, int N, int O>
struct TReduceW {
  static __device__ __forceinline__ void run(Real* v, Real w, int dl) {
    static_assert(N > 1 && O > 0, "at least one halving round");
    const bool hi = (dl & O) != 0;
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const Real send = w * (hi ? v[i] : v[i + N / 2]);
      const Real keep = hi ? v[i + N / 2] : v[i];
      v[i] = fma(keep, w, __shfl_xor_sync(FULL, send, O));
    }
    TReduce<Real, N / 2, O / 2>::run(v, dl);
  }
};

// cp.async helpers (global -> shared, zero-fill when the source is absent).
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
template <class Real>
__device__ __forceinline__ void cp_async(Real* smem, const Real* gmem, bool valid) {
  if constexpr (sizeof(Real) == 8)
    cp_async_8(smem, gmem, valid);
  else
    cp_async_4(smem, gmem, valid);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }


}  // namespace sweep_detail
}  // namespace rte
