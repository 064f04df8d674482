// Rows of the stored dense inverses of the coarsest level (exact or MG-DD, Sec.
// 4) applied to a vector: shared by the per-colour local-product launches
// (k_dense.cu) and the persistent MG-DD coarsest solve (k_coarse_persist.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"

namespace ehs {

__device__ __forceinline__ float2 ldlp(const float2* p) { return *p; }
__device__ __forceinline__ float2 ldlp(const __half2* p) { return __half22float2(*p); }
__device__ __forceinline__ float2 ldlp(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }

// x[row0 .. row0+3] = (A r)[row0 .. row0+3] for one warp, A stored as N x N
// entries of TI (complex64, FP16 or BF16 pairs; FP32 accumulation) of which the
// leading n x n are live (the rest is identity padding; columns beyond n are
// skipped, rows beyond n are not written).  16-byte loads: every lane keeps
// four matrix loads in flight and reuses each chunk of r for the four rows (E
// entries per load; N a multiple of 4 and of E, so every row starts 16-byte
// aligned).  mat: the matrix, r and x: the item's vectors.  RCG: r is read
// through L2 only (r written earlier by the same launch on other SMs).
// With map (SCATTER), the four results are added to xg[map[row]] instead (rows
// whose map entry is -1 are dropped), read through L2: the scatter-add of an MG-DD
// correction into the coarsest vector.
template <typename TI, bool RCG = false, bool SCATTER = false>
__device__ __forceinline__ void dense_rows4(int N, int n, int row0, const TI* __restrict__ mat,
                                            const float2* __restrict__ r, float2* __restrict__ x,
                                            const int* __restrict__ map = nullptr, float2* xg = nullptr) {
  constexpr int E = 16 / (int)sizeof(TI);
  constexpr int R = 4;
  const int lane = threadIdx.x & 31;
  const int nq = (n + E - 1) / E;                  // 16-byte chunks per live row
  const uint4* m0 = (const uint4*)(mat + (long long)row0 * N);
  const int qs = N / E;                            // chunks per stored row
  const float4* rv = (const float4*)r;
  union U { uint4 u; TI t[E]; };
  float ax[R], ay[R];
#pragma unroll
  for (int k = 0; k < R; ++k) { ax[k] = 0.f; ay[k] = 0.f; }
  for (int q = lane; q < nq; q += 32) {
    U a[R];
#pragma unroll
    for (int k = 0; k < R; ++k) a[k].u = __ldg(m0 + (long long)k * qs + q);
#pragma unroll
    for (int e = 0; e < E; e += 2) {
      const float4 b = RCG ? __ldcg(rv + (q * E + e) / 2) : __ldg(rv + (q * E + e) / 2);
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const float2 c0 = ldlp(&a[k].t[e]), c1 = ldlp(&a[k].t[e + 1]);
        ax[k] = fmaf(c0.x, b.x, fmaf(-c0.y, b.y, ax[k]));
        ay[k] = fmaf(c0.x, b.y, fmaf(c0.y, b.x, ay[k]));
        ax[k] = fmaf(c1.x, b.z, fmaf(-c1.y, b.w, ax[k]));
        ay[k] = fmaf(c1.x, b.w, fmaf(c1.y, b.z, ay[k]));
      }
    }
  }
#pragma unroll
  for (int k = 0; k < R; ++k)
    for (int o = 16; o > 0; o >>= 1) {
      ax[k] += __shfl_xor_sync(0xffffffffu, ax[k], o);
      ay[k] += __shfl_xor_sync(0xffffffffu, ay[k], o);
    }
  if (lane < R) {
    float vx = ax[0], vy = ay[0];
#pragma unroll
    for (int k = 1; k < R; ++k)
      if (lane == k) { vx = ax[k]; vy = ay[k]; }
    if constexpr (SCATTER) {
      const int gs = map[row0 + lane];
      if (gs >= 0) {
        const float2 o = __ldcg(xg + gs);
        xg[gs] = make_float2(o.x + vx, o.y + vy);
      }
    } else {
      x[row0 + lane] = make_float2(vx, vy);
    }
  }
}

}  // namespace ehs
