// Rows of the stored Galerkin operators (Sec. 2.2 eq. coarseGridMatrix): the
// table element loads and the compile-time unrolled row sums shared by the
// Galerkin-level kernels (k_stencil.cu) and the persistent MG-DD coarsest solve
// (k_coarse_persist.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"

namespace ehs {

// Stencil-table element load: complex64/complex128 tables as stored, and the
// half-precision table formats (FP16 or BF16 real/imag pairs) widened to
// complex64 so that accumulation stays in FP32.
template <typename T> __device__ __forceinline__ typename CT<T>::type ldtab(const typename CT<T>::type* p) {
  return __ldg(p);
}
template <typename T> __device__ __forceinline__ float2 ldtab(const __half2* p) {
  return __half22float2(__ldg(p));
}
template <typename T> __device__ __forceinline__ float2 ldtab(const __nv_bfloat162* p) {
  return __bfloat1622float2(__ldg(p));
}

namespace rows {

// Compact slot and mirror flag of box position ti of pair Q in a half table
// (half_index in common.cuh with the pair's constants folded).
template <int D, int LV, int Q>
__device__ __forceinline__ int half_slot_of(int ti, bool& mir) {
  constexpr StencilLayout L = level_layout(D, LV);
  constexpr int a = L.p[Q].a, b = L.p[Q].b;
  constexpr int ne = L.p[Q].ext[0] * L.p[Q].ext[1] * L.p[Q].ext[2];
  constexpr int hb = half_base(L, Q);
  if constexpr (a < b) {
    mir = false;
    return hb + ti;
  } else if constexpr (a == b) {
    constexpr int tc = (ne - 1) / 2;
    mir = ti < tc;
    return hb + (mir ? tc - ti : ti - tc);
  } else {
    constexpr int hbm = half_base(L, L.pidx[b][a]);
    mir = true;
    return hbm + (ne - 1 - ti);
  }
}

// Row a of the stored operator at cell c (coords i), with the stencil box of
// Galerkin level variant LV (1 = first coarse level, 2 = all coarser ones)
// known at compile time so that every table and vector load of the row is
// issued back to back.  SYM: the table is stored half (common.cuh HalfMap), an
// unstored coefficient read from its mirror at the neighbour cell.
// XCG: x is read through L2 only (x written earlier by the same launch on other SMs).
// NS > 1: only the coefficients whose slot index is SI modulo NS (a share of the row, the
// rest summed by NS - 1 other threads).
template <typename T, typename TT, int D, int LV, bool SYM, int Q, int QE, bool XCG = false, int NS = 1, int SI = 0>
__device__ __forceinline__ void row_acc(typename CT<T>::type& y, const Grid& g,
                                        const TT* __restrict__ tab,
                                        long long c, const int i[3],
                                        const typename CT<T>::type* __restrict__ x) {
  if constexpr (Q < QE) {
    constexpr StencilLayout L = level_layout(D, LV);
    constexpr int b = L.p[Q].b, base = L.p[Q].base;
    constexpr int lo0 = L.p[Q].lo[0], lo1 = L.p[Q].lo[1], lo2 = L.p[Q].lo[2];
    constexpr int e0 = L.p[Q].ext[0], e1 = L.p[Q].ext[1], e2 = L.p[Q].ext[2];
    const long long N = g.ncell;
    const long long sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
    const typename CT<T>::type* xb = x + (long long)b * N;
#pragma unroll
    for (int oz = 0; oz < e2; ++oz) {
      const int jz = i[2] + lo2 + oz;
#pragma unroll
      for (int oy = 0; oy < e1; ++oy) {
        const int jy = i[1] + lo1 + oy;
        const bool rin = (D < 3 || (jz >= 0 && jz < g.n[2])) && jy >= 0 && jy < g.n[1];
#pragma unroll
        for (int ox = 0; ox < e0; ++ox) {
          const int jx = i[0] + lo0 + ox;
          if ((NS == 1 || (base + (oz * e1 + oy) * e0 + ox) % NS == SI) && rin && jx >= 0 && jx < g.n[0]) {
            const int ti = (oz * e1 + oy) * e0 + ox;
            const long long cj = c + (lo2 + oz) * sz + (lo1 + oy) * sy + (lo0 + ox);
            const TT* tp;
            if constexpr (SYM) {
              bool mir = false;
              const int hs = half_slot_of<D, LV, Q>(ti, mir);
              tp = tab + (long long)hs * N + (mir ? cj : c);
            } else {
              tp = tab + (long long)(base + ti) * N + c;
            }
            y = cfma(ldtab<T>(tp), XCG ? __ldcg(xb + cj) : __ldg(xb + cj), y);
          }
        }
      }
    }
    row_acc<T, TT, D, LV, SYM, Q + 1, QE, XCG, NS, SI>(y, g, tab, c, i, x);
  }
}

template <typename T, typename TT, int D, int LV, bool SYM, int A, bool XCG = false, int NS = 1, int SI = 0>
__device__ __forceinline__ typename CT<T>::type st_row_ct(const Grid& g, const TT* tab,
                                                           long long c, const int i[3],
                                                           const typename CT<T>::type* x) {
  constexpr StencilLayout L = level_layout(D, LV);
  typename CT<T>::type y = czero<typename CT<T>::type>();
  row_acc<T, TT, D, LV, SYM, L.row_first[A], L.row_first[A + 1], XCG, NS, SI>(y, g, tab, c, i, x);
  return y;
}

}  // namespace rows
using rows::st_row_ct;
using rows::half_slot_of;

}  // namespace ehs
