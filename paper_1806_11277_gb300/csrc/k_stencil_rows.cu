// Residual passes over the Galerkin levels' stored stencils (Sec. 2.2 eq.
// coarseGridMatrix: y = K_c x or b - K_c x row by row from the tables built by
// k_stencil.cu's Galerkin product), in the launch shapes the setup autotuner
// chooses from.  Kept apart from k_stencil.cu so that the two compile in
// parallel.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"
#include "stencil_rows.cuh"

namespace ehs {
namespace {

// Residual pass of a Galerkin-level operation: one thread per (cell, row
// type); blockIdx.z selects the row type, so control flow is uniform across
// a warp and the row's stencil loop is fully unrolled.  mode 0: y = A x,
// mode 1: y = b - A x.  colour >= 0 restricts the pressure rows to cells of
// that colour (the rows a red-black half-sweep needs).
template <typename T, typename TT, int D, int LV, bool SYM, int A>
__device__ __forceinline__ void st_one_row(const Grid& g, const TT* ts, long long c,
                                           const int i[3], const typename CT<T>::type* xv,
                                           const typename CT<T>::type* bv, typename CT<T>::type* yv,
                                           int mode) {
  typedef typename CT<T>::type Cx;
  const long long N = g.ncell;
  Cx r = czero<Cx>();
  if (slot_valid(A, D, i)) {
    r = st_row_ct<T, TT, D, LV, SYM, A>(g, ts, c, i, xv);
    if (mode) r = csub(__ldg(bv + (long long)A * N + c), r);
  }
  yv[(long long)A * N + c] = r;
}

template <typename T, typename TT, int D, int LV, bool SYM>
__global__ void __launch_bounds__(256) k_st_rows(Grid g, int nrhs, const TT* __restrict__ tab,
                                                 const typename CT<T>::type* __restrict__ x,
                                                 const typename CT<T>::type* __restrict__ b,
                                                 typename CT<T>::type* __restrict__ y, int mode, int colour,
                                                 const int* __restrict__ il) {
  constexpr StencilLayout L = level_layout(D, LV);
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int a = blockIdx.z;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  int i[3];
  cell_coords(g, c, i);
  if (a == D && colour >= 0 && ((i[0] + i[1] + i[2]) & 1) != colour) return;
  const long long N = g.ncell;
  const long long vo = (long long)item * (D + 1) * N;
  constexpr int nslot = SYM ? half_base(L, L.npair) : L.nslot;
  const TT* ts = tab + (long long)(item / nrhs) * nslot * N;
  const typename CT<T>::type* bv = mode ? b + vo : nullptr;
  if (a == 0) st_one_row<T, TT, D, LV, SYM, 0>(g, ts, c, i, x + vo, bv, y + vo, mode);
  else if (a == 1) st_one_row<T, TT, D, LV, SYM, 1>(g, ts, c, i, x + vo, bv, y + vo, mode);
  else if (a == 2) st_one_row<T, TT, D, LV, SYM, 2>(g, ts, c, i, x + vo, bv, y + vo, mode);
  else if constexpr (D == 3) st_one_row<T, TT, D, LV, SYM, 3>(g, ts, c, i, x + vo, bv, y + vo, mode);
}

// Two-cells-per-thread variant of the residual pass: cells c and c+1 (same x
// row; n_x is even on every level that uses it) share one vector load of
// their two table coefficients per stencil entry, doubling the bytes each
// load brings in.  Same arithmetic, per cell, as k_st_rows.
template <typename TT> struct Pair2;
template <> struct Pair2<float2> {
  typedef float4 V;
  static __device__ __forceinline__ void ld(const float2* p, float2& a, float2& b) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    a = make_float2(v.x, v.y); b = make_float2(v.z, v.w);
  }
};
template <> struct Pair2<double2> {
  static __device__ __forceinline__ void ld(const double2* p, double2& a, double2& b) {
    a = __ldg(p); b = __ldg(p + 1);
  }
};
template <> struct Pair2<__half2> {
  static __device__ __forceinline__ void ld(const __half2* p, float2& a, float2& b) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
    b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
  }
};
template <> struct Pair2<__nv_bfloat162> {
  static __device__ __forceinline__ void ld(const __nv_bfloat162* p, float2& a, float2& b) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.x));
    b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v.y));
  }
};

template <typename T, typename TT, int D, int LV, bool SYM, int Q, int QE>
__device__ __forceinline__ void row_acc2(typename CT<T>::type& y0, typename CT<T>::type& y1, const Grid& g,
                                         const TT* __restrict__ tab, long long c, const int i[3],
                                         const typename CT<T>::type* __restrict__ x) {
  if constexpr (Q < QE) {
    typedef typename CT<T>::type Cx;
    constexpr StencilLayout L = level_layout(D, LV);
    constexpr int b = L.p[Q].b, base = L.p[Q].base;
    constexpr int lo0 = L.p[Q].lo[0], lo1 = L.p[Q].lo[1], lo2 = L.p[Q].lo[2];
    constexpr int e0 = L.p[Q].ext[0], e1 = L.p[Q].ext[1], e2 = L.p[Q].ext[2];
    const long long N = g.ncell;
    const long long sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
    const Cx* xb = x + (long long)b * N;
#pragma unroll
    for (int oz = 0; oz < e2; ++oz) {
      const int jz = i[2] + lo2 + oz;
#pragma unroll
      for (int oy = 0; oy < e1; ++oy) {
        const int jy = i[1] + lo1 + oy;
        const bool rin = (D < 3 || (jz >= 0 && jz < g.n[2])) && jy >= 0 && jy < g.n[1];
#pragma unroll
        for (int ox = 0; ox < e0; ++ox) {
          const int jx = i[0] + lo0 + ox;       // neighbour of cell c; jx + 1 is the one of c + 1
          const int ti = (oz * e1 + oy) * e0 + ox;
          const long long cj = c + (lo2 + oz) * sz + (lo1 + oy) * sy + (lo0 + ox);
          Cx t0 = czero<Cx>(), t1 = czero<Cx>();
          if constexpr (SYM) {
            // the mirror of cell c's coefficient sits at cell cj, c + 1's at cj + 1; cj is even
            // (aligned pair load) when the x offset is even (n_x is even here)
            bool mir = false;
            const int hs = half_slot_of<D, LV, Q>(ti, mir);
            const TT* tp = tab + (long long)hs * N + (mir ? cj : c);
            const bool in0 = rin && jx >= 0 && jx < g.n[0], in1 = rin && jx + 1 >= 0 && jx + 1 < g.n[0];
            if (!mir || ((lo0 + ox) & 1) == 0) {
              if (!mir || (in0 && in1)) Pair2<TT>::ld(tp, t0, t1);
              else {                            // a mirror cell outside the grid is not read
                if (in0) t0 = ldtab<T>(tp);
                if (in1) t1 = ldtab<T>(tp + 1);
              }
            } else {
              if (in0) t0 = ldtab<T>(tp);
              if (in1) t1 = ldtab<T>(tp + 1);
            }
          } else {
            Pair2<TT>::ld(tab + (long long)(base + ti) * N + c, t0, t1);
          }
          if (rin && jx >= 0 && jx < g.n[0]) y0 = cfma(t0, __ldg(xb + cj), y0);
          if (rin && jx + 1 >= 0 && jx + 1 < g.n[0]) y1 = cfma(t1, __ldg(xb + cj + 1), y1);
        }
      }
    }
    row_acc2<T, TT, D, LV, SYM, Q + 1, QE>(y0, y1, g, tab, c, i, x);
  }
}

template <typename T, typename TT, int D, int LV, bool SYM, int A>
__device__ __forceinline__ void st_two_rows(const Grid& g, const TT* ts, long long c, const int i[3],
                                            const typename CT<T>::type* xv, const typename CT<T>::type* bv,
                                            typename CT<T>::type* yv, int mode, int colour) {
  typedef typename CT<T>::type Cx;
  constexpr StencilLayout L = level_layout(D, LV);
  const long long N = g.ncell;
  Cx y0 = czero<Cx>(), y1 = czero<Cx>();
  row_acc2<T, TT, D, LV, SYM, L.row_first[A], L.row_first[A + 1]>(y0, y1, g, ts, c, i, xv);
  const int i1[3] = {i[0] + 1, i[1], i[2]};
  const bool v0 = slot_valid(A, D, i), v1 = slot_valid(A, D, i1);
  const int par = (i[0] + i[1] + i[2]) & 1;
  const bool w0 = !(A == D && colour >= 0 && par != colour), w1 = !(A == D && colour >= 0 && par == colour);
  if (mode) {
    if (v0) y0 = csub(__ldg(bv + (long long)A * N + c), y0);
    if (v1) y1 = csub(__ldg(bv + (long long)A * N + c + 1), y1);
  }
  if (w0) yv[(long long)A * N + c] = v0 ? y0 : czero<Cx>();
  if (w1) yv[(long long)A * N + c + 1] = v1 ? y1 : czero<Cx>();
}

template <typename T, typename TT, int D, int LV, bool SYM>
__global__ void k_st_rows2(Grid g, int nrhs, const TT* __restrict__ tab, const typename CT<T>::type* __restrict__ x,
                           const typename CT<T>::type* __restrict__ b, typename CT<T>::type* __restrict__ y,
                           int mode, int colour, const int* __restrict__ il) {
  constexpr StencilLayout L = level_layout(D, LV);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.ncell / 2) return;
  const long long c = 2 * t;
  const int a = blockIdx.z;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  int i[3];
  cell_coords(g, c, i);
  const long long N = g.ncell;
  const long long vo = (long long)item * (D + 1) * N;
  constexpr int nslot = SYM ? half_base(L, L.npair) : L.nslot;
  const TT* ts = tab + (long long)(item / nrhs) * nslot * N;
  const typename CT<T>::type* bv = mode ? b + vo : nullptr;
  if (a == 0) st_two_rows<T, TT, D, LV, SYM, 0>(g, ts, c, i, x + vo, bv, y + vo, mode, colour);
  else if (a == 1) st_two_rows<T, TT, D, LV, SYM, 1>(g, ts, c, i, x + vo, bv, y + vo, mode, colour);
  else if (a == 2) st_two_rows<T, TT, D, LV, SYM, 2>(g, ts, c, i, x + vo, bv, y + vo, mode, colour);
  else if constexpr (D == 3) st_two_rows<T, TT, D, LV, SYM, 3>(g, ts, c, i, x + vo, bv, y + vo, mode, colour);
}

// residual-pass launch shapes the autotuner chooses from: (cells per thread, threads per block)
static const int kRowsCpt[ST_ROWS_VARIANTS] = {1, 2, 1, 2};
static const int kRowsBs[ST_ROWS_VARIANTS] = {128, 128, 256, 64};

template <typename T, typename TT, bool SYM>
static void st_apply_t(const Grid& g, int items, int nrhs, int v, const TT* tab, const typename CT<T>::type* x,
                       const typename CT<T>::type* b, typename CT<T>::type* y, int mode, int colour,
                       int var, cudaStream_t s) {
  if (var < 0 || var >= ST_ROWS_VARIANTS || (kRowsCpt[var] == 2 && (g.n[0] & 1))) var = 0;
  const int bs = kRowsBs[var];
  if (kRowsCpt[var] == 1) {
    const dim3 gr((unsigned)((g.ncell + bs - 1) / bs), sel_items(items), g.d + 1);
    if (g.d == 2) {
      if (v == 1) k_st_rows<T, TT, 2, 1, SYM><<<gr, bs, 0, s>>>(g, nrhs, tab, x, b, y, mode, colour, g_sel.list);
      else k_st_rows<T, TT, 2, 2, SYM><<<gr, bs, 0, s>>>(g, nrhs, tab, x, b, y, mode, colour, g_sel.list);
    } else if constexpr (!SYM) {
      if (v == 1) k_st_rows<T, TT, 3, 1, SYM><<<gr, bs, 0, s>>>(g, nrhs, tab, x, b, y, mode, colour, g_sel.list);
      else k_st_rows<T, TT, 3, 2, SYM><<<gr, bs, 0, s>>>(g, nrhs, tab, x, b, y, mode, colour, g_sel.list);
    }
  } else {
    const dim3 gr((unsigned)((g.ncell / 2 + bs - 1) / bs), sel_items(items), g.d + 1);
    if (g.d == 2) {
      if (v == 1) k_st_rows2<T, TT, 2, 1, SYM><<<gr, bs, 0, s>>>(g, nrhs, tab, x, b, y, mode, colour, g_sel.list);
      else k_st_rows2<T, TT, 2, 2, SYM><<<gr, bs, 0, s>>>(g, nrhs, tab, x, b, y, mode, colour, g_sel.list);
    } else if constexpr (!SYM) {
      if (v == 1) k_st_rows2<T, TT, 3, 1, SYM><<<gr, bs, 0, s>>>(g, nrhs, tab, x, b, y, mode, colour, g_sel.list);
      else k_st_rows2<T, TT, 3, 2, SYM><<<gr, bs, 0, s>>>(g, nrhs, tab, x, b, y, mode, colour, g_sel.list);
    }
  }
}
// dispatch on the table storage format (0: as T, full; 1: FP16 pairs, 2: BF16 pairs; T = float
// only).  In 2D the half formats are stored half by symmetry (launch_table_half_sym); in 3D
// they are full (the mirrored reads of the 3D boxes cost more registers than they save).
template <typename T>
static void st_apply_any(const Grid& g, int items, int nrhs, int v, const void* tab, int fmt,
                         const typename CT<T>::type* x, const typename CT<T>::type* b, typename CT<T>::type* y,
                         int mode, int colour, int var, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (fmt == 1 && g.d == 2)
      return st_apply_t<T, __half2, true>(g, items, nrhs, v, (const __half2*)tab, x, b, y, mode, colour, var, s);
    if (fmt == 2 && g.d == 2)
      return st_apply_t<T, __nv_bfloat162, true>(g, items, nrhs, v, (const __nv_bfloat162*)tab, x, b, y, mode, colour,
                                                 var, s);
    if (fmt == 1)
      return st_apply_t<T, __half2, false>(g, items, nrhs, v, (const __half2*)tab, x, b, y, mode, colour, var, s);
    if (fmt == 2)
      return st_apply_t<T, __nv_bfloat162, false>(g, items, nrhs, v, (const __nv_bfloat162*)tab, x, b, y, mode,
                                                  colour, var, s);
  }
  st_apply_t<T, typename CT<T>::type, false>(g, items, nrhs, v, (const typename CT<T>::type*)tab, x, b, y, mode,
                                             colour, var, s);
}
}  // namespace

template <typename T>
void launch_st_rows(const Grid& g, int items, int nrhs, int v, const void* tab, int fmt,
                    const typename CT<T>::type* x, const typename CT<T>::type* b, typename CT<T>::type* y, int mode,
                    int colour, int var, cudaStream_t s) {
  st_apply_any<T>(g, items, nrhs, v, tab, fmt, x, b, y, mode, colour, var, s);
}

template <typename T>
void launch_st_apply(const Grid& g, int items, int nrhs, const StencilLayout& L, const void* tab, int fmt,
                     const typename CT<T>::type* x, const typename CT<T>::type* b, typename CT<T>::type* y,
                     int mode, int var, cudaStream_t s) {
  launch_st_rows<T>(g, items, nrhs, layout_variant(L, g.d), tab, fmt, x, b, y, mode, -1, var, s);
}

#define INST(T)                                                                                            \
  template void launch_st_rows<T>(const Grid&, int, int, int, const void*, int, const CT<T>::type*,          \
                                  const CT<T>::type*, CT<T>::type*, int, int, int, cudaStream_t);            \
  template void launch_st_apply<T>(const Grid&, int, int, const StencilLayout&, const void*, int,            \
                                   const CT<T>::type*, const CT<T>::type*, CT<T>::type*, int, int,           \
                                   cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace ehs
