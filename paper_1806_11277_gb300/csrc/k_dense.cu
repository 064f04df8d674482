// Coarsest level: the Galerkin operator is assembled densely, inverted once in
// FP64 at setup (Gauss-Jordan with partial pivoting), and every cycle applies
// the stored inverse (Algorithm TwoCycle step 3 solved exactly, as the paper's
// coarsest LU does).  Boundary slots are identity rows so the dense index is
// simply comp * ncell + cell.
//
// MG-DD (Sec. 4): the same machinery for the subdomains of the coarsest grid.
// Each box's local matrix (the coarsest operator restricted to the box
// unknowns, padded with identity rows to nloc) is assembled from the stencil
// table and inverted in FP64 together with the others; per colour one launch
// multiplies every subdomain's stored inverse (double-float, complex64, FP16
// or BF16 pairs) with its local residuals, skipping the padding rows.
#include "kernels.h"
#include "dense_rows.cuh"

namespace ehs {
namespace {

template <int D>
__global__ void k_dense_assemble(Grid g, StencilLayout L, const double2* __restrict__ tab,
                                 double2* __restrict__ A) {
  const long long N = (long long)(D + 1) * g.ncell;
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const int set = blockIdx.y;
  const double2* ts = tab + (long long)set * L.nslot * g.ncell;
  double2* row = A + ((long long)set * N + r) * (2 * N);
  const int a = (int)(r / g.ncell);
  const long long c = r % g.ncell;
  for (long long j = 0; j < 2 * N; ++j) row[j] = make_double2(0, 0);
  row[N + r] = make_double2(1, 0);  // augmented identity
  int i[3];
  cell_coords(g, c, i);
  if (!slot_valid(a, D, i)) { row[r] = make_double2(1, 0); return; }
  for (int q = L.row_first[a]; q < L.row_first[a + 1]; ++q) {
    const PairBox& P = L.p[q];
    int s = P.base;
    for (int oz = 0; oz < P.ext[2]; ++oz)
      for (int oy = 0; oy < P.ext[1]; ++oy)
        for (int ox = 0; ox < P.ext[0]; ++ox, ++s) {
          const int j[3] = {i[0] + P.lo[0] + ox, i[1] + P.lo[1] + oy, i[2] + P.lo[2] + oz};
          bool in = true;
          for (int k = 0; k < 3; ++k) in = in && j[k] >= 0 && j[k] < g.n[k];
          if (!in || !slot_valid(P.b, D, j)) continue;
          const double2 v = ts[(long long)s * g.ncell + c];
          const long long col = (long long)P.b * g.ncell + cell_index(g, j);
          row[col].x += v.x;
          row[col].y += v.y;
        }
  }
}

// pivot search of column k (one block per set): piv[set] = argmax_{i>=k} |M[i][k]|
__global__ void k_gj_pivot(int N, int k, const double2* __restrict__ M, int* piv, double2* f, int* err) {
  const int set = blockIdx.x;
  const double2* Ms = M + (long long)set * N * 2 * N;
  __shared__ double bv[1024];
  __shared__ int bi[1024];
  double best = -1.0;
  int besti = k;
  for (int i = k + threadIdx.x; i < N; i += blockDim.x) {
    const double2 v = Ms[(long long)i * 2 * N + k];
    const double m = v.x * v.x + v.y * v.y;
    if (m > best) { best = m; besti = i; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = besti;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = bv[threadIdx.x + s];
      const int oi = bi[threadIdx.x + s];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    piv[set] = bi[0];
    f[(long long)set * (N + 1) + N] = Ms[(long long)bi[0] * 2 * N + k];  // pivot value
    if (!(bv[0] > 0.0)) atomicOr(err, EHS_DEVERR_SINGULAR);
  }
}

// swap rows k and piv, scale row k by 1/pivot (pivot value saved by k_gj_pivot)
__global__ void k_gj_swap(int N, int k, double2* __restrict__ M, const int* piv, double2* f) {
  const int set = blockIdx.y;
  double2* Ms = M + (long long)set * N * 2 * N;
  const int p = piv[set];
  const double2 inv = cinv(f[(long long)set * (N + 1) + N]);
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x + k;
  if (j < 2 * N) {
    double2 a = Ms[(long long)k * 2 * N + j];
    double2 b = Ms[(long long)p * 2 * N + j];
    Ms[(long long)p * 2 * N + j] = a;
    Ms[(long long)k * 2 * N + j] = cmul(b, inv);
  }
}
__global__ void k_gj_col(int N, int k, const double2* __restrict__ M, double2* f) {
  const int set = blockIdx.y;
  const double2* Ms = M + (long long)set * N * 2 * N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) f[(long long)set * (N + 1) + i] = (i == k) ? make_double2(0, 0) : Ms[(long long)i * 2 * N + k];
}
// M[i][j] -= f_i M[k][j] for i != k, j >= k
__global__ void k_gj_elim(int N, int k, double2* __restrict__ M, const double2* __restrict__ f) {
  const int set = blockIdx.z;
  double2* Ms = M + (long long)set * N * 2 * N;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x + k;
  const int i = blockIdx.y;
  if (j >= 2 * N || i == k) return;
  const double2 fi = f[(long long)set * (N + 1) + i];
  if (fi.x == 0.0 && fi.y == 0.0) return;
  const double2 rk = Ms[(long long)k * 2 * N + j];
  double2& m = Ms[(long long)i * 2 * N + j];
  m = csub(m, cmul(fi, rk));
}
__global__ void k_gj_extract(int N, const double2* __restrict__ M, double2* __restrict__ inv) {
  const int set = blockIdx.z;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= N) return;
  inv[((long long)set * N + i) * N + j] = M[((long long)set * N + i) * 2 * N + N + j];
}

// x = Ainv r, one warp per dense row; input/output in the working precision
template <typename T>
__global__ void k_dense_apply(int N, int nrhs, const double2* __restrict__ inv,
                              const typename CT<T>::type* __restrict__ r,
                              typename CT<T>::type* __restrict__ x, const int* __restrict__ il) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  if (warp >= N) return;
  const double2* row = inv + ((long long)(item / nrhs) * N + warp) * N;
  const typename CT<T>::type* rv = r + (long long)item * N;
  double sx = 0.0, sy = 0.0;
  for (int j = lane; j < N; j += 32) {
    const double2 a = __ldg(row + j);
    const typename CT<T>::type b = __ldg(rv + j);
    sx = fma(a.x, (double)b.x, fma(-a.y, (double)b.y, sx));
    sy = fma(a.x, (double)b.y, fma(a.y, (double)b.x, sy));
  }
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  if (lane == 0) {
    typename CT<T>::type v;
    v.x = (T)sx; v.y = (T)sy;
    x[(long long)item * N + warp] = v;
  }
}

// MG-DD local problems (Sec. 4): row e of local matrix (set, s) is the
// coarsest-level row of global slot map[s][e], restricted to the columns that
// are local unknowns of subdomain s (g2l[s][slot] >= 0); padding rows (map -1)
// are identity rows.  Augmented with the identity like k_dense_assemble.
template <int D>
__global__ void k_dense_assemble_sub(Grid g, StencilLayout L, const double2* __restrict__ tab, int nsub,
                                     int nloc, const int* __restrict__ map, const int* __restrict__ g2l,
                                     double2* __restrict__ A) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nloc) return;
  const int ms = blockIdx.y;                 // set * nsub + s
  const int set = ms / nsub, sub = ms % nsub;
  const long long NG = (long long)(D + 1) * g.ncell;
  const double2* ts = tab + (long long)set * L.nslot * g.ncell;
  double2* row = A + ((long long)ms * nloc + e) * (2 * nloc);
  for (int j = 0; j < 2 * nloc; ++j) row[j] = make_double2(0, 0);
  row[nloc + e] = make_double2(1, 0);
  const int gs = map[(long long)sub * nloc + e];
  if (gs < 0) { row[e] = make_double2(1, 0); return; }
  const int* gl = g2l + (long long)sub * NG;
  const int a = (int)(gs / g.ncell);
  const long long c = gs % g.ncell;
  int i[3];
  cell_coords(g, c, i);
  for (int q = L.row_first[a]; q < L.row_first[a + 1]; ++q) {
    const PairBox& P = L.p[q];
    int sl = P.base;
    for (int oz = 0; oz < P.ext[2]; ++oz)
      for (int oy = 0; oy < P.ext[1]; ++oy)
        for (int ox = 0; ox < P.ext[0]; ++ox, ++sl) {
          const int j[3] = {i[0] + P.lo[0] + ox, i[1] + P.lo[1] + oy, i[2] + P.lo[2] + oz};
          bool in = true;
          for (int k = 0; k < 3; ++k) in = in && j[k] >= 0 && j[k] < g.n[k];
          if (!in || !slot_valid(P.b, D, j)) continue;
          const int lc = gl[(long long)P.b * g.ncell + cell_index(g, j)];
          if (lc < 0) continue;
          const double2 v = ts[(long long)sl * g.ncell + c];
          row[lc].x += v.x;
          row[lc].y += v.y;
        }
  }
}

// x = Ainv r with Ainv stored in complex64, FP16 or BF16 pairs (FP32
// accumulation); one warp per row, four independent loads in flight per lane

template <typename TI>
__global__ void k_dense_apply_lp(int N, int nrhs, const TI* __restrict__ inv, const float2* __restrict__ r,
                                 float2* __restrict__ x, const int* __restrict__ il) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  if (warp >= N) return;
  const TI* row = inv + ((long long)(item / nrhs) * N + warp) * N;
  const float2* rv = r + (long long)item * N;
  float sx0 = 0.f, sy0 = 0.f, sx1 = 0.f, sy1 = 0.f;
  int j = lane;
  for (; j + 96 < N; j += 128) {
    const float2 a0 = ldlp(row + j), a1 = ldlp(row + j + 32), a2 = ldlp(row + j + 64), a3 = ldlp(row + j + 96);
    const float2 b0 = __ldg(rv + j), b1 = __ldg(rv + j + 32), b2 = __ldg(rv + j + 64), b3 = __ldg(rv + j + 96);
    sx0 = fmaf(a0.x, b0.x, fmaf(-a0.y, b0.y, sx0)); sy0 = fmaf(a0.x, b0.y, fmaf(a0.y, b0.x, sy0));
    sx1 = fmaf(a1.x, b1.x, fmaf(-a1.y, b1.y, sx1)); sy1 = fmaf(a1.x, b1.y, fmaf(a1.y, b1.x, sy1));
    sx0 = fmaf(a2.x, b2.x, fmaf(-a2.y, b2.y, sx0)); sy0 = fmaf(a2.x, b2.y, fmaf(a2.y, b2.x, sy0));
    sx1 = fmaf(a3.x, b3.x, fmaf(-a3.y, b3.y, sx1)); sy1 = fmaf(a3.x, b3.y, fmaf(a3.y, b3.x, sy1));
  }
  for (; j < N; j += 32) {
    const float2 a = ldlp(row + j), b = __ldg(rv + j);
    sx0 = fmaf(a.x, b.x, fmaf(-a.y, b.y, sx0)); sy0 = fmaf(a.x, b.y, fmaf(a.y, b.x, sy0));
  }
  float sx = sx0 + sx1, sy = sy0 + sy1;
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  if (lane == 0) x[(long long)item * N + warp] = make_float2(sx, sy);
}

// The same product with 16-byte loads (dense_rows4 in dense_rows.cuh): each warp
// computes 4 consecutive rows of the matrix set (item / nrhs), whose live size is
// sizes[set % nsub]; groups of rows at or beyond it are skipped.
template <typename TI>
__global__ void __launch_bounds__(256) k_dense_apply_v(int N, int nrhs, int nsub, const int* __restrict__ sizes,
                                                       const TI* __restrict__ inv, const float2* __restrict__ r,
                                                       float2* __restrict__ x, const int* __restrict__ il) {
  const int row0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const int set = item / nrhs;
  const int n = sizes ? sizes[set % nsub] : N;
  if (row0 >= n) return;
  dense_rows4<TI>(N, n, row0, inv + (long long)set * N * N, r + (long long)item * N, x + (long long)item * N);
}

// The MG-DD form that also scatters: sub-item = ((m * nsub) + s) * nrhs + r, its four results
// added to the coarsest vector xg of item m * nrhs + r at the subdomain's unknowns map[s][row]
// (subdomains of one colour are disjoint, so no two threads add to the same entry).
template <typename TI>
__global__ void __launch_bounds__(256) k_dense_apply_vs(int N, int nrhs, int nsub, const int* __restrict__ sizes,
                                                        const TI* __restrict__ inv, const float2* __restrict__ r,
                                                        const int* __restrict__ map, long long NG, float2* xg,
                                                        const int* __restrict__ il) {
  const int row0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const int set = item / nrhs, sub = set % nsub;
  const int n = sizes[sub];
  if (row0 >= n) return;
  const long long gi = (long long)(set / nsub) * nrhs + item % nrhs;
  dense_rows4<TI, false, true>(N, n, row0, inv + (long long)set * N * N, r + (long long)item * N, nullptr,
                               map + (long long)sub * N, xg + gi * NG);
}

}  // namespace

bool launch_dense_apply_scatter(int N, int items, int nrhs, int nsub, const int* sizes, const void* inv, int fmt,
                                const float2* r, const int* map, long long NG, float2* xg, cudaStream_t s) {
  const int wpb = 8;
  const int E = fmt >= 2 ? 4 : 2;
  if (N % 4 != 0 || N % E != 0 || !sizes) return false;
  const dim3 gv((N / 4 + wpb - 1) / wpb, sel_items(items));   // a warp per 4 rows
  if (fmt == 2)
    k_dense_apply_vs<__half2><<<gv, 32 * wpb, 0, s>>>(N, nrhs, nsub, sizes, (const __half2*)inv, r, map, NG, xg,
                                                       g_sel.list);
  else if (fmt == 3)
    k_dense_apply_vs<__nv_bfloat162><<<gv, 32 * wpb, 0, s>>>(N, nrhs, nsub, sizes, (const __nv_bfloat162*)inv, r, map,
                                                              NG, xg, g_sel.list);
  else
    k_dense_apply_vs<float2><<<gv, 32 * wpb, 0, s>>>(N, nrhs, nsub, sizes, (const float2*)inv, r, map, NG, xg,
                                                      g_sel.list);
  return true;
}

void launch_dense_assemble(const Grid& g, int nsets, const StencilLayout& L, const double2* tab,
                           double2* A, cudaStream_t s) {
  const long long N = (long long)(g.d + 1) * g.ncell;
  dim3 grid((unsigned)((N + 127) / 128), nsets);
  if (g.d == 2) k_dense_assemble<2><<<grid, 128, 0, s>>>(g, L, tab, A);
  else k_dense_assemble<3><<<grid, 128, 0, s>>>(g, L, tab, A);
}

void dense_invert(int N, int nsets, double2* M, double2* inv, double2* fbuf, int* pivbuf, int* err,
                  cudaStream_t s) {
  for (int k = 0; k < N; ++k) {
    k_gj_pivot<<<nsets, 1024, 0, s>>>(N, k, M, pivbuf, fbuf, err);
    const int ncol = 2 * N - k;
    k_gj_swap<<<dim3((ncol + 255) / 256, nsets), 256, 0, s>>>(N, k, M, pivbuf, fbuf);
    k_gj_col<<<dim3((N + 255) / 256, nsets), 256, 0, s>>>(N, k, M, fbuf);
    k_gj_elim<<<dim3((ncol + 255) / 256, N, nsets), 256, 0, s>>>(N, k, M, fbuf);
  }
  k_gj_extract<<<dim3((N + 255) / 256, N, nsets), 256, 0, s>>>(N, M, inv);
}

template <typename T>
void launch_dense_apply(int N, int items, int nrhs, const double2* inv, const typename CT<T>::type* r,
                        typename CT<T>::type* x, cudaStream_t s) {
  const int wpb = 8;
  dim3 grid((N + wpb - 1) / wpb, sel_items(items));
  k_dense_apply<T><<<grid, 32 * wpb, 0, s>>>(N, nrhs, inv, r, x, g_sel.list);
}

void launch_dense_assemble_sub(const Grid& g, int nsets, int nsub, int nloc, const StencilLayout& L,
                               const double2* tab, const int* map, const int* g2l, double2* A, cudaStream_t s) {
  const dim3 grid((unsigned)((nloc + 127) / 128), nsets * nsub);
  if (g.d == 2) k_dense_assemble_sub<2><<<grid, 128, 0, s>>>(g, L, tab, nsub, nloc, map, g2l, A);
  else k_dense_assemble_sub<3><<<grid, 128, 0, s>>>(g, L, tab, nsub, nloc, map, g2l, A);
}

void launch_dense_apply_lp(int N, int items, int nrhs, int nsub, const int* sizes, const void* inv, int fmt,
                           const float2* r, float2* x, cudaStream_t s) {
  const int wpb = 8;
  const dim3 grid((N + wpb - 1) / wpb, sel_items(items));
  const int E = fmt >= 2 ? 4 : 2;
  if (N % 4 == 0 && N % E == 0) {
    const dim3 gv((N / 4 + wpb - 1) / wpb, sel_items(items));   // a warp per 4 rows
    if (fmt == 2)
      k_dense_apply_v<__half2><<<gv, 32 * wpb, 0, s>>>(N, nrhs, nsub, sizes, (const __half2*)inv, r, x, g_sel.list);
    else if (fmt == 3)
      k_dense_apply_v<__nv_bfloat162><<<gv, 32 * wpb, 0, s>>>(N, nrhs, nsub, sizes, (const __nv_bfloat162*)inv, r, x,
                                                              g_sel.list);
    else
      k_dense_apply_v<float2><<<gv, 32 * wpb, 0, s>>>(N, nrhs, nsub, sizes, (const float2*)inv, r, x, g_sel.list);
    return;
  }
  if (fmt == 2)
    k_dense_apply_lp<__half2><<<grid, 32 * wpb, 0, s>>>(N, nrhs, (const __half2*)inv, r, x, g_sel.list);
  else if (fmt == 3)
    k_dense_apply_lp<__nv_bfloat162><<<grid, 32 * wpb, 0, s>>>(N, nrhs, (const __nv_bfloat162*)inv, r, x, g_sel.list);
  else
    k_dense_apply_lp<float2><<<grid, 32 * wpb, 0, s>>>(N, nrhs, (const float2*)inv, r, x, g_sel.list);
}

template void launch_dense_apply<float>(int, int, int, const double2*, const float2*, float2*, cudaStream_t);
template void launch_dense_apply<double>(int, int, int, const double2*, const double2*, double2*, cudaStream_t);

}  // namespace ehs
