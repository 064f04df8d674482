// Restriction r_c = P^T r_f and prolongation x_f += P e_c (Algorithm TwoCycle
// steps 2 and 4) with the bilinear staggered-grid transfer of Sec. 3: per
// component a tensor product of 1D rules (vertex-like along the component's
// own direction, cell-like with zero ghosts across it, cell-like with clamped
// ghosts for p).  The 1D weights come from pw4() in common.cuh (exact quarters).
#include "kernels.h"

namespace ehs {
namespace {

template <typename T, int D>
__global__ void k_restrict(Grid gf, Grid gc, const typename CT<T>::type* __restrict__ rf,
                           typename CT<T>::type* __restrict__ rc, const int* __restrict__ il) {
  typedef typename CT<T>::type C;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= gc.ncell) return;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const C* f = rf + (long long)item * (D + 1) * gf.ncell;
  C* o = rc + (long long)item * (D + 1) * gc.ncell;
  int I[3];
  cell_coords(gc, c, I);
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    C acc = czero<C>();
    if (slot_valid(a, D, I)) {
      int fi[3][4];
      T fw[3][4];
      int nf[3] = {1, 1, 1};
      for (int k = 0; k < 3; ++k) {
        if (k >= D) { fi[k][0] = 0; fw[k][0] = 1; continue; }
        int n = 0;
        const int kind = tkind(a, k, D);
        for (int i = 2 * I[k] - 1; i <= 2 * I[k] + 2; ++i) {
          const int v = pw4(kind, i, I[k], gc.n[k]);
          if (v != 0) { fi[k][n] = i; fw[k][n] = T(0.25) * (T)v; ++n; }
        }
        nf[k] = n;
      }
      const C* fa = f + (long long)a * gf.ncell;
      for (int z = 0; z < nf[2]; ++z)
        for (int y = 0; y < nf[1]; ++y) {
          const long long row = ((long long)fi[2][z] * gf.n[1] + fi[1][y]) * gf.n[0];
          const T wzy = fw[2][z] * fw[1][y];
          for (int x = 0; x < nf[0]; ++x)
            acc = cfma(mk<T>(wzy * fw[0][x], 0), __ldg(fa + row + fi[0][x]), acc);
        }
    }
    o[(long long)a * gc.ncell + c] = acc;
  }
}

template <typename T, int D>
__global__ void k_prolong_add(Grid gf, Grid gc, const typename CT<T>::type* __restrict__ ec,
                              typename CT<T>::type* __restrict__ xf, const int* __restrict__ il) {
  typedef typename CT<T>::type C;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= gf.ncell) return;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const C* e = ec + (long long)item * (D + 1) * gc.ncell;
  C* x = xf + (long long)item * (D + 1) * gf.ncell;
  int i[3];
  cell_coords(gf, c, i);
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    if (!slot_valid(a, D, i)) continue;
    int ci[3][3];
    T cw[3][3];
    int nc[3] = {1, 1, 1};
    for (int k = 0; k < 3; ++k) {
      if (k >= D) { ci[k][0] = 0; cw[k][0] = 1; continue; }
      int n = 0;
      const int kind = tkind(a, k, D);
      for (int J = (i[k] >> 1) - 1; J <= (i[k] >> 1) + 1; ++J) {
        const int v = pw4(kind, i[k], J, gc.n[k]);
        if (v != 0) { ci[k][n] = J; cw[k][n] = T(0.25) * (T)v; ++n; }
      }
      nc[k] = n;
    }
    const C* ea = e + (long long)a * gc.ncell;
    C acc = czero<C>();
    for (int z = 0; z < nc[2]; ++z)
      for (int y = 0; y < nc[1]; ++y) {
        const long long row = ((long long)ci[2][z] * gc.n[1] + ci[1][y]) * gc.n[0];
        const T wzy = cw[2][z] * cw[1][y];
        for (int xx = 0; xx < nc[0]; ++xx)
          acc = cfma(mk<T>(wzy * cw[0][xx], 0), __ldg(ea + row + ci[0][xx]), acc);
      }
    const long long idx = (long long)a * gf.ncell + c;
    x[idx] = cadd(x[idx], acc);
  }
}

inline dim3 grid1(long long n, int items, int bs) { return dim3((unsigned)((n + bs - 1) / bs), items, 1); }

}  // namespace

template <typename T>
void launch_restrict(const Grid& gf, const Grid& gc, int items, const typename CT<T>::type* rf,
                     typename CT<T>::type* rc, cudaStream_t s) {
  if (gf.d == 2)
    k_restrict<T, 2><<<grid1(gc.ncell, sel_items(items), 128), 128, 0, s>>>(gf, gc, rf, rc, g_sel.list);
  else
    k_restrict<T, 3><<<grid1(gc.ncell, sel_items(items), 128), 128, 0, s>>>(gf, gc, rf, rc, g_sel.list);
}

template <typename T>
void launch_prolong_add(const Grid& gf, const Grid& gc, int items, const typename CT<T>::type* ec,
                        typename CT<T>::type* xf, cudaStream_t s) {
  if (gf.d == 2)
    k_prolong_add<T, 2><<<grid1(gf.ncell, sel_items(items), 256), 256, 0, s>>>(gf, gc, ec, xf, g_sel.list);
  else
    k_prolong_add<T, 3><<<grid1(gf.ncell, sel_items(items), 256), 256, 0, s>>>(gf, gc, ec, xf, g_sel.list);
}

#define INST(T)                                                                                 \
  template void launch_restrict<T>(const Grid&, const Grid&, int, const CT<T>::type*, CT<T>::type*, \
                                   cudaStream_t);                                                \
  template void launch_prolong_add<T>(const Grid&, const Grid&, int, const CT<T>::type*,          \
                                      CT<T>::type*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace ehs
