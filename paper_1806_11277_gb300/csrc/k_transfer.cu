// Restriction r_c = P^T r_f and prolongation x_f += P e_c (Algorithm TwoCycle
// steps 2 and 4) with the bilinear staggered-grid transfer of Sec. 3: per
// component a tensor product of 1D rules (vertex-like along the component's
// own direction, cell-like with zero ghosts across it, cell-like with clamped
// ghosts for p).  The 1D weights come from pw4() / pw_pair() in common.cuh
// (exact quarters); every tap loop has a fixed trip count and is unrolled, so
// a thread issues all of its loads back to back.  (The 2D complex64 fine
// level of the cycle uses the fused kernels of k_fine_fused.cu instead.)
#include "kernels.h"

namespace ehs {
namespace {

// thread per coarse cell: fine offsets -1..2 around 2I along every direction
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
  constexpr int NZ = D == 3 ? 4 : 1;
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    C acc = czero<C>();
    if (slot_valid(a, D, I)) {
      T w[3][4];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int t = 0; t < 4; ++t)
          w[k][t] = k < D ? T(0.25) * (T)pw4(tkind(a, k, D), 2 * I[k] - 1 + t, I[k], gc.n[k]) : T(t == 0);
      const C* fa = f + (long long)a * gf.ncell;
#pragma unroll
      for (int z = 0; z < NZ; ++z) {
        const int fz = D == 3 ? 2 * I[2] - 1 + z : 0;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const T wzy = w[2][z] * w[1][y];
          if (wzy == T(0)) continue;
          const long long row = ((long long)fz * gf.n[1] + (2 * I[1] - 1 + y)) * gf.n[0];
#pragma unroll
          for (int x = 0; x < 4; ++x)
            if (w[0][x] != T(0)) acc = cfma(mk<T>(wzy * w[0][x], 0), __ldg(fa + row + 2 * I[0] - 1 + x), acc);
        }
      }
    }
    o[(long long)a * gc.ncell + c] = acc;
  }
}

// thread per fine cell: at most two coarse indices per direction (pw_pair)
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
  constexpr int NZ = D == 3 ? 2 : 1;
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    if (!slot_valid(a, D, i)) continue;
    int J[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    T w[3][2] = {{T(1), T(0)}, {T(1), T(0)}, {T(1), T(0)}};
#pragma unroll
    for (int k = 0; k < D; ++k) pw_pair<T>(tkind(a, k, D), i[k], gc.n[k], J[k][0], w[k][0], J[k][1], w[k][1]);
    const C* ea = e + (long long)a * gc.ncell;
    C acc = czero<C>();
#pragma unroll
    for (int z = 0; z < NZ; ++z)
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        const T wzy = w[2][z] * w[1][y];
        if (wzy == T(0)) continue;
        const long long row = ((long long)J[2][z] * gc.n[1] + J[1][y]) * gc.n[0];
#pragma unroll
        for (int xx = 0; xx < 2; ++xx)
          if (w[0][xx] != T(0)) acc = cfma(mk<T>(wzy * w[0][xx], 0), __ldg(ea + row + J[0][xx]), acc);
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
