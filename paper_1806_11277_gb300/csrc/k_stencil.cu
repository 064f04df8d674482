// Galerkin coarse operators K_c = P^T K P (Sec. 2.2 eq. coarseGridMatrix,
// built on the shifted operator as Sec. 3 prescribes) stored as per-cell
// stencil tables, and the kernels that apply and relax them.
//
// The table keeps, for every (row component a, column component b) pair, a
// box of offsets; the coarse box of a pair follows from the fine box and the
// 1D transfer supports, so the hierarchy never stores offsets it cannot use.
#include <algorithm>
#include <stdexcept>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"
#include "stencil_rows.cuh"

namespace ehs {

// ------------------------------------------------------------------ layout
void coarse_layout(int d, const StencilLayout& F, StencilLayout* C) { *C = make_coarse_layout(d, F); }

namespace {

#define EHS_MAXROW 512

// 1D list of (fine index, weight) of coarse index I, and of (coarse index,
// weight) of fine index j.
__device__ __forceinline__ int fine_support(int kind, int I, int nc, int* idx, double* w) {
  int n = 0;
  for (int i = 2 * I - 2; i <= 2 * I + 3; ++i) {
    const double v = pw(kind, i, I, nc);
    if (v != 0.0) { idx[n] = i; w[n] = v; ++n; }
  }
  return n;
}
__device__ __forceinline__ int coarse_support(int kind, int j, int nc, int* idx, double* w) {
  int n = 0;
  for (int J = (j >> 1) - 1; J <= (j >> 1) + 1; ++J) {
    const double v = pw(kind, j, J, nc);
    if (v != 0.0) { idx[n] = J; w[n] = v; ++n; }
  }
  return n;
}

// one thread per (coarse cell, row component)
template <int D>
__global__ void k_galerkin(Grid gf, Grid gc, StencilLayout Lf, const double2* __restrict__ tf,
                           StencilLayout Lc, double2* __restrict__ tc, int* err) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gc.ncell * (D + 1)) return;
  const int a = (int)(t / gc.ncell);
  const long long C = t % gc.ncell;
  const int set = blockIdx.y;
  const double2* TF = tf + (long long)set * Lf.nslot * gf.ncell;
  double2* TC = tc + (long long)set * Lc.nslot * gc.ncell;
  const int q0 = Lc.row_first[a], q1 = Lc.row_first[a + 1];
  const int s0 = Lc.p[q0].base;
  const int s1 = (q1 < Lc.npair) ? Lc.p[q1].base : Lc.nslot;
  double2 acc[EHS_MAXROW];
  for (int s = 0; s < s1 - s0; ++s) acc[s] = make_double2(0, 0);
  int Ic[3];
  cell_coords(gc, C, Ic);
  if (slot_valid(a, D, Ic)) {
    int fi[3][6];
    double fw[3][6];
    int nf[3] = {1, 1, 1};
    for (int k = 0; k < 3; ++k) {
      if (k < D) nf[k] = fine_support(tkind(a, k, D), Ic[k], gc.n[k], fi[k], fw[k]);
      else { fi[k][0] = 0; fw[k][0] = 1.0; }
    }
    for (int az = 0; az < nf[2]; ++az)
      for (int ay = 0; ay < nf[1]; ++ay)
        for (int ax = 0; ax < nf[0]; ++ax) {
          const int i[3] = {fi[0][ax], fi[1][ay], fi[2][az]};
          if (!slot_valid(a, D, i)) continue;
          const double wi = fw[0][ax] * fw[1][ay] * fw[2][az];
          const long long ci = cell_index(gf, i);
          for (int q = Lf.row_first[a]; q < Lf.row_first[a + 1]; ++q) {
            const PairBox& P = Lf.p[q];
            const int b = P.b;
            const int qc = Lc.pidx[a][b];
            const PairBox& Q = Lc.p[qc];
            for (int oz = 0; oz < P.ext[2]; ++oz)
              for (int oy = 0; oy < P.ext[1]; ++oy)
                for (int ox = 0; ox < P.ext[0]; ++ox) {
                  const int s = P.base + (oz * P.ext[1] + oy) * P.ext[0] + ox;
                  const double2 kv = TF[(long long)s * gf.ncell + ci];
                  if (kv.x == 0.0 && kv.y == 0.0) continue;
                  const int j[3] = {i[0] + P.lo[0] + ox, i[1] + P.lo[1] + oy, i[2] + P.lo[2] + oz};
                  bool in = true;
                  for (int k = 0; k < D; ++k) in = in && j[k] >= 0 && j[k] < gf.n[k];
                  if (!in || !slot_valid(b, D, j)) continue;
                  int ci2[3][3];
                  double cw[3][3];
                  int nn[3] = {1, 1, 1};
                  for (int k = 0; k < 3; ++k) {
                    if (k < D) nn[k] = coarse_support(tkind(b, k, D), j[k], gc.n[k], ci2[k], cw[k]);
                    else { ci2[k][0] = 0; cw[k][0] = 1.0; }
                  }
                  for (int bz = 0; bz < nn[2]; ++bz)
                    for (int by = 0; by < nn[1]; ++by)
                      for (int bx = 0; bx < nn[0]; ++bx) {
                        const double w = wi * cw[0][bx] * cw[1][by] * cw[2][bz];
                        const int O[3] = {ci2[0][bx] - Ic[0], ci2[1][by] - Ic[1], ci2[2][bz] - Ic[2]};
                        const int lx = O[0] - Q.lo[0], ly = O[1] - Q.lo[1], lz = O[2] - Q.lo[2];
                        if (lx < 0 || ly < 0 || lz < 0 || lx >= Q.ext[0] || ly >= Q.ext[1] ||
                            lz >= Q.ext[2]) {
                          atomicOr(err, EHS_DEVERR_BOX);
                          continue;
                        }
                        const int sl = Q.base - s0 + (lz * Q.ext[1] + ly) * Q.ext[0] + lx;
                        acc[sl].x += w * kv.x;
                        acc[sl].y += w * kv.y;
                      }
                }
          }
        }
  }
  for (int s = 0; s < s1 - s0; ++s) TC[(long long)(s0 + s) * gc.ncell + C] = acc[s];
}

template <typename C>
__global__ void k_table_cast(long long n, const double2* in, C* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double2 v = in[i];
    C r; r.x = v.x; r.y = v.y;
    out[i] = r;
  }
}

// Update pass of one colour: the economic cell block (stored diagonal and
// displacement-pressure couplings) is solved for every cell of the colour
// from the residual r of the residual pass; xo receives the new iterate.
// Coefficient (row A, column B, offset O) of the row at cell c from a full table
// (slot of the layout at cell c) or a half table (compact slot at c, or its
// mirror's at c + O; off = the linear cell offset of O), slots folded at
// compile time.
template <typename T, typename TT, int D, int LV, bool SYM, int A, int B, int OX, int OY, int OZ>
__device__ __forceinline__ typename CT<T>::type tab_coef(const TT* ts, long long N, long long c, long long off) {
  constexpr StencilLayout L = level_layout(D, LV);
  constexpr int sl = st_slot(L, A, B, OX, OY, OZ);
  static_assert(sl >= 0, "coefficient outside the stored box");
  if constexpr (SYM) {
    constexpr int q = L.pidx[A][B];
    constexpr bool mir = half_mir_c(L, q, sl - L.p[q].base);
    constexpr int hs = half_slot_c(L, q, sl - L.p[q].base);
    return ldtab<T>(ts + (long long)hs * N + (mir ? c + off : c));
  } else {
    return ldtab<T>(ts + (long long)sl * N + c);
  }
}

// the block coefficients of component K of the economic cell update: diagonals of the low
// and high face, their couplings to the cell's pressure, and back
template <typename T, typename TT, int D, int LV, bool SYM, int K>
__device__ __forceinline__ void vupd_coefs(const TT* ts, long long N, long long c, long long sk, bool lo_ok,
                                           bool hi_ok, typename CT<T>::type* dg, typename CT<T>::type* gr,
                                           typename CT<T>::type* gc) {
  constexpr int E0 = K == 0, E1 = K == 1, E2 = K == 2;
  if (lo_ok) {
    dg[K] = tab_coef<T, TT, D, LV, SYM, K, K, 0, 0, 0>(ts, N, c, 0);
    gr[K] = tab_coef<T, TT, D, LV, SYM, K, D, 0, 0, 0>(ts, N, c, 0);
    gc[K] = tab_coef<T, TT, D, LV, SYM, D, K, 0, 0, 0>(ts, N, c, 0);
  }
  if (hi_ok) {
    dg[D + K] = tab_coef<T, TT, D, LV, SYM, K, K, 0, 0, 0>(ts, N, c + sk, 0);
    gr[D + K] = tab_coef<T, TT, D, LV, SYM, K, D, -E0, -E1, -E2>(ts, N, c + sk, -sk);
    gc[D + K] = tab_coef<T, TT, D, LV, SYM, D, K, E0, E1, E2>(ts, N, c, sk);
  }
}

template <typename T, typename TT, int D, int LV, bool SYM>
__global__ void __launch_bounds__(128) k_st_vupd(Grid g, int nrhs, const TT* __restrict__ tab,
                                                 T wu, T wp, int colour,
                                                 const typename CT<T>::type* __restrict__ res,
                                                 const typename CT<T>::type* __restrict__ xi,
                                                 typename CT<T>::type* __restrict__ xo,
                                                 const int* __restrict__ il) {
  typedef typename CT<T>::type Cx;
  constexpr StencilLayout L = level_layout(D, LV);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long N = g.ncell;
  if (t >= N / 2) return;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const long long vo = (long long)item * (D + 1) * N;
  constexpr int nslot = SYM ? half_base(L, L.npair) : L.nslot;
  const TT* ts = tab + (long long)(item / nrhs) * nslot * N;
  const Cx* x = xi + vo;
  const Cx* rr = res + vo;
  Cx* xout = xo + vo;
  long long c = 2 * t;
  int i[3];
  cell_coords(g, c, i);
  if (((i[0] + i[1] + i[2]) & 1) != colour) { ++c; ++i[0]; }
  const long long co = (c & 1) ? c - 1 : c + 1;
  xout[(long long)D * N + co] = __ldg(x + (long long)D * N + co);
  Cx r[2 * D + 1], dg[2 * D], gr[2 * D], gc_[2 * D];
  bool ok[2 * D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const long long sk = stride_of(g, k);
    ok[k] = i[k] >= 1;
    ok[D + k] = i[k] + 1 < g.n[k];
    if (ok[k]) r[k] = __ldg(rr + (long long)k * N + c);
    if (ok[D + k]) r[D + k] = __ldg(rr + (long long)k * N + c + sk);
  }
  vupd_coefs<T, TT, D, LV, SYM, 0>(ts, N, c, stride_of(g, 0), ok[0], ok[D], dg, gr, gc_);
  vupd_coefs<T, TT, D, LV, SYM, 1>(ts, N, c, stride_of(g, 1), ok[1], ok[D + 1], dg, gr, gc_);
  if constexpr (D == 3) vupd_coefs<T, TT, D, LV, SYM, 2>(ts, N, c, stride_of(g, 2), ok[2], ok[D + 2], dg, gr, gc_);
  r[2 * D] = __ldg(rr + (long long)D * N + c);
  Cx sch = tab_coef<T, TT, D, LV, SYM, D, D, 0, 0, 0>(ts, N, c, 0);
  Cx rp = r[2 * D];
  Cx dinv[2 * D];
#pragma unroll
  for (int a = 0; a < 2 * D; ++a) {
    if (!ok[a]) continue;
    dinv[a] = cinv(dg[a]);
    const Cx gd = cmul(gc_[a], dinv[a]);
    sch = csub(sch, cmul(gd, gr[a]));
    rp = csub(rp, cmul(gd, r[a]));
  }
  const Cx dp = cmul(rp, cinv(sch));
  xout[(long long)D * N + c] = cfma(mk<T>(wp, 0), dp, __ldg(x + (long long)D * N + c));
#pragma unroll
  for (int a = 0; a < 2 * D; ++a) {
    if (!ok[a]) continue;
    const int k = a % D;
    const long long idx = (long long)k * N + c + (a >= D ? stride_of(g, k) : 0);
    const Cx du = cmul(csub(r[a], cmul(gr[a], dp)), dinv[a]);
    xout[idx] = cfma(mk<T>(wu, 0), du, __ldg(x + idx));
  }
}

// Full cell-wise Vanka on a Galerkin level (Sec. 4.2, with the setup-time
// block inversion of the implementation remark in Sec. 4): the cell block is
// B_c = K_c[I_c, I_c] over the 2d faces and the pressure of cell c, all
// couplings kept.  DOF a of the block: a < d the low face of u_a (cell c),
// d <= a < 2d the high face of u_{a-d} (cell c + e_{a-d}), 2d the pressure.
// Boundary faces are not unknowns: their rows and columns are the identity.
// Output layout per set: [colour][a * (2d+1) + b][t], t = cell pair index, so
// the update pass of one colour reads its inverses contiguously.
template <int D, int LV>
__global__ void k_block_inv(Grid g, const double2* __restrict__ tab, double2* __restrict__ out,
                            int* __restrict__ err) {
  constexpr StencilLayout L = level_layout(D, LV);
  constexpr int NB = 2 * D + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long N = g.ncell, H = N / 2;
  if (t >= H) return;
  const int set = blockIdx.y, colour = blockIdx.z;
  const double2* ts = tab + (long long)set * L.nslot * N;
  long long c = 2 * t;
  int i[3];
  cell_coords(g, c, i);
  if (((i[0] + i[1] + i[2]) & 1) != colour) { ++c; ++i[0]; }
  int comp[NB], off[NB][3];
  bool ok[NB];
  long long cell[NB];
  for (int a = 0; a < NB; ++a) {
    const int k = a < D ? a : (a < 2 * D ? a - D : D);
    comp[a] = k;
    off[a][0] = off[a][1] = off[a][2] = 0;
    cell[a] = c;
    if (a < D) ok[a] = i[k] >= 1;
    else if (a < 2 * D) { ok[a] = i[k] + 1 < g.n[k]; off[a][k] = 1; cell[a] = c + stride_of(g, k); }
    else ok[a] = true;
  }
  double2 M[NB][2 * NB];   // [B | I] reduced to [I | B^{-1}]
  for (int a = 0; a < NB; ++a)
    for (int b = 0; b < NB; ++b) {
      double2 v = make_double2(a == b ? 1.0 : 0.0, 0.0);
      if (ok[a] && ok[b]) {
        const int sl = st_slot(L, comp[a], comp[b], off[b][0] - off[a][0], off[b][1] - off[a][1],
                               off[b][2] - off[a][2]);
        v = sl >= 0 ? ts[(long long)sl * N + cell[a]] : make_double2(0.0, 0.0);
      }
      M[a][b] = v;
      M[a][NB + b] = make_double2(a == b ? 1.0 : 0.0, 0.0);
    }
  for (int k = 0; k < NB; ++k) {          // Gauss-Jordan with partial pivoting
    int pr = k;
    double best = M[k][k].x * M[k][k].x + M[k][k].y * M[k][k].y;
    for (int a = k + 1; a < NB; ++a) {
      const double m2 = M[a][k].x * M[a][k].x + M[a][k].y * M[a][k].y;
      if (m2 > best) { best = m2; pr = a; }
    }
    if (!(best > 0.0)) { atomicOr(err, EHS_DEVERR_SINGULAR); return; }
    if (pr != k)
      for (int b = 0; b < 2 * NB; ++b) { const double2 tmp = M[k][b]; M[k][b] = M[pr][b]; M[pr][b] = tmp; }
    const double2 piv = cinv(M[k][k]);
    for (int b = 0; b < 2 * NB; ++b) M[k][b] = cmul(M[k][b], piv);
    for (int a = 0; a < NB; ++a) {
      if (a == k) continue;
      const double2 f = M[a][k];
      for (int b = 0; b < 2 * NB; ++b) M[a][b] = csub(M[a][b], cmul(f, M[k][b]));
    }
  }
  double2* o = out + ((long long)set * 2 + colour) * NB * NB * H + t;
  for (int a = 0; a < NB; ++a)
    for (int b = 0; b < NB; ++b) o[(long long)(a * NB + b) * H] = M[a][NB + b];
}

// Update pass of one colour with the stored full block inverses (storage TI:
// complex T, or FP16 / BF16 pairs widened to FP32): x[I_c] += W B_c^{-1} r[I_c].
template <typename T, typename TI, int D>
__global__ void __launch_bounds__(128) k_st_vupd_full(Grid g, int nrhs, const TI* __restrict__ binv,
                                                      T wu, T wp, int colour,
                                                      const typename CT<T>::type* __restrict__ res,
                                                      const typename CT<T>::type* __restrict__ xi,
                                                      typename CT<T>::type* __restrict__ xo,
                                                      const int* __restrict__ il) {
  typedef typename CT<T>::type Cx;
  constexpr int NB = 2 * D + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long N = g.ncell, H = N / 2;
  if (t >= H) return;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const long long vo = (long long)item * (D + 1) * N;
  const TI* bs = binv + ((long long)(item / nrhs) * 2 + colour) * NB * NB * H + t;
  const Cx* x = xi + vo;
  const Cx* rr = res + vo;
  Cx* xout = xo + vo;
  long long c = 2 * t;
  int i[3];
  cell_coords(g, c, i);
  if (((i[0] + i[1] + i[2]) & 1) != colour) { ++c; ++i[0]; }
  const long long co = (c & 1) ? c - 1 : c + 1;
  xout[(long long)D * N + co] = __ldg(x + (long long)D * N + co);
  Cx r[NB];
  long long idx[NB];
  bool ok[NB];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    idx[k] = (long long)k * N + c;
    idx[D + k] = (long long)k * N + c + stride_of(g, k);
    ok[k] = i[k] >= 1;
    ok[D + k] = i[k] + 1 < g.n[k];
  }
  idx[2 * D] = (long long)D * N + c;
  ok[2 * D] = true;
#pragma unroll
  for (int a = 0; a < NB; ++a) r[a] = ok[a] ? __ldg(rr + idx[a]) : czero<Cx>();
#pragma unroll
  for (int a = 0; a < NB; ++a) {
    if (!ok[a]) continue;
    Cx acc = czero<Cx>();
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (ok[b]) acc = cfma(ldtab<T>(bs + (long long)(a * NB + b) * H), r[b], acc);
    xout[idx[a]] = cfma(mk<T>(a < 2 * D ? wu : wp, 0), acc, __ldg(x + idx[a]));
  }
}

// MG-DD colour residual fused with its gather: local unknown e of sub-item bl
// (= ((m * nsub) + s) * nrhs + r) receives (b - K_c x) at coarsest slot
// map[s][e] of item m * nrhs + r, or 0 on padding (map -1); only the rows of
// the colour's subdomains are evaluated.  Two warps share 32 rows, each summing
// the coefficients of one slot parity (a warp-uniform split: no divergence),
// so that twice as many loads are in flight (the launch is small: the box
// unknowns of one colour); the halves meet in shared memory.
template <typename T, typename TT, int D, int LV, bool SYM>
__device__ __forceinline__ typename CT<T>::type gather_row_half(const Grid& g, const TT* ts, long long c,
                                                                const int i[3], const typename CT<T>::type* x,
                                                                int a, int part) {
  if (part == 0) {
    if (a == 0) return st_row_ct<T, TT, D, LV, SYM, 0, false, 2, 0>(g, ts, c, i, x);
    if (a == 1) return st_row_ct<T, TT, D, LV, SYM, 1, false, 2, 0>(g, ts, c, i, x);
    if (a == 2) return st_row_ct<T, TT, D, LV, SYM, 2, false, 2, 0>(g, ts, c, i, x);
    if constexpr (D == 3) return st_row_ct<T, TT, D, LV, SYM, 3, false, 2, 0>(g, ts, c, i, x);
  } else {
    if (a == 0) return st_row_ct<T, TT, D, LV, SYM, 0, false, 2, 1>(g, ts, c, i, x);
    if (a == 1) return st_row_ct<T, TT, D, LV, SYM, 1, false, 2, 1>(g, ts, c, i, x);
    if (a == 2) return st_row_ct<T, TT, D, LV, SYM, 2, false, 2, 1>(g, ts, c, i, x);
    if constexpr (D == 3) return st_row_ct<T, TT, D, LV, SYM, 3, false, 2, 1>(g, ts, c, i, x);
  }
  return czero<typename CT<T>::type>();
}

template <typename T, typename TT, int D, int LV, bool SYM>
__global__ void __launch_bounds__(128) k_st_resid_gather(Grid g, int nrhs, int nsub, int nloc,
                                                         const int* __restrict__ map, const TT* __restrict__ tab,
                                                         const typename CT<T>::type* __restrict__ x,
                                                         const typename CT<T>::type* __restrict__ b,
                                                         typename CT<T>::type* __restrict__ out,
                                                         const int* __restrict__ il) {
  typedef typename CT<T>::type Cx;
  constexpr StencilLayout L = level_layout(D, LV);
  __shared__ Cx half1[2][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int part = w & 1;                                  // slot parity this warp sums
  const int e = blockIdx.x * 64 + (w >> 1) * 32 + lane;
  const int bl = il ? il[blockIdx.y] : blockIdx.y;
  const int r = bl % nrhs, s = (bl / nrhs) % nsub, m = bl / (nrhs * nsub);
  const long long N = g.ncell;
  const int gs = e < nloc ? map[(long long)s * nloc + e] : -1;
  Cx v = czero<Cx>();
  const long long vo = (long long)(m * nrhs + r) * (D + 1) * N;
  if (gs >= 0) {
    const int a = (int)(gs / N);
    const long long c = gs % N;
    constexpr int nslot = SYM ? half_base(L, L.npair) : L.nslot;
    const TT* ts = tab + (long long)m * nslot * N;
    int i[3];
    cell_coords(g, c, i);
    v = gather_row_half<T, TT, D, LV, SYM>(g, ts, c, i, x + vo, a, part);
  }
  if (part) half1[w >> 1][lane] = v;
  __syncthreads();
  if (!part && e < nloc) {
    const Cx v1 = half1[w >> 1][lane];
    v.x += v1.x;
    v.y += v1.y;
    if (gs >= 0) v = csub(__ldg(b + vo + gs), v);
    out[(long long)bl * nloc + e] = v;
  }
}

inline dim3 grid1(long long n, int items, int bs) { return dim3((unsigned)((n + bs - 1) / bs), items, 1); }

}  // namespace

void launch_galerkin(const Grid& gf, const Grid& gc, int nsets, const StencilLayout& Lf,
                     const double2* tf, const StencilLayout& Lc, double2* tc, int* err,
                     cudaStream_t s) {
  int mx = 0;
  for (int a = 0; a <= gf.d; ++a) {
    const int q0 = Lc.row_first[a], q1 = Lc.row_first[a + 1];
    const int s1 = q1 < Lc.npair ? Lc.p[q1].base : Lc.nslot;
    mx = std::max(mx, s1 - Lc.p[q0].base);
  }
  if (mx > EHS_MAXROW) throw std::runtime_error("coarse stencil row exceeds EHS_MAXROW");
  const long long n = gc.ncell * (gf.d + 1);
  if (gf.d == 2)
    k_galerkin<2><<<grid1(n, nsets, 64), 64, 0, s>>>(gf, gc, Lf, tf, Lc, tc, err);
  else
    k_galerkin<3><<<grid1(n, nsets, 64), 64, 0, s>>>(gf, gc, Lf, tf, Lc, tc, err);
}

template <typename T>
void launch_table_cast(long long n, const double2* in, typename CT<T>::type* out, cudaStream_t s) {
  k_table_cast<typename CT<T>::type><<<grid1(n, 1, 256), 256, 0, s>>>(n, in, out);
}

// which compile-time layout variant a runtime layout is (1 or 2)
int layout_variant(const StencilLayout& L, int d) {
  if (d == 2) {
    if (same_layout(L, level_layout(2, 1))) return 1;
    if (same_layout(L, level_layout(2, 2))) return 2;
  } else {
    if (same_layout(L, level_layout(3, 1))) return 1;
    if (same_layout(L, level_layout(3, 2))) return 2;
  }
  throw std::runtime_error("unexpected Galerkin stencil layout");
}

template <typename T, typename TT, bool SYM>
static void st_vupd_t(const Grid& g, int items, int nrhs, int v, const TT* tab, T wu, T wp, int colour,
                      const typename CT<T>::type* r, const typename CT<T>::type* xi, typename CT<T>::type* xo,
                      cudaStream_t s) {
  const dim3 gu((unsigned)((g.ncell / 2 + 127) / 128), sel_items(items), 1);
  if (g.d == 2) {
    if (v == 1) k_st_vupd<T, TT, 2, 1, SYM><<<gu, 128, 0, s>>>(g, nrhs, tab, wu, wp, colour, r, xi, xo, g_sel.list);
    else k_st_vupd<T, TT, 2, 2, SYM><<<gu, 128, 0, s>>>(g, nrhs, tab, wu, wp, colour, r, xi, xo, g_sel.list);
  } else if constexpr (!SYM) {
    if (v == 1) k_st_vupd<T, TT, 3, 1, SYM><<<gu, 128, 0, s>>>(g, nrhs, tab, wu, wp, colour, r, xi, xo, g_sel.list);
    else k_st_vupd<T, TT, 3, 2, SYM><<<gu, 128, 0, s>>>(g, nrhs, tab, wu, wp, colour, r, xi, xo, g_sel.list);
  }
}
// dispatch on the table storage format (0: as T, full; 1: FP16 pairs, 2: BF16 pairs; T = float
// only).  In 2D the half formats are stored half by symmetry (launch_table_half_sym); in 3D
// they are full (the mirrored reads of the 3D boxes cost more registers than they save).
template <typename T>
static void st_vupd_any(const Grid& g, int items, int nrhs, int v, const void* tab, int fmt, T wu, T wp,
                        int colour, const typename CT<T>::type* r, const typename CT<T>::type* xi,
                        typename CT<T>::type* xo, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (fmt == 1 && g.d == 2)
      return st_vupd_t<T, __half2, true>(g, items, nrhs, v, (const __half2*)tab, wu, wp, colour, r, xi, xo, s);
    if (fmt == 2 && g.d == 2)
      return st_vupd_t<T, __nv_bfloat162, true>(g, items, nrhs, v, (const __nv_bfloat162*)tab, wu, wp, colour, r, xi,
                                                xo, s);
    if (fmt == 1)
      return st_vupd_t<T, __half2, false>(g, items, nrhs, v, (const __half2*)tab, wu, wp, colour, r, xi, xo, s);
    if (fmt == 2)
      return st_vupd_t<T, __nv_bfloat162, false>(g, items, nrhs, v, (const __nv_bfloat162*)tab, wu, wp, colour, r,
                                                 xi, xo, s);
  }
  st_vupd_t<T, typename CT<T>::type, false>(g, items, nrhs, v, (const typename CT<T>::type*)tab, wu, wp, colour, r,
                                            xi, xo, s);
}

// one colour of red-black economic Vanka on a Galerkin level: residual pass
// into rbuf (u rows of every cell, p rows of the colour), then the update pass
template <typename T>
void launch_st_vanka(const Grid& g, int items, int nrhs, const StencilLayout& L, const void* tab, int fmt,
                     T wu, T wp, int colour, const typename CT<T>::type* b, const typename CT<T>::type* xi,
                     typename CT<T>::type* xo, typename CT<T>::type* rbuf, int var, cudaStream_t s) {
  const int v = layout_variant(L, g.d);
  launch_st_rows<T>(g, items, nrhs, v, tab, fmt, xi, b, rbuf, 1, colour, var, s);
  st_vupd_any<T>(g, items, nrhs, v, tab, fmt, wu, wp, colour, rbuf, xi, xo, s);
}

// FP64 master table -> half-precision pairs (fmt 1: FP16, 2: BF16)
__global__ void k_table_half(long long n, const double2* __restrict__ in, void* out, int fmt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = in[i];
  if (fmt == 1) ((__half2*)out)[i] = __floats2half2_rn((float)v.x, (float)v.y);
  else ((__nv_bfloat162*)out)[i] = __floats2bfloat162_rn((float)v.x, (float)v.y);
}
template <typename T, typename TT, bool SYM>
static void resid_gather_t(const Grid& g, int items_l, int nrhs, int nsub, int nloc, const int* map, int v,
                           const TT* tab, const typename CT<T>::type* x, const typename CT<T>::type* b,
                           typename CT<T>::type* out, cudaStream_t s) {
  const dim3 gr((unsigned)((nloc + 63) / 64), sel_items(items_l));   // 64 unknowns per 128-thread block
  if (g.d == 2) {
    if (v == 1) k_st_resid_gather<T, TT, 2, 1, SYM><<<gr, 128, 0, s>>>(g, nrhs, nsub, nloc, map, tab, x, b, out, g_sel.list);
    else k_st_resid_gather<T, TT, 2, 2, SYM><<<gr, 128, 0, s>>>(g, nrhs, nsub, nloc, map, tab, x, b, out, g_sel.list);
  } else if constexpr (!SYM) {
    if (v == 1) k_st_resid_gather<T, TT, 3, 1, SYM><<<gr, 128, 0, s>>>(g, nrhs, nsub, nloc, map, tab, x, b, out, g_sel.list);
    else k_st_resid_gather<T, TT, 3, 2, SYM><<<gr, 128, 0, s>>>(g, nrhs, nsub, nloc, map, tab, x, b, out, g_sel.list);
  }
}

template <typename T>
void launch_st_resid_gather(const Grid& g, int items_l, int nrhs, int nsub, int nloc, const int* map,
                            const StencilLayout& L, const void* tab, int fmt, const typename CT<T>::type* x,
                            const typename CT<T>::type* b, typename CT<T>::type* out, cudaStream_t s) {
  const int v = layout_variant(L, g.d);
  if constexpr (sizeof(T) == 4) {
    if (fmt == 1 && g.d == 2)
      return resid_gather_t<T, __half2, true>(g, items_l, nrhs, nsub, nloc, map, v, (const __half2*)tab, x, b, out, s);
    if (fmt == 2 && g.d == 2)
      return resid_gather_t<T, __nv_bfloat162, true>(g, items_l, nrhs, nsub, nloc, map, v,
                                                     (const __nv_bfloat162*)tab, x, b, out, s);
    if (fmt == 1)
      return resid_gather_t<T, __half2, false>(g, items_l, nrhs, nsub, nloc, map, v, (const __half2*)tab, x, b, out,
                                               s);
    if (fmt == 2)
      return resid_gather_t<T, __nv_bfloat162, false>(g, items_l, nrhs, nsub, nloc, map, v,
                                                      (const __nv_bfloat162*)tab, x, b, out, s);
  }
  resid_gather_t<T, typename CT<T>::type, false>(g, items_l, nrhs, nsub, nloc, map, v,
                                                 (const typename CT<T>::type*)tab, x, b, out, s);
}

void launch_table_half(long long n, const double2* in, void* out, int fmt, cudaStream_t s) {
  k_table_half<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, in, out, fmt);
}

// full FP64 table [set][full slot][cell] -> half-precision half table [set][compact slot][cell]
#define EHS_MAXHALF 512
struct HalfFull {
  int full[EHS_MAXHALF];
};
__global__ void k_table_half_sym(long long ncell, int nfull, int nhalf, HalfFull hf, const double2* __restrict__ in,
                                 void* out, int fmt) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int hs = blockIdx.y, set = blockIdx.z;
  const double2 v = in[((long long)set * nfull + hf.full[hs]) * ncell + c];
  const long long o = ((long long)set * nhalf + hs) * ncell + c;
  if (fmt == 1) ((__half2*)out)[o] = __floats2half2_rn((float)v.x, (float)v.y);
  else ((__nv_bfloat162*)out)[o] = __floats2bfloat162_rn((float)v.x, (float)v.y);
}

int half_table_slots(const StencilLayout& L) { return make_half_map(L).nslot; }

void launch_table_half_sym(const Grid& g, int nsets, const StencilLayout& L, const double2* in, void* out, int fmt,
                           cudaStream_t s) {
  const HalfMap H = make_half_map(L);
  if (!H.ok || H.nslot > EHS_MAXHALF) throw std::runtime_error("half table map");
  HalfFull hf{};
  for (int k = 0; k < H.nslot; ++k) hf.full[k] = H.full[k];
  const dim3 gr((unsigned)((g.ncell + 255) / 256), H.nslot, nsets);
  k_table_half_sym<<<gr, 256, 0, s>>>(g.ncell, L.nslot, H.nslot, hf, in, out, fmt);
}

void launch_block_inv(const Grid& g, int nsets, const StencilLayout& L, const double2* tab, double2* out,
                      int* err, cudaStream_t s) {
  const dim3 gr((unsigned)((g.ncell / 2 + 63) / 64), nsets, 2);
  const int v = layout_variant(L, g.d);
  if (g.d == 2) {
    if (v == 1) k_block_inv<2, 1><<<gr, 64, 0, s>>>(g, tab, out, err);
    else k_block_inv<2, 2><<<gr, 64, 0, s>>>(g, tab, out, err);
  } else {
    if (v == 1) k_block_inv<3, 1><<<gr, 64, 0, s>>>(g, tab, out, err);
    else k_block_inv<3, 2><<<gr, 64, 0, s>>>(g, tab, out, err);
  }
}

template <typename T, typename TI>
static void st_vupd_full_t(const Grid& g, int items, int nrhs, const TI* binv, T wu, T wp, int colour,
                           const typename CT<T>::type* r, const typename CT<T>::type* xi,
                           typename CT<T>::type* xo, cudaStream_t s) {
  const dim3 gu((unsigned)((g.ncell / 2 + 127) / 128), sel_items(items), 1);
  if (g.d == 2) k_st_vupd_full<T, TI, 2><<<gu, 128, 0, s>>>(g, nrhs, binv, wu, wp, colour, r, xi, xo, g_sel.list);
  else k_st_vupd_full<T, TI, 3><<<gu, 128, 0, s>>>(g, nrhs, binv, wu, wp, colour, r, xi, xo, g_sel.list);
}

// one colour of red-black full Vanka on a Galerkin level: residual pass, then
// the update with the stored block inverses binv (format bfmt as for tables)
template <typename T>
void launch_st_vanka_full(const Grid& g, int items, int nrhs, const StencilLayout& L, const void* tab, int fmt,
                          const void* binv, int bfmt, T wu, T wp, int colour, const typename CT<T>::type* b,
                          const typename CT<T>::type* xi, typename CT<T>::type* xo, typename CT<T>::type* rbuf,
                          int var, cudaStream_t s) {
  const int v = layout_variant(L, g.d);
  launch_st_rows<T>(g, items, nrhs, v, tab, fmt, xi, b, rbuf, 1, colour, var, s);
  if constexpr (sizeof(T) == 4) {
    if (bfmt == 1) return st_vupd_full_t<T, __half2>(g, items, nrhs, (const __half2*)binv, wu, wp, colour, rbuf, xi, xo, s);
    if (bfmt == 2)
      return st_vupd_full_t<T, __nv_bfloat162>(g, items, nrhs, (const __nv_bfloat162*)binv, wu, wp, colour, rbuf, xi, xo, s);
  }
  st_vupd_full_t<T, typename CT<T>::type>(g, items, nrhs, (const typename CT<T>::type*)binv, wu, wp, colour, rbuf, xi,
                                          xo, s);
}

#define INST(T)                                                                                   \
  template void launch_table_cast<T>(long long, const double2*, CT<T>::type*, cudaStream_t);       \
  template void launch_st_resid_gather<T>(const Grid&, int, int, int, int, const int*, const StencilLayout&,   \
                                          const void*, int, const CT<T>::type*, const CT<T>::type*,          \
                                          CT<T>::type*, cudaStream_t);                                       \
  template void launch_st_vanka<T>(const Grid&, int, int, const StencilLayout&, const void*, int, T, \
                                   T, int, const CT<T>::type*, const CT<T>::type*, CT<T>::type*,    \
                                   CT<T>::type*, int, cudaStream_t); \
  template void launch_st_vanka_full<T>(const Grid&, int, int, const StencilLayout&, const void*, int, \
                                        const void*, int, T, T, int, const CT<T>::type*,               \
                                        const CT<T>::type*, CT<T>::type*, CT<T>::type*, int, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace ehs
