// Fine-level (matrix-free) kernels of the mixed elastic Helmholtz operator.
//
// Operator (Sec. 2.1 eq. elasticHelmSystem / Sec. 3 eq.
// elasticHelmReformulatedSystem, shifted per eq. shift with the zero-padded
// shift matrix of Sec. 3):
//   row u_k at face f (low face of cell c):
//     sum_j [w+ (u_f - u_{f+e_j}) + w- (u_f - u_{f-e_j})] / h^2
//     + (-mr_f + i (mi_f + alpha mr_f)) u_f + (p_c - p_{c-e_k}) / h
//     with w = mu at the cell centre for j = k and the mean of the 4 cells
//     around the edge for j != k (indices clamped); mr_f, mi_f are the face
//     means of omega^2 rho and omega rho gamma;
//   row p at cell c: sum_k (u_k(c) - u_k(c+e_k)) / h - p_c / (lambda+mu).
// Outside the grid u is zero; the i_k == 0 slot of u_k is a boundary face.
#include "kernels.h"

namespace ehs {

namespace {

template <typename T>
__device__ __forceinline__ Coef4<T> ldcf(const Coef4<T>* p, long long c) {
  Coef4<T> r;
  if constexpr (sizeof(T) == 4) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p) + c);
    r.mu = v.x; r.kap = v.y; r.mr = v.z; r.mi = v.w;
  } else {
    const double2* q = reinterpret_cast<const double2*>(p) + 2 * c;
    double2 a = __ldg(q), b = __ldg(q + 1);
    r.mu = a.x; r.kap = a.y; r.mr = b.x; r.mi = b.y;
  }
  return r;
}
template <typename C> __device__ __forceinline__ C ldc(const C* p, long long i) { return __ldg(p + i); }

template <typename T> struct FineP {
  T h2inv, hinv, alpha;
};

// value and diagonal of row u_k at the face whose high cell is c (coords i)
template <typename T, int D>
__device__ __forceinline__ typename CT<T>::type row_u(
    const Grid& g, int k, long long c, const int i[3], const Coef4<T>* cf,
    const typename CT<T>::type* xk, const typename CT<T>::type* p, const FineP<T>& P,
    typename CT<T>::type* diag) {
  typedef typename CT<T>::type C;
  const long long sk = stride_of(g, k);
  const Coef4<T> c0 = ldcf(cf, c), c1 = ldcf(cf, c - sk);
  const C xc = ldc(xk, c);
  C xp = czero<C>(), xm = czero<C>();
  if (i[k] + 1 < g.n[k]) xp = ldc(xk, c + sk);
  if (i[k] - 1 >= 1) xm = ldc(xk, c - sk);
  T wsum = c0.mu + c1.mu;
  C nb = cadd(cscale(xp, c0.mu), cscale(xm, c1.mu));
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (j == k) continue;
    const long long sj = stride_of(g, j);
    const bool hp = i[j] + 1 < g.n[j], hm = i[j] - 1 >= 0;
    const long long cp = hp ? c + sj : c, cm = hm ? c - sj : c;
    const T base = c0.mu + c1.mu;
    const T wp = T(0.25) * (base + ldcf(cf, cp).mu + ldcf(cf, cp - sk).mu);
    const T wm = T(0.25) * (base + ldcf(cf, cm).mu + ldcf(cf, cm - sk).mu);
    wsum += wp + wm;
    if (hp) nb = cfma(mk<T>(wp, 0), ldc(xk, c + sj), nb);
    if (hm) nb = cfma(mk<T>(wm, 0), ldc(xk, c - sj), nb);
  }
  const T rf = T(0.5) * (c0.mr + c1.mr), gf = T(0.5) * (c0.mi + c1.mi);
  C dg = mk<T>(wsum * P.h2inv - rf, gf + P.alpha * rf);
  *diag = dg;
  C y = csub(cmul(dg, xc), cscale(nb, P.h2inv));
  const C pc = ldc(p, c), pm = ldc(p, c - sk);
  y = cadd(y, cscale(csub(pc, pm), P.hinv));
  return y;
}

template <typename T, int D>
__device__ __forceinline__ typename CT<T>::type row_p(
    const Grid& g, long long c, const int i[3], const Coef4<T>& c0,
    const typename CT<T>::type* x, const FineP<T>& P) {
  typedef typename CT<T>::type C;
  const long long N = g.ncell;
  C y = cscale(ldc(x + (long long)D * N, c), -c0.kap);
  C s = czero<C>();
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const C* xk = x + (long long)k * N;
    if (i[k] >= 1) s = cadd(s, ldc(xk, c));
    if (i[k] + 1 < g.n[k]) s = csub(s, ldc(xk, c + stride_of(g, k)));
  }
  return cadd(y, cscale(s, P.hinv));
}

template <typename T, int D>
__global__ void k_fine_apply(Grid g, int nrhs, const Coef4<T>* __restrict__ cf, FineP<T> P,
                             const typename CT<T>::type* __restrict__ x,
                             const typename CT<T>::type* __restrict__ b,
                             typename CT<T>::type* __restrict__ y, int mode, const int* __restrict__ il) {
  typedef typename CT<T>::type C;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const long long N = g.ncell;
  const long long vo = (long long)item * (D + 1) * N;
  const Coef4<T>* cs = cf + (long long)(item / nrhs) * N;
  const C* xv = x + vo;
  int i[3];
  cell_coords(g, c, i);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    C r = czero<C>();
    if (i[k] >= 1) {
      C dg;
      r = row_u<T, D>(g, k, c, i, cs, xv + (long long)k * N, xv + (long long)D * N, P, &dg);
      if (mode) r = csub(ldc(b + vo + (long long)k * N, c), r);
    }
    y[vo + (long long)k * N + c] = r;
  }
  C r = row_p<T, D>(g, c, i, ldcf(cs, c), xv, P);
  if (mode) r = csub(ldc(b + vo + (long long)D * N, c), r);
  y[vo + (long long)D * N + c] = r;
}

// One colour of red-black cell-wise Vanka (Sec. 4.2).  Thread = pair of cells
// along x (2t, 2t+1); the one of the requested colour is relaxed, the other
// one's p is copied.  All u faces are written (each face belongs to exactly one
// cell of each colour), so xo is a complete new iterate.
// FULL = false: economic block (eq. RelaxationMatrix: diagonal of the
// displacement block, displacement-pressure couplings, pressure diagonal).
// FULL = true: the whole (2d+1)^2 block of K_s.  On the fine level the only
// displacement couplings inside one cell are between the low and high face of
// the same component, K[u_k(c), u_k(c+e_k)] = -mu_c/h^2 (the normal difference
// across the cell), so the block is an arrowhead with d 2x2 diagonal blocks and
// is solved in closed form through the pressure Schur complement.
template <typename T, int D, bool FULL>
__global__ void k_fine_vanka(Grid g, int nrhs, const Coef4<T>* __restrict__ cf, FineP<T> P,
                             T wu, T wp, int colour, const typename CT<T>::type* __restrict__ b,
                             const typename CT<T>::type* __restrict__ xi,
                             typename CT<T>::type* __restrict__ xo, const int* __restrict__ il) {
  typedef typename CT<T>::type C;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long npair = g.ncell >> 1;
  if (t >= npair) return;
  const int item = il ? il[blockIdx.y] : blockIdx.y;
  const long long N = g.ncell;
  const long long vo = (long long)item * (D + 1) * N;
  const Coef4<T>* cs = cf + (long long)(item / nrhs) * N;
  const C* x = xi + vo;
  const C* bb = b + vo;
  C* xout = xo + vo;
  long long c = 2 * t;
  int i[3];
  cell_coords(g, c, i);
  if (((i[0] + i[1] + i[2]) & 1) != colour) { ++c; ++i[0]; }
  const long long co = ((c & 1) ? c - 1 : c + 1);  // the other cell of the pair
  xout[(long long)D * N + co] = ldc(x + (long long)D * N, co);

  const Coef4<T> c0 = ldcf(cs, c);
  C r[2 * D + 1], dg[2 * D], g_[2 * D];
  bool ok[2 * D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const long long sk = stride_of(g, k);
    const C* xk = x + (long long)k * N;
    const C* pp = x + (long long)D * N;
    ok[k] = i[k] >= 1;
    if (ok[k]) {
      r[k] = csub(ldc(bb + (long long)k * N, c), row_u<T, D>(g, k, c, i, cs, xk, pp, P, &dg[k]));
    } else {
      r[k] = czero<C>(); dg[k] = mk<T>(1, 0);
    }
    g_[k] = mk<T>(P.hinv, 0);            // K[u_k(c), p(c)] = +1/h
    ok[D + k] = i[k] + 1 < g.n[k];
    if (ok[D + k]) {
      int ih[3] = {i[0], i[1], i[2]};
      ih[k] += 1;
      r[D + k] = csub(ldc(bb + (long long)k * N, c + sk),
                      row_u<T, D>(g, k, c + sk, ih, cs, xk, pp, P, &dg[D + k]));
    } else {
      r[D + k] = czero<C>(); dg[D + k] = mk<T>(1, 0);
    }
    g_[D + k] = mk<T>(-P.hinv, 0);       // K[u_k(c+e_k), p(c)] = -1/h
  }
  r[2 * D] = csub(ldc(bb + (long long)D * N, c), row_p<T, D>(g, c, i, c0, x, P));
  if constexpr (FULL) {
    // B = [[A, g], [g^T, -kap]], A = blockdiag_k [[dg_lo, e], [e, dg_hi]], e = -mu_c/h^2.
    // s = A^{-1} r_u, q = A^{-1} g; dp = (r_p - g.s) / (-kap - g.q); du = s - q dp.
    const T e = -c0.mu * P.h2inv;
    C sch = mk<T>(-c0.kap, 0);
    C rp = r[2 * D];
    C sv[2 * D], qv[2 * D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int lo = k, hi = D + k;
      if (ok[lo] && ok[hi]) {
        const C det = csub(cmul(dg[lo], dg[hi]), mk<T>(e * e, 0));
        const C di = cinv(det);
        sv[lo] = cmul(di, csub(cmul(dg[hi], r[lo]), cscale(r[hi], e)));
        sv[hi] = cmul(di, csub(cmul(dg[lo], r[hi]), cscale(r[lo], e)));
        qv[lo] = cmul(di, csub(cmul(dg[hi], g_[lo]), cscale(g_[hi], e)));
        qv[hi] = cmul(di, csub(cmul(dg[lo], g_[hi]), cscale(g_[lo], e)));
      } else {
#pragma unroll
        for (int a = lo; a <= hi; a += D) {
          if (!ok[a]) { sv[a] = czero<C>(); qv[a] = czero<C>(); continue; }
          const C dinv = cinv(dg[a]);
          sv[a] = cmul(r[a], dinv);
          qv[a] = cmul(g_[a], dinv);
        }
      }
#pragma unroll
      for (int a = lo; a <= hi; a += D) {
        if (!ok[a]) continue;
        sch = csub(sch, cmul(g_[a], qv[a]));
        rp = csub(rp, cmul(g_[a], sv[a]));
      }
    }
    const C dp = cmul(rp, cinv(sch));
    xout[(long long)D * N + c] = cfma(mk<T>(wp, 0), dp, ldc(x + (long long)D * N, c));
#pragma unroll
    for (int a = 0; a < 2 * D; ++a) {
      if (!ok[a]) continue;
      const int k = a % D;
      const long long idx = (long long)k * N + c + (a >= D ? stride_of(g, k) : 0);
      const C du = csub(sv[a], cmul(qv[a], dp));
      xout[idx] = cfma(mk<T>(wu, 0), du, ldc(x, idx));
    }
    return;
  }
  // economic arrowhead solve: B = [[diag(dg), g], [g^T, -kap]]
  C sch = mk<T>(-c0.kap, 0);
  C rp = r[2 * D];
  C dinv[2 * D];
#pragma unroll
  for (int a = 0; a < 2 * D; ++a) {
    if (!ok[a]) continue;
    dinv[a] = cinv(dg[a]);
    const C gd = cmul(g_[a], dinv[a]);
    sch = csub(sch, cmul(gd, g_[a]));
    rp = csub(rp, cmul(gd, r[a]));
  }
  const C dp = cmul(rp, cinv(sch));
  xout[(long long)D * N + c] = cfma(mk<T>(wp, 0), dp, ldc(x + (long long)D * N, c));
#pragma unroll
  for (int a = 0; a < 2 * D; ++a) {
    if (!ok[a]) continue;
    const int k = a % D;
    const long long idx = (long long)k * N + c + (a >= D ? stride_of(g, k) : 0);
    const C du = cmul(csub(r[a], cmul(g_[a], dp)), dinv[a]);
    xout[idx] = cfma(mk<T>(wu, 0), du, ldc(x, idx));
  }
}

// The same economic half-sweep for 2D complex64, staged through shared memory:
// a CTA owns a VT_X x VT_Y tile of cells of one item, loads u_0, u_1, p and
// the coefficients of the tile plus a 2-cell halo once (coalesced), and each
// thread relaxes the colour cell of one x-pair from shared memory.  Outside
// the grid the displacements read 0 (the Dirichlet slots and the implicit high
// boundary faces) and the coefficients repeat the nearest cell (the clamped
// edge averages), so the rows need no per-load bounds checks; the arithmetic
// is that of k_fine_vanka term by term.
constexpr int VT_X = 32, VT_Y = 8, VT_H = 2;
constexpr int VS_X = VT_X + 2 * VT_H, VS_Y = VT_Y + 2 * VT_H;

// asynchronous global -> shared copies (cp.async): all of a thread's staging
// loads are in flight at once; nbytes = 0 fills the destination with zeros
// (the source address is then not read, but is kept valid all the same)
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int nbytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__global__ void __launch_bounds__(VT_X * VT_Y / 2) k_fine_vanka_tile(Grid g, int nrhs, const Coef4<float>* __restrict__ cf,
                                                                     FineP<float> P, float wu, float wp, int colour,
                                                                     const float2* __restrict__ b,
                                                                     const float2* __restrict__ xi,
                                                                     float2* __restrict__ xo, const int* __restrict__ il) {
  __shared__ __align__(16) float2 xs[3][VS_Y][VS_X];
  __shared__ __align__(16) float4 cs[VS_Y][VS_X];
  const int item = il ? il[blockIdx.z] : blockIdx.z;
  const long long N = g.ncell;
  const int nx = g.n[0], ny = g.n[1];
  const long long vo = (long long)item * 3 * N;
  const float4* cfs = reinterpret_cast<const float4*>(cf + (long long)(item / nrhs) * N);
  const float2* x = xi + vo;
  const int x0 = blockIdx.x * VT_X - VT_H, y0 = blockIdx.y * VT_Y - VT_H;
  for (int idx = threadIdx.x; idx < VS_X * VS_Y; idx += blockDim.x) {
    const int lx = idx % VS_X, ly = idx / VS_X;
    const int gx = x0 + lx, gy = y0 + ly;
    const bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
    const int cx = min(max(gx, 0), nx - 1), cy = min(max(gy, 0), ny - 1);
    const long long gc = (long long)cy * nx + cx;                  // a valid address in every case
    cp_async8(&xs[0][ly][lx], x + gc, (in && gx >= 1) ? 8 : 0);    // u_0 slot 0 is a boundary face
    cp_async8(&xs[1][ly][lx], x + N + gc, (in && gy >= 1) ? 8 : 0);  // u_1 slot 0 likewise
    cp_async8(&xs[2][ly][lx], x + 2 * N + gc, in ? 8 : 0);
    cp_async16(&cs[ly][lx], cfs + gc);                              // clamped: the edge averages' rule
  }
  cp_async_wait_all();
  __syncthreads();
  const int t = threadIdx.x;
  int lx = 2 * (t % (VT_X / 2)), ly = t / (VT_X / 2);
  int i0 = blockIdx.x * VT_X + lx, i1 = blockIdx.y * VT_Y + ly;
  if (((i0 + i1) & 1) != colour) { ++lx; ++i0; }
  const int sx = lx + VT_H, sy = ly + VT_H;                        // the colour cell in shared memory
  const int ox = ((lx & 1) ? lx - 1 : lx + 1) + VT_H;              // the other cell of the pair
  const long long c = (long long)i1 * nx + i0;
  const long long co = (long long)i1 * nx + (((i0 & 1) ? i0 - 1 : i0 + 1));
  const float2* bb = b + vo;
  float2* xout = xo + vo;
  xout[2 * N + co] = xs[2][sy][ox];
  const float4 cc = cs[sy][sx];
  // row of u_k at the face whose high cell is (ax, ay) (smem coordinates), diagonal in *dg
  auto row_u = [&](int k, int ax, int ay, float2* dg) -> float2 {
    const int ex = k == 0, ey = k == 1;
    const float4 c0 = cs[ay][ax], c1 = cs[ay - ey][ax - ex];
    const float2 xc = xs[k][ay][ax];
    const float2 xp = xs[k][ay + ey][ax + ex], xm = xs[k][ay - ey][ax - ex];
    float wsum = c0.x + c1.x;
    float2 nb = cadd(cscale(xp, c0.x), cscale(xm, c1.x));
    const int jx = 1 - ex, jy = 1 - ey;                             // the tangential direction
    const float base = c0.x + c1.x;
    const float wpl = 0.25f * (base + cs[ay + jy][ax + jx].x + cs[ay + jy - ey][ax + jx - ex].x);
    const float wmi = 0.25f * (base + cs[ay - jy][ax - jx].x + cs[ay - jy - ey][ax - jx - ex].x);
    wsum += wpl + wmi;
    nb = cfma(make_float2(wpl, 0.f), xs[k][ay + jy][ax + jx], nb);
    nb = cfma(make_float2(wmi, 0.f), xs[k][ay - jy][ax - jx], nb);
    const float rf = 0.5f * (c0.z + c1.z), gf = 0.5f * (c0.w + c1.w);
    const float2 d = make_float2(wsum * P.h2inv - rf, gf + P.alpha * rf);
    *dg = d;
    float2 y = csub(cmul(d, xc), cscale(nb, P.h2inv));
    return cadd(y, cscale(csub(xs[2][ay][ax], xs[2][ay - ey][ax - ex]), P.hinv));
  };
  const int ic[2] = {i0, i1}, nn[2] = {nx, ny};
  float2 r[5], dg[4], g_[4];
  bool ok[4];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const long long sk = k == 0 ? 1 : nx;
    ok[k] = ic[k] >= 1;
    if (ok[k]) r[k] = csub(__ldg(bb + (long long)k * N + c), row_u(k, sx, sy, &dg[k]));
    else { r[k] = make_float2(0.f, 0.f); dg[k] = make_float2(1.f, 0.f); }
    g_[k] = make_float2(P.hinv, 0.f);
    ok[2 + k] = ic[k] + 1 < nn[k];
    if (ok[2 + k]) r[2 + k] = csub(__ldg(bb + (long long)k * N + c + sk), row_u(k, sx + (k == 0), sy + (k == 1), &dg[2 + k]));
    else { r[2 + k] = make_float2(0.f, 0.f); dg[2 + k] = make_float2(1.f, 0.f); }
    g_[2 + k] = make_float2(-P.hinv, 0.f);
  }
  {   // pressure row: -kap p + (div u) / h
    float2 y = cscale(xs[2][sy][sx], -cc.y);
    float2 sdiv = make_float2(0.f, 0.f);
    sdiv = cadd(sdiv, xs[0][sy][sx]);
    sdiv = csub(sdiv, xs[0][sy][sx + 1]);
    sdiv = cadd(sdiv, xs[1][sy][sx]);
    sdiv = csub(sdiv, xs[1][sy + 1][sx]);
    r[4] = csub(__ldg(bb + 2 * N + c), cadd(y, cscale(sdiv, P.hinv)));
  }
  float2 sch = make_float2(-cc.y, 0.f);
  float2 rp = r[4];
  float2 dinv[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (!ok[a]) continue;
    dinv[a] = cinv(dg[a]);
    const float2 gd = cmul(g_[a], dinv[a]);
    sch = csub(sch, cmul(gd, g_[a]));
    rp = csub(rp, cmul(gd, r[a]));
  }
  const float2 dp = cmul(rp, cinv(sch));
  xout[2 * N + c] = cfma(make_float2(wp, 0.f), dp, xs[2][sy][sx]);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (!ok[a]) continue;
    const int k = a % 2;
    const long long idx = (long long)k * N + c + (a >= 2 ? (k == 0 ? 1 : nx) : 0);
    const float2 xv = xs[k][sy + (a >= 2 && k == 1)][sx + (a >= 2 && k == 0)];
    const float2 du = cmul(csub(r[a], cmul(g_[a], dp)), dinv[a]);
    xout[idx] = cfma(make_float2(wu, 0.f), du, xv);
  }
}

__device__ __forceinline__ double abl_ramp(const Grid& g, const int i[3], int L) {
  if (L <= 0) return 0.0;
  double r = 0.0;
  for (int k = 0; k < g.d; ++k) {
    int dep = max(max(L - i[k], i[k] - (g.n[k] - 1 - L)), 0);
    double t = (double)dep / L;
    r = fmax(r, t * t);
  }
  return r;
}

template <typename T>
__global__ void k_fine_coef(Grid g, const double* lam, const double* mu, const double* rho,
                            const double* omegas, int L, double abl_max, double gamma_add,
                            Coef4<T>* out) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const long long o = (long long)blockIdx.y * g.ncell + c;
  const double omega = omegas[blockIdx.y];
  int i[3];
  cell_coords(g, c, i);
  const double gam = gamma_add + omega * abl_max * abl_ramp(g, i, L);
  Coef4<T> r;
  r.mu = (T)mu[o];
  r.kap = (T)(1.0 / (lam[o] + mu[o]));
  r.mr = (T)(omega * omega * rho[o]);
  r.mi = (T)(omega * rho[o] * gam);
  out[o] = r;
}

template <typename T>
__global__ void k_coef_cast(long long n, const Coef4<double>* in, Coef4<T>* out) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  Coef4<double> v = in[c];
  Coef4<T> r;
  r.mu = (T)v.mu; r.kap = (T)v.kap; r.mr = (T)v.mr; r.mi = (T)v.mi;
  out[c] = r;
}

// Subdomain coefficients (Algorithm DD, padded subdomains with an absorbing
// layer in the padding).  blockIdx.y = subdomain-set index.
template <typename T>
__global__ void k_sub_coef(Grid gl, Grid gg, int nsub, const int* origin, const int* omlo,
                           const int* omhi, const int* padlo, const int* padhi, const int* subset,
                           const Coef4<double>* glob, double ddabl, Coef4<T>* out) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= gl.ncell) return;
  const int s = blockIdx.y;            // = set * nsub + sub
  const int sub = s % nsub;
  const int gset = subset[s];
  int i[3], gi[3];
  cell_coords(gl, c, i);
  double ramp = 0.0;
  for (int k = 0; k < 3; ++k) {
    int gk = origin[sub * 3 + k] + i[k];
    gk = min(max(gk, omlo[sub * 3 + k]), omhi[sub * 3 + k] - 1);
    gi[k] = gk;
    if (k < gl.d) {
      const int plo = padlo[sub * 3 + k], phi = padhi[sub * 3 + k];
      const int ext = omhi[sub * 3 + k] - omlo[sub * 3 + k];
      double dep = 0.0;
      if (plo && i[k] < plo) dep = (double)(plo - i[k]) / plo;
      if (phi && i[k] >= plo + ext) dep = (double)(i[k] - (plo + ext) + 1) / phi;
      ramp = fmax(ramp, dep * dep);
    }
  }
  Coef4<double> v = glob[(long long)gset * gg.ncell + cell_index(gg, gi)];
  Coef4<T> r;
  r.mu = (T)v.mu; r.kap = (T)v.kap; r.mr = (T)v.mr;
  r.mi = (T)(v.mi + v.mr * ddabl * ramp);   // omega rho (gamma + omega*ddabl*ramp)
  out[(long long)s * gl.ncell + c] = r;
}

// level-0 stencil table of K_s (double), layout from fine_table_layout
template <int D>
__global__ void k_fine_table(Grid g, const Coef4<double>* __restrict__ cf, FineP<double> P,
                             StencilLayout L, double2* __restrict__ tab) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const long long N = g.ncell;
  const int set = blockIdx.y;
  const Coef4<double>* cs = cf + (long long)set * N;
  double2* T0 = tab + (long long)set * L.nslot * N;
  for (int q = 0; q < L.nslot; ++q) T0[(long long)q * N + c] = make_double2(0, 0);
  int i[3];
  cell_coords(g, c, i);
  const Coef4<double> c0 = cs[c];
  for (int k = 0; k < D; ++k) {
    if (i[k] < 1) continue;
    const long long sk = stride_of(g, k);
    const Coef4<double> c1 = cs[c - sk];
    int o[3] = {0, 0, 0};
    double wsum = c0.mu + c1.mu;
    // normal neighbours
    if (i[k] + 1 < g.n[k]) { o[k] = 1; T0[(long long)st_slot(L, k, k, o[0], o[1], o[2]) * N + c].x = -c0.mu * P.h2inv; }
    if (i[k] - 1 >= 1) { o[k] = -1; T0[(long long)st_slot(L, k, k, o[0], o[1], o[2]) * N + c].x = -c1.mu * P.h2inv; }
    o[k] = 0;
    for (int j = 0; j < D; ++j) {
      if (j == k) continue;
      const long long sj = stride_of(g, j);
      const bool hp = i[j] + 1 < g.n[j], hm = i[j] - 1 >= 0;
      const long long cp = hp ? c + sj : c, cm = hm ? c - sj : c;
      const double base = c0.mu + c1.mu;
      const double wp = 0.25 * (base + cs[cp].mu + cs[cp - sk].mu);
      const double wm = 0.25 * (base + cs[cm].mu + cs[cm - sk].mu);
      wsum += wp + wm;
      if (hp) { o[j] = 1; T0[(long long)st_slot(L, k, k, o[0], o[1], o[2]) * N + c].x = -wp * P.h2inv; }
      if (hm) { o[j] = -1; T0[(long long)st_slot(L, k, k, o[0], o[1], o[2]) * N + c].x = -wm * P.h2inv; }
      o[j] = 0;
    }
    const double rf = 0.5 * (c0.mr + c1.mr), gf = 0.5 * (c0.mi + c1.mi);
    T0[(long long)st_slot(L, k, k, 0, 0, 0) * N + c] =
        make_double2(wsum * P.h2inv - rf, gf + P.alpha * rf);
    T0[(long long)st_slot(L, k, D, 0, 0, 0) * N + c].x = P.hinv;
    o[k] = -1;
    T0[(long long)st_slot(L, k, D, o[0], o[1], o[2]) * N + c].x = -P.hinv;
  }
  for (int k = 0; k < D; ++k) {
    if (i[k] >= 1) T0[(long long)st_slot(L, D, k, 0, 0, 0) * N + c].x = P.hinv;
    if (i[k] + 1 < g.n[k]) {
      int o[3] = {0, 0, 0};
      o[k] = 1;
      T0[(long long)st_slot(L, D, k, o[0], o[1], o[2]) * N + c].x = -P.hinv;
    }
  }
  T0[(long long)st_slot(L, D, D, 0, 0, 0) * N + c].x = -c0.kap;
}

template <typename T> FineP<T> mkP(double h, double alpha) {
  FineP<T> P;
  P.h2inv = (T)(1.0 / (h * h));
  P.hinv = (T)(1.0 / h);
  P.alpha = (T)alpha;
  return P;
}

inline dim3 grid1(long long n, int items, int bs) { return dim3((unsigned)((n + bs - 1) / bs), items, 1); }

}  // namespace

template <typename T>
void launch_fine_coef(const Grid& g, int nsets, const double* lam, const double* mu,
                      const double* rho, const double* omegas, int abl_cells, double abl_max,
                      double gamma_add, Coef4<T>* out, cudaStream_t s) {
  k_fine_coef<T><<<grid1(g.ncell, nsets, 256), 256, 0, s>>>(g, lam, mu, rho, omegas, abl_cells,
                                                             abl_max, gamma_add, out);
}

template <typename T>
void launch_sub_coef(const Grid& gl, const Grid& gg, int nsets_glob, int nsub, const int* d_origin,
                     const int* d_omlo, const int* d_omhi, const int* d_padlo, const int* d_padhi,
                     const int* d_subset, const Coef4<double>* glob, double ddabl,
                     Coef4<T>* out, cudaStream_t s) {
  k_sub_coef<T><<<grid1(gl.ncell, nsets_glob * nsub, 256), 256, 0, s>>>(
      gl, gg, nsub, d_origin, d_omlo, d_omhi, d_padlo, d_padhi, d_subset, glob, ddabl, out);
}

template <typename T>
void launch_coef_cast(long long n, const Coef4<double>* in, Coef4<T>* out, cudaStream_t s) {
  k_coef_cast<T><<<grid1(n, 1, 256), 256, 0, s>>>(n, in, out);
}

template <typename T>
void launch_fine_apply(const Grid& g, int items, int nrhs, const Coef4<T>* cf, double h,
                       double alpha, const typename CT<T>::type* x,
                       const typename CT<T>::type* b, typename CT<T>::type* y, int mode,
                       cudaStream_t s) {
  const FineP<T> P = mkP<T>(h, alpha);
  const dim3 gr((unsigned)((g.ncell + 255) / 256), sel_items(items));
  if (g.d == 2)
    k_fine_apply<T, 2><<<gr, 256, 0, s>>>(g, nrhs, cf, P, x, b, y, mode, g_sel.list);
  else
    k_fine_apply<T, 3><<<gr, 256, 0, s>>>(g, nrhs, cf, P, x, b, y, mode, g_sel.list);
}

template <typename T>
void launch_fine_vanka(const Grid& g, int items, int nrhs, const Coef4<T>* cf, double h,
                       double alpha, T wu, T wp, int colour,
                       const typename CT<T>::type* b, const typename CT<T>::type* xi,
                       typename CT<T>::type* xo, cudaStream_t s, int full) {
  const FineP<T> P = mkP<T>(h, alpha);
  if constexpr (sizeof(T) == 4) {
    if (g.d == 2 && !full && g.n[0] % VT_X == 0 && g.n[1] % VT_Y == 0) {   // shared-memory tiles
      const dim3 gt(g.n[0] / VT_X, g.n[1] / VT_Y, sel_items(items));
      k_fine_vanka_tile<<<gt, VT_X * VT_Y / 2, 0, s>>>(g, nrhs, cf, P, wu, wp, colour, b, xi, xo, g_sel.list);
      return;
    }
  }
  const long long np = g.ncell / 2;
  const dim3 gr((unsigned)((np + 127) / 128), sel_items(items));
  if (g.d == 2) {
    if (full) k_fine_vanka<T, 2, true><<<gr, 128, 0, s>>>(g, nrhs, cf, P, wu, wp, colour, b, xi, xo, g_sel.list);
    else k_fine_vanka<T, 2, false><<<gr, 128, 0, s>>>(g, nrhs, cf, P, wu, wp, colour, b, xi, xo, g_sel.list);
  } else {
    if (full) k_fine_vanka<T, 3, true><<<gr, 128, 0, s>>>(g, nrhs, cf, P, wu, wp, colour, b, xi, xo, g_sel.list);
    else k_fine_vanka<T, 3, false><<<gr, 128, 0, s>>>(g, nrhs, cf, P, wu, wp, colour, b, xi, xo, g_sel.list);
  }
}

void fine_table_layout(int d, StencilLayout* L) { *L = make_fine_layout(d); }

void launch_fine_table(const Grid& g, int nsets, const Coef4<double>* cf, double h,
                       double alpha, const StencilLayout& L, double2* tab, cudaStream_t s) {
  const FineP<double> P = mkP<double>(h, alpha);
  if (g.d == 2)
    k_fine_table<2><<<grid1(g.ncell, nsets, 128), 128, 0, s>>>(g, cf, P, L, tab);
  else
    k_fine_table<3><<<grid1(g.ncell, nsets, 128), 128, 0, s>>>(g, cf, P, L, tab);
}

#define INST(T)                                                                                  \
  template void launch_fine_coef<T>(const Grid&, int, const double*, const double*, const double*, \
                                    const double*, int, double, double, Coef4<T>*, cudaStream_t);  \
  template void launch_sub_coef<T>(const Grid&, const Grid&, int, int, const int*, const int*,     \
                                   const int*, const int*, const int*, const int*,                 \
                                   const Coef4<double>*, double, Coef4<T>*, cudaStream_t);         \
  template void launch_coef_cast<T>(long long, const Coef4<double>*, Coef4<T>*, cudaStream_t);     \
  template void launch_fine_apply<T>(const Grid&, int, int, const Coef4<T>*, double,              \
                                     double, const CT<T>::type*, const CT<T>::type*,              \
                                     CT<T>::type*, int, cudaStream_t);                             \
  template void launch_fine_vanka<T>(const Grid&, int, int, const Coef4<T>*, double,              \
                                     double, T, T, int, const CT<T>::type*, const CT<T>::type*,    \
                                     CT<T>::type*, cudaStream_t, int);
INST(float)
INST(double)
#undef INST

}  // namespace ehs
