// Fused fine-level kernels of the 2D complex64 cycle (economic cell-wise
// Vanka, Sec. 3 and Sec. 4.2; Algorithm TwoCycle steps 2 and 4 of Sec. 2.2).
//
// k_fine_sweep_tile: one whole red-black sweep in one launch.  A CTA owns a
//   SW_X x SW_Y tile of fine cells of one item and stages x (u_0, u_1, p) and
//   the coefficient terms of the tile plus a halo (2 cells below, 3 above) in
//   shared memory.  It
//   relaxes every red cell of the tile and of the one-cell ring around it from
//   the staged iterate (all red updates from the same old iterate, as in the
//   red half-sweep), applies them in shared memory, then relaxes the black
//   cells of the tile and writes the new iterate.  Every interior face belongs
//   to exactly one black cell, whose CTA writes it; each CTA writes the
//   pressures of its tile and zeros on its Dirichlet slots, so the output is a
//   complete iterate.  The staged x is either the input iterate, zero (a zero
//   initial guess: pre-smoothing of a cycle, no read of x), or the input
//   iterate plus the prolongated coarse correction P e_c (Algorithm TwoCycle
//   step 4 folded into the first post-smoothing sweep).
// k_fine_resid_restrict_tile: r_c = P^T (b - K_s x) in one pass.  A CTA stages
//   x and the coefficients of a RR_X x RR_Y fine tile plus a 2-cell halo,
//   evaluates the fine residual on the tile plus a one-cell ring into shared
//   memory, and forms the restriction of the tile's coarse cells from there;
//   the fine residual is never written to memory.
//
// The row arithmetic is that of k_fine_apply / k_fine_vanka, with the
// quantities that depend on the coefficients alone formed once instead of once
// per use: the mean of mu over the 4 cells around each vertex (the tangential
// weight of the two face rows that meet there), the diagonal of each face row
// (residual kernel: per staged tile) or its inverse, and the inverse pressure
// Schur complement of each relaxed cell's arrowhead block (eq.
// RelaxationMatrix; sweep: setup-time tables); weights carry the 1/h^2
// factor.  Outside the
// grid the displacements read zero (Dirichlet slots and the implicit high
// boundary faces) and the coefficients repeat the nearest cell (the clamped
// edge averages), so the rows need no per-load bounds checks.  Each cell update
// loads every neighbouring value it needs once.
#include "kernels.h"

namespace ehs {
namespace {

constexpr int SW_X = 32, SW_Y = 16, SW_H = 2;                 // sweep tile, staged halo below it
constexpr int SWS_X = SW_X + 2 * SW_H + 2, SWS_Y = SW_Y + 2 * SW_H + 1;   // and one (x: two) more above
// A warp relaxes the cells of one colour in a pair of rows, lane j the cell of column j (in
// the row of the pair where it has that colour).  With an even row pitch the staged words
// the 32 lanes read at any one offset then fall in 32 different banks (16 different 8-byte
// bank pairs per half warp for the complex values), where lanes two columns apart in one row
// would meet in pairs.
static_assert(SWS_X % 2 == 0, "even staged row pitch");
constexpr int SW_RX = SW_X + 2, SW_RY = SW_Y + 2;             // red region: tile + one-cell ring
constexpr int SW_NRED = SW_RX * SW_RY / 2;                    // 306 red cells
constexpr int SW_TB = SW_X * SW_Y / 2;                        // 256 black cells: one per thread
constexpr int SW_T = 320;                                     // 10 warps: every red cell in one round
constexpr int SW_RPT = (SW_NRED + SW_T - 1) / SW_T;           // red cells per thread (1)
static_assert(SW_T >= SW_TB && SW_T % 32 == 0, "sweep threads");

constexpr int RR_X = 32, RR_Y = 16, RR_H = 2;                 // residual + restriction tile
constexpr int RRS_X = RR_X + 2 * RR_H, RRS_Y = RR_Y + 2 * RR_H;
constexpr int RR_RX = RR_X + 2, RR_RY = RR_Y + 2;             // fine residual region
constexpr int RR_T = 256;                                     // 8 warps (10 measured slower here)
constexpr int RR_RPT = (RR_RX * RR_RY + RR_T - 1) / RR_T;     // residual cells per thread (3)
static_assert(RR_T >= RR_X * RR_Y / 2, "one restriction output per thread");

static_assert(SW_X % 2 == 0 && RR_X % 4 == 0 && RR_Y % 2 == 0, "tile shapes");

struct FP {
  float h2inv, hinv, alpha;
};

// Staged tile of W x H cells (local (lx, ly) = global (x0 + lx, y0 + ly)).
//   x:   u_0, u_1, p (zero outside the grid and on Dirichlet slots)
//   mu:  cell mu / h^2 (clamped outside the grid); kap: cell 1/(lambda+mu)
//   mm:  (sweep tile) the inverse Schur complement 1/(-kap - sum_faces (1/h^2) / dg)
//        of the cell's block
//   vm:  vm[ly][lx] = mean of mu / h^2 over cells (lx-1..lx, ly-1..ly), the
//        vertex at the low corner of cell (lx, ly)
//   fx / fy: per face of u_0 (between cells lx-1 and lx) / u_1 (between cells
//        ly-1 and ly) the diagonal dg of its row (residual tile) or its inverse
//        (sweep tile: the cell solve needs only 1/dg).  mm, vm, fx and fy come
//        from the setup-time tables.
template <int W, int H>
struct Tile {
  float2 x[3][H][W];
  float mu[H][W], kap[H][W], vm[H][W];
  float2 mm[H][W];
  float2 fx[H][W], fy[H][W];
};

__device__ __forceinline__ void cpa8(void* dst, const void* src, int nbytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void cpa4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// (P e_c) of component a at fine cell (gx, gy): coarse item vector ec ([3][ncc])
__device__ __forceinline__ float2 prolong_at(const float2* __restrict__ ec, int a, int gx, int gy, int ncx,
                                             int ncy) {
  const int kx = a == 2 ? 2 : (a == 0 ? 0 : 1);
  const int ky = a == 2 ? 2 : (a == 1 ? 0 : 1);
  int X0, X1, Y0, Y1;
  float wx0, wx1, wy0, wy1;
  pw_pair<float>(kx, gx, ncx, X0, wx0, X1, wx1);
  pw_pair<float>(ky, gy, ncy, Y0, wy0, Y1, wy1);
  const float2* e = ec + (long long)a * ncx * ncy;
  float2 acc = make_float2(0.f, 0.f);
  if (wy0 != 0.0f) {
    const float2* row = e + (long long)Y0 * ncx;
    if (wx0 != 0.0f) acc = cfma(make_float2(wy0 * wx0, 0.f), __ldg(row + X0), acc);
    if (wx1 != 0.0f) acc = cfma(make_float2(wy0 * wx1, 0.f), __ldg(row + X1), acc);
  }
  if (wy1 != 0.0f) {
    const float2* row = e + (long long)Y1 * ncx;
    if (wx0 != 0.0f) acc = cfma(make_float2(wy1 * wx0, 0.f), __ldg(row + X0), acc);
    if (wx1 != 0.0f) acc = cfma(make_float2(wy1 * wx1, 0.f), __ldg(row + X1), acc);
  }
  return acc;
}

// The coefficient terms of the rows, formed into the setup-time tables below: the
// mean of mu / h^2 over the four cells around a vertex, and the diagonal of a
// face row from the mu / h^2 of its two cells, the vertex means at its two ends and
// the two cells' (omega^2 rho, omega rho gamma).
__device__ __forceinline__ float vertex_mean(float m00, float m01, float m10, float m11) {
  return 0.25f * ((m00 + m01) + m10 + m11);
}
__device__ __forceinline__ float2 face_diag(float mu0, float mu1, float vhi, float vlo, float2 m0, float2 m1,
                                            float alpha) {
  const float wsum = (mu0 + mu1) + vhi + vlo;
  const float rf = 0.5f * (m0.x + m1.x), gf = 0.5f * (m0.y + m1.y);
  return make_float2(wsum - rf, gf + alpha * rf);
}

// Setup-time tables of the fused kernels, per medium: the diagonals of each cell's
// low u_0 and u_1 face rows (gdx, gdy, [ncell]) and their inverses (dvx, dvy), the
// inverse pressure Schur
// complement of each cell's block (sinv, [ncell]) and the vertex means of mu / h^2
// (vm, [(nx + 1) (ny + 1)], vertex (vx, vy) the low corner of cell (vx, vy)).  The
// clamped coefficients outside the grid (the clamped edge averages), formed once
// instead of in every sweep; entries on Dirichlet faces are formed but never used.
__device__ __forceinline__ float mu_cl(const float4* cfs, int gx, int gy, int nx, int ny, float h2inv) {
  return __ldg(cfs + min(max(gy, 0), ny - 1) * nx + min(max(gx, 0), nx - 1)).x * h2inv;
}
__device__ __forceinline__ float2 mm_cl(const float4* cfs, int gx, int gy, int nx, int ny) {
  const float4 c = __ldg(cfs + min(max(gy, 0), ny - 1) * nx + min(max(gx, 0), nx - 1));
  return make_float2(c.z, c.w);
}
__device__ __forceinline__ float vm_cl(const float4* cfs, int vx, int vy, int nx, int ny, float h2inv) {
  return vertex_mean(mu_cl(cfs, vx, vy, nx, ny, h2inv), mu_cl(cfs, vx - 1, vy, nx, ny, h2inv),
                     mu_cl(cfs, vx, vy - 1, nx, ny, h2inv), mu_cl(cfs, vx - 1, vy - 1, nx, ny, h2inv));
}
__global__ void k_sweep_tables_faces(Grid g, const float4* __restrict__ cf, FP P, float2* __restrict__ dvx,
                                     float2* __restrict__ dvy, float2* __restrict__ gdx, float2* __restrict__ gdy,
                                     float* __restrict__ vm) {
  const int nx = g.n[0], ny = g.n[1];
  const int nv = (nx + 1) * (ny + 1);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv) return;
  const int set = blockIdx.y;
  const float4* cfs = cf + (long long)set * g.ncell;
  const int vx = t % (nx + 1), vy = t / (nx + 1);
  const float h2 = P.h2inv;
  vm[(long long)set * nv + t] = vm_cl(cfs, vx, vy, nx, ny, h2);
  if (vx >= nx || vy >= ny) return;
  const long long c = (long long)set * g.ncell + vy * nx + vx;
  const float mc = mu_cl(cfs, vx, vy, nx, ny, h2), v00 = vm_cl(cfs, vx, vy, nx, ny, h2);
  const float2 m0 = mm_cl(cfs, vx, vy, nx, ny);
  const float2 dx = face_diag(mc, mu_cl(cfs, vx - 1, vy, nx, ny, h2), vm_cl(cfs, vx, vy + 1, nx, ny, h2), v00, m0,
                              mm_cl(cfs, vx - 1, vy, nx, ny), P.alpha);
  const float2 dy = face_diag(mc, mu_cl(cfs, vx, vy - 1, nx, ny, h2), vm_cl(cfs, vx + 1, vy, nx, ny, h2), v00, m0,
                              mm_cl(cfs, vx, vy - 1, nx, ny), P.alpha);
  gdx[c] = dx;
  gdy[c] = dy;
  dvx[c] = cinv(dx);
  dvy[c] = cinv(dy);
}
__global__ void k_sweep_tables_schur(Grid g, const float4* __restrict__ cf, FP P, const float2* __restrict__ dvx,
                                     const float2* __restrict__ dvy, float2* __restrict__ sinv) {
  const int nx = g.n[0], ny = g.n[1];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.ncell) return;
  const long long c = (long long)blockIdx.y * g.ncell + t;
  const int gx = t % nx, gy = t / nx;
  float2 sd = make_float2(0.f, 0.f);                               // sum of the faces' 1/dg
  if (gx >= 1) sd = cadd(sd, dvx[c]);
  if (gx + 1 < nx) sd = cadd(sd, dvx[c + 1]);
  if (gy >= 1) sd = cadd(sd, dvy[c]);
  if (gy + 1 < ny) sd = cadd(sd, dvy[c + nx]);
  const float kap = __ldg(cf + c).y;
  sinv[c] = cinv(make_float2(-kap - P.h2inv * sd.x, -P.h2inv * sd.y));
}

// Stage the tile (x0, y0) of x: from xv (null: the zero iterate), plus P e when e is
// given, zero outside the grid and on Dirichlet slots; with mu / h^2 and
// 1/(lambda+mu) of the (clamped) cells and the setup-time tables: fx, fy the
// face diagonals or their inverses (tx, ty), mm the inverse Schur complements (ts;
// not staged when null), vm the vertex means (tv).
template <int W, int H, int NT>
__device__ __forceinline__ void stage_tab(Tile<W, H>& S, const float4* __restrict__ cfs, const float2* __restrict__ tx,
                                          const float2* __restrict__ ty, const float2* __restrict__ ts,
                                          const float* __restrict__ tv, const float2* __restrict__ xv,
                                          const float2* __restrict__ e, const Grid& gc, int N, int nx, int ny,
                                          int x0, int y0, float h2inv) {
#pragma unroll 4
  for (int idx = threadIdx.x; idx < W * H; idx += NT) {
    const int lx = idx % W, ly = idx / W;
    const int gx = x0 + lx, gy = y0 + ly;
    const bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
    const int cx = min(max(gx, 0), nx - 1), cy = min(max(gy, 0), ny - 1);
    const int gcl = cy * nx + cx;                                  // a valid address in every case
    const bool v0 = in && gx >= 1, v1 = in && gy >= 1;            // u_k slot 0 is a boundary face
    if (!e) {
      if (xv) {
        cpa8(&S.x[0][ly][lx], xv + gcl, v0 ? 8 : 0);
        cpa8(&S.x[1][ly][lx], xv + N + gcl, v1 ? 8 : 0);
        cpa8(&S.x[2][ly][lx], xv + 2 * N + gcl, in ? 8 : 0);
      } else {
        const float2 z = make_float2(0.f, 0.f);
        S.x[0][ly][lx] = z; S.x[1][ly][lx] = z; S.x[2][ly][lx] = z;
      }
    } else {
      float2 u0 = make_float2(0.f, 0.f), u1 = u0, pv = u0;
      if (v0) u0 = cadd(xv ? __ldg(xv + gcl) : u0, prolong_at(e, 0, gx, gy, gc.n[0], gc.n[1]));
      if (v1) u1 = cadd(xv ? __ldg(xv + N + gcl) : u1, prolong_at(e, 1, gx, gy, gc.n[0], gc.n[1]));
      if (in) pv = cadd(xv ? __ldg(xv + 2 * N + gcl) : pv, prolong_at(e, 2, gx, gy, gc.n[0], gc.n[1]));
      S.x[0][ly][lx] = u0; S.x[1][ly][lx] = u1; S.x[2][ly][lx] = pv;
    }
    cpa8(&S.fx[ly][lx], tx + gcl, 8);
    cpa8(&S.fy[ly][lx], ty + gcl, 8);
    if (ts) cpa8(&S.mm[ly][lx], ts + gcl, 8);
    cpa4(&S.vm[ly][lx], tv + min(max(gy, 0), ny) * (nx + 1) + min(max(gx, 0), nx));
    const float2 mk = __ldg(reinterpret_cast<const float2*>(cfs + gcl));   // mu, 1/(lambda+mu)
    S.mu[ly][lx] = mk.x * h2inv;
    S.kap[ly][lx] = mk.y;
  }
}

// Complex arithmetic on the paired FP32 instructions (one instruction for the
// real and imaginary parts; per part the rounding of the scalar operation).
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
// a * x + y, a real
__device__ __forceinline__ float2 rfma2(float a, float2 x, float2 y) { return __ffma2_rn(bc2(a), x, y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
// a * b complex: (a.x b.x - a.y b.y, a.x b.y + a.y b.x)
__device__ __forceinline__ float2 cmul2(float2 a, float2 b) {
  return __ffma2_rn(bc2(a.y), make_float2(-b.y, b.x), __fmul2_rn(bc2(a.x), b));
}

// Off-diagonal part of a face row and its pressure coupling:
// b - (K_s row - dg xc) = b + (wpn xn+ + wmn xn- + wtp xt+ + wtm xt-) - (p_high - p_low) / h
__device__ __forceinline__ float2 face_rhs(float2 b, float wpn, float2 xnp, float wmn, float2 xnm, float wtp,
                                           float2 xtp, float wtm, float2 xtm, float2 phi, float2 plo, float hinv) {
  float2 s = rfma2(wpn, xnp, b);
  s = rfma2(wmn, xnm, s);
  s = rfma2(wtp, xtp, s);
  s = rfma2(wtm, xtm, s);
  return rfma2(-hinv, sub2(phi, plo), s);
}

// Economic cell update (eq. RelaxationMatrix: diagonal of the displacement block,
// displacement-pressure couplings g = (+1/h, +1/h, -1/h, -1/h), pressure diagonal)
// of the cell at staged (sx, sy), global (gx, gy), in-item index c: new values
// of its low faces (o[0] u_0, o[1] u_1), high faces (o[2] u_0 of cell + e_x,
// o[3] u_1 of cell + e_y) and pressure (o[4]); ok[a] marks the faces that are
// unknowns.  With r the residual of the block's rows and t_a = r_a / dg_a
// = (b_a - offdiag_a) / dg_a - x_a:
//   dp = (r_p - sum_a g_a t_a) / S,  du_a = t_a - g_a dp / dg_a,
// S = -kap - sum_a g_a^2 / dg_a (stored inverted per cell).
template <int W, int H>
__device__ __forceinline__ void cell_update(const Tile<W, H>& S, int sx, int sy, int gx, int gy, int nx, int ny,
                                            int N, int c, const float2* __restrict__ bb, const FP& P,
                                            float wu, float wp, float2 o[5], bool ok[4]) {
  ok[0] = gx >= 1;
  ok[1] = gy >= 1;
  ok[2] = gx + 1 < nx;
  ok[3] = gy + 1 < ny;
  // right-hand sides first (global loads in flight while the rows are formed)
  const float2 z = make_float2(0.f, 0.f);
  const float2 b0 = ok[0] ? __ldg(bb + c) : z, b1 = ok[1] ? __ldg(bb + N + c) : z;
  const float2 b2 = ok[2] ? __ldg(bb + c + 1) : z, b3 = ok[3] ? __ldg(bb + N + c + nx) : z;
  const float2 b4 = __ldg(bb + 2 * N + c);
  // every staged value the five rows read, once
  const float2 u0m = S.x[0][sy][sx - 1], u00 = S.x[0][sy][sx], u01 = S.x[0][sy][sx + 1], u02 = S.x[0][sy][sx + 2];
  const float2 u0dn = S.x[0][sy - 1][sx], u0up = S.x[0][sy + 1][sx];
  const float2 u1dn = S.x[0][sy - 1][sx + 1], u1up = S.x[0][sy + 1][sx + 1];
  const float2 v0m = S.x[1][sy - 1][sx], v00 = S.x[1][sy][sx], v01 = S.x[1][sy + 1][sx], v02 = S.x[1][sy + 2][sx];
  const float2 v0l = S.x[1][sy][sx - 1], v0r = S.x[1][sy][sx + 1];
  const float2 v1l = S.x[1][sy + 1][sx - 1], v1r = S.x[1][sy + 1][sx + 1];
  const float2 pc = S.x[2][sy][sx], pl = S.x[2][sy][sx - 1], pr = S.x[2][sy][sx + 1];
  const float2 pd = S.x[2][sy - 1][sx], pu = S.x[2][sy + 1][sx];
  const float mc = S.mu[sy][sx], ml = S.mu[sy][sx - 1], mr = S.mu[sy][sx + 1];
  const float md = S.mu[sy - 1][sx], mup = S.mu[sy + 1][sx];
  const float w00 = S.vm[sy][sx], w10 = S.vm[sy][sx + 1], w01 = S.vm[sy + 1][sx], w11 = S.vm[sy + 1][sx + 1];
  const float hinv = P.hinv;
  float2 dinv[4];
  dinv[0] = S.fx[sy][sx];
  dinv[1] = S.fy[sy][sx];
  dinv[2] = S.fx[sy][sx + 1];
  dinv[3] = S.fy[sy + 1][sx];
  float2 t[4];
  t[0] = sub2(cmul2(dinv[0], face_rhs(b0, mc, u01, ml, u0m, w01, u0up, w00, u0dn, pc, pl, hinv)), u00);
  t[1] = sub2(cmul2(dinv[1], face_rhs(b1, mc, v01, md, v0m, w10, v0r, w00, v0l, pc, pd, hinv)), v00);
  t[2] = sub2(cmul2(dinv[2], face_rhs(b2, mr, u02, mc, u00, w11, u1up, w10, u1dn, pr, pc, hinv)), u01);
  t[3] = sub2(cmul2(dinv[3], face_rhs(b3, mup, v02, mc, v00, w11, v1r, w01, v1l, pu, pc, hinv)), v01);
  // pressure row residual: b - (-kap p + (div u) / h)
  const float kap = S.kap[sy][sx];
  const float2 sdiv = __fadd2_rn(sub2(u00, u01), sub2(v00, v01));
  float2 rp = sub2(b4, rfma2(-kap, pc, __fmul2_rn(bc2(hinv), sdiv)));
  const float gk[4] = {hinv, hinv, -hinv, -hinv};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (!ok[a]) continue;
    rp = rfma2(-gk[a], t[a], rp);
  }
  const float2 dp = cmul2(rp, S.mm[sy][sx]);
  o[4] = rfma2(wp, dp, pc);
  const float2 xv[4] = {u00, v00, u01, v01};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (!ok[a]) { o[a] = xv[a]; continue; }
    const float2 q = cmul2(dp, dinv[a]);
    const float2 du = rfma2(-gk[a], q, t[a]);
    o[a] = rfma2(wu, du, xv[a]);
  }
}

typedef Tile<SWS_X, SWS_Y> SweepTile;
typedef Tile<RRS_X, RRS_Y> ResTile;

// 4 CTAs per SM (48 registers; a few bytes of spill) measured faster than 3 (64 registers)
__global__ void __launch_bounds__(SW_T, 4) k_fine_sweep_tile(Grid g, Grid gc, int nrhs, const float4* __restrict__ cf,
                                                             const float2* __restrict__ tdx,
                                                             const float2* __restrict__ tdy,
                                                             const float2* __restrict__ tsi,
                                                             const float* __restrict__ tvm,
                                                             FP P, float wu, float wp,
                                                             const float2* __restrict__ b,
                                                             const float2* __restrict__ xi,
                                                             const float2* __restrict__ ec,
                                                             float2* __restrict__ xo, const int* __restrict__ il) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SweepTile& S = *reinterpret_cast<SweepTile*>(smem_raw);
  const int item = il ? il[blockIdx.z] : blockIdx.z;
  const int N = (int)g.ncell;                                      // ncell < 2^31 on every level
  const int nx = g.n[0], ny = g.n[1];
  const long long vo = (long long)item * 3 * N;
  const float4* cfs = cf + (long long)(item / nrhs) * N;
  const float2* x = xi ? xi + vo : nullptr;
  const float2* e = ec ? ec + (long long)item * 3 * gc.ncell : nullptr;
  const int X0 = blockIdx.x * SW_X, Y0 = blockIdx.y * SW_Y;
  const int x0 = X0 - SW_H, y0 = Y0 - SW_H;
  const int set = item / nrhs;
  const long long nvt = (long long)(nx + 1) * (ny + 1);
  stage_tab<SWS_X, SWS_Y, SW_T>(S, cfs, tdx + (long long)set * N, tdy + (long long)set * N, tsi + (long long)set * N,
                                tvm + set * nvt, x, e, gc, N, nx, ny, x0, y0, P.h2inv);
  cpa_wait();
  __syncthreads();
  const float2* bb = b + vo;
  float2* xout = xo + vo;
  // ---- red cells of the tile and its one-cell ring, all from the staged iterate
  float2 ro[SW_RPT][5];
  bool rok[SW_RPT][4];
  int rsx[SW_RPT], rsy[SW_RPT];
#pragma unroll
  for (int q = 0; q < SW_RPT; ++q) {
    rsx[q] = -1;
    const int id = threadIdx.x + q * SW_T;
    if (id >= SW_NRED) continue;
    const int pr = id / SW_RX, j = id % SW_RX;                     // row pair, column
    const int gx = X0 - 1 + j, gy0 = Y0 - 1 + 2 * pr;
    const int gy = gy0 + ((gx + gy0) & 1);                         // (gx + gy) even: red
    if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;
    const int sx = gx - x0, sy = gy - y0;
    cell_update<SWS_X, SWS_Y>(S, sx, sy, gx, gy, nx, ny, N, gy * nx + gx, bb, P, wu, wp, ro[q], rok[q]);
    rsx[q] = sx; rsy[q] = sy;
  }
  __syncthreads();                                                 // every red row has read the old iterate
#pragma unroll
  for (int q = 0; q < SW_RPT; ++q) {
    if (rsx[q] < 0) continue;
    const int sx = rsx[q], sy = rsy[q];
    if (rok[q][0]) S.x[0][sy][sx] = ro[q][0];
    if (rok[q][1]) S.x[1][sy][sx] = ro[q][1];
    if (rok[q][2]) S.x[0][sy][sx + 1] = ro[q][2];
    if (rok[q][3]) S.x[1][sy + 1][sx] = ro[q][3];
    S.x[2][sy][sx] = ro[q][4];
  }
  __syncthreads();
  // ---- black cells of the tile from the red-updated iterate; outputs
  const int t = threadIdx.x;
  if (t >= SW_TB) return;                                          // no barrier follows
  const int gx = X0 + t % SW_X, gy0 = Y0 + 2 * (t / SW_X);         // column, row pair
  const int gyb = gy0 + ((gx + gy0 + 1) & 1), gyr = gyb ^ 1;       // (gx + gy) odd: black; the red one
  const int cb = gyb * nx + gx, cr = gyr * nx + gx;
  const int sx = gx - x0, sy = gyb - y0;
  // red pressure of the column's red cell: the red update
  xout[2 * N + cr] = S.x[2][gyr - y0][sx];
  // Dirichlet slots of the column's two cells (never written by any update)
  if (gx == 0) { xout[cb] = make_float2(0.f, 0.f); xout[cr] = make_float2(0.f, 0.f); }
  if (gyb == 0) xout[N + cb] = make_float2(0.f, 0.f);
  if (gyr == 0) xout[N + cr] = make_float2(0.f, 0.f);
  float2 o[5];
  bool ok[4];
  cell_update<SWS_X, SWS_Y>(S, sx, sy, gx, gyb, nx, ny, N, cb, bb, P, wu, wp, o, ok);
  xout[2 * N + cb] = o[4];
  if (ok[0]) xout[cb] = o[0];
  if (ok[1]) xout[N + cb] = o[1];
  if (ok[2]) xout[cb + 1] = o[2];
  if (ok[3]) xout[N + cb + nx] = o[3];
}

// 1D restriction weight of fine index j in coarse index J (pw4 in quarters)
__device__ __forceinline__ float rw(int kind, int j, int J, int nc) { return 0.25f * (float)pw4(kind, j, J, nc); }

__global__ void __launch_bounds__(RR_T, 4) k_fine_resid_restrict_tile(Grid g, Grid gc, int nrhs,
                                                                      const float4* __restrict__ cf,
                                                                      const float2* __restrict__ tgx,
                                                                      const float2* __restrict__ tgy,
                                                                      const float* __restrict__ tvm, FP P,
                                                                      const float2* __restrict__ x,
                                                                      const float2* __restrict__ b,
                                                                      float2* __restrict__ rc,
                                                                      const int* __restrict__ il) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ResTile& S = *reinterpret_cast<ResTile*>(smem_raw);
  const int item = il ? il[blockIdx.z] : blockIdx.z;
  const int N = (int)g.ncell;                                      // ncell < 2^31 on every level
  const int nx = g.n[0], ny = g.n[1];
  const long long vo = (long long)item * 3 * N;
  const float4* cfs = cf + (long long)(item / nrhs) * N;
  const int X0 = blockIdx.x * RR_X, Y0 = blockIdx.y * RR_Y;
  const int x0 = X0 - RR_H, y0 = Y0 - RR_H;
  const int set = item / nrhs;
  const long long nvt = (long long)(nx + 1) * (ny + 1);
  stage_tab<RRS_X, RRS_Y, RR_T>(S, cfs, tgx + (long long)set * N, tgy + (long long)set * N, nullptr, tvm + set * nvt,
                                x + vo, nullptr, gc, N, nx, ny, x0, y0, P.h2inv);
  cpa_wait();
  __syncthreads();
  const float2* bb = b + vo;
  const float hinv = P.hinv;
  // fine residual b - K_s x on the tile and its one-cell ring (zero outside the grid and on
  // the Dirichlet slots): the low-face rows of u_0 and u_1 and the pressure row of each cell
  float2 rr[RR_RPT][3];
#pragma unroll
  for (int q = 0; q < RR_RPT; ++q) {
    const int id = threadIdx.x + q * RR_T;
    rr[q][0] = rr[q][1] = rr[q][2] = make_float2(0.f, 0.f);
    if (id >= RR_RX * RR_RY) continue;
    const int rx = id % RR_RX, ry = id / RR_RX;
    const int gx = X0 - 1 + rx, gy = Y0 - 1 + ry;
    if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;
    const int sx = gx - x0, sy = gy - y0;
    const int c = gy * nx + gx;
    const float2 z = make_float2(0.f, 0.f);
    const float2 b0 = gx >= 1 ? __ldg(bb + c) : z;
    const float2 b1 = gy >= 1 ? __ldg(bb + N + c) : z;
    const float2 b2 = __ldg(bb + 2 * N + c);
    const float2 u0m = S.x[0][sy][sx - 1], u00 = S.x[0][sy][sx], u01 = S.x[0][sy][sx + 1];
    const float2 u0dn = S.x[0][sy - 1][sx], u0up = S.x[0][sy + 1][sx];
    const float2 v0m = S.x[1][sy - 1][sx], v00 = S.x[1][sy][sx], v01 = S.x[1][sy + 1][sx];
    const float2 v0l = S.x[1][sy][sx - 1], v0r = S.x[1][sy][sx + 1];
    const float2 pc = S.x[2][sy][sx], pl = S.x[2][sy][sx - 1], pd = S.x[2][sy - 1][sx];
    const float mc = S.mu[sy][sx], ml = S.mu[sy][sx - 1], md = S.mu[sy - 1][sx];
    const float w00 = S.vm[sy][sx], w10 = S.vm[sy][sx + 1], w01 = S.vm[sy + 1][sx];
    if (gx >= 1) rr[q][0] = sub2(face_rhs(b0, mc, u01, ml, u0m, w01, u0up, w00, u0dn, pc, pl, hinv), cmul2(S.fx[sy][sx], u00));
    if (gy >= 1) rr[q][1] = sub2(face_rhs(b1, mc, v01, md, v0m, w10, v0r, w00, v0l, pc, pd, hinv), cmul2(S.fy[sy][sx], v00));
    const float kap = S.kap[sy][sx];
    const float2 sdiv = __fadd2_rn(sub2(u00, u01), sub2(v00, v01));
    rr[q][2] = sub2(b2, rfma2(-kap, pc, __fmul2_rn(bc2(hinv), sdiv)));
  }
  __syncthreads();                                                 // the staged x is no longer read
  float2(*rs)[RR_RY][RR_RX] = reinterpret_cast<float2(*)[RR_RY][RR_RX]>(&S.x[0][0][0]);   // [3][RY][RX]
  static_assert(sizeof(float2) * 3 * RR_RY * RR_RX <= sizeof(ResTile::x), "residual fits in the staged x");
#pragma unroll
  for (int q = 0; q < RR_RPT; ++q) {
    const int id = threadIdx.x + q * RR_T;
    if (id >= RR_RX * RR_RY) continue;
    const int rx = id % RR_RX, ry = id / RR_RX;
    rs[0][ry][rx] = rr[q][0];
    rs[1][ry][rx] = rr[q][1];
    rs[2][ry][rx] = rr[q][2];
  }
  __syncthreads();
  // restriction: thread t < 128 forms u_0 and u_1 of coarse cell t, thread t >= 128 its pressure
  constexpr int CX = RR_X / 2, CY = RR_Y / 2;
  if (threadIdx.x >= 2 * CX * CY) return;                          // no barrier follows
  const int t = threadIdx.x % (CX * CY), half = threadIdx.x / (CX * CY);
  const int I = X0 / 2 + t % CX, J = Y0 / 2 + t / CX;
  if (I >= gc.n[0] || J >= gc.n[1]) return;
  const int ncx = gc.n[0], ncy = gc.n[1];
  const long long Nc = gc.ncell;
  float2* o = rc + (long long)item * 3 * Nc + (long long)J * ncx + I;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int a = half ? 2 : s;                                    // half 0: u_0, u_1; half 1: p
    if (half && s) break;
    float2 acc = make_float2(0.f, 0.f);
    const bool valid = a == 2 || (a == 0 ? I >= 1 : J >= 1);
    if (valid) {
      const int kx = a == 2 ? 2 : (a == 0 ? 0 : 1);
      const int ky = a == 2 ? 2 : (a == 1 ? 0 : 1);
#pragma unroll
      for (int dy = -1; dy <= 2; ++dy) {
        const int j = 2 * J + dy;
        const float wy = rw(ky, j, J, ncy);
        if (wy == 0.0f) continue;
#pragma unroll
        for (int dx = -1; dx <= 2; ++dx) {
          const int i = 2 * I + dx;
          const float wx = rw(kx, i, I, ncx);
          if (wx == 0.0f) continue;
          acc = cfma(make_float2(wy * wx, 0.f), rs[a][j - (Y0 - 1)][i - (X0 - 1)], acc);
        }
      }
    }
    o[(long long)a * Nc] = acc;
  }
}

// dynamic shared memory above the 48 KB default: set once per process and device
template <typename K> void smem_attr(K kernel, size_t bytes) {
  static int done[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  if (dev >= 0 && dev < 64 && !done[dev]) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done[dev] = 1;
  }
}

}  // namespace

bool fine_tiles_fit(const Grid& g) {
  return g.d == 2 && g.n[0] % SW_X == 0 && g.n[1] % SW_Y == 0 && g.n[0] % RR_X == 0 && g.n[1] % RR_Y == 0;
}

static FP make_fp(double h, double alpha) {
  FP P;
  P.h2inv = (float)(1.0 / (h * h));
  P.hinv = (float)(1.0 / h);
  P.alpha = (float)alpha;
  return P;
}

long long sweep_table_vertices(const Grid& g) { return (long long)(g.n[0] + 1) * (g.n[1] + 1); }

void launch_sweep_tables(const Grid& g, int nsets, const Coef4<float>* cf, double h, double alpha,
                         const SweepTab& T, cudaStream_t s) {
  const FP P = make_fp(h, alpha);
  const float4* c4 = reinterpret_cast<const float4*>(cf);
  const long long nv = sweep_table_vertices(g);
  k_sweep_tables_faces<<<dim3((unsigned)((nv + 255) / 256), nsets), 256, 0, s>>>(g, c4, P, T.dvx, T.dvy, T.gdx,
                                                                                    T.gdy, T.vm);
  k_sweep_tables_schur<<<dim3((unsigned)((g.ncell + 255) / 256), nsets), 256, 0, s>>>(g, c4, P, T.dvx, T.dvy,
                                                                                       T.sinv);
}

void launch_fine_sweep_tile(const Grid& g, const Grid& gc, int items, int nrhs, const Coef4<float>* cf,
                            const SweepTab& T, double h, double alpha, float wu, float wp, const float2* b,
                            const float2* xi, const float2* ec, float2* xo, cudaStream_t s) {
  const FP P = make_fp(h, alpha);
  smem_attr(k_fine_sweep_tile, sizeof(SweepTile));
  const dim3 gr(g.n[0] / SW_X, g.n[1] / SW_Y, sel_items(items));
  k_fine_sweep_tile<<<gr, SW_T, sizeof(SweepTile), s>>>(g, gc, nrhs, reinterpret_cast<const float4*>(cf), T.dvx,
                                                         T.dvy, T.sinv, T.vm, P, wu, wp, b, xi, ec, xo, g_sel.list);
}

void launch_fine_resid_restrict_tile(const Grid& g, const Grid& gc, int items, int nrhs, const Coef4<float>* cf,
                                     const SweepTab& T, double h, double alpha, const float2* x, const float2* b,
                                     float2* rc, cudaStream_t s) {
  const FP P = make_fp(h, alpha);
  smem_attr(k_fine_resid_restrict_tile, sizeof(ResTile));
  const dim3 gr(g.n[0] / RR_X, g.n[1] / RR_Y, sel_items(items));
  k_fine_resid_restrict_tile<<<gr, RR_T, sizeof(ResTile), s>>>(g, gc, nrhs, reinterpret_cast<const float4*>(cf),
                                                                T.gdx, T.gdy, T.vm, P, x, b, rc, g_sel.list);
}

}  // namespace ehs
