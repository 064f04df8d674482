// Launchers of the device kernels (host side).  All launches are
// asynchronous on the given stream; items = batch size of the vectors,
// nrhs = items per coefficient set (item b uses coefficient set b / nrhs).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace ehs {

// Active-item selection: when list != nullptr, per-item launches cover only
// the n listed items (blockIdx.y indexes the list), so items of a batch that
// have converged stop consuming bandwidth.  Set by the solver around the
// launches it issues (per host thread).
struct ItemSel {
  const int* list = nullptr;
  int n = 0;
};
extern thread_local ItemSel g_sel;
inline unsigned sel_items(int items) { return (unsigned)(g_sel.list ? g_sel.n : items); }

// ---- fine level (matrix-free) -------------------------------------------
// cell coefficients from lambda, mu, rho (double, one set per medium, device)
// and the absorbing layer; gamma = gamma_add + omega*abl_max*max_k(depth_k/L)^2;
// omegas: device array, one frequency per set
template <typename T>
void launch_fine_coef(const Grid& g, int nsets, const double* lam, const double* mu,
                      const double* rho, const double* omegas, int abl_cells, double abl_max,
                      double gamma_add, Coef4<T>* out, cudaStream_t s);
// DD subdomain coefficients: clamped copy of a global coefficient set plus the
// interface absorbing ramp; origin = global index of local cell 0 (may be
// negative), om_lo/om_hi = Omega_i in global indices, pad = padding per side.
template <typename T>
void launch_sub_coef(const Grid& gl, const Grid& gg, int nsets_glob, int nsub,
                     const int* d_origin /*[nsub*3]*/, const int* d_omlo, const int* d_omhi,
                     const int* d_padlo, const int* d_padhi, const int* d_subset /*glob set of sub set*/,
                     const Coef4<double>* glob, double dd_abl_max, Coef4<T>* out,
                     cudaStream_t s);
template <typename T>
void launch_coef_cast(long long n, const Coef4<double>* in, Coef4<T>* out, cudaStream_t s);

// y = K_s x (mode 0) or y = b - K_s x (mode 1), alpha = shift (0: unshifted)
template <typename T>
void launch_fine_apply(const Grid& g, int items, int nrhs, const Coef4<T>* cf, double h,
                       double alpha, const typename CT<T>::type* x,
                       const typename CT<T>::type* b, typename CT<T>::type* y, int mode,
                       cudaStream_t s);
// one colour of red-black economic cell-wise relaxation: xo = xi + W B^{-1}(b - K_s xi)
template <typename T>
void launch_fine_vanka(const Grid& g, int items, int nrhs, const Coef4<T>* cf, double h,
                       double alpha, T wu, T wp, int colour,
                       const typename CT<T>::type* b, const typename CT<T>::type* xi,
                       typename CT<T>::type* xo, cudaStream_t s, int full = 0);
// Fused fine-level kernels of the 2D complex64 cycle (economic block), for grids
// that split into their tiles (fine_tiles_fit).  One whole red-black sweep:
// xo = sweep(x_in), x_in = (xi or 0) + (P ec if ec), xo != xi; ec: coarse
// vector of grid gc (ignored when null).  And r_c = P^T (b - K_s x) in one pass.
bool fine_tiles_fit(const Grid& g);
// Setup-time tables of the fused fine kernels, per medium (k_fine_fused.cu): the diagonals of
// each cell's low u_0 / u_1 face rows, their inverses and the inverse pressure Schur complement
// of its block ([nsets][ncell] each), vertex means of mu / h^2 ([nsets][sweep_table_vertices(g)])
struct SweepTab {
  float2* gdx = nullptr;
  float2* gdy = nullptr;
  float2* dvx = nullptr;
  float2* dvy = nullptr;
  float2* sinv = nullptr;
  float* vm = nullptr;
};
long long sweep_table_vertices(const Grid& g);
void launch_sweep_tables(const Grid& g, int nsets, const Coef4<float>* cf, double h, double alpha,
                         const SweepTab& T, cudaStream_t s);
void launch_fine_sweep_tile(const Grid& g, const Grid& gc, int items, int nrhs, const Coef4<float>* cf,
                            const SweepTab& T, double h, double alpha, float wu, float wp, const float2* b,
                            const float2* xi, const float2* ec, float2* xo, cudaStream_t s);
void launch_fine_resid_restrict_tile(const Grid& g, const Grid& gc, int items, int nrhs, const Coef4<float>* cf,
                                     const SweepTab& T, double h, double alpha, const float2* x, const float2* b,
                                     float2* rc, cudaStream_t s);
// level-0 stencil table (double) of K_s for the Galerkin setup
void fine_table_layout(int d, StencilLayout* L);
void launch_fine_table(const Grid& g, int nsets, const Coef4<double>* cf, double h,
                       double alpha, const StencilLayout& L, double2* tab, cudaStream_t s);

// ---- stored stencils (Galerkin levels) ----------------------------------
void coarse_layout(int d, const StencilLayout& fine, StencilLayout* coarse);
void launch_galerkin(const Grid& gf, const Grid& gc, int nsets, const StencilLayout& Lf,
                     const double2* tf, const StencilLayout& Lc, double2* tc, int* err,
                     cudaStream_t s);
template <typename T>
void launch_table_cast(long long n, const double2* in, typename CT<T>::type* out, cudaStream_t s);
// tab: stencil table of level-layout L in format fmt (0: complex T, full; 1: FP16
// pairs, 2: BF16 pairs, in half storage (launch_table_half_sym) in 2D and full in
// 3D; the half formats serve the complex64 cycle only)
// var: residual-pass launch shape, 0 .. ST_ROWS_VARIANTS-1 (chosen by the setup autotuner)
#define ST_ROWS_VARIANTS 4
// layout variant of a Galerkin level: 1 = first coarse level, 2 = all coarser ones (throws otherwise)
int layout_variant(const StencilLayout& L, int d);
// residual pass on a Galerkin level of layout variant v (mode 0: y = K_c x, 1: y = b - K_c x;
// colour >= 0: pressure rows of that colour only)
template <typename T>
void launch_st_rows(const Grid& g, int items, int nrhs, int v, const void* tab, int fmt,
                    const typename CT<T>::type* x, const typename CT<T>::type* b, typename CT<T>::type* y, int mode,
                    int colour, int var, cudaStream_t s);
template <typename T>
void launch_st_apply(const Grid& g, int items, int nrhs, const StencilLayout& L, const void* tab, int fmt,
                     const typename CT<T>::type* x, const typename CT<T>::type* b, typename CT<T>::type* y,
                     int mode, int var, cudaStream_t s);
void launch_table_half(long long n, const double2* in, void* out, int fmt, cudaStream_t s);
// Galerkin table in half storage (common.cuh HalfMap: one coefficient of every mirrored pair,
// K_c = K_c^T) and FP16 (fmt 1) / BF16 (fmt 2) pairs: out [nsets][half_table_slots(L)][ncell];
// the complex64 cycle reads its fmt 1 / 2 tables in this form
int half_table_slots(const StencilLayout& L);
void launch_table_half_sym(const Grid& g, int nsets, const StencilLayout& L, const double2* in, void* out, int fmt,
                           cudaStream_t s);
// one colour of red-black Vanka on a Galerkin level; rbuf: residual scratch of x's size
template <typename T>
void launch_st_vanka(const Grid& g, int items, int nrhs, const StencilLayout& L, const void* tab, int fmt,
                     T wu, T wp, int colour, const typename CT<T>::type* b, const typename CT<T>::type* xi,
                     typename CT<T>::type* xo, typename CT<T>::type* rbuf, int var, cudaStream_t s);
// full Vanka (whole cell block): setup inverses of a smoothed Galerkin level,
// out [nsets][2 colours][(2d+1)^2][ncell/2] complex FP64; err gets EHS_DEVERR_SINGULAR
void launch_block_inv(const Grid& g, int nsets, const StencilLayout& L, const double2* tab, double2* out,
                      int* err, cudaStream_t s);
// one colour of red-black full Vanka on a Galerkin level (binv in format bfmt, as fmt for tables)
template <typename T>
void launch_st_vanka_full(const Grid& g, int items, int nrhs, const StencilLayout& L, const void* tab, int fmt,
                          const void* binv, int bfmt, T wu, T wp, int colour, const typename CT<T>::type* b,
                          const typename CT<T>::type* xi, typename CT<T>::type* xo, typename CT<T>::type* rbuf,
                          int var, cudaStream_t s);

// MG-DD: colour residual b - A x of a Galerkin level evaluated only at the local
// unknowns of the listed sub-items, written as their local vectors (map as launch_dd_gather)
template <typename T>
void launch_st_resid_gather(const Grid& g, int items_l, int nrhs, int nsub, int nloc, const int* map,
                            const StencilLayout& L, const void* tab, int fmt, const typename CT<T>::type* x,
                            const typename CT<T>::type* b, typename CT<T>::type* out, cudaStream_t s);

// ---- transfer -------------------------------------------------------------
template <typename T>
void launch_restrict(const Grid& gf, const Grid& gc, int items, const typename CT<T>::type* rf,
                     typename CT<T>::type* rc, cudaStream_t s);
template <typename T>
void launch_prolong_add(const Grid& gf, const Grid& gc, int items, const typename CT<T>::type* ec,
                        typename CT<T>::type* xf, cudaStream_t s);

// ---- coarsest level (dense FP64) ----------------------------------------
void launch_dense_assemble(const Grid& g, int nsets, const StencilLayout& L, const double2* tab,
                           double2* A /*[nsets][N][2N]*/, cudaStream_t s);
void dense_invert(int N, int nsets, double2* M /*[nsets][N][2N] augmented*/, double2* inv /*[nsets][N][N]*/,
                  double2* fbuf, int* pivbuf, int* err, cudaStream_t s);
template <typename T>
void launch_dense_apply(int N, int items, int nrhs, const double2* inv, const typename CT<T>::type* r,
                        typename CT<T>::type* x, cudaStream_t s);
// MG-DD: local dense matrices of the coarsest-grid subdomains ([nsets*nsub][nloc][2 nloc], augmented)
void launch_dense_assemble_sub(const Grid& g, int nsets, int nsub, int nloc, const StencilLayout& L,
                               const double2* tab, const int* map, const int* g2l, double2* A, cudaStream_t s);
// x = inv r with a low-precision inverse, FP32 accumulation; fmt 1 complex64, 2 FP16 pairs,
// 3 BF16 pairs; matrix of item b: inv + (b / nrhs) N^2 entries.  sizes (device, optional):
// live size of matrix set s is sizes[s % nsub], the rest identity padding (skipped)
// MG-DD local products of one colour with the scatter-add folded in: x[item][map[sub][row]] +=
// (A_sub^{-1} r_sub)[row] for every sub-item of the selection (complex64 r, x; inverses in format fmt
// as launch_dense_apply_lp); false (nothing launched) where the 4-row form does not apply
bool launch_dense_apply_scatter(int N, int items, int nrhs, int nsub, const int* sizes, const void* inv, int fmt,
                                const float2* r, const int* map, long long NG, float2* xg, cudaStream_t s);
void launch_dense_apply_lp(int N, int items, int nrhs, int nsub, const int* sizes, const void* inv, int fmt,
                           const float2* r, float2* x, cudaStream_t s);
// The MG-DD coarsest solve of the 2D complex64 cycle in one persistent launch (every colour's
// residual gather, local products and scatter, separated by bounded grid barriers; the result
// of the per-colour launches).  lv: layout variant of the coarsest level (1, 2); tfmt: table
// format (0 complex64, 1 FP16, 2 BF16 pairs); ifmt: coarse_fmt of the inverses (1..3); act/nact:
// active items (act null: all nact items); col_subs[k] / ncs[k]: subdomains of colour k; bar: two
// device words of barrier state (cleared by the launch); err: set to 1 if a barrier gave up.
bool coarse_persist_supported(const Grid& g, int coarse_fmt);
void launch_coarse_dd_persist(const Grid& g, int lv, int tfmt, int ifmt, int nrhs, int nsub, int nloc, const int* map,
                              const int* sizes, const void* tab, const void* inv, const float2* b, float2* x,
                              float2* rs, float2* zs, const int* act, int nact, const int* const* col_subs,
                              const int* ncs, int ncol, unsigned* bar, int* err, cudaStream_t s);
// sub-item list of MG-DD / DD: out[j * ncs + q] = ((m * nsub) + subs[q]) * nrhs + r for the
// j-th active item b = m * nrhs + r (all items when list is null)
void launch_expand_items(const int* list, int nact, int nrhs, int nsub, const int* subs, int ncs, int* out,
                         cudaStream_t s);
// gather of global slots into local vectors (map[s][e] = global slot or -1) and
// scatter-add back; sub-item bl = ((m * nsub) + s) * nrhs + r reads/writes item m * nrhs + r
template <typename T>
void launch_dd_gather(long long nl, int items_l, int nsub, int nrhs, long long nglob_item,
                      const int* map, const typename CT<T>::type* res, typename CT<T>::type* out,
                      cudaStream_t s);
template <typename T>
void launch_dd_scatter(long long nl, int items_l, int nsub, int nrhs, long long nglob_item,
                       const int* map, const typename CT<T>::type* xs, typename CT<T>::type* x,
                       cudaStream_t s);

// ---- Krylov (FP64) --------------------------------------------------------
void launch_cast_c128_c64(long long n, const double2* in, float2* out, cudaStream_t s);
void launch_cast_c64_c128(long long n, const float2* in, double2* out, cudaStream_t s);
void launch_copy(long long nbytes, const void* in, void* out, cudaStream_t s);
// partial dot products: part[item][i][blk] = sum conj(V_i) w over block blk
// V: [m+1][items][n] (vector i of item b at V + (i*items + b)*n)
int krylov_nblk(long long n);
void launch_mdot(long long n, int items, int nv, const double2* V, const double2* w, double2* part,
                 int nblk, cudaStream_t s);
// w -= sum_i V_i h_i; if dot: partial dots of V with the new w; if nrm: partial |w|^2
void launch_mupdate(long long n, int items, int nv, const double2* V, const double2* h, double2* w,
                    double2* part, int nblk, int dot, double* nrm_part, cudaStream_t s);
void launch_reduce_parts(int items, int nv, int nblk, const double2* part, double2* out, int accumulate,
                         cudaStream_t s);
void launch_norm_part(long long n, int items, const double2* w, double* part, int nblk, cudaStream_t s);
void launch_reduce_norm(int items, int nblk, const double* part, double* out, cudaStream_t s);
// v_out = w / nrm (per item)
void launch_scale_inv(long long n, int items, const double2* w, const double* nrm, double2* out,
                      cudaStream_t s);
// x += sum_{i<k_b} Z_i y_i, Z: [m][items][n] of CZ
template <typename CZ>
void launch_xupdate(long long n, int items, int m, const CZ* Z, const double2* y /*[items][m]*/,
                    const int* kused, double2* x, cudaStream_t s);

// ---- FP64-class (double-float) Krylov, operator and coarsest ----------------
// complex df64 = float4 {re.hi, im.hi, re.lo, im.lo} (dfc_st); real df64 = float2 {hi, lo}
// With cnt (device counters [items], zero, reset by the kernels), the last block of each item
// also reduces the partials: dots into out (df64) and outd (double copy for the host), the norm
// into nrm (double) and inv (df64 1/norm) -- the results of launch_reduce_parts_df /
// launch_reduce_norm_df, summed in the same order, without their launches.
void launch_mdot_df(long long n, int items, int nv, const float4* V, const float4* w, float4* part,
                    int nblk, cudaStream_t s, int* cnt = nullptr, float4* out = nullptr, double2* outd = nullptr);
void launch_mupdate_df(long long n, int items, int nv, const float4* V, const float4* h, float4* w,
                       float4* part, int nblk, int dot, float2* nrm_part, cudaStream_t s, int* cnt = nullptr,
                       float4* out = nullptr, double2* outd = nullptr, double* nrm = nullptr, float2* inv = nullptr,
                       int store = 1);
// out = w / norm (inv per item) and out32 = its complex64 copy
// V_{j+1} = (w - V (h0 + h)) * inv and its complex64 copy (the last pass of an Arnoldi step; h0 may be null)
void launch_update_scale_cast_df(long long n, int items, int nv, const float4* V, const float4* h, const float4* w,
                                 const float2* inv, float4* out, float2* out32, int nblk, cudaStream_t s,
                                 const float4* h0 = nullptr);
void launch_scale_cast_df(long long n, int items, const float4* w, const float2* inv, float4* out, float2* out32,
                          cudaStream_t s);
// Delayed CGS2 (one dot pass and one update pass per Arnoldi step j; slot j of V holds u_j,
// the direction the preconditioner was applied to).  launch_mdot2_df forms, with its last block
// per item (cnt: device counters [items], zero, reset by the kernel), the FP64 coefficients:
// coef[item * KDS ...] (df64) for launch_dupdate_df and outd[item * KDS ...] (double, for the
// host) = a_0..a_{j-1}, sigma, b_0..b_{j-1}, h_j, rho; part: [items][2][j + 2][nblk] partials.
// launch_dupdate_df rewrites slot j as v_j and writes u_{j+1} into slot j + 1 and its complex64
// copy into out32.
constexpr int KDS = 24;   // per-item stride of those arrays (2 j + 3 <= 23 for j <= 10)
void launch_mdot2_df(long long n, int items, int j, const float4* V, const float4* w, float4* part, int nblk,
                     cudaStream_t s, int* cnt, float4* coef, double2* outd);
void launch_dupdate_df(long long n, int items, int j, float4* V, const float4* w, const float4* coef,
                       float2* out32, cudaStream_t s);
void launch_norm_part_df(long long n, int items, const float4* w, float2* part, int nblk, cudaStream_t s);
// out (df64, device use) and outd (double copy for the host)
void launch_reduce_parts_df(int items, int nv, int nblk, const float4* part, float4* out, double2* outd,
                            cudaStream_t s);
// out = norm (double), inv = 1/norm (df64; may be null)
void launch_reduce_norm_df(int items, int nblk, const float2* part, double* out, float2* inv, cudaStream_t s);
void launch_scale_df(long long n, int items, const float4* w, const float2* inv, float4* out, cudaStream_t s);
void launch_xupdate_df(long long n, int items, int m, const float2* Z, const float4* y, const int* kused,
                       float4* x, cudaStream_t s);
void launch_d2_to_df(long long n, const double2* in, float4* out, cudaStream_t s);
void launch_df_to_d2(long long n, const float4* in, double2* out, cudaStream_t s);
void launch_df_to_f2(long long n, const float4* in, float2* out, cudaStream_t s);
void launch_coef_df(long long n, const Coef4<double>* in, void* out /*Coef4df*/, cudaStream_t s);
// y = K x (mode 0) or b - K x (mode 1); x complex64 (x_is_c64) or complex df64
// Setup-time tables of the 2D operator K (alpha = 0) for launch_fine_apply_df: dg [nsets][2][ncell]
// complex df64 (the low u_0 / u_1 face-row diagonals), vm [nsets][(nx + 1) (ny + 1)] df64 (vertex
// means of mu)
void launch_apply_df_tables(const Grid& g, int nsets, const Coef4<double>* cf, double h, float4* dg, float2* vm,
                            cudaStream_t s);
// with dg, vm (2D, alpha = 0) the rows read the tables above
void launch_fine_apply_df(const Grid& g, int items, int nrhs, const void* cf, double h, double alpha,
                          const void* x, int x_is_c64, const float4* b, float4* y, int mode, cudaStream_t s,
                          const float4* dg = nullptr, const float2* vm = nullptr);
void launch_dense_apply_df(int N, int items, int nrhs, const float4* inv, const float2* r, float2* x,
                           cudaStream_t s);

// adjoint-state gradient -Re(w^H dK/dm x) per cell, summed over each medium's rhs
void launch_gradient(const Grid& g, int nsets, int nrhs, const Coef4<double>* cf, const double* rho,
                     const double* omegas, double h, const double2* x, const double2* w, double* gl,
                     double* gm, double* gr, cudaStream_t s);

}  // namespace ehs
