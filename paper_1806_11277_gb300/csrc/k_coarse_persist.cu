// The MG-DD coarsest solve of the 2D complex64 cycle (Sec. 4: Algorithm DD
// over the coarsest Galerkin operator, dense local inverses, one sweep from a
// zero guess) in one persistent launch.  For every colour in turn, the CTAs
// of one grid take, in a fixed grid-stride order, the work items of two
// phases over all active items x subdomains of the colour:
//   A  the local residual r_loc = (b - K_c x) at the subdomain's unknowns (b at
//      the first colour, where x = 0; the clearing of x runs in that phase);
//   B  the local products A_s^{-1} r_loc, four rows per warp, each result added
//      to x at its unknown (subdomains of one colour are disjoint);
// separated by grid barriers.  This replaces the 17 launches of the per-colour
// form (clearing x, and per colour the item-list expansion, residual gather,
// local products and scatter) with one; the arithmetic of every element is
// that of those kernels (the same row sums and dense rows), so the results
// agree with them.
//
// Data one phase writes and a later phase reads again after other SMs changed
// it (x, across the colours) is read through L2 only (L1 is not coherent
// across SMs); each colour's local vectors are written once and then read.  The grid
// barrier is an arrival counter and a generation word; a CTA that
// waits longer than a fixed cycle budget (about a second; the launch sizes the
// grid so every CTA is resident, so this only happens if another workload
// holds the SMs) sets the error flag and returns, and so does every CTA at
// its next barrier: the solve then reports EHS_ERR_TIMEOUT instead of hanging.
#include "dense_rows.cuh"
#include "kernels.h"
#include "stencil_rows.cuh"

namespace ehs {
namespace {

constexpr int CP_T = 256;
#ifndef EHS_CP_MINBLOCKS
#define EHS_CP_MINBLOCKS 4      // CTAs per SM the register budget is sized for (best of 3..6 measured)
#endif
constexpr long long CP_SPIN_CYCLES = 2000000000LL;   // ~1 s at the GB300's SM clock

struct CoarsePersistArgs {
  Grid g;
  int nrhs, nsub, nloc;
  const int* map;       // [nsub][nloc] coarsest slot or -1
  const int* sizes;     // [nsub] live unknowns
  const void* tab;      // coarsest Galerkin table (format of TT)
  const void* inv;      // [nsets * nsub][nloc][nloc] local inverses (format of TI)
  const float2* b;
  float2* x;
  float2* rs;           // local vectors [items * nsub][nloc]
  float2* zs;
  const int* act;       // active items (null: all)
  int nact;
  const int* col_subs[8];
  int ncs[8];
  unsigned* bar;        // [2]: arrivals, generation
  int* err;
};

// bounded grid barrier; false once any CTA has given up
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
      atomicExch(bar, 0u);                 // reset before the release
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g0) {
        if (clock64() - t0 > CP_SPIN_CYCLES) { atomicOr(err, 1); break; }
        __nanosleep(128);
      }
    }
    __threadfence();
    if (*(volatile int*)err) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

template <typename TT, typename TI, int LV, bool SYM>
__global__ void __launch_bounds__(CP_T, EHS_CP_MINBLOCKS) k_coarse_dd_persist(CoarsePersistArgs A) {
  constexpr int D = 2;
  const Grid& g = A.g;
  const long long N = g.ncell;
  const long long NG = (long long)(D + 1) * N;
  const int nloc = A.nloc;
  const int nitems = A.nact;
  const long long gtid = (long long)blockIdx.x * CP_T + threadIdx.x;
  const long long gthreads = (long long)gridDim.x * CP_T;
  constexpr StencilLayout L = level_layout(D, LV);
  constexpr int nslot = SYM ? half_base(L, L.npair) : L.nslot;
  bool first = true;
  for (int col = 0; col < 8; ++col) {
    const int ncs = A.ncs[col];
    if (!ncs) continue;
    const int* subs = A.col_subs[col];
    const long long nsi = (long long)nitems * ncs;   // sub-items of this colour
    // ---- A: local residuals (first colour: x = 0 on the active items and r_loc = b)
    if (first)
      for (long long t = gtid; t < (long long)nitems * NG; t += gthreads) {
        const int j = (int)(t / NG);
        const int item = A.act ? A.act[j] : j;
        A.x[(long long)item * NG + t % NG] = make_float2(0.f, 0.f);
      }
    for (long long t = gtid; t < nsi * nloc; t += gthreads) {
      const int jj = (int)(t / nloc), e = (int)(t % nloc);
      const int item = A.act ? A.act[jj / ncs] : jj / ncs;
      const int s = subs[jj % ncs];
      const int m = item / A.nrhs, r = item % A.nrhs;
      const long long bl = ((long long)m * A.nsub + s) * A.nrhs + r;
      const int gs = A.map[(long long)s * nloc + e];
      float2 v = make_float2(0.f, 0.f);
      if (gs >= 0) {
        const long long vo = (long long)item * NG;
        v = __ldg(A.b + vo + gs);
        if (!first) {
          const int a = (int)(gs / N);
          const long long c = gs % N;
          const TT* ts = (const TT*)A.tab + (long long)m * nslot * N;
          int i[3];
          cell_coords(g, c, i);
          float2 y;
          if (a == 0) y = st_row_ct<float, TT, D, LV, SYM, 0, true>(g, ts, c, i, A.x + vo);
          else if (a == 1) y = st_row_ct<float, TT, D, LV, SYM, 1, true>(g, ts, c, i, A.x + vo);
          else y = st_row_ct<float, TT, D, LV, SYM, 2, true>(g, ts, c, i, A.x + vo);
          v = csub(v, y);
        }
      }
      A.rs[bl * nloc + e] = v;
    }
    first = false;
    if (!grid_sync(A.bar, A.err)) return;
    // ---- B: local products, four rows per warp, each result added to x at its unknown
    {
      const int rg = nloc / 4;
      const long long gw = gtid >> 5, nw = gthreads >> 5;
      for (long long w = gw; w < nsi * rg; w += nw) {
        const int jj = (int)(w / rg), row0 = (int)(w % rg) * 4;
        const int item = A.act ? A.act[jj / ncs] : jj / ncs;
        const int s = subs[jj % ncs];
        const int m = item / A.nrhs, r = item % A.nrhs;
        const long long set = (long long)m * A.nsub + s;
        const long long bl = set * A.nrhs + r;
        const int n = A.sizes[s];
        if (row0 >= n) continue;                       // warp-uniform
        // r_loc through L1 (__ldg): the sub-items of a colour are first read here, after this
        // launch wrote them, so no SM holds an older copy (a local vector is a whole number of
        // 32-byte sectors: nloc is a multiple of 8)
        dense_rows4<TI, false, true>(nloc, n, row0, (const TI*)A.inv + set * nloc * nloc, A.rs + bl * nloc,
                                     nullptr, A.map + (long long)s * nloc, A.x + (long long)item * NG);
      }
    }
    if (!grid_sync(A.bar, A.err)) return;
  }
}

template <typename TT, typename TI, int LV, bool SYM>
void launch_t(const CoarsePersistArgs& a, cudaStream_t s) {
  static int grid[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  if (!grid[dev]) {   // every CTA resident: SMs x the kernel's occupancy
    int nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_coarse_dd_persist<TT, TI, LV, SYM>, CP_T, 0);
    grid[dev] = nsm * (per < 1 ? 1 : per);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid[dev]);
  cfg.blockDim = dim3(CP_T);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;     // co-residency of all CTAs
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_coarse_dd_persist<TT, TI, LV, SYM>, a);
}

template <typename TT, typename TI>
void launch_lv(const CoarsePersistArgs& a, int lv, bool sym, cudaStream_t s) {
  if (sym) {
    if (lv == 1) launch_t<TT, TI, 1, true>(a, s);
    else launch_t<TT, TI, 2, true>(a, s);
  } else {
    if (lv == 1) launch_t<TT, TI, 1, false>(a, s);
    else launch_t<TT, TI, 2, false>(a, s);
  }
}
template <typename TT>
void launch_ti(const CoarsePersistArgs& a, int lv, bool sym, int ifmt, cudaStream_t s) {
  if (ifmt == 2) launch_lv<TT, __half2>(a, lv, sym, s);
  else if (ifmt == 3) launch_lv<TT, __nv_bfloat162>(a, lv, sym, s);
  else launch_lv<TT, float2>(a, lv, sym, s);
}

}  // namespace

bool coarse_persist_supported(const Grid& g, int coarse_fmt) { return g.d == 2 && coarse_fmt >= 1 && coarse_fmt <= 3; }

void launch_coarse_dd_persist(const Grid& g, int lv, int tfmt, int ifmt, int nrhs, int nsub, int nloc, const int* map,
                              const int* sizes, const void* tab, const void* inv, const float2* b, float2* x,
                              float2* rs, float2* zs, const int* act, int nact, const int* const* col_subs,
                              const int* ncs, int ncol, unsigned* bar, int* err, cudaStream_t s) {
  CoarsePersistArgs a{};
  a.g = g;
  a.nrhs = nrhs; a.nsub = nsub; a.nloc = nloc;
  a.map = map; a.sizes = sizes; a.tab = tab; a.inv = inv;
  a.b = b; a.x = x; a.rs = rs; a.zs = zs;
  a.act = act; a.nact = nact;
  for (int k = 0; k < 8; ++k) {
    a.col_subs[k] = k < ncol ? col_subs[k] : nullptr;
    a.ncs[k] = k < ncol ? ncs[k] : 0;
  }
  a.bar = bar; a.err = err;
  cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  // table formats: 0 complex64 (full), 1 FP16 / 2 BF16 pairs (half storage in 2D)
  if (tfmt == 1) launch_ti<__half2>(a, lv, true, ifmt, s);
  else if (tfmt == 2) launch_ti<__nv_bfloat162>(a, lv, true, ifmt, s);
  else launch_ti<float2>(a, lv, false, ifmt, s);
}

}  // namespace ehs
