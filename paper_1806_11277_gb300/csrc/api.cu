// Host side of the GB300 elastic Helmholtz library: hierarchy setup, the
// multigrid cycle, the multicolour DD sweep and the FGMRES driver, behind the
// C ABI of include/ehs.h.  Every arithmetic step runs in the kernels of this
// directory; the host only sequences launches and runs the (m+1) x m
// Hessenberg least-squares update of FGMRES.
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <complex>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "ehs.h"
#include "kernels.h"

namespace ehs {
std::atomic<long long> g_launches{0};
thread_local ItemSel g_sel;
}

using namespace ehs;
typedef std::complex<double> zc;

namespace {

struct CudaError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct ArgError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      throw CudaError(std::string(#call) + ": " + cudaGetErrorString(e_));               \
  } while (0)

inline void cnt(long long k = 1) { g_launches += k; }
inline void post() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw CudaError(std::string("kernel launch: ") + cudaGetErrorString(e));
}

struct Level {
  Grid g{};
  StencilLayout L{};
  double2* tab64 = nullptr;   // Galerkin levels and coarsest: [nsets][nslot][ncell]
  float2* tab32 = nullptr;
  void* tabh = nullptr;       // half-precision copy (FP16 or BF16 pairs) for the complex64 cycle
  double2* inv = nullptr;     // coarsest: [nsets][N][N]
  float4* invdf = nullptr;    // coarsest inverse in complex df64 (used by the complex64 cycle)
  void* invlp = nullptr;      // coarsest inverse in complex64 / FP16 / BF16 pairs (coarse_fmt 1..3)
  void* binv[2] = {nullptr, nullptr};  // full Vanka block inverses [prec: 0 double2, 1 float2 or half pairs]
  void* ws[2][4] = {{nullptr}};  // [prec: 0 double, 1 float][b, x, t, r]
  int rows_var[2] = {0, 0};      // residual-pass launch shape per precision (setup autotuner)
  double w = 0.5;
};

// MG-DD coarsest solver (Sec. 4): subdomains of the coarsest grid, their
// dense local inverses and the per-colour sub-item lists
struct CoarseDD {
  int nsub = 0;                 // 0: exact dense coarsest solve
  int nloc = 0;                 // local dense size (largest subdomain; smaller ones padded)
  int* d_map = nullptr;         // [nsub][nloc] coarsest slot (comp * ncell + cell) or -1
  int* d_sizes = nullptr;       // [nsub] live unknowns of each subdomain (<= nloc)
  std::vector<int> sizes;
  std::vector<std::vector<int>> col_subs;  // subdomains of each colour (2^d colours)
  std::vector<int*> d_col_subs;
  std::vector<int*> d_list;     // per colour: expanded sub-item list [items * ncs]
  std::vector<int*> d_list_all; // per colour: the sub-item list with every item active (setup)
  void* loc[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [prec][r, z] [items * nsub][nloc]
};

struct Hier {
  Grid g0{};
  int nlev = 0, nsets = 0, nrhs = 1, items = 0;
  double h = 1, alpha = 0;
  double wp_ratio = 1;
  int nu1 = 1, nu2 = 1, cyc = 1;
  int half = 0;                // Galerkin tables of the complex64 cycle: 0 complex64, 1 FP16, 2 BF16
  int full = 0;                // 1: full cell-block Vanka instead of the economic block
  int cdd_split[3] = {1, 1, 1};  // MG-DD subdomains per axis of the coarsest grid
  int cdd_overlap = 2;
  int coarse_fmt = 0;          // coarsest inverses of the complex64 cycle: 0 df64, 1 c64, 2 FP16, 3 BF16
  CoarseDD cdd;
  bool coef_only = false;      // only the fine coefficients were built (global problem of a DD context)
  bool fused0 = false;         // 2D complex64 cycle: fused fine-level sweep and residual + restriction
  SweepTab stab;               // setup-time tables of the fused sweep (fused0)
  bool persist = false;        // complex64 MG-DD coarsest solve in one persistent launch
  unsigned* pbar = nullptr;    // its grid-barrier state (2 words)
  Coef4<double>* cf64 = nullptr;
  Coef4<float>* cf32 = nullptr;
  void* cfdf = nullptr;        // df64 coefficients (outer-Krylov operator of the global problem)
  float4* kdg = nullptr;       // 2D: df64 tables of that operator (face-row diagonals, vertex means)
  float2* kvm = nullptr;
  std::vector<Level> lv;
};

struct DDGroup {          // subdomains of one colour that share one shape
  Hier H;
  int* d_sub_act = nullptr;  // active sub-items (derived from the active global items)
  int nsub_act = 0;
  int nsub = 0;
  std::vector<int> subs;  // global subdomain ids
  int* d_map = nullptr;   // [nsub][ncell_local] -> global cell index or -1 (outside Omega_i)
  int* d_origin = nullptr;
};

}  // namespace

struct ehs_ctx {
  cudaStream_t s = nullptr;
  int* derr = nullptr;       // device flag: a bounded grid barrier of a persistent launch gave up
  ehs_problem prob{};
  ehs_opts opt{};
  int d = 2;
  long long n0 = 0;       // complex values per item at the fine level
  Hier H;
  std::vector<DDGroup> dd[8];
  std::vector<void*> allocs;
  // Krylov workspace
  double2 *V = nullptr, *Z = nullptr, *w = nullptr, *part = nullptr, *hd = nullptr, *y = nullptr;
  double2 *qd = nullptr, *ud = nullptr, *rd = nullptr;
  double *npart = nullptr, *nrm = nullptr;
  int* kused = nullptr;
  float2 *f_in = nullptr, *f_out = nullptr;
  // df64 Krylov workspace (complex64 preconditioner form)
  float4 *Vq = nullptr, *wq = nullptr, *rq = nullptr, *qq = nullptr, *xq = nullptr, *partq = nullptr;
  float4 *hq = nullptr, *h2q = nullptr, *yq = nullptr;
  float4* dcoef = nullptr;    // [items][KDS] delayed-CGS2 update coefficients (df64)
  float2 *Zf = nullptr, *npq = nullptr, *invq = nullptr;
  int* kcnt = nullptr;        // [3][items] last-block counters of the fused Krylov reductions
  double2* hhost = nullptr;   // device double copies of h for the host
  double* d_rho = nullptr;   // media kept for the gradient: rho and omega per set
  double* d_om = nullptr;
  double2* dd_x = nullptr;   // DD accumulated correction (c128 or c64 view)
  double2* dd_r = nullptr;
  int nblk = 1;
  double* hpin = nullptr;    // pinned host scratch
  double2* hstep = nullptr;  // pinned host copies of one Arnoldi step: h1 [items][12], h2 [items][12], norms
                             // (delayed CGS2: the step's FP64 coefficients, [items][KDS])
  cudaEvent_t ev_step = nullptr;   // recorded after the copies of one Arnoldi step
  // CUDA graphs of the preconditioner application, one per Krylov direction j
  // (the input/output pointers differ per j), captured on a private stream
  bool use_graphs = true;
  cudaStream_t cap = nullptr;
  std::vector<cudaGraphExec_t> pg;
  std::vector<long long> pg_nodes;
  std::vector<int> pg_ver;
  // active items of the current Arnoldi step (batch compaction)
  int* d_act = nullptr;
  std::vector<int> act;      // host copy; empty = all items
  int act_ver = 0;
  std::string err;
};

static std::string g_create_err;

namespace {

template <typename P> P* dalloc(ehs_ctx* c, size_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&p, count * sizeof(P));
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) throw std::bad_alloc();
    throw CudaError(std::string("cudaMalloc: ") + cudaGetErrorString(e));   // no device, driver, ...
  }
  c->allocs.push_back(p);
  CK(cudaMemsetAsync(p, 0, count * sizeof(P), c->s));
  return (P*)p;
}
void dfree(ehs_ctx* c, void* p) {
  if (!p) return;
  for (auto& q : c->allocs)
    if (q == p) { cudaFree(p); q = nullptr; return; }
}

Grid mkgrid(int d, int nx, int ny, int nz) {
  Grid g;
  g.d = d; g.n[0] = nx; g.n[1] = ny; g.n[2] = d == 3 ? nz : 1;
  g.ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  return g;
}

// Installs the active item list (or none) for the launches in its scope.
struct SelScope {
  ItemSel old;
  SelScope(const int* list, int n) : old(g_sel) { g_sel.list = list; g_sel.n = n; }
  ~SelScope() { g_sel = old; }
};
inline SelScope global_sel(ehs_ctx* c) {
  return c->act.empty() ? SelScope(nullptr, 0) : SelScope(c->d_act, (int)c->act.size());
}

// ------------------------------------------------------------ hierarchy
template <typename T> void autotune_rows(ehs_ctx* c, Hier& H);

// Builds the hierarchy of H from H.cf64.  precs: work buffers for the FP64
// cycle (bit 0) and the complex64 cycle (bit 1).  coef_only: only the fine
// coefficients (the global problem of a DD context, whose cycles run on the
// subdomain hierarchies).
void build_hier(ehs_ctx* c, Hier& H, int precs, bool coef_only) {
  const int d = H.g0.d;
  H.cf32 = dalloc<Coef4<float>>(c, (size_t)H.nsets * H.g0.ncell);
  launch_coef_cast<float>((long long)H.nsets * H.g0.ncell, H.cf64, H.cf32, c->s); cnt(); post();
  if (coef_only) {
    H.lv.resize(1);
    H.lv[0].g = H.g0;
    H.coef_only = true;
    return;
  }
  H.lv.resize(H.nlev);
  Grid g = H.g0;
  for (int l = 0; l < H.nlev; ++l) {
    Level& L = H.lv[l];
    L.g = g;
    L.w = c->opt.w[l < 8 ? l : 7];
    const long long nv = (long long)H.items * (d + 1) * g.ncell;
    for (int k = 0; k < 4; ++k) {
      if (precs & 1) L.ws[0][k] = dalloc<double2>(c, nv);
      if (precs & 2) L.ws[1][k] = dalloc<float2>(c, nv);
    }
    if (l + 1 < H.nlev) g = mkgrid(d, g.n[0] / 2, g.n[1] / 2, g.n[2] / 2);
  }
  // level-0 table of K_s, then Galerkin products level by level
  StencilLayout Lf;
  fine_table_layout(d, &Lf);
  double2* tf = dalloc<double2>(c, (size_t)H.nsets * Lf.nslot * H.g0.ncell);
  launch_fine_table(H.g0, H.nsets, H.cf64, H.h, H.alpha, Lf, tf, c->s); cnt(); post();
  int* derr = dalloc<int>(c, 1);
  for (int l = 1; l < H.nlev; ++l) {
    Level& L = H.lv[l];
    coarse_layout(d, Lf, &L.L);
    L.tab64 = dalloc<double2>(c, (size_t)H.nsets * L.L.nslot * L.g.ncell);
    launch_galerkin(H.lv[l - 1].g, L.g, H.nsets, Lf, tf, L.L, L.tab64, derr, c->s); cnt(); post();
    if (l == 1) dfree(c, tf);   // the level-0 table is only needed for the first product
    const long long nt = (long long)H.nsets * L.L.nslot * L.g.ncell;
    L.tab32 = dalloc<float2>(c, nt);
    launch_table_cast<float>(nt, L.tab64, L.tab32, c->s); cnt(); post();
    if (H.half && d == 2) {   // 4 bytes per complex coefficient, one of each mirrored pair (K_c = K_c^T)
      L.tabh = dalloc<float>(c, (size_t)H.nsets * half_table_slots(L.L) * L.g.ncell);
      launch_table_half_sym(L.g, H.nsets, L.L, L.tab64, L.tabh, H.half, c->s); cnt(); post();
    } else if (H.half) {      // 3D: the whole table, 4 bytes per complex coefficient
      L.tabh = dalloc<float>(c, nt);
      launch_table_half(nt, L.tab64, L.tabh, H.half, c->s); cnt(); post();
    }
    Lf = L.L;
    tf = L.tab64;
  }
  // full Vanka: block inverses of every smoothed Galerkin level (FP64, then the cycle's formats)
  for (int l = 1; H.full && l + 1 < H.nlev; ++l) {
    Level& L = H.lv[l];
    const long long nb = (long long)H.nsets * 2 * (2 * d + 1) * (2 * d + 1) * (L.g.ncell / 2);
    double2* b64 = dalloc<double2>(c, nb);
    launch_block_inv(L.g, H.nsets, L.L, L.tab64, b64, derr, c->s); cnt(); post();
    if (precs & 2) {
      if (H.half) {
        L.binv[1] = dalloc<float>(c, nb);
        launch_table_half(nb, b64, L.binv[1], H.half, c->s); cnt(); post();
      } else {
        L.binv[1] = dalloc<float2>(c, nb);
        launch_table_cast<float>(nb, b64, (float2*)L.binv[1], c->s); cnt(); post();
      }
    }
    if (precs & 1) L.binv[0] = b64;
    else dfree(c, b64);
  }
  // coarsest: dense FP64 inverse of the whole level, or of every MG-DD subdomain
  Level& C = H.lv[H.nlev - 1];
  const long long NG = (long long)(d + 1) * C.g.ncell;
  int nloc = (int)NG, nmat = H.nsets;
  int *d_g2l = nullptr;
  const bool mgdd = H.cdd_split[0] * H.cdd_split[1] * H.cdd_split[2] > 1;
  if (mgdd) {
    CoarseDD& D = H.cdd;
    std::vector<std::vector<int>> sp(3);
    for (int k = 0; k < 3; ++k) {
      const int n = k < d ? C.g.n[k] : 1, ns = k < d ? H.cdd_split[k] : 1;
      if (ns < 1 || ns > n) throw ArgError("coarse_dd split larger than the coarsest grid");
      sp[k].push_back(0);
      for (int q = 0; q < ns; ++q) sp[k].push_back(sp[k].back() + n / ns + (q < n % ns ? 1 : 0));
      for (int q = 0; q < ns && ns > 1; ++q)
        if (2 * H.cdd_overlap > sp[k][q + 1] - sp[k][q])
          throw ArgError("coarse_dd_overlap larger than half a coarsest-grid core");
    }
    if (H.cdd_overlap < 1) throw ArgError("coarse_dd_overlap must be >= 1");
    D.nsub = (d == 3 ? H.cdd_split[2] : 1) * H.cdd_split[1] * H.cdd_split[0];
    D.col_subs.assign(1 << d, {});
    std::vector<std::vector<int>> dofs(D.nsub);
    int sidx = 0;
    for (int iz = 0; iz < (d == 3 ? H.cdd_split[2] : 1); ++iz)
      for (int iy = 0; iy < H.cdd_split[1]; ++iy)
        for (int ix = 0; ix < H.cdd_split[0]; ++ix, ++sidx) {
          const int id[3] = {ix, iy, iz};
          int lo[3], hi[3], col = 0;
          for (int k = 0; k < 3; ++k) {
            if (k >= d) { lo[k] = 0; hi[k] = 1; continue; }
            lo[k] = std::max(sp[k][id[k]] - H.cdd_overlap, 0);
            hi[k] = std::min(sp[k][id[k] + 1] + H.cdd_overlap, C.g.n[k]);
            col |= (id[k] & 1) << k;
          }
          D.col_subs[col].push_back(sidx);
          // unknowns of the box: pressures of its cells, faces with both cells inside
          for (int a = 0; a <= d; ++a)
            for (int z = lo[2]; z < hi[2]; ++z)
              for (int y = lo[1]; y < hi[1]; ++y)
                for (int x = lo[0]; x < hi[0]; ++x) {
                  const int j3[3] = {x, y, z};
                  if (a < d && j3[a] - 1 < lo[a]) continue;
                  dofs[sidx].push_back((int)((long long)a * C.g.ncell + cell_index(C.g, j3)));
                }
        }
    nloc = 0;
    for (auto& v : dofs) {
      nloc = std::max(nloc, (int)v.size());
      D.sizes.push_back((int)v.size());
    }
    nloc = (nloc + 7) / 8 * 8;   // rows start 16-byte aligned for the vectorised local products
    D.nloc = nloc;
    D.d_sizes = dalloc<int>(c, D.nsub);
    CK(cudaMemcpyAsync(D.d_sizes, D.sizes.data(), D.nsub * sizeof(int), cudaMemcpyHostToDevice, c->s));
    std::vector<int> map((size_t)D.nsub * nloc, -1), g2l((size_t)D.nsub * NG, -1);
    for (int q = 0; q < D.nsub; ++q)
      for (int e = 0; e < (int)dofs[q].size(); ++e) {
        map[(size_t)q * nloc + e] = dofs[q][e];
        g2l[(size_t)q * NG + dofs[q][e]] = e;
      }
    D.d_map = dalloc<int>(c, map.size());
    d_g2l = dalloc<int>(c, g2l.size());
    CK(cudaMemcpyAsync(D.d_map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(d_g2l, g2l.data(), g2l.size() * sizeof(int), cudaMemcpyHostToDevice, c->s));
    for (int col = 0; col < (1 << d); ++col) {
      const auto& cs = D.col_subs[col];
      int* ds = nullptr;
      int* dl = nullptr;
      if (!cs.empty()) {
        ds = dalloc<int>(c, cs.size());
        CK(cudaMemcpyAsync(ds, cs.data(), cs.size() * sizeof(int), cudaMemcpyHostToDevice, c->s));
        dl = dalloc<int>(c, (size_t)H.items * cs.size());
      }
      D.d_col_subs.push_back(ds);
      D.d_list.push_back(dl);
      int* da = nullptr;
      if (!cs.empty()) {
        std::vector<int> all;
        for (int b = 0; b < H.items; ++b)
          for (int q : cs) all.push_back(((b / H.nrhs) * D.nsub + q) * H.nrhs + b % H.nrhs);
        da = dalloc<int>(c, all.size());
        CK(cudaMemcpyAsync(da, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice, c->s));
        CK(cudaStreamSynchronize(c->s));
      }
      D.d_list_all.push_back(da);
    }
    for (int p = 0; p < 2; ++p)
      if (precs & (1 << p))
        for (int k = 0; k < 2; ++k)
          D.loc[p][k] = p == 0 ? (void*)dalloc<double2>(c, (size_t)H.items * D.nsub * nloc)
                               : (void*)dalloc<float2>(c, (size_t)H.items * D.nsub * nloc);
    CK(cudaStreamSynchronize(c->s));   // the host arrays above are temporaries
    nmat = H.nsets * D.nsub;
  } else if (NG > 16384) {
    throw ArgError("coarsest grid too large for the dense FP64 inverse (use more levels or coarse_dd)");
  }
  if (nloc > 16384) throw ArgError("coarse_dd subdomains too large for dense local inverses");
  const long long N = nloc;
  double2* M = dalloc<double2>(c, (size_t)nmat * N * 2 * N);
  double2* fb = dalloc<double2>(c, (size_t)nmat * (N + 1));
  int* pv = dalloc<int>(c, nmat);
  if (mgdd)
    launch_dense_assemble_sub(C.g, H.nsets, H.cdd.nsub, nloc, C.L, C.tab64, H.cdd.d_map, d_g2l, M, c->s);
  else
    launch_dense_assemble(C.g, H.nsets, C.L, C.tab64, M, c->s);
  cnt(); post();
  C.inv = dalloc<double2>(c, (size_t)nmat * N * N);
  dense_invert((int)N, nmat, M, C.inv, fb, pv, derr, c->s); cnt(4 * N + 1); post();
  if (precs & 2) {
    if (H.coarse_fmt == 1) {
      C.invlp = dalloc<float2>(c, (size_t)nmat * N * N);
      launch_table_cast<float>((long long)nmat * N * N, C.inv, (float2*)C.invlp, c->s); cnt(); post();
    } else if (H.coarse_fmt >= 2) {
      C.invlp = dalloc<float>(c, (size_t)nmat * N * N);   // 4 bytes per complex entry
      launch_table_half((long long)nmat * N * N, C.inv, C.invlp, H.coarse_fmt - 1, c->s); cnt(); post();
    } else {
      C.invdf = dalloc<float4>(c, (size_t)nmat * N * N);
      launch_d2_to_df((long long)nmat * N * N, C.inv, C.invdf, c->s); cnt(); post();
    }
  }
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  dfree(c, M); dfree(c, fb); dfree(c, pv); dfree(c, derr);
  if (d_g2l) dfree(c, d_g2l);
  if (!(precs & 1)) { dfree(c, C.inv); C.inv = nullptr; }
  if (herr & EHS_DEVERR_BOX) throw CudaError("Galerkin stencil fell outside its box");
  if (herr & EHS_DEVERR_SINGULAR) throw ArgError("coarsest Galerkin operator is singular");
  if (precs & 2) autotune_rows<float>(c, H);
  if (precs & 1) autotune_rows<double>(c, H);
  // the fused fine-level kernels serve the economic 2D complex64 cycle on grids that split into
  // their tiles; EHS_FINE_UNFUSED=1 selects the per-colour kernels instead (tests compare both)
  const char* uf = getenv("EHS_FINE_UNFUSED");
  H.fused0 = (precs & 2) && d == 2 && !H.full && fine_tiles_fit(H.g0) && !(uf && uf[0] == '1');
  if (H.fused0) {
    const size_t nc = (size_t)H.nsets * H.g0.ncell;
    H.stab.gdx = dalloc<float2>(c, nc);
    H.stab.gdy = dalloc<float2>(c, nc);
    H.stab.dvx = dalloc<float2>(c, nc);
    H.stab.dvy = dalloc<float2>(c, nc);
    H.stab.sinv = dalloc<float2>(c, nc);
    H.stab.vm = dalloc<float>(c, (size_t)H.nsets * sweep_table_vertices(H.g0));
    launch_sweep_tables(H.g0, H.nsets, H.cf32, H.h, H.alpha, H.stab, c->s); cnt(2); post();
  }
  // opts.coarse_persist: the MG-DD coarsest solve of the 2D complex64 cycle as one persistent launch
  H.persist = (precs & 2) && mgdd && c->opt.coarse_persist && coarse_persist_supported(C.g, H.coarse_fmt);
  if (H.persist) H.pbar = dalloc<unsigned>(c, 2);
  if (const char* f = getenv("EHS_ROWS_VARIANT")) {   // fixed launch shape (tests)
    const int v = atoi(f);
    if (v >= 0 && v < ST_ROWS_VARIANTS)
      for (Level& L : H.lv) L.rows_var[0] = L.rows_var[1] = v;
  }
}

template <typename T> struct PT;
template <> struct PT<double> { static const int i = 0; };
template <> struct PT<float> { static const int i = 1; };

template <typename T> const Coef4<T>* cfp(const Hier& H);
template <> const Coef4<double>* cfp<double>(const Hier& H) { return H.cf64; }
template <> const Coef4<float>* cfp<float>(const Hier& H) { return H.cf32; }
// stencil table of a Galerkin level for the cycle precision T, and its format
template <typename T> const void* tabp(const Hier& H, const Level& L, int* fmt);
template <> const void* tabp<double>(const Hier&, const Level& L, int* fmt) { *fmt = 0; return L.tab64; }
template <> const void* tabp<float>(const Hier& H, const Level& L, int* fmt) {
  if (H.half && L.tabh) { *fmt = H.half; return L.tabh; }
  *fmt = 0;
  return L.tab32;
}

template <typename T>
void level_apply(ehs_ctx* c, const Hier& H, int l, double alpha, const typename CT<T>::type* x,
                 const typename CT<T>::type* b, typename CT<T>::type* y, int mode) {
  const Level& L = H.lv[l];
  if (l == 0) {
    launch_fine_apply<T>(L.g, H.items, H.nrhs, cfp<T>(H), H.h, alpha, x, b, y, mode, c->s);
  } else {
    int fmt = 0;
    const void* tab = tabp<T>(H, L, &fmt);
    launch_st_apply<T>(L.g, H.items, H.nrhs, L.L, tab, fmt, x, b, y, mode, L.rows_var[PT<T>::i], c->s);
  }
  cnt(); post();
}

// one red-black sweep on level l: x -> t -> x
template <typename T>
void level_sweep(ehs_ctx* c, const Hier& H, int l, const typename CT<T>::type* b,
                 typename CT<T>::type* x, typename CT<T>::type* t) {
  const Level& L = H.lv[l];
  const T wu = (T)L.w, wp = (T)(L.w * H.wp_ratio);
  if (l == 0) {
    launch_fine_vanka<T>(L.g, H.items, H.nrhs, cfp<T>(H), H.h, H.alpha, wu, wp, 0, b, x, t, c->s, H.full);
    launch_fine_vanka<T>(L.g, H.items, H.nrhs, cfp<T>(H), H.h, H.alpha, wu, wp, 1, b, t, x, c->s, H.full);
  } else {
    typedef typename CT<T>::type C;
    C* rb = (C*)L.ws[PT<T>::i][3];
    int fmt = 0;
    const void* tab = tabp<T>(H, L, &fmt);
    const int var = L.rows_var[PT<T>::i];
    if (H.full) {
      const void* bi = L.binv[PT<T>::i];
      const int bfmt = sizeof(T) == 4 ? H.half : 0;
      launch_st_vanka_full<T>(L.g, H.items, H.nrhs, L.L, tab, fmt, bi, bfmt, wu, wp, 0, b, x, t, rb, var, c->s);
      launch_st_vanka_full<T>(L.g, H.items, H.nrhs, L.L, tab, fmt, bi, bfmt, wu, wp, 1, b, t, x, rb, var, c->s);
    } else {
      launch_st_vanka<T>(L.g, H.items, H.nrhs, L.L, tab, fmt, wu, wp, 0, b, x, t, rb, var, c->s);
      launch_st_vanka<T>(L.g, H.items, H.nrhs, L.L, tab, fmt, wu, wp, 1, b, t, x, rb, var, c->s);
    }
    cnt(2);
  }
  cnt(2); post();
}

// Setup autotuner: times every residual-pass launch shape of each smoothed
// Galerkin level, and of the coarsest level under MG-DD (its working precision
// and table format, on the level's own buffers) and keeps the fastest.  Runs
// at setup, outside any capture.
template <typename T>
void autotune_rows(ehs_ctx* c, Hier& H) {
  typedef typename CT<T>::type C;
  const int p = PT<T>::i;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // smoothed Galerkin levels, and the coarsest level when the MG-DD sweep takes residuals there
  const int ltop = H.cdd.nsub ? H.nlev : H.nlev - 1;
  for (int l = 1; l < ltop; ++l) {
    Level& L = H.lv[l];
    int fmt = 0;
    const void* tab = tabp<T>(H, L, &fmt);
    float best = 1e30f;
    int bestv = 0;
    for (int v = 0; v < ST_ROWS_VARIANTS; ++v) {
      float tsum = 0.0f;
      for (int rep = 0; rep < 4; ++rep) {
        CK(cudaEventRecord(e0, c->s));
        launch_st_apply<T>(L.g, H.items, H.nrhs, L.L, tab, fmt, (const C*)L.ws[p][1], (const C*)L.ws[p][0],
                           (C*)L.ws[p][3], 1, v, c->s);
        CK(cudaEventRecord(e1, c->s));
        CK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (rep) tsum += ms;                // the first run warms caches and code
      }
      cnt(4); post();
      if (tsum < best) { best = tsum; bestv = v; }
    }
    L.rows_var[p] = bestv;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

// x = K_c^{-1} b through the stored dense inverses of the coarsest level (the
// whole level, or the MG-DD subdomains: items are then sub-items)
template <typename T>
void coarse_gemv(ehs_ctx* c, const Hier& H, const Level& L, int N, int items, const typename CT<T>::type* b,
                 typename CT<T>::type* x) {
  if (PT<T>::i == 1) {
    if (L.invlp)   // complex64 / FP16 / BF16 inverse, FP32 accumulation
      launch_dense_apply_lp(N, items, H.nrhs, H.cdd.nsub ? H.cdd.nsub : 1, H.cdd.nsub ? H.cdd.d_sizes : nullptr,
                            L.invlp, H.coarse_fmt, (const float2*)b, (float2*)x, c->s);
    else           // FP64-class (df64) inverse on the FP32 pipe
      launch_dense_apply_df(N, items, H.nrhs, L.invdf, (const float2*)b, (float2*)x, c->s);
  } else {
    launch_dense_apply<T>(N, items, H.nrhs, L.inv, b, x, c->s);
  }
  cnt(); post();
}

// MG-DD coarsest solve (Sec. 4 with Algorithm DD): one multiplicative sweep
// over the colours from x = 0; before every colour but the first the residual
// b - K_c x is recomputed at the colour's subdomain unknowns (fused with their
// gather), solved with the subdomains' dense inverses and scatter-added on the
// subdomain unknowns.
template <typename T>
void coarse_dd_solve(ehs_ctx* c, Hier& H, const typename CT<T>::type* b, typename CT<T>::type* x) {
  typedef typename CT<T>::type C;
  const int l = H.nlev - 1;
  const Level& L = H.lv[l];
  CoarseDD& D = H.cdd;
  const int p = PT<T>::i;
  if constexpr (sizeof(T) == 4) {
    if (H.persist) {   // every colour in one persistent launch
      int fmt = 0;
      const void* tab = tabp<float>(H, L, &fmt);
      const int ncol = (int)D.col_subs.size();
      const int* cs[8] = {nullptr};
      int ncs[8] = {0};
      for (int k = 0; k < ncol && k < 8; ++k) {
        cs[k] = D.d_col_subs[k];
        ncs[k] = (int)D.col_subs[k].size();
      }
      launch_coarse_dd_persist(L.g, l >= 2 ? 2 : 1, fmt, H.coarse_fmt, H.nrhs, D.nsub, D.nloc, D.d_map, D.d_sizes, tab,
                               L.invlp, (const float2*)b, (float2*)x, (float2*)D.loc[1][0], (float2*)D.loc[1][1],
                               g_sel.list, (int)sel_items(H.items), cs, ncs, ncol, H.pbar, c->derr, c->s);
      cnt(); post();
      return;
    }
  }
  const long long NG = (long long)(L.g.d + 1) * L.g.ncell;
  C* rs = (C*)D.loc[p][0];
  C* zs = (C*)D.loc[p][1];
  CK(cudaMemsetAsync(x, 0, (size_t)H.items * NG * sizeof(C), c->s));
  const int nact = (int)sel_items(H.items);
  const int* act = g_sel.list;
  bool first = true;
  for (int col = 0; col < (int)D.col_subs.size(); ++col) {
    const int ncs = (int)D.col_subs[col].size();
    if (!ncs) continue;
    const int* lst = D.d_list_all[col];   // every item active: the list built at setup
    if (act) {
      launch_expand_items(act, nact, H.nrhs, D.nsub, D.d_col_subs[col], ncs, D.d_list[col], c->s); cnt(); post();
      lst = D.d_list[col];
    }
    SelScope sel(lst, nact * ncs);
    const int items_l = H.items * D.nsub;
    if (first) {   // x = 0: the residual is b
      launch_dd_gather<T>(D.nloc, items_l, D.nsub, H.nrhs, NG, D.d_map, b, rs, c->s);
    } else {       // b - K_c x at the colour's box unknowns only, straight into the local vectors
      int fmt = 0;
      const void* tab = tabp<T>(H, L, &fmt);
      launch_st_resid_gather<T>(L.g, items_l, H.nrhs, D.nsub, D.nloc, D.d_map, L.L, tab, fmt, x, b, rs, c->s);
    }
    cnt(); post();
    first = false;
    if constexpr (sizeof(T) == 4) {   // local products with the scatter-add folded in
      if (L.invlp && launch_dense_apply_scatter(D.nloc, items_l, H.nrhs, D.nsub, D.d_sizes, L.invlp, H.coarse_fmt,
                                                (const float2*)rs, D.d_map, NG, (float2*)x, c->s)) {
        cnt(); post();
        continue;
      }
    }
    coarse_gemv<T>(c, H, L, D.nloc, items_l, rs, zs);
    launch_dd_scatter<T>(D.nloc, items_l, D.nsub, H.nrhs, NG, D.d_map, zs, x, c->s); cnt(); post();
  }
}

template <typename T>
void cycle_rec(ehs_ctx* c, Hier& H, int l, const typename CT<T>::type* b, typename CT<T>::type* x,
               bool guess);

// Fine level of the 2D complex64 cycle with the fused kernels: pre-smoothing
// sweeps (the first from the zero guess without reading x), residual and
// restriction in one pass, the coarse cycle, and post-smoothing sweeps whose
// first adds the prolongated correction while staging x.  Each sweep writes the
// buffer it does not read (x or the level's t), chosen so that the last lands
// in x.
void cycle_fine_fused(ehs_ctx* c, Hier& H, const float2* b, float2* x, bool guess) {
  Level& L = H.lv[0];
  Level& Lc = H.lv[1];
  float2* t = (float2*)L.ws[1][2];
  float2* bc = (float2*)Lc.ws[1][0];
  float2* xc = (float2*)Lc.ws[1][1];
  const float wu = (float)L.w, wp = (float)(L.w * H.wp_ratio);
  const float2* cur = guess ? x : nullptr;            // nullptr: the zero iterate
  float2* out = guess ? t : (((H.nu1 + H.nu2) & 1) ? x : t);
  auto sweep = [&](const float2* ec) {
    launch_fine_sweep_tile(L.g, Lc.g, H.items, H.nrhs, H.cf32, H.stab, H.h, H.alpha, wu, wp, b, cur, ec, out, c->s);
    cnt(); post();
    cur = out;
    out = out == t ? x : t;
  };
  for (int s = 0; s < H.nu1; ++s) sweep(nullptr);
  launch_fine_resid_restrict_tile(L.g, Lc.g, H.items, H.nrhs, H.cf32, H.stab, H.h, H.alpha, cur, b, bc, c->s);
  cnt(); post();
  const int reps = (1 == H.nlev - 1) ? 1 : H.cyc;
  for (int k = 0; k < reps; ++k) cycle_rec<float>(c, H, 1, bc, xc, k > 0);
  for (int s = 0; s < H.nu2; ++s) sweep(s == 0 ? xc : nullptr);
  if (cur != x) {   // only with an initial guess and an odd number of sweeps; copies every item
                    // (the vectors of items outside an active list are not read afterwards)
    const long long nv = (long long)H.items * 3 * L.g.ncell;
    CK(cudaMemcpyAsync(x, cur, nv * sizeof(float2), cudaMemcpyDeviceToDevice, c->s));
  }
}

template <typename T>
void cycle_rec(ehs_ctx* c, Hier& H, int l, const typename CT<T>::type* b, typename CT<T>::type* x,
               bool guess) {
  typedef typename CT<T>::type C;
  Level& L = H.lv[l];
  const int p = PT<T>::i;
  const long long nv = (long long)H.items * (L.g.d + 1) * L.g.ncell;
  if (l == H.nlev - 1) {
    if (H.cdd.nsub) coarse_dd_solve<T>(c, H, b, x);
    else coarse_gemv<T>(c, H, L, (int)((L.g.d + 1) * L.g.ncell), H.items, b, x);
    return;
  }
  if constexpr (sizeof(T) == 4) {
    if (l == 0 && H.fused0 && H.nu1 >= 1 && H.nu2 >= 1) {
      cycle_fine_fused(c, H, b, x, guess);
      return;
    }
  }
  C* t = (C*)L.ws[p][2];
  C* r = (C*)L.ws[p][3];
  if (!guess) CK(cudaMemsetAsync(x, 0, nv * sizeof(C), c->s));
  for (int s = 0; s < H.nu1; ++s) level_sweep<T>(c, H, l, b, x, t);
  level_apply<T>(c, H, l, H.alpha, x, b, r, 1);
  Level& Lc = H.lv[l + 1];
  C* bc = (C*)Lc.ws[p][0];
  C* xc = (C*)Lc.ws[p][1];
  launch_restrict<T>(L.g, Lc.g, H.items, r, bc, c->s); cnt(); post();
  const int reps = (l + 1 == H.nlev - 1) ? 1 : H.cyc;
  for (int k = 0; k < reps; ++k) cycle_rec<T>(c, H, l + 1, bc, xc, k > 0);
  launch_prolong_add<T>(L.g, Lc.g, H.items, xc, x, c->s); cnt(); post();
  for (int s = 0; s < H.nu2; ++s) level_sweep<T>(c, H, l, b, x, t);
}

// ------------------------------------------------------------------ checks
bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void validate(const ehs_problem* P, const ehs_opts* O) {
  if (!P || !O) throw ArgError("null problem or options");
  if (P->dim != 2 && P->dim != 3) throw ArgError("dim must be 2 or 3");
  if (O->levels < 2 || O->levels > 8) throw ArgError("levels must be in [2, 8]");
  const int f = 1 << (O->levels - 1);
  for (int k = 0; k < P->dim; ++k)
    if (P->n[k] < 2 * f || P->n[k] % f) throw ArgError("every n[k] must be a multiple of 2^(levels-1), at least twice it");
  if (!(P->h > 0) || (!P->omegas && (!std::isfinite(P->omega) || !(P->omega > 0))))
    throw ArgError("h and omega must be positive and finite");
  if (P->nmedia < 1 || O->nrhs < 1) throw ArgError("nmedia and nrhs must be >= 1");
  if (!P->lambda || !P->mu || !P->rho) throw ArgError("null media pointer");
  if (O->restart < 1 || O->restart > 11) throw ArgError("restart must be in [1, 11]");
  if (O->prec != EHS_C64 && O->prec != EHS_C128) throw ArgError("prec must be EHS_C64 or EHS_C128");
  if (O->cycle != 1 && O->cycle != 2) throw ArgError("cycle must be 1 (V) or 2 (W)");
  if (O->nu_pre < 0 || O->nu_post < 0) throw ArgError("negative sweep count");
  if (!(O->tol > 0)) throw ArgError("tol must be positive");
  if (P->abl_cells < 0 || 2 * P->abl_cells > P->n[0]) throw ArgError("bad abl_cells");
  if (O->precond != EHS_PRECOND_MG && O->precond != EHS_PRECOND_DD) throw ArgError("bad precond");
  if (O->coef_half < 0 || O->coef_half > 2) throw ArgError("coef_half must be 0, 1 (FP16) or 2 (BF16)");
  if (O->vanka_full != 0 && O->vanka_full != 1) throw ArgError("vanka_full must be 0 or 1");
  if (O->coarse_fmt < 0 || O->coarse_fmt > 3) throw ArgError("coarse_fmt must be 0..3");
  if (O->coarse_persist != 0 && O->coarse_persist != 1) throw ArgError("coarse_persist must be 0 or 1");
  if (O->ortho != 0 && O->ortho != 1) throw ArgError("ortho must be 0 (CGS2) or 1 (delayed CGS2)");
  for (int k = 0; k < 3; ++k)
    if (O->coarse_dd[k] < 0) throw ArgError("coarse_dd must be >= 0");
  // MG-DD on the global hierarchy: the coarsest grid is known here (DD contexts split the
  // coarsest grids of their subdomain hierarchies, checked when those are built)
  if (O->precond == EHS_PRECOND_MG && (O->coarse_dd[0] > 1 || O->coarse_dd[1] > 1 || (P->dim == 3 && O->coarse_dd[2] > 1))) {
    if (O->coarse_dd_overlap < 1) throw ArgError("coarse_dd_overlap must be >= 1");
    for (int k = 0; k < P->dim; ++k) {
      const int nc = P->n[k] >> (O->levels - 1), ns = std::max(O->coarse_dd[k], 1);
      if (ns > nc) throw ArgError("coarse_dd split larger than the coarsest grid");
      if (ns > 1 && 2 * O->coarse_dd_overlap > nc / ns)
        throw ArgError("coarse_dd_overlap larger than half a coarsest-grid core");
    }
  }
  // dense inverses of the global coarsest level: the whole level, or every MG-DD box
  if (O->precond == EHS_PRECOND_MG) {
    int nc[3] = {1, 1, 1}, ns[3] = {1, 1, 1};
    long long cells = 1;
    for (int k = 0; k < P->dim; ++k) {
      nc[k] = P->n[k] >> (O->levels - 1);
      ns[k] = std::max(O->coarse_dd[k], 1);
      cells *= nc[k];
    }
    if (ns[0] * ns[1] * ns[2] == 1) {
      if ((P->dim + 1) * cells > 16384)
        throw ArgError("coarsest grid too large for the dense FP64 inverse (use more levels or coarse_dd)");
    } else {
      long long big = 0;   // unknowns of the largest box: its pressures and the faces with both cells inside
      int id[3];
      for (id[2] = 0; id[2] < ns[2]; ++id[2])
        for (id[1] = 0; id[1] < ns[1]; ++id[1])
          for (id[0] = 0; id[0] < ns[0]; ++id[0]) {
            long long ext[3] = {1, 1, 1};
            for (int k = 0; k < P->dim; ++k) {
              const int lo0 = id[k] * (nc[k] / ns[k]) + std::min(id[k], nc[k] % ns[k]);
              const int hi0 = lo0 + nc[k] / ns[k] + (id[k] < nc[k] % ns[k] ? 1 : 0);
              ext[k] = std::min(hi0 + O->coarse_dd_overlap, nc[k]) - std::max(lo0 - O->coarse_dd_overlap, 0);
            }
            long long nbox = ext[0] * ext[1] * ext[2];
            for (int a = 0; a < P->dim; ++a) nbox += ext[0] * ext[1] * ext[2] / ext[a] * (ext[a] - 1);
            big = std::max(big, nbox);
          }
      if ((big + 7) / 8 * 8 > 16384) throw ArgError("coarse_dd subdomains too large for dense local inverses");
    }
  }
}

void check_media(ehs_ctx* c, const double* lam, const double* mu, const double* rho, long long n) {
  std::vector<double> L(n), M(n), R(n);
  CK(cudaMemcpy(L.data(), lam, n * sizeof(double), cudaMemcpyDefault));
  CK(cudaMemcpy(M.data(), mu, n * sizeof(double), cudaMemcpyDefault));
  CK(cudaMemcpy(R.data(), rho, n * sizeof(double), cudaMemcpyDefault));
  for (long long i = 0; i < n; ++i) {
    if (!std::isfinite(L[i]) || !std::isfinite(M[i]) || !std::isfinite(R[i])) throw ArgError("non-finite medium value");
    if (!(R[i] > 0)) throw ArgError("rho must be positive");
    if (M[i] < 0) throw ArgError("mu must be non-negative");
    if (!(L[i] + M[i] > 0)) throw ArgError("lambda + mu must be positive");
  }
}

}  // namespace

namespace {

// Sets the active item list from the Arnoldi state (no list when every item
// is active) and derives the DD sub-item lists; bumps the graph version when
// the set changes.
void set_active(ehs_ctx* c, const std::vector<int>& active) {
  std::vector<int> list;
  for (int b = 0; b < (int)active.size(); ++b)
    if (active[b]) list.push_back(b);
  if ((int)list.size() == (int)active.size()) list.clear();
  if (list == c->act) return;
  c->act = list;
  ++c->act_ver;
  if (list.empty()) return;
  CK(cudaMemcpyAsync(c->d_act, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice, c->s));
  const int nrhs = c->H.nrhs;
  for (int col = 0; col < 8; ++col)
    for (DDGroup& grp : c->dd[col]) {
      std::vector<int> sl;
      for (int b : list) {
        const int m = b / nrhs, r = b % nrhs;
        for (int sdx = 0; sdx < grp.nsub; ++sdx) sl.push_back((m * grp.nsub + sdx) * nrhs + r);
      }
      grp.nsub_act = (int)sl.size();
      CK(cudaMemcpyAsync(grp.d_sub_act, sl.data(), sl.size() * sizeof(int), cudaMemcpyHostToDevice, c->s));
    }
  CK(cudaStreamSynchronize(c->s));   // the host lists above are temporaries
}


}  // namespace

// ------------------------------------------------------------------- DD
#include "dd_impl.inc"

// ------------------------------------------------------------------ FGMRES
namespace {

void givens(zc a, zc b, double* cs, zc* sn, zc* r) {
  if (b == 0.0) { *cs = 1; *sn = 0; *r = a; return; }
  if (a == 0.0) { *cs = 0; *sn = std::conj(b) / std::abs(b); *r = std::abs(b); return; }
  const double t = std::abs(a), nr = std::hypot(t, std::abs(b));
  *cs = t / nr;
  *sn = (a / t) * std::conj(b) / nr;
  *r = (a / t) * nr;
}

// Host side of FGMRES(m) for every item: Hessenberg columns, complex Givens
// rotations, residual estimates, per-item convergence and iteration counts.
// The (m+1) x m least-squares problem is tiny; everything of length n runs in
// the kernels.
struct Arnoldi {
  int items, m, maxit;
  double tol;
  std::vector<zc> H, g, sn;
  std::vector<zc> Hr;          // unrotated Hessenberg matrix (delayed CGS2 corrects a column later)
  std::vector<double> cs, bnorm, beta, rho;
  std::vector<int> iters, done, kused, active;
  bool breakdown = false, nonfinite = false;

  Arnoldi(int items_, int m_, int maxit_, double tol_)
      : items(items_), m(m_), maxit(maxit_), tol(tol_), H((size_t)items_ * (m_ + 1) * m_),
        g((size_t)items_ * (m_ + 1)), sn((size_t)items_ * m_), Hr((size_t)items_ * (m_ + 1) * m_),
        cs((size_t)items_ * m_), bnorm(items_), beta(items_), rho(items_, 0.0), iters(items_, 0),
        done(items_, 0), kused(items_, 0), active(items_, 0) {}

  void set_b(const double* nrm) {
    for (int b = 0; b < items; ++b) {
      bnorm[b] = beta[b] = nrm[b];
      done[b] = !(bnorm[b] > 0);
    }
  }
  bool all_done() const {
    for (int b = 0; b < items; ++b) if (!done[b]) return false;
    return true;
  }
  bool maxed() const {
    for (int b = 0; b < items; ++b) if (!done[b] && iters[b] < maxit) return false;
    return true;
  }
  void start_cycle() {
    std::fill(H.begin(), H.end(), zc(0));
    std::fill(Hr.begin(), Hr.end(), zc(0));
    std::fill(g.begin(), g.end(), zc(0));
    for (int b = 0; b < items; ++b) {
      g[(size_t)b * (m + 1)] = beta[b];
      kused[b] = 0;
      active[b] = !done[b] && iters[b] < maxit;
    }
  }
  // applies the rotations of columns < j to column j of item b's H, forms the rotation of
  // column j and applies it to g
  void rotate(int b, int j) {
    zc* Hb = &H[(size_t)b * (m + 1) * m];
    zc* gb = &g[(size_t)b * (m + 1)];
    for (int i = 0; i < j; ++i) {
      const zc t = cs[b * m + i] * Hb[i * m + j] + sn[b * m + i] * Hb[(i + 1) * m + j];
      Hb[(i + 1) * m + j] = -std::conj(sn[b * m + i]) * Hb[i * m + j] + cs[b * m + i] * Hb[(i + 1) * m + j];
      Hb[i * m + j] = t;
    }
    zc rr;
    givens(Hb[j * m + j], Hb[(j + 1) * m + j], &cs[b * m + j], &sn[b * m + j], &rr);
    Hb[j * m + j] = rr;
    Hb[(j + 1) * m + j] = 0.0;
    gb[j + 1] = -std::conj(sn[b * m + j]) * gb[j];
    gb[j] = cs[b * m + j] * gb[j];
  }
  // counts step j of item b and tests its residual estimate; false once the item stops
  bool count(int b, int j, double hn) {
    iters[b] += 1;
    kused[b] = j + 1;
    const double res = std::abs(g[(size_t)b * (m + 1) + j + 1]) / bnorm[b];
    if (!std::isfinite(res)) { nonfinite = true; active[b] = 0; return false; }
    if (hn == 0.0) { active[b] = 0; if (res > tol) breakdown = true; return false; }
    if (res <= tol || iters[b] >= maxit) { active[b] = 0; return false; }
    return true;
  }
  // column j of H from h = h1 + h2 ([items][j+1]) and hn; true if an item is still active
  bool step(int j, const double2* h1, const double2* h2, const double* hn) {
    const int nv = j + 1;
    bool any = false;
    for (int b = 0; b < items; ++b) {
      if (!active[b]) continue;
      zc* Hb = &H[(size_t)b * (m + 1) * m];
      for (int i = 0; i < nv; ++i)
        Hb[i * m + j] = zc(h1[b * nv + i].x + h2[b * nv + i].x, h1[b * nv + i].y + h2[b * nv + i].y);
      Hb[(j + 1) * m + j] = hn[b];
      rotate(b, j);
      any = count(b, j, hn[b]) || any;
    }
    return any;
  }
  // Delayed CGS2: p[b * stride ...] = a_0..a_{j-1}, sigma, b_0..b_{j-1}, h_j, rho of step j.
  // Corrects column j - 1 of the unrotated matrix Hr (u_j = V_j a + sigma v_j, so its
  // column gains rho_{j-1} a above the diagonal and its subdiagonal becomes
  // rho_{j-1} sigma), sets column j to (b, h_j, rho), and redoes the Givens QR of
  // columns 0..j from Hr (column j - 1 changed after its rotation was formed).
  bool step_delayed(int j, const double2* p, int stride) {
    bool any = false;
    for (int b = 0; b < items; ++b) {
      if (!active[b]) continue;
      const double2* pa = p + (size_t)b * stride;
      const double2* pb = pa + j + 1;
      zc* R = &Hr[(size_t)b * (m + 1) * m];
      if (j > 0) {
        for (int i = 0; i < j; ++i) R[i * m + j - 1] += rho[b] * zc(pa[i].x, pa[i].y);
        R[j * m + j - 1] = rho[b] * pa[j].x;
      }
      for (int i = 0; i <= j; ++i) R[i * m + j] = zc(pb[i].x, pb[i].y);
      R[(j + 1) * m + j] = pb[j + 1].x;
      rho[b] = pb[j + 1].x;
      zc* Hb = &H[(size_t)b * (m + 1) * m];
      zc* gb = &g[(size_t)b * (m + 1)];
      std::fill(gb, gb + m + 1, zc(0));
      gb[0] = beta[b];
      for (int l = 0; l <= j; ++l) {
        for (int i = 0; i <= l + 1; ++i) Hb[i * m + l] = R[i * m + l];
        rotate(b, l);
      }
      any = count(b, j, rho[b]) || any;
    }
    return any;
  }
  // y = R^{-1} g per item, [items][m] (zero beyond kused)
  void solve_y(std::vector<double2>& y) const {
    y.assign((size_t)items * m, make_double2(0, 0));
    for (int b = 0; b < items; ++b) {
      const int k = kused[b];
      const zc* Hb = &H[(size_t)b * (m + 1) * m];
      const zc* gb = &g[(size_t)b * (m + 1)];
      std::vector<zc> yv(k);
      for (int i = k - 1; i >= 0; --i) {
        zc acc = gb[i];
        for (int l = i + 1; l < k; ++l) acc -= Hb[i * m + l] * yv[l];
        yv[i] = acc / Hb[i * m + i];
      }
      for (int i = 0; i < k; ++i) y[(size_t)b * m + i] = make_double2(yv[i].real(), yv[i].imag());
    }
  }
  void end_cycle(const double* rnorm) {
    for (int b = 0; b < items; ++b) {
      beta[b] = rnorm[b];
      if (!std::isfinite(beta[b])) { nonfinite = true; done[b] = 1; }
      if (!done[b] && beta[b] / bnorm[b] <= tol) done[b] = 1;
    }
  }
  ehs_status finish(ehs_ctx* c, ehs_solve_info* info) const {
    bool allconv = true;
    for (int b = 0; b < items; ++b) {
      const double rel = bnorm[b] > 0 ? beta[b] / bnorm[b] : 0.0;
      const int conv = rel <= tol;
      allconv = allconv && conv;
      if (info) { info[b].iters = iters[b]; info[b].relres = rel; info[b].converged = conv; }
    }
    if (nonfinite) { c->err = "non-finite residual norm"; return EHS_ERR_NONFINITE; }
    if (!allconv && breakdown) { c->err = "Arnoldi breakdown before tol"; return EHS_ERR_BREAKDOWN; }
    if (!allconv) { c->err = "maxit reached before tol"; return EHS_ERR_NOCONV; }
    return EHS_OK;
  }
};

void sync_read(ehs_ctx* c, void* host, const void* dev, size_t bytes) {
  CK(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
}

// Runs body() (a fixed sequence of launches on c->s) directly, or replays it
// from a CUDA graph captured on the first call for slot j.
template <typename F> void graphed(ehs_ctx* c, int j, F body) {
  if (!c->use_graphs) { body(); return; }
  if (c->pg[j] && c->pg_ver[j] != c->act_ver) {   // the active item set changed
    cudaGraphExecDestroy(c->pg[j]);
    c->pg[j] = nullptr;
  }
  if (!c->pg[j]) {
    cudaStream_t user = c->s;
    const long long l0 = g_launches.load();
    c->s = c->cap;
    CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    cudaGraph_t graph = nullptr;
    try {
      body();
    } catch (...) {
      cudaStreamEndCapture(c->cap, &graph);
      if (graph) cudaGraphDestroy(graph);
      c->s = user;
      throw;
    }
    c->s = user;
    CK(cudaStreamEndCapture(c->cap, &graph));
    cudaGraphExec_t ex = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    c->pg[j] = ex;
    c->pg_ver[j] = c->act_ver;
    c->pg_nodes[j] = g_launches.load() - l0;
    g_launches -= c->pg_nodes[j];          // counted when replayed
  }
  CK(cudaGraphLaunch(c->pg[j], c->s));
  g_launches += c->pg_nodes[j];
}

// ---- plain FP64 form: complex128 vectors, FP64 kernels, FP64 cycle -------
ehs_status fgmres_c128(ehs_ctx* c, const double2* q, double2* u, ehs_solve_info* info) {
  const int items = c->H.items, m = c->opt.restart, nblk = c->nblk;
  const long long n = c->n0;
  cudaStream_t s = c->s;
  Arnoldi A(items, m, c->opt.maxit, c->opt.tol);
  launch_norm_part(n, items, q, c->npart, nblk, s);
  launch_reduce_norm(items, nblk, c->npart, c->nrm, s); cnt(2); post();
  sync_read(c, c->hpin, c->nrm, items * sizeof(double));
  A.set_b(c->hpin);
  CK(cudaMemsetAsync(u, 0, (size_t)items * n * sizeof(double2), s));
  CK(cudaMemcpyAsync(c->rd, q, (size_t)items * n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  std::vector<double2> yh;
  while (!A.all_done() && !A.maxed()) {
    CK(cudaMemcpyAsync(c->nrm, A.beta.data(), items * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_scale_inv(n, items, c->rd, c->nrm, c->V, s); cnt(); post();
    A.start_cycle();
    for (int j = 0; j < m; ++j) {
      double2* Vj = c->V + (size_t)j * items * n;
      double2* Zj = c->Z + (size_t)j * items * n;
      graphed(c, j, [&]() {
        if (c->opt.precond == EHS_PRECOND_DD) dd_apply_t<double>(c, Vj, Zj);
        else cycle_rec<double>(c, c->H, 0, Vj, Zj, false);
      });
      launch_fine_apply<double>(c->H.g0, items, c->H.nrhs, c->H.cf64, c->H.h, 0.0, Zj, nullptr, c->w, 0, s);
      const int nv = j + 1;
      launch_mdot(n, items, nv, c->V, c->w, c->part, nblk, s);
      launch_reduce_parts(items, nv, nblk, c->part, c->hd, 0, s);
      launch_mupdate(n, items, nv, c->V, c->hd, c->w, c->part, nblk, 1, nullptr, s);
      launch_reduce_parts(items, nv, nblk, c->part, c->y, 0, s);
      launch_mupdate(n, items, nv, c->V, c->y, c->w, nullptr, nblk, 0, c->npart, s);
      launch_reduce_norm(items, nblk, c->npart, c->nrm, s);
      cnt(7); post();
      double2* ph1 = c->hstep;                         // pinned: no pageable copies
      double2* ph2 = c->hstep + (size_t)items * 12;
      double* phn = (double*)(c->hstep + (size_t)items * 24);
      CK(cudaMemcpyAsync(ph1, c->hd, (size_t)items * nv * sizeof(double2), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(ph2, c->y, (size_t)items * nv * sizeof(double2), cudaMemcpyDeviceToHost, s));
      sync_read(c, phn, c->nrm, items * sizeof(double));
      if (!A.step(j, ph1, ph2, phn)) break;
      launch_scale_inv(n, items, c->w, c->nrm, c->V + (size_t)(j + 1) * items * n, s); cnt(); post();
    }
    A.solve_y(yh);
    CK(cudaMemcpyAsync(c->y, yh.data(), (size_t)items * m * sizeof(double2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->kused, A.kused.data(), items * sizeof(int), cudaMemcpyHostToDevice, s));
    launch_xupdate<double2>(n, items, m, c->Z, c->y, c->kused, u, s);
    launch_fine_apply<double>(c->H.g0, items, c->H.nrhs, c->H.cf64, c->H.h, 0.0, u, q, c->rd, 1, s);
    launch_norm_part(n, items, c->rd, c->npart, nblk, s);
    launch_reduce_norm(items, nblk, c->npart, c->nrm, s); cnt(4); post();
    sync_read(c, c->hpin, c->nrm, items * sizeof(double));
    A.end_cycle(c->hpin);
    if (A.nonfinite || A.breakdown) break;
  }
  return A.finish(c, info);
}

// ---- mixed form: complex64 cycle, FP64-class (df64) Krylov ----------------
ehs_status fgmres_df(ehs_ctx* c, const double2* q, double2* u, ehs_solve_info* info) {
  const int items = c->H.items, m = c->opt.restart, nblk = c->nblk;
  const long long n = c->n0;
  const long long nall = (long long)items * n;
  cudaStream_t s = c->s;
  Arnoldi A(items, m, c->opt.maxit, c->opt.tol);
  launch_d2_to_df(nall, q, c->qq, s);
  launch_norm_part_df(n, items, c->qq, c->npq, nblk, s);
  launch_reduce_norm_df(items, nblk, c->npq, c->nrm, c->invq, s); cnt(3); post();
  sync_read(c, c->hpin, c->nrm, items * sizeof(double));
  A.set_b(c->hpin);
  CK(cudaMemsetAsync(c->xq, 0, nall * sizeof(float4), s));
  CK(cudaMemcpyAsync(c->rq, c->qq, nall * sizeof(float4), cudaMemcpyDeviceToDevice, s));
  std::vector<double2> yh;
  while (!A.all_done() && !A.maxed()) {
    A.start_cycle();
    set_active(c, A.active);
    {  // V_0 = r / beta (invq holds 1/||r|| from the last norm) and its complex64 copy
      SelScope sel = global_sel(c);
      launch_scale_cast_df(n, items, c->rq, c->invq, c->Vq, c->f_in, s); cnt(); post();
    }
    for (int j = 0; j < m; ++j) {
      float2* Zj = c->Zf + (size_t)j * items * n;
      SelScope sel = global_sel(c);      // only the items still iterating
      graphed(c, j, [&]() {               // f_in holds V_j in complex64
        if (c->opt.precond == EHS_PRECOND_DD) dd_apply_t<float>(c, c->f_in, Zj);
        else cycle_rec<float>(c, c->H, 0, c->f_in, Zj, false);
      });
      launch_fine_apply_df(c->H.g0, items, c->H.nrhs, c->H.cfdf, c->H.h, 0.0, Zj, 1, nullptr, c->wq, 0, s, c->H.kdg,
                           c->H.kvm);
      if (c->opt.ortho == 1) {
        // delayed CGS2: one pass for V^H u_j, V^H w and the norms, whose last block forms the
        // coefficients; one pass for v_j and u_{j+1} (and its complex64 copy in f_in)
        launch_mdot2_df(n, items, j, c->Vq, c->wq, c->partq, nblk, s, c->kcnt, c->dcoef, c->hhost);
        CK(cudaMemcpyAsync(c->hstep, c->hhost, (size_t)items * KDS * sizeof(double2), cudaMemcpyDeviceToHost, s));
        CK(cudaEventRecord(c->ev_step, s));
        launch_dupdate_df(n, items, j, c->Vq, c->wq, c->dcoef, c->f_in, s);
        cnt(3); post();                      // with the operator launch above
        CK(cudaEventSynchronize(c->ev_step));
        if (!A.step_delayed(j, c->hstep, KDS)) break;
        set_active(c, A.active);
        continue;
      }
      // CGS2: h1 = V^H w; w' = w - V h1 (not stored) with h2 = V^H w' and ||w'||^2 in the same
      // pass, whose last block also forms ||w' - V h2|| = sqrt(||w'||^2 - ||h2||^2); then one pass
      // forms V_{j+1} = (w - V (h1 + h2)) / ||.|| and its complex64 copy.  Each reduction is done
      // by the launch's last block.
      const int nv = j + 1;
      int* k0 = c->kcnt;
      int* k1 = c->kcnt + items;
      launch_mdot_df(n, items, nv, c->Vq, c->wq, c->partq, nblk, s, k0, c->hq, c->hhost);
      launch_mupdate_df(n, items, nv, c->Vq, c->hq, c->wq, c->partq, nblk, 1, c->npq, s, k1, c->h2q,
                        c->hhost + (size_t)items * 12, c->nrm, c->invq, 0);
      // one round trip into pinned memory (h1, h2 and the norms), overlapped with the last pass
      double2* ph1 = c->hstep;
      double2* ph2 = c->hstep + (size_t)items * 12;
      double* phn = (double*)(c->hstep + (size_t)items * 24);
      CK(cudaMemcpyAsync(ph1, c->hhost, (size_t)items * 24 * sizeof(double2), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(phn, c->nrm, items * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaEventRecord(c->ev_step, s));
      launch_update_scale_cast_df(n, items, nv, c->Vq, c->h2q, c->wq, c->invq, c->Vq + (size_t)(j + 1) * items * n,
                                  c->f_in, nblk, s, c->hq);
      cnt(4); post();                        // with the operator launch above
      CK(cudaEventSynchronize(c->ev_step));
      if (!A.step(j, ph1, ph2, phn)) break;
      set_active(c, A.active);
    }
    A.solve_y(yh);
    // y to df64 on the device via the double2 -> df64 conversion
    CK(cudaMemcpyAsync(c->hhost, yh.data(), (size_t)items * m * sizeof(double2), cudaMemcpyHostToDevice, s));
    launch_d2_to_df((long long)items * m, c->hhost, c->yq, s);
    CK(cudaMemcpyAsync(c->kused, A.kused.data(), items * sizeof(int), cudaMemcpyHostToDevice, s));
    launch_xupdate_df(n, items, m, c->Zf, c->yq, c->kused, c->xq, s);
    launch_fine_apply_df(c->H.g0, items, c->H.nrhs, c->H.cfdf, c->H.h, 0.0, c->xq, 0, c->qq, c->rq, 1, s, c->H.kdg,
                         c->H.kvm);
    launch_norm_part_df(n, items, c->rq, c->npq, nblk, s);
    launch_reduce_norm_df(items, nblk, c->npq, c->nrm, c->invq, s); cnt(5); post();
    sync_read(c, c->hpin, c->nrm, items * sizeof(double));
    A.end_cycle(c->hpin);
    if (A.nonfinite || A.breakdown) break;
  }
  launch_df_to_d2(nall, c->xq, u, s); cnt(); post();
  return A.finish(c, info);
}

// a persistent launch whose grid barrier gave up (EHS_ERR_TIMEOUT); clears the flag
bool device_timeout(ehs_ctx* c) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, c->derr, sizeof(int), cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  if (h) CK(cudaMemsetAsync(c->derr, 0, sizeof(int), c->s));
  return h != 0;
}

ehs_status fgmres(ehs_ctx* c, const double2* q, double2* u, ehs_solve_info* info) {
  const ehs_status st = c->opt.prec == EHS_C64 ? fgmres_df(c, q, u, info) : fgmres_c128(c, q, u, info);
  if (device_timeout(c)) {
    c->err = "a persistent launch's grid barrier waited past its limit (the SMs were held by other work)";
    return EHS_ERR_TIMEOUT;
  }
  return st;
}

__global__ void k_conj(long long n, double2* v) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) v[e].y = -v[e].y;
}

template <typename F> ehs_status guard(ehs_ctx* c, F f) {
  try {
    return f();
  } catch (const ArgError& e) {
    if (c) c->err = e.what();
    return EHS_ERR_ARG;
  } catch (const CudaError& e) {
    if (c) c->err = e.what();
    return EHS_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    if (c) c->err = "device allocation failed";
    return EHS_ERR_OOM;
  } catch (const std::exception& e) {
    if (c) c->err = e.what();
    return EHS_ERR_CUDA;
  }
}

ehs_status solve_common(ehs_ctx* c, const void* qin, void* uout, ehs_solve_info* info, bool adjoint) {
  const size_t bytes = (size_t)c->H.items * c->n0 * sizeof(double2);
  const bool qdev = is_device_ptr(qin), udev = is_device_ptr(uout);
  const double2* q = (const double2*)qin;
  double2* u = (double2*)uout;
  if (!qdev || adjoint) {
    CK(cudaMemcpyAsync(c->qd, qin, bytes, qdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->s));
    q = c->qd;
  }
  if (!udev) u = c->ud;
  const long long n = (long long)c->H.items * c->n0;
  if (adjoint) { k_conj<<<(unsigned)((n + 255) / 256), 256, 0, c->s>>>(n, c->qd); cnt(); post(); }
  ehs_status st = fgmres(c, q, u, info);
  if (adjoint) { k_conj<<<(unsigned)((n + 255) / 256), 256, 0, c->s>>>(n, u); cnt(); post(); }
  if (!udev) {
    CK(cudaMemcpyAsync(uout, u, bytes, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
  }
  return st;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

void ehs_default_opts(ehs_opts* o) {
  std::memset(o, 0, sizeof(*o));
  o->levels = 3;
  o->alpha = 0.2;
  const double w[8] = {0.75, 0.5, 0.25, 0.25, 0.25, 0.25, 0.25, 0.25};
  for (int i = 0; i < 8; ++i) o->w[i] = w[i];
  o->wp_ratio = 1.0;
  o->nu_pre = o->nu_post = 1;
  o->cycle = 1;
  o->restart = 10;
  o->maxit = 500;
  o->tol = 1e-6;
  o->precond = EHS_PRECOND_MG;
  o->prec = EHS_C64;
  o->nrhs = 1;
  o->dd[0] = o->dd[1] = o->dd[2] = 1;
  o->dd_overlap = 4;
  o->dd_pad = 8;
  o->dd_abl_max = 1.0;
  o->coarse_dd[0] = o->coarse_dd[1] = o->coarse_dd[2] = 1;
  o->coarse_dd_overlap = 2;
  o->ortho = 1;
}

ehs_status ehs_create(const ehs_problem* prob, const ehs_opts* opts, void* stream, ehs_ctx** out) {
  if (!out) { g_create_err = "null output pointer"; return EHS_ERR_ARG; }
  *out = nullptr;
  ehs_ctx* c = new ehs_ctx();
  ehs_status st = guard(c, [&]() -> ehs_status {
    validate(prob, opts);
    c->s = (cudaStream_t)stream;
    c->prob = *prob;
    c->opt = *opts;
    c->d = prob->dim;
    Hier& H = c->H;
    H.g0 = mkgrid(prob->dim, prob->n[0], prob->n[1], prob->n[2]);
    H.nlev = opts->levels;
    H.nsets = prob->nmedia;
    H.nrhs = opts->nrhs;
    H.items = H.nsets * H.nrhs;
    H.h = prob->h; H.alpha = opts->alpha;
    H.wp_ratio = opts->wp_ratio > 0 ? opts->wp_ratio : 1.0;
    H.nu1 = opts->nu_pre; H.nu2 = opts->nu_post; H.cyc = opts->cycle;
    H.half = opts->coef_half;
    H.full = opts->vanka_full;
    for (int k = 0; k < 3; ++k) H.cdd_split[k] = k < prob->dim ? std::max(opts->coarse_dd[k], 1) : 1;
    H.cdd_overlap = opts->coarse_dd_overlap;
    H.coarse_fmt = opts->coarse_fmt;
    c->n0 = (long long)(c->d + 1) * H.g0.ncell;
    c->derr = dalloc<int>(c, 1);
    const long long nc = (long long)H.nsets * H.g0.ncell;
    check_media(c, prob->lambda, prob->mu, prob->rho, nc);
    // media to the device (the caller's buffers are only read here)
    double* dl = dalloc<double>(c, nc);
    double* dm = dalloc<double>(c, nc);
    double* dr = dalloc<double>(c, nc);
    CK(cudaMemcpyAsync(dl, prob->lambda, nc * sizeof(double), cudaMemcpyDefault, c->s));
    CK(cudaMemcpyAsync(dm, prob->mu, nc * sizeof(double), cudaMemcpyDefault, c->s));
    CK(cudaMemcpyAsync(dr, prob->rho, nc * sizeof(double), cudaMemcpyDefault, c->s));
    std::vector<double> om(H.nsets);
    for (int m = 0; m < H.nsets; ++m) om[m] = prob->omegas ? prob->omegas[m] : prob->omega;
    for (double w : om)
      if (!std::isfinite(w) || !(w > 0)) throw ArgError("omega must be positive and finite");
    double* dom = dalloc<double>(c, H.nsets);
    CK(cudaMemcpyAsync(dom, om.data(), H.nsets * sizeof(double), cudaMemcpyHostToDevice, c->s));
    H.cf64 = dalloc<Coef4<double>>(c, nc);
    launch_fine_coef<double>(H.g0, H.nsets, dl, dm, dr, dom, prob->abl_cells, prob->abl_max,
                             prob->gamma_add, H.cf64, c->s);
    cnt(); post();
    CK(cudaStreamSynchronize(c->s));
    dfree(c, dl); dfree(c, dm);
    c->d_rho = dr;
    c->d_om = dom;
    build_hier(c, H, 3, opts->precond == EHS_PRECOND_DD);
    if (opts->precond == EHS_PRECOND_DD) dd_build(c);
    // Krylov workspace
    const int m = opts->restart, items = H.items;
    const long long n = c->n0;
    c->nblk = krylov_nblk(n);
    c->V = dalloc<double2>(c, (size_t)(m + 1) * items * n);
    c->Z = dalloc<double2>(c, (size_t)m * items * n);
    c->w = dalloc<double2>(c, (size_t)items * n);
    c->rd = dalloc<double2>(c, (size_t)items * n);
    c->qd = dalloc<double2>(c, (size_t)items * n);
    c->ud = dalloc<double2>(c, (size_t)items * n);
    c->part = dalloc<double2>(c, (size_t)items * 12 * c->nblk);
    c->hd = dalloc<double2>(c, (size_t)items * 12);
    c->y = dalloc<double2>(c, (size_t)items * 12);
    c->npart = dalloc<double>(c, (size_t)items * c->nblk);
    c->nrm = dalloc<double>(c, items);
    c->kused = dalloc<int>(c, items);
    c->f_in = dalloc<float2>(c, (size_t)items * n);
    c->f_out = dalloc<float2>(c, (size_t)items * n);
    if (opts->prec == EHS_C64) {   // df64 Krylov workspace of the mixed form
      H.cfdf = dalloc<float4>(c, (size_t)2 * H.nsets * H.g0.ncell);
      launch_coef_df((long long)H.nsets * H.g0.ncell, H.cf64, H.cfdf, c->s); cnt(); post();
      if (H.g0.d == 2) {
        H.kdg = dalloc<float4>(c, (size_t)2 * H.nsets * H.g0.ncell);
        H.kvm = dalloc<float2>(c, (size_t)H.nsets * (H.g0.n[0] + 1) * (H.g0.n[1] + 1));
        launch_apply_df_tables(H.g0, H.nsets, H.cf64, H.h, H.kdg, H.kvm, c->s); cnt(); post();
      }
      c->Vq = dalloc<float4>(c, (size_t)(m + 1) * items * n);
      c->Zf = dalloc<float2>(c, (size_t)m * items * n);
      c->wq = dalloc<float4>(c, (size_t)items * n);
      c->rq = dalloc<float4>(c, (size_t)items * n);
      c->qq = dalloc<float4>(c, (size_t)items * n);
      c->xq = dalloc<float4>(c, (size_t)items * n);
      c->partq = dalloc<float4>(c, (size_t)items * 24 * c->nblk);   // 2 x 12 sums per item (delayed CGS2)
      c->dcoef = dalloc<float4>(c, (size_t)items * KDS);
      c->hq = dalloc<float4>(c, (size_t)items * 12);
      c->h2q = dalloc<float4>(c, (size_t)items * 12);
      c->yq = dalloc<float4>(c, (size_t)items * 12);
      c->npq = dalloc<float2>(c, (size_t)items * c->nblk);
      c->invq = dalloc<float2>(c, items);
      static_assert(KDS <= 24, "hhost and hstep hold 24 double2 per item");
      c->hhost = dalloc<double2>(c, (size_t)items * 24);            // h1, h2 or the delayed-CGS2 coefficients
      c->kcnt = dalloc<int>(c, (size_t)items * 3);
    }
    CK(cudaMallocHost((void**)&c->hpin, 64 * sizeof(double) + items * sizeof(double)));
    CK(cudaMallocHost((void**)&c->hstep, (size_t)items * 25 * sizeof(double2)));
    CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_step, cudaEventDisableTiming));
    c->pg.assign(m, nullptr);
    c->pg_nodes.assign(m, 0);
    c->pg_ver.assign(m, -1);
    c->d_act = dalloc<int>(c, items);
    for (int col = 0; col < 8; ++col)
      for (DDGroup& grp : c->dd[col]) grp.d_sub_act = dalloc<int>(c, grp.H.items);
    const char* ng = getenv("EHS_NO_GRAPHS");
    c->use_graphs = !(ng && ng[0] == '1');
    CK(cudaStreamSynchronize(c->s));
    return EHS_OK;
  });
  if (st != EHS_OK) {
    g_create_err = c->err;
    ehs_destroy(c);
    return st;
  }
  *out = c;
  return EHS_OK;
}

ehs_status ehs_destroy(ehs_ctx* c) {
  if (!c) return EHS_OK;
  cudaStreamSynchronize(c->s);
  for (cudaGraphExec_t g : c->pg)
    if (g) cudaGraphExecDestroy(g);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->ev_step) cudaEventDestroy(c->ev_step);
  for (void* p : c->allocs)
    if (p) cudaFree(p);
  if (c->hpin) cudaFreeHost(c->hpin);
  if (c->hstep) cudaFreeHost(c->hstep);
  delete c;
  return EHS_OK;
}

ehs_status ehs_op_apply(ehs_ctx* c, int level, int shifted, int prec, const void* x, void* y) {
  if (!c) return EHS_ERR_ARG;
  return guard(c, [&]() -> ehs_status {
    if (level > 0 && c->H.coef_only) throw ArgError("a DD context builds no global coarse levels");
    if (level < 0 || level >= c->H.nlev) throw ArgError("level out of range");
    if (prec != EHS_C64 && prec != EHS_C128) throw ArgError("bad prec");
    if (!x || !y) throw ArgError("null vector");
    const double alpha = (level == 0 && !shifted) ? 0.0 : c->H.alpha;
    if (prec == EHS_C128) level_apply<double>(c, c->H, level, alpha, (const double2*)x, nullptr, (double2*)y, 0);
    else level_apply<float>(c, c->H, level, alpha, (const float2*)x, nullptr, (float2*)y, 0);
    return EHS_OK;
  });
}

ehs_status ehs_smooth(ehs_ctx* c, int level, int nsweeps, int prec, const void* b, void* x) {
  if (!c) return EHS_ERR_ARG;
  return guard(c, [&]() -> ehs_status {
    if (c->H.coef_only) throw ArgError("a DD context builds no global multigrid hierarchy");
    if (level < 0 || level >= c->H.nlev - 1) throw ArgError("level out of range (the coarsest level is solved, not smoothed)");
    if (prec != EHS_C64 && prec != EHS_C128) throw ArgError("bad prec");
    if (!b || !x || nsweeps < 0) throw ArgError("bad argument");
    if (prec == EHS_C64 && level == 0 && c->H.fused0) {   // whole sweeps, x -> t -> x
      Hier& H = c->H;
      const Level& L = H.lv[0];
      float2* t = (float2*)L.ws[1][2];
      const float wu = (float)L.w, wp = (float)(L.w * H.wp_ratio);
      const float2* cur = (const float2*)x;
      for (int s = 0; s < nsweeps; ++s) {
        float2* out = cur == (const float2*)x ? t : (float2*)x;
        launch_fine_sweep_tile(L.g, H.lv[1].g, H.items, H.nrhs, H.cf32, H.stab, H.h, H.alpha, wu, wp,
                               (const float2*)b, cur, nullptr, out, c->s);
        cnt(); post();
        cur = out;
      }
      if (cur != (const float2*)x)
        CK(cudaMemcpyAsync(x, cur, (size_t)H.items * 3 * L.g.ncell * sizeof(float2), cudaMemcpyDeviceToDevice,
                           c->s));
      return EHS_OK;
    }
    for (int s = 0; s < nsweeps; ++s) {
      if (prec == EHS_C128)
        level_sweep<double>(c, c->H, level, (const double2*)b, (double2*)x, (double2*)c->H.lv[level].ws[0][2]);
      else
        level_sweep<float>(c, c->H, level, (const float2*)b, (float2*)x, (float2*)c->H.lv[level].ws[1][2]);
    }
    return EHS_OK;
  });
}

ehs_status ehs_vcycle(ehs_ctx* c, int prec, const void* b, void* x) {
  if (!c) return EHS_ERR_ARG;
  return guard(c, [&]() -> ehs_status {
    if (c->H.coef_only) throw ArgError("a DD context builds no global multigrid hierarchy");
    if (prec != EHS_C64 && prec != EHS_C128) throw ArgError("bad prec");
    if (!b || !x) throw ArgError("null vector");
    if (prec == EHS_C128) cycle_rec<double>(c, c->H, 0, (const double2*)b, (double2*)x, false);
    else cycle_rec<float>(c, c->H, 0, (const float2*)b, (float2*)x, false);
    return EHS_OK;
  });
}

ehs_status ehs_residual_restrict(ehs_ctx* c, int level, int prec, const void* b, const void* x, void* rc) {
  if (!c) return EHS_ERR_ARG;
  return guard(c, [&]() -> ehs_status {
    if (c->H.coef_only) throw ArgError("a DD context builds no global multigrid hierarchy");
    if (level < 0 || level >= c->H.nlev - 1) throw ArgError("level out of range (0 .. levels-2)");
    if (prec != EHS_C64 && prec != EHS_C128) throw ArgError("bad prec");
    if (!b || !x || !rc) throw ArgError("null vector");
    Hier& H = c->H;
    const Level& L = H.lv[level];
    const Level& Lc = H.lv[level + 1];
    if (prec == EHS_C64 && level == 0 && H.fused0) {
      launch_fine_resid_restrict_tile(L.g, Lc.g, H.items, H.nrhs, H.cf32, H.stab, H.h, H.alpha, (const float2*)x,
                                      (const float2*)b, (float2*)rc, c->s);
      cnt(); post();
    } else if (prec == EHS_C64) {
      float2* r = (float2*)L.ws[1][3];
      level_apply<float>(c, H, level, H.alpha, (const float2*)x, (const float2*)b, r, 1);
      launch_restrict<float>(L.g, Lc.g, H.items, r, (float2*)rc, c->s); cnt(); post();
    } else {
      double2* r = (double2*)L.ws[0][3];
      level_apply<double>(c, H, level, H.alpha, (const double2*)x, (const double2*)b, r, 1);
      launch_restrict<double>(L.g, Lc.g, H.items, r, (double2*)rc, c->s); cnt(); post();
    }
    return EHS_OK;
  });
}

ehs_status ehs_prolong_add(ehs_ctx* c, int level, int prec, const void* ec, void* x) {
  if (!c) return EHS_ERR_ARG;
  return guard(c, [&]() -> ehs_status {
    if (c->H.coef_only) throw ArgError("a DD context builds no global multigrid hierarchy");
    if (level < 0 || level >= c->H.nlev - 1) throw ArgError("level out of range (0 .. levels-2)");
    if (prec != EHS_C64 && prec != EHS_C128) throw ArgError("bad prec");
    if (!ec || !x) throw ArgError("null vector");
    const Hier& H = c->H;
    if (prec == EHS_C64)
      launch_prolong_add<float>(H.lv[level].g, H.lv[level + 1].g, H.items, (const float2*)ec, (float2*)x, c->s);
    else
      launch_prolong_add<double>(H.lv[level].g, H.lv[level + 1].g, H.items, (const double2*)ec, (double2*)x, c->s);
    cnt(); post();
    return EHS_OK;
  });
}

ehs_status ehs_coarse_solve(ehs_ctx* c, int prec, const void* b, void* x) {
  if (!c) return EHS_ERR_ARG;
  return guard(c, [&]() -> ehs_status {
    if (c->H.coef_only) throw ArgError("a DD context builds no global multigrid hierarchy");
    if (prec != EHS_C64 && prec != EHS_C128) throw ArgError("bad prec");
    if (!b || !x) throw ArgError("null vector");
    const int l = c->H.nlev - 1;
    if (prec == EHS_C128) cycle_rec<double>(c, c->H, l, (const double2*)b, (double2*)x, false);
    else cycle_rec<float>(c, c->H, l, (const float2*)b, (float2*)x, false);
    return EHS_OK;
  });
}

ehs_status ehs_coarse_dims(const ehs_ctx* c, int* nsub, int* nloc, int* sizes) {
  if (!c || !nsub || !nloc) return EHS_ERR_ARG;
  if (c->H.coef_only) return EHS_ERR_ARG;
  const Hier& H = c->H;
  const Level& L = H.lv.back();
  if (H.cdd.nsub) {
    *nsub = H.cdd.nsub;
    *nloc = H.cdd.nloc;
    if (sizes)
      for (int q = 0; q < H.cdd.nsub; ++q) sizes[q] = H.cdd.sizes[q];
  } else {
    *nsub = 1;
    *nloc = (int)((L.g.d + 1) * L.g.ncell);
    if (sizes) sizes[0] = *nloc;
  }
  return EHS_OK;
}

ehs_status ehs_coarse_local_apply(ehs_ctx* c, int prec, int colour, const void* r, void* z) {
  if (!c) return EHS_ERR_ARG;
  return guard(c, [&]() -> ehs_status {
    if (c->H.coef_only) throw ArgError("a DD context builds no global multigrid hierarchy");
    if (prec != EHS_C64 && prec != EHS_C128) throw ArgError("bad prec");
    if (!r || !z) throw ArgError("null vector");
    Hier& H = c->H;
    const Level& L = H.lv.back();
    CoarseDD& D = H.cdd;
    if (!D.nsub) {
      if (colour != 0) throw ArgError("the exact coarsest solve has colour 0 only");
      const int N = (int)((L.g.d + 1) * L.g.ncell);
      if (prec == EHS_C128) coarse_gemv<double>(c, H, L, N, H.items, (const double2*)r, (double2*)z);
      else coarse_gemv<float>(c, H, L, N, H.items, (const float2*)r, (float2*)z);
      return EHS_OK;
    }
    if (colour < 0 || colour >= (int)D.col_subs.size() || D.col_subs[colour].empty())
      throw ArgError("no coarsest subdomain has this colour");
    const int ncs = (int)D.col_subs[colour].size();
    SelScope sel(D.d_list_all[colour], H.items * ncs);   // one launch: the local products alone
    if (prec == EHS_C128)
      coarse_gemv<double>(c, H, L, D.nloc, H.items * D.nsub, (const double2*)r, (double2*)z);
    else
      coarse_gemv<float>(c, H, L, D.nloc, H.items * D.nsub, (const float2*)r, (float2*)z);
    return EHS_OK;
  });
}

ehs_status ehs_coarse_local_add(ehs_ctx* c, int prec, int colour, const void* r, void* x) {
  if (!c) return EHS_ERR_ARG;
  return guard(c, [&]() -> ehs_status {
    if (c->H.coef_only) throw ArgError("a DD context builds no global multigrid hierarchy");
    if (prec != EHS_C64 && prec != EHS_C128) throw ArgError("bad prec");
    if (!r || !x) throw ArgError("null vector");
    Hier& H = c->H;
    const Level& L = H.lv.back();
    CoarseDD& D = H.cdd;
    if (!D.nsub) throw ArgError("the coarsest grid is not split (opts.coarse_dd)");
    if (colour < 0 || colour >= (int)D.col_subs.size() || D.col_subs[colour].empty())
      throw ArgError("no coarsest subdomain has this colour");
    if (!D.loc[prec == EHS_C128 ? 0 : 1][1]) throw ArgError("the context was not set up for this precision");
    const long long NG = (long long)(L.g.d + 1) * L.g.ncell;
    const int ncs = (int)D.col_subs[colour].size();
    const int items_l = H.items * D.nsub;
    SelScope sel(D.d_list_all[colour], H.items * ncs);
    if (prec == EHS_C64 && L.invlp &&
        launch_dense_apply_scatter(D.nloc, items_l, H.nrhs, D.nsub, D.d_sizes, L.invlp, H.coarse_fmt,
                                   (const float2*)r, D.d_map, NG, (float2*)x, c->s)) {
      cnt(); post();
      return EHS_OK;
    }
    if (prec == EHS_C128) {
      double2* zs = (double2*)D.loc[0][1];
      coarse_gemv<double>(c, H, L, D.nloc, items_l, (const double2*)r, zs);
      launch_dd_scatter<double>(D.nloc, items_l, D.nsub, H.nrhs, NG, D.d_map, zs, (double2*)x, c->s);
    } else {
      float2* zs = (float2*)D.loc[1][1];
      coarse_gemv<float>(c, H, L, D.nloc, items_l, (const float2*)r, zs);
      launch_dd_scatter<float>(D.nloc, items_l, D.nsub, H.nrhs, NG, D.d_map, zs, (float2*)x, c->s);
    }
    cnt(); post();
    return EHS_OK;
  });
}

ehs_status ehs_dd_precond(ehs_ctx* c, int prec, const void* r, void* z) {
  if (!c) return EHS_ERR_ARG;
  return guard(c, [&]() -> ehs_status {
    if (c->opt.precond != EHS_PRECOND_DD) throw ArgError("context was not created with the DD preconditioner");
    if (prec != c->opt.prec) throw ArgError("a DD context runs its subdomain cycles in opts.prec only");
    if (!r || !z) throw ArgError("null vector");
    dd_apply(c, prec, (const double2*)r, (double2*)z);
    return EHS_OK;
  });
}

ehs_status ehs_fgmres_solve(ehs_ctx* c, const void* q, void* u, ehs_solve_info* info) {
  if (!c) return EHS_ERR_ARG;
  return guard(c, [&]() -> ehs_status {
    if (!q || !u) throw ArgError("null vector");
    return solve_common(c, q, u, info, false);
  });
}

ehs_status ehs_adjoint_solve(ehs_ctx* c, const void* g, void* w, ehs_solve_info* info) {
  if (!c) return EHS_ERR_ARG;
  return guard(c, [&]() -> ehs_status {
    if (!g || !w) throw ArgError("null vector");
    return solve_common(c, g, w, info, true);
  });
}

ehs_status ehs_gradient(ehs_ctx* c, const void* x, const void* w, double* g_lambda, double* g_mu,
                        double* g_rho) {
  if (!c) return EHS_ERR_ARG;
  return guard(c, [&]() -> ehs_status {
    if (!x || !w || !g_lambda || !g_mu || !g_rho) throw ArgError("null argument");
    if (!is_device_ptr(x) || !is_device_ptr(w) || !is_device_ptr(g_lambda) || !is_device_ptr(g_mu) ||
        !is_device_ptr(g_rho))
      throw ArgError("ehs_gradient takes device pointers");
    launch_gradient(c->H.g0, c->H.nsets, c->H.nrhs, c->H.cf64, c->d_rho, c->d_om, c->H.h,
                    (const double2*)x, (const double2*)w, g_lambda, g_mu, g_rho, c->s);
    cnt(); post();
    return EHS_OK;
  });
}

int ehs_items(const ehs_ctx* c) { return c ? c->H.items : 0; }
long long ehs_level_len(const ehs_ctx* c, int level) {
  if (!c || level < 0 || level >= (int)c->H.lv.size()) return -1;
  return (long long)(c->d + 1) * c->H.lv[level].g.ncell;
}
int ehs_level_dims(const ehs_ctx* c, int level, int n[3]) {
  if (!c || !n || level < 0 || level >= (int)c->H.lv.size()) return -1;
  for (int k = 0; k < 3; ++k) n[k] = c->H.lv[level].g.n[k];
  return 0;
}
ehs_status ehs_sync(ehs_ctx* c) {
  if (!c) return EHS_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(c->s);
  if (e != cudaSuccess) { c->err = cudaGetErrorString(e); return EHS_ERR_CUDA; }
  return guard(c, [&]() -> ehs_status {
    if (device_timeout(c)) {
      c->err = "a persistent launch's grid barrier waited past its limit (the SMs were held by other work)";
      return EHS_ERR_TIMEOUT;
    }
    return EHS_OK;
  });
}
long long ehs_kernel_launches(void) { return g_launches.load(); }
const char* ehs_last_error(const ehs_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

}  // extern "C"
