// Shared device/host definitions of the GB300 elastic Helmholtz library.
//
// Layout of every vector (the "slot layout" of include/ehs.h): per batch
// item, d+1 component arrays of ncell complex values each, [u_1, .., u_d, p];
// x is the fastest index.  u_k[c] is the value on the low face of cell c in
// direction k; the slot with i_k == 0 is a Dirichlet boundary face and is
// always zero.  Complex numbers are interleaved (re, im).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define EHS_HD __host__ __device__ __forceinline__

namespace ehs {

template <typename T> struct CT;
template <> struct CT<float> { typedef float2 type; };
template <> struct CT<double> { typedef double2 type; };

template <typename T> EHS_HD typename CT<T>::type mk(T re, T im) {
  typename CT<T>::type z; z.x = re; z.y = im; return z;
}
EHS_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
EHS_HD double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
EHS_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
EHS_HD double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
EHS_HD float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
EHS_HD double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
EHS_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
EHS_HD double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// a + b * c
EHS_HD float2 cfma(float2 b, float2 c, float2 a) {
  return make_float2(fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x)), fmaf(b.x, c.y, fmaf(b.y, c.x, a.y)));
}
EHS_HD double2 cfma(double2 b, double2 c, double2 a) {
  return make_double2(fma(b.x, c.x, fma(-b.y, c.y, a.x)), fma(b.x, c.y, fma(b.y, c.x, a.y)));
}
template <typename C> EHS_HD C czero() { C z; z.x = 0; z.y = 0; return z; }
// 1 / z
EHS_HD float2 cinv(float2 z) { float s = 1.0f / (z.x * z.x + z.y * z.y); return make_float2(z.x * s, -z.y * s); }
EHS_HD double2 cinv(double2 z) { double s = 1.0 / (z.x * z.x + z.y * z.y); return make_double2(z.x * s, -z.y * s); }
EHS_HD float2 to_c(float2 z, float) { return z; }
EHS_HD float2 to_c(double2 z, float) { return make_float2((float)z.x, (float)z.y); }
EHS_HD double2 to_c(float2 z, double) { return make_double2(z.x, z.y); }
EHS_HD double2 to_c(double2 z, double) { return z; }

// Grid of one multigrid level; n[0] = n_x, n[1] = n_y, n[2] = n_z (1 in 2D).
struct Grid {
  int d;
  int n[3];
  long long ncell;
};

EHS_HD void cell_coords(const Grid& g, long long c, int i[3]) {
  const unsigned cc = (unsigned)c;                 // ncell < 2^31 on every level
  const unsigned t = cc / (unsigned)g.n[0];
  i[0] = (int)(cc - t * (unsigned)g.n[0]);
  const unsigned z = t / (unsigned)g.n[1];
  i[1] = (int)(t - z * (unsigned)g.n[1]);
  i[2] = (int)z;
}
EHS_HD long long cell_index(const Grid& g, const int i[3]) {
  return ((long long)i[2] * g.n[1] + i[1]) * g.n[0] + i[0];
}
EHS_HD long long stride_of(const Grid& g, int k) {
  return k == 0 ? 1 : (k == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1]);
}

// Fine-level cell coefficients of the matrix-free operator: mu, 1/(lambda+mu),
// mr = omega^2 rho and mi = omega rho gamma, so that the face mass term
// -omega^2 A_f(rho (1 - i gamma/omega)) is -A_f(mr) + i A_f(mi) and each
// coefficient set (medium) carries its own frequency.
template <typename T> struct Coef4 { T mu, kap, mr, mi; };

// ------------------------------------------------------------ stencil table
// Stored operators of Galerkin levels: for each (row comp a, col comp b)
// pair a box of offsets [lo, lo+ext) per direction.  Coefficients are stored
// per coefficient set as [slot][cell] (cell fastest), slot = base + linear
// offset index (x fastest).
#define EHS_MAXPAIR 16
struct PairBox {
  int a, b;
  int lo[3];
  int ext[3];
  int base;  // first slot of this pair
};
struct StencilLayout {
  int npair;
  int nslot;            // coefficients per cell
  int row_first[5];     // pairs are sorted by row; pairs of row a: [row_first[a], row_first[a+1])
  int pidx[4][4];       // pair index of (a, b), -1 if the pair is structurally zero
  PairBox p[EHS_MAXPAIR];
};

// slot of coefficient (a, b, offset o) or -1 if outside the stored box
__host__ __device__ constexpr int st_slot(const StencilLayout& L, int a, int b, int ox, int oy, int oz) {
  int q = L.pidx[a][b];
  if (q < 0) return -1;
  const PairBox& P = L.p[q];
  int ix = ox - P.lo[0], iy = oy - P.lo[1], iz = oz - P.lo[2];
  if (ix < 0 || iy < 0 || iz < 0 || ix >= P.ext[0] || iy >= P.ext[1] || iz >= P.ext[2]) return -1;
  return P.base + (iz * P.ext[1] + iy) * P.ext[0] + ix;
}

// Transfer weights (1D).  Kinds: 0 = vertex-like (u_k along k; interior faces
// 1..n-1 are unknowns), 1 = cell-like with zero ghosts (u tangential),
// 2 = cell-like with clamped ghosts (p).  pw(kind, j, J, nc) is the weight of
// coarse index J in fine index j (fine grid has 2 nc cells).
__host__ __device__ constexpr double pw(int kind, int j, int J, int nc) {
  const int nf = 2 * nc;
  if (kind == 0) {
    if (j < 1 || j > nf - 1 || J < 1 || J > nc - 1) return 0.0;
    if ((j & 1) == 0) return (j == 2 * J) ? 1.0 : 0.0;
    return (J == (j - 1) / 2 || J == (j + 1) / 2) ? 0.5 : 0.0;
  }
  if (j < 0 || j > nf - 1 || J < 0 || J > nc - 1) return 0.0;
  const int Jc = j >> 1;
  const int nb = (j & 1) ? Jc + 1 : Jc - 1;
  double w = 0.0;
  if (J == Jc) w += 0.75;
  if (nb >= 0 && nb < nc) {
    if (J == nb) w += 0.25;
  } else if (kind == 2 && J == Jc) {
    w += 0.25;
  }
  return w;
}
// pw() in quarters as an integer (all transfer weights are multiples of 1/4):
// the transfer kernels use this so they never touch the FP64 pipe
__host__ __device__ constexpr int pw4(int kind, int j, int J, int nc) {
  const int nf = 2 * nc;
  if (kind == 0) {
    if (j < 1 || j > nf - 1 || J < 1 || J > nc - 1) return 0;
    if ((j & 1) == 0) return (j == 2 * J) ? 4 : 0;
    return (J == (j - 1) / 2 || J == (j + 1) / 2) ? 2 : 0;
  }
  if (j < 0 || j > nf - 1 || J < 0 || J > nc - 1) return 0;
  const int Jc = j >> 1;
  const int nb = (j & 1) ? Jc + 1 : Jc - 1;
  int w = 0;
  if (J == Jc) w += 3;
  if (nb >= 0 && nb < nc) {
    if (J == nb) w += 1;
  } else if (kind == 2 && J == Jc) {
    w += 1;
  }
  return w;
}

// kind of component a along direction k
__host__ __device__ constexpr int tkind(int a, int k, int d) { return a == d ? 2 : (a == k ? 0 : 1); }

// The same 1D rules seen from a fine index j: at most two coarse indices J0,
// J1 carry a weight (w0, w1; a zero weight is unused and its index is a valid
// in-range placeholder).  Fine indices are those of unknowns (1..nf-1 for
// kind 0, 0..nf-1 otherwise); pw(kind, j, J, nc) == w0 at J0 plus w1 at J1.
template <typename T>
__host__ __device__ constexpr void pw_pair(int kind, int j, int nc, int& J0, T& w0, int& J1, T& w1) {
  if (kind == 0) {
    if ((j & 1) == 0) {
      J0 = j >> 1; w0 = (J0 >= 1 && J0 <= nc - 1) ? T(1) : T(0);
      J1 = J0; w1 = T(0);
    } else {
      J0 = (j - 1) >> 1; w0 = (J0 >= 1 && J0 <= nc - 1) ? T(0.5) : T(0);
      J1 = (j + 1) >> 1; w1 = (J1 >= 1 && J1 <= nc - 1) ? T(0.5) : T(0);
      if (w1 == T(0)) J1 = J0;
      if (w0 == T(0)) J0 = J1;
    }
    return;
  }
  J0 = j >> 1; w0 = T(0.75);
  J1 = (j & 1) ? J0 + 1 : J0 - 1; w1 = T(0.25);
  if (J1 < 0 || J1 >= nc) {
    w1 = T(0); J1 = J0;
    if (kind == 2) w0 = T(1);
  }
}
// pw_pair() against pw() for every kind and unknown index of a coarse grid of nc cells
__host__ __device__ constexpr bool pw_pair_agrees(int nc) {
  for (int kind = 0; kind < 3; ++kind)
    for (int j = (kind == 0 ? 1 : 0); j <= 2 * nc - 1; ++j) {
      int J0 = 0, J1 = 0;
      double w0 = 0, w1 = 0;
      pw_pair<double>(kind, j, nc, J0, w0, J1, w1);
      if (J0 < 0 || J0 >= nc || J1 < 0 || J1 >= nc) return false;
      for (int J = 0; J < nc; ++J) {
        const double w = (J == J0 ? w0 : 0.0) + (J == J1 ? w1 : 0.0);   // a placeholder adds 0
        if (w != pw(kind, j, J, nc)) return false;
      }
    }
  return true;
}
static_assert(pw_pair_agrees(2) && pw_pair_agrees(3) && pw_pair_agrees(4) && pw_pair_agrees(9),
              "fine-index transfer rule = pw()");

// Level-0 stencil layout of the mixed operator: (u_k, u_k) a 3^d box, (u_k, p)
// offsets -1..0 along k, (p, u_k) offsets 0..1 along k, (p, p) the centre.
__host__ __device__ constexpr StencilLayout make_fine_layout(int d) {
  StencilLayout L{};
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) L.pidx[a][b] = -1;
  int q = 0, base = 0;
  for (int a = 0; a <= d; ++a) {
    L.row_first[a] = q;
    const int nb = a < d ? 2 : d + 1;
    for (int t = 0; t < nb; ++t) {
      const int b = a < d ? (t == 0 ? a : d) : t;
      PairBox& P = L.p[q];
      P.a = a; P.b = b;
      for (int k = 0; k < 3; ++k) { P.lo[k] = 0; P.ext[k] = 1; }
      for (int k = 0; k < d; ++k) {
        if (a < d && b == a) { P.lo[k] = -1; P.ext[k] = 3; }
        else if (a < d && k == a) { P.lo[k] = -1; P.ext[k] = 2; }
        else if (a == d && b < d && k == b) { P.lo[k] = 0; P.ext[k] = 2; }
      }
      P.base = base;
      base += P.ext[0] * P.ext[1] * P.ext[2];
      L.pidx[a][b] = q++;
    }
  }
  L.row_first[d + 1] = q;
  L.npair = q;
  L.nslot = base;
  return L;
}

// Galerkin coarse layout: the box of each pair on the next coarser level,
// from the fine box and the 1D transfer supports (interior rows).
__host__ __device__ constexpr StencilLayout make_coarse_layout(int d, const StencilLayout& F) {
  StencilLayout C{};
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) C.pidx[a][b] = -1;
  const int nc = 64, I = 32;
  int base = 0;
  for (int q = 0; q < F.npair; ++q) {
    const PairBox& P = F.p[q];
    PairBox& Q = C.p[q];
    Q.a = P.a; Q.b = P.b;
    for (int k = 0; k < 3; ++k) {
      if (k >= d) { Q.lo[k] = 0; Q.ext[k] = 1; continue; }
      const int ka = tkind(P.a, k, d), kb = tkind(P.b, k, d);
      int mn = 1 << 30, mx = -(1 << 30);
      for (int i = 2 * I - 4; i <= 2 * I + 5; ++i) {
        if (pw(ka, i, I, nc) == 0.0) continue;
        for (int o = P.lo[k]; o < P.lo[k] + P.ext[k]; ++o) {
          const int j = i + o;
          for (int J = j / 2 - 3; J <= j / 2 + 3; ++J) {
            if (pw(kb, j, J, nc) == 0.0) continue;
            mn = J - I < mn ? J - I : mn;
            mx = J - I > mx ? J - I : mx;
          }
        }
      }
      Q.lo[k] = mn;
      Q.ext[k] = mx - mn + 1;
    }
    Q.base = base;
    base += Q.ext[0] * Q.ext[1] * Q.ext[2];
    C.pidx[Q.a][Q.b] = q;
  }
  C.npair = F.npair;
  C.nslot = base;
  for (int a = 0; a < 5; ++a) C.row_first[a] = F.row_first[a];
  return C;
}

// layout of Galerkin level lv >= 1 (the boxes are the same from level 2 on)
__host__ __device__ constexpr StencilLayout level_layout(int d, int lv) {
  StencilLayout L = make_fine_layout(d);
  for (int l = 0; l < lv; ++l) L = make_coarse_layout(d, L);
  return L;
}
__host__ __device__ constexpr bool same_layout(const StencilLayout& A, const StencilLayout& B) {
  if (A.npair != B.npair || A.nslot != B.nslot) return false;
  for (int q = 0; q < A.npair; ++q) {
    if (A.p[q].a != B.p[q].a || A.p[q].b != B.p[q].b || A.p[q].base != B.p[q].base) return false;
    for (int k = 0; k < 3; ++k)
      if (A.p[q].lo[k] != B.p[q].lo[k] || A.p[q].ext[k] != B.p[q].ext[k]) return false;
  }
  return true;
}
static_assert(same_layout(level_layout(2, 2), level_layout(2, 3)), "2D Galerkin boxes settle at level 2");
static_assert(same_layout(level_layout(3, 2), level_layout(3, 3)), "3D Galerkin boxes settle at level 2");
static_assert(level_layout(2, 1).nslot == 87 && level_layout(2, 2).nslot == 135, "2D table sizes");

// Half ("symmetric") storage of a Galerkin table.  K_c = P^T K_s P is complex
// symmetric (P real, K_s = K_s^T), so the coefficient (row a, column b, offset
// o) at cell c equals (row b, column a, offset -o) at cell c + o.  Stored: pairs
// a < b whole, pairs a == b for offsets o >= 0 in lexicographic (z, y, x)
// order, pairs a > b not at all; a row reads an unstored coefficient from its
// mirror's compact slot at the neighbour cell c + o.
#define EHS_MAXSLOT 960
struct HalfMap {
  int nslot;                  // stored coefficients per cell
  int slot[EHS_MAXSLOT];      // per full slot: the compact slot holding it (its own or its mirror's)
  bool mir[EHS_MAXSLOT];      // the full slot is read from its mirror at cell c + o
  int full[EHS_MAXSLOT];      // per compact slot: the full slot stored there
  bool ok;                    // every unstored coefficient has a stored mirror
};
__host__ __device__ constexpr bool half_stored(int a, int b, int ox, int oy, int oz) {
  return a < b || (a == b && (oz > 0 || (oz == 0 && (oy > 0 || (oy == 0 && ox >= 0)))));
}
__host__ __device__ constexpr HalfMap make_half_map(const StencilLayout& L) {
  HalfMap H{};
  H.ok = L.nslot <= EHS_MAXSLOT;
  int n = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int q = 0; q < L.npair; ++q) {
      const PairBox& P = L.p[q];
      for (int iz = 0; iz < P.ext[2]; ++iz)
        for (int iy = 0; iy < P.ext[1]; ++iy)
          for (int ix = 0; ix < P.ext[0]; ++ix) {
            const int ox = P.lo[0] + ix, oy = P.lo[1] + iy, oz = P.lo[2] + iz;
            const int sl = P.base + (iz * P.ext[1] + iy) * P.ext[0] + ix;
            if (sl >= EHS_MAXSLOT) { H.ok = false; continue; }
            const bool st = half_stored(P.a, P.b, ox, oy, oz);
            if (pass == 0 && st) {             // stored entries, numbered in full-slot order
              H.slot[sl] = n; H.mir[sl] = false; H.full[n] = sl; ++n;
            } else if (pass == 1 && !st) {     // the others read their mirror
              const int ms = st_slot(L, P.b, P.a, -ox, -oy, -oz);
              if (ms < 0 || !half_stored(P.b, P.a, -ox, -oy, -oz)) { H.ok = false; continue; }
              H.slot[sl] = H.slot[ms]; H.mir[sl] = true;
            }
          }
    }
  H.nslot = n;
  return H;
}
// The same numbering in closed form, for kernels that walk a row's boxes with the
// pair index q known at compile time and the box position ti (x fastest, as the
// full slots) unrolled: pairs a < b store their box whole from half_base(q);
// a diagonal pair's box is symmetric about 0, so its offsets o >= 0 are the
// positions ti >= (n-1)/2 of its n entries, and the mirror of ti is n-1-ti;
// the box of a pair a > b is the point reflection of pair (b, a)'s box.
__host__ __device__ constexpr int half_base(const StencilLayout& L, int q) {
  int n = 0;
  for (int k = 0; k < q; ++k) {
    const PairBox& P = L.p[k];
    const int ne = P.ext[0] * P.ext[1] * P.ext[2];
    n += P.a < P.b ? ne : (P.a == P.b ? (ne + 1) / 2 : 0);
  }
  return n;
}
__host__ __device__ constexpr int half_index(const StencilLayout& L, int q, int ti, bool& mir) {
  const PairBox& P = L.p[q];
  const int ne = P.ext[0] * P.ext[1] * P.ext[2];
  if (P.a < P.b) { mir = false; return half_base(L, q) + ti; }
  if (P.a == P.b) {
    const int tc = (ne - 1) / 2;
    mir = ti < tc;
    return half_base(L, q) + (mir ? tc - ti : ti - tc);
  }
  mir = true;
  return half_base(L, L.pidx[P.b][P.a]) + (ne - 1 - ti);
}
__host__ __device__ constexpr int half_slot_c(const StencilLayout& L, int q, int ti) {
  bool m = false;
  return half_index(L, q, ti, m);
}
__host__ __device__ constexpr bool half_mir_c(const StencilLayout& L, int q, int ti) {
  bool m = false;
  half_index(L, q, ti, m);
  return m;
}
// the closed form agrees with make_half_map on every slot
__host__ __device__ constexpr bool half_index_agrees(const StencilLayout& L) {
  const HalfMap H = make_half_map(L);
  if (!H.ok) return false;
  for (int q = 0; q < L.npair; ++q) {
    const PairBox& P = L.p[q];
    const int ne = P.ext[0] * P.ext[1] * P.ext[2];
    if (P.a == P.b && (ne % 2 == 0 || P.lo[0] != -(P.ext[0] - 1) / 2 || P.lo[1] != -(P.ext[1] - 1) / 2 ||
                       P.lo[2] != -(P.ext[2] - 1) / 2))
      return false;
    for (int ti = 0; ti < ne; ++ti) {
      bool mir = false;
      const int hs = half_index(L, q, ti, mir);
      if (hs != H.slot[P.base + ti] || mir != H.mir[P.base + ti]) return false;
    }
  }
  return true;
}
static_assert(half_index_agrees(level_layout(2, 1)) && half_index_agrees(level_layout(2, 2)) &&
              half_index_agrees(level_layout(3, 1)) && half_index_agrees(level_layout(3, 2)),
              "closed-form half-table index");
static_assert(make_half_map(level_layout(2, 1)).ok && make_half_map(level_layout(2, 1)).nslot == 45,
              "2D level-1 half table");
static_assert(make_half_map(level_layout(2, 2)).ok && make_half_map(level_layout(2, 2)).nslot == 69,
              "2D half table from level 2 on");
static_assert(make_half_map(level_layout(3, 1)).ok && make_half_map(level_layout(3, 2)).ok, "3D half tables");

// a valid unknown slot?  (u_k at i_k == 0 is a boundary face)
EHS_HD bool slot_valid(int a, int d, const int i[3]) { return a == d || i[a] >= 1; }

enum { EHS_DEVERR_BOX = 1, EHS_DEVERR_SINGULAR = 2, EHS_DEVERR_NONFINITE = 4 };

}  // namespace ehs
