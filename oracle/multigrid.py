"""Shifted-Laplacian multigrid for the mixed system (oracle).

* Transfer (Sec. 3, "standard bilinear transfer operators ... for face-based
  staggered discretization"): per component, a tensor product of 1D
  interpolations.  Along its own direction u_k is interpolated like a vertex
  quantity (fine face 2I = coarse face I, fine face 2I+1 = mean of coarse
  faces I and I+1); along the other directions u_k and, along every
  direction, p are interpolated like cell quantities (weights 3/4 and 1/4).
  u uses zero ghosts, p clamped ghosts.  Restriction is P^T (Sec. 2.2).
* Coarse operators: Galerkin products P^T K_s P (eq. coarseGridMatrix).
* Relaxation: damped cell-wise (Vanka) relaxation, full or economic block
  (Sec. 3; economic block = eq. RelaxationMatrix), red-black or
  lexicographic cell order.
* Cycle: Algorithm TwoCycle applied recursively (once: V, twice: W); the
  coarsest level is solved exactly with a sparse LU, or (MG-DD, Sec. 4) by
  one multiplicative sweep of Algorithm DD over subdomains of the coarsest
  grid with exact local solves (`CoarseDD`).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .operators import comp_shape, kron_axes


# ------------------------------------------------------------------ transfer
def interp_vertex(nc):
    """(2nc-1) x (nc-1): interior faces of the fine grid from interior coarse faces."""
    rows, cols, vals = [], [], []
    for I in range(1, nc):          # coarse interior face I -> column I-1
        for f, w in ((2 * I - 1, 0.5), (2 * I, 1.0), (2 * I + 1, 0.5)):
            rows.append(f - 1); cols.append(I - 1); vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * nc - 1, nc - 1))


def interp_cell(nc, clamp):
    """2nc x nc cell-centred linear interpolation (3/4, 1/4); zero or clamped ghosts."""
    rows, cols, vals = [], [], []
    for i in range(2 * nc):
        J = i // 2
        nb = J - 1 if i % 2 == 0 else J + 1
        rows.append(i); cols.append(J); vals.append(0.75)
        if 0 <= nb < nc:
            rows.append(i); cols.append(nb); vals.append(0.25)
        elif clamp:
            rows.append(i); cols.append(J); vals.append(0.25)
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * nc, nc)).tocsr()


def prolongation(coarse_shape):
    """Block-diagonal P from the coarse grid to the grid twice as fine."""
    d = len(coarse_shape)
    blocks = []
    for k in range(d):
        mats = []
        for a in range(d):
            nc = coarse_shape[a]
            if a == d - 1 - k:
                mats.append(interp_vertex(nc))
            else:
                mats.append(interp_cell(nc, clamp=False))
        blocks.append(kron_axes(mats))
    blocks.append(kron_axes([interp_cell(nc, clamp=True) for nc in coarse_shape]))
    return sp.block_diag(blocks, format="csr")


# ------------------------------------------------------------- cell blocks
def cell_dofs(shape):
    """(N_c, 2d+1) DOF indices of each cell's block: low faces, high faces, p.

    -1 marks a face that lies on the boundary (not an unknown)."""
    d = len(shape)
    idx = np.indices(shape).reshape(d, -1)          # idx[a] = index along numpy axis a
    ncell = idx.shape[1]
    out = -np.ones((ncell, 2 * d + 1), dtype=np.int64)
    off = 0
    for k in range(d):
        cs = comp_shape(shape, k)
        ak = d - 1 - k
        for side in (0, 1):
            f = idx[ak] + side                      # face index along k (low face = cell index)
            ok = (f >= 1) & (f <= shape[ak] - 1)
            coords = [idx[a].copy() for a in range(d)]
            coords[ak] = f - 1
            lin = np.zeros(ncell, dtype=np.int64)
            for a in range(d):
                lin = lin * cs[a] + np.where(ok, coords[a], 0)
            out[:, side * d + k] = np.where(ok, off + lin, -1)
        off += int(np.prod(cs))
    out[:, 2 * d] = off + np.arange(ncell)
    return out


def cell_colour(shape):
    idx = np.indices(shape).reshape(len(shape), -1)
    return idx.sum(axis=0) % 2


def extract_blocks(K, dofs, economic):
    """Dense local blocks K[I_c, I_c]; missing DOFs become identity rows/cols.

    economic=True keeps only the diagonal of the displacement block plus the
    displacement-pressure couplings and the pressure diagonal (eq.
    RelaxationMatrix)."""
    K = K.tocsr()
    ncell, nb = dofs.shape
    d = (nb - 1) // 2
    B = np.zeros((ncell, nb, nb), dtype=np.complex128)
    for a in range(nb):
        for b in range(nb):
            if economic and a != b and a < 2 * d and b < 2 * d:
                continue
            ok = (dofs[:, a] >= 0) & (dofs[:, b] >= 0)
            if not ok.any():
                continue
            vals = np.asarray(K[dofs[ok, a], dofs[ok, b]]).ravel()
            B[ok, a, b] = vals
    for a in range(nb):
        miss = dofs[:, a] < 0
        B[miss, a, :] = 0.0
        B[miss, :, a] = 0.0
        B[miss, a, a] = 1.0
    return B


# --------------------------------------------------------------- relaxation
class Level:
    def __init__(self, K, shape, w, economic, wu=None, wp=None):
        self.K = K.tocsr()
        self.shape = shape
        self.dofs = cell_dofs(shape)
        self.colour = cell_colour(shape)
        self.Binv = np.linalg.inv(extract_blocks(self.K, self.dofs, economic))
        d = len(shape)
        nb = 2 * d + 1
        wu = w if wu is None else wu
        wp = w if wp is None else wp
        self.wvec = np.array([wu] * (2 * d) + [wp])
        self.valid = self.dofs >= 0
        self.safe = np.where(self.valid, self.dofs, 0)
        assert self.Binv.shape[1] == nb

    def _update_cells(self, x, r, cells):
        """x[I_c] += W B_c^{-1} r[I_c] for every listed cell (one shared residual)."""
        rl = np.where(self.valid[cells], r[self.safe[cells]], 0.0)
        dl = np.einsum("cab,cb->ca", self.Binv[cells], rl) * self.wvec
        dl = np.where(self.valid[cells], dl, 0.0)
        np.add.at(x, self.safe[cells].ravel(), dl.ravel())
        return x

    def relax_rb(self, b, x):
        """One red-black sweep: residual recomputed before each colour, then
        all cells of that colour updated simultaneously."""
        x = x.copy()
        for col in (0, 1):
            r = b - self.K @ x
            x = self._update_cells(x, r, np.nonzero(self.colour == col)[0])
        return x

    def relax_lex(self, b, x):
        """One lexicographic (x fastest) multiplicative sweep."""
        x = x.copy()
        K = self.K
        for c in range(self.dofs.shape[0]):
            I = self.dofs[c][self.valid[c]]
            r = b[I] - K[I, :] @ x
            Bi = self.Binv[c][np.ix_(self.valid[c], self.valid[c])]
            # the inverse of the reduced block equals the reduced inverse because
            # missing DOFs were identity rows/cols decoupled from the rest
            x[I] += self.wvec[self.valid[c]] * (Bi @ r)
        return x


# ------------------------------------------------------ coarse-grid DD
def near_equal_edges(n, s):
    """Edges of s nearly equal consecutive parts of n cells (larger parts first)."""
    base, rem = divmod(n, s)
    edges = [0]
    for i in range(s):
        edges.append(edges[-1] + base + (1 if i < rem else 0))
    return edges


def box_dofs(shape, lo, hi):
    """Oracle DOF numbers of the unknowns inside the cell box [lo, hi) (numpy
    axis order): the pressures of its cells and the faces whose two cells both
    lie in the box.  Faces on the box surface are not unknowns of the local
    problem (homogeneous Dirichlet), as on the outer boundary."""
    d = len(shape)
    out = []
    off = 0
    for k in range(d):
        cs = comp_shape(shape, k)
        ak = d - 1 - k
        # u_k array index j along axis ak is the face between cells j and j+1
        rng = [np.arange(lo[a], hi[a]) if a != ak else np.arange(lo[a], hi[a] - 1) for a in range(d)]
        grid = np.meshgrid(*rng, indexing="ij")
        lin = np.ravel_multi_index(tuple(g.ravel() for g in grid), cs)
        out.append(off + lin)
        off += int(np.prod(cs))
    grid = np.meshgrid(*[np.arange(lo[a], hi[a]) for a in range(d)], indexing="ij")
    out.append(off + np.ravel_multi_index(tuple(g.ravel() for g in grid), shape))
    return np.sort(np.concatenate(out))


class CoarseDD:
    """Algorithm DD as the coarsest-grid solver of MG-DD (Sec. 4), applied to
    the assembled coarsest Galerkin operator.

    Readings: cores split each direction into nsub near-equal parts
    (nsub in direction order x, y, z); Omega_i = core grown by `overlap` cells
    on every side, clipped to the grid; the local matrix is the coarsest
    operator restricted to the unknowns inside Omega_i (`box_dofs`), solved
    exactly; colours by the parity of the subdomain index along each
    direction, c = sum_k 2^k (i_k mod 2), visited in increasing order; the
    residual is recomputed before each colour and the subdomains of one colour
    are corrected from that same residual; one sweep from a zero guess.
    """

    def __init__(self, K, shape, nsub, overlap):
        d = len(shape)
        self.K = K.tocsr()
        self.subs = []            # (colour, dof indices, LU of the local matrix)
        edges = [near_equal_edges(shape[d - 1 - k], nsub[k]) for k in range(d)]
        for sidx in np.ndindex(*[nsub[k] for k in range(d)]):
            lo = [0] * d
            hi = [0] * d
            colour = 0
            for k in range(d):
                a = d - 1 - k
                lo[a] = max(edges[k][sidx[k]] - overlap, 0)
                hi[a] = min(edges[k][sidx[k] + 1] + overlap, shape[a])
                colour += (sidx[k] % 2) << k
            idx = box_dofs(shape, lo, hi)
            lu = spla.splu(self.K[idx][:, idx].tocsc())
            self.subs.append((colour, idx, lu))
        self.colours = sorted({c for c, _, _ in self.subs})

    def solve(self, b):
        x = np.zeros_like(b)
        for col in self.colours:
            r = b - self.K @ x
            dx = np.zeros_like(b)
            for c, idx, lu in self.subs:
                if c == col:
                    dx[idx] += lu.solve(r[idx])
            x = x + dx
        return x


# ------------------------------------------------------------- hierarchy
DEFAULT_W = {2: [0.75], 3: [0.75, 0.5], 4: [0.5, 0.5, 0.2]}


class Hierarchy:
    """Multigrid hierarchy of the shifted operator K_s = K_0, K_{l+1} = P_l^T K_l P_l."""

    def __init__(self, Ks, shape, levels, w=None, economic=True, order="rb",
                 wu=None, wp=None, coarse_dd=None):
        """coarse_dd = (nsub, overlap): MG-DD, the coarsest level solved by
        one sweep of `CoarseDD` instead of the exact LU."""
        if w is None:
            w = DEFAULT_W.get(levels, [0.75, 0.5] + [0.25] * max(0, levels - 3))
        self.levels = levels
        self.order = order
        self.shapes = [tuple(shape)]
        self.K = [Ks.tocsr()]
        self.P = []
        for l in range(levels - 1):
            cs = tuple(s // 2 for s in self.shapes[-1])
            assert all(2 * c == s for c, s in zip(cs, self.shapes[-1])), "grid not divisible"
            P = prolongation(cs)
            self.P.append(P)
            self.K.append((P.T @ self.K[-1] @ P).tocsr())
            self.shapes.append(cs)
        self.lv = [Level(self.K[l], self.shapes[l], w[l], economic, wu, wp)
                   for l in range(levels - 1)]
        if coarse_dd is None:
            self.lu = spla.splu(self.K[-1].tocsc())
            self.coarse_solve = self.lu.solve
        else:
            self.cdd = CoarseDD(self.K[-1], self.shapes[-1], *coarse_dd)
            self.coarse_solve = self.cdd.solve

    def relax(self, l, b, x):
        lv = self.lv[l]
        return lv.relax_rb(b, x) if self.order == "rb" else lv.relax_lex(b, x)

    def cycle(self, b, l=0, x=None, nu1=1, nu2=1, gamma=1):
        """Algorithm TwoCycle applied recursively: gamma = 1 V-cycle, 2 W-cycle."""
        if l == self.levels - 1:
            return self.coarse_solve(b)
        x = np.zeros_like(b) if x is None else x.copy()
        for _ in range(nu1):
            x = self.relax(l, b, x)
        rc = self.P[l].T @ (b - self.K[l] @ x)
        ec = None
        for _ in range(gamma):
            ec = self.cycle(rc, l + 1, ec, nu1, nu2, gamma)
            if l + 1 == self.levels - 1:
                break                   # one coarsest solve per visit (exact or DD)
        x = x + self.P[l] @ ec
        for _ in range(nu2):
            x = self.relax(l, b, x)
        return x
