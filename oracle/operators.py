"""Assembly of the staggered-grid elastic Helmholtz operators (oracle).

Follows Sec. 2.1 (eq. elasticHelmSystem and eq. elasticHelmMass), Sec. 2.2
(eq. shift) and Sec. 3 (eq. pressure, eq. elasticHelmReformulatedSystem and
the zero-padded shift matrix).  Readings of points the paper leaves open:

* boundary: homogeneous Dirichlet for u; the boundary-normal faces are not
  unknowns and tangential neighbours outside the grid are zero;
* A_e / A_f: arithmetic means; the normal derivative of u_k is weighted by
  the cell-centre mu, a tangential one by the mean of the 4 cells around the
  edge (indices clamped at the boundary);
* gamma = gamma_add + omega * abl_max * (depth / L)^2 inside an L-cell layer
  on every side (max over directions at corners);
* shift: the artificial attenuation has the same sign as the physical one,
  K_s = K + i alpha omega^2 diag(A_f(rho), 0).

Directions: k = 0, 1, 2 is x, y, z; numpy axis of direction k is d - 1 - k.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------- 1D pieces
def d_face_to_centre(n, h):
    """n x (n-1): (u_{c+1} - u_c)/h at cell c from interior faces 1..n-1."""
    rows, cols, vals = [], [], []
    for c in range(n):
        if c + 1 <= n - 1:
            rows.append(c); cols.append(c); vals.append(1.0 / h)      # face c+1 -> column c
        if c >= 1:
            rows.append(c); cols.append(c - 1); vals.append(-1.0 / h)  # face c   -> column c-1
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n - 1))


def d_cell_to_edge(n, h):
    """(n+1) x n: (u_e - u_{e-1})/h at edge e = 0..n, zero ghosts outside."""
    rows, cols, vals = [], [], []
    for e in range(n + 1):
        if e <= n - 1:
            rows.append(e); cols.append(e); vals.append(1.0 / h)
        if e >= 1:
            rows.append(e); cols.append(e - 1); vals.append(-1.0 / h)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n + 1, n))


def grad_centre_to_face(n, h):
    """(n-1) x n: (p_f - p_{f-1})/h on interior face f = 1..n-1."""
    rows, cols, vals = [], [], []
    for f in range(1, n):
        rows += [f - 1, f - 1]; cols += [f - 1, f]; vals += [-1.0 / h, 1.0 / h]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n - 1, n))


def avg_centre_to_face(n):
    """(n-1) x n: mean of the two cells beside interior face f."""
    rows, cols, vals = [], [], []
    for f in range(1, n):
        rows += [f - 1, f - 1]; cols += [f - 1, f]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n - 1, n))


def avg_centre_to_edge_clamped(n):
    """(n+1) x n: mean of cells e-1 and e with indices clamped into [0, n-1]."""
    rows, cols, vals = [], [], []
    for e in range(n + 1):
        for c in (e - 1, e):
            cc = min(max(c, 0), n - 1)
            rows.append(e); cols.append(cc); vals.append(0.5)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n + 1, n)).tocsr()


def kron_axes(mats):
    """Kronecker product over numpy axes (first = slowest)."""
    out = sp.csr_matrix(mats[0])
    for m in mats[1:]:
        out = sp.kron(out, m, format="csr")
    return out


def comp_shape(shape, k):
    """Array shape of the u_k unknowns: n_k - 1 along direction k."""
    d = len(shape)
    s = list(shape)
    s[d - 1 - k] -= 1
    return tuple(s)


def dof_sizes(shape):
    d = len(shape)
    sizes = [int(np.prod(comp_shape(shape, k))) for k in range(d)]
    sizes.append(int(np.prod(shape)))
    return sizes


# ------------------------------------------------------------------- media
def gamma_profile(shape, omega, abl_cells, abl_max=1.0, gamma_add=0.01 * np.pi):
    """gamma = gamma_add + omega * abl_max * max_k (depth_k / L)^2 (eq. elasticHelmMass).

    depth_k counts cells into the layer from its inner edge: the outermost
    cell has depth L, the innermost layer cell depth 1, interior cells 0.
    """
    d = len(shape)
    ramp = np.zeros(shape)
    L = abl_cells
    if L > 0:
        for ax in range(d):
            n = shape[ax]
            i = np.arange(n)
            depth = np.maximum(np.maximum(L - i, i - (n - 1 - L)), 0).astype(float)
            r = (depth / L) ** 2
            sh = [1] * d
            sh[ax] = n
            ramp = np.maximum(ramp, r.reshape(sh))
    return gamma_add + omega * abl_max * ramp


# ------------------------------------------------------------ operator parts
class Parts:
    """The named blocks of eq. elasticHelmSystem / elasticHelmReformulatedSystem."""

    def __init__(self, lam, mu, rho, gamma, omega, h):
        self.shape = lam.shape
        d = self.d = lam.ndim
        self.omega, self.h = omega, h
        n = lambda k: self.shape[d - 1 - k]
        ax = lambda k: d - 1 - k
        self.L = []      # weighted Laplacian per component: sum_j D^T A_e(mu) D
        self.terms = []  # per component: list of (D, W) with the term D^T diag(W mu) D
        self.A = []      # face-averaging matrix per component (cells -> u_k faces)
        self.M = []      # A_f(rho (1 - i gamma / omega)) per component (diagonal)
        self.Ms = []     # A_f(rho) per component (shift mass)
        self.G = []      # centres -> u_k faces gradient
        mass_cell = rho * (1.0 - 1j * gamma / omega)
        for k in range(d):
            Lk = None
            tk = []
            for j in range(d):
                mats, wmats = [], []
                for a in range(d):
                    na = self.shape[a]
                    if a == ax(k) and a == ax(j):
                        mats.append(d_face_to_centre(na, h))
                        wmats.append(sp.identity(na, format="csr"))      # mu at centres
                    elif a == ax(k):
                        mats.append(sp.identity(na - 1, format="csr"))
                        wmats.append(avg_centre_to_face(na))
                    elif a == ax(j):
                        mats.append(d_cell_to_edge(na, h))
                        wmats.append(avg_centre_to_edge_clamped(na))
                    else:
                        mats.append(sp.identity(na, format="csr"))
                        wmats.append(sp.identity(na, format="csr"))
                D = kron_axes(mats)
                Wm = kron_axes(wmats)
                w = Wm @ mu.ravel()
                tk.append((D, Wm))
                term = D.T @ sp.diags(w) @ D
                Lk = term if Lk is None else Lk + term
            self.L.append(Lk.tocsr())
            self.terms.append(tk)
            A = kron_axes([avg_centre_to_face(self.shape[a]) if a == ax(k)
                           else sp.identity(self.shape[a], format="csr") for a in range(d)])
            self.A.append(A)
            self.M.append(sp.diags(A @ mass_cell.ravel()))
            self.Ms.append(sp.diags(A @ rho.ravel()))
            self.G.append(kron_axes([grad_centre_to_face(self.shape[a], h) if a == ax(k)
                                     else sp.identity(self.shape[a], format="csr")
                                     for a in range(d)]))
        self.lam_mu = (lam + mu).ravel()
        self.gamma = gamma.ravel()


def assemble_mixed(parts: Parts, alpha=0.0):
    """K (alpha = 0) or K_s: [[L - w^2 M + i alpha w^2 M_s, G], [G^T, -D_c(1/(lam+mu))]]."""
    d, w2 = parts.d, parts.omega ** 2
    blocks = [[None] * (d + 1) for _ in range(d + 1)]
    for k in range(d):
        blocks[k][k] = parts.L[k] - w2 * parts.M[k] + 1j * alpha * w2 * parts.Ms[k]
        blocks[k][d] = parts.G[k]
        blocks[d][k] = parts.G[k].T
    blocks[d][d] = sp.diags(-1.0 / parts.lam_mu)
    return sp.bmat(blocks, format="csr").astype(np.complex128)


def assemble_displacement(parts: Parts, alpha=0.0):
    """H^e = grad_h D_c(lam+mu) grad_h^T + L_mu - w^2 M (eq. elasticHelmSystem)."""
    d, w2 = parts.d, parts.omega ** 2
    G = sp.vstack(parts.G, format="csr")
    GDGt = G @ sp.diags(parts.lam_mu) @ G.T
    blocks = [[None] * d for _ in range(d)]
    for k in range(d):
        blocks[k][k] = parts.L[k] - w2 * parts.M[k] + 1j * alpha * w2 * parts.Ms[k]
    A = sp.bmat(blocks, format="csr")
    return (A + GDGt).tocsr().astype(np.complex128)


def parts_for(medium, abl_max=1.0, gamma_add=0.01 * np.pi):
    gamma = gamma_profile(medium.lam.shape, medium.omega, medium.abl_cells, abl_max, gamma_add)
    return Parts(medium.lam, medium.mu, medium.rho, gamma, medium.omega, medium.h)


# ------------------------------------------------------------ layout helpers
def slots_to_dofs(v, shape):
    """Slot layout (d+1, *shape) -> oracle DOF vector (drops Dirichlet slots)."""
    d = len(shape)
    parts = []
    for k in range(d):
        sl = [slice(None)] * d
        sl[d - 1 - k] = slice(1, None)
        parts.append(np.asarray(v[k])[tuple(sl)].ravel())
    parts.append(np.asarray(v[d]).ravel())
    return np.concatenate(parts)


def dofs_to_slots(x, shape):
    """Oracle DOF vector -> slot layout (d+1, *shape) with zero Dirichlet slots."""
    d = len(shape)
    out = np.zeros((d + 1,) + tuple(shape), dtype=np.result_type(x.dtype, np.complex128))
    off = 0
    for k in range(d):
        cs = comp_shape(shape, k)
        m = int(np.prod(cs))
        sl = [slice(None)] * d
        sl[d - 1 - k] = slice(1, None)
        out[(k,) + tuple(sl)] = x[off:off + m].reshape(cs)
        off += m
    out[d] = x[off:].reshape(shape)
    return out
