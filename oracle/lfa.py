"""Local Fourier analysis of lexicographic cell-wise (Vanka) relaxation (oracle).

Sec. 5 of the paper: the 2D mixed operator with constant coefficients, the
economic block B of eq. RelaxationMatrix, a lexicographic sweep (x fastest),
per-component damping (w_u, w_v, w_p).  The smoothing factor mu_loc is the
largest spectral radius of the symbol S(theta) over the high frequencies
T_high = [-pi/2, 3pi/2]^2 minus [-pi/2, pi/2]^2 (Definition def_mu_loc).

The 5 x 5 / 5 x 3 relation between partially/fully updated and un-updated
amplitudes (eq. PQdef) is generated here from first principles instead of
being typed in from the printed matrices: for the cell being relaxed, every
DOF in the stencil of its five rows is classified as un-updated, partially
updated or fully updated by counting how many of the cells that own it come
earlier in the lexicographic order; the update equation
    e_after = e_before - W B^{-1} (A e_before)_local
is then written in amplitudes, which gives one linear relation per local DOF.
The operator stencil values are passed in, so a caller can take them from
an assembled matrix.

Red-black order (the order the solver uses; Sec. 5 analyses only the
lexicographic one): a half-step relaxes every cell of one colour from one
residual, so a plane wave theta mixes only with theta + (pi, pi).  The 6 x 6
symbol of a red-black sweep is obtained by applying both half-steps to the
two harmonics on the infinite grid, cell by cell, and reading the new
amplitudes back at two cells of opposite colour; the smoothing factor takes
the high harmonics of each pair.  Either block (economic or full) can be
analysed.
"""
from __future__ import annotations

import numpy as np

# local DOF order of a cell (i, j): u left, u right, v bottom, v top, p
# positions are in half-cell units relative to the cell centre.
LOCAL = [("u", (-1, 0)), ("u", (1, 0)), ("v", (0, -1)), ("v", (0, 1)), ("p", (0, 0))]


def _owners(comp, pos):
    """Cells (in cell units, relative to the relaxed cell) that own a DOF."""
    px, py = pos
    if comp == "u":           # face between cells (px-1)/2 and (px+1)/2 along x
        return [((px - 1) // 2, py // 2), ((px + 1) // 2, py // 2)]
    if comp == "v":
        return [(px // 2, (py - 1) // 2), (px // 2, (py + 1) // 2)]
    return [(px // 2, py // 2)]


def _before(cell):
    """Lexicographic order, x fastest: is ``cell`` relaxed before (0, 0)?"""
    ci, cj = cell
    return cj < 0 or (cj == 0 and ci < 0)


def _state(comp, pos, include_self):
    n = sum(1 for c in _owners(comp, pos) if _before(c) or (include_self and c == (0, 0)))
    if comp == "p":
        return 2 if n else 0
    return n                   # 0 un-updated, 1 partially, 2 fully updated


def row_stencil(comp, s):
    """Neighbours (comp, offset in half units, coefficient) of a row of the
    2D operator [[-mu Lap - w^2 M, d_x], [.., -mu Lap - w^2 M, d_y], [-d_x, -d_y, -1/(l+m)]].

    s: dict with keys s00, sx (x-neighbour), sy (y-neighbour), g (1/h), c (1/(lam+mu))."""
    if comp == "u":
        return [("u", (0, 0), s["s00"]), ("u", (2, 0), s["sx"]), ("u", (-2, 0), s["sx"]),
                ("u", (0, 2), s["sy"]), ("u", (0, -2), s["sy"]),
                ("p", (1, 0), s["g"]), ("p", (-1, 0), -s["g"])]
    if comp == "v":
        return [("v", (0, 0), s["s00"]), ("v", (0, 2), s["sx"]), ("v", (0, -2), s["sx"]),
                ("v", (2, 0), s["sy"]), ("v", (-2, 0), s["sy"]),
                ("p", (0, 1), s["g"]), ("p", (0, -1), -s["g"])]
    return [("u", (1, 0), -s["g"]), ("u", (-1, 0), s["g"]),
            ("v", (0, 1), -s["g"]), ("v", (0, -1), s["g"]), ("p", (0, 0), -s["c"])]


def economic_block(s):
    """Arrowhead B: diagonal displacement block, its pressure couplings, p-p entry."""
    B = np.zeros((5, 5), dtype=np.complex128)
    for a, (ca, pa) in enumerate(LOCAL):
        for (cb, off, val) in row_stencil(ca, s):
            pb = (pa[0] + off[0], pa[1] + off[1])
            for b, (cl, pl) in enumerate(LOCAL):
                if cl == cb and pl == pb:
                    if a < 4 and b < 4 and a != b:
                        continue
                    B[a, b] += val
    return B


# unknown amplitude vector X = [u_half, v_half, u_full, v_full, p_full]
# known amplitudes Y = [u0, v0, p0]
def _var(comp, state):
    if state == 0:
        return ("Y", {"u": 0, "v": 1, "p": 2}[comp])
    if state == 1:
        return ("X", {"u": 0, "v": 1}[comp])
    return ("X", {"u": 2, "v": 3, "p": 4}[comp])


def symbol(theta, s, wu, wv, wp, B=None):
    """3 x 3 amplification matrix S(theta) of one lexicographic sweep."""
    t1, t2 = theta
    ph = lambda pos: np.exp(0.5j * (t1 * pos[0] + t2 * pos[1]))
    B = economic_block(s) if B is None else B
    Binv = np.linalg.inv(B)
    W = np.array([wu, wu, wv, wv, wp])
    # R[a] = residual row a as linear form in (X, Y): coefficient arrays
    RX = np.zeros((5, 5), dtype=np.complex128)
    RY = np.zeros((5, 3), dtype=np.complex128)
    for a, (ca, pa) in enumerate(LOCAL):
        for (cb, off, val) in row_stencil(ca, s):
            pb = (pa[0] + off[0], pa[1] + off[1])
            kind, i = _var(cb, _state(cb, pb, include_self=False))
            (RX if kind == "X" else RY)[a, i] += val * ph(pb)
    # update: after(q) phase(q) = before(q) phase(q) - W[q] (Binv R)[q]
    CX = -(W[:, None] * (Binv @ RX))
    CY = -(W[:, None] * (Binv @ RY))
    PX = np.zeros((5, 5), dtype=np.complex128)
    QY = np.zeros((5, 3), dtype=np.complex128)
    for q, (cq, pq) in enumerate(LOCAL):
        kb, ib = _var(cq, _state(cq, pq, include_self=False))
        ka, ia = _var(cq, _state(cq, pq, include_self=True))
        # after - before - C = 0
        PX[q, ia] += ph(pq)
        if kb == "X":
            PX[q, ib] -= ph(pq)
        else:
            QY[q, ib] += ph(pq)
        PX[q] -= CX[q]
        QY[q] += CY[q]
    T = np.linalg.solve(PX, QY)
    return T[2:5]


def stencil_values(h, omega, gamma, lam, mu, rho):
    """Constant-coefficient stencil with the LFA mass rho (1 - i gamma) (Sec. 5)."""
    return dict(s00=4 * mu / h ** 2 - rho * omega ** 2 * (1 - 1j * gamma),
                sx=-mu / h ** 2, sy=-mu / h ** 2, g=1.0 / h, c=1.0 / (lam + mu))


def mu_loc(s, wu, wv=None, wp=None, nsamp=63):
    """sup over the sampled high frequencies of rho(S(theta))."""
    wv = wu if wv is None else wv
    wp = wu if wp is None else wp
    th = np.linspace(-np.pi / 2, 3 * np.pi / 2, nsamp)
    B = economic_block(s)
    best = 0.0
    for t1 in th:
        for t2 in th:
            if abs(t1) <= np.pi / 2 and abs(t2) <= np.pi / 2:
                continue
            S = symbol((t1, t2), s, wu, wv, wp, B)
            best = max(best, np.max(np.abs(np.linalg.eigvals(S))))
    return best


def full_block(s):
    """Full (2d+1)^2 cell block: every coupling among the cell's five DOFs."""
    B = np.zeros((5, 5), dtype=np.complex128)
    for a, (ca, pa) in enumerate(LOCAL):
        for (cb, off, val) in row_stencil(ca, s):
            pb = (pa[0] + off[0], pa[1] + off[1])
            for b, (cl, pl) in enumerate(LOCAL):
                if cl == cb and pl == pb:
                    B[a, b] += val
    return B


# ------------------------------------------------------------ red-black
# Cells (i, j) have centres at half-unit position (2i+1, 2j+1) and colour
# (i + j) mod 2 (0 = red, relaxed first).  A red-black half-step updates all
# cells of one colour at once from one residual, so the pair of harmonics
# theta and theta + (pi, pi) spans an invariant space: the amplitudes are
# A = [u, v, p of phi_theta, u, v, p of phi_(theta+(pi,pi))].
_TYPES = ("u", "v", "p")


def _dof_pos(t, i, j):
    """Half-unit position of the type-t DOF that belongs to cell (i, j) on its low side."""
    return {"u": (2 * i, 2 * j + 1), "v": (2 * i + 1, 2 * j), "p": (2 * i + 1, 2 * j + 1)}[t]


def _owners_rb(t, i, j):
    """(cell, local index) pairs owning the type-t DOF of cell (i, j)."""
    if t == "u":
        return [((i - 1, j), 1), ((i, j), 0)]
    if t == "v":
        return [((i, j - 1), 3), ((i, j), 2)]
    return [((i, j), 4)]


def _half_step_rb(theta, s, W, Binv, colour, A):
    t1, t2 = theta
    ph = lambda X, sh: np.exp(0.5j * ((t1 + sh * np.pi) * X[0] + (t2 + sh * np.pi) * X[1]))

    def err(t, X):
        k = _TYPES.index(t)
        return A[k] * ph(X, 0) + A[3 + k] * ph(X, 1)

    def delta(ci, cj):
        cx, cy = 2 * ci + 1, 2 * cj + 1
        r = np.zeros(5, dtype=np.complex128)
        for a, (ca, pa) in enumerate(LOCAL):
            for (cb, off, val) in row_stencil(ca, s):
                r[a] -= val * err(cb, (cx + pa[0] + off[0], cy + pa[1] + off[1]))
        return W * (Binv @ r)

    out = np.zeros(6, dtype=np.complex128)
    for k, t in enumerate(_TYPES):
        rows, rhs = [], []
        for q in (0, 1):                        # two cells of opposite colour parity
            X = _dof_pos(t, q, 0)
            v = err(t, X)
            for (ci, cj), a in _owners_rb(t, q, 0):
                if (ci + cj) % 2 == colour:
                    v += delta(ci, cj)[a]
            rows.append([ph(X, 0), ph(X, 1)])
            rhs.append(v)
        out[k], out[3 + k] = np.linalg.solve(np.array(rows), np.array(rhs))
    return out


def symbol_rb(theta, s, wu, wv, wp, B=None):
    """6 x 6 amplification matrix of one red-black sweep (red, then black) on the
    harmonic pair theta, theta + (pi, pi)."""
    B = economic_block(s) if B is None else B
    Binv = np.linalg.inv(B)
    W = np.array([wu, wu, wv, wv, wp])
    S = []
    for colour in (0, 1):
        M = np.zeros((6, 6), dtype=np.complex128)
        for col in range(6):
            e = np.zeros(6, dtype=np.complex128)
            e[col] = 1.0
            M[:, col] = _half_step_rb(theta, s, W, Binv, colour, e)
        S.append(M)
    return S[1] @ S[0]


def mu_loc_rb(s, wu, wv=None, wp=None, nsamp=32, B=None):
    """Smoothing factor of one red-black sweep: over theta in the low box, the
    largest spectral radius of the sweep restricted to the high harmonics of the
    pairs (theta, theta + (pi, pi)) (theta low, so only its partner is high)
    and (theta + (pi, 0), theta + (0, pi)) (both high)."""
    wv = wu if wv is None else wv
    wp = wu if wp is None else wp
    th = -np.pi / 2 + np.pi * (np.arange(nsamp) + 0.5) / nsamp
    best = 0.0
    for t1 in th:
        for t2 in th:
            S = symbol_rb((t1, t2), s, wu, wv, wp, B)
            best = max(best, np.max(np.abs(np.linalg.eigvals(S[3:, 3:]))))
            S2 = symbol_rb((t1 + np.pi, t2), s, wu, wv, wp, B)
            best = max(best, np.max(np.abs(np.linalg.eigvals(S2))))
    return best
