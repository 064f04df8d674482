"""Right-preconditioned flexible GMRES(m) (oracle).

The shifted-Laplacian framework of Sec. 2.2 uses a multigrid cycle on the
shifted matrix as the preconditioner of a (flexible) GMRES solve of the
original system; Sec. 6 solves to a 1e-6 relative residual from a zero
initial guess and counts preconditioner applications.  Arnoldi uses
classical Gram-Schmidt applied twice (CGS2) and complex Givens rotations.
"""
from __future__ import annotations

import numpy as np


def _givens(a, b):
    """Complex Givens rotation (c real, s complex) with c a + s b = r, -conj(s) a + c b = 0."""
    if b == 0:
        return 1.0, 0.0j, a
    if a == 0:
        return 0.0, np.conj(b) / abs(b), abs(b)
    t = abs(a)
    nrm = np.hypot(t, abs(b))
    c = t / nrm
    s = (a / t) * np.conj(b) / nrm
    return c, s, (a / t) * nrm


def fgmres(matvec, precond, b, m=10, tol=1e-6, maxit=500, x0=None):
    """Returns (x, info) with info = dict(iters, relres, history, converged)."""
    n = b.shape[0]
    x = np.zeros(n, dtype=np.complex128) if x0 is None else x0.astype(np.complex128).copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return x, dict(iters=0, relres=0.0, history=[0.0], converged=True)
    r = b - matvec(x) if x0 is not None else b.astype(np.complex128).copy()
    beta = np.linalg.norm(r)
    hist = [beta / bnorm]
    iters = 0
    converged = beta / bnorm <= tol
    while not converged and iters < maxit:
        V = np.zeros((m + 1, n), dtype=np.complex128)
        Z = np.zeros((m, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_used = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = matvec(Z[j])
            h = np.zeros(j + 1, dtype=np.complex128)
            for _ in range(2):                       # CGS2
                hh = V[:j + 1].conj() @ w
                w = w - hh @ V[:j + 1]
                h += hh
            hn = np.linalg.norm(w)
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            iters += 1
            j_used = j + 1
            for i in range(j):                       # apply previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            c, s, rr = _givens(H[j, j], H[j + 1, j])
            cs[j], sn[j] = c, s
            H[j, j] = rr
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            res = abs(g[j + 1]) / bnorm
            hist.append(res)
            if hn == 0.0:
                break
            V[j + 1] = w / hn
            if res <= tol or iters >= maxit:
                break
        k = j_used
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):               # back substitution
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + y @ Z[:k]
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        converged = beta / bnorm <= tol
    return x, dict(iters=iters, relres=beta / bnorm, history=hist, converged=converged)
