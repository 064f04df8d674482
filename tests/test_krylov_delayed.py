"""The Arnoldi scheme of the double-float solve, restated in numpy (no GPU).

The paper does not say how the Arnoldi vectors are orthogonalised.  The oracle
uses CGS2 (classical Gram-Schmidt applied twice).  The GPU's double-float solve
uses delayed CGS2 instead: the second projection of direction u_j is formed in
the pass that forms the first projection of w = K z_j, and the preconditioner is
applied to the once-orthogonalised u_j (flexible GMRES allows any z_j).  Only
the second projection is carried in full precision; the first projection of w
is formed from single-precision products.

Here that scheme is written out step by step (FP64 for the second projection,
complex64 products and sums for the first) and held to the oracle's CGS2 FGMRES
with the oracle's multigrid preconditioner:

* the same iteration counts and solutions within 1e-9 (restart 10 and 3),
* K Z = U H column by column (U: the final basis plus the last provisional
  direction) and an orthonormal basis, both to 1e-12, although the first
  projection is single precision.
"""
import numpy as np
import pytest

from oracle import krylov, multigrid as mg, operators as op
from paper_1806_11277_gb300 import synth


def _lsq_residual(H, beta, k):
    """min_y ||beta e1 - H[:k+1, :k] y|| and its minimiser."""
    rhs = np.zeros(k + 1, complex)
    rhs[0] = beta
    y = np.linalg.lstsq(H[:k + 1, :k], rhs, rcond=None)[0]
    return np.linalg.norm(rhs - H[:k + 1, :k] @ y), y


def fgmres_delayed(matvec, precond, b, m=10, tol=1e-6, maxit=500, trace=None):
    """Right-preconditioned FGMRES(m) with delayed CGS2; slot j of U holds u_j
    (the direction handed to the preconditioner) until step j turns it into
    v_j.  Returns (x, iterations)."""
    n = b.shape[0]
    x = np.zeros(n, complex)
    bnorm = np.linalg.norm(b)
    r = b.astype(complex)
    beta = np.linalg.norm(r)
    iters = 0
    while beta / bnorm > tol and iters < maxit:
        U = np.zeros((m + 1, n), complex)
        Z = np.zeros((m, n), complex)
        H = np.zeros((m + 1, m), complex)
        U[0] = r / beta
        rho = 0.0
        k = 0
        for j in range(m):
            u = U[j].copy()
            Z[j] = precond(u)
            w = matvec(Z[j])
            Vf = U[:j]
            # second projection of u_j, full precision
            a = Vf.conj() @ u
            d = np.vdot(u, u).real
            # first projection of w: complex64 products and sums
            t = (U[:j + 1].astype(np.complex64).conj() @ w.astype(np.complex64)).astype(complex)
            bw, c = t[:j], t[j]
            e = float(np.vdot(w.astype(np.complex64), w.astype(np.complex64)).real)
            if j > 0:
                sig = np.sqrt(d - np.vdot(a, a).real)
                H[:j, j - 1] += rho * a            # u_j = V a + sigma v_j, scaled by the last rho
                H[j, j - 1] = rho * sig
            else:
                sig = 1.0                          # u_0 = r / ||r||
            hj = (c - np.vdot(a, bw)) / sig
            rho = np.sqrt(max(e - np.vdot(bw, bw).real - abs(hj) ** 2, 1e-12 * e))
            H[:j, j] = bw
            H[j, j] = hj
            H[j + 1, j] = rho
            U[j] = (u - a @ Vf) / sig
            U[j + 1] = (w - (bw - a * hj / sig) @ Vf - u * (hj / sig)) / rho
            iters += 1
            k = j + 1
            res, _ = _lsq_residual(H, beta, k)
            if res / bnorm <= tol or iters >= maxit:
                break
        _, y = _lsq_residual(H, beta, k)
        if trace is not None:
            trace.append((U[:k + 1].copy(), Z[:k].copy(), H[:k + 1, :k].copy()))
        x = x + y @ Z[:k]
        r = b - matvec(x)
        beta = np.linalg.norm(r)
    return x, iters


def _problem(sigma, n=64):
    med = synth.random_2d(n=n, sigma=sigma, seed=0)
    parts = op.parts_for(med)
    K = op.assemble_mixed(parts)
    H = mg.Hierarchy(op.assemble_mixed(parts, 0.2), med.shape, 2, w=[0.75, 0.5])
    q = op.slots_to_dofs(synth.point_rhs(med.shape, med.sources)[0], med.shape)
    return K, H, q


@pytest.mark.parametrize("m", [10, 3])
def test_delayed_cgs2_matches_oracle_cgs2(m):
    for sigma in (0.25, 0.49):
        K, H, q = _problem(sigma)
        xo, io = krylov.fgmres(lambda v: K @ v, H.cycle, q, m=m, tol=1e-6)
        xd, it = fgmres_delayed(lambda v: K @ v, H.cycle, q, m=m, tol=1e-6)
        assert it == io["iters"], (sigma, m, it, io["iters"])
        assert np.abs(xd - xo).max() <= 1e-9 * np.abs(xo).max()
        assert np.linalg.norm(q - K @ xd) <= 1e-6 * np.linalg.norm(q)


def test_delayed_cgs2_arnoldi_relation_and_orthogonality():
    K, H, q = _problem(0.4)
    trace = []
    fgmres_delayed(lambda v: K @ v, H.cycle, q, m=10, tol=1e-6, trace=trace)
    U, Z, Hm = trace[0]
    k = Z.shape[0]
    KZ = np.stack([K @ z for z in Z])
    # K z_j = sum_i U_i H[i, j]: the columns as corrected by the next step, the last one provisional
    assert np.linalg.norm(KZ - Hm.T @ U) <= 1e-12 * np.linalg.norm(KZ)
    V = U[:k]                                      # v_0 .. v_{k-1} are final
    assert np.abs(V.conj() @ V.T - np.eye(k)).max() <= 1e-12
