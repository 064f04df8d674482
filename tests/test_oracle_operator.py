"""Pins of the oracle's operator assembly against closed forms (no GPU).

* discrete Fourier symbol of H^e with constant coefficients: P and S
  dispersion relations (Sec. 2.1; the symbol of the stencils eq. LStencil /
  eq. GStencil),
* complex symmetry of K, K_s and H^e,
* H^e is the Schur complement of the mixed system (Sec. 3),
* acoustic limit mu = 0: eliminating u gives the cell-centred acoustic
  operator (Sec. 3, "relation between the acoustic and elastic equations"),
* second-order convergence on a manufactured solution,
* the absorbing-layer profile of eq. elasticHelmMass.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import operators as op
from paper_1806_11277_gb300 import synth


def _const_parts(shape, lam, mu, rho, omega, gamma, h=1.0):
    f = lambda v: np.full(shape, float(v))
    return op.Parts(f(lam), f(mu), f(rho), f(gamma), omega, h)


def _face_positions(shape, k, h):
    """Physical coordinates (x, y[, z]) of every u_k slot, in numpy array shape."""
    d = len(shape)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    coords = []
    for kk in range(d):
        ax = d - 1 - kk
        c = grids[ax].astype(float) + 0.5
        if kk == k:
            c = c - 0.5
        coords.append(c * h)
    return coords


@pytest.mark.parametrize("shape", [(24, 28), (10, 12, 14)])
def test_symbol_matches_p_and_s_dispersion(shape):
    d = len(shape)
    lam, mu, rho, omega, gamma, h = 3.0, 1.3, 1.7, 0.9, 0.25, 0.5
    parts = _const_parts(shape, lam, mu, rho, omega, gamma, h)
    He = op.assemble_displacement(parts)
    rng = np.random.default_rng(0)
    theta = rng.uniform(0.3, 2.5, d)
    sh = 2 * np.sin(theta / 2) / h
    khat2 = np.sum(sh ** 2)
    rhot = rho * (1 - 1j * gamma / omega)
    for kind in ("P", "S"):
        if kind == "P":
            a = sh / np.linalg.norm(sh)
            expect = (lam + 2 * mu) * khat2 - omega ** 2 * rhot
        else:
            a = np.zeros(d); a[0], a[1] = -sh[1], sh[0]
            a /= np.linalg.norm(a)
            expect = mu * khat2 - omega ** 2 * rhot
        slots = np.zeros((d + 1,) + shape, dtype=np.complex128)
        for k in range(d):
            X = _face_positions(shape, k, h)
            slots[k] = a[k] * np.exp(1j * sum(theta[j] * X[j] / h for j in range(d)))
        u = op.slots_to_dofs(slots, shape)[:He.shape[0]]
        y = op.dofs_to_slots(np.concatenate([He @ u, np.zeros(int(np.prod(shape)))]), shape)
        inner = tuple(slice(3, n - 3) for n in shape)
        scale = abs(expect)
        for k in range(d):
            got = y[k][inner]
            want = expect * slots[k][inner]
            assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * scale)


@pytest.mark.parametrize("shape", [(16, 20), (8, 10, 12)])
def test_complex_symmetry(shape):
    d = len(shape)
    rng = np.random.default_rng(1)
    lam = 1 + rng.random(shape); mu = 0.5 + rng.random(shape); rho = 1 + rng.random(shape)
    gamma = op.gamma_profile(shape, 0.8, 3)
    parts = op.Parts(lam, mu, rho, gamma, 0.8, 1.0)
    for M in (op.assemble_mixed(parts), op.assemble_mixed(parts, 0.3),
              op.assemble_displacement(parts)):
        assert abs(M - M.T).max() <= 1e-15 * abs(M).max()
        assert abs(M.imag).max() > 0            # really complex, not Hermitian
    K = op.assemble_mixed(parts)
    nu = sum(op.dof_sizes(shape)[:d])
    assert K.shape[0] == nu + int(np.prod(shape))


def test_schur_complement_is_displacement_operator():
    shape = (12, 14)
    rng = np.random.default_rng(2)
    lam = 2 + rng.random(shape); mu = 0.5 + rng.random(shape); rho = 1 + rng.random(shape)
    parts = op.Parts(lam, mu, rho, op.gamma_profile(shape, 0.7, 2), 0.7, 1.0)
    K = op.assemble_mixed(parts, 0.2)
    He = op.assemble_displacement(parts, 0.2)
    nu = He.shape[0]
    A, B, C = K[:nu, :nu], K[:nu, nu:], K[nu:, nu:]
    S = A - B @ sp.diags(1.0 / C.diagonal()) @ B.T
    assert abs(S - He).max() <= 1e-12 * abs(He).max()
    q = rng.standard_normal(nu) + 1j * rng.standard_normal(nu)
    up = spla.spsolve(K.tocsc(), np.concatenate([q, np.zeros(K.shape[0] - nu)]))
    u = spla.spsolve(He.tocsc(), q)
    assert np.linalg.norm(up[:nu] - u) <= 1e-10 * np.linalg.norm(u)
    # the pressure block is the scaled divergence of eq. pressure
    p = up[nu:]
    G = sp.vstack(parts.G)
    assert np.allclose(p, (lam + mu).ravel() * (G.T @ u), atol=1e-10 * np.abs(p).max())


def test_acoustic_limit():
    """mu = 0, gamma = 0: eliminating u from K gives
    -1/lambda + omega^-2 (acoustic 5-point operator with face densities)."""
    ny, nx, h, omega = 6, 7, 0.5, 1.3
    rng = np.random.default_rng(3)
    lam = 1 + rng.random((ny, nx)); rho = 1 + rng.random((ny, nx))
    parts = op.Parts(lam, np.zeros((ny, nx)), rho, np.zeros((ny, nx)), omega, h)
    K = op.assemble_mixed(parts).toarray()
    nu = K.shape[0] - ny * nx
    S = K[nu:, nu:] - K[nu:, :nu] @ np.linalg.solve(K[:nu, :nu], K[:nu, nu:])
    # brute-force cell loop: flux (p_nb - p_c) / (h^2 * mean(rho)) through interior faces
    A = np.zeros((ny * nx, ny * nx))
    cid = lambda j, i: j * nx + i
    for j in range(ny):
        for i in range(nx):
            for dj, di in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                jj, ii = j + dj, i + di
                if 0 <= jj < ny and 0 <= ii < nx:
                    rf = 0.5 * (rho[j, i] + rho[jj, ii])
                    A[cid(j, i), cid(jj, ii)] += 1.0 / (h * h * rf)
                    A[cid(j, i), cid(j, i)] -= 1.0 / (h * h * rf)
    expect = -np.diag(1.0 / lam.ravel()) - A / omega ** 2
    assert np.allclose(S, expect, atol=1e-12 * np.abs(expect).max())


def test_manufactured_solution_second_order():
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    pi = sympy.pi
    u1 = sympy.sin(pi * x) * sympy.sin(pi * y) ** 2
    u2 = sympy.sin(pi * x) ** 2 * sympy.sin(pi * y)
    lam_e = 2 + x * y
    mu_e = 1 + x ** 2 / 2
    rho_e = 1 + y / 4
    om = 2.0
    div = sympy.diff(u1, x) + sympy.diff(u2, y)
    f1 = -(sympy.diff((lam_e + mu_e) * div, x)
           + sympy.diff(mu_e * sympy.diff(u1, x), x) + sympy.diff(mu_e * sympy.diff(u1, y), y)) \
        - om ** 2 * rho_e * u1
    f2 = -(sympy.diff((lam_e + mu_e) * div, y)
           + sympy.diff(mu_e * sympy.diff(u2, x), x) + sympy.diff(mu_e * sympy.diff(u2, y), y)) \
        - om ** 2 * rho_e * u2
    F = [sympy.lambdify((x, y), f, "numpy") for f in (f1, f2)]
    U = [sympy.lambdify((x, y), u, "numpy") for u in (u1, u2)]
    C = [sympy.lambdify((x, y), c, "numpy") for c in (lam_e, mu_e, rho_e)]
    errs = []
    ns = [16, 32, 64, 128]
    for n in ns:
        h = 1.0 / n
        yc, xc = np.meshgrid((np.arange(n) + 0.5) * h, (np.arange(n) + 0.5) * h, indexing="ij")
        lam, mu, rho = [np.broadcast_to(c(xc, yc), (n, n)).astype(float) for c in C]
        parts = op.Parts(lam, mu, rho, np.zeros((n, n)), om, h)
        He = op.assemble_displacement(parts)
        fs = np.zeros((3, n, n), dtype=np.complex128)
        us = np.zeros((3, n, n), dtype=np.complex128)
        for k in range(2):
            X, Y = _face_positions((n, n), k, h)
            fs[k] = F[k](X, Y)
            us[k] = U[k](X, Y)
        f = op.slots_to_dofs(fs, (n, n))[:He.shape[0]]
        ue = op.slots_to_dofs(us, (n, n))[:He.shape[0]]
        uh = spla.spsolve(He.tocsc(), f)
        errs.append(np.sqrt(np.mean(np.abs(uh - ue) ** 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders[1:] - 2.0) < 0.15), (errs, orders)


def test_gamma_profile():
    omega, L = 0.7, 4
    g = op.gamma_profile((12, 16), omega, L, abl_max=1.0, gamma_add=0.05)
    assert np.isclose(g[6, 8], 0.05)
    assert np.isclose(g[0, 8], 0.05 + omega)                 # outermost: gamma / omega = 1
    assert np.isclose(g[6, 15], 0.05 + omega)
    assert np.isclose(g[6, 3], 0.05 + omega * (1 / L) ** 2)  # innermost layer cell
    assert np.isclose(g[1, 2], 0.05 + omega * (3 / L) ** 2)  # corner: max over directions
    assert np.allclose(g, g[::-1, ::-1])


def test_schur_complement_is_displacement_operator_3d():
    """Eliminating p from the 3D mixed system gives H^e = S + grad D(lambda+mu) div."""
    shape = (6, 7, 8)
    rng = np.random.default_rng(12)
    lam = 2 + rng.random(shape); mu = 0.5 + rng.random(shape); rho = 1 + rng.random(shape)
    parts = op.Parts(lam, mu, rho, op.gamma_profile(shape, 0.7, 2), 0.7, 1.0)
    K = op.assemble_mixed(parts, 0.2)
    He = op.assemble_displacement(parts, 0.2)
    nu = He.shape[0]
    A, B, C = K[:nu, :nu], K[:nu, nu:], K[nu:, nu:]
    S = A - B @ sp.diags(1.0 / C.diagonal()) @ B.T
    assert abs(S - He).max() <= 1e-12 * abs(He).max()


def test_manufactured_solution_second_order_3d():
    """3D manufactured solution (Dirichlet-compatible sines, smooth lambda, mu,
    rho, no attenuation): the displacement error falls at second order."""
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    pi, s = sympy.pi, sympy.sin
    u = [s(pi * x) * s(pi * y) ** 2 * s(pi * z) ** 2,
         s(pi * x) ** 2 * s(pi * y) * s(pi * z) ** 2,
         s(pi * x) ** 2 * s(pi * y) ** 2 * s(pi * z)]
    X = (x, y, z)
    lam_e, mu_e, rho_e = 2 + x * y * z, 1 + x ** 2 / 2 + z / 4, 1 + y / 4
    om = 2.0
    div = sum(sympy.diff(u[k], X[k]) for k in range(3))
    f = [-(sympy.diff((lam_e + mu_e) * div, X[k]) + sum(sympy.diff(mu_e * sympy.diff(u[k], X[j]), X[j])
                                                      for j in range(3))) - om ** 2 * rho_e * u[k]
         for k in range(3)]
    F = [sympy.lambdify(X, e, "numpy") for e in f]
    U = [sympy.lambdify(X, e, "numpy") for e in u]
    Cf = [sympy.lambdify(X, e, "numpy") for e in (lam_e, mu_e, rho_e)]
    errs = []
    for n in (8, 16, 32):
        h = 1.0 / n
        shape = (n, n, n)
        zc, yc, xc = np.meshgrid(*[(np.arange(n) + 0.5) * h] * 3, indexing="ij")
        lam, mu, rho = [np.broadcast_to(c(xc, yc, zc), shape).astype(float) for c in Cf]
        He = op.assemble_displacement(op.Parts(lam, mu, rho, np.zeros(shape), om, h)).real.tocsr()
        fs = np.zeros((4,) + shape)
        us = np.zeros((4,) + shape)
        for k in range(3):
            Xk, Yk, Zk = _face_positions(shape, k, h)
            fs[k] = F[k](Xk, Yk, Zk)
            us[k] = U[k](Xk, Yk, Zk)
        fv = op.slots_to_dofs(fs, shape)[:He.shape[0]].real
        ue = op.slots_to_dofs(us, shape)[:He.shape[0]].real
        uh, info = spla.cg(He, fv, rtol=1e-12, maxiter=20000)   # SPD at this omega
        assert info == 0
        errs.append(np.sqrt(np.mean((uh - ue) ** 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert abs(orders[-1] - 2.0) < 0.2, (errs, orders)
