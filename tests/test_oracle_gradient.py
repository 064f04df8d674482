"""Pin of the oracle's adjoint-state gradient: central finite differences of a
receiver misfit J(m) = 1/2 sum_r |u(r) - d_r|^2 with exact sparse solves."""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import gradient as og, operators as op
from paper_1806_11277_gb300 import synth


def _misfit(lam, mu, rho, gamma, omega, q, rec, d):
    parts = op.Parts(lam, mu, rho, gamma, omega, 1.0)
    K = op.assemble_mixed(parts)
    x = spla.spsolve(K.tocsc(), q)
    r = x[rec] - d
    return 0.5 * np.real(np.vdot(r, r)), x, parts, K


def test_gradient_matches_central_differences():
    med = synth.random_2d(n=16, sigma=0.4, seed=4, corr=3.0, abl=3)
    gamma = op.gamma_profile(med.shape, med.omega, med.abl_cells)
    q = op.slots_to_dofs(synth.point_rhs(med.shape, med.sources)[0], med.shape)
    nu1 = op.dof_sizes(med.shape)[0]
    rec = np.arange(20, nu1, 7)                 # receivers: a set of u_1 faces
    rng = np.random.default_rng(0)
    d = rng.standard_normal(rec.size) * 1e-2 + 1j * rng.standard_normal(rec.size) * 1e-2
    J0, x, parts, K = _misfit(med.lam, med.mu, med.rho, gamma, med.omega, q, rec, d)
    e = np.zeros_like(x)
    e[rec] = x[rec] - d
    w = spla.spsolve(K.conj().T.tocsc(), e)
    g = og.gradient(parts, x, w)
    for name, gi in zip(("lam", "mu", "rho"), g):
        for cell in ((5, 7), (8, 8), (3, 12), (10, 2)):
            m = {"lam": med.lam.copy(), "mu": med.mu.copy(), "rho": med.rho.copy()}
            base = m[name][cell]
            eps = 1e-6 * abs(base)
            m[name][cell] = base + eps
            Jp = _misfit(m["lam"], m["mu"], m["rho"], gamma, med.omega, q, rec, d)[0]
            m[name][cell] = base - eps
            Jm = _misfit(m["lam"], m["mu"], m["rho"], gamma, med.omega, q, rec, d)[0]
            fd = (Jp - Jm) / (2 * eps)
            assert abs(fd - gi[cell]) <= 1e-5 * np.abs(gi).max(), (name, cell, fd, gi[cell])


def test_gradient_matches_central_differences_3d():
    """The same pin in 3D (two tangential directions per face, clamped edge
    averages at the boundary), including boundary and corner cells."""
    med = synth.layered_3d(n=8, seed=3, corr=2.0, abl=2)
    gamma = op.gamma_profile(med.shape, med.omega, med.abl_cells)
    q = op.slots_to_dofs(synth.point_rhs(med.shape, med.sources)[0], med.shape)
    nu1 = op.dof_sizes(med.shape)[0]
    rec = np.arange(5, nu1, 11)
    rng = np.random.default_rng(1)
    d = rng.standard_normal(rec.size) * 1e-2 + 1j * rng.standard_normal(rec.size) * 1e-2
    J0, x, parts, K = _misfit(med.lam, med.mu, med.rho, gamma, med.omega, q, rec, d)
    e = np.zeros_like(x)
    e[rec] = x[rec] - d
    w = spla.spsolve(K.conj().T.tocsc(), e)
    g = og.gradient(parts, x, w)
    for name, gi in zip(("lam", "mu", "rho"), g):
        for cell in ((4, 3, 5), (0, 0, 0), (7, 2, 7), (2, 7, 0)):
            m = {"lam": med.lam.copy(), "mu": med.mu.copy(), "rho": med.rho.copy()}
            base = m[name][cell]
            eps = 1e-6 * abs(base)
            m[name][cell] = base + eps
            Jp = _misfit(m["lam"], m["mu"], m["rho"], gamma, med.omega, q, rec, d)[0]
            m[name][cell] = base - eps
            Jm = _misfit(m["lam"], m["mu"], m["rho"], gamma, med.omega, q, rec, d)[0]
            fd = (Jp - Jm) / (2 * eps)
            assert abs(fd - gi[cell]) <= 1e-5 * np.abs(gi).max(), (name, cell, fd, gi[cell])
