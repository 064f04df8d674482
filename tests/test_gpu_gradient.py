"""Adjoint-state gradient through the C ABI and torch.autograd.

* ehs_gradient against the oracle's -Re(w^H dK/dm x) on the same x and w
  (both FP64; 1e-10 relative, element-wise over every cell);
* the autograd Function (forward solve, adjoint solve, fused gradient) against
  central finite differences of a receiver misfit (step 1e-6 relative,
  complex128 solves at 1e-11), 2 media x 2 sources.
"""
import numpy as np
import pytest

from oracle import gradient as og, operators as op
from paper_1806_11277_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _meds(n=32):
    return [synth.random_2d(n=n, sigma=s, seed=i + 5, corr=4.0, abl=6) for i, s in enumerate((0.3, 0.45))]


def test_gradient_kernel_matches_oracle():
    from paper_1806_11277_gb300 import ehs
    meds = _meds(32)
    S = ehs.solver_for(meds, levels=3, prec=ehs.EHS_C128, nrhs=2, tol=1e-10)
    rng = np.random.default_rng(1)
    shape = meds[0].shape
    x = rng.standard_normal((4, 3) + shape) + 1j * rng.standard_normal((4, 3) + shape)
    w = rng.standard_normal((4, 3) + shape) + 1j * rng.standard_normal((4, 3) + shape)
    for v in (x, w):
        v[:, 0, :, 0] = 0
        v[:, 1, 0, :] = 0
    xd, wd = torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda()
    gl, gm, gr = [t.cpu().numpy() for t in S.gradient(xd, wd)]
    for m, med in enumerate(meds):
        parts = op.parts_for(med)
        acc = [np.zeros(shape) for _ in range(3)]
        for r in range(2):
            b = m * 2 + r
            go = og.gradient(parts, op.slots_to_dofs(x[b], shape), op.slots_to_dofs(w[b], shape))
            for a, g in zip(acc, go):
                a += g
        for got, want in zip((gl[m], gm[m], gr[m]), acc):
            assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    S.close()


def test_gradient_kernel_matches_oracle_3d():
    """The 3D instance of the fused gradient (two tangential directions per
    face) against the oracle's formula, one medium with two right-hand sides."""
    from paper_1806_11277_gb300 import ehs
    med = synth.layered_3d(n=8, seed=3, corr=2.0, abl=2)
    S = ehs.solver_for([med], levels=2, prec=ehs.EHS_C128, nrhs=2, tol=1e-10)
    shape = med.shape
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 4) + shape) + 1j * rng.standard_normal((2, 4) + shape)
    w = rng.standard_normal((2, 4) + shape) + 1j * rng.standard_normal((2, 4) + shape)
    for v in (x, w):                     # boundary slots: u_k at i_k = 0
        v[:, 0, :, :, 0] = 0
        v[:, 1, :, 0, :] = 0
        v[:, 2, 0, :, :] = 0
    gl, gm, gr = [t.cpu().numpy() for t in S.gradient(torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda())]
    parts = op.parts_for(med)
    acc = [np.zeros(shape) for _ in range(3)]
    for r in range(2):
        go = og.gradient(parts, op.slots_to_dofs(x[r], shape), op.slots_to_dofs(w[r], shape))
        for a, g in zip(acc, go):
            a += g
    for got, want in zip((gl[0], gm[0], gr[0]), acc):
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    S.close()


def test_autograd_matches_finite_differences():
    from paper_1806_11277_gb300 import autograd as ag
    meds = _meds(32)
    shape = meds[0].shape
    lam = torch.tensor(np.stack([m.lam for m in meds]), dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(np.stack([m.mu for m in meds]), dtype=torch.float64, requires_grad=True)
    rho = torch.tensor(np.stack([m.rho for m in meds]), dtype=torch.float64, requires_grad=True)
    omegas = [m.omega for m in meds]
    q = np.zeros((4, 3) + shape, dtype=np.complex128)
    for b in range(4):
        q[b, 0, 8, 10 + 6 * (b % 2)] = 1.0                     # two x-forces per medium
    qd = torch.from_numpy(q).cuda()
    rec = (slice(None), 0, 9, slice(6, 26, 2))                  # a line of u_x receivers
    rng = np.random.default_rng(2)
    d = torch.from_numpy(1e-3 * (rng.standard_normal((4, 10)) + 1j * rng.standard_normal((4, 10)))).cuda()
    kw = dict(levels=3, prec=0, nrhs=2, tol=1e-11, maxit=400)

    def misfit(l, m_, r_):
        x = ag.solve(l, m_, r_, qd, omegas, 1.0, 6, **kw)
        res = x[rec] - d
        return 0.5 * (res.real ** 2 + res.imag ** 2).sum()

    J = misfit(lam, mu, rho)
    J.backward()
    for name, t in (("lam", lam), ("mu", mu), ("rho", rho)):
        for cell in ((0, 10, 12), (1, 16, 16), (0, 20, 9)):
            base = t.detach().clone()
            eps = 1e-6 * float(base[cell].abs())
            vals = []
            for sgn in (1, -1):
                pert = base.clone()
                pert[cell] += sgn * eps
                args = {"lam": lam.detach(), "mu": mu.detach(), "rho": rho.detach()}
                args[name] = pert
                with torch.no_grad():
                    vals.append(float(misfit(args["lam"], args["mu"], args["rho"])))
            fd = (vals[0] - vals[1]) / (2 * eps)
            g = float(t.grad[cell])
            scale = float(t.grad.abs().max())
            assert abs(fd - g) <= 2e-4 * scale, (name, cell, fd, g, scale)


def test_autograd_backward_twice_and_release():
    """backward with retain_graph=True may run twice (the solver context lives
    with the graph): the second pass adds the same gradient again; the context
    is released with the graph."""
    import gc
    import weakref
    from paper_1806_11277_gb300 import autograd as ag
    meds = _meds(32)[:1]
    shape = meds[0].shape
    lam = torch.tensor(meds[0].lam[None], dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(meds[0].mu[None], dtype=torch.float64, requires_grad=True)
    rho = torch.tensor(meds[0].rho[None], dtype=torch.float64, requires_grad=True)
    q = np.zeros((1, 3) + shape, dtype=np.complex128)
    q[0, 0, 8, 16] = 1.0
    qd = torch.from_numpy(q).cuda()
    x = ag.solve(lam, mu, rho, qd, [meds[0].omega], 1.0, 6, levels=3, prec=0)
    J = (x[0, 0, 9, 6:26].abs() ** 2).sum()
    J.backward(retain_graph=True)
    g1 = [t.grad.clone() for t in (lam, mu, rho)]
    J.backward()
    for t, g in zip((lam, mu, rho), g1):
        assert torch.allclose(t.grad, 2 * g, rtol=1e-9, atol=1e-12 * float(g.abs().max()))
    S_ref = weakref.ref(x.grad_fn.S) if hasattr(x.grad_fn, "S") else None
    del x, J
    gc.collect()
    if S_ref is not None:
        assert S_ref() is None
