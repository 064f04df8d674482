"""Allocation-free fine-level smoothing through the C ABI.

ehs_fine_smooth_noalloc serves callers that may not allocate device memory
when they relax a vector -- a host program that gave all of the device memory
to its own pool at start-up and forbids its libraries to call cudaMalloc, or a
latency-bound loop that must not stall on the allocator -- and so cannot
build a context.  Its result must equal ehs_smooth on level 0 of a context
built from the same problem; two calls in a row check that the shared static
scratch left by one call does not leak into the next, and the device's free
memory must not change across a call.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1806_11277_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(ehs, meds, lam, mu, rho, omegas):
    p = ehs.Problem()
    shape = meds[0].shape
    p.dim = len(shape)
    n = list(reversed(shape)) + [1] * (3 - len(shape))
    for k in range(3):
        p.n[k] = n[k]
    p.h = meds[0].h
    p.omega = float(omegas[0])
    p.omegas = omegas.ctypes.data
    p.nmedia = len(meds)
    p.lam, p.mu, p.rho = lam.data_ptr(), mu.data_ptr(), rho.data_ptr()
    p.abl_cells = meds[0].abl_cells
    p.abl_max = 1.0
    p.gamma_add = 0.01 * np.pi
    return p


def _slots(shape, items, seed):
    rng = np.random.default_rng(seed)
    d = len(shape)
    v = rng.standard_normal((items, d + 1) + shape) + 1j * rng.standard_normal((items, d + 1) + shape)
    v[:, 0, ..., 0] = 0                       # u_x boundary slots
    if d == 2:
        v[:, 1, 0, :] = 0                     # u_y boundary slots
    else:
        v[:, 1, :, 0, :] = 0
        v[:, 2, 0, :, :] = 0
    return v


@pytest.mark.parametrize("prec_name", ["c128", "c64"])
def test_noalloc_smooth_matches_context_smooth(prec_name):
    from paper_1806_11277_gb300 import ehs
    lib = ehs.load()
    prec = ehs.EHS_C128 if prec_name == "c128" else ehs.EHS_C64
    dt = torch.complex128 if prec_name == "c128" else torch.complex64
    tol = 1e-12 if prec_name == "c128" else 1e-6
    meds = [synth.random_2d(n=64, sigma=s, seed=i, corr=6.0, abl=8) for i, s in enumerate((0.3, 0.45))]
    alpha, w = 0.2, 0.75
    S = ehs.solver_for(meds, levels=3, alpha=alpha, w=[w, 0.5])
    lam = torch.from_numpy(np.stack([m.lam for m in meds])).cuda()
    mu = torch.from_numpy(np.stack([m.mu for m in meds])).cuda()
    rho = torch.from_numpy(np.stack([m.rho for m in meds])).cuda()
    omegas = np.array([m.omega for m in meds])
    prob = _problem(ehs, meds, lam, mu, rho, omegas)
    for call, seed in enumerate((11, 12)):           # two calls in a row
        b = torch.from_numpy(_slots(meds[0].shape, 2, seed)).to("cuda", dt)
        x0 = torch.from_numpy(_slots(meds[0].shape, 2, seed + 100)).to("cuda", dt)
        x_ref = x0.clone()
        S.smooth(b, x_ref, level=0, nsweeps=2)
        x_new = x0.clone()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = lib.ehs_fine_smooth_noalloc(C.byref(prob), 1, alpha, w, w, 2, prec,
                                         C.c_void_p(b.data_ptr()), C.c_void_p(x_new.data_ptr()), None)
        torch.cuda.synchronize()
        assert st == 0, (call, st)
        if call:                                     # the first call loaded the kernels
            assert torch.cuda.mem_get_info()[0] == free0, (call, free0, torch.cuda.mem_get_info()[0])
        err = (torch.abs(x_new - x_ref).max() / torch.abs(x_ref).max()).item()
        assert err <= tol, (call, err)
        assert torch.abs(x_new - x0).max().item() > 0      # it did relax
    S.close()


def test_noalloc_rejects_oversize_and_host_pointers():
    from paper_1806_11277_gb300 import ehs
    lib = ehs.load()
    med = synth.homogeneous_2d(n=1024, abl=10)
    lam = torch.from_numpy(med.lam[None]).cuda()
    mu = torch.from_numpy(med.mu[None]).cuda()
    rho = torch.from_numpy(med.rho[None]).cuda()
    omegas = np.array([med.omega])
    prob = _problem(ehs, [med], lam, mu, rho, omegas)
    b = torch.zeros((1, 3, 1024, 1024), dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(b)
    st = lib.ehs_fine_smooth_noalloc(C.byref(prob), 1, 0.2, 0.75, 0.75, 1, ehs.EHS_C128,
                                     C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), None)
    assert st == 3                                   # EHS_ERR_OOM: beyond the 32 MiB scratch
    xh = np.zeros((1, 3, 1024, 1024), dtype=np.complex128)
    st = lib.ehs_fine_smooth_noalloc(C.byref(prob), 1, 0.2, 0.75, 0.75, 1, ehs.EHS_C128,
                                     C.c_void_p(b.data_ptr()), C.c_void_p(xh.ctypes.data), None)
    assert st == 1                                   # EHS_ERR_ARG: host pointer
    small = synth.homogeneous_2d(n=32, abl=4)
    lam = torch.from_numpy(small.lam[None]).cuda()
    mu = torch.from_numpy(small.mu[None]).cuda()
    rho = torch.from_numpy(small.rho[None]).cuda()
    prob = _problem(ehs, [small], lam, mu, rho, np.array([small.omega]))
    prob.abl_cells = 17                              # wider than half the grid
    b = torch.zeros((1, 3, 32, 32), dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(b)
    st = lib.ehs_fine_smooth_noalloc(C.byref(prob), 1, 0.2, 0.75, 0.75, 1, ehs.EHS_C128,
                                     C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), None)
    assert st == 1                                   # EHS_ERR_ARG: absorbing layer out of range
