"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Every comparison is element-wise: max_i |got_i - ref_i| / max_i |ref_i| over
the whole vector (boundary faces, absorbing layer and subdomain overlaps
included), so an error confined to a few rows is not diluted by the norm of
the rest.  Tolerances:
* operator apply: 1e-12 in complex128, 1e-5 in complex64;
* one relaxation sweep / one cycle: 1e-11 in complex128 (a few operator
  applications deep), 1e-5 in complex64;
* FGMRES: same iteration count as the oracle with the complex128
  preconditioner (+-1 with complex64), true residual <= 1e-6 and solution
  within 1e-5 of the oracle's solution.
Grids span several multigrid tiles, odd numbers of interior faces and
absorbing layers; 2D and 3D; batches of media and of right-hand sides.
"""
import numpy as np
import pytest

from oracle import dd as odd, krylov, multigrid as mg, operators as op
from paper_1806_11277_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ehs():
    from paper_1806_11277_gb300 import ehs
    return ehs


def _rand_slots(shape, items, seed, dtype=np.complex128):
    rng = np.random.default_rng(seed)
    d = len(shape)
    v = rng.standard_normal((items, d + 1) + shape) + 1j * rng.standard_normal((items, d + 1) + shape)
    for k in range(d):                           # Dirichlet slots are zero
        sl = [slice(None)] * (d + 2)
        sl[0] = slice(None); sl[1] = k; sl[2 + d - 1 - k] = 0
        v[tuple(sl)] = 0
    return v.astype(dtype)


def _media_2d(n=64, nmed=2):
    return [synth.random_2d(n=n, sigma=s, seed=i, corr=6.0, abl=8) for i, s in
            zip(range(nmed), (0.3, 0.49, 0.45, 0.4))]


def _media_3d(n=16, nmed=1):
    return [synth.layered_3d(n=n, seed=i, corr=3.0, abl=3) for i in range(nmed)]


def _err(a, b):
    """Element-wise error of a against the reference b: max |a - b| / max |b|."""
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.abs(a - b).max() / np.abs(b).max())


def _oracle_parts(med, alpha=0.0):
    return op.assemble_mixed(op.parts_for(med), alpha)


@pytest.mark.parametrize("case", ["2d", "3d"])
@pytest.mark.parametrize("shifted", [False, True])
def test_op_apply_fine(case, shifted):
    ehs = _ehs()
    meds = _media_2d(48, 2) if case == "2d" else _media_3d(16, 1)
    S = ehs.solver_for(meds, levels=3, alpha=0.2)
    shape = meds[0].shape
    x = _rand_slots(shape, S.items, 1)
    for prec, dt, tol in ((ehs.EHS_C128, torch.complex128, 1e-12), (ehs.EHS_C64, torch.complex64, 1e-5)):
        xd = torch.from_numpy(x).to("cuda", dt)
        yd = torch.zeros_like(xd)
        S.op_apply(xd, yd, level=0, shifted=shifted)
        y = yd.cpu().numpy()
        for b, med in enumerate(meds):
            K = _oracle_parts(med, 0.2 if shifted else 0.0)
            xe = op.slots_to_dofs(xd[b].cpu().numpy().astype(np.complex128), shape)
            ye = op.dofs_to_slots(K @ xe, shape)
            assert _err(y[b], ye) <= tol, (prec, b, _err(y[b], ye))
    S.close()


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_galerkin_levels_match_oracle(case):
    ehs = _ehs()
    meds = _media_2d(64, 2) if case == "2d" else _media_3d(16, 1)
    levels = 3
    S = ehs.solver_for(meds, levels=levels, alpha=0.2)
    for b, med in enumerate(meds):
        H = mg.Hierarchy(_oracle_parts(med, 0.2), med.shape, levels)
        for l in range(1, levels):
            shp = S.level_shape(l)
            x = _rand_slots(tuple(shp[2:]), S.items, 10 + l)
            for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5)):
                xd = torch.from_numpy(x).to("cuda", dt)
                yd = torch.zeros_like(xd)
                S.op_apply(xd, yd, level=l)
                xe = op.slots_to_dofs(xd[b].cpu().numpy().astype(np.complex128), tuple(shp[2:]))
                ye = op.dofs_to_slots(H.K[l] @ xe, tuple(shp[2:]))
                assert _err(yd[b].cpu().numpy(), ye) <= tol, (l, dt, _err(yd[b].cpu().numpy(), ye))
    S.close()


@pytest.mark.parametrize("case,nsweeps,rows,half", [("2d", 1, None, 0), ("3d", 1, None, 0), ("2d", 2, None, 0),
                                                    ("2d", 3, None, 0), ("2d", 1, 0, 1), ("2d", 1, 1, 1),
                                                    ("2d", 1, 3, 0), ("3d", 1, 1, 0)])
def test_smooth_matches_oracle(case, nsweeps, rows, half, monkeypatch):
    """nsweeps red-black sweeps of every smoothed level (2D complex64 level 0:
    the fused whole-sweep kernel, ping-ponging between x and the level's
    scratch).  rows: a fixed residual-pass launch shape on the Galerkin levels
    (0: one cell per thread; 1, 3: two cells per thread); half: FP16 Galerkin
    tables (stored half in 2D), against the oracle's exact operator."""
    ehs = _ehs()
    if rows is not None:
        monkeypatch.setenv("EHS_ROWS_VARIANT", str(rows))
    meds = _media_2d(32, 2) if case == "2d" else _media_3d(16, 1)
    levels = 3
    S = ehs.solver_for(meds, levels=levels, alpha=0.2, coef_half=half)
    for l in range(levels - 1):
        shp = S.level_shape(l)
        gshape = tuple(shp[2:])
        b_ = _rand_slots(gshape, S.items, 20 + l)
        x_ = _rand_slots(gshape, S.items, 30 + l)
        for dt, tol in ((torch.complex128, 1e-11), (torch.complex64, 2e-5 if not half or l == 0 else 2e-3)):
            bd = torch.from_numpy(b_).to("cuda", dt)
            xd = torch.from_numpy(x_).to("cuda", dt)
            S.smooth(bd, xd, level=l, nsweeps=nsweeps)
            for it, med in enumerate(meds):
                H = mg.Hierarchy(_oracle_parts(med, 0.2), med.shape, levels)
                be = op.slots_to_dofs(bd[it].cpu().numpy().astype(np.complex128), gshape)
                xe = op.slots_to_dofs(torch.from_numpy(x_[it]).to(dt).numpy().astype(np.complex128), gshape)
                for _ in range(nsweeps):
                    xe = H.relax(l, be, xe)
                xr = op.dofs_to_slots(xe, gshape)
                got = xd[it].cpu().numpy()
                assert _err(got, xr) <= tol, (l, dt, it, _err(got, xr))
    S.close()


@pytest.mark.parametrize("case,levels,n,nu,unfused", [("2d", 3, 64, 1, 0), ("2d", 4, 64, 1, 0), ("3d", 3, 16, 1, 0),
                                                     ("2d", 3, 64, 1, 1), ("2d", 3, 48, 1, 0), ("2d", 3, 64, 2, 0),
                                                     ("2d", 3, 64, 3, 0)])
def test_vcycle_matches_oracle(case, levels, n, nu, unfused, monkeypatch):
    """One V(nu, nu) cycle.  In 2D complex64 the fine level runs the fused
    kernels (whole red-black sweeps, residual + restriction in one pass,
    prolongation folded into the first post-smoothing sweep) when the grid
    splits into their tiles (64 x 64); 48 x 48 and EHS_FINE_UNFUSED=1 run the
    per-colour kernels and the separate transfers."""
    ehs = _ehs()
    if unfused:
        monkeypatch.setenv("EHS_FINE_UNFUSED", "1")
    meds = _media_2d(n, 2) if case == "2d" else _media_3d(n, 1)
    S = ehs.solver_for(meds, levels=levels, alpha=0.2, nu_pre=nu, nu_post=nu)
    shape = meds[0].shape
    b_ = _rand_slots(shape, S.items, 5)
    for dt, tol in ((torch.complex128, 1e-10), (torch.complex64, 5e-5)):
        bd = torch.from_numpy(b_).to("cuda", dt)
        xd = torch.full_like(bd, 7.0)                # the cycle ignores the input of x
        S.vcycle(bd, xd)
        for it, med in enumerate(meds):
            H = mg.Hierarchy(_oracle_parts(med, 0.2), med.shape, levels,
                             w=[0.75, 0.5, 0.25, 0.25, 0.25][:levels - 1])
            xr = op.dofs_to_slots(H.cycle(op.slots_to_dofs(b_[it], shape), nu1=nu, nu2=nu), shape)
            assert _err(xd[it].cpu().numpy(), xr) <= tol, (dt, it, _err(xd[it].cpu().numpy(), xr))
    S.close()


@pytest.mark.parametrize("n,unfused", [(64, 0), (64, 1), (48, 0)])
def test_transfers_match_oracle(n, unfused, monkeypatch):
    """ehs_residual_restrict (P^T (b - K_l x), Algorithm TwoCycle step 2) and
    ehs_prolong_add (x + P e_c, step 4) on every level pair against the
    oracle's assembled K_l and P_l; 2D complex64 level 0 of a 64 x 64 grid runs
    the fused residual + restriction kernel, 48 x 48 or EHS_FINE_UNFUSED=1 the
    residual pass and the separate restriction.  Also 3D (16^3)."""
    ehs = _ehs()
    if unfused:
        monkeypatch.setenv("EHS_FINE_UNFUSED", "1")
    for meds in (_media_2d(n, 2), _media_3d(16, 1)):
        S = ehs.solver_for(meds, levels=3, alpha=0.2)
        for l in range(2):
            fs, cs = tuple(S.level_shape(l)[2:]), tuple(S.level_shape(l + 1)[2:])
            b_ = _rand_slots(fs, S.items, 60 + l)
            x_ = _rand_slots(fs, S.items, 70 + l)
            e_ = _rand_slots(cs, S.items, 80 + l)
            for dt, npt, tol in ((torch.complex128, np.complex128, 1e-12), (torch.complex64, np.complex64, 1e-5)):
                bd = torch.from_numpy(b_).to("cuda", dt)
                xd = torch.from_numpy(x_).to("cuda", dt)
                ed = torch.from_numpy(e_).to("cuda", dt)
                rc = torch.full((S.items, len(fs) + 1) + cs, 3.0, dtype=dt, device="cuda")
                S.residual_restrict(bd, xd, rc, level=l)
                S.prolong_add(ed, xd, level=l)
                for it, med in enumerate(meds):
                    H = mg.Hierarchy(_oracle_parts(med, 0.2), med.shape, 3)
                    xe = op.slots_to_dofs(x_[it].astype(npt).astype(np.complex128), fs)
                    be = op.slots_to_dofs(b_[it].astype(npt).astype(np.complex128), fs)
                    ee = op.slots_to_dofs(e_[it].astype(npt).astype(np.complex128), cs)
                    rr = op.dofs_to_slots(H.P[l].T @ (be - H.K[l] @ xe), cs)
                    xr = op.dofs_to_slots(xe + H.P[l] @ ee, fs)
                    assert _err(rc[it].cpu().numpy(), rr) <= tol, (n, l, dt, it, _err(rc[it].cpu().numpy(), rr))
                    assert _err(xd[it].cpu().numpy(), xr) <= tol, (n, l, dt, it, _err(xd[it].cpu().numpy(), xr))
        S.close()


def _solve_both(meds, levels, prec, nrhs=1, host=False, **kw):
    ehs = _ehs()
    S = ehs.solver_for(meds, levels=levels, prec=prec, nrhs=nrhs, **kw)
    shape = meds[0].shape
    qs = []
    for med in meds:
        srcs = med.sources * nrhs if len(med.sources) < nrhs else med.sources[:nrhs]
        for r in range(nrhs):
            k, idx = srcs[r]
            idx = tuple(i + r for i in idx)
            qs.append(synth.point_rhs(shape, [(k, idx)])[0])
    q = np.stack(qs)
    if host:
        u = np.zeros_like(q)
        info = S.fgmres_solve(q, u)
    else:
        qd = torch.from_numpy(q).cuda()
        ud = torch.zeros_like(qd)
        info = S.fgmres_solve(qd, ud)
        u = ud.cpu().numpy()
    S.close()
    return q, u, info


@pytest.mark.parametrize("prec_name,ortho,restart", [("c128", 0, 10), ("c64", 0, 10), ("c64", 1, 10), ("c64", 1, 3)])
def test_fgmres_matches_oracle_2d(prec_name, ortho, restart):
    """Four media in one batch against the oracle's FGMRES(restart); the double-float
    solve with CGS2 (ortho 0) or delayed CGS2 (ortho 1), which the oracle's CGS2
    equals in exact arithmetic; restart 3 runs several restart cycles."""
    ehs = _ehs()
    prec = ehs.EHS_C128 if prec_name == "c128" else ehs.EHS_C64
    meds = _media_2d(64, 4)
    q, u, info = _solve_both(meds, 3, prec, ortho=ortho, restart=restart)
    for it, med in enumerate(meds):
        K = _oracle_parts(med)
        H = mg.Hierarchy(_oracle_parts(med, 0.2), med.shape, 3)
        qo = op.slots_to_dofs(q[it], med.shape)
        xo, io = krylov.fgmres(lambda v: K @ v, H.cycle, qo, m=restart)
        ug = op.slots_to_dofs(u[it], med.shape)
        res = np.linalg.norm(qo - K @ ug) / np.linalg.norm(qo)
        assert info[it]["converged"] and res <= 1e-6
        if prec == ehs.EHS_C128:
            assert info[it]["iters"] == io["iters"], (info[it], io["iters"])
        else:
            assert abs(info[it]["iters"] - io["iters"]) <= 1, (info[it], io["iters"])
        assert _err(ug, xo) <= 1e-5


def test_fgmres_config1_host_buffers():
    """64 x 64 homogeneous Vp=2, Vs=1, 3 levels, alpha 0.2, FGMRES(10); host q/u."""
    ehs = _ehs()
    med = synth.homogeneous_2d()
    q, u, info = _solve_both([med], 3, ehs.EHS_C128, host=True)
    K = _oracle_parts(med)
    H = mg.Hierarchy(_oracle_parts(med, 0.2), med.shape, 3)
    qo = op.slots_to_dofs(q[0], med.shape)
    xo, io = krylov.fgmres(lambda v: K @ v, H.cycle, qo, m=10)
    import scipy.sparse.linalg as spla
    xe = spla.spsolve(K.tocsc(), qo)
    ug = op.slots_to_dofs(u[0], med.shape)
    assert info[0]["iters"] == io["iters"]
    assert _err(ug, xo) <= 1e-5
    assert _err(ug, xe) <= 1e-5


@pytest.mark.parametrize("ortho", [0, 1])
def test_fgmres_multi_rhs_3d(ortho):
    """Two sources of one 3D medium in one batch (complex64 cycle; CGS2 or delayed
    CGS2): each source's iteration count within 1 of the oracle's, its true
    residual <= 1e-6 and its solution within 1e-5 of the oracle's, element by
    element."""
    ehs = _ehs()
    meds = _media_3d(16, 1)
    q, u, info = _solve_both(meds, 3, ehs.EHS_C64, nrhs=2, ortho=ortho)
    K = _oracle_parts(meds[0])
    H = mg.Hierarchy(_oracle_parts(meds[0], 0.2), meds[0].shape, 3)
    for it in range(2):
        qo = op.slots_to_dofs(q[it], meds[0].shape)
        ug = op.slots_to_dofs(u[it], meds[0].shape)
        xo, io = krylov.fgmres(lambda v: K @ v, H.cycle, qo, m=10)
        assert np.linalg.norm(qo - K @ ug) / np.linalg.norm(qo) <= 1e-6
        assert info[it]["converged"]
        assert abs(info[it]["iters"] - io["iters"]) <= 1, (it, info[it], io["iters"])
        assert _err(ug, xo) <= 1e-5, (it, _err(ug, xo))


@pytest.mark.parametrize("ortho", [0, 1])
def test_fgmres_zero_rhs_item(ortho):
    """A zero right-hand side in a batch (the degenerate case of the solve): that item takes
    no iteration and returns u = 0 with relative residual 0 (the convention for q = 0), while
    the other item of the batch is solved as the oracle solves it alone."""
    ehs = _ehs()
    meds = _media_2d(64, 2)
    q = np.stack([synth.point_rhs(m.shape, m.sources)[0] for m in meds])
    q[0] = 0
    S = ehs.solver_for(meds, levels=3, prec=ehs.EHS_C64, ortho=ortho)
    qd = torch.from_numpy(q).cuda()
    ud = torch.ones_like(qd)                      # the solve starts from zero whatever u holds
    info = S.fgmres_solve(qd, ud)
    u = ud.cpu().numpy()
    S.close()
    assert info[0]["iters"] == 0 and info[0]["converged"] and info[0]["relres"] == 0.0
    assert not np.any(u[0])
    med = meds[1]
    K = _oracle_parts(med)
    H = mg.Hierarchy(_oracle_parts(med, 0.2), med.shape, 3)
    qo = op.slots_to_dofs(q[1], med.shape)
    xo, io = krylov.fgmres(lambda v: K @ v, H.cycle, qo, m=10)
    ug = op.slots_to_dofs(u[1], med.shape)
    assert info[1]["converged"] and abs(info[1]["iters"] - io["iters"]) <= 1, (info[1], io["iters"])
    assert _err(ug, xo) <= 1e-5


def test_adjoint_solve():
    ehs = _ehs()
    med = _media_2d(32, 1)[0]
    S = ehs.solver_for(med, levels=3, prec=ehs.EHS_C64)
    g = _rand_slots(med.shape, 1, 7)
    gd = torch.from_numpy(g).cuda()
    wd = torch.zeros_like(gd)
    info = S.adjoint_solve(gd, wd)[0]
    K = _oracle_parts(med)
    go = op.slots_to_dofs(g[0], med.shape)
    wo = op.slots_to_dofs(wd[0].cpu().numpy(), med.shape)
    assert info["converged"]
    assert np.linalg.norm(K.conj().T @ wo - go) / np.linalg.norm(go) <= 1e-6
    S.close()


@pytest.mark.parametrize("prec_name", ["c128", "c64"])
def test_dd_precond_matches_oracle(prec_name):
    ehs = _ehs()
    prec = ehs.EHS_C128 if prec_name == "c128" else ehs.EHS_C64
    tol = 1e-10 if prec == ehs.EHS_C128 else 5e-5
    med = synth.random_2d(n=64, sigma=0.4, seed=2, corr=6.0, abl=8)
    S = ehs.solver_for(med, levels=3, precond=ehs.EHS_PRECOND_DD, dd=(2, 2, 1), dd_overlap=4,
                       dd_pad=8, prec=prec)
    D = odd.DD(med, (2, 2), 4, 8, 3, 0.2)
    r = _rand_slots(med.shape, 1, 9)
    rd = torch.from_numpy(r).cuda()
    zd = torch.zeros_like(rd)
    S.dd_precond(rd, zd, prec=prec)
    zo = op.dofs_to_slots(D.apply(op.slots_to_dofs(r[0], med.shape)), med.shape)
    assert _err(zd[0].cpu().numpy(), zo) <= tol
    S.close()


def test_dd_fgmres_iterations_match_oracle():
    ehs = _ehs()
    med = synth.homogeneous_2d()
    q, u, info = _solve_both([med], 3, ehs.EHS_C128, precond=ehs.EHS_PRECOND_DD, dd=(2, 2, 1),
                             dd_overlap=4, dd_pad=8)
    D = odd.DD(med, (2, 2), 4, 8, 3, 0.2)
    qo = op.slots_to_dofs(q[0], med.shape)
    xo, io = krylov.fgmres(lambda v: D.K @ v, D.apply, qo, m=10)
    ug = op.slots_to_dofs(u[0], med.shape)
    assert info[0]["iters"] == io["iters"]
    assert _err(ug, xo) <= 1e-5


def test_invalid_arguments_rejected():
    ehs = _ehs()
    med = synth.homogeneous_2d(n=36)
    with pytest.raises(ehs.EhsError, match="ERR_ARG"):
        ehs.solver_for(med, levels=4)              # 36 not divisible by 8
    bad = synth.homogeneous_2d(n=32)
    bad.rho[3, 3] = -1.0
    with pytest.raises(ehs.EhsError, match="ERR_ARG"):
        ehs.solver_for(bad, levels=3)
    bad = synth.homogeneous_2d(n=32)
    bad.lam[1, 1] = np.nan
    with pytest.raises(ehs.EhsError, match="ERR_ARG"):
        ehs.solver_for(bad, levels=3)


@pytest.mark.parametrize("ortho", [0, 1])
def test_noconv_reports_best_iterate(ortho):
    ehs = _ehs()
    med = synth.homogeneous_2d()
    S = ehs.solver_for(med, levels=3, maxit=3, ortho=ortho)
    q = synth.point_rhs(med.shape, med.sources)[0][None]
    qd = torch.from_numpy(q).cuda()
    ud = torch.zeros_like(qd)
    info = S.fgmres_solve(qd, ud, raise_noconv=False)[0]
    assert info["iters"] == 3 and not info["converged"]
    assert 0 < info["relres"] < 1
    S.close()


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_wcycle_matches_oracle(case):
    ehs = _ehs()
    meds = _media_2d(64, 2) if case == "2d" else _media_3d(16, 1)
    levels = 4 if case == "2d" else 3
    S = ehs.solver_for(meds, levels=levels, alpha=0.4, cycle=2)
    shape = meds[0].shape
    b_ = _rand_slots(shape, S.items, 15)
    for dt, tol in ((torch.complex128, 1e-10), (torch.complex64, 5e-5)):
        bd = torch.from_numpy(b_).to("cuda", dt)
        xd = torch.zeros_like(bd)
        S.vcycle(bd, xd)
        for it, med in enumerate(meds):
            H = mg.Hierarchy(_oracle_parts(med, 0.4), med.shape, levels,
                             w=[0.75, 0.5, 0.25][:levels - 1])
            xr = op.dofs_to_slots(H.cycle(op.slots_to_dofs(b_[it], shape), gamma=2), shape)
            assert _err(xd[it].cpu().numpy(), xr) <= tol, (dt, it, _err(xd[it].cpu().numpy(), xr))
    S.close()


def test_fgmres_wcycle_iterations_match_oracle():
    ehs = _ehs()
    meds = _media_2d(64, 2)
    q, u, info = _solve_both(meds, 4, ehs.EHS_C128, alpha=0.4, cycle=2)
    for it, med in enumerate(meds):
        K = _oracle_parts(med)
        H = mg.Hierarchy(_oracle_parts(med, 0.4), med.shape, 4, w=[0.75, 0.5, 0.25])
        qo = op.slots_to_dofs(q[it], med.shape)
        xo, io = krylov.fgmres(lambda v: K @ v, lambda v: H.cycle(v, gamma=2), qo, m=10)
        ug = op.slots_to_dofs(u[it], med.shape)
        assert info[it]["iters"] == io["iters"], (info[it], io["iters"])
        assert _err(ug, xo) <= 1e-5


@pytest.mark.parametrize("ortho", [0, 1])
def test_dd_fgmres_batched_media_compaction(ortho):
    """Two media converging at different iteration counts in one DD-MG batch:
    each item's count and solution must equal its own oracle solve."""
    ehs = _ehs()
    meds = _media_2d(64, 2)
    q, u, info = _solve_both(meds, 3, ehs.EHS_C64, precond=ehs.EHS_PRECOND_DD, dd=(2, 2, 1),
                             dd_overlap=4, dd_pad=8, ortho=ortho)
    for it, med in enumerate(meds):
        D = odd.DD(med, (2, 2), 4, 8, 3, 0.2)
        qo = op.slots_to_dofs(q[it], med.shape)
        xo, io = krylov.fgmres(lambda v: D.K @ v, D.apply, qo, m=10)
        ug = op.slots_to_dofs(u[it], med.shape)
        assert abs(info[it]["iters"] - io["iters"]) <= 1, (it, info[it], io["iters"])
        assert _err(ug, xo) <= 1e-5
    assert info[0]["iters"] != info[1]["iters"]


@pytest.mark.parametrize("fmt,tol", [(1, 2e-3), (2, 1.5e-2)])
def test_half_tables_operator(fmt, tol):
    """Galerkin levels with FP16 (fmt 1) / BF16 (fmt 2) coefficient storage,
    FP32 accumulation: relative error of K_l x against the FP64 oracle within
    the format's rounding (unit roundoff 4.9e-4 FP16, 3.9e-3 BF16)."""
    ehs = _ehs()
    meds = _media_2d(64, 2)
    S = ehs.solver_for(meds, levels=4, alpha=0.4, coef_half=fmt)
    for b, med in enumerate(meds):
        H = mg.Hierarchy(_oracle_parts(med, 0.4), med.shape, 4, w=[0.75, 0.5, 0.25])
        for l in (1, 2):
            shp = S.level_shape(l)
            x = _rand_slots(tuple(shp[2:]), S.items, 40 + l)
            xd = torch.from_numpy(x).to("cuda", torch.complex64)
            yd = torch.zeros_like(xd)
            S.op_apply(xd, yd, level=l)
            xe = op.slots_to_dofs(xd[b].cpu().numpy().astype(np.complex128), tuple(shp[2:]))
            ye = op.dofs_to_slots(H.K[l] @ xe, tuple(shp[2:]))
            err = _err(yd[b].cpu().numpy(), ye)
            assert err <= tol, (fmt, l, err)
    S.close()


@pytest.mark.parametrize("fmt", [1, 2])
def test_half_tables_fgmres(fmt):
    """Half-precision Galerkin tables inside the complex64 W-cycle: the FP64-class
    outer FGMRES still reaches 1e-6, the solution stays within 1e-5 of the
    oracle's, and the iteration count moves by at most 2."""
    ehs = _ehs()
    meds = _media_2d(64, 4)
    q, u, info = _solve_both(meds, 4, ehs.EHS_C64, alpha=0.4, cycle=2, coef_half=fmt)
    for it, med in enumerate(meds):
        K = _oracle_parts(med)
        H = mg.Hierarchy(_oracle_parts(med, 0.4), med.shape, 4, w=[0.75, 0.5, 0.25])
        qo = op.slots_to_dofs(q[it], med.shape)
        xo, io = krylov.fgmres(lambda v: K @ v, lambda v: H.cycle(v, gamma=2), qo, m=10)
        ug = op.slots_to_dofs(u[it], med.shape)
        assert info[it]["converged"] and np.linalg.norm(qo - K @ ug) / np.linalg.norm(qo) <= 1e-6
        assert abs(info[it]["iters"] - io["iters"]) <= 2, (fmt, it, info[it], io["iters"])
        assert _err(ug, xo) <= 1e-5


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_galerkin_rows_launch_shapes_agree(variant, monkeypatch):
    """Every residual-pass launch shape the setup autotuner can pick (1 or 2
    cells per thread, 64..256 threads) gives the oracle's Galerkin operator."""
    ehs = _ehs()
    monkeypatch.setenv("EHS_ROWS_VARIANT", str(variant))
    meds = _media_2d(64, 2)
    for fmt in (0, 1):
        S = ehs.solver_for(meds, levels=4, alpha=0.4, coef_half=fmt)
        for b, med in enumerate(meds):
            H = mg.Hierarchy(_oracle_parts(med, 0.4), med.shape, 4, w=[0.75, 0.5, 0.25])
            for l in (1, 2):
                shp = S.level_shape(l)
                x = _rand_slots(tuple(shp[2:]), S.items, 50 + l)
                for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5 if fmt == 0 else 2e-3)):
                    if fmt and dt == torch.complex128:
                        continue
                    xd = torch.from_numpy(x).to("cuda", dt)
                    yd = torch.zeros_like(xd)
                    S.op_apply(xd, yd, level=l)
                    xe = op.slots_to_dofs(xd[b].cpu().numpy().astype(np.complex128), tuple(shp[2:]))
                    ye = op.dofs_to_slots(H.K[l] @ xe, tuple(shp[2:]))
                    assert _err(yd[b].cpu().numpy(), ye) <= tol, (variant, fmt, l, dt)
        S.close()
    # a full solve with this launch shape keeps the oracle's iteration counts
    q, u, info = _solve_both(meds, 4, ehs.EHS_C64, alpha=0.4, cycle=2)
    for it, med in enumerate(meds):
        K = _oracle_parts(med)
        H = mg.Hierarchy(_oracle_parts(med, 0.4), med.shape, 4, w=[0.75, 0.5, 0.25])
        qo = op.slots_to_dofs(q[it], med.shape)
        _, io = krylov.fgmres(lambda v: K @ v, lambda v: H.cycle(v, gamma=2), qo, m=10)
        assert abs(info[it]["iters"] - io["iters"]) <= 1


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_full_vanka_smooth_matches_oracle(case):
    """Full cell-block Vanka (closed form on the fine level, stored FP64-built
    inverses on Galerkin levels) against the oracle's dense block inverses."""
    ehs = _ehs()
    meds = _media_2d(32, 2) if case == "2d" else _media_3d(16, 1)
    levels = 3
    S = ehs.solver_for(meds, levels=levels, alpha=0.2, vanka_full=1)
    for l in range(levels - 1):
        gshape = tuple(S.level_shape(l)[2:])
        b_ = _rand_slots(gshape, S.items, 40 + l)
        x_ = _rand_slots(gshape, S.items, 50 + l)
        for dt, tol in ((torch.complex128, 1e-11), (torch.complex64, 2e-5)):
            bd = torch.from_numpy(b_).to("cuda", dt)
            xd = torch.from_numpy(x_).to("cuda", dt)
            S.smooth(bd, xd, level=l, nsweeps=1)
            for it, med in enumerate(meds):
                H = mg.Hierarchy(_oracle_parts(med, 0.2), med.shape, levels, economic=False)
                be = op.slots_to_dofs(bd[it].cpu().numpy().astype(np.complex128), gshape)
                xe = op.slots_to_dofs(torch.from_numpy(x_[it]).to(dt).numpy().astype(np.complex128), gshape)
                xr = op.dofs_to_slots(H.relax(l, be, xe), gshape)
                assert _err(xd[it].cpu().numpy(), xr) <= tol, (l, dt, it, _err(xd[it].cpu().numpy(), xr))
    S.close()


@pytest.mark.parametrize("fmt,tol", [(1, 3e-3), (2, 2e-2)])
def test_full_vanka_half_inverses(fmt, tol):
    """Block inverses stored as FP16 / BF16 pairs (the half-precision storage of
    Sec. 4's implementation remark): one Galerkin-level sweep within the
    storage rounding of the FP64 result."""
    ehs = _ehs()
    meds = _media_2d(32, 1)
    S = ehs.solver_for(meds, levels=3, alpha=0.2, vanka_full=1, coef_half=fmt)
    gshape = tuple(S.level_shape(1)[2:])
    b_ = _rand_slots(gshape, S.items, 61)
    x_ = _rand_slots(gshape, S.items, 62)
    bd = torch.from_numpy(b_).to("cuda", torch.complex64)
    xd = torch.from_numpy(x_).to("cuda", torch.complex64)
    S.smooth(bd, xd, level=1, nsweeps=1)
    H = mg.Hierarchy(_oracle_parts(meds[0], 0.2), meds[0].shape, 3, economic=False)
    xr = op.dofs_to_slots(H.relax(1, op.slots_to_dofs(b_[0], gshape), op.slots_to_dofs(x_[0], gshape)), gshape)
    err = _err(xd[0].cpu().numpy(), xr)
    assert err <= tol, err
    S.close()


@pytest.mark.parametrize("prec_name", ["c128", "c64"])
def test_full_vanka_fgmres_matches_oracle(prec_name):
    ehs = _ehs()
    prec = ehs.EHS_C128 if prec_name == "c128" else ehs.EHS_C64
    meds = _media_2d(64, 2)
    q, u, info = _solve_both(meds, 4, prec, alpha=0.4, cycle=2, vanka_full=1)
    for it, med in enumerate(meds):
        K = _oracle_parts(med)
        H = mg.Hierarchy(_oracle_parts(med, 0.4), med.shape, 4, w=[0.75, 0.5, 0.25], economic=False)
        qo = op.slots_to_dofs(q[it], med.shape)
        xo, io = krylov.fgmres(lambda v: K @ v, lambda v: H.cycle(v, gamma=2), qo, m=10)
        ug = op.slots_to_dofs(u[it], med.shape)
        assert info[it]["converged"]
        if prec == ehs.EHS_C128:
            assert info[it]["iters"] == io["iters"], (info[it], io["iters"])
        else:
            assert abs(info[it]["iters"] - io["iters"]) <= 1, (info[it], io["iters"])
        assert _err(ug, xo) <= 1e-5


def test_full_vanka_dd_fgmres():
    """DD whose subdomain cycles use full Vanka: same iteration count and
    solution as the oracle DD with full-block subdomain smoothers."""
    ehs = _ehs()
    med = synth.homogeneous_2d()
    q, u, info = _solve_both([med], 3, ehs.EHS_C128, precond=ehs.EHS_PRECOND_DD, dd=(2, 2, 1),
                             dd_overlap=4, dd_pad=8, vanka_full=1)
    D = odd.DD(med, (2, 2), 4, 8, 3, 0.2, economic=False)
    qo = op.slots_to_dofs(q[0], med.shape)
    xo, io = krylov.fgmres(lambda v: D.K @ v, D.apply, qo, m=10)
    ug = op.slots_to_dofs(u[0], med.shape)
    assert info[0]["iters"] == io["iters"], (info[0], io["iters"])
    assert _err(ug, xo) <= 1e-5


# ------------------------------------------------------------- MG-DD, DD-MG-DD
@pytest.mark.parametrize("case,cyc", [("2d", 1), ("2d", 2), ("3d", 1)])
def test_mgdd_cycle_matches_oracle(case, cyc):
    """MG-DD (Sec. 4): the coarsest grid solved by one multicolour DD sweep with
    dense local solves; one cycle against the oracle's CoarseDD."""
    ehs = _ehs()
    if case == "2d":
        meds, levels, split, ov = _media_2d(64, 2), 3, (2, 2, 1), 2
    else:
        meds, levels, split, ov = _media_3d(16, 1), 3, (2, 2, 2), 1
    S = ehs.solver_for(meds, levels=levels, alpha=0.4, cycle=cyc, coarse_dd=split, coarse_dd_overlap=ov)
    shape = meds[0].shape
    d = len(shape)
    b_ = _rand_slots(shape, S.items, 71)
    for dt, tol in ((torch.complex128, 1e-10), (torch.complex64, 5e-5)):
        bd = torch.from_numpy(b_).to("cuda", dt)
        xd = torch.zeros_like(bd)
        S.vcycle(bd, xd)
        for it, med in enumerate(meds):
            H = mg.Hierarchy(_oracle_parts(med, 0.4), med.shape, levels,
                             w=[0.75, 0.5, 0.25][:levels - 1], coarse_dd=(split[:d], ov))
            xr = op.dofs_to_slots(H.cycle(op.slots_to_dofs(b_[it], shape), gamma=cyc), shape)
            assert _err(xd[it].cpu().numpy(), xr) <= tol, (dt, it, _err(xd[it].cpu().numpy(), xr))
    S.close()


@pytest.mark.parametrize("prec_name,fmt,persist,ortho", [("c128", 0, 0, 0), ("c64", 0, 0, 0), ("c64", 1, 0, 0),
                                                         ("c64", 2, 0, 0), ("c64", 3, 0, 0), ("c64", 1, 1, 0),
                                                         ("c64", 2, 1, 0), ("c64", 3, 1, 0), ("c64", 0, 0, 1),
                                                         ("c64", 2, 0, 1)])
def test_mgdd_fgmres_matches_oracle(prec_name, fmt, persist, ortho):
    """MG-DD inside FGMRES; the local inverses in double-float, complex64, FP16 or
    BF16 storage (FP32 accumulation) for the complex64 cycle; with persist the
    complex64 coarsest solve runs as one persistent launch (opts.coarse_persist); with
    ortho the double-float solve uses delayed CGS2."""
    ehs = _ehs()
    prec = ehs.EHS_C128 if prec_name == "c128" else ehs.EHS_C64
    meds = _media_2d(64, 2)
    q, u, info = _solve_both(meds, 3, prec, alpha=0.4, cycle=2, coarse_dd=(2, 2, 1), coarse_dd_overlap=2,
                             coarse_fmt=fmt, coarse_persist=persist, ortho=ortho)
    for it, med in enumerate(meds):
        K = _oracle_parts(med)
        H = mg.Hierarchy(_oracle_parts(med, 0.4), med.shape, 3, w=[0.75, 0.5], coarse_dd=((2, 2), 2))
        qo = op.slots_to_dofs(q[it], med.shape)
        xo, io = krylov.fgmres(lambda v: K @ v, lambda v: H.cycle(v, gamma=2), qo, m=10)
        ug = op.slots_to_dofs(u[it], med.shape)
        assert info[it]["converged"]
        if prec == ehs.EHS_C128:
            assert info[it]["iters"] == io["iters"], (info[it], io["iters"])
        else:
            assert abs(info[it]["iters"] - io["iters"]) <= (1 if fmt < 2 else 2), (info[it], io["iters"])
        assert _err(ug, xo) <= 1e-5


def test_coarse_fmt_inverse_fgmres():
    """Exact coarsest solve with the inverse stored in complex64: same counts as
    the oracle (+-1) and the same solution."""
    ehs = _ehs()
    meds = _media_2d(64, 2)
    q, u, info = _solve_both(meds, 3, ehs.EHS_C64, coarse_fmt=1)
    for it, med in enumerate(meds):
        K = _oracle_parts(med)
        H = mg.Hierarchy(_oracle_parts(med, 0.2), med.shape, 3)
        qo = op.slots_to_dofs(q[it], med.shape)
        xo, io = krylov.fgmres(lambda v: K @ v, H.cycle, qo, m=10)
        ug = op.slots_to_dofs(u[it], med.shape)
        assert info[it]["converged"] and abs(info[it]["iters"] - io["iters"]) <= 1, (info[it], io["iters"])
        assert _err(ug, xo) <= 1e-5


def test_dd_mg_dd_fgmres_matches_oracle():
    """DD-MG-DD (Sec. 4): top-level DD whose subdomain cycles solve their
    coarsest grids by DD; iteration count and solution as the oracle's."""
    ehs = _ehs()
    med = synth.homogeneous_2d()
    q, u, info = _solve_both([med], 3, ehs.EHS_C128, precond=ehs.EHS_PRECOND_DD, dd=(2, 2, 1),
                             dd_overlap=4, dd_pad=8, coarse_dd=(2, 2, 1), coarse_dd_overlap=2)
    D = odd.DD(med, (2, 2), 4, 8, 3, 0.2, coarse_dd=((2, 2), 2))
    qo = op.slots_to_dofs(q[0], med.shape)
    xo, io = krylov.fgmres(lambda v: D.K @ v, D.apply, qo, m=10)
    ug = op.slots_to_dofs(u[0], med.shape)
    assert info[0]["iters"] == io["iters"], (info[0], io["iters"])
    assert _err(ug, xo) <= 1e-5


def test_mgdd_rejects_bad_split():
    ehs = _ehs()
    meds = _media_2d(32, 1)
    with pytest.raises(ehs.EhsError, match="ERR_ARG"):
        ehs.solver_for(meds, levels=3, coarse_dd=(3, 3, 1), coarse_dd_overlap=2)   # cores of 2-3 cells


@pytest.mark.parametrize("split,fmt,tol", [((1, 1, 1), 1, 2e-5), ((2, 2, 1), 0, 1e-10), ((2, 2, 1), 1, 2e-5),
                                           ((2, 2, 1), 2, 3e-3)])
def test_coarse_solve_and_local_apply(split, fmt, tol):
    """ehs_coarse_solve against the oracle's coarsest solve (exact LU or the
    CoarseDD sweep), every colour's ehs_coarse_local_apply against the
    oracle's dense solve of the subdomain matrix (the coarsest operator
    restricted to the box unknowns), and ehs_coarse_local_add (the same
    products added into a random coarsest vector at the boxes' unknowns)."""
    ehs = _ehs()
    meds = _media_2d(64, 2)
    cdd = split[0] * split[1] > 1
    S = ehs.solver_for(meds, levels=3, alpha=0.4, coarse_dd=split, coarse_dd_overlap=2, coarse_fmt=fmt)
    cshape = tuple(S.level_shape(2)[2:])
    dt = torch.complex128 if (fmt == 0 and cdd) else torch.complex64
    b_ = _rand_slots(cshape, S.items, 81)
    bd = torch.from_numpy(b_).to("cuda", dt)
    xd = torch.zeros_like(bd)
    S.coarse_solve(bd, xd, prec=ehs.EHS_C128 if dt == torch.complex128 else ehs.EHS_C64)
    ns, nloc, sizes = S.coarse_dims()
    assert ns == (4 if cdd else 1)
    if cdd:
        assert nloc % 8 == 0 and max(sizes) <= nloc
    rng = np.random.default_rng(5)
    rl = rng.standard_normal((S.items, ns, nloc)) + 1j * rng.standard_normal((S.items, ns, nloc))
    for s_, n in enumerate(sizes):
        rl[:, s_, n:] = 0
    rld = torch.from_numpy(rl).to("cuda", dt)
    zs, xs = {}, {}
    x0 = _rand_slots(cshape, S.items, 82)
    for col in (range(4) if cdd else [0]):
        zd = torch.zeros_like(rld)
        S.coarse_local_apply(col, rld, zd, prec=ehs.EHS_C128 if dt == torch.complex128 else ehs.EHS_C64)
        zs[col] = zd.cpu().numpy()
        if cdd:   # the same products added into a coarsest vector at the boxes' unknowns
            xa = torch.from_numpy(x0).to("cuda", dt)
            S.coarse_local_add(col, rld, xa, prec=ehs.EHS_C128 if dt == torch.complex128 else ehs.EHS_C64)
            xs[col] = xa.cpu().numpy()
    for it, med in enumerate(meds):
        H = mg.Hierarchy(_oracle_parts(med, 0.4), med.shape, 3, w=[0.75, 0.5],
                         coarse_dd=((split[0], split[1]), 2) if cdd else None)
        xr = op.dofs_to_slots(H.coarse_solve(op.slots_to_dofs(b_[it], cshape)), cshape)
        assert _err(xd[it].cpu().numpy(), xr) <= tol, (it, _err(xd[it].cpu().numpy(), xr))
        Kc = H.K[-1].tocsc()
        if not cdd:
            continue
        nx = split[0]
        xadd = {col: op.slots_to_dofs(x0[it].astype(np.complex128), cshape) for col in xs}
        for p_, (col, idx, _) in enumerate(H.cdd.subs):
            ix, iy = divmod(p_, split[1])          # oracle order: y index fastest
            s_ = iy * nx + ix                      # library order: x index fastest
            assert sizes[s_] == idx.size
            ze = np.linalg.solve(Kc[idx][:, idx].toarray(), rl[it, s_, :idx.size])
            got = zs[col][it, s_, :idx.size]
            assert _err(got, ze) <= tol, (it, s_, _err(got, ze))
            xadd[col][idx] += ze
        for col, xe in xadd.items():
            got = op.slots_to_dofs(xs[col][it], cshape)
            assert _err(got, xe) <= tol, (it, col, _err(got, xe))
    S.close()


def test_dd_mg_dd_3d_fgmres_matches_oracle():
    """3D DD-MG-DD (Sec. 4, the paper's 3D method): top-level DD 2x2x2 whose
    subdomain cycles split their coarsest grids 2x2x1; iteration count and
    solution as the oracle's (FP64 form)."""
    ehs = _ehs()
    med = synth.layered_3d(n=24, seed=1, corr=4.0, abl=4)
    q, u, info = _solve_both([med], 3, ehs.EHS_C128, precond=ehs.EHS_PRECOND_DD, dd=(2, 2, 2), dd_overlap=2,
                             dd_pad=4, alpha=0.5, w=[0.5, 0.5], coarse_dd=(2, 2, 1), coarse_dd_overlap=1)
    D = odd.DD(med, (2, 2, 2), 2, 4, 3, 0.5, w=[0.5, 0.5], coarse_dd=((2, 2, 1), 1))
    qo = op.slots_to_dofs(q[0], med.shape)
    xo, io = krylov.fgmres(lambda v: D.K @ v, D.apply, qo, m=10)
    ug = op.slots_to_dofs(u[0], med.shape)
    assert info[0]["iters"] == io["iters"], (info[0], io["iters"])
    assert _err(ug, xo) <= 1e-5


@pytest.mark.parametrize("fmt", [1, 2])
def test_mgdd_multi_rhs_local_products(fmt):
    """Five sources per medium share each MG-DD subdomain inverse: every
    source's local solve (local vectors in [nmedia][nsub][nrhs][nloc] order)
    equals the dense solve of its subdomain matrix, and FGMRES keeps the
    oracle's iteration counts (+-1) and solutions for every source."""
    ehs = _ehs()
    meds = _media_2d(64, 1)
    nrhs = 5
    S = ehs.solver_for(meds, levels=3, alpha=0.4, nrhs=nrhs, coarse_dd=(2, 2, 1), coarse_dd_overlap=2,
                       coarse_fmt=fmt)
    ns, nloc, sizes = S.coarse_dims()
    rng = np.random.default_rng(8)
    shp = (1, ns, nrhs, nloc)                  # local vectors: [nmedia][nsub][nrhs][nloc]
    rl = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    for s_, n in enumerate(sizes):
        rl[:, s_, :, n:] = 0
    rld = torch.from_numpy(rl).to("cuda", torch.complex64)
    H = mg.Hierarchy(_oracle_parts(meds[0], 0.4), meds[0].shape, 3, w=[0.75, 0.5], coarse_dd=((2, 2), 2))
    Kc = H.K[-1].tocsc()
    tol = 2e-5 if fmt == 1 else 3e-3
    for col in range(4):
        zd = torch.zeros_like(rld)
        S.coarse_local_apply(col, rld, zd, prec=ehs.EHS_C64)
        z = zd.cpu().numpy()
        for p_, (c_, idx, _) in enumerate(H.cdd.subs):
            if c_ != col:
                continue
            ix, iy = divmod(p_, 2)
            s_ = iy * 2 + ix
            A = Kc[idx][:, idx].toarray()
            for it in range(nrhs):
                ze = np.linalg.solve(A, rl[0, s_, it, :idx.size])
                err = _err(z[0, s_, it, :idx.size], ze)
                assert err <= tol, (col, it, s_, err)
    S.close()
    q, u, info = _solve_both(meds, 3, ehs.EHS_C64, nrhs=nrhs, alpha=0.4, coarse_dd=(2, 2, 1),
                             coarse_dd_overlap=2, coarse_fmt=fmt)
    K = _oracle_parts(meds[0])
    for it in range(nrhs):
        qo = op.slots_to_dofs(q[it], meds[0].shape)
        xo, io = krylov.fgmres(lambda v: K @ v, H.cycle, qo, m=10)
        ug = op.slots_to_dofs(u[it], meds[0].shape)
        assert info[it]["converged"] and abs(info[it]["iters"] - io["iters"]) <= 1, (it, info[it], io["iters"])
        assert _err(ug, xo) <= 1e-5


# ------------------------------------------ uneven DD subdomains (shape groups)
# Algorithm DD (Sec. 2.3) on splits whose subdomains of one colour have different
# padded shapes, so that the library batches each colour as several shape groups
# (one hierarchy per group).  The geometry of both cases is checked on the CPU in
# tests/test_oracle_dd.py (test_uneven_parity_splits_have_several_shape_groups).
UNEVEN_2D = dict(split=(3, 3, 1), osplit=(3, 3), overlap=2, pad=4)
UNEVEN_3D = dict(split=(3, 3, 2), osplit=(2, 3, 3), overlap=3, pad=4)


def _med_uneven_2d():
    """44 x 32 cells (non-square), 4-cell absorbing layer."""
    return synth.random_2d(n=32, nx=44, sigma=0.4, seed=3, corr=6.0, abl=4)


def _med_uneven_3d():
    """28 x 28 x 16 cells: the top 16 layers of a 28^3 layered medium, two x-forces."""
    m = synth.layered_3d(n=28, seed=1, corr=4.0, abl=4)
    sl = slice(0, 16)
    return synth.Medium(m.lam[sl].copy(), m.mu[sl].copy(), m.rho[sl].copy(), m.omega, m.h, m.abl_cells,
                        [(0, (6, 14, 10)), (0, (6, 14, 17))], name="layered28x28x16")


def _uneven(case):
    if case == "2d":
        return _med_uneven_2d(), UNEVEN_2D, 0.2, [0.75, 0.5], 1
    return _med_uneven_3d(), UNEVEN_3D, 0.5, [0.5, 0.5], 2


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_dd_uneven_split_apply_matches_oracle(case):
    """One sweep of Algorithm DD over an uneven split (several shape groups per
    colour): complex128 within 1e-10, complex64 within 5e-5 of the oracle."""
    ehs = _ehs()
    med, g, alpha, w, _ = _uneven(case)
    D = odd.DD(med, g["osplit"], g["overlap"], g["pad"], 3, alpha, w=w)
    r = _rand_slots(med.shape, 1, 19)
    zo = op.dofs_to_slots(D.apply(op.slots_to_dofs(r[0], med.shape)), med.shape)
    for prec, tol in ((ehs.EHS_C128, 1e-10), (ehs.EHS_C64, 5e-5)):
        S = ehs.solver_for(med, levels=3, alpha=alpha, w=w, precond=ehs.EHS_PRECOND_DD, dd=g["split"],
                           dd_overlap=g["overlap"], dd_pad=g["pad"], prec=prec)
        rd = torch.from_numpy(r).cuda()
        zd = torch.zeros_like(rd)
        S.dd_precond(rd, zd, prec=prec)
        assert _err(zd[0].cpu().numpy(), zo) <= tol, (case, prec, _err(zd[0].cpu().numpy(), zo))
        S.close()


@pytest.mark.parametrize("case", ["2d", "3d"])
@pytest.mark.parametrize("form", ["dd-mg", "dd-mg-dd"])
def test_dd_uneven_split_fgmres_matches_oracle(case, form):
    """FGMRES preconditioned by Algorithm DD on an uneven split (DD-MG with exact
    subdomain coarsest solves, or DD-MG-DD with the subdomain coarsest grids split
    2 x 2 (x 1)), in 3D with two sources in one batch: the oracle's iteration count
    exactly in complex128 (+-1 in complex64), true residual <= 1e-6, solution
    within 1e-5 of the oracle's element by element, for every source."""
    ehs = _ehs()
    med, g, alpha, w, nrhs = _uneven(case)
    d = len(med.shape)
    cdd = ((2, 2, 1)[:d], 1) if form == "dd-mg-dd" else None
    D = odd.DD(med, g["osplit"], g["overlap"], g["pad"], 3, alpha, w=w, coarse_dd=cdd)
    extra = dict(coarse_dd=(2, 2, 1), coarse_dd_overlap=1) if cdd else {}
    for prec in (ehs.EHS_C128, ehs.EHS_C64):
        q, u, info = _solve_both([med], 3, prec, nrhs=nrhs, alpha=alpha, w=w, precond=ehs.EHS_PRECOND_DD,
                                 dd=g["split"], dd_overlap=g["overlap"], dd_pad=g["pad"], **extra)
        for it in range(nrhs):
            qo = op.slots_to_dofs(q[it], med.shape)
            xo, io = krylov.fgmres(lambda v: D.K @ v, D.apply, qo, m=10)
            ug = op.slots_to_dofs(u[it], med.shape)
            assert info[it]["converged"] and np.linalg.norm(qo - D.K @ ug) / np.linalg.norm(qo) <= 1e-6
            if prec == ehs.EHS_C128:
                assert info[it]["iters"] == io["iters"], (case, form, it, info[it], io["iters"])
            else:
                assert abs(info[it]["iters"] - io["iters"]) <= 1, (case, form, it, info[it], io["iters"])
            assert _err(ug, xo) <= 1e-5, (case, form, prec, it, _err(ug, xo))


@pytest.mark.parametrize("fmt,tfmt", [(1, 0), (2, 1), (3, 2)])
def test_coarse_persistent_equals_per_colour_launches(fmt, tfmt):
    """The persistent MG-DD coarsest solve (one launch, grid barriers between the
    colours' residual, local-product and scatter phases) gives the result of the
    per-colour launches (the same arithmetic per element), with several sources
    per medium so that sub-items of many media and sources share each phase; and
    both match the oracle's CoarseDD within the storage rounding."""
    ehs = _ehs()
    meds = _media_2d(64, 2)
    outs = {}
    for persist in (1, 0):
        S = ehs.solver_for(meds, levels=3, alpha=0.4, nrhs=3, coarse_dd=(2, 2, 1), coarse_dd_overlap=2,
                           coarse_fmt=fmt, coef_half=tfmt, coarse_persist=persist)
        cshape = tuple(S.level_shape(2)[2:])
        b_ = _rand_slots(cshape, S.items, 91)
        bd = torch.from_numpy(b_).to("cuda", torch.complex64)
        xd = torch.full_like(bd, 5.0)
        S.coarse_solve(bd, xd)
        S.sync()
        outs[persist] = xd.cpu().numpy()
        S.close()
    assert _err(outs[1], outs[0]) <= 1e-6, _err(outs[1], outs[0])
    tol = {1: 2e-5, 2: 3e-3, 3: 2e-2}[fmt]
    for it in range(6):
        H = mg.Hierarchy(_oracle_parts(meds[it // 3], 0.4), meds[0].shape, 3, w=[0.75, 0.5], coarse_dd=((2, 2), 2))
        xr = op.dofs_to_slots(H.coarse_solve(op.slots_to_dofs(b_[it], cshape)), cshape)
        assert _err(outs[1][it], xr) <= tol, (it, _err(outs[1][it], xr))
