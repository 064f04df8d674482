"""Full-size checks in the configuration bench.py times (512 x 512, four
Poisson ratios batched, MG-DD: 3-level complex64 V(1,1) cycle with a DD
coarsest solve over 8 x 8 subdomains, FP16 tables and local inverses,
double-float FGMRES).

The oracle's full solves take minutes, so the per-medium iteration counts it
produced are stored in tests/golden/c2_oracle_iters.json and its solutions at
1088 sampled DOFs per medium in tests/golden/c2_oracle_samples.json (both
written by tests/golden/make_c2_oracle_iters.py, which calls only oracle/).
The GPU counts must match them (+-2: the complex64 cycle with FP16 tables and
local inverses against the FP64 oracle), the GPU solution must lie within
1e-5 of the oracle's at every sampled DOF (relative to the largest entry of
the oracle's solution), the true residual of every GPU solution is
recomputed with the oracle's own assembled complex128 operator, and sampled
operator rows are compared element-wise.
"""
import json
import os

import numpy as np
import pytest

from oracle import operators as op

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("ortho", [0, 1])
def test_bench_workload_iterations_and_residuals(ortho):
    """The bench workload with either Arnoldi orthogonalisation of the double-float
    solve (CGS2, delayed CGS2)."""
    import bench
    from paper_1806_11277_gb300 import ehs
    gold = json.load(open(os.path.join(HERE, "golden", "c2_oracle_iters.json")))
    smp = json.load(open(os.path.join(HERE, "golden", "c2_oracle_samples.json")))["media"]
    kw = dict(bench.default_kw(), ortho=ortho)
    assert gold["levels"] == kw["levels"] and gold["alpha"] == kw["alpha"] and gold["w"] == kw["w"]
    assert gold["cycle"] == ("W(1,1)" if kw["cycle"] == 2 else "V(1,1)")
    assert tuple(gold["coarse_dd"]) == tuple(kw["coarse_dd"][:2])
    assert gold["coarse_dd_overlap"] == kw["coarse_dd_overlap"]
    meds = bench.media()
    S = ehs.solver_for(meds, **kw)
    q = bench.rhs(meds)
    qd = torch.from_numpy(q).cuda()
    ud = torch.zeros_like(qd)
    info = S.fgmres_solve(qd, ud)
    u = ud.cpu().numpy()
    for it, med in enumerate(meds):
        assert abs(info[it]["iters"] - gold["iters"][it]) <= 2, (it, info[it], gold["iters"][it])
        K = op.assemble_mixed(op.parts_for(med))
        qo = op.slots_to_dofs(q[it], med.shape)
        uo = op.slots_to_dofs(u[it], med.shape)
        assert np.linalg.norm(qo - K @ uo) / np.linalg.norm(qo) <= 1e-6
        # the solution against the FP64 oracle's at the stored DOFs
        m = smp[it]
        assert m["sigma"] == bench.SIGMAS[it] and m["ndof"] == uo.size
        idx = np.asarray(m["idx"])
        ref = np.asarray(m["re"]) + 1j * np.asarray(m["im"])
        err = np.abs(uo[idx] - ref).max() / m["maxabs"]
        assert err <= 1e-5, (it, err)
        assert np.linalg.norm(uo) == pytest.approx(m["norm2"], rel=1e-5)
    # sampled rows of the FP64 operator at full size
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(q.shape) + 1j * rng.standard_normal(q.shape))
    x[:, 0, :, 0] = 0
    x[:, 1, 0, :] = 0
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    S.op_apply(xd, yd, level=0)
    y = yd.cpu().numpy()
    for it, med in enumerate(meds):
        K = op.assemble_mixed(op.parts_for(med)).tocsr()
        ye = K @ op.slots_to_dofs(x[it], med.shape)
        yg = op.slots_to_dofs(y[it], med.shape)
        rows = rng.choice(ye.size, 2000, replace=False)
        assert np.allclose(yg[rows], ye[rows], rtol=1e-12, atol=1e-12 * np.abs(ye).max())
    S.close()
