"""The benchmark's default solver options and the oracle configuration behind
the stored iteration counts (tests/golden/c2_oracle_iters.json) must agree;
checked here without a GPU so that a change to either side shows up at once."""
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def test_default_line_matches_golden_oracle_config():
    import bench
    gold = json.load(open(os.path.join(HERE, "golden", "c2_oracle_iters.json")))
    kw = bench.default_kw()
    assert gold["levels"] == kw["levels"]
    assert gold["alpha"] == kw["alpha"]
    assert gold["w"] == list(kw["w"])
    assert gold["cycle"] == ("W(1,1)" if kw["cycle"] == 2 else "V(1,1)")
    assert list(gold["coarse_dd"]) == list(kw["coarse_dd"][:2])
    assert gold["coarse_dd_overlap"] == kw["coarse_dd_overlap"]
    assert gold["sigmas"] == list(bench.SIGMAS)
    assert gold["restart"] == 10 and gold["tol"] == 1e-6
    assert len(gold["iters"]) == len(bench.SIGMAS) and all(r <= 1e-6 for r in gold["relres"])


def test_bench_configs_are_complete():
    import bench
    for name, cfg in bench.OTHER.items():
        assert cfg is not None, name
        assert {"workload", "media", "kw", "kernel"} <= set(cfg), name
        assert cfg.get("roof") == "coarse" or "rows_l1_bytes" in cfg, name


def test_fwi_workload_generator():
    """The gradient line's inputs: 16 x-forces and 200 distinct receivers on the
    line y = ABL + 2 inside the interior; the true model scales lambda and mu
    by (1 + 0.05 b)^2 with b a unit Gaussian bump, rho unchanged."""
    import numpy as np
    from paper_1806_11277_gb300 import synth
    base, true, (ry, rx) = synth.fwi_2d()
    n, abl = base.shape[0], base.abl_cells
    assert len(base.sources) == 16 and all(k == 0 and idx[0] == abl + 2 for k, idx in base.sources)
    assert len(set(rx.tolist())) == 200 and (ry == abl + 2).all()
    assert rx.min() >= abl and rx.max() < n - abl
    f = true.lam / base.lam
    assert np.allclose(true.mu / base.mu, f) and np.array_equal(true.rho, base.rho)
    assert 1.0 <= f.min() and abs(f.max() - 1.05 ** 2) < 1e-3


def test_clock_sampler_parses_clocks_and_reasons(tmp_path, monkeypatch):
    """The bench's clock record (median SM clock under load, max clock, active
    throttle reasons) from the nvidia-smi CSV it samples, with a stand-in
    nvidia-smi on PATH: 'Not Active' is not a reason, N/A rows are skipped."""
    import bench
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '1980, 2070, 1390.5, Not Active, Not Active, Not Active, Active'\n"
                    "echo '[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]'\n"
                    "echo '2040, 2070, 1200.0, Not Active, Not Active, Not Active, Not Active'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    s = bench.ClockSampler(0)
    s.start()
    import time
    t0 = time.time()
    while len(s.rows) < 4 and time.time() - t0 < 20:
        time.sleep(0.05)
    rec = s.stop()
    assert rec["sm_mhz"] == 2040.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]


def test_every_bench_config_passes_host_validation():
    """Every bench workload (the default line, its small profiling case and each --config) gets past
    ehs_create's host-side checks of its options against its grid (levels,
    MG-DD split and overlap, formats): on a host without a GPU the create call
    then stops at its first CUDA call (EHS_ERR_CUDA), never at EHS_ERR_ARG."""
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("with a GPU present the create call would build the full hierarchy")
    import bench
    from paper_1806_11277_gb300 import build, ehs
    try:
        ehs.load(build.build())
    except FileNotFoundError:
        pytest.skip("nvcc not available")
    cases = {"c2": (bench.media, {}), "small": (lambda: bench.small_case()[0], bench.small_case()[1])}
    cases.update({k: (v["media"], v["kw"]) for k, v in bench.OTHER.items()})
    for name, (mk, over) in cases.items():
        kw = bench.default_kw()
        kw.update(over)
        with pytest.raises(ehs.EhsError) as e:
            ehs.solver_for(mk(), **kw)
        assert e.value.status == 2, (name, str(e.value))


def test_oracle_dd_sample_of_the_3d_lines():
    """The CPU baseline of the 3D DD lines (one global residual, one cycle of the
    largest subdomain and ten Krylov iterations of the oracle, extrapolated to a
    DD-preconditioned iteration) runs on a small medium with the lines' DD-MG and
    DD-MG-DD options and reports a positive rate with its sample description."""
    import bench
    from paper_1806_11277_gb300 import synth
    med = synth.layered_3d(n=32, seed=0, corr=4.0, abl=4)
    base = dict(levels=3, alpha=0.5, w=[0.5, 0.5], dd=(2, 2, 2), dd_overlap=2, dd_pad=4, coarse_dd=(1, 1, 1))
    for kw in (base, dict(base, coarse_dd=(2, 2, 1), coarse_dd_overlap=1)):
        r = bench.oracle_dd_sample(med, kw, [20, 22])
        assert r["value"] > 0 and r["kind"] == "oracle" and "8 subdomain cycles" in r["sample"]
