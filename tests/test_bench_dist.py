"""The multi-rank part of bench.py on CPU: two gloo ranks, each timing its own
replica, agree on the maximum time, so the whole-job value divides the units
of all ranks by the slowest rank's time."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total = bench.max_over_ranks(1.0 + rank, dist, torch.device("cpu"))
    out.put((rank, total))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 2.0, 1: 2.0}


def test_reference_arm_only_rank0_prints(tmp_path, monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, ref_iters, gpus = 1, 0, 1, 2
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_json_contract(monkeypatch, capsys):
    """Rank 0 of the reference arm prints one JSON line with the keys the
    benchmark contract asks for (on small 64x64 media so that the oracle runs
    in seconds; the solver options are the default line's, with a coarsest
    split that fits the smaller grid)."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    from paper_1806_11277_gb300 import synth
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(bench, "media", lambda seed=0: [synth.random_2d(n=64, sigma=s, seed=seed, corr=6.0, abl=8)
                                                       for s in bench.SIGMAS])
    monkeypatch.setattr(bench, "COARSE_DD", (2, 2, 1))
    monkeypatch.setattr(bench, "COARSE_OVERLAP", 1)
    monkeypatch.setattr(bench, "_ORACLE_CACHE", {})

    class A:
        steps, warmup, ref_iters, gpus = 2, 1, 2, 1
    assert bench.run_reference(A()) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["metric"] == bench.METRIC and j["unit"] == "solves/s"
    assert j["higher_is_better"] is True and j["value"] > 0 and j["steps"] == 2 and j["warmup"] == 1
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == j["value"] and cb["cores"] >= 1 and cb["sample"]
    assert j["e2e"] == {"value": j["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert j["config"]["workload"] == bench.WORKLOAD
