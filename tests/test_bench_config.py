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
