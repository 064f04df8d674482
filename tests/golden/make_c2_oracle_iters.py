"""Writes c2_oracle_iters.json: the CPU oracle's FGMRES(10) iteration counts
(and final relative residuals) for the 512 x 512 four-Poisson-ratio workload
of bench.py: 3-level V(1,1) cycle, alpha 0.25, damping 0.75/0.5, economic
red-black Vanka, MG-DD coarsest solve (128 x 128 coarsest grid split 8 x 8,
overlap 3), tol 1e-6.  Calls only oracle/ and the seeded input generator.
Run from the repository root:
    python tests/golden/make_c2_oracle_iters.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import krylov, multigrid as mg, operators as op  # noqa: E402
from paper_1806_11277_gb300 import synth  # noqa: E402

SIGMAS = (0.25, 0.4, 0.45, 0.49)
LEVELS, ALPHA, W, GAMMA = 3, 0.25, [0.75, 0.5], 1
COARSE_DD, COARSE_OVERLAP = (8, 8), 3


def main():
    iters, relres, secs = [], [], []
    for s in SIGMAS:
        med = synth.random_2d(n=512, sigma=s, seed=0)
        parts = op.parts_for(med)
        K = op.assemble_mixed(parts)
        H = mg.Hierarchy(op.assemble_mixed(parts, ALPHA), med.shape, LEVELS, w=W,
                         coarse_dd=(COARSE_DD, COARSE_OVERLAP))
        q = op.slots_to_dofs(synth.point_rhs(med.shape, med.sources)[0], med.shape)
        t = time.time()
        _, info = krylov.fgmres(lambda v: K @ v, lambda v: H.cycle(v, gamma=GAMMA), q, m=10, tol=1e-6)
        secs.append(time.time() - t)
        iters.append(info["iters"])
        relres.append(info["relres"])
        print(s, info["iters"], info["relres"], f"{secs[-1]:.0f}s", flush=True)
    out = dict(workload="512x512 GRF media, seed 0, sigma 0.25/0.4/0.45/0.49, 8 ppw, 20-cell ABL",
               levels=LEVELS, alpha=ALPHA, w=W, cycle="W(1,1)" if GAMMA == 2 else "V(1,1)",
               coarse_dd=list(COARSE_DD), coarse_dd_overlap=COARSE_OVERLAP, restart=10, tol=1e-6,
               sigmas=list(SIGMAS), iters=iters, relres=relres)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_oracle_iters.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
