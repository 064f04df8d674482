"""Writes c2_oracle_iters.json: the CPU oracle's FGMRES(10) iteration counts
(and final relative residuals) for the 512 x 512 four-Poisson-ratio workload
of bench.py: 3-level V(1,1) cycle, alpha 0.2, damping 0.75/0.5, economic
red-black Vanka, MG-DD coarsest solve (128 x 128 coarsest grid split 8 x 8,
overlap 3), tol 1e-6.  Also writes c2_oracle_samples.json: per medium the
oracle's solution at a fixed seeded sample of DOFs (uniform over the whole
mixed vector, plus the largest entries around the source), with the 2-norm
and the largest magnitude of the whole solution, so that a GPU solution of
the same workload can be compared with the FP64 oracle's entry by entry.
Calls only oracle/ and the seeded input generator.
Run from the repository root:
    python tests/golden/make_c2_oracle_iters.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import krylov, multigrid as mg, operators as op  # noqa: E402
from paper_1806_11277_gb300 import synth  # noqa: E402

SIGMAS = (0.25, 0.4, 0.45, 0.49)
LEVELS, ALPHA, W, GAMMA = 3, 0.2, [0.75, 0.5], 1
COARSE_DD, COARSE_OVERLAP = (8, 8), 3
N_UNIFORM, N_LARGEST, SAMPLE_SEED = 1024, 64, 2024


def sample_dofs(x, seed=SAMPLE_SEED):
    """Indices into the oracle's DOF vector: N_UNIFORM drawn uniformly without
    replacement (seeded, the same for every medium) and the N_LARGEST entries of
    largest magnitude of this solution (around the source)."""
    rng = np.random.default_rng(seed)
    uni = rng.choice(x.size, N_UNIFORM, replace=False)
    big = np.argsort(-np.abs(x))[:N_LARGEST]
    return np.unique(np.concatenate([uni, big]))


def main():
    iters, relres, secs, samples = [], [], [], []
    for s in SIGMAS:
        med = synth.random_2d(n=512, sigma=s, seed=0)
        parts = op.parts_for(med)
        K = op.assemble_mixed(parts)
        H = mg.Hierarchy(op.assemble_mixed(parts, ALPHA), med.shape, LEVELS, w=W,
                         coarse_dd=(COARSE_DD, COARSE_OVERLAP))
        q = op.slots_to_dofs(synth.point_rhs(med.shape, med.sources)[0], med.shape)
        t = time.time()
        x, info = krylov.fgmres(lambda v: K @ v, lambda v: H.cycle(v, gamma=GAMMA), q, m=10, tol=1e-6)
        secs.append(time.time() - t)
        idx = sample_dofs(x)
        samples.append(dict(sigma=s, ndof=int(x.size), norm2=float(np.linalg.norm(x)),
                            maxabs=float(np.abs(x).max()), idx=[int(i) for i in idx],
                            re=[float("%.12e" % v) for v in x[idx].real],
                            im=[float("%.12e" % v) for v in x[idx].imag]))
        iters.append(info["iters"])
        relres.append(info["relres"])
        print(s, info["iters"], info["relres"], f"{secs[-1]:.0f}s", flush=True)
    out = dict(workload="512x512 GRF media, seed 0, sigma 0.25/0.4/0.45/0.49, 8 ppw, 20-cell ABL",
               levels=LEVELS, alpha=ALPHA, w=W, cycle="W(1,1)" if GAMMA == 2 else "V(1,1)",
               coarse_dd=list(COARSE_DD), coarse_dd_overlap=COARSE_OVERLAP, restart=10, tol=1e-6,
               sigmas=list(SIGMAS), iters=iters, relres=relres)
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "c2_oracle_iters.json"), "w") as f:
        json.dump(out, f, indent=1)
    smp = dict(workload=out["workload"], solver="as c2_oracle_iters.json", dof_order="oracle DOF vector "
               "(operators.slots_to_dofs: u_x interior faces, u_y interior faces, p; x fastest)",
               sample=f"{N_UNIFORM} DOFs uniform (seed {SAMPLE_SEED}) + the {N_LARGEST} largest |x|",
               media=samples)
    with open(os.path.join(here, "c2_oracle_samples.json"), "w") as f:
        json.dump(smp, f, separators=(",", ":"))


if __name__ == "__main__":
    main()
