"""Benchmark: elastic Helmholtz solves/s to a 1e-6 residual on GB300.

Workload (one step): four 512 x 512 heterogeneous media (smooth Gaussian
random fields, correlation 20 cells, Vp in [1.5, 4.5], rho in [1, 2.5]) with
Poisson ratios 0.25 / 0.4 / 0.45 / 0.49, 8 points per shortest S-wavelength,
20-cell absorbing layer, one x-force each; an MG-DD preconditioner (a
complex64 3-level V-cycle whose coarsest grid is solved by one DD sweep over
8 x 8 subdomains) inside an FP64-class (double-float) FGMRES(10) with
delayed CGS2 to 1e-6 relative residual.  The four media are one batched context, so one step is
four solves.

Timing: W warm-up steps, then K steps timed with CUDA events on the solver's
stream, L2 flushed (a 512 MiB write) between steps outside the events;
barrier + synchronize around the timed loop; max over ranks.  N > 1 ranks
run independent replicas (weak scaling, no collective on the data path).

Also reported: e2e (the same solves through the C ABI with host buffers,
copies inside the timed region), the roofline of the dominant kernel timed
live with CUDA events, SM clocks sampled during the timed region, and the
CPU oracle timed on a bounded sample (``--impl reference`` times the oracle
alone on this workload).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "elastic Helmholtz solves/s to 1e-6 residual; stencil HBM GB/s vs peak"
SIGMAS = (0.25, 0.4, 0.45, 0.49)
N_GRID = 512
# The solver of the 512x512 line: MG-DD (Sec. 4), a 3-level V(1,1) cycle whose
# 128x128 coarsest grid is solved by one multicolour DD sweep over 8x8
# overlapping subdomains; 16-bit storage of the Galerkin stencils and of the
# coarse local inverses (the paper's half-precision inverses, Sec. 4), FP32
# arithmetic in the cycle, double-float FGMRES.
LEVELS = 3
ALPHA = 0.2
W_LEVELS = (0.75, 0.5)
CYCLE = 1                          # V(1,1)
COARSE_DD = (8, 8, 1)
COARSE_OVERLAP = 3
COARSE_FMT = 2                     # FP16 pairs
COEF_HALF = 1                      # FP16 pairs
ORTHO = 1                          # delayed CGS2 Arnoldi
WORKLOAD = ("2D heterogeneous media 512x512 (GRF corr 20, Vp 1.5-4.5, rho 1-2.5), Poisson "
            "0.25/0.4/0.45/0.49, 8 points per S-wavelength, 20-cell ABL; MG-DD preconditioner: complex64 "
            f"V(1,1) cycle ({LEVELS} levels, alpha {ALPHA}), coarsest 128x128 grid solved by one DD sweep over "
            f"8x8 subdomains (overlap {COARSE_OVERLAP}, dense local inverses), FP16 Galerkin tables and local "
            "inverses; FP64-class (double-float) FGMRES(10) with delayed CGS2 to 1e-6")


def default_kw():
    """Solver options of the default 512x512 line (the C ABI's ehs_opts fields)."""
    return dict(levels=LEVELS, alpha=ALPHA, w=list(W_LEVELS), prec=1, cycle=CYCLE, coarse_dd=COARSE_DD,
                coarse_dd_overlap=COARSE_OVERLAP, coarse_fmt=COARSE_FMT, coef_half=COEF_HALF, ortho=ORTHO)


# Roofline kernel of the default line: the MG-DD coarsest local products with the scatter-add
# (k_dense_apply_vs, the largest share of the solve in the ncu launch list); per launch (one
# colour) the live n_s x n_s entries of every subdomain inverse of the colour (4 B each, FP16
# pairs) + r read and the coarsest vector read and written at the live rows
ROOF = "coarse"
ROOF_KERNEL = ("k_dense_apply_vs<__half2> (MG-DD coarsest local products with the scatter-add: one colour = "
               "16 subdomain inverses x 4 media)")
# Galerkin level-1 apply (k_st_rows): 45 stored stencil coefficients of the half table (FP16 pairs,
# 4 B; 87 per row set, the mirrored ones read at the neighbour cell) + x 24 + y 24
ST_ROWS_L1_BYTES_PER_CELL = 45 * 4 + 24 + 24
# DRAM read + write bytes of one roofline-kernel launch (one colour) of the default line, from an
# ncu capture of the kernel as it stands (None whenever the kernel changes): mean of 7 warm launches
ROOF_TRAFFIC_C2 = 447.13e6 + 0.59e6

# Stencil kernels of the default line (the metric's "stencil HBM GB/s"), each timed through the
# C ABI call that launches it alone: algorithmic bytes per cell of the level it runs on (each
# input read once, each output written once; complex64 vectors 8 B per value, 3 values per cell).
#  fine sweep: one launch of the fused red-black sweep, x 24 + b 24 + x' 24 + mu and 1/(lambda+mu) 8
#    + the setup-time tables 28 (inverse diagonals of the two low faces 16, inverse Schur complement
#    8, vertex mean 4)
#  fine residual + restriction: one fused launch, x 24 + b 24 + mu and 1/(lambda+mu) 8 + the
#    setup-time tables 20 (face diagonals 16, vertex mean 4) + coarse r 6
#  level-1 rows: the Galerkin residual pass, the FP16 table in half storage (45 of the 87
#    coefficients per cell kept, K_c = K_c^T) x 4 B + x 24 + y 24
#  level-1 prolongation: x += P e, x 24 read + 24 written + e 6 (per level-1 cell)
STENCIL = (
    ("k_fine_sweep_tile (fine level, whole red-black sweep)", "sweep", 0, 108),
    ("k_fine_resid_restrict_tile (fine residual + restriction)", "resid_restrict", 0, 82),
    ("k_st_rows / k_st_rows2 <float,__half2,2,1,true> (Galerkin level 1, all rows, FP16 half table; the "
     "setup autotuner's launch shape)", "rows", 1, 45 * 4 + 48),
    ("k_prolong_add<float,2> (level 2 -> level 1 correction)", "prolong", 1, 54),
)


def media(seed=0):
    from paper_1806_11277_gb300 import synth
    return [synth.random_2d(n=N_GRID, sigma=s, seed=seed) for s in SIGMAS]


def small_case():
    """The default line's solver on 4 media of 256x256 (the same Poisson ratios): every
    kernel of the line with the same tile and subdomain shapes (coarsest 64x64 in 4x4
    subdomains of 16x16 cells, as the 128x128 coarsest grid's 8x8), its vectors and
    tables still larger than L2, a few GB on the device: the case ncu section captures
    run on."""
    from paper_1806_11277_gb300 import synth
    kw = default_kw()
    kw["coarse_dd"] = (4, 4, 1)
    return [synth.random_2d(n=256, sigma=s, seed=0) for s in SIGMAS], kw


_EXACT5W = dict(levels=5, alpha=0.4, w=[0.75, 0.5, 0.25, 0.25], cycle=2, coarse_dd=(1, 1, 1), coarse_fmt=0,
                coef_half=0)
_W5 = WORKLOAD.split("; MG-DD")[0] + ("; complex64 W(1,1) cycle (5 levels, alpha 0.4, damping 0.75/0.5/0.25/0.25), "
                                      "exact dense coarsest 32x32 solve (double-float inverse); FP64-class "
                                      "(double-float) FGMRES(10) to 1e-6")
_ROWS_C64 = "k_st_rows<float,float2,2,1> (Galerkin level 1, all rows, complex64 table)"
_ROWS_H = "k_st_rows<float,__half2,2,1> (Galerkin level 1, all rows, FP16 table)"

# Other workloads (bench.py --config NAME); "c2" above is the default line.
OTHER = {
    # 128^3 layered + random 3D medium, DD into 2x2x2 overlapping subdomains,
    # one shifted-Laplacian V-cycle per subdomain, complex64 preconditioner
    "c3": dict(
        workload=("3D layered+random medium 128^3 (5 layers Vp 1.5-4.5 x (1 + 0.1 GRF), Poisson 0.25-0.45, "
                  "rho = 0.25 Vp + 1.5), 8 points per S-wavelength, 16-cell ABL; DD 2x2x2 (overlap 4, "
                  "pad 8) with one complex64 5-level V(1,1) cycle per subdomain (damping 0.5/0.5/0.2/0.2) inside "
                  "double-float FGMRES(10)"),
        media=lambda: [__import__("paper_1806_11277_gb300.synth", fromlist=["x"]).layered_3d(
            n=128, seed=0, corr=10.0, abl=16)],
        kw=dict(levels=5, alpha=0.4, w=[0.5, 0.5, 0.2, 0.2], cycle=1, precond=1, dd=(2, 2, 2),
                dd_overlap=4, dd_pad=8, coarse_dd=(1, 1, 1), coarse_fmt=0, coef_half=0),
        roof_level=0, rows_l1_bytes=32 + 16 + 32,
        kernel="k_fine_apply<float,3> (fine K x: x 32 + coefficients 16 + y 32 B per cell)"),
    # batched multi-source 3D: 192^3, 8 x-forces on a surface line in one batch,
    # uneven 3x3x2 subdomains (shape groups per colour), complex64 V-cycles
    "c4": dict(
        workload=("3D layered+random medium 192^3, 8 x-forces on the line z = ABL+2, y = n/2 solved as one "
                  "batch; DD 3x3x2 (uneven subdomains, overlap 4, pad 8), one complex64 5-level V(1,1) per "
                  "subdomain, double-float FGMRES(10)"),
        media=lambda: [__import__("paper_1806_11277_gb300.synth", fromlist=["x"]).layered_3d(
            n=192, seed=0, corr=10.0, abl=16, nsrc=8)],
        nrhs=8,
        kw=dict(levels=5, alpha=0.4, w=[0.5, 0.5, 0.2, 0.2], cycle=1, precond=1, dd=(3, 3, 2),
                dd_overlap=4, dd_pad=8, nrhs=8, maxit=800, coarse_dd=(1, 1, 1), coarse_fmt=0, coef_half=0),
        roof_level=0, rows_l1_bytes=32 + 16 + 32,
        kernel="k_fine_apply<float,3> (fine K x: x 32 + coefficients 16 + y 32 B per cell)"),
    "c4b": None,   # filled below: c4 with BF16 Galerkin tables
    # the 512x512 workload with the 5-level W(1,1) cycle and the exact dense coarsest solve
    "c2w5": dict(workload=_W5, media=lambda: media(), kw=dict(_EXACT5W), rows_l1_bytes=87 * 8 + 24 + 24,
                 kernel=_ROWS_C64),
    # the default line with complex64 tables and complex64 local inverses (no 16-bit storage)
    "c2c64": dict(workload=WORKLOAD.replace("FP16 Galerkin tables and local inverses", "complex64 Galerkin "
                                            "tables and local inverses"),
                  media=lambda: media(), kw=dict(coarse_fmt=1, coef_half=0), roof="coarse",
                  kernel="k_dense_apply_vs<float2> (MG-DD coarsest local products with the scatter-add, complex64 inverses)"),
    # the default line in the plain FP64 GPU form: complex128 cycle, FP64 inverses, FP64 Krylov
    "c2f64": dict(workload=WORKLOAD.replace("complex64 V(1,1)", "complex128 V(1,1)").replace(
                      "FP16 Galerkin tables and local inverses", "FP64 Galerkin tables and local inverses").replace(
                      "FP64-class (double-float) FGMRES", "FP64 FGMRES") + "; plain FP64 GPU form",
                  media=lambda: media(), kw=dict(prec=0, coarse_fmt=0, coef_half=0), rows_l1_bytes=87 * 16 + 48 + 48,
                  kernel="k_st_rows<double,double2,2,1> (Galerkin level 1, all rows)"),
    # the default line with the MG-DD coarsest solve as one persistent launch per solve
    "c2p": dict(workload=WORKLOAD + "; MG-DD coarsest solve as one persistent launch (bounded grid barriers "
                "between the colours' residual and local-product phases) instead of graph-replayed per-colour "
                "launches", media=lambda: media(), kw=dict(coarse_persist=1), roof="coarse", kernel=ROOF_KERNEL),
    # the default line with the three-pass CGS2 Arnoldi instead of delayed CGS2
    "c2cgs2": dict(workload=WORKLOAD.replace("with delayed CGS2", "with CGS2 (three passes over the basis per "
                                            "Arnoldi step instead of two)"),
                   media=lambda: media(), kw=dict(ortho=0), roof="coarse", kernel=ROOF_KERNEL),
    # the default line with full cell-block Vanka
    "c2v": dict(workload=WORKLOAD + "; full (2d+1)^2 cell-block Vanka instead of the economic block",
                media=lambda: media(), kw=dict(vanka_full=1), roof="coarse", kernel=ROOF_KERNEL),
    # 4-level MG-DD with the W(1,1) cycle (coarsest 64x64 split 4x4)
    "c2dd4": dict(workload=WORKLOAD.split("; MG-DD")[0] + "; MG-DD: complex64 W(1,1) cycle (4 levels, alpha 0.4), "
                  "coarsest 64x64 grid split 4x4 (overlap 2), complex64 local inverses; double-float FGMRES(10)",
                  media=lambda: media(), kw=dict(levels=4, alpha=0.4, w=[0.75, 0.5, 0.25], cycle=2,
                                                 coarse_dd=(4, 4, 1), coarse_dd_overlap=2, coarse_fmt=1, coef_half=0),
                  roof="coarse", kernel="k_dense_apply_vs<float2> (MG-DD coarsest local products with the scatter-add, complex64 inverses)"),
    # the 64x64 homogeneous case: 3-level V-cycle, alpha 0.2, complex128
    "c1": dict(
        workload=("2D homogeneous 64x64, Vp 2, Vs 1, rho 1, 10 points per S-wavelength, 10-cell ABL, centred "
                  "x-force; 3-level V(1,1), alpha 0.2, complex128 FGMRES(10)"),
        media=lambda: [__import__("paper_1806_11277_gb300.synth", fromlist=["x"]).homogeneous_2d()],
        kw=dict(levels=3, alpha=0.2, w=[0.75, 0.5], cycle=1, prec=0, coarse_dd=(1, 1, 1), coarse_fmt=0, coef_half=0),
        rows_l1_bytes=87 * 16 + 48 + 48, kernel="k_st_rows<double,double2,2,1> (Galerkin level 1, all rows)"),
}


def rhs(meds, nrhs=1):
    """nrhs right-hand sides per medium (the medium's first nrhs sources)."""
    from paper_1806_11277_gb300 import synth
    out = []
    for m in meds:
        out += synth.point_rhs(m.shape, m.sources[:nrhs])
    return np.stack(out)


OTHER["c4b"] = dict(OTHER["c4"], workload=OTHER["c4"]["workload"] + "; Galerkin tables stored as BF16 pairs",
                    kw=dict(OTHER["c4"]["kw"], coef_half=2))
# adjoint-state gradient (FWI) workload: 256x256, 16 sources, 200 receivers; one step = forward
# solves of the 16 sources, receiver residual against data of the blob-perturbed true model,
# adjoint solves, fused gradient (solves/s counts forward and adjoint solves)
OTHER["c5"] = dict(
    workload=("2D adjoint-state gradient: 256x256 random medium (Poisson 0.45, GRF corr 20), 16 x-forces and "
              "200 u_x receivers on the line y = ABL+2, data from the true model (+5% Gaussian blob of "
              "radius 20 cells); one step = 16 forward solves + receiver residual + 16 adjoint solves + fused "
              "dJ/d(lambda, mu, rho); MG-DD preconditioner (3-level complex64 V(1,1), alpha 0.25, 64x64 "
              "coarsest grid split 4x4, overlap 3, FP16 tables and local inverses), double-float FGMRES(10)"),
    media=lambda: [__import__("paper_1806_11277_gb300.synth", fromlist=["x"]).fwi_2d()[0]],
    nrhs=16, fwi=True,
    kw=dict(nrhs=16, coarse_dd=(4, 4, 1)), roof="coarse",
    kernel="k_dense_apply_vs<__half2> (MG-DD coarsest local products with the scatter-add: one colour = 4 subdomain inverses x 16 sources)")

# DD-MG-DD (Sec. 4, the paper's 3D method): the same top-level DD, 4-level V(1,1) cycles per subdomain
# whose coarsest grids are themselves split 2x2x1 (overlap 2, FP16 local inverses), alpha 0.5
_DDMGDD = dict(levels=4, alpha=0.5, w=[0.5, 0.5, 0.2], coarse_dd=(2, 2, 1), coarse_dd_overlap=2, coarse_fmt=2,
               coef_half=1)
OTHER["c3dd"] = dict(OTHER["c3"], workload=OTHER["c3"]["workload"].replace(
    "with one complex64 5-level V(1,1) cycle per subdomain (damping 0.5/0.5/0.2/0.2)",
    "with one complex64 4-level V(1,1) cycle per subdomain (damping 0.5/0.5/0.2, alpha 0.5) whose coarsest "
    "grid is split 2x2x1 (DD-MG-DD, overlap 2, FP16 local inverses and tables)"),
    kw=dict(OTHER["c3"]["kw"], **_DDMGDD))
OTHER["c4dd"] = dict(OTHER["c4"], workload=OTHER["c4"]["workload"].replace(
    "one complex64 5-level V(1,1) per subdomain",
    "one complex64 4-level V(1,1) per subdomain (alpha 0.5) whose coarsest grid is split 2x2x1 (DD-MG-DD, "
    "overlap 2, FP16 local inverses and tables)"),
    kw=dict(OTHER["c4"]["kw"], **_DDMGDD))
OTHER["c4"]["kernel"] = OTHER["c4b"]["kernel"] = OTHER["c3"]["kernel"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 3 + i and r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(sm)}


# --------------------------------------------------------------- oracle leg
_ORACLE_CACHE = {}


def oracle_sample(meds, iters_per_sample, which=0):
    """Oracle (as it stands) FGMRES on one medium from a zero guess, iters_per_sample preconditioner
    applications (10 = one whole restart cycle: ten Arnoldi steps with their CGS2 passes, the
    x-update and the true residual); seconds per iteration.  The medium's operator and hierarchy
    are built once and reused (setup is not timed)."""
    from oracle import krylov, multigrid as mg, operators as op
    k = which % len(meds)
    if k not in _ORACLE_CACHE:
        med = meds[k]
        parts = op.parts_for(med)
        K = op.assemble_mixed(parts)
        H = mg.Hierarchy(op.assemble_mixed(parts, ALPHA), med.shape, LEVELS, w=list(W_LEVELS),
                         coarse_dd=(COARSE_DD[:2], COARSE_OVERLAP))
        q = op.slots_to_dofs(rhs([med])[0], med.shape)
        _ORACLE_CACHE[k] = (K, H, q)
    K, H, q = _ORACLE_CACHE[k]
    t, c = time.perf_counter(), time.process_time()
    _, info = krylov.fgmres(lambda v: K @ v, lambda v: H.cycle(v, gamma=CYCLE), q, m=10,
                            maxit=iters_per_sample, tol=1e-30)
    dt = time.perf_counter() - t
    _CPU_METER["wall"] += dt
    _CPU_METER["cpu"] += time.process_time() - c
    return dt / max(1, info["iters"]), info["iters"]


# wall and process CPU seconds of the timed oracle work (all threads of the process)
_CPU_METER = {"wall": 0.0, "cpu": 0.0}


def cores_used(meter):
    """Threads the timed oracle work kept busy on average: process CPU time / wall time."""
    return max(1, int(round(meter["cpu"] / meter["wall"]))) if meter["wall"] > 0 else 1


def oracle_dd_sample(med, kw, gpu_iters):
    """Bounded oracle sample of a 3D DD line (Algorithm DD with one shifted-Laplacian cycle per
    subdomain).  Outside the timer: the global operator K and the hierarchy of the largest padded
    subdomain.  Timed: ten oracle FGMRES iterations on K with the identity as preconditioner (the
    Krylov work and the operator product of an iteration: CGS2 over the growing basis, x-update,
    true residual), one global residual K x, and one cycle of that subdomain's shifted operator.
    One DD-preconditioned iteration = Krylov part + one residual per colour + one cycle per
    subdomain.  The oracle's own iteration count at this size is not available (its solve would
    take hours), so the GPU line's mean count is used; in the parity tests of the same DD forms
    (24^3 and 28 x 28 x 16) the counts are equal."""
    import itertools
    from oracle import dd as odd, krylov, multigrid as mg, operators as op
    shape = med.lam.shape
    d = len(shape)
    nsub = tuple(kw["dd"][d - 1 - a] for a in range(d))          # per numpy axis
    splits = [odd.split_axis(shape[a], nsub[a]) for a in range(d)]
    align = 2 ** (kw["levels"] - 1)
    subs = [odd.Subdomain(shape, si, splits, kw["dd_overlap"], kw["dd_pad"], align)
            for si in itertools.product(*[range(n) for n in nsub])]
    big = max(subs, key=lambda sd: int(np.prod(sd.shape)))
    ncol = len({sd.colour for sd in subs})
    parts = op.parts_for(med)
    K = op.assemble_mixed(parts)
    gamma = op.gamma_profile(shape, med.omega, med.abl_cells, 1.0, 0.01 * np.pi)
    lm = big.local_medium(med.lam, med.mu, med.rho, gamma, med.omega, 1.0)
    cdd = None
    if max(kw.get("coarse_dd", (1, 1, 1))) > 1:
        cdd = (tuple(kw["coarse_dd"][:d]), kw.get("coarse_dd_overlap", 2))
    H = mg.Hierarchy(op.assemble_mixed(op.Parts(*lm, med.omega, med.h), kw["alpha"]), big.shape, kw["levels"],
                     w=list(kw["w"])[:kw["levels"] - 1], coarse_dd=cdd)
    q = op.slots_to_dofs(synth_rhs(med), shape)
    rng = np.random.default_rng(0)
    rl = rng.standard_normal(H.K[0].shape[0]) + 0j
    meter = {"wall": 0.0, "cpu": 0.0}
    t, c = time.perf_counter(), time.process_time()
    krylov.fgmres(lambda v: K @ v, lambda v: v, q, m=10, maxit=10, tol=1e-30)
    t_kry = (time.perf_counter() - t) / 10
    t1 = time.perf_counter()
    _ = q - K @ q
    t_res = time.perf_counter() - t1
    t2 = time.perf_counter()
    H.cycle(rl)
    t_cyc = time.perf_counter() - t2
    meter["wall"] = time.perf_counter() - t
    meter["cpu"] = time.process_time() - c
    t_iter = t_kry + ncol * t_res + len(subs) * t_cyc
    mean_it = float(np.mean(gpu_iters))
    return {"value": 1.0 / (t_iter * mean_it), "unit": "solves/s", "cores": cores_used(meter),
            "threads_available": cpu_threads(), "kind": "oracle",
            "sample": (f"oracle on one source, setup excluded: 10 identity-preconditioned FGMRES iterations on "
                       f"the global K ({t_kry:.2f} s/iteration), one global residual ({t_res:.2f} s), one cycle of "
                       f"the largest subdomain {big.shape} ({t_cyc:.2f} s); per DD iteration {t_iter:.1f} s = "
                       f"Krylov + {ncol} residuals + {len(subs)} subdomain cycles; x the GPU line's mean count "
                       f"{mean_it:.1f} (the oracle's own count at this size is not available)")}


def synth_rhs(med):
    from paper_1806_11277_gb300 import synth
    return synth.point_rhs(med.shape, med.sources[:1])[0]


def oracle_iteration_counts():
    p = os.path.join(ROOT, "tests", "golden", "c2_oracle_iters.json")
    try:
        with open(p) as f:
            return json.load(f)["iters"]
    except Exception:
        return None


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        nt = [i.get("num_threads", 1) for i in threadpool_info()]
        return max(nt) if nt else 1
    except Exception:
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args):
    """--impl reference: the CPU oracle on this workload, per step a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    meds = media()
    iters = oracle_iteration_counts()
    per = []
    for s in range(args.warmup + args.steps):
        if s == args.warmup:
            _CPU_METER.update(wall=0.0, cpu=0.0)
        t_it, n_it = oracle_sample(meds, args.ref_iters, which=s)
        if s >= args.warmup:
            per.append((s % len(meds), t_it))
    mean_iters = float(np.mean(iters)) if iters else None
    t_iter = float(np.mean([t for _, t in per]))
    value = 1.0 / (t_iter * mean_iters) if mean_iters else None
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_iter * args.ref_iters * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [N_GRID, N_GRID], "media": len(SIGMAS),
                   "arithmetic": ("the oracle: FP64 throughout (scipy.sparse complex128 cycle and coarsest "
                                  "local solves, FGMRES(10) with CGS2)")},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores_used(_CPU_METER),
                         "threads_available": cpu_threads(), "kind": "oracle",
                         "sample": (f"{args.ref_iters} oracle FGMRES iterations per step on one medium "
                                    f"(media cycled; 10 = one whole restart cycle with its x-update and true "
                                    f"residual), setup excluded, seconds/iteration x the oracle's own mean "
                                    f"iteration count per solve ({mean_iters}) from tests/golden/c2_oracle_iters.json")},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _dofs_2d(v):
    """Slot layout (3, n_y, n_x) -> the oracle's DOF order (u_x interior faces, u_y interior faces,
    p; x fastest): index marshalling only, for comparing with stored oracle samples."""
    return np.concatenate([v[0][:, 1:].ravel(), v[1][1:, :].ravel(), v[2].ravel()])


def err_vs_oracle(u):
    """Per medium: the GPU solution against the FP64 oracle's at the DOFs stored in
    tests/golden/c2_oracle_samples.json (written by a script that calls only oracle/):
    max |u - u_oracle| / max |u_oracle| over the samples (relative to the largest entry of the
    oracle's whole solution), and the 2-norm over the samples relative to theirs."""
    p = os.path.join(ROOT, "tests", "golden", "c2_oracle_samples.json")
    try:
        with open(p) as f:
            media_s = json.load(f)["media"]
    except Exception:
        return None
    out = []
    for it, m in enumerate(media_s):
        x = _dofs_2d(u[it])
        idx = np.asarray(m["idx"])
        ref = np.asarray(m["re"]) + 1j * np.asarray(m["im"])
        d = x[idx] - ref
        out.append({"sigma": m["sigma"], "max_rel": float(np.abs(d).max() / m["maxabs"]),
                    "l2_rel_samples": float(np.linalg.norm(d) / np.linalg.norm(ref)), "samples": int(idx.size)})
    return {"reference": "FP64 oracle solutions at 1e-6 residual, sampled (tests/golden/c2_oracle_samples.json)",
            "media": out}


def fp64_form_sample(meds, q_host, stream, dev, flush, steps=3):
    """The same workload in the plain FP64 GPU form (complex128 cycle, FP64 tables and local
    inverses, FP64 FGMRES): a short timed sample of solves/s with the same timing rules."""
    import torch
    from paper_1806_11277_gb300 import ehs
    kw = default_kw()
    kw.update(prec=0, coarse_fmt=0, coef_half=0)
    with torch.cuda.stream(stream):
        S = ehs.solver_for(meds, stream=stream.cuda_stream, **kw)
    qd = torch.from_numpy(q_host).to(dev)
    ud = torch.zeros_like(qd)
    info = S.fgmres_solve(qd, ud)          # warm-up (graph capture)
    times = []
    for _ in range(steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = S.fgmres_solve(qd, ud)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    S.close()
    err = err_vs_oracle(ud.cpu().numpy())
    return {"value": len(meds) * steps / sum(times), "unit": "solves/s", "steps": steps,
            "iters": [i["iters"] for i in info], "dtype": "c128",
            "err_vs_oracle": err["media"] if err else None,
            "note": "plain FP64 GPU form of the same workload and solver (complex128 cycle, FP64 Galerkin "
                    "tables and MG-DD local inverses, FP64 FGMRES); one warm-up solve, CUDA events, L2 flushed"}


# ----------------------------------------------------------------- GPU leg
def max_over_ranks(total, dist, dev):
    """Whole-job time: the maximum of the ranks' timed totals (replicas, weak scaling)."""
    if not dist:
        return total
    import torch
    t = torch.tensor([total], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def run_gpu(args):
    import torch
    from paper_1806_11277_gb300 import ehs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream()
    cfg = OTHER.get(args.config)
    meds = media() if cfg is None else cfg["media"]()
    kw = default_kw()
    if cfg is not None:
        kw.update(cfg["kw"])
    if args.profile_small:
        if cfg is not None:
            raise SystemExit("--profile-small applies to the default line")
        meds, kw = small_case()
    nsolve = len(meds) * (1 if cfg is None else cfg.get("nrhs", 1))
    fwi = cfg is not None and cfg.get("fwi", False)
    if fwi:
        nsolve *= 2                       # forward and adjoint solves per step
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        S = ehs.solver_for(meds, stream=stream.cuda_stream, **kw)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    nrhs = 1 if cfg is None else cfg.get("nrhs", 1)
    q_host = rhs(meds, nrhs)
    qd = torch.from_numpy(q_host).to(dev)
    ud = torch.zeros_like(qd)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    roof_note = []

    def roofline_coarse():
        # roofline of the dominant kernel of the MG-DD line, the coarsest local products: one
        # launch = one colour (every subdomain of that colour, every item), events on the
        # solver's stream.  The complex64 form times ehs_coarse_local_add, the launch the solve
        # makes (k_dense_apply_vs: products and scatter-add, r read, x read and written per
        # live row); the FP64 form ehs_coarse_local_apply (k_dense_apply, r read, z written).
        ns, nloc, sizes = S.coarse_dims()
        c64 = kw["prec"] == ehs.EHS_C64
        eb = {0: 16, 1: 8, 2: 4, 3: 4}[kw.get("coarse_fmt", 0)] if c64 else 16
        vb = 8 if c64 else 16
        nx = kw["coarse_dd"][0]
        nsets = len(meds)
        r = torch.randn((S.items, ns, nloc), dtype=torch.complex64 if c64 else torch.complex128, device=dev)
        for q, n in enumerate(sizes):
            r[:, q, n:] = 0
        z = torch.zeros_like(r)
        xc = torch.zeros(tuple(S.level_shape(kw["levels"] - 1)), dtype=r.dtype, device=dev)
        cols = {}
        for q, n in enumerate(sizes):
            col = (q % nx) % 2 + 2 * ((q // nx) % 2)
            cols[col] = cols.get(col, 0) + nsets * n * n * eb + S.items * n * (3 if c64 else 2) * vb
        # Every launch reads more than L2 holds (the colour's inverses, ~445 MB), so no
        # flush is needed between them: per sample the four colours run back to back
        # between one pair of events, queued behind a read-only 512 MiB pass (which
        # leaves L2 clean and keeps host launch gaps outside the events).
        kt = []
        for rep in range(args.kernel_reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush.sum()
                e0.record(stream)
                for col in cols:
                    if c64:
                        S.coarse_local_add(col, r, xc)
                    else:
                        S.coarse_local_apply(col, r, z)
                e1.record(stream)
            e1.synchronize()
            kt.append(e0.elapsed_time(e1) / 1e3)
        tsum = statistics.median(kt)
        bsum = sum(cols.values())
        roof_note.append("the %d colour launches back to back per event pair (each reads > L2), median of %d "
                         "samples; per-launch time = sample / %d" % (len(cols), args.kernel_reps, len(cols)))
        return tsum / len(cols), bsum / len(cols), bsum / tsum / 1e9

    def roofline():
        if (cfg is None and ROOF == "coarse") or (cfg is not None and cfg.get("roof") == "coarse"):
            return roofline_coarse()
        # roofline of the dominant kernel family, the Galerkin-level stencil rows
        # (k_st_rows): one launch = ehs_op_apply on level 1 (all rows, every cell),
        # one launch per sample, L2 flushed before each, events on the solver's stream
        lvl = 1 if cfg is None else cfg.get("roof_level", 1)
        shp1 = S.level_shape(lvl)
        ncell1 = int(np.prod(shp1[2:])) * nsolve
        x1 = torch.randn(shp1, dtype=torch.complex64 if kw["prec"] == ehs.EHS_C64 else torch.complex128, device=dev)
        x1[:, 0, ..., 0] = 0         # boundary slots: u_k at i_k = 0
        if len(shp1) == 4:
            x1[:, 1, 0, :] = 0
        else:
            x1[:, 1, :, 0, :] = 0
            x1[:, 2, 0, :, :] = 0
        y1 = torch.zeros_like(x1)
        kt = []
        for r in range(args.kernel_reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                # the 512 MiB flush runs long enough that the events and the launch
                # are queued behind it: no host gap lands inside the events
                flush.fill_(1)
                e0.record(stream)
                S.op_apply(x1, y1, level=lvl)
                e1.record(stream)
            e1.synchronize()
            kt.append(e0.elapsed_time(e1) / 1e3)
        t_launch = statistics.median(kt)
        peak, peak_kind = peaks()
        alg = (ST_ROWS_L1_BYTES_PER_CELL if cfg is None else cfg["rows_l1_bytes"]) * ncell1
        achieved = alg / t_launch / 1e9
        return t_launch, alg, achieved

    def stencil_roofline():
        """Achieved HBM GB/s of each stencil kernel of the default line (STENCIL), timed with CUDA
        events on the solver's stream around the C ABI call that launches it, queued behind a
        read-only 512 MiB pass that empties L2, median of samples.  The sweep is timed as ehs_smooth with two
        sweeps (two launches, x -> t -> x; a single sweep would add a copy back into x), reported
        per launch."""
        if cfg is not None:
            return None
        peak, _ = peaks()
        shp = [S.level_shape(lv) for lv in range(kw["levels"])]

        def rnd(lv):
            v = torch.randn(shp[lv], dtype=torch.complex64, device=dev)
            v[:, 0, :, 0] = 0           # Dirichlet slots
            v[:, 1, 0, :] = 0
            return v
        x0, b0, x1, y1, e2 = rnd(0), rnd(0), rnd(1), rnd(1), rnd(2)
        rc1 = torch.zeros_like(x1)
        calls = {"sweep": (lambda: S.smooth(b0, x0, level=0, nsweeps=2), 2),
                 "resid_restrict": (lambda: S.residual_restrict(b0, x0, rc1, level=0), 1),
                 "rows": (lambda: S.op_apply(x1, y1, level=1), 1),
                 "prolong": (lambda: S.prolong_add(e2, x1, level=1), 1)}
        out = []
        for name, what, lvl, bpc in STENCIL:
            fn, nl = calls[what]
            ncell = int(np.prod(shp[lvl][2:])) * S.items
            kt = []
            for _ in range(args.kernel_reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    # a read-only 512 MiB pass: it evicts the kernel's data from L2 without leaving
                    # dirty lines whose write-back would land inside the timed launch, and runs
                    # long enough that the host-side call is queued before the events
                    flush.sum()
                    e0.record(stream)
                    fn()
                    e1.record(stream)
                e1.synchronize()
                kt.append(e0.elapsed_time(e1) / 1e3 / nl)
            t = statistics.median(kt)
            gbs = bpc * ncell / t / 1e9
            out.append({"kernel": name, "bytes_per_cell": bpc, "cells_per_launch": ncell,
                        "alg_bytes_per_launch": bpc * ncell, "launch_us": t * 1e6, "achieved": gbs,
                        "unit": "GB/s", "frac": gbs / peak, "launches_per_sample": nl})
        return out

    if args.roofline_only:              # the roofline kernel loop alone (for ncu captures)
        t_launch, alg, achieved = roofline()
        print(json.dumps({"roofline_kernel_us": t_launch * 1e6, "alg_bytes": alg, "achieved_gbs": achieved}))
        S.close()
        return 0

    def step():
        return S.fgmres_solve(qd, ud)

    if fwi:
        # observed data: the same sources solved in the true (blob-perturbed) model, before timing
        from paper_1806_11277_gb300 import synth
        _, true_med, (ry, rx) = synth.fwi_2d()
        with torch.cuda.stream(stream):
            St = ehs.solver_for([true_med], stream=stream.cuda_stream, **kw)
        dobs = torch.zeros_like(qd)
        St.fgmres_solve(qd, dobs)
        St.close()
        ryd = torch.as_tensor(ry, device=dev)
        rxd = torch.as_tensor(rx, device=dev)
        d_rec = dobs[:, 0, ryd, rxd].clone()
        gsrc = torch.zeros_like(qd)
        wd = torch.zeros_like(qd)
        grads = [torch.empty((len(meds),) + tuple(meds[0].shape), dtype=torch.float64, device=dev) for _ in range(3)]

        def step():
            with torch.cuda.stream(stream):
                info_f = S.fgmres_solve(qd, ud)
                # J = 1/2 sum |u_x(receivers) - d|^2: the adjoint source is the receiver residual
                gsrc[:, 0, ryd, rxd] = ud[:, 0, ryd, rxd] - d_rec
                S.adjoint_solve(gsrc, wd)
                S.gradient(ud, wd, grads)
            return info_f

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()
    if args.profile_step or args.profile_small:   # one solve step between profiler start/stop
        torch.cuda.cudart().cudaProfilerStart()
        step()
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        S.close()
        return 0
    if dist:
        dist.barrier()
    clocks = ClockSampler(dev.index)
    clocks.start()
    l0 = ehs.kernel_launches()
    times = []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    torch.cuda.synchronize()
    launches = ehs.kernel_launches() - l0
    clk = clocks.stop()
    total = max_over_ranks(sum(times), dist, dev)
    solves = nsolve * args.steps * world
    value = solves / total
    its = [i["iters"] for i in info]
    relres = [i["relres"] for i in info]

    # e2e: same solves through the C ABI with host buffers (copies inside)
    q_pin = torch.from_numpy(q_host).pin_memory().numpy()
    u_pin = torch.zeros(q_host.shape, dtype=torch.complex128).pin_memory().numpy()
    e2e_t = []
    h2d, d2h = int(q_host.nbytes), int(q_host.nbytes)
    if fwi:
        q_src = torch.from_numpy(q_host).pin_memory()
        g_host = [torch.empty(g.shape, dtype=g.dtype).pin_memory() for g in grads]
        d2h = int(sum(g.numel() * 8 for g in grads))
    for _ in range(max(1, min(args.steps, 5))):
        flush.fill_(1)
        torch.cuda.synchronize()
        t = time.perf_counter()
        if fwi:    # sources in from pinned host memory, gradient back out
            with torch.cuda.stream(stream):
                qd.copy_(q_src, non_blocking=True)
            step()
            with torch.cuda.stream(stream):
                for gh, g in zip(g_host, grads):
                    gh.copy_(g, non_blocking=True)
            stream.synchronize()
        else:
            S.fgmres_solve(q_pin, u_pin)
        e2e_t.append(time.perf_counter() - t)
    # median over the calls: one call slowed by the host (page faults, scheduling) would pull a mean
    e2e_val = nsolve * world / statistics.median(e2e_t)

    t_launch, alg, achieved = roofline()
    peak, peak_kind = peaks()
    stencil = stencil_roofline()
    err_o = err_vs_oracle(ud.cpu().numpy()) if cfg is None else None

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        # arithmetic of the path: complex64 preconditioner with a double-float (FP32-pair) Krylov
        # solve in the mixed form, complex128 everywhere in the plain FP64 form
        "dtype": "c128" if kw.get("prec", 1) == 0 else "c64+df64", "data": "synthetic",
        "arithmetic": ("complex128 cycle and FP64 FGMRES (plain FP64 form)" if kw.get("prec", 1) == 0 else
                       "complex64 cycle with FP32 accumulation; Galerkin tables stored as %s, coarsest "
                       "inverses as %s; FGMRES vectors, operator, Arnoldi and true residual in double-float "
                       "(FP32 pairs, about 48-bit significands; no IEEE FP64 on the path)" % (
                           ["complex64", "FP16 pairs", "BF16 pairs"][kw.get("coef_half", 0)],
                           ["double-float", "complex64", "FP16 pairs", "BF16 pairs"][kw.get("coarse_fmt", 0)])),
        "config": {"name": args.config, "workload": WORKLOAD if cfg is None else cfg["workload"],
                   "grid": list(meds[0].shape), "media": nsolve,
                   "sigmas": list(SIGMAS) if cfg is None else None, "levels": kw["levels"],
                   "alpha": kw["alpha"], "cycle": "W(1,1)" if kw["cycle"] == 2 else "V(1,1)",
                   "krylov": "FGMRES(10), " + ("double-float (FP64-class)" if kw["prec"] == 1 else "FP64")
                   + " vectors and operator, " + ("delayed CGS2" if kw["prec"] == 1 and kw.get("ortho", 1)
                                                  else "CGS2"), "precond_dtype": "complex64" if kw["prec"] == 1 else "complex128",
                   "coarsest": ("MG-DD %s subdomains, overlap %d" % ("x".join(map(str, kw["coarse_dd"][:2])),
                                                                   kw.get("coarse_dd_overlap", 2))
                                if max(kw.get("coarse_dd", (1,))) > 1 else "exact dense inverse"),
                   "storage": {"galerkin_tables": ["complex", "FP16", "BF16"][kw.get("coef_half", 0)],
                               "coarsest_inverses": ["double-float", "complex64", "FP16", "BF16"][kw.get("coarse_fmt", 0)]
                               if kw["prec"] == 1 else "FP64"},
                   "l2": "flushed between steps (512 MiB write)", "parallelism": f"replicas x{world}"},
        "iters": its, "relres": relres, "setup_s": setup_s,
        "gridpoints_x_iters_per_s": float(np.prod(meds[0].shape) * sum(its) * args.steps * world / total),
        "e2e": {"value": e2e_val, "unit": "solves/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": ROOF_KERNEL if cfg is None else cfg["kernel"],
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs",
                     "traffic": args.traffic if args.traffic is not None else
                     (ROOF_TRAFFIC_C2 if cfg is None else None), "alg_bytes_per_launch": alg,
                     "launch_us": t_launch * 1e6,
                     "timing": roof_note[-1] if roof_note else
                     "one launch per event pair, queued behind a 512 MiB L2-flushing write"},
        "clocks": clk,
    }
    if stencil:
        line["roofline"]["stencil"] = stencil
    if err_o:
        line["err_vs_oracle"] = err_o
    if cfg is None and not args.no_fp64_form:
        line["fp64_form"] = fp64_form_sample(meds, q_host, stream, dev, flush)
    if rank == 0 and world == 1 and not args.no_cpu and cfg is None:
        iters_o = oracle_iteration_counts()
        t_it = []
        _CPU_METER.update(wall=0.0, cpu=0.0)
        for s in range(len(SIGMAS)):
            ti, _ = oracle_sample(meds, args.cpu_iters, which=s)
            t_it.append(ti)
        mean_iters = float(np.mean(iters_o)) if iters_o else float(np.mean(its))
        src = "tests/golden/c2_oracle_iters.json" if iters_o else "this run's GPU counts"
        cpu_val = 1.0 / (float(np.mean(t_it)) * mean_iters)
        line["cpu_baseline"] = {
            "value": cpu_val, "unit": "solves/s", "cores": cores_used(_CPU_METER),
            "threads_available": cpu_threads(), "kind": "oracle",
            "sample": (f"{args.cpu_iters} oracle FGMRES iterations (one whole restart cycle: Arnoldi steps, "
                       f"x-update and true residual) on each of the 4 media, setup excluded; seconds/iteration "
                       f"x mean iterations per solve ({mean_iters:.1f}, {src})")}
    if rank == 0 and world == 1 and not args.no_cpu and cfg is not None and kw.get("precond", 0) == 1 \
            and len(meds[0].shape) == 3:
        line["cpu_baseline"] = oracle_dd_sample(meds[0], kw, its)
    if rank == 0 and world == 1 and not args.no_cpu and args.config == "c1":
        # the 64x64 case is small enough for whole oracle solves (3-level V(1,1), alpha 0.2)
        from oracle import krylov, multigrid as mg, operators as op
        med = meds[0]
        parts = op.parts_for(med)
        K = op.assemble_mixed(parts)
        H = mg.Hierarchy(op.assemble_mixed(parts, kw["alpha"]), med.shape, kw["levels"], w=list(kw["w"]))
        qo = op.slots_to_dofs(q_host[0], med.shape)
        t, c = time.perf_counter(), time.process_time()
        reps = 3
        for _ in range(reps):
            krylov.fgmres(lambda v: K @ v, H.cycle, qo, m=10)
        wall = time.perf_counter() - t
        meter = {"wall": wall, "cpu": time.process_time() - c}
        cpu_val = reps / wall
        line["cpu_baseline"] = {"value": cpu_val, "unit": "solves/s", "cores": cores_used(meter),
                                "threads_available": cpu_threads(), "kind": "oracle",
                                "sample": f"{reps} whole oracle solves of the 64x64 case (hierarchy built beforehand)"}
    S.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40,
                    help="timed steps (the default keeps the 512x512 line's timed region near 1.3 s, so the "
                         "clock sampler sees several samples)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ehs", choices=["ehs", "reference"])
    ap.add_argument("--config", default="c2", choices=["c2"] + sorted(OTHER),
                    help="c2: the 512x512 four-Poisson-ratio line (default); c3: 3D 128^3 DD-MG; c1: 64x64")
    ap.add_argument("--kernel-reps", type=int, default=20)
    ap.add_argument("--cpu-iters", type=int, default=10,
                    help="oracle iterations per medium in the CPU baseline (10 = one whole restart cycle)")
    ap.add_argument("--ref-iters", type=int, default=10)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the roofline kernel from an ncu capture "
                         "(default: the capture of the current kernel for the c2 line)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="skip the short timed sample of the plain FP64 GPU form of the default line")
    ap.add_argument("--roofline-only", action="store_true",
                    help="skip the solves; only the roofline kernel timing loop (for ncu captures)")
    ap.add_argument("--profile-step", action="store_true",
                    help="run warm-up, then one step between cudaProfilerStart/Stop and exit")
    ap.add_argument("--profile-small", action="store_true",
                    help="as --profile-step, on the small case of the default line's kernels (small_case(): "
                         "4 media of 256x256, a few GB on the device) for ncu section captures")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
