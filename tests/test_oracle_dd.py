"""Structural pins of the oracle's Algorithm DD pieces (Sec. 2.3, Sec. 4; no GPU).

A non-square grid and an uneven split are used so that a swapped axis, an
off-by-one in the overlap or the padding, or a misplaced absorbing ramp fails:

* the local operator of every padded subdomain, restricted to the DOFs whose
  stencil stays inside Omega_i, equals the global operator's rows mapped
  through the subdomain's index maps (same medium, same attenuation there);
* the padding holds a clamped copy of the medium and gamma grows by
  omega * dd_abl_max * (depth / pad)^2, reaching omega * dd_abl_max at the
  outer cell; no padding on sides at the domain boundary;
* every padded extent is a multiple of the coarsening factor 2^(levels-1);
* with exact subdomain solves the iteration count rises as the domain is
  split more aggressively (the trend of Table DDexact).
"""
import itertools

import numpy as np

from oracle import dd, operators as op
from paper_1806_11277_gb300 import synth

SHAPE = (40, 48)                  # (n_y, n_x)
NSUB = (2, 3)                     # per numpy axis
OVERLAP, PAD, LEVELS, DD_ABL = 3, 4, 3, 1.0


def _subdomains(med):
    splits = [dd.split_axis(SHAPE[a], NSUB[a]) for a in range(2)]
    for sidx in itertools.product(*[range(n) for n in NSUB]):
        yield dd.Subdomain(SHAPE, sidx, splits, OVERLAP, PAD, 2 ** (LEVELS - 1))


def test_local_operator_equals_global_rows_inside_omega():
    med = synth.random_2d(n=SHAPE[0], nx=SHAPE[1], sigma=0.4, seed=2, corr=5.0, abl=6)
    parts = op.parts_for(med)
    K = op.assemble_mixed(parts).tocsr()
    gamma = op.gamma_profile(SHAPE, med.omega, med.abl_cells)
    nchecked = 0
    for sd in _subdomains(med):
        lm = sd.local_medium(med.lam, med.mu, med.rho, gamma, med.omega, DD_ABL)
        Kl = op.assemble_mixed(op.Parts(*lm, med.omega, med.h)).tocsr()
        loc, glo = sd.index_maps(SHAPE)
        g2l = -np.ones(K.shape[0], dtype=np.int64)
        g2l[glo] = loc
        # slots whose cells lie at least 2 cells inside Omega_i on every interface side
        lidx = dd.slot_dof_index(sd.shape)
        keep = np.ones(sd.shape, dtype=bool)
        for a in range(2):
            l = np.arange(sd.shape[a])
            lo = sd.pad_lo[a] + (2 if sd.pad_lo[a] else 0)
            hi = sd.shape[a] - sd.pad_hi[a] - (2 if sd.pad_hi[a] else 0)
            sh = [1, 1]
            sh[a] = sd.shape[a]
            keep &= ((l >= lo) & (l < hi)).reshape(sh)
        rows_l = np.concatenate([lidx[c][keep & (lidx[c] >= 0)] for c in range(3)])
        l2g = -np.ones(Kl.shape[0], dtype=np.int64)
        l2g[loc] = glo
        rows_g = l2g[rows_l]
        assert (rows_g >= 0).all()
        A = Kl[rows_l].toarray()
        B = K[rows_g].toarray()
        # every global column these rows touch is inside Omega_i, in the same place
        cols = np.nonzero(np.abs(B).sum(0))[0]
        assert (g2l[cols] >= 0).all()
        Bl = np.zeros_like(A)
        Bl[:, g2l[cols]] = B[:, cols]
        assert np.abs(A - Bl).max() <= 1e-12 * np.abs(B).max()
        nchecked += rows_l.size
    assert nchecked > 2000


def test_padding_medium_and_absorbing_ramp():
    med = synth.random_2d(n=SHAPE[0], nx=SHAPE[1], sigma=0.4, seed=2, corr=5.0, abl=6)
    gamma = op.gamma_profile(SHAPE, med.omega, med.abl_cells)
    for sd in _subdomains(med):
        lam, mu, rho, gl = sd.local_medium(med.lam, med.mu, med.rho, gamma, med.omega, DD_ABL)
        assert all(n % 2 ** (LEVELS - 1) == 0 for n in sd.shape)
        for a in range(2):
            assert (sd.pad_lo[a] > 0) == (sd.om_lo[a] > 0) and (sd.pad_hi[a] > 0) == (sd.om_hi[a] < SHAPE[a])
            assert sd.pad_lo[a] in (0,) or sd.pad_lo[a] >= PAD
            assert sd.pad_hi[a] in (0,) or sd.pad_hi[a] >= PAD
        ylo, xlo = sd.pad_lo
        ny, nx = sd.om_hi[0] - sd.om_lo[0], sd.om_hi[1] - sd.om_lo[1]
        core = (slice(ylo, ylo + ny), slice(xlo, xlo + nx))
        gsl = (slice(sd.om_lo[0], sd.om_hi[0]), slice(sd.om_lo[1], sd.om_hi[1]))
        assert np.array_equal(lam[core], med.lam[gsl]) and np.array_equal(gl[core], gamma[gsl])
        # clamped copy: every padding cell repeats the nearest Omega_i cell
        yy = np.clip(np.arange(sd.shape[0]) - ylo, 0, ny - 1) + sd.om_lo[0]
        xx = np.clip(np.arange(sd.shape[1]) - xlo, 0, nx - 1) + sd.om_lo[1]
        assert np.array_equal(mu, med.mu[np.ix_(yy, xx)]) and np.array_equal(rho, med.rho[np.ix_(yy, xx)])
        extra = gl - gamma[np.ix_(yy, xx)]
        assert np.allclose(extra[core], 0.0, atol=0)
        # outermost padding cell of an interface side: depth = pad, extra = omega * dd_abl_max
        if sd.pad_lo[1]:
            col = extra[ylo:ylo + ny, 0]
            assert np.allclose(col, med.omega * DD_ABL, rtol=1e-14)
            inner = extra[ylo:ylo + ny, sd.pad_lo[1] - 1]           # depth 1 of pad_lo
            assert np.allclose(inner, med.omega * DD_ABL / sd.pad_lo[1] ** 2, rtol=1e-14)
        if sd.pad_hi[0]:
            row = extra[-1, xlo:xlo + nx]
            assert np.allclose(row, med.omega * DD_ABL, rtol=1e-14)


def test_exact_dd_deteriorates_with_aggressive_splitting():
    """The trend of Table DDexact (exact subdomain solves with absorbing
    interface padding): on a shallow, wide 2D model at 12 points per
    S-wavelength the FGMRES count grows with every halving of the subdomains
    along x, and the 16 x 1 split needs several times the 2 x 1 count (the
    paper: 28 -> 130 on its smallest grid)."""
    from oracle import krylov
    ny, nx = 32, 128
    med = synth.random_2d(n=ny, nx=nx, sigma=0.3, seed=0, corr=8.0, abl=8, ppw=12.0)
    med.sources = [(0, (ny // 2, nx // 2))]
    K = op.assemble_mixed(op.parts_for(med))
    q = op.slots_to_dofs(synth.point_rhs(med.shape, med.sources)[0], med.shape)
    its = []
    for sx in (2, 4, 8, 16):
        D = dd.DD(med, (1, sx), 4, 8, 2, 0.05, local="exact")
        _, info = krylov.fgmres(lambda v: K @ v, D.apply, q, maxit=300)
        assert info["converged"], sx
        its.append(info["iters"])
    assert all(a < b for a, b in zip(its, its[1:])), its
    assert its[-1] >= 4 * its[0], its


def test_near_equal_splits_agree():
    """Both DD layers split an axis the same way: nearly equal consecutive
    parts, the larger ones first, covering the axis exactly."""
    from oracle import multigrid as mg
    for n in range(1, 70):
        for s in range(1, min(n, 17) + 1):
            e = dd.split_axis(n, s)
            assert list(e) == list(mg.near_equal_edges(n, s))
            sizes = np.diff(e)
            assert e[0] == 0 and e[-1] == n and sizes.max() - sizes.min() <= 1
            assert np.all(np.diff(sizes) <= 0)


def _shape_groups(shape, nsub, overlap, pad, levels):
    """Padded subdomain shapes of each colour (Algorithm DD geometry)."""
    splits = [dd.split_axis(shape[a], nsub[a]) for a in range(len(shape))]
    groups = {}
    for sidx in itertools.product(*[range(n) for n in nsub]):
        sd = dd.Subdomain(shape, sidx, splits, overlap, pad, 2 ** (levels - 1))
        groups.setdefault(sd.colour, set()).add(sd.shape)
    return groups


def test_uneven_parity_splits_have_several_shape_groups():
    """The uneven splits of the GPU parity tests (44 x 32 split 3 x 3, overlap 2,
    pad 4; 28 x 28 x 16 split 3 x 3 x 2, overlap 3, pad 4; 3 levels) give some
    colour several padded shapes, so the library's per-colour shape groups
    (one batched hierarchy per shape) are exercised, and every shape divides by
    the coarsening factor."""
    g2 = _shape_groups((32, 44), (3, 3), 2, 4, 3)
    g3 = _shape_groups((16, 28, 28), (2, 3, 3), 3, 4, 3)
    assert max(len(v) for v in g2.values()) == 4 and len(g2) == 4
    assert max(len(v) for v in g3.values()) == 4 and len(g3) == 8
    for g in (g2, g3):
        for shapes in g.values():
            assert all(s % 4 == 0 for sh in shapes for s in sh)
