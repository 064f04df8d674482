"""The seeded input generators follow the stated recipe (no GPU).

* wave speeds: Vp = sqrt((lambda + 2 mu) / rho), Vs = sqrt(mu / rho) (Sec. 2.1)
  and the Poisson ratio sigma = lambda / (2 (lambda + mu)) come back exactly,
* 2D random media: Vp spans [1.5, 4.5] and rho [1, 2.5] (affine maps of two
  independent smooth fields), omega gives 8 points per shortest S-wavelength,
  the field is smooth on the correlation length,
* 3D layered media: five layers with Vp 1.5 .. 4.5 perturbed by at most 10 %,
  Poisson ratio 0.25 .. 0.45 over the layers, rho = 0.25 Vp + 1.5 (Sec. 6.3),
* the 64x64 homogeneous case: mu = 1, lambda = 2, rho = 1, omega = 0.2 pi,
* the same seed gives the same medium; another seed another one.
"""
import math

import numpy as np
import pytest

from paper_1806_11277_gb300 import synth


def _speeds(m):
    vp = np.sqrt((m.lam + 2 * m.mu) / m.rho)
    vs = np.sqrt(m.mu / m.rho)
    return vp, vs


@pytest.mark.parametrize("sigma", [0.25, 0.4, 0.45, 0.49])
def test_random_2d_recipe(sigma):
    m = synth.random_2d(n=128, sigma=sigma, seed=0, corr=8.0, abl=10)
    vp, vs = _speeds(m)
    assert abs(vp.min() - 1.5) < 1e-12 and abs(vp.max() - 4.5) < 1e-12
    assert abs(m.rho.min() - 1.0) < 1e-12 and abs(m.rho.max() - 2.5) < 1e-12
    pois = m.lam / (2 * (m.lam + m.mu))
    assert np.allclose(pois, sigma, rtol=0, atol=1e-12)
    assert math.isclose(m.omega, 2 * math.pi * vs.min() / 8.0, rel_tol=1e-14)
    # the shortest S-wavelength 2 pi Vs_min / omega spans 8 cells
    assert math.isclose(2 * math.pi * vs.min() / m.omega, 8.0, rel_tol=1e-14)
    # density is an independent field: not an affine function of Vp
    assert abs(np.corrcoef(vp.ravel(), m.rho.ravel())[0, 1]) < 0.9
    # smooth on the correlation length: neighbouring cells differ far less than the range
    assert np.abs(np.diff(vp, axis=1)).max() < 0.15 * 3.0
    k, (iy, ix) = m.sources[0]
    assert k == 0 and iy == m.abl_cells + 2 and ix == 64


def test_random_2d_seeded():
    a = synth.random_2d(n=64, seed=3, corr=6.0, abl=8)
    b = synth.random_2d(n=64, seed=3, corr=6.0, abl=8)
    c = synth.random_2d(n=64, seed=4, corr=6.0, abl=8)
    assert np.array_equal(a.lam, b.lam) and np.array_equal(a.rho, b.rho) and a.omega == b.omega
    assert not np.allclose(a.lam, c.lam)


def test_layered_3d_recipe():
    n = 40
    m = synth.layered_3d(n=n, seed=1, corr=4.0, abl=4, nsrc=3)
    vp, vs = _speeds(m)
    layer = np.minimum((np.arange(n) * 5) // n, 4)
    base = np.linspace(1.5, 4.5, 5)[layer][:, None, None]
    assert np.abs(vp / base - 1).max() <= 0.1 + 1e-12
    assert np.abs(vp / base - 1).max() >= 0.1 - 1e-12           # max|g| = 1 is reached
    assert np.allclose(m.rho, 0.25 * vp + 1.5, rtol=1e-13)
    pois = m.lam / (2 * (m.lam + m.mu))
    sig = np.linspace(0.25, 0.45, 5)[layer][:, None, None]
    assert np.allclose(pois, np.broadcast_to(sig, pois.shape), atol=1e-12)
    assert math.isclose(2 * math.pi * vs.min() / m.omega, 8.0, rel_tol=1e-14)
    assert len(m.sources) == 3 and all(k == 0 and idx[0] == 6 and idx[1] == n // 2 for k, idx in m.sources)


def test_homogeneous_2d_case():
    m = synth.homogeneous_2d()
    assert m.shape == (64, 64)
    assert np.all(m.mu == 1.0) and np.all(m.lam == 2.0) and np.all(m.rho == 1.0)
    assert math.isclose(m.omega, 0.2 * math.pi, rel_tol=1e-15)
    assert m.abl_cells == 10 and m.sources == [(0, (32, 32))]


def test_point_rhs_unit_force():
    shape = (6, 8)
    q = synth.point_rhs(shape, [(0, (2, 3)), (1, (4, 5))])
    assert len(q) == 2 and q[0].shape == (3, 6, 8)
    assert q[0][0, 2, 3] == 1 and np.count_nonzero(q[0]) == 1
    assert q[1][1, 4, 5] == 1 and np.count_nonzero(q[1]) == 1
    assert not q[0][2].any()                                   # zero pressure block
