"""Seeded synthetic media and sources for the elastic Helmholtz solver.

This module produces inputs only: cell-centred Lame parameters and density,
the angular frequency, and point-force right-hand sides.  It holds none of
the solver's arithmetic (no operator, no absorbing layer, no multigrid), so
both the CUDA path and the CPU oracle can be fed from it.

Grid convention (shared with the C ABI): a 2D grid has shape (n_y, n_x), a
3D grid (n_z, n_y, n_x); x is the fastest axis.  Direction k = 0, 1, 2 means
x, y, z.  The last axis listed in ``n`` tuples below is always x, i.e. the
``shape`` tuple is the numpy array shape.

Velocity-to-Lame conversion follows the definitions of the two wave speeds in
Sec. 2.1 of the paper: Vp = sqrt((lambda + 2 mu) / rho), Vs = sqrt(mu / rho).
The 3D density rule rho = 0.25 Vp + 1.5 is the one quoted in Sec. 6.3.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np
from scipy import ndimage


@dataclass
class Medium:
    """One synthetic problem: media on cells, frequency, spacing, sources."""
    lam: np.ndarray          # cell-centred lambda, array shape = grid shape
    mu: np.ndarray           # cell-centred mu
    rho: np.ndarray          # cell-centred rho
    omega: float
    h: float
    abl_cells: int
    sources: list = field(default_factory=list)   # list of (k, index tuple) unit point forces
    name: str = ""

    @property
    def shape(self):
        return self.lam.shape

    @property
    def dim(self):
        return self.lam.ndim


def lame_from_velocities(vp, vs, rho):
    """mu = rho Vs^2 and lambda = rho Vp^2 - 2 mu (wave-speed definitions, Sec. 2.1)."""
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    return lam, mu


def vs_from_poisson(vp, sigma):
    """Vs for a given Poisson ratio sigma = lambda / (2 (lambda + mu)) (Sec. 6.1)."""
    return vp * np.sqrt((1.0 - 2.0 * sigma) / (2.0 - 2.0 * sigma))


def gaussian_random_field(shape, corr, seed):
    """White noise smoothed by a Gaussian kernel exp(-r^2 / (2 corr^2)); mean 0."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(shape)
    g = ndimage.gaussian_filter(g, sigma=corr, mode="reflect")
    return g - g.mean()


def _affine(g, lo, hi):
    gmin, gmax = float(g.min()), float(g.max())
    return lo + (hi - lo) * (g - gmin) / (gmax - gmin)


def homogeneous_2d(n=64, vp=2.0, vs=1.0, rho=1.0, ppw=10.0, abl=10, h=1.0):
    """Constant medium; omega set for ``ppw`` points per S-wavelength.

    The default is the 64 x 64 case with Vp = 2, Vs = 1, rho = 1 (Poisson 1/3)
    and a unit x-force on the centred u_1 face.
    """
    shape = (n, n)
    vp_a = np.full(shape, vp)
    vs_a = np.full(shape, vs)
    rho_a = np.full(shape, rho)
    lam, mu = lame_from_velocities(vp_a, vs_a, rho_a)
    omega = 2.0 * math.pi * vs / (ppw * h)
    src = [(0, (n // 2, n // 2))]       # (component k, (iy, ix))
    return Medium(lam, mu, rho_a, omega, h, abl, src, name=f"homog{n}")


def constant_2d(ny, nx, lam, mu, rho, omega, abl, h=1.0, sources=None):
    """Constant-coefficient medium with explicit Lame values (test helper)."""
    shape = (ny, nx)
    return Medium(np.full(shape, float(lam)), np.full(shape, float(mu)),
                  np.full(shape, float(rho)), float(omega), h, abl,
                  sources if sources is not None else [(0, (ny // 2, nx // 2))],
                  name=f"const{ny}x{nx}")


def random_2d(n=512, sigma=0.25, seed=0, corr=20.0, ppw=8.0, abl=20, h=1.0,
              vp_range=(1.5, 4.5), rho_range=(1.0, 2.5), nx=None):
    """Heterogeneous 2D medium from smooth Gaussian random fields.

    Vp in [1.5, 4.5] and rho in [1, 2.5] from two independent fields (seed and
    seed + 1000), correlation length ``corr`` cells; Vs from the Poisson ratio;
    omega for ``ppw`` points per shortest S-wavelength; one x-force at the
    middle of the first row below the absorbing layer.
    """
    nx = n if nx is None else nx
    shape = (n, nx)
    vp = _affine(gaussian_random_field(shape, corr, seed), *vp_range)
    rho = _affine(gaussian_random_field(shape, corr, seed + 1000), *rho_range)
    vs = vs_from_poisson(vp, sigma)
    lam, mu = lame_from_velocities(vp, vs, rho)
    omega = 2.0 * math.pi * float(vs.min()) / (ppw * h)
    src = [(0, (abl + 2, nx // 2))]
    return Medium(lam, mu, rho, omega, h, abl, src, name=f"rand{n}_s{sigma}_seed{seed}")


def fwi_2d(n=256, sigma=0.45, seed=0, nsrc=16, nrec=200, blob=0.05, radius=20.0, corr=20.0, ppw=8.0, abl=20):
    """Adjoint-state gradient workload: a base medium (``random_2d``) with
    ``nsrc`` x-forces on the line y = abl + 2, x evenly spaced over the
    interior; the true medium scales the wave speeds by (1 + blob * b), b a
    Gaussian bump of ``radius`` cells at the centre (lambda and mu scale by
    (1 + blob * b)^2, rho unchanged); ``nrec`` receivers (u_x faces) on the same
    line.  Returns (base, true, receivers) with receivers as (y, x) index
    arrays."""
    base = random_2d(n=n, sigma=sigma, seed=seed, corr=corr, ppw=ppw, abl=abl)
    lo, hi = abl + 2, n - abl - 2
    xs = np.linspace(lo, hi, nsrc).round().astype(int)
    base.sources = [(0, (abl + 2, int(x))) for x in xs]
    yy, xx = np.indices(base.shape)
    bump = np.exp(-((yy - n / 2) ** 2 + (xx - n / 2) ** 2) / (2.0 * radius ** 2))
    f = (1.0 + blob * bump) ** 2
    true = Medium(base.lam * f, base.mu * f, base.rho.copy(), base.omega, base.h, base.abl_cells,
                  list(base.sources), name=base.name + "_true")
    rx = np.linspace(lo, hi, nrec).round().astype(int)
    ry = np.full(nrec, abl + 2)
    return base, true, (ry, rx)


def layered_3d(n=128, seed=0, corr=10.0, ppw=8.0, abl=16, h=1.0, nlayers=5,
               sigma_range=(0.25, 0.45), pert=0.1, nsrc=1):
    """3D layered medium: 5 horizontal layers in z with Vp 1.5 .. 4.5, each
    perturbed by (1 + pert * g) with g a Gaussian random field scaled to
    max|g| = 1; Poisson ratio linear over the layers; rho = 0.25 Vp + 1.5.
    ``nsrc`` x-forces on the line z = abl + 2, y = n / 2."""
    shape = (n, n, n)
    vp_layers = np.linspace(1.5, 4.5, nlayers)
    sig_layers = np.linspace(*sigma_range, nlayers)
    z = np.arange(n)
    layer = np.minimum((z * nlayers) // n, nlayers - 1)
    g = gaussian_random_field(shape, corr, seed)
    g = g / np.abs(g).max()
    vp = vp_layers[layer][:, None, None] * (1.0 + pert * g)
    sig = np.broadcast_to(sig_layers[layer][:, None, None], shape)
    rho = 0.25 * vp + 1.5
    vs = vs_from_poisson(vp, sig)
    lam, mu = lame_from_velocities(vp, vs, rho)
    omega = 2.0 * math.pi * float(vs.min()) / (ppw * h)
    lo, hi = abl + 2, n - abl - 2
    xs = np.linspace(lo, hi, nsrc).round().astype(int) if nsrc > 1 else [n // 2]
    src = [(0, (abl + 2, n // 2, int(x))) for x in xs]
    return Medium(lam, mu, rho, omega, h, abl, src, name=f"layered{n}_seed{seed}")


def point_rhs(shape, sources, dtype=np.complex128):
    """Right-hand sides in the slot layout: one (d+1, *shape) array per source,
    zero everywhere except a unit value on the chosen u_k face."""
    d = len(shape)
    out = []
    for (k, idx) in sources:
        q = np.zeros((d + 1,) + tuple(shape), dtype=dtype)
        q[(k,) + tuple(idx)] = 1.0
        out.append(q)
    return out
