"""Adjoint-state gradient of the mixed elastic Helmholtz system (oracle).

The paper motivates the solver by full-waveform inversion (Sec. 1), where
misfits J(m) of the solution x = K(m)^{-1} q are differentiated with respect
to the cell-centred medium m = (lambda, mu, rho).  With the adjoint state w,
K^H w = dJ/dx* (here K = K^T, so K^H = conj(K)), the standard adjoint-state
identity gives

    dJ/dm_c = -Re( w^H (dK/dm_c) x ).

dK/dm_c is written out from the assembly of oracle/operators.py (Sec. 2.1
eq. elasticHelmSystem and eq. elasticHelmMass, Sec. 3 eq.
elasticHelmReformulatedSystem): the weighted Laplacian is linear in mu
(sum of D^T diag(W mu) D), the mass is linear in rho, and the pressure block
-1/(lambda+mu) has derivative 1/(lambda+mu)^2 in both lambda and mu.
"""
from __future__ import annotations

import numpy as np


def gradient(parts, x, w):
    """(g_lambda, g_mu, g_rho), each of shape parts.shape, for oracle-layout vectors x, w."""
    d = parts.d
    sizes = [parts.A[k].shape[0] for k in range(d)]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    xp, wp = x[offs[d]:], w[offs[d]:]
    pp = -np.real(np.conj(wp) * xp) / parts.lam_mu ** 2      # from -1/(lambda+mu)
    g_lam = pp.copy()
    g_mu = pp.copy()
    g_rho = np.zeros_like(pp)
    om = parts.omega
    mass_fac = -om ** 2 * (1.0 - 1j * parts.gamma / om)       # d(-w^2 rho (1 - i g/w))/d rho
    for k in range(d):
        xk, wk = x[offs[k]:offs[k + 1]], w[offs[k]:offs[k + 1]]
        for (D, Wm) in parts.terms[k]:
            g_mu += -np.real(Wm.T @ (np.conj(D @ wk) * (D @ xk)))
        g_rho += -np.real(mass_fac * (parts.A[k].T @ (np.conj(wk) * xk)))
    shp = parts.shape
    return g_lam.reshape(shp), g_mu.reshape(shp), g_rho.reshape(shp)
