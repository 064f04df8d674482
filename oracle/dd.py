"""Multicolour overlapping domain decomposition (oracle), Algorithm DD.

Sec. 2.3 and Sec. 4 of the paper.  Readings of what the paper leaves open:

* cores split every axis into nearly equal parts; Omega_i is the core grown
  by ``overlap`` cells on each side (clipped at the domain boundary);
* each Omega_i is padded by ``pad`` cells on every side that is not on the
  domain boundary; the padding holds a clamped copy of the medium and an
  absorbing layer, gamma += omega * dd_abl_max * (depth / pad)^2 (the
  interface absorbing layer of Sec. 2.3); the padded extent is rounded up
  (more padding) to a multiple of 2^(levels-1);
* 2^d colours by the parity of the subdomain index along each axis,
  c = sum_k 2^k (i_k mod 2) with k = 0 for x; colours are visited in
  increasing c and the global residual is recomputed before each colour
  (Algorithm DD, step 1);
* the local correction solves the local operator H_i, and in the hybrid
  DD-MG form (Sec. 4) this solve is one multigrid cycle of the shifted local
  operator; the correction is added on the DOFs that lie inside Omega_i (cells
  of Omega_i, faces with both neighbouring cells in Omega_i).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse.linalg as spla

from . import operators as op
from .multigrid import Hierarchy


def split_axis(n, s):
    """Core boundaries of s nearly equal parts (larger parts first)."""
    base, rem = divmod(n, s)
    edges = [0]
    for i in range(s):
        edges.append(edges[-1] + base + (1 if i < rem else 0))
    return edges


def slot_dof_index(shape):
    """Oracle DOF number of every slot of the slot layout; -1 on Dirichlet slots."""
    d = len(shape)
    idx = -np.ones((d + 1,) + tuple(shape), dtype=np.int64)
    off = 0
    for k in range(d):
        cs = op.comp_shape(shape, k)
        m = int(np.prod(cs))
        sl = [slice(None)] * d
        sl[d - 1 - k] = slice(1, None)
        idx[(k,) + tuple(sl)] = off + np.arange(m).reshape(cs)
        off += m
    idx[d] = off + np.arange(int(np.prod(shape))).reshape(shape)
    return idx


class Subdomain:
    def __init__(self, shape, sub_index, splits, overlap, pad, align):
        d = len(shape)
        self.index = sub_index                        # per numpy axis
        # colour c = sum_k 2^k (index along direction k mod 2), k = 0 for x
        self.colour = sum((sub_index[a] % 2) << (d - 1 - a) for a in range(d))
        self.om_lo, self.om_hi, self.pad_lo, self.pad_hi = [], [], [], []
        for a in range(d):
            e = splits[a]
            lo = max(e[sub_index[a]] - overlap, 0)
            hi = min(e[sub_index[a] + 1] + overlap, shape[a])
            plo = pad if lo > 0 else 0
            phi = pad if hi < shape[a] else 0
            ext = hi - lo + plo + phi
            extra = (-ext) % align
            if extra:
                if plo and phi:
                    plo += extra // 2
                    phi += extra - extra // 2
                elif plo:
                    plo += extra
                elif phi:
                    phi += extra
                else:
                    raise ValueError("axis not divisible by the coarsening factor")
            self.om_lo.append(lo); self.om_hi.append(hi)
            self.pad_lo.append(plo); self.pad_hi.append(phi)
        self.shape = tuple(self.om_hi[a] - self.om_lo[a] + self.pad_lo[a] + self.pad_hi[a]
                           for a in range(d))

    def local_medium(self, lam, mu, rho, gamma, omega, dd_abl_max):
        d = len(self.shape)
        gidx = []
        for a in range(d):
            l = np.arange(self.shape[a])
            g = self.om_lo[a] - self.pad_lo[a] + l
            gidx.append(np.clip(g, self.om_lo[a], self.om_hi[a] - 1))
        mesh = np.ix_(*gidx)
        ramp = np.zeros(self.shape)
        for a in range(d):
            l = np.arange(self.shape[a])
            ext = self.om_hi[a] - self.om_lo[a]
            dep = np.zeros(self.shape[a])
            if self.pad_lo[a]:
                m = l < self.pad_lo[a]
                dep[m] = (self.pad_lo[a] - l[m]) / self.pad_lo[a]
            if self.pad_hi[a]:
                m = l >= self.pad_lo[a] + ext
                dep[m] = (l[m] - (self.pad_lo[a] + ext) + 1) / self.pad_hi[a]
            sh = [1] * d
            sh[a] = self.shape[a]
            ramp = np.maximum(ramp, (dep ** 2).reshape(sh))
        return (lam[mesh], mu[mesh], rho[mesh],
                gamma[mesh] + omega * dd_abl_max * ramp)

    def index_maps(self, gshape):
        """(local DOF numbers, global DOF numbers) of the DOFs inside Omega_i."""
        d = len(self.shape)
        lidx = slot_dof_index(self.shape)
        gidx = slot_dof_index(gshape)
        inside = []
        for a in range(d):
            l = np.arange(self.shape[a])
            inside.append((l >= self.pad_lo[a]) & (l < self.shape[a] - self.pad_hi[a]))
        loc, glo = [], []
        for c in range(d + 1):
            mask = np.ones(self.shape, dtype=bool)
            for a in range(d):
                sh = [1] * d
                sh[a] = self.shape[a]
                ins = inside[a]
                if c < d and a == d - 1 - c:          # face slot f: cells f-1 and f
                    prev = np.concatenate([[False], ins[:-1]])
                    ins = ins & prev
                mask = mask & ins.reshape(sh)
            mask = mask & (lidx[c] >= 0)
            pos = np.nonzero(mask)
            gpos = tuple(pos[a] + self.om_lo[a] - self.pad_lo[a] for a in range(d))
            loc.append(lidx[c][pos])
            glo.append(gidx[c][gpos])
        loc = np.concatenate(loc); glo = np.concatenate(glo)
        assert (glo >= 0).all()
        return loc, glo


class DD:
    """Multicolour DD preconditioner for the unshifted global K."""

    def __init__(self, medium, nsub, overlap, pad, levels, alpha, dd_abl_max=1.0,
                 local="mg", w=None, economic=True, abl_max=1.0, gamma_add=0.01 * np.pi,
                 coarse_dd=None):
        shape = medium.lam.shape
        d = len(shape)
        self.shape = shape
        parts = op.parts_for(medium, abl_max, gamma_add)
        self.K = op.assemble_mixed(parts)
        gamma = op.gamma_profile(shape, medium.omega, medium.abl_cells, abl_max, gamma_add)
        splits = [split_axis(shape[a], nsub[a]) for a in range(d)]
        align = 2 ** (levels - 1)
        self.subs = []
        for sidx in itertools.product(*[range(nsub[a]) for a in range(d)]):
            sd = Subdomain(shape, sidx, splits, overlap, pad, align)
            lm = sd.local_medium(medium.lam, medium.mu, medium.rho, gamma, medium.omega, dd_abl_max)
            lparts = op.Parts(*lm, medium.omega, medium.h)
            sd.loc, sd.glo = sd.index_maps(shape)
            sd.ndof = sum(op.dof_sizes(sd.shape))
            if local == "mg":
                Ks = op.assemble_mixed(lparts, alpha)
                sd.hier = Hierarchy(Ks, sd.shape, levels, w=w, economic=economic,
                                    coarse_dd=coarse_dd)   # DD-MG-DD with coarse_dd (Sec. 4)
                sd.solve = lambda r, H=sd.hier: H.cycle(r)
            else:                                      # exact local solve of H_i
                lu = spla.splu(op.assemble_mixed(lparts, 0.0).tocsc())
                sd.solve = lu.solve
            self.subs.append(sd)
        self.ncolours = 2 ** d

    def apply(self, r):
        x = np.zeros_like(r, dtype=np.complex128)
        for c in range(self.ncolours):
            subs = [s for s in self.subs if s.colour == c]
            if not subs:
                continue
            res = r - self.K @ x
            for sd in subs:
                ri = np.zeros(sd.ndof, dtype=np.complex128)
                ri[sd.loc] = res[sd.glo]
                ei = sd.solve(ri)
                x[sd.glo] += ei[sd.loc]
        return x
