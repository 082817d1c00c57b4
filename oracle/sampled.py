"""The FP64 oracle's right-hand side of Eq. 4-5 at a sample of particles of a large
wake (test infrastructure: only tests/ and bench.py's cpu_baseline leg use it).

For a million particles and more the oracle cannot evaluate every particle, so the
right-hand side is assembled at sampled particles i from the oracle's own routines
(nothing here comes from the CUDA library):

  dx/dt_i    = u_i + u_inf, u_i from every particle and every segment;
  nu_t,i     = Vreman's eddy viscosity of the full gradient J_i;
  dGamma/dt_i = the stretching of J_i plus the exchange sum of Eq. 5 over every
               particle j, p_i = (2/sigma^2) sum_j nu_ij (v_i Gamma_j - v_j Gamma_i)
               zeta_sigma(r_ij), nu_ij = nu + (nu_t,i + nu_t,j)/2.

The exchange sum needs nu_t,j of the other particles, i.e. their full gradients.
With c_V = 0 it needs none and the result is exact.  With c_V > 0 the gradients are
evaluated at every particle within ``cut`` sigma of a sampled one; for the particles
beyond, nu_t,j is taken as 0.  Their exchange weight zeta(r) / zeta(0) is below
exp(-cut^2 / 2) (1.3e-14 at the default cut of 8), so this changes p_i by less
than that fraction of one neighbour's term.  Sampled particles that come in runs of
consecutive indices (neighbours along a vortex filament) share most of their
neighbourhoods, which keeps the gradient evaluations few.
"""
from __future__ import annotations

import numpy as np

from . import p2p, pse_at, segments, stretch, vreman


def _neighbours(P, idx, radius):
    from scipy.spatial import cKDTree

    tree = cKDTree(P)
    nb = set()
    for lst in tree.query_ball_point(P[idx], radius):
        nb.update(lst)
    nb.update(int(i) for i in idx)
    return np.array(sorted(nb), dtype=np.int64)


def _uJ(w, sel):
    u, J = p2p(w.pos, w.strength, w.pos[sel], w.sigma)
    if w.m > 0:
        us, Js = segments(w.seg_a, w.seg_b, w.pos[sel], w.seg_core, w.vatistas_n)
        u, J = u + us, J + Js
    return u, J


def rhs_at(w, idx, c_v=None, cut=8.0, classic=False):
    """(dx/dt [k, 3], dGamma/dt [k, 3], nu_t [k]) at the particles idx of wake w
    (a synth.Wake: pos, strength, seg_a, seg_b, sigma, nu, c_v, seg_core,
    vatistas_n, u_inf), with c_V = w.c_v unless given."""
    idx = np.asarray(idx, dtype=np.int64)
    c_v = w.c_v if c_v is None else c_v
    u, J = _uJ(w, idx)
    nut_i = vreman(J, w.sigma, c_v)
    s = stretch(J, w.strength[idx], classic=classic)
    if c_v > 0.0:
        P = w.pos[:, :3].astype(np.float64)
        nb = _neighbours(P, idx, cut * w.sigma)
        rest = np.setdiff1d(nb, idx)
        nut = np.zeros(w.n)
        nut[idx] = nut_i
        if rest.size:
            _, Jr = _uJ(w, rest)
            nut[rest] = vreman(Jr, w.sigma, c_v)
        p = pse_at(w.pos, w.strength, nut, w.sigma, w.nu, idx)
    else:
        p = pse_at(w.pos, w.strength, None, w.sigma, w.nu, idx)
    dxdt = u + np.asarray(w.u_inf, dtype=np.float64)
    return dxdt, s + p, nut_i
