"""Prescribed blade motion of the oracle's near-wake loop (test infrastructure: only
tests/ and the oracle's own loop use it).  Written independently of the product's
lattice generator: each blade is one rigid body placed by a rotation matrix, and
its angular velocity is read off the time derivative of that matrix.

Blade b of a rotor with N_b blades sits at azimuth psi_b = Omega t + 2 pi b / N_b
(psi = 0 downstream along +x, counter-clockwise about +z seen from above).  Its
pitch and flap follow the first-harmonic schedules of Sec. IV.B (Eq. 12 form),
  theta(psi) = theta_0 + theta_1c cos psi + theta_1s sin psi,
  beta(psi)  = beta_0  + beta_1c  cos psi + beta_1s  sin psi      [deg],
with the flap hinge and the feathering axis through the hub (a teetering hub).  In
the blade's own frame (span along +x, direction of travel +y, up +z) a point at
span r and chordwise distance s behind the leading edge is
  q(r, s) = R_x(tw(r)) (r, -(s - c/4), 0),   tw(r) = twist (r/R - twist_ref),
i.e. the blade twisted about its quarter-chord line.  In the rotor frame it is
  x = hub + M(t) q,   M = R_z(psi) R_y(-beta) R_x(theta):
pitch about the span axis (nose up), flap about the hinge (tip up), azimuth about
+z.  The angular velocity is the axial vector of dM/dt M^T, with dM/dt from the
product rule and the schedules' analytic rates, and every point of the blade moves
with omega x (x - hub).

The vortex-ring lattice on each blade (Sec. II.A): panel (i, j) between radial
stations r_i, r_{i+1} (root cut-out to tip, uniform) and chordwise stations
xi_j, xi_{j+1} (uniform over the chord); its ring is the panel shifted a quarter
panel chord aft, corners in the order leading-root, trailing-root, trailing-tip,
leading-tip; its control point is the middle of the three-quarter panel chord line;
its normal is the blade's up direction at the panel's mid-span, M R_x(tw) e_z.
"""
from __future__ import annotations

import numpy as np


def _rx(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def _ry(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def _rz(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _drx(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[0.0, 0.0, 0.0], [0.0, -s, -c], [0.0, c, -s]])


def _dry(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[-s, 0.0, c], [0.0, 0.0, 0.0], [-c, 0.0, -s]])


def _drz(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[-s, -c, 0.0], [c, -s, 0.0], [0.0, 0.0, 0.0]])


def schedule(coef, psi):
    """(angle, d angle / d psi) in radians of c0 + c1c cos psi + c1s sin psi [deg]."""
    c0, c1c, c1s = coef
    a = c0 + c1c * np.cos(psi) + c1s * np.sin(psi)
    da = -c1c * np.sin(psi) + c1s * np.cos(psi)
    return np.deg2rad(a), np.deg2rad(da)


def blade_attitude(kin, t, b, n_blades):
    """(M, dM/dt) of blade b at time t: rotation matrix of the blade frame and its rate."""
    W = kin.omega
    psi = W * t + 2.0 * np.pi * b / n_blades
    th, dth = schedule(kin.theta, psi)
    be, dbe = schedule(kin.beta, psi)
    Z, Y, X = _rz(psi), _ry(-be), _rx(th)
    # d/dt with d psi/dt = Omega: each angle's rate is Omega times its psi-derivative
    dM = W * (_drz(psi) @ Y @ X - dbe * (Z @ _dry(-be) @ X) + dth * (Z @ Y @ _drx(th)))
    return Z @ Y @ X, dM


def angular_velocity(M, dM):
    """The axial vector w of the skew matrix dM M^T (w x v = dM M^T v)."""
    S = dM @ M.T
    return np.array([0.5 * (S[2, 1] - S[1, 2]), 0.5 * (S[0, 2] - S[2, 0]), 0.5 * (S[1, 0] - S[0, 1])])


class Lattice:
    """The blade-ring lattice of a rotor at one instant (float64)."""

    def __init__(self, rings, colloc, normal, v_rel, omega_b, te, te_idx):
        self.rings, self.colloc, self.normal, self.v_rel = rings, colloc, normal, v_rel
        self.omega_b, self.te, self.te_idx = omega_b, te, te_idx


def lattice(kin, t, n_blades, n_span, n_chord, hub=(0.0, 0.0, 0.0)):
    """Rings [n, 4, 3], control points, normals and v_rel = u_inf - omega x (y - hub)
    [n, 3] (n = n_blades n_span n_chord, blade-major, then span, then chord), each
    blade's angular velocity [n_blades, 3], trailing-edge node lines [n_blades,
    n_span + 1, 3] and the trailing-edge ring indices [n_blades, n_span]."""
    hub = np.asarray(hub, dtype=np.float64)
    Rr, c = kin.radius, kin.chord
    u_inf = np.array([kin.mu * kin.omega * Rr, 0.0, 0.0])
    r_st = kin.root + (Rr - kin.root) * np.arange(n_span + 1) / n_span
    d_xi = c / n_chord
    rings, colloc, normal, v_rel, omegas = [], [], [], [], []
    te = np.zeros((n_blades, n_span + 1, 3))
    te_idx = np.zeros((n_blades, n_span), dtype=np.int64)

    for b in range(n_blades):
        M, dM = blade_attitude(kin, t, b, n_blades)
        w = angular_velocity(M, dM)
        omegas.append(w)

        def point(r, s):
            tw = np.deg2rad(kin.twist) * (r / Rr - kin.twist_ref)
            return hub + M @ (_rx(tw) @ np.array([r, -(s - 0.25 * c), 0.0]))

        for i in range(n_span):
            ra, rb = r_st[i], r_st[i + 1]
            rm = 0.5 * (ra + rb)
            up = M @ (_rx(np.deg2rad(kin.twist) * (rm / Rr - kin.twist_ref)) @ np.array([0.0, 0.0, 1.0]))
            for j in range(n_chord):
                s_lead = j * d_xi + 0.25 * d_xi
                s_trail = (j + 1) * d_xi + 0.25 * d_xi
                rings.append([point(ra, s_lead), point(ra, s_trail), point(rb, s_trail), point(rb, s_lead)])
                y = point(rm, j * d_xi + 0.75 * d_xi)
                colloc.append(y)
                normal.append(up)
                v_rel.append(u_inf - np.cross(w, y - hub))
            k = (b * n_span + i) * n_chord + n_chord - 1
            te_idx[b, i] = k
            te[b, i] = rings[k][1]
        te[b, n_span] = rings[te_idx[b, n_span - 1]][2]
    return Lattice(np.asarray(rings), np.asarray(colloc), np.asarray(normal), np.asarray(v_rel),
                   np.asarray(omegas), te, te_idx)


def ring_segments(rings, gamma):
    """Segments c_k -> c_(k+1 mod 4) of every ring [n, 4, 3] with its circulation:
    seg_a [4 n, 4] = (start, circulation), seg_b [4 n, 4] = (end, 0)."""
    n = rings.shape[0]
    a = np.zeros((4 * n, 4))
    b = np.zeros((4 * n, 4))
    for i in range(n):
        for k in range(4):
            a[4 * i + k, :3] = rings[i, k, :3]
            a[4 * i + k, 3] = gamma[i]
            b[4 * i + k, :3] = rings[i, (k + 1) % 4, :3]
    return a, b
