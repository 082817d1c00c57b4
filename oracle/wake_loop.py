"""FP64 CPU reference of the near-wake time loop (Sec. II.A-C) that
paper_2511_11430_gb300.wake.RotorWake runs through the library.  TEST
INFRASTRUCTURE ONLY: only tests/ use it.

Every step uses the oracle's own routines (plain FP64 loops in vpm_oracle.c) in
the same order as the library's driver: blade circulations from the AIC with the
velocity the particles and the wake rows induce at the control points (textbook LU),
the near-wake node lines convected by explicit Euler, the particles by one
low-storage RK3 step (the right-hand side evaluated on the state rounded to FP32,
the library's precision reading), a new row shed with the trailing-edge panels'
circulation (Kutta), and the oldest row beyond max_rows converted by Eq. 6-8.  The
blade geometry and motion are the same synthetic input (rounded to FP32, as the
library gets it): hover, or forward flight with the pitch and flapping schedules of
Eq. 12 form and a free stream, which convects the node lines and the particles and
enters the loads with each blade's own angular velocity.  The blade placement, its
angular velocity and the lattice come from oracle/kinematics.py, written apart from
the product's generator; only the rotor's static description (synth.Kinematics:
radius, chord, schedule coefficients) and the air constants are shared.
"""
from __future__ import annotations

import numpy as np

import oracle
from oracle import kinematics
from paper_2511_11430_gb300 import synth


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


class OracleRotorWake:
    def __init__(self, n_blades=2, n_span=20, n_chord=4, sigma=None, dt=None, max_rows=2, n_tip=2,
                 n_shed=1, adaptive=True, seg_core=None, nu=synth.NU_AIR, c_v=synth.C_V, kin=None):
        self.kin = synth.Kinematics() if kin is None else kin
        self.nb, self.S, self.nc = n_blades, n_span, n_chord
        sigma = 0.02 * self.kin.radius if sigma is None else sigma
        dt = np.deg2rad(5.0) / self.kin.omega if dt is None else dt
        self.sigma, self.dt, self.max_rows = float(sigma), float(dt), int(max_rows)
        self.u_inf = _f32(self.kin.u_inf)
        self.n_tip = int(n_tip) if adaptive else -int(n_tip)
        self.n_shed = int(n_shed)
        self.core = float(sigma if seg_core is None else seg_core)
        self.nu, self.c_v = nu, c_v
        self.t = 0.0
        self.x = np.zeros((0, 3))
        self.G = np.zeros((0, 3))
        te = self._geometry(0.0)[4]
        self.nodes = te.reshape(1, self.nb, self.S + 1, 3).copy()
        self.gammas = np.zeros((0, self.nb, self.S))
        self.rho = 1.225
        self.gam_prev = None
        self.history = []

    def _geometry(self, t):
        L = kinematics.lattice(self.kin, t, self.nb, self.S, self.nc)
        return _f32(L.rings), _f32(L.colloc), _f32(L.normal), _f32(L.v_rel), L.te, L.te_idx, L.omega_b

    @property
    def rows(self):
        return self.gammas.shape[0]

    def _wake_segments(self):
        sa, sb = [], []
        for r in range(self.rows):
            for b in range(self.nb):
                U, D = self.nodes[r, b], self.nodes[r + 1, b]
                for p in range(self.S):
                    c = [U[p], U[p + 1], D[p + 1], D[p]]
                    for k in range(4):
                        sa.append([*_f32(c[k]), np.float32(self.gammas[r, b, p])])
                        sb.append([*_f32(c[(k + 1) % 4]), 0.0])
        return np.array(sa).reshape(-1, 4), np.array(sb).reshape(-1, 4)

    def _velocity(self, tgt, sa, sb):
        u = np.zeros((len(tgt), 3))
        if len(self.x):
            pos = np.concatenate([_f32(self.x), np.full((len(self.x), 1), np.float32(self.sigma ** 3))], 1)
            u += oracle.p2p(pos, _f32(self.G), tgt, self.sigma, grad=False)
        if len(sa):
            u += oracle.segments(sa, sb, tgt, self.core, 2, grad=False)
        return u

    def step(self):
        rings, colloc, normal, vrel, _, te_idx, omega_b = self._geometry(self.t)
        wsa, wsb = self._wake_segments()
        u_c = self._velocity(colloc, wsa, wsb)
        A = oracle.aic_build(rings, colloc, normal, self.core)
        b = oracle.aic_rhs(vrel, _f32(u_c), normal)
        gam = oracle.lu_solve(_f32(A), b)
        bsa, bsb = kinematics.ring_segments(rings, _f32(gam))
        sa = np.concatenate([bsa, wsa]) if len(wsa) else bsa
        sb = np.concatenate([bsb, wsb]) if len(wsb) else bsb
        self._loads(rings, normal, gam, te_idx, omega_b, bsa, bsb, sa, sb)
        pts = self.nodes.reshape(-1, 3)
        u_n = self._velocity(pts, sa, sb)
        x_old, G_old = self.x, self.G
        self.nodes = (pts + self.dt * (_f32(u_n) + self.u_inf)).reshape(self.nodes.shape)
        if len(x_old):
            vol = np.full(len(x_old), np.float32(self.sigma ** 3))
            self.x, self.G = oracle.step(x_old, G_old, vol, sa, sb, self.sigma, self.dt, nu=self.nu, c_v=self.c_v,
                                         seg_core=self.core, u_inf=self.u_inf, cast_f32=True)
        te_next = self._geometry(self.t + self.dt)[4]
        self.nodes = np.concatenate([te_next.reshape(1, self.nb, self.S + 1, 3), self.nodes])
        shed = -gam[te_idx.ravel()].reshape(1, self.nb, self.S)
        self.gammas = np.concatenate([shed, self.gammas])
        if self.rows > self.max_rows:
            self._convert_oldest()
        self.t += self.dt
        return gam

    def _loads(self, rings, normal, gam, te_idx, omega_b, bsa, bsb, sa, sb):
        # the bound segments: every side of every blade ring, except the trailing-edge sides,
        # whose net circulation with the row shed this step is zero (Kutta condition)
        ba, bb = _f32(bsa).copy(), _f32(bsb)
        ba[4 * te_idx.ravel() + 1, 3] = 0.0
        mid = ((ba[:, :3].astype(np.float32) + bb[:, :3].astype(np.float32)) * np.float32(0.5)).astype(np.float64)
        u_mid = _f32(self._velocity(mid, sa, sb))
        F, M = np.zeros(3), np.zeros(3)
        nr = len(rings) // self.nb
        for b in range(self.nb):  # each blade with its own angular velocity about the hub
            r, s = slice(b * nr, (b + 1) * nr), slice(4 * b * nr, 4 * (b + 1) * nr)
            Fb, Mb = oracle.blade_loads(ba[s], bb[s], u_mid[s], omega_b[b], [0.0, 0.0, 0.0], self.u_inf, rings[r],
                                        normal[r], gam[r], None if self.gam_prev is None else self.gam_prev[r],
                                        self.dt, self.rho)
            F, M = F + Fb, M + Mb
        Rr, W = self.kin.radius, self.kin.omega
        q = self.rho * np.pi * Rr ** 2 * (W * Rr) ** 2
        self.history.append((self.t, F[2] / q, -M[2] / (q * Rr)))
        self.gam_prev = gam.copy()

    def _convert_oldest(self):
        R = self.rows
        xs, Gs = [], []
        for b in range(self.nb):
            U, D = self.nodes[R - 1, b], self.nodes[R, b]
            d = D[-1] - U[-1]
            ds_tip = float(np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]))
            ea, eb, g, gnb, hn, tr = oracle.wake_row_edges(U, D, self.gammas[R - 1, b])
            xw, Gw, _ = oracle.wake_convert(ea, eb, g, gnb, hn, tr, ds_tip, self.n_tip, self.n_shed)
            xs.append(xw)
            Gs.append(Gw)
        self.x = np.concatenate([self.x] + xs)
        self.G = np.concatenate([self.G] + Gs)
        self.nodes = self.nodes[:R]
        self.gammas = self.gammas[:R - 1]
