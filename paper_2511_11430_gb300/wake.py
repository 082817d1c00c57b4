"""A rotor shedding its near wake and converting it into vortex particles (Sec. II.A-C),
in hover or in forward flight with prescribed pitch and flapping (Eq. 12 form), driven
through the C ABI.

Each step of ``RotorWake.step``:
  1. the blade lattice at time t (prescribed motion ``synth.Kinematics``: rotation,
     collective and cyclic pitch, flapping, free stream; synthetic geometry);
  2. the velocity the particles and the near-wake rows induce at the control points,
     the AIC build and solve for the blade circulations (Neumann condition);
  3. the near-wake node lines convected by the local velocity plus the free stream
     (explicit Euler) and the particles advanced by one low-storage RK3 step, both with
     the blade rings and the wake rings frozen as Vatistas-cored segments;
  4. a new wake row shed between the trailing edge at t + dt and the convected
     trailing-edge line of t, carrying the trailing-edge panels' circulation (Kutta
     condition; upstream rows keep their strength);
  5. the oldest row beyond ``max_rows`` converted into particles (Eq. 6-8; adaptive
     counts, or the conventional uniform count with ``adaptive=False``) and appended;
  6. the blade loads at time t: Kutta-Joukowski on every bound segment (the blade rings'
     sides but the trailing-edge ones, whose net circulation with the row shed at this
     step vanishes) with the velocity relative to the blade at its midpoint (free stream
     minus the blade's own motion omega_b x r plus the induced velocity; one call per
     blade, each with its angular velocity), and the unsteady Bernoulli term of every
     panel; thrust and torque coefficients C_T = T / (rho pi R^2 (Omega R)^2),
     C_Q = Q / (rho pi R^3 (Omega R)^2) (thrust along the shaft +z, torque about it) are
     kept in ``history``.

Rows use the ring convention of vpm_wake_convert_row (U[p] -> U[p+1] -> D[p+1] ->
D[p]); the blade's trailing-edge segments run root -> tip, so a row shed behind a panel
of circulation Gamma carries -Gamma in that convention (the same sense of rotation).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib, api, synth
from ._lib import check


def _dev(a, dtype, device):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).to(device)


class RotorWake:
    def __init__(self, n_blades=2, n_span=20, n_chord=4, sigma=None, dt=None, max_rows=2, n_tip=2,
                 n_shed=1, adaptive=True, compensated=True, seg_core=None, nu=synth.NU_AIR, c_v=synth.C_V,
                 kin=None, tree=None, device="cuda"):
        """sigma defaults to 0.02 R, dt to 5 deg of azimuth; kin to the hover rotor
        (synth.Kinematics(): 8 deg collective, no flapping, no free stream).  tree =
        (theta, order) advances the particles with the treecode right-hand side
        (vpm_step_tree) instead of the direct sums, for wakes of a million particles."""
        self.tree = tree
        self.kin = synth.Kinematics() if kin is None else kin
        self.nb, self.S, self.nc = n_blades, n_span, n_chord
        sigma = 0.02 * self.kin.radius if sigma is None else sigma
        dt = np.deg2rad(5.0) / self.kin.omega if dt is None else dt
        self.sigma, self.dt, self.max_rows = float(sigma), float(dt), int(max_rows)
        self.u_inf = tuple(float(np.float32(v)) for v in self.kin.u_inf)  # the library's FP32 free stream
        self.n_tip = int(n_tip) if adaptive else -int(n_tip)
        self.n_shed = int(n_shed)
        self.core = float(sigma if seg_core is None else seg_core)
        self.dev = torch.device(device)
        self.prm = api.Params(sigma=self.sigma, nu=nu, c_v=c_v, seg_core=self.core, u_inf=self.u_inf,
                              compensated=compensated)
        self.compensated = compensated
        self.t = 0.0
        self.steps = 0
        self.ws = api.Workspace(self.dev)
        self.x = torch.zeros((3, 0), dtype=torch.float64, device=self.dev)
        self.G = torch.zeros((3, 0), dtype=torch.float64, device=self.dev)
        self.vol = torch.zeros((0,), dtype=torch.float32, device=self.dev)
        te = self._geometry_host(0.0)[4]
        self.nodes = _dev(te, torch.float64, self.dev).reshape(1, self.nb, self.S + 1, 3).contiguous()
        self.gammas = torch.zeros((0, self.nb, self.S), dtype=torch.float64, device=self.dev)
        self.converted = 0  # particles created so far
        self.rho = 1.225
        self.gam_prev = None
        self.history = []  # (t, C_T, C_Q) per step

    # ---- geometry (prescribed motion: synthetic input) ---------------------------
    def _geometry_host(self, t):
        # each step asks for the lattice at t and at t + dt: keep the last one
        if getattr(self, "_geo_t", None) == t:
            return self._geo
        L = synth.rotor_lattice(self.kin, t, self.nb, self.S, self.nc)
        r4 = np.zeros(L.rings.shape[:2] + (4,))
        r4[..., :3] = L.rings
        pad = lambda a: np.concatenate([a, np.zeros((a.shape[0], 1))], 1)
        self._geo_t = t
        self._geo = (r4, pad(L.colloc), pad(L.normal), pad(L.v_rel), L.te, L.te_idx, L.omega_b)
        return self._geo

    @property
    def rows(self) -> int:
        return int(self.gammas.shape[0])

    @property
    def n(self) -> int:
        return int(self.x.shape[1])

    def _wake_segments(self):
        R = self.rows
        m = 4 * R * self.nb * self.S
        sa = torch.empty((m, 4), dtype=torch.float32, device=self.dev)
        sb = torch.empty_like(sa)
        if m:
            check(_lib.load().vpm_wake_segments(api._void(self.nodes), api._void(self.gammas), R, self.nb, self.S,
                                                api._void(sa), api._void(sb), api._stream()))
        return sa, sb

    def _velocity(self, tgt, seg_a, seg_b, pos, strn):
        """u [3, n_tgt] at FP32 targets from the particles and the given segments."""
        u = torch.zeros((3, tgt.shape[0]), dtype=torch.float32, device=self.dev)
        if self.n > 0:
            u += api.induce(pos, strn, tgt, self.sigma, compensated=self.compensated, grad=False, ws=self.ws)
        if seg_a.shape[0] > 0:
            u += api.segments_induce(seg_a, seg_b, tgt, self.core, 2, compensated=self.compensated, grad=False,
                                     ws=self.ws)
        return u

    def step(self):
        lib = _lib.load()
        r4, colloc, normal, vrel, _, te_idx, omega_b = self._geometry_host(self.t)
        rings = _dev(r4, torch.float32, self.dev)
        colloc, normal, vrel = (_dev(a, torch.float32, self.dev) for a in (colloc, normal, vrel))
        pos = strn = None
        if self.n > 0:
            pos, strn = api.pack_state(self.x, self.G, self.vol)
        wsa, wsb = self._wake_segments()
        # 2. blade circulations
        u_c = self._velocity(colloc, wsa, wsb, pos, strn)
        A, b = api.aic_build(rings, colloc, normal, self.core, 2, v_rel=vrel, w_ind=u_c.contiguous())
        gam_b, _, _ = api.aic_solve(A, b, tol=1e-12, max_iter=30, ws=self.ws)
        nr = rings.shape[0]
        bsa = torch.empty((4 * nr, 4), dtype=torch.float32, device=self.dev)
        bsb = torch.empty_like(bsa)
        check(lib.vpm_ring_segments(api._void(rings), api._void(gam_b), nr, api._void(bsa), api._void(bsb),
                                    api._stream()))
        seg_a = torch.cat([bsa, wsa]).contiguous()
        seg_b = torch.cat([bsb, wsb]).contiguous()
        self._loads(lib, rings, normal, gam_b, te_idx, omega_b, bsa, bsb, seg_a, seg_b, pos, strn)
        # 3. convect the node lines, advance the particles
        pts = self.nodes.reshape(-1, 3)
        npts = pts.shape[0]
        tgt = torch.empty((npts, 4), dtype=torch.float32, device=self.dev)
        check(lib.vpm_points_pack(api._void(pts), npts, api._void(tgt), api._stream()))
        u_n = self._velocity(tgt, seg_a, seg_b, pos, strn).contiguous()
        check(lib.vpm_points_advect(api._void(pts), api._void(u_n), npts, ctypes.c_double(self.dt),
                                    (ctypes.c_float * 3)(*self.u_inf), api._stream()))
        if self.n > 0:
            if self.tree is None:
                api.step(self.x, self.G, self.vol, seg_a, seg_b, self.prm, self.dt, ws=self.ws)
            else:
                api.step_tree(self.x, self.G, self.vol, seg_a, seg_b, self.prm, self.dt, theta=self.tree[0],
                              order=self.tree[1], ws=self.ws)
        # 4. shed a row behind the trailing edge of t + dt
        te_next = self._geometry_host(self.t + self.dt)[4]
        line0 = _dev(te_next, torch.float64, self.dev).reshape(1, self.nb, self.S + 1, 3)
        self.nodes = torch.cat([line0, self.nodes]).contiguous()
        shed = -gam_b[torch.from_numpy(te_idx.ravel()).to(self.dev)].reshape(1, self.nb, self.S)
        self.gammas = torch.cat([shed, self.gammas]).contiguous()
        # 5. convert the oldest row beyond max_rows
        if self.rows > self.max_rows:
            self._convert_oldest()
        self.t += self.dt
        self.steps += 1
        return gam_b

    def _loads(self, lib, rings, normal, gam_b, te_idx, omega_b, bsa, bsb, seg_a, seg_b, pos, strn):
        # the bound segments: every side of every blade ring, except the trailing-edge sides,
        # whose net circulation with the row shed this step is zero (Kutta condition)
        ba = bsa.clone()
        ba[torch.from_numpy(4 * te_idx.ravel() + 1).to(self.dev), 3] = 0.0
        bb = bsb
        m = ba.shape[0]
        mid = torch.empty((m, 4), dtype=torch.float32, device=self.dev)
        check(lib.vpm_segment_midpoints(api._void(ba), api._void(bb), m, api._void(mid), api._stream()))
        u_mid = self._velocity(mid, seg_a, seg_b, pos, strn)
        # one call per blade: each blade moves with its own angular velocity about the hub
        nr = rings.shape[0] // self.nb
        ms = 4 * nr
        out = torch.empty((self.nb, 6), dtype=torch.float64, device=self.dev)
        D3 = ctypes.c_double * 3
        w = self.ws.get(api.workspace_size(_lib.VPM_OP_LOADS, 0, nr, ms, 0))
        for b in range(self.nb):
            r0, s0 = b * nr, b * ms
            um = u_mid[:, s0:s0 + ms].contiguous()
            gp = None if self.gam_prev is None else self.gam_prev[r0:r0 + nr]
            check(lib.vpm_blade_loads(api._void(ba[s0:]), api._void(bb[s0:]), ms, api._void(um), D3(*omega_b[b]),
                                      D3(0.0, 0.0, 0.0), D3(*self.u_inf), api._void(rings[r0:]),
                                      api._void(normal[r0:]), api._void(gam_b[r0:]), api._void(gp), nr,
                                      ctypes.c_double(self.dt), ctypes.c_double(self.rho), api._void(out[b]),
                                      api._void(w), w.numel(), api._stream()))
        F = out.sum(0).cpu().numpy()
        Rr, W = self.kin.radius, self.kin.omega
        q = self.rho * np.pi * Rr ** 2 * (W * Rr) ** 2
        self.history.append((self.t, F[2] / q, -F[5] / (q * Rr)))
        self.gam_prev = gam_b.clone()

    def _convert_oldest(self):
        R = self.rows
        U = self.nodes[R - 1]  # [nb, S+1, 3]
        D = self.nodes[R]
        Uh, Dh = U[:, -1].cpu().numpy(), D[:, -1].cpu().numpy()
        xs, Gs = [], []
        for b in range(self.nb):
            d = Dh[b] - Uh[b]
            ds_tip = float(np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]))  # the tip's trailed edge
            xw, Gw = api.wake_convert_row(U[b].contiguous(), D[b].contiguous(), self.gammas[R - 1, b].contiguous(),
                                          ds_tip, self.n_tip, self.n_shed, ws=self.ws)
            xs.append(xw)
            Gs.append(Gw)
        xn = torch.cat(xs, 1)
        Gn = torch.cat(Gs, 1)
        self.converted += int(xn.shape[1])
        self.x = torch.cat([self.x, xn], 1).contiguous()
        self.G = torch.cat([self.G, Gn], 1).contiguous()
        vol = torch.full((xn.shape[1],), self.sigma ** 3, dtype=torch.float32, device=self.dev)
        self.vol = torch.cat([self.vol, vol]).contiguous()
        self.nodes = self.nodes[:R].contiguous()
        self.gammas = self.gammas[:R - 1].contiguous()
