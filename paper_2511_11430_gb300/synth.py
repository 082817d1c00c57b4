"""Seeded synthetic rotor-wake inputs.

The paper's cases (Caradonna-Tung hover, AH-1G forward flight with blade-vortex
interaction, Sweet's side-by-side rotors; Sec. IV) need experimental geometry and
wakes that are not available, so these generators stand in for them with the
same structure: helical tip-vortex particle spirals behind rectangular blades
carrying a vortex-ring lattice (Sec. II.A, Fig. 1), the skewed wake of forward
flight, wakes of two counter-rotating rotors merging between the hubs.

This module holds geometry only: positions, directions, magnitudes and the ring
lattice layout.  It computes nothing of the method (no induced velocity, no
kernel, no solve); both the CUDA path and the FP64 oracle consume what it
returns.  Every value is built in float64 from ``numpy.random.default_rng(seed)``
and rounded once to float32, so both sides read bit-identical inputs.

Layouts (float32, C-contiguous):
  pos[n, 4] = (x, y, z, volume)       strength[n, 4] = (Gx, Gy, Gz, 0)
  seg_a[m, 4] = (ax, ay, az, circulation)   seg_b[m, 4] = (bx, by, bz, 0)
  rings[nr, 4, 4] corners (xyz, 0) ordered leading-root, trailing-root,
      trailing-tip, leading-tip: right-handed about the panel normal
  colloc[nr, 4], normal[nr, 4], v_rel[nr, 4] (free stream minus blade motion)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

R = 1.0  # rotor radius [m]
OMEGA = 200.0  # rotor speed [rad/s], Omega R = 200 m/s
NU_AIR = 1.5e-5  # kinematic viscosity [m^2/s]
C_V = 0.07  # Vreman coefficient used by the paper
DT = np.deg2rad(5.0) / OMEGA  # 5 deg azimuth per step (N_steps = 72)


@dataclass
class Wake:
    name: str
    sigma: float
    pos: np.ndarray
    strength: np.ndarray
    seg_a: np.ndarray
    seg_b: np.ndarray
    rings: np.ndarray
    colloc: np.ndarray
    normal: np.ndarray
    v_rel: np.ndarray
    seg_core: float
    u_inf: tuple = (0.0, 0.0, 0.0)
    dt: float = DT
    nu: float = NU_AIR
    c_v: float = C_V
    vatistas_n: int = 2
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def m(self) -> int:
        return int(self.seg_a.shape[0])

    @property
    def n_ctrl(self) -> int:
        return int(self.colloc.shape[0])


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def _pad4(xyz, w):
    out = np.zeros((xyz.shape[0], 4), dtype=np.float64)
    out[:, :3] = xyz
    out[:, 3] = w
    return out


def helix(rng, n, phase, revs, pitch, r_of_age, gamma_mag=(0.9e-3, 1.1e-3), jitter=0.0,
          centre=(0.0, 0.0, 0.0), spin=1.0, drift=(0.0, 0.0), z0=-0.01):
    """n particles on one trailing tip-vortex spiral.

    Wake age psi in (0, 2 pi revs); the particle shed at age psi sits at azimuth
    phase - spin*psi, radius r_of_age(psi), height z0 - pitch*psi/(2 pi), shifted by
    drift = (dx, dz) per revolution (skew or merging).  The strength is tangent to
    the spiral in the direction of increasing age, with magnitude drawn uniformly
    from gamma_mag, then positions get uniform jitter in [-jitter, jitter]^3.
    """
    psi = (np.arange(n, dtype=np.float64) + 0.5) * (2.0 * np.pi * revs / n)
    h = 1e-6
    def curve(p):
        t = phase - spin * p
        r = r_of_age(p)
        x = centre[0] + r * np.cos(t) + drift[0] * p / (2 * np.pi)
        y = centre[1] + r * np.sin(t)
        z = centre[2] + z0 - pitch * p / (2 * np.pi) + drift[1] * p / (2 * np.pi)
        return np.stack([x, y, z], axis=1)
    xyz = curve(psi)
    tan = curve(psi + h) - curve(psi - h)
    tan /= np.linalg.norm(tan, axis=1, keepdims=True)
    mag = rng.uniform(gamma_mag[0], gamma_mag[1], size=n)
    G = tan * mag[:, None]
    if jitter > 0:
        xyz = xyz + rng.uniform(-jitter, jitter, size=xyz.shape)
    return xyz, G


def blade_lattice(n_blades, n_span, n_chord, chord=R / 6, root=0.15 * R, pitch_deg=8.0, phase=0.0,
                  hub=(0.0, 0.0, 0.0), spin=1.0, gamma0=2.0, u_inf=(0.0, 0.0, 0.0)):
    """Flat rectangular blades with a vortex-ring lattice (Sec. II.A).

    Panel (i, j) spans radial stations i..i+1 and chordwise stations j..j+1; its
    ring is the panel shifted a quarter panel chord aft, its collocation point the
    centre of the three-quarter-chord line.  Blades rotate about +z with sense
    ``spin`` (+1 counter-clockwise seen from above).  Ring circulations follow the
    fixed profile gamma0 (r/R) sqrt(1 - (r/R)^2) shared linearly over the chord.
    """
    th = np.deg2rad(pitch_deg)
    rings, colloc, normal, vrel, gam = [], [], [], [], []
    r_nodes = np.linspace(root, R, n_span + 1)
    xi = np.linspace(0.0, chord, n_chord + 1)
    dxi = chord / n_chord
    w = np.arange(n_chord, 0, -1, dtype=np.float64)
    w /= w.sum()
    for b in range(n_blades):
        psi = phase + spin * 2.0 * np.pi * b / n_blades
        er = np.array([np.cos(psi), np.sin(psi), 0.0])
        epsi = spin * np.array([-np.sin(psi), np.cos(psi), 0.0])  # direction of travel
        cdir = -epsi * np.cos(th) - np.array([0.0, 0.0, 1.0]) * np.sin(th)  # leading -> trailing edge
        nrm = np.cross(cdir, er)
        nrm /= np.linalg.norm(nrm)
        if nrm[2] < 0:
            nrm = -nrm
        hubv = np.asarray(hub, dtype=np.float64)
        def pt(r, s):
            return hubv + r * er + (s - 0.25 * chord) * cdir
        for i in range(n_span):
            r0, r1 = r_nodes[i], r_nodes[i + 1]
            rm = 0.5 * (r0 + r1)
            for j in range(n_chord):
                s0, s1 = xi[j] + 0.25 * dxi, xi[j + 1] + 0.25 * dxi
                c = [pt(r0, s0), pt(r0, s1), pt(r1, s1), pt(r1, s0)]
                if spin < 0:  # keep the corner order right-handed about the normal
                    c = [c[0], c[3], c[2], c[1]]
                rings.append(c)
                y = pt(rm, xi[j] + 0.75 * dxi)
                colloc.append(y)
                normal.append(nrm)
                omega_cross_y = spin * OMEGA * np.array([-(y[1] - hubv[1]), y[0] - hubv[0], 0.0])
                vrel.append(np.asarray(u_inf) - omega_cross_y)
                gam.append(gamma0 * (rm / R) * np.sqrt(max(1.0 - (rm / R) ** 2, 0.0)) * w[j] * n_chord)
    rings = np.asarray(rings)
    colloc = np.asarray(colloc)
    normal = np.asarray(normal)
    vrel = np.asarray(vrel)
    gam = np.asarray(gam)
    return rings, colloc, normal, vrel, gam


@dataclass(frozen=True)
class Kinematics:
    """Prescribed motion of a rotor with rigid rectangular blades (Sec. IV.B, Eq. 12 form).

    Blade b sits at azimuth psi_b = Omega t + 2 pi b / N_b (psi = 0 downstream, +x;
    rotation counter-clockwise about +z seen from above).  Its pitch and flap angles
    follow first-harmonic schedules in psi_b [deg]:
        theta(psi) = theta_0 + theta_1c cos psi + theta_1s sin psi   (plus the twist),
        beta(psi)  = beta_0  + beta_1c  cos psi + beta_1s  sin psi.
    The flap hinge and the feathering axis pass through the hub (a teetering hub: no
    hinge offset).  The linear twist adds twist (r/R - twist_ref) to the pitch.  The
    free stream (mu Omega R, 0, 0) lies in the disk plane (no shaft tilt)."""
    radius: float = R
    chord: float = R / 6
    root: float = 0.15 * R
    omega: float = OMEGA
    theta: tuple = (8.0, 0.0, 0.0)
    beta: tuple = (0.0, 0.0, 0.0)
    twist: float = 0.0
    twist_ref: float = 0.75
    mu: float = 0.0

    @property
    def u_inf(self):
        return (self.mu * self.omega * self.radius, 0.0, 0.0)


# The AH-1G main rotor of the forward-flight case: geometry of its table of rotor
# properties (2 blades, R 6.7 m, c 0.7283 m, -10 deg linear twist, root cut-out 0.154 R),
# the pitch and flapping schedules of Eq. 12, advance ratio 0.19 and tip Mach number
# 0.65 (speed of sound 340.3 m/s).
AH1G = Kinematics(radius=6.7, chord=0.7283, root=0.154 * 6.7, omega=0.65 * 340.3 / 6.7, theta=(6.0, 1.7, -5.5),
                  beta=(0.0, 2.13, -0.15), twist=-10.0, mu=0.19)


@dataclass
class RotorLattice:
    rings: np.ndarray    # [nr, 4, 3] corners, ordered as blade_lattice's
    colloc: np.ndarray   # [nr, 3]
    normal: np.ndarray   # [nr, 3]
    v_rel: np.ndarray    # [nr, 3] free stream minus the blade's velocity at the control point
    omega_b: np.ndarray  # [n_blades, 3] angular velocity of each blade (about the hub)
    te: np.ndarray       # [n_blades, n_span + 1, 3] trailing-edge node lines
    te_idx: np.ndarray   # [n_blades, n_span] trailing-edge ring indices


def _harmonic(c, psi):
    """(value, d/dpsi) of c0 + c1c cos psi + c1s sin psi, c in degrees, result in radians."""
    v = c[0] + c[1] * np.cos(psi) + c[2] * np.sin(psi)
    d = -c[1] * np.sin(psi) + c[2] * np.cos(psi)
    return np.deg2rad(v), np.deg2rad(d)


def rotor_lattice(kin: Kinematics, t, n_blades, n_span, n_chord, hub=(0.0, 0.0, 0.0)) -> RotorLattice:
    """The vortex-ring lattice of the blades of ``kin`` at time t.

    Each blade is placed by three rotations about axes through the hub: pitch about
    the blade axis, flap about the hinge axis e_r x e_z, azimuth about e_z.  Its
    angular velocity is therefore the sum Omega e_z + beta' (e_r x e_z) + theta'
    e_r,flapped (each rate d/dt of the schedule), and every point x of the blade moves
    with omega_b x (x - hub).  Panel layout as in blade_lattice (rings a quarter panel
    chord aft, control points at the three-quarter chord); with twist the rings are
    not planar and each control point takes the normal of the local chord line.
    """
    W, Rr, c = kin.omega, kin.radius, kin.chord
    hubv = np.asarray(hub, dtype=np.float64)
    ez = np.array([0.0, 0.0, 1.0])
    u_inf = np.asarray(kin.u_inf)
    r_nodes = np.linspace(kin.root, Rr, n_span + 1)
    xi = np.linspace(0.0, c, n_chord + 1)
    dxi = c / n_chord
    rings, colloc, normal, vrel, omegas = [], [], [], [], []
    for b in range(n_blades):
        psi = W * t + 2.0 * np.pi * b / n_blades
        er = np.array([np.cos(psi), np.sin(psi), 0.0])
        tg = np.array([-np.sin(psi), np.cos(psi), 0.0])  # direction of travel
        beta, dbeta = _harmonic(kin.beta, psi)
        theta, dtheta = _harmonic(kin.theta, psi)
        erf = np.cos(beta) * er + np.sin(beta) * ez  # flapped blade axis
        nf = np.cos(beta) * ez - np.sin(beta) * er   # flapped disk normal
        om = W * ez + W * dbeta * np.cross(er, ez) + W * dtheta * erf
        omegas.append(om)

        def cdir(r):  # leading -> trailing edge at radius r
            a = theta + np.deg2rad(kin.twist) * (r / Rr - kin.twist_ref)
            return -tg * np.cos(a) - nf * np.sin(a)

        def pt(r, s):
            return hubv + r * erf + (s - 0.25 * c) * cdir(r)

        for i in range(n_span):
            r0, r1 = r_nodes[i], r_nodes[i + 1]
            rm = 0.5 * (r0 + r1)
            nrm = np.cross(cdir(rm), erf)
            nrm /= np.linalg.norm(nrm)
            for j in range(n_chord):
                s0, s1 = xi[j] + 0.25 * dxi, xi[j + 1] + 0.25 * dxi
                rings.append([pt(r0, s0), pt(r0, s1), pt(r1, s1), pt(r1, s0)])
                y = pt(rm, xi[j] + 0.75 * dxi)
                colloc.append(y)
                normal.append(nrm)
                vrel.append(u_inf - np.cross(om, y - hubv))
    rings = np.asarray(rings)
    te, te_idx = blade_trailing_edge(rings, n_blades, n_span, n_chord)
    return RotorLattice(rings=rings, colloc=np.asarray(colloc), normal=np.asarray(normal), v_rel=np.asarray(vrel),
                        omega_b=np.asarray(omegas), te=te, te_idx=te_idx)


def ring_segments(rings, gam):
    """The four straight segments c0->c1->c2->c3->c0 of every ring, carrying its circulation."""
    nr = rings.shape[0]
    a = np.zeros((4 * nr, 4))
    b = np.zeros((4 * nr, 4))
    for s in range(4):
        a[s::4, :3] = rings[:, s, :3]
        b[s::4, :3] = rings[:, (s + 1) % 4, :3]
        a[s::4, 3] = gam
    return a, b


def _pack(name, sigma, xyz, G, rings, colloc, normal, vrel, gam, seg_core=None, u_inf=(0.0, 0.0, 0.0), meta=None):
    a, b = ring_segments(rings, gam)
    ring4 = np.zeros(rings.shape[:2] + (4,))
    ring4[..., :3] = rings
    return Wake(
        name=name,
        sigma=float(np.float32(sigma)),
        pos=_f32(_pad4(xyz, sigma ** 3)),
        strength=_f32(_pad4(G, 0.0)),
        seg_a=_f32(a),
        seg_b=_f32(b),
        rings=_f32(ring4),
        colloc=_f32(_pad4(colloc, 0.0)),
        normal=_f32(_pad4(normal, 0.0)),
        v_rel=_f32(_pad4(vrel, 0.0)),
        seg_core=float(np.float32(sigma if seg_core is None else seg_core)),
        u_inf=tuple(float(np.float32(v)) for v in u_inf),
        meta=meta or {},
    )


def _landgrebe(ct=0.005):
    lam = 0.145 + 27.0 * ct
    return lambda psi: R * (0.78 + 0.22 * np.exp(-lam * psi))


def small_hover(seed=0, n=2000):
    """2-blade hover, 20 x 4 panels per blade, n particles on 2 tip spirals over 3 revolutions, sigma 0.02R."""
    rng = np.random.default_rng(seed)
    sigma = 0.02 * R
    parts = []
    for h in range(2):
        nh = n // 2 + (1 if h < n % 2 else 0)
        parts.append(helix(rng, nh, phase=np.pi * h, revs=3, pitch=0.1 * R, r_of_age=lambda p: R + 0 * p,
                           jitter=0.01 * R))
    xyz = np.concatenate([p[0] for p in parts])
    G = np.concatenate([p[1] for p in parts])
    rings, colloc, normal, vrel, gam = blade_lattice(2, 20, 4)
    return _pack("small_hover_2k", sigma, xyz, G, rings, colloc, normal, vrel, gam,
                 meta={"blades": 2, "panels": "20x4", "revs": 3})


def hover(seed=1, n=100_000, n_blades=4):
    """4-blade hover, 40 x 8 panels, n particles on 4 contracting tip spirals (10 revs), sigma 0.01R."""
    rng = np.random.default_rng(seed)
    sigma = 0.01 * R
    rofa = _landgrebe()
    parts = []
    for h in range(n_blades):
        nh = n // n_blades + (1 if h < n % n_blades else 0)
        parts.append(helix(rng, nh, phase=2 * np.pi * h / n_blades, revs=10, pitch=0.1 * R, r_of_age=rofa,
                           jitter=0.005 * R))
    xyz = np.concatenate([p[0] for p in parts])
    G = np.concatenate([p[1] for p in parts])
    rings, colloc, normal, vrel, gam = blade_lattice(n_blades, 40, 8)
    return _pack(f"hover4_{n // 1000}k", sigma, xyz, G, rings, colloc, normal, vrel, gam,
                 meta={"blades": n_blades, "panels": "40x8", "revs": 10})


def bvi(seed=2, n=1_000_000):
    """4-blade rotor at advance ratio 0.15, wake skewed 20 deg aft, plus three straight filaments
    parallel to blade 0 at 0.5, 1 and 2 sigma above its panels (blade-vortex interaction)."""
    rng = np.random.default_rng(seed)
    sigma = 0.01 * R
    mu = 0.15
    u_inf = (mu * OMEGA * R, 0.0, 0.0)
    aft = 2 * np.pi * mu * R
    descent = aft * np.tan(np.deg2rad(20.0))
    n_fil, per_fil = 3, 2000
    n_hel = n - n_fil * per_fil
    parts = []
    for h in range(4):
        nh = n_hel // 4 + (1 if h < n_hel % 4 else 0)
        parts.append(helix(rng, nh, phase=np.pi / 2 * h, revs=10, pitch=0.0, r_of_age=lambda p: R + 0 * p,
                           jitter=0.005 * R, drift=(aft, -descent)))
    rings, colloc, normal, vrel, gam = blade_lattice(4, 40, 8, u_inf=u_inf)
    # blade 0 lies along +x with 8 deg pitch: leading->trailing direction and panel normal
    th = np.deg2rad(8.0)
    cdir = np.array([0.0, -np.cos(th), -np.sin(th)])
    nrm = np.array([0.0, -np.sin(th), np.cos(th)])
    for hgt in (0.5 * sigma, 1.0 * sigma, 2.0 * sigma):
        s = np.linspace(0.15 * R, R, per_fil)
        xyz = (s[:, None] * np.array([1.0, 0.0, 0.0]) + (R / 6) * 0.25 * cdir + hgt * nrm)
        mag = rng.uniform(0.9e-3, 1.1e-3, size=per_fil)
        G = np.stack([mag, np.zeros_like(mag), np.zeros_like(mag)], axis=1)
        parts.append((xyz, G))
    xyz = np.concatenate([p[0] for p in parts])
    G = np.concatenate([p[1] for p in parts])
    return _pack(f"bvi4_{n // 1000}k", sigma, xyz, G, rings, colloc, normal, vrel, gam, u_inf=u_inf,
                 meta={"blades": 4, "panels": "40x8", "advance_ratio": mu, "skew_deg": 20})


def adjoint_hover(seed=3, n=200_000):
    """The hover wake of ``hover`` with n particles, for the downwash-loss adjoint at 1,280 control points."""
    w = hover(seed=seed, n=n)
    w.name = f"adjoint_hover4_{n // 1000}k"
    return w


def multirotor(seed=4, n=2_000_000):
    """Two 3-blade counter-rotating rotors, hubs 2.2R apart, 40 x 8 panels, wakes drifting toward
    the mid-plane (0.05R per revolution) so that they merge, sigma 0.008R."""
    rng = np.random.default_rng(seed)
    sigma = 0.008 * R
    rofa = _landgrebe()
    parts = []
    rings_l, coll_l, norm_l, vrel_l, gam_l = [], [], [], [], []
    for rot, (hx, spin) in enumerate(((-1.1 * R, 1.0), (1.1 * R, -1.0))):
        for h in range(3):
            k = rot * 3 + h
            nh = n // 6 + (1 if k < n % 6 else 0)
            parts.append(helix(rng, nh, phase=2 * np.pi * h / 3 * spin, revs=10, pitch=0.1 * R, r_of_age=rofa,
                               jitter=0.004 * R, centre=(hx, 0.0, 0.0), spin=spin,
                               drift=(-np.sign(hx) * 0.05 * R, 0.0)))
        rg, co, no, vr, ga = blade_lattice(3, 40, 8, hub=(hx, 0.0, 0.0), spin=spin)
        rings_l.append(rg), coll_l.append(co), norm_l.append(no), vrel_l.append(vr), gam_l.append(ga)
    xyz = np.concatenate([p[0] for p in parts])
    G = np.concatenate([p[1] for p in parts])
    return _pack(f"twin3_{n // 1000}k", sigma, xyz, G, np.concatenate(rings_l), np.concatenate(coll_l),
                 np.concatenate(norm_l), np.concatenate(vrel_l), np.concatenate(gam_l),
                 meta={"rotors": 2, "blades": 3, "panels": "40x8", "hub_spacing": 2.2})


CONFIGS = {1: small_hover, 2: hover, 3: bvi, 4: adjoint_hover, 5: multirotor}


def make(config: int, n: int | None = None) -> Wake:
    """Workload of the given configuration (1..5), seeded with config - 1; n overrides the particle count."""
    fn = CONFIGS[int(config)]
    return fn(seed=int(config) - 1) if n is None else fn(seed=int(config) - 1, n=int(n))


def random_cloud(seed, n, box=1.0, sigma=0.05, gamma=1e-3):
    """n particles uniform in a cube of side ``box`` with random strengths (ragged-size tests)."""
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-0.5 * box, 0.5 * box, size=(n, 3))
    G = rng.normal(size=(n, 3)) * gamma
    return _f32(_pad4(xyz, sigma ** 3)), _f32(_pad4(G, 0.0))


def random_segments(seed, m, box=1.0, length=0.1, gamma=1.0):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-0.5 * box, 0.5 * box, size=(m, 3))
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    b = a + length * d
    g = rng.uniform(-gamma, gamma, size=m)
    return _f32(_pad4(a, g)), _f32(_pad4(b, 0.0))


def random_rings(seed, n_rings, box=1.0, size=0.1, gamma=1.0):
    """Closed four-sided vortex rings as segments (4 per ring, side k from corner k to
    corner k + 1 mod 4, the ring's circulation on every side; end points shared bit
    for bit): non-planar random quadrilaterals of about `size` in a cube `box`."""
    rng = np.random.default_rng(seed)
    centre = rng.uniform(-0.5 * box, 0.5 * box, size=(n_rings, 1, 3))
    ang = np.sort(rng.uniform(0.0, 2.0 * np.pi, size=(n_rings, 4)), axis=1)
    rad = size * rng.uniform(0.3, 0.7, size=(n_rings, 4))
    c = np.stack([rad * np.cos(ang), rad * np.sin(ang), 0.2 * size * rng.normal(size=(n_rings, 4))], axis=2)
    rot = np.linalg.qr(rng.normal(size=(n_rings, 3, 3)))[0]
    corners = _f32(centre + np.einsum("rij,rkj->rki", rot, c))  # [n_rings, 4, 3]
    g = np.repeat(rng.uniform(-gamma, gamma, size=n_rings), 4)
    a = corners.reshape(-1, 3)
    b = np.roll(corners, -1, axis=1).reshape(-1, 3)
    return _f32(_pad4(a, g)), _f32(_pad4(b, 0.0))


def sample_targets(seed, n, k):
    """k distinct target indices out of n, sorted (subsampled parity and oracle timing)."""
    rng = np.random.default_rng(seed + 1000)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False))


def sample_runs(seed, n, n_runs, run, lo=0, hi=None):
    """n_runs runs of ``run`` consecutive particle indices in [lo, hi), sorted and
    non-overlapping (sampled checks of large wakes: consecutive particles of a
    filament share their neighbourhoods)."""
    hi = n if hi is None else hi
    rng = np.random.default_rng(seed + 2000)
    slots = (hi - lo) // run
    starts = lo + run * np.sort(rng.choice(slots, size=min(n_runs, slots), replace=False))
    return np.concatenate([np.arange(s, s + run) for s in starts])


def rotor_wake_edges(seed, n_rows, n_span=40, n_blades=4, dpsi_deg=5.0):
    """Edges of n_rows x n_blades near-wake panel rows behind a hover rotor (FP64):
    each row spans r = 0.15R..R between the trailing-edge line at one azimuth and the
    same line one time step (dpsi) earlier, dropped by a small inflow, so the trailed
    edges lengthen with radius (the geometry behind the adaptive count).  Panel
    circulations follow Gamma_0 (r/R) sqrt(1 - (r/R)^2) with a few percent of noise.
    Returns a, b [m, 3], gamma, gamma_nb [m], has_nb, trailed [m] (int32) and the
    length of the tip's trailed edge."""
    rng = np.random.default_rng(seed)
    r = np.linspace(0.15 * R, R, n_span + 1)
    dpsi = np.deg2rad(dpsi_deg)
    rc = 0.5 * (r[1:] + r[:-1])
    A, B, g, gnb, hn, tr = [], [], [], [], [], []
    for row in range(n_rows):
        for bl in range(n_blades):
            psi = 2 * np.pi * bl / n_blades + row * dpsi
            z0 = -0.01 * R * (row + 1)
            up = np.stack([r * np.cos(psi), r * np.sin(psi), np.full_like(r, z0)], 1)
            dn = np.stack([r * np.cos(psi - dpsi), r * np.sin(psi - dpsi), np.full_like(r, z0 - 0.01 * R)], 1)
            gam = 2.0 * (rc / R) * np.sqrt(1 - (rc / R) ** 2) * (1 + 0.02 * rng.normal(size=n_span))
            for q in range(n_span + 1):  # trailed edges, as a panel row's conversion lists them
                end = q == n_span
                A.append(up[q] if end else dn[q])
                B.append(dn[q] if end else up[q])
                g.append(gam[-1] if end else gam[q])
                has = (not end) and q > 0
                gnb.append(gam[q - 1] if has else 0.0)
                hn.append(int(has))
                tr.append(1)
            for p in range(n_span):  # shed edges, downstream then upstream lines
                A.append(dn[p + 1]), B.append(dn[p]), g.append(gam[p]), gnb.append(0.0), hn.append(0), tr.append(0)
            for p in range(n_span):
                A.append(up[p]), B.append(up[p + 1]), g.append(gam[p]), gnb.append(0.0), hn.append(0), tr.append(0)
    ds_tip = float(np.linalg.norm(np.array(B[n_span]) - np.array(A[n_span])))
    return (np.array(A), np.array(B), np.array(g), np.array(gnb), np.array(hn, dtype=np.int32),
            np.array(tr, dtype=np.int32), ds_tip)


def blade_trailing_edge(rings, n_blades, n_span, n_chord):
    """Trailing-edge node lines [n_blades, n_span + 1, 3] of blade_lattice rings (blades
    turning with spin +1: ring corners leading-root, trailing-root, trailing-tip,
    leading-tip), and the indices [n_blades, n_span] of the trailing-edge rings."""
    idx = np.zeros((n_blades, n_span), dtype=np.int64)
    te = np.zeros((n_blades, n_span + 1, 3))
    for b in range(n_blades):
        for i in range(n_span):
            k = (b * n_span + i) * n_chord + (n_chord - 1)
            idx[b, i] = k
            te[b, i] = rings[k, 1, :3]
        te[b, n_span] = rings[idx[b, n_span - 1], 2, :3]
    return te, idx
