"""The prescribed rotor motion (Sec. IV.B, Eq. 12 form) of the synthetic input module:
the blade lattice of ``synth.rotor_lattice`` against the closed forms it must meet.

* hover kinematics reproduce ``synth.blade_lattice`` bit for bit;
* the AH-1G preset carries the values printed in Sec. IV.B (tests/golden), and the pitch
  and flap angles read back from the lattice equal the Eq. 12 schedules at psi = 0, 90,
  180 and 270 deg, with the -10 deg linear twist of the rotor's property table;
* every ring corner and control point moves with omega_b x (x - hub): central finite
  differences of the lattice in time against the stated angular velocity, and v_rel is
  the free stream minus that motion;
* a two-bladed teetering rotor with first-harmonic schedules and no coning turns as one
  rigid body (both blades share one angular velocity);
* the free stream is mu Omega R along +x (psi = 0 downstream).
"""
import dataclasses
import os

import numpy as np
import pytest

from paper_2511_11430_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ah1g_forward_flight.txt")


def golden_ah1g():
    """The AH-1G values printed in Sec. IV.B (Eq. 12, Tables 3 and 4)."""
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if len(line) == 2:
            out[line[0]] = float(line[1])
    return out


def test_ah1g_preset_is_the_printed_case():
    g = golden_ah1g()
    k = synth.AH1G
    assert k.theta == (g["theta_0"], g["theta_1c"], g["theta_1s"])
    assert k.beta == (0.0, g["beta_1c"], g["beta_1s"])
    assert (k.radius, k.chord, k.twist) == (g["radius"], g["chord"], g["twist"])
    assert k.root == pytest.approx(g["root_cutout"] * g["radius"], rel=1e-15)
    assert k.mu == g["advance_ratio"]
    assert k.omega * k.radius == pytest.approx(g["tip_mach"] * 340.3, rel=1e-15)


def test_hover_kinematics_reduce_to_blade_lattice():
    for nb, S, nc, t in ((2, 10, 3, 0.0), (4, 7, 2, 0.0), (3, 5, 4, 0.0123)):
        L = synth.rotor_lattice(synth.Kinematics(), t, nb, S, nc)
        r, c, n, v, _ = synth.blade_lattice(nb, S, nc, phase=synth.OMEGA * t)
        assert np.array_equal(L.rings, r) and np.array_equal(L.colloc, c)
        assert np.array_equal(L.normal, n) and np.array_equal(L.v_rel, v)
        assert np.allclose(L.omega_b, [[0.0, 0.0, synth.OMEGA]] * nb, rtol=0, atol=0)


def _flap(L, b, S, nc, i):
    """Flap angle [deg] and azimuth of blade b's strip i, from its leading edge (no twist)."""
    c = L.rings[(b * S + i) * nc]
    span = c[3] - c[0]  # leading-root -> leading-tip corner, along the flapped blade axis
    span /= np.linalg.norm(span)
    return np.degrees(np.arcsin(span[2])), np.arctan2(span[1], span[0])


def _pitch(L, b, S, nc, i, psi, beta_deg):
    """Pitch [deg] of blade b's strip i at its root radius: the chord line (corner 0 -> 1)
    against the disk plane flapped by beta."""
    c = L.rings[(b * S + i) * nc]
    chord = (c[1] - c[0]) / np.linalg.norm(c[1] - c[0])
    be = np.radians(beta_deg)
    nf = np.array([-np.sin(be) * np.cos(psi), -np.sin(be) * np.sin(psi), np.cos(be)])
    return np.degrees(np.arcsin(-chord @ nf))  # trailing edge below the flapped disk plane


@pytest.mark.parametrize("psi_deg", [0.0, 90.0, 180.0, 270.0])
def test_eq12_schedules_read_back(psi_deg):
    g = golden_ah1g()
    c, sn = np.cos(np.radians(psi_deg)), np.sin(np.radians(psi_deg))
    theta = g["theta_0"] + g["theta_1c"] * c + g["theta_1s"] * sn
    beta = g["beta_1c"] * c + g["beta_1s"] * sn
    S, nc = 16, 3
    kin = synth.AH1G
    t = np.radians(psi_deg) / kin.omega
    flat = synth.rotor_lattice(dataclasses.replace(kin, twist=0.0), t, 2, S, nc)
    L = synth.rotor_lattice(kin, t, 2, S, nc)
    r_nodes = np.linspace(kin.root, kin.radius, S + 1)
    psi = np.radians(psi_deg)
    for i in (0, 7, 15):
        flap, az = _flap(flat, 0, S, nc, i)
        assert flap == pytest.approx(beta, abs=1e-9)
        assert np.cos(az - psi) == pytest.approx(1.0, abs=1e-12)
        twist = kin.twist * (r_nodes[i] / kin.radius - kin.twist_ref)
        assert _pitch(L, 0, S, nc, i, psi, beta) == pytest.approx(theta + twist, abs=1e-9)
    # blade 1 sits half a turn later: the schedules at psi + 180 deg
    flap1, _ = _flap(flat, 1, S, nc, 3)
    assert flap1 == pytest.approx(-beta, abs=1e-9)
    th1 = g["theta_0"] - (theta - g["theta_0"]) + kin.twist * (r_nodes[3] / kin.radius - kin.twist_ref)
    assert _pitch(L, 1, S, nc, 3, psi + np.pi, -beta) == pytest.approx(th1, abs=1e-9)


@pytest.mark.parametrize("t", [0.0, 0.0137, 0.0911])
def test_lattice_moves_with_the_blade_angular_velocity(t):
    kin = synth.AH1G
    nb, S, nc = 2, 6, 3
    h = 1e-6 / kin.omega
    Lm = synth.rotor_lattice(kin, t - h, nb, S, nc)
    L0 = synth.rotor_lattice(kin, t, nb, S, nc)
    Lp = synth.rotor_lattice(kin, t + h, nb, S, nc)
    vel_c = (Lp.rings - Lm.rings) / (2 * h)   # [nr, 4, 3]
    vel_y = (Lp.colloc - Lm.colloc) / (2 * h)
    per = S * nc
    scale = kin.omega * kin.radius
    for b in range(nb):
        sl = slice(b * per, (b + 1) * per)
        om = L0.omega_b[b]
        want_c = np.cross(om, L0.rings[sl])
        want_y = np.cross(om, L0.colloc[sl])
        assert np.abs(vel_c[sl] - want_c).max() <= 1e-6 * scale
        assert np.abs(vel_y[sl] - want_y).max() <= 1e-6 * scale
    assert np.abs(L0.v_rel - (np.asarray(kin.u_inf) - vel_y)).max() <= 1e-6 * scale
    # the angular velocity has the shaft speed plus the flap and pitch rates
    assert np.all(np.abs(L0.omega_b[:, 2] - kin.omega) < 0.1 * kin.omega)


def test_teetering_rotor_turns_as_one_body():
    kin = synth.AH1G
    assert kin.beta[0] == 0.0
    for t in (0.0, 0.021, 0.05):
        L = synth.rotor_lattice(kin, t, 2, 4, 2)
        assert np.allclose(L.omega_b[0], L.omega_b[1], rtol=0, atol=1e-12 * kin.omega)
    # with coning the two blades no longer share it
    coned = synth.Kinematics(theta=(6.0, 1.7, -5.5), beta=(3.0, 2.13, -0.15))
    L = synth.rotor_lattice(coned, 0.01, 2, 4, 2)
    assert not np.allclose(L.omega_b[0], L.omega_b[1])


def test_free_stream_and_normals():
    kin = synth.AH1G
    assert kin.u_inf[0] == pytest.approx(0.19 * 0.65 * 340.3)
    assert kin.u_inf[1] == kin.u_inf[2] == 0.0
    L = synth.rotor_lattice(kin, 0.03, 2, 8, 3)
    assert np.allclose(np.linalg.norm(L.normal, axis=1), 1.0)
    assert np.all(L.normal[:, 2] > 0.9)  # pitch and flap of a few degrees: normals near +z
    # on the advancing side (psi = 90 deg) the relative wind at the tip is
    # (1 + mu) Omega R, on the retreating side (psi = 270 deg) (1 - mu) Omega R in size
    Ladv = synth.rotor_lattice(synth.Kinematics(mu=0.19, theta=(0, 0, 0)), np.pi / 2 / synth.OMEGA, 2, 8, 1)
    tip = 7  # blade 0's outermost strip, one chordwise panel
    y = Ladv.colloc[tip]
    want = synth.OMEGA * np.hypot(y[0], y[1]) + 0.19 * synth.OMEGA * synth.R
    assert np.linalg.norm(Ladv.v_rel[tip]) == pytest.approx(want, rel=0.02)
    ret = 8 + 7  # blade 1 at psi = 270 deg
    y = Ladv.colloc[ret]
    want = synth.OMEGA * np.hypot(y[0], y[1]) - 0.19 * synth.OMEGA * synth.R
    assert np.linalg.norm(Ladv.v_rel[ret]) == pytest.approx(want, rel=0.02)
