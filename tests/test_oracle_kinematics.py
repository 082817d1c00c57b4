"""Pins of the oracle's blade kinematics (oracle/kinematics.py), the prescribed motion
of Sec. IV.B (Eq. 12 pitch and flapping schedules) that the oracle's near-wake loop
uses: the schedules read back from the placed lattice, the blade velocity against
central differences of the lattice in time, hover in closed form, and agreement
with the product's own lattice generator (an independent implementation)."""
import dataclasses

import numpy as np
import pytest

from oracle import kinematics as K
from paper_2511_11430_gb300 import synth


def _flat(kin):
    return dataclasses.replace(kin, twist=0.0)


@pytest.mark.parametrize("psi_deg", [0.0, 37.0, 90.0, 200.0, 311.0])
def test_schedules_read_back_from_the_lattice(psi_deg):
    """Blade 0 at azimuth psi: the span axis rises at the flap angle beta(psi) and the
    chord line is pitched nose up by theta(psi) relative to the flapped disk plane."""
    kin = _flat(synth.AH1G)
    psi = np.deg2rad(psi_deg)
    t = psi / kin.omega
    nb, S, nc = 2, 6, 1
    L = K.lattice(kin, t, nb, S, nc)
    r0 = L.rings[0]          # root panel of blade 0: corners LR, TR, TT, LT
    rS = L.rings[S - 1]      # tip panel
    span = rS[3] - r0[0]     # leading corners, same chordwise station
    span /= np.linalg.norm(span)
    beta = np.arcsin(span[2])
    chord = r0[1] - r0[0]    # leading -> trailing at the root station
    chord /= np.linalg.norm(chord)
    e_r = np.array([np.cos(psi), np.sin(psi), 0.0])
    n_f = np.cos(beta) * np.array([0.0, 0.0, 1.0]) - np.sin(beta) * e_r
    theta = -np.arcsin(chord @ n_f)
    th = kin.theta[0] + kin.theta[1] * np.cos(psi) + kin.theta[2] * np.sin(psi)
    be = kin.beta[0] + kin.beta[1] * np.cos(psi) + kin.beta[2] * np.sin(psi)
    assert np.rad2deg(beta) == pytest.approx(be, abs=1e-9)
    assert np.rad2deg(theta) == pytest.approx(th, abs=1e-9)
    # the span axis lies in the vertical plane of the azimuth
    assert abs(span @ np.array([-np.sin(psi), np.cos(psi), 0.0])) < 1e-12


@pytest.mark.parametrize("kin", [synth.AH1G, dataclasses.replace(synth.AH1G, beta=(3.0, 2.13, -0.15))],
                         ids=["ah1g", "coned"])
def test_blade_velocity_equals_central_differences_of_the_lattice(kin):
    """omega_b x (y - hub) equals d y / dt of every control point and ring corner by
    central differences in time (rigid-body motion of each blade)."""
    nb, S, nc = 2, 5, 2
    t, h = 0.021, 1e-6
    Lm, L0, Lp = (K.lattice(kin, tt, nb, S, nc) for tt in (t - h, t, t + h))
    u_inf = np.array([kin.mu * kin.omega * kin.radius, 0.0, 0.0])
    dy = (Lp.colloc - Lm.colloc) / (2 * h)
    np.testing.assert_allclose(u_inf - L0.v_rel, dy, rtol=1e-7, atol=1e-7 * np.abs(dy).max())
    per = S * nc
    for b in range(nb):
        c = L0.rings[b * per:(b + 1) * per]
        dc = (Lp.rings[b * per:(b + 1) * per] - Lm.rings[b * per:(b + 1) * per]) / (2 * h)
        np.testing.assert_allclose(np.cross(L0.omega_b[b], c), dc, rtol=1e-7, atol=1e-7 * np.abs(dc).max())


def test_hover_is_steady_rotation():
    kin = synth.Kinematics()
    L = K.lattice(kin, 0.004, 3, 4, 2)
    np.testing.assert_allclose(L.omega_b, [[0.0, 0.0, kin.omega]] * 3, atol=1e-12)
    ez = np.array([0.0, 0.0, 1.0])
    np.testing.assert_allclose(L.v_rel, -np.cross(kin.omega * ez, L.colloc), atol=1e-10)
    # 8 deg collective: the normals tilt 8 deg from the axis, towards the direction of travel
    assert np.allclose(L.normal @ ez, np.cos(np.deg2rad(8.0)))


def test_ring_segments_close_each_ring():
    L = K.lattice(synth.AH1G, 0.01, 2, 3, 2)
    g = np.arange(L.rings.shape[0], dtype=np.float64) + 1.0
    a, b = K.ring_segments(L.rings, g)
    assert np.array_equal(a[:, 3], np.repeat(g, 4))
    np.testing.assert_array_equal(b[0::4, :3], a[1::4, :3])
    np.testing.assert_array_equal(b[3::4, :3], a[0::4, :3])


@pytest.mark.parametrize("t", [0.0, 0.013, 0.37])
def test_oracle_lattice_agrees_with_the_product_generator(t):
    """The product's lattice (synth.rotor_lattice, written from the blade-axis form of
    the angular velocity) and the oracle's (rotation matrices) agree to round-off."""
    for kin in (synth.Kinematics(), synth.AH1G):
        P = synth.rotor_lattice(kin, t, 2, 6, 3)
        O = K.lattice(kin, t, 2, 6, 3)
        for a, b in ((P.rings, O.rings), (P.colloc, O.colloc), (P.normal, O.normal), (P.te, O.te)):
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * kin.radius)
        np.testing.assert_allclose(P.v_rel, O.v_rel, rtol=0, atol=1e-12 * np.abs(O.v_rel).max())
        np.testing.assert_allclose(P.omega_b, O.omega_b, rtol=0, atol=1e-12 * kin.omega)
        assert np.array_equal(P.te_idx, O.te_idx)
