"""Pins of the oracle's near-wake time loop (Sec. II.A-C) on a small hover rotor:
the shed rows convect downwards at the induced velocity of a hovering rotor (a wrong
Kutta sign or ring orientation makes the wake rise), every conversion conserves the
closed rings' zero net circulation, and Eq. 8 needs fewer particles than the uniform
count with the same tip resolution."""
import numpy as np

from oracle.wake_loop import OracleRotorWake
from paper_2511_11430_gb300 import synth


def test_shed_rows_move_down_at_the_hover_induced_velocity():
    o = OracleRotorWake(n_blades=2, n_span=12, n_chord=3, max_rows=5, n_tip=3)
    for _ in range(4):
        o.step()
    z = o.nodes[..., 2].mean(axis=(1, 2))  # line 0 at the trailing edge, then older lines
    assert z[1] < z[0] and z[2] < z[1] and z[3] < z[2]
    w = -(z[2] - z[1]) / o.dt  # descent per step between two free lines
    # momentum theory for the synthetic blades' loading: O(10 m/s) at Omega R = 200 m/s
    assert 2.0 < w < 30.0


def test_conversions_keep_zero_net_circulation_and_adaptive_is_leaner():
    kw = dict(n_blades=2, n_span=12, n_chord=3, max_rows=1, n_tip=4, n_shed=1)
    a = OracleRotorWake(adaptive=True, **kw)
    c = OracleRotorWake(adaptive=False, **kw)
    a.step(), c.step()
    n_before = len(a.x)
    a.step(), c.step()  # the first conversion (no particles to convect yet before it)
    assert n_before == 0 and len(a.x) > 0
    np.testing.assert_allclose(a.G.sum(0), 0.0, atol=1e-12)
    np.testing.assert_allclose(c.G.sum(0), 0.0, atol=1e-12)
    assert len(a.x) < len(c.x)
    # the conventional count is exact: n_tip per trailed edge, n_shed per shed edge
    S, nb = kw["n_span"], kw["n_blades"]
    assert len(c.x) == nb * ((S + 1) * 4 + 2 * S * 1)


def test_kutta_joukowski_pins():
    """A closed ring in a uniform stream carries no force; one straight bound segment of
    circulation Gamma and length L across a stream V carries rho Gamma |V| L along V x dl;
    a panel whose circulation grows at dGamma/dt gets rho dGamma/dt A along its normal."""
    import oracle

    ring = np.array([[[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]]], float)
    a, b = synth.ring_segments(ring, np.array([2.0]))
    nrm = np.array([[0.0, 0.0, 1.0, 0.0]])
    F, _ = oracle.blade_loads(a, b, np.zeros((4, 3)), [0, 0, 0], [0, 0, 0], [3.0, 1.0, 0.5], ring, nrm, [2.0], None,
                              1e-3, rho=1.2)
    np.testing.assert_allclose(F, 0.0, atol=1e-14)
    sa = np.array([[0.0, 0.0, 0.0, 1.5]])
    sb = np.array([[0.0, 2.0, 0.0, 0.0]])
    F, M = oracle.blade_loads(sa, sb, np.zeros((1, 3)), [0, 0, 0], [0, 0, 0], [10.0, 0.0, 0.0], ring, nrm, [0.0],
                              None, 1e-3, rho=1.2)
    np.testing.assert_allclose(F, [0.0, 0.0, 1.2 * 1.5 * 10.0 * 2.0], rtol=1e-15)  # (10,0,0) x (0,2,0) = +z
    np.testing.assert_allclose(M, np.cross([0.0, 1.0, 0.0], F), rtol=1e-15)
    F, _ = oracle.blade_loads(sa[:0], sb[:0], np.zeros((0, 3)), [0, 0, 0], [0, 0, 0], [0, 0, 0], ring, nrm, [3.0],
                              [1.0], 0.5, rho=1.2)
    np.testing.assert_allclose(F, [0.0, 0.0, 1.2 * (3.0 - 1.0) / 0.5 * 1.0], rtol=1e-15)


def test_rotor_thrust_builds_up_to_the_momentum_theory_range():
    """Started impulsively, the synthetic rotor's thrust coefficient grows as the starting
    vortex leaves the trailing edge and settles in the range blade-element momentum
    theory gives for 8 deg collective and this solidity (C_T of order 0.01)."""
    o = OracleRotorWake(n_blades=2, n_span=12, n_chord=3, max_rows=4, n_tip=3)
    for _ in range(10):
        o.step()
    ct = np.array([h[1] for h in o.history])
    cq = np.array([h[2] for h in o.history])
    assert ct[-1] > ct[2] > 0
    assert 0.004 < ct[-1] < 0.02
    assert 0.0 < cq[-1] < 0.1 * ct[-1]
