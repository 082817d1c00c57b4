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
