"""Pins of the oracle's near-wake time loop (Sec. II.A-C) on a small hover rotor:
the shed rows convect downwards at the induced velocity of a hovering rotor (a wrong
Kutta sign or ring orientation makes the wake rise), every conversion conserves the
closed rings' zero net circulation, and Eq. 8 needs fewer particles than the uniform
count with the same tip resolution."""
import numpy as np

from oracle import kinematics
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
    a, b = kinematics.ring_segments(ring, np.array([2.0]))
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


def test_zero_lift_forward_flight_convects_with_the_free_stream():
    """Flat blades at zero pitch in the disk plane, free stream in that plane: the Neumann
    condition has a zero right-hand side, every circulation and load vanishes, and the
    wake is carried by the free stream alone.  Each node line is then the trailing edge
    of its shedding time moved by the free stream for its age, and every particle moves
    by dt u_inf per step (closed forms of Euler and of the RK3 step for a constant
    velocity)."""
    kin = synth.Kinematics(mu=0.19, theta=(0.0, 0.0, 0.0))
    o = OracleRotorWake(n_blades=2, n_span=6, n_chord=2, max_rows=2, n_tip=2, kin=kin)
    u = o.u_inf
    assert u[0] > 30.0 and u[1] == u[2] == 0.0
    x_prev = None
    for k in range(5):
        gam = o.step()
        assert np.all(gam == 0.0) and o.history[-1][1] == 0.0 and o.history[-1][2] == 0.0
        for r in range(o.rows + 1):  # line r was shed at time t - r dt (t after the step)
            te = kinematics.lattice(kin, o.t - r * o.dt, 2, 6, 2).te
            np.testing.assert_allclose(o.nodes[r], te + r * o.dt * u, rtol=0, atol=1e-12)
        if x_prev is not None and len(x_prev):
            np.testing.assert_allclose(o.x[:len(x_prev)], x_prev + o.dt * u, rtol=0, atol=1e-12)
            assert np.all(o.G == 0.0)
        x_prev = o.x.copy()
    assert len(o.x) > 0


def test_forward_flight_thrust_of_the_ah1g_case():
    """The AH-1G rotor of the forward-flight case with the pitch and flapping schedules of
    Eq. 12 at advance ratio 0.19: over the first revolution (after the starting transient)
    the thrust coefficient averages within 25 % of the paper's printed NL-UVLM-VPM value,
    C_T = 0.00478 (Table 4).  A loose bound: the 2D viscous coupling is not part of this
    path and the lattice is coarse (12 x 3 panels per blade, 10 deg steps)."""
    kin = synth.AH1G
    o = OracleRotorWake(n_blades=2, n_span=12, n_chord=3, max_rows=2, n_tip=3, kin=kin,
                        dt=np.deg2rad(10.0) / kin.omega)
    for _ in range(24):
        o.step()
    ct = np.array([h[1] for h in o.history])
    assert np.all(ct[3:] > 0)
    from tests.test_synth_kinematics import golden_ah1g

    assert abs(ct[6:].mean() / golden_ah1g()["C_T_NL_UVLM_VPM"] - 1.0) < 0.25
