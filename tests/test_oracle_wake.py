"""Pins of the oracle's wake panel -> particle conversion (Sec. II.C, Eq. 6-8).

The conversion is a plain definition (counts, positions, strengths), so the pins are
the equations themselves on hand-checkable cases, exact rational arithmetic for the
integer counts of Eq. 8, conservation of the converted circulation, and the velocity
of the converted particles converging to that of the panel row they replace."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _edges(lens, trailed=1):
    m = len(lens)
    a = np.zeros((m, 3))
    b = np.zeros((m, 3))
    b[:, 0] = lens
    a[:, 1] = np.arange(m)
    b[:, 1] = np.arange(m)
    return a, b, np.ones(m), np.zeros(m), np.zeros(m, dtype=np.int32), np.full(m, trailed, dtype=np.int32)


@pytest.mark.parametrize("n_tip", [1, 2, 3, 7])
def test_tip_edge_gets_exactly_n_tip(n_tip):
    a, b, g, gnb, hn, tr = _edges([0.37])
    x, G, c = oracle.wake_convert(a, b, g, gnb, hn, tr, ds_tip=0.37, n_tip=n_tip)
    assert c.tolist() == [n_tip]


def test_counts_are_the_exact_ceiling_of_eq8():
    rng = np.random.default_rng(0)
    lens = rng.uniform(0.01, 3.0, size=400)
    ds_tip, n_tip = 0.23, 3
    a, b, g, gnb, hn, tr = _edges(lens)
    _, _, c = oracle.wake_convert(a, b, g, gnb, hn, tr, ds_tip=ds_tip, n_tip=n_tip)
    for L, n in zip(lens, c):
        exact = Fraction(float(L)) / Fraction(ds_tip) * n_tip
        if abs(exact - round(exact)) < Fraction(1, 10**9):
            continue  # a near-tie is decided by rounding; skip it
        assert n == math.ceil(exact)


def test_conventional_strategy_is_one_particle_per_edge():
    lens = [0.1, 0.4, 0.9, 1.0]
    a, b, g, gnb, hn, tr = _edges(lens)
    _, _, c = oracle.wake_convert(a, b, g, gnb, hn, tr, ds_tip=max(lens), n_tip=1)
    assert c.tolist() == [1, 1, 1, 1]
    a, b, g, gnb, hn, tr = _edges(lens, trailed=0)
    _, _, c = oracle.wake_convert(a, b, g, gnb, hn, tr, ds_tip=0.1, n_tip=5, n_shed=1)
    assert c.tolist() == [1, 1, 1, 1]  # shed edges take n_shed, not Eq. 8


def test_eq6_strengths_sum_to_delta_gamma_dl_and_eq7_neighbour_rule():
    a = np.array([[0.1, 0.2, 0.3], [1.0, -1.0, 0.5]])
    b = np.array([[0.9, -0.4, 1.3], [-0.5, 0.25, 2.0]])
    g = np.array([2.0, -1.5])
    gnb = np.array([0.5, 7.0])
    hn = np.array([1, 0], dtype=np.int32)
    x, G, c = oracle.wake_convert(a, b, g, gnb, hn, [1, 1], ds_tip=0.3, n_tip=2)
    o = 0
    for i, n in enumerate(c):
        dG = g[i] - gnb[i] if hn[i] else g[i]
        np.testing.assert_allclose(G[o:o + n].sum(0), dG * (b[i] - a[i]), rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(G[o:o + n], np.tile(dG * (b[i] - a[i]) / n, (n, 1)), rtol=1e-15)
        o += n


def test_particles_sit_at_the_centres_of_equal_pieces():
    a = np.array([[1.0, 2.0, 3.0]])
    b = np.array([[3.0, 2.0, 7.0]])
    x, G, c = oracle.wake_convert(a, b, [1.0], None, None, [1], ds_tip=float(np.linalg.norm(b - a)), n_tip=4)
    assert c.tolist() == [4]
    t = np.array([0.125, 0.375, 0.625, 0.875])
    np.testing.assert_allclose(x, a + t[:, None] * (b - a), rtol=0, atol=1e-15)
    np.testing.assert_allclose(x.mean(0), 0.5 * (a[0] + b[0]), atol=1e-15)  # symmetric about the midpoint


def _row(S=6, span=1.0, chord=0.3, seed=0):
    rng = np.random.default_rng(seed)
    y = np.linspace(0.2, 0.2 + span, S + 1)
    U = np.stack([np.zeros(S + 1), y, 0.02 * rng.normal(size=S + 1)], 1)
    D = np.stack([chord * (0.5 + y), y, 0.02 * rng.normal(size=S + 1)], 1)  # longer outboard, like a rotor wake
    gamma = 1.0 + rng.uniform(-0.3, 0.3, size=S)
    return U, D, gamma


def test_row_edges_topology_and_closed_rings_sum_to_zero():
    U, D, gamma = _row()
    a, b, g, gnb, hn, tr = oracle.wake_row_edges(U, D, gamma)
    S = gamma.size
    assert len(a) == 3 * S + 1 and tr.sum() == S + 1 and hn.sum() == S - 1
    # trailed edge at the tip is the longest, use it as the reference
    ds_tip = np.linalg.norm(b[S] - a[S])
    x, G, c = oracle.wake_convert(a, b, g, gnb, hn, tr, ds_tip=ds_tip, n_tip=3, n_shed=2)
    assert c[S] == 3 and all(c[:S + 1] <= 3) and all(c[S + 1:] == 2)
    np.testing.assert_allclose(G.sum(0), 0.0, atol=1e-14)  # every ring is a closed loop


def test_converted_particles_induce_the_velocity_of_the_panel_row():
    """Far from the row, the converted particles (point vortices: Gaussian blobs of tiny
    sigma) reproduce the velocity of the row's rings as vortex segments, with an error
    that falls at second order in the particle spacing."""
    U, D, gamma = _row(S=4)
    a, b, g, gnb, hn, tr = oracle.wake_row_edges(U, D, gamma)
    # the rings as segments: four per panel
    sa, sb = [], []
    for p in range(gamma.size):
        corners = [U[p], U[p + 1], D[p + 1], D[p]]
        for k in range(4):
            sa.append([*corners[k], gamma[p]])
            sb.append([*corners[(k + 1) % 4], 0.0])
    tgt = np.array([[0.2, 0.6, 1.5, 0.0], [-1.0, 0.4, 0.8, 0.0], [0.9, 2.2, -1.1, 0.0]])
    u_ref = oracle.segments(np.array(sa), np.array(sb), tgt, 1e-9, grad=False)
    ds_tip = np.linalg.norm(b[gamma.size] - a[gamma.size])
    errs = []
    for nt in (2, 4, 8):
        x, G, c = oracle.wake_convert(a, b, g, gnb, hn, tr, ds_tip=ds_tip, n_tip=nt, n_shed=nt)
        pos = np.concatenate([x, np.full((len(x), 1), 1e-27)], 1)
        u = oracle.p2p(pos, G, tgt, 1e-6, grad=False)
        errs.append(np.abs(u - u_ref).max() / np.abs(u_ref).max())
    assert errs[-1] < 1e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0  # second order


def test_conventional_strategy_gives_every_trailed_edge_the_same_count():
    """A negative n_tip: -n_tip particles on every trailed edge whatever its length
    (the uniform strategy Eq. 8 replaces); shed edges keep n_shed."""
    U, D, gamma = _row()
    a, b, g, gnb, hn, tr = oracle.wake_row_edges(U, D, gamma)
    S = gamma.size
    ds_tip = np.linalg.norm(b[S] - a[S])
    _, _, conv = oracle.wake_convert(a, b, g, gnb, hn, tr, ds_tip=ds_tip, n_tip=-3, n_shed=1)
    _, _, adap = oracle.wake_convert(a, b, g, gnb, hn, tr, ds_tip=ds_tip, n_tip=3, n_shed=1)
    assert all(conv[:S + 1] == 3) and all(conv[S + 1:] == 1)
    assert adap[S] == 3 and adap[:S + 1].sum() < conv[:S + 1].sum()
