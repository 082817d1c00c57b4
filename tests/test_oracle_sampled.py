"""The sampled assembly of the oracle's right-hand side (oracle/sampled.py) that the
full-size GPU checks use: on a wake small enough for the oracle's full right-hand
side, the sampled values equal the full ones at those particles."""
import numpy as np
import pytest

import oracle
from oracle import sampled
from paper_2511_11430_gb300 import synth
from tests._util import rel_l2


@pytest.fixture(scope="module")
def wake():
    return synth.make(1)


def test_pse_at_equals_pse_rows(wake):
    w = wake
    nut = np.random.default_rng(0).uniform(0.0, 1e-4, w.n)
    p = oracle.pse(w.pos, w.strength, nut, w.sigma, w.nu)
    idx = np.array([0, 5, 777, w.n - 1])
    np.testing.assert_array_equal(oracle.pse_at(w.pos, w.strength, nut, w.sigma, w.nu, idx), p[idx])


@pytest.mark.parametrize("c_v", [0.07, 0.0])
def test_sampled_rhs_equals_full_rhs(wake, c_v):
    w = wake
    rdx, rdG, rnut = oracle.rhs(w.pos, w.strength, w.seg_a, w.seg_b, w.sigma, nu=w.nu, c_v=c_v,
                                seg_core=w.seg_core, u_inf=w.u_inf)
    idx = synth.sample_runs(1, w.n, 4, 16)
    dx, dG, nut = sampled.rhs_at(w, idx, c_v=c_v)
    assert rel_l2(dx, rdx[idx]) <= 1e-14
    assert rel_l2(dG, rdG[idx]) <= 1e-14
    if c_v > 0:
        assert rel_l2(nut, rnut[idx]) <= 1e-14


def test_sample_runs_are_disjoint_runs():
    idx = synth.sample_runs(3, 1000, 5, 16)
    assert len(idx) == 80 and len(set(idx.tolist())) == 80
    starts = idx[::16]
    assert np.all(idx.reshape(5, 16) == starts[:, None] + np.arange(16)[None, :])
