"""The near-wake time loop (shedding, convection, conversion, loads: Sec. II.A-C) run
through the library against the FP64 oracle loop on a small rotor, in hover and in the
forward flight of the AH-1G case (Eq. 12 schedules, free stream): blade circulations
and thrust/torque coefficients each step, the particle count after conversions (an
integer decided in FP64 on both sides), and the converted and convected particles."""
import numpy as np
import pytest

from oracle.wake_loop import OracleRotorWake
from tests._util import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wake_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11430_gb300 import build, wake

    build.build()
    return wake


@pytest.mark.parametrize("adaptive, flight", [(True, "hover"), (False, "hover"), (True, "ah1g"), (False, "ah1g")])
def test_rotor_wake_loop_matches_oracle(wake_mod, adaptive, flight):
    kw = dict(n_blades=2, n_span=12, n_chord=3, max_rows=2, n_tip=3, n_shed=1, adaptive=adaptive)
    if flight == "ah1g":  # forward flight: Eq. 12 pitch and flapping, advance ratio 0.19, 10 deg steps
        from paper_2511_11430_gb300 import synth

        kw.update(kin=synth.AH1G, dt=np.deg2rad(10.0) / synth.AH1G.omega)
    g = wake_mod.RotorWake(**kw)
    o = OracleRotorWake(**kw)
    for _ in range(6):
        gg = g.step().cpu().numpy()
        go = o.step()
        assert rel_l2(gg, go) <= 2e-5
    torch.cuda.synchronize()
    assert g.n == len(o.x) > 0 and g.rows == o.rows
    assert rel_l2(g.x.cpu().numpy().T, o.x) <= 1e-6
    assert rel_l2(g.G.cpu().numpy().T, o.G) <= 2e-5
    assert rel_l2(g.nodes.cpu().numpy(), o.nodes) <= 1e-6
    hg, ho = np.array(g.history), np.array(o.history)
    np.testing.assert_allclose(hg[:, 1], ho[:, 1], rtol=1e-4, atol=1e-8)  # C_T per step
    np.testing.assert_allclose(hg[:, 2], ho[:, 2], rtol=1e-3, atol=1e-3 * np.abs(ho[:, 2]).max())  # C_Q


def test_adaptive_conversion_creates_fewer_particles(wake_mod):
    """Eq. 8 against the uniform count: same tip resolution, fewer particles inboard."""
    kw = dict(n_blades=2, n_span=12, n_chord=3, max_rows=1, n_tip=4, n_shed=1)
    a = wake_mod.RotorWake(adaptive=True, **kw)
    c = wake_mod.RotorWake(adaptive=False, **kw)
    for _ in range(4):
        a.step()
        c.step()
    assert 0 < a.n < c.n


def test_rotor_wake_with_the_treecode_step(wake_mod):
    """The driver with the treecode step at theta = 0 (every cluster opened: the direct
    sums in plain FP32) follows the driver with the direct compensated step."""
    kw = dict(n_blades=2, n_span=12, n_chord=3, max_rows=2, n_tip=3, n_shed=1)
    a = wake_mod.RotorWake(**kw)
    b = wake_mod.RotorWake(tree=(0.0, 4), **kw)
    for _ in range(6):
        ga = a.step().cpu().numpy()
        gb = b.step().cpu().numpy()
        assert rel_l2(gb, ga) <= 1e-4
    torch.cuda.synchronize()
    assert a.n == b.n > 0
    assert rel_l2(b.x.cpu().numpy(), a.x.cpu().numpy()) <= 1e-6
    assert rel_l2(b.G.cpu().numpy(), a.G.cpu().numpy()) <= 1e-4


def test_ah1g_with_overlapping_particles_matches_oracle(wake_mod):
    """The AH-1G case with the particle size of the rotor bench (sigma 0.075 R, blade
    segments' core 0.02 R), twelve 10-deg steps: circulations and loads per step,
    particles at the end."""
    from paper_2511_11430_gb300 import synth

    kin = synth.AH1G
    kw = dict(n_blades=2, n_span=12, n_chord=3, max_rows=2, n_tip=3, n_shed=1, kin=kin,
              dt=np.deg2rad(10.0) / kin.omega, sigma=0.075 * kin.radius, seg_core=0.02 * kin.radius)
    g = wake_mod.RotorWake(**kw)
    o = OracleRotorWake(**kw)
    for _ in range(12):
        assert rel_l2(g.step().cpu().numpy(), o.step()) <= 2e-5
    torch.cuda.synchronize()
    assert g.n == len(o.x) > 0
    assert rel_l2(g.x.cpu().numpy().T, o.x) <= 1e-6
    assert rel_l2(g.G.cpu().numpy().T, o.G) <= 2e-5
    hg, ho = np.array(g.history), np.array(o.history)
    np.testing.assert_allclose(hg[:, 1], ho[:, 1], rtol=1e-4, atol=1e-8)
