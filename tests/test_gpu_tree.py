"""The treecode (vpm_tree_induce, the fast summation of Sec. II.B) against the direct
sum as its oracle:

* theta = 0 opens every cluster, so the result is the direct sum: it matches the
  FP64 oracle to the plain-FP32 tolerance, on sizes that leave ragged leaves;
* with clusters accepted, the truncation error falls with the expansion order p as
  (a / L)^(p + 1) for a source cluster of radius a at distance L (a wrong term of the
  derivative recurrence, the moments or their shift breaks this rate), and it falls
  with the opening angle theta;
* on the hover wake and on the million-particle BVI wake the default settings
  (theta = 0.5, p = 4) stay within stated error bounds against the FP64 oracle on
  sampled targets;
* degenerate inputs: one particle, coincident particles, particles on a line.
"""
import numpy as np
import pytest

import oracle
from paper_2511_11430_gb300 import synth
from tests._util import TOL_PLAIN, grad_rows, planar_to_rows, rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# default settings' error bound against the FP64 oracle (relative L2 over sampled targets)
TREE_TOL_U = 1e-3
TREE_TOL_G = 5e-4


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11430_gb300 import api as a
    from paper_2511_11430_gb300 import build

    build.build()
    return a


def _oracle_on(pos, strn, sigma, idx):
    return oracle.p2p(pos, strn, pos[idx], sigma, grad=True)


def _errors(u, g, ref_u, ref_J, idx):
    eu = rel_l2(planar_to_rows(u, 3)[idx], ref_u)
    eg = rel_l2(grad_rows(g)[idx], ref_J)
    return eu, eg


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 129, 3001])
def test_theta_zero_is_the_direct_sum(api, n):
    w = synth.make(1, n=max(n, 2))
    pos, strn = w.pos[:n], w.strength[:n]
    P, S = to_dev(pos), to_dev(strn)
    u, g = api.tree_induce(P, S, w.sigma, theta=0.0, order=4)
    if n == 1:
        assert torch.count_nonzero(u) == 0 and torch.count_nonzero(g) == 0
        return
    ref_u, ref_J = oracle.p2p(pos, strn, pos, w.sigma, grad=True)
    assert rel_l2(planar_to_rows(u, 3), ref_u) <= TOL_PLAIN
    assert rel_l2(grad_rows(g), ref_J) <= TOL_PLAIN
    uv = api.tree_induce(P, S, w.sigma, theta=0.0, order=4, grad=False)
    assert torch.equal(uv, u)


def _two_clusters(a, seed=0, L=1.0):
    """64 zero-strength targets in a ball of radius 1e-3 at the origin, 448 sources in
    a ball of radius a about (L, 0, 0)."""
    rng = np.random.default_rng(seed)

    def ball(m, r):
        v = rng.normal(size=(m, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        return v * (r * rng.uniform(0, 1, size=(m, 1)) ** (1 / 3))

    x = np.concatenate([ball(64, 1e-3), ball(448, a) + [L, 0.0, 0.0]])
    G = np.concatenate([np.zeros((64, 3)), rng.normal(size=(448, 3))])
    pos = np.zeros((512, 4), np.float32)
    pos[:, :3] = x
    strn = np.zeros((512, 4), np.float32)
    strn[:, :3] = G
    return pos, strn


@pytest.mark.parametrize("order, radii", [(2, (0.2, 0.1, 0.05)), (3, (0.3, 0.15, 0.075)), (4, (0.4, 0.2, 0.1))])
def test_truncation_error_falls_at_the_expansion_order(api, order, radii):
    """Halving the source cluster's radius divides the far-field error by about
    2^(p + 1); the direct sum of the same FP32 inputs is the reference.  The radii
    keep the smallest error well above the FP32 floor."""
    sigma = 1e-4
    errs = []
    for a in radii:
        pos, strn = _two_clusters(a)
        P, S = to_dev(pos), to_dev(strn)
        u, g = api.tree_induce(P, S, sigma, theta=1.0, order=order)
        u0, g0 = api.tree_induce(P, S, sigma, theta=0.0, order=order)
        tu, ru = planar_to_rows(u, 3)[:64], planar_to_rows(u0, 3)[:64]
        tg, rg = grad_rows(g)[:64], grad_rows(g0)[:64]
        errs.append((rel_l2(tu, ru), rel_l2(tg, rg)))
    errs = np.array(errs)
    assert np.all(errs[0] > 1e-6), errs  # the expansion is in use
    rate = errs[:-1] / errs[1:]
    # the expected ratio is 2^(p+1) (8, 16, 32); half of it allows for the FP32 floor
    # and the clusters' actual extent
    assert np.all(rate >= 0.5 * 2 ** (order + 1)), (order, errs, rate)


def test_error_falls_with_theta(api):
    rng = np.random.default_rng(5)
    n = 20000
    pos = np.zeros((n, 4), np.float32)
    pos[:, :3] = rng.uniform(-1, 1, size=(n, 3))
    strn = np.zeros((n, 4), np.float32)
    strn[:, :3] = rng.normal(size=(n, 3)) * 1e-3
    sigma = 1e-3
    P, S = to_dev(pos), to_dev(strn)
    idx = np.sort(rng.choice(n, 200, replace=False))
    ref_u, ref_J = _oracle_on(pos, strn, sigma, idx)
    errs = []
    for theta in (1.0, 0.8, 0.6, 0.4):
        u, g = api.tree_induce(P, S, sigma, theta=theta, order=4)
        errs.append(_errors(u, g, ref_u, ref_J, idx))
    errs = np.array(errs)
    # strictly falling while above the plain FP32 floor of a 20,000-term sum (about 2e-6
    # here), then at that floor
    assert np.all(np.diff(errs[:3, 0]) < 0) and np.all(np.diff(errs[:3, 1]) < 0), errs
    assert errs[-1, 0] < 1e-5 and errs[-1, 1] < 1e-5, errs


def test_degenerate_inputs(api):
    # every particle at one point: all pairs at zero distance contribute nothing
    pos = np.zeros((300, 4), np.float32)
    pos[:, :3] = [0.3, -0.2, 0.1]
    strn = np.ones((300, 4), np.float32)
    u, g = api.tree_induce(to_dev(pos), to_dev(strn), 0.01, theta=0.5, order=3)
    assert torch.count_nonzero(u) == 0 and torch.count_nonzero(g) == 0
    # particles on one line (a filament), a size that leaves ragged leaves
    n = 777
    pos = np.zeros((n, 4), np.float32)
    pos[:, 0] = np.linspace(0, 1, n)
    strn = np.zeros((n, 4), np.float32)
    strn[:, 1] = 1e-3
    P, S = to_dev(pos), to_dev(strn)
    u, g = api.tree_induce(P, S, 0.002, theta=0.5, order=4)
    ref_u, ref_J = oracle.p2p(pos, strn, pos, 0.002, grad=True)
    assert rel_l2(planar_to_rows(u, 3), ref_u) <= TREE_TOL_U
    assert rel_l2(grad_rows(g), ref_J) <= TREE_TOL_G


@pytest.mark.parametrize("config", [2, 3])
def test_default_settings_on_rotor_wakes(api, config):
    """Hover (100,000 particles) and BVI (1,000,000) wakes, theta = 0.5, p = 4, against
    the FP64 oracle on 64 sampled targets."""
    w = synth.make(config)
    P, S = to_dev(w.pos), to_dev(w.strength)
    u, g = api.tree_induce(P, S, w.sigma, theta=0.5, order=4)
    idx = synth.sample_targets(11, w.n, 64)
    ref_u, ref_J = _oracle_on(w.pos, w.strength, w.sigma, idx)
    eu, eg = _errors(u, g, ref_u, ref_J, idx)
    assert eu <= TREE_TOL_U and eg <= TREE_TOL_G, (eu, eg)


@pytest.mark.parametrize("classic", [False, True])
def test_rhs_tree_theta_zero_matches_the_oracle(api, classic):
    """The treecode right-hand side with every cluster opened is the direct right-hand
    side: u and grad u of the particles, the segments, Vreman, the stretching (here from
    J^T Gamma of the summed gradient) and PSE over the tree's near pairs."""
    w = synth.make(1)
    rdx, rdG, rnut = oracle.rhs(w.pos, w.strength, w.seg_a, w.seg_b, w.sigma, nu=w.nu, c_v=w.c_v,
                                seg_core=w.seg_core, u_inf=w.u_inf, classic=classic)
    prm = api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core, u_inf=w.u_inf, compensated=False,
                     classic=classic)
    dx, dG, nut = api.rhs_tree(to_dev(w.pos), to_dev(w.strength), to_dev(w.seg_a), to_dev(w.seg_b), prm, theta=0.0)
    torch.cuda.synchronize()
    assert rel_l2(planar_to_rows(dx, 3), rdx) <= TOL_PLAIN
    assert rel_l2(planar_to_rows(dG, 3), rdG) <= TOL_PLAIN
    assert rel_l2(nut.cpu().numpy(), rnut) <= 1e-3


def test_rhs_tree_with_strong_diffusion(api):
    """A viscosity large enough that the PSE term is a large part of dGamma/dt, no
    segments, no eddy viscosity: the tree's PSE walk against the oracle's sum."""
    w = synth.make(1)
    rdx, rdG, rnut = oracle.rhs(w.pos, w.strength, None, None, w.sigma, nu=5e-2, c_v=0.0)
    dx, dG, nut = api.rhs_tree(to_dev(w.pos), to_dev(w.strength), None, None,
                               api.Params(sigma=w.sigma, nu=5e-2, c_v=0.0), theta=0.0)
    torch.cuda.synchronize()
    assert rel_l2(planar_to_rows(dG, 3), rdG) <= TOL_PLAIN


def test_rhs_tree_default_against_the_direct_rhs(api):
    """Hover wake, 100,000 particles: theta = 0.5, order 4 against the direct right-hand
    side of the library (itself within 1e-4 of the oracle)."""
    w = synth.make(2)
    prm = api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core, u_inf=w.u_inf, compensated=False)
    P, S, A, B = to_dev(w.pos), to_dev(w.strength), to_dev(w.seg_a), to_dev(w.seg_b)
    dx0, dG0, nt0 = api.rhs(P, S, A, B, prm)
    dx, dG, nt = api.rhs_tree(P, S, A, B, prm, theta=0.5, order=4)
    torch.cuda.synchronize()
    ex = rel_l2(planar_to_rows(dx, 3), planar_to_rows(dx0, 3))
    eG = rel_l2(planar_to_rows(dG, 3), planar_to_rows(dG0, 3))
    en = rel_l2(nt.cpu().numpy(), nt0.cpu().numpy())
    assert ex <= TREE_TOL_U and eG <= 1e-2 and en <= 1e-2, (ex, eG, en)


def _segment_field(api, w, theta, order, vn=2):
    """dx/dt and nu_t of particles of zero strength: the velocity and (through nu_t)
    the gradient of the blade segments alone, by the treecode and by the direct sweep."""
    strn = np.zeros_like(w.strength)
    prm = api.Params(sigma=w.sigma, nu=0.0, c_v=w.c_v, seg_core=w.seg_core, vatistas_n=vn, compensated=False)
    P, S, A, B = to_dev(w.pos), to_dev(strn), to_dev(w.seg_a), to_dev(w.seg_b)
    dx0, _, nt0 = api.rhs(P, S, A, B, prm)
    dx, _, nt = api.rhs_tree(P, S, A, B, prm, theta=theta, order=order)
    torch.cuda.synchronize()
    ex = rel_l2(planar_to_rows(dx, 3), planar_to_rows(dx0, 3))
    en = rel_l2(nt.cpu().numpy(), nt0.cpu().numpy())
    return ex, en


def test_segment_tree_far_field(api):
    """The segment tree alone (5,120 blade segments onto 30,000 wake particles): theta = 0
    is the direct segment sum; with far nodes accepted the error stays within the
    treecode's bounds and falls with the expansion order (the line-strength moments or
    their quadrature wrong would break this)."""
    w = synth.make(2, n=30000)
    ex0, en0 = _segment_field(api, w, 0.0, 4)
    assert ex0 <= TOL_PLAIN and en0 <= 1e-3, (ex0, en0)
    errs = {p: _segment_field(api, w, 0.5, p) for p in (2, 4)}
    assert errs[4][0] <= TREE_TOL_U and errs[4][1] <= 1e-2, errs
    assert errs[4][0] < errs[2][0], errs


def test_segment_tree_with_zero_length_segments(api):
    """Zero-length segments with a nonzero circulation in the segment tree (in leaves and
    in far nodes) induce nothing, as in the direct sum."""
    w = synth.make(2, n=20000)
    sa, sb = w.seg_a.copy(), w.seg_b.copy()
    sb[::7, :3] = sa[::7, :3]
    strn = np.zeros_like(w.strength)
    prm = api.Params(sigma=w.sigma, nu=0.0, c_v=w.c_v, seg_core=w.seg_core, compensated=False)
    P, S, A, B = to_dev(w.pos), to_dev(strn), to_dev(sa), to_dev(sb)
    dx0, _, _ = api.rhs(P, S, A, B, prm)
    dx, _, nt = api.rhs_tree(P, S, A, B, prm, theta=0.5, order=4)
    torch.cuda.synchronize()
    assert torch.isfinite(dx).all() and torch.isfinite(nt).all()
    assert rel_l2(planar_to_rows(dx, 3), planar_to_rows(dx0, 3)) <= TREE_TOL_U


def test_segment_tree_first_order_vatistas_core(api):
    """With the n = 1 core, which decays slowly (a far node must be about 700 cores
    away), the segment tree still matches the direct sum."""
    w = synth.make(2, n=20000)
    ex, en = _segment_field(api, w, 0.5, 4, vn=1)
    assert ex <= TREE_TOL_U and en <= 1e-2, (ex, en)


def test_step_tree_theta_zero_matches_the_direct_step(api):
    w = synth.make(1)
    prm = api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core, u_inf=w.u_inf, compensated=False)
    x0 = torch.from_numpy(w.pos[:, :3].T.astype(np.float64).copy()).cuda()
    G0 = torch.from_numpy(w.strength[:, :3].T.astype(np.float64).copy()).cuda()
    vol = torch.from_numpy(w.pos[:, 3].copy()).cuda()
    A, B = to_dev(w.seg_a), to_dev(w.seg_b)
    x1, G1 = api.step(x0.clone(), G0.clone(), vol, A, B, prm, w.dt)
    x2, G2 = api.step_tree(x0.clone(), G0.clone(), vol, A, B, prm, w.dt, theta=0.0)
    torch.cuda.synchronize()
    dx_ref = (x1 - x0).cpu().numpy()
    dG_ref = (G1 - G0).cpu().numpy()
    assert rel_l2((x2 - x0).cpu().numpy(), dx_ref) <= TOL_PLAIN
    assert rel_l2((G2 - G0).cpu().numpy(), dG_ref) <= TOL_PLAIN


def test_tree_is_independent_of_the_input_order(api):
    """The Morton sort makes the tree canonical: a permuted particle list gives the same
    u and grad u bit for bit once un-permuted (distinct positions, so no key ties)."""
    w = synth.make(2, n=20000)
    perm = np.random.default_rng(3).permutation(w.n)
    u, g = api.tree_induce(to_dev(w.pos), to_dev(w.strength), w.sigma, theta=0.5, order=4)
    up, gp = api.tree_induce(to_dev(w.pos[perm]), to_dev(w.strength[perm]), w.sigma, theta=0.5, order=4)
    torch.cuda.synchronize()
    inv = np.argsort(perm)
    assert np.array_equal(up.cpu().numpy()[:, inv], u.cpu().numpy())
    assert np.array_equal(gp.cpu().numpy()[:, inv], g.cpu().numpy())


def test_velocity_only_tree_matches_the_gradient_tree(api):
    w = synth.make(2, n=30000)
    P, S = to_dev(w.pos), to_dev(w.strength)
    u, g = api.tree_induce(P, S, w.sigma, theta=0.5, order=4)
    uv = api.tree_induce(P, S, w.sigma, theta=0.5, order=4, grad=False)
    torch.cuda.synchronize()
    assert rel_l2(uv.cpu().numpy(), u.cpu().numpy()) <= 1e-6
