"""GPU parity at the workloads' full sizes, in the launch configuration the benchmark
times, checked on sampled outputs that the FP64 oracle evaluates one by one."""
import numpy as np
import pytest

import oracle
from paper_2511_11430_gb300 import synth
from tests._util import TOL_COMP, TOL_PLAIN, grad_rows, planar_to_rows, rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11430_gb300 import api as a
    from paper_2511_11430_gb300 import build

    build.build()
    return a


def _rows(t, idx, k):
    return t[:, idx].detach().cpu().numpy().T.astype(np.float64).reshape(len(idx), *([3, 3] if k == 9 else [3]))


def _sampled_rhs_reference(w, idx, cut=12.0):
    """Oracle dx/dt and dGamma/dt at particles idx.  Velocity and gradient come from all
    particles and segments; the exchange sum of particle i runs over the particles
    within cut*sigma of it (beyond 12 sigma the Gaussian weight is below 1e-31 of its
    peak), for which nu_t is evaluated from their own full velocity gradients."""
    from scipy.spatial import cKDTree

    P = w.pos[:, :3].astype(np.float64)
    tree = cKDTree(P)
    neigh = sorted(set(j for i in idx for j in tree.query_ball_point(P[i], cut * w.sigma)))
    sub = np.array(neigh)
    u, J = oracle.p2p(w.pos, w.strength, w.pos[sub], w.sigma)
    us, Js = oracle.segments(w.seg_a, w.seg_b, w.pos[sub], w.seg_core, w.vatistas_n)
    J = J + Js
    nut = oracle.vreman(J, w.sigma, w.c_v)
    s = oracle.stretch(J, w.strength[sub])
    p = oracle.pse(w.pos[sub], w.strength[sub], nut, w.sigma, w.nu)
    loc = {j: k for k, j in enumerate(neigh)}
    k = np.array([loc[i] for i in idx])
    dxdt = (u + us + np.array(w.u_inf))[k]
    dGdt = (s + p)[k]
    return dxdt, dGdt


def test_hover_100k_rhs_sampled(api):
    w = synth.make(2)
    prm = api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core, u_inf=w.u_inf, compensated=True)
    dx, dG, nut = api.rhs(to_dev(w.pos), to_dev(w.strength), to_dev(w.seg_a), to_dev(w.seg_b), prm)
    torch.cuda.synchronize()
    idx = synth.sample_targets(2, w.n, 24)
    rdx, rdG = _sampled_rhs_reference(w, idx)
    assert rel_l2(_rows(dx, idx, 3), rdx) <= TOL_COMP
    assert rel_l2(_rows(dG, idx, 3), rdG) <= TOL_COMP


@pytest.mark.parametrize("compensated", [True, False])
def test_hover_100k_induce_sampled(api, compensated):
    w = synth.make(2)
    P = to_dev(w.pos)
    u, g = api.induce(P, to_dev(w.strength), P, w.sigma, compensated=compensated)
    torch.cuda.synchronize()
    idx = synth.sample_targets(2, w.n, 512)
    ru, rJ = oracle.p2p(w.pos, w.strength, w.pos[idx], w.sigma)
    tol = TOL_COMP if compensated else TOL_PLAIN
    assert rel_l2(_rows(u, idx, 3), ru) <= tol
    assert rel_l2(_rows(g, idx, 9), rJ) <= tol


@pytest.mark.parametrize("compensated", [True, False])
def test_bvi_1m_induce_sampled(api, compensated):
    w = synth.make(3)
    P = to_dev(w.pos)
    u, g = api.induce(P, to_dev(w.strength), P, w.sigma, compensated=compensated)
    torch.cuda.synchronize()
    # half random, half on the filaments passing 0.5-2 sigma over the blade
    idx = np.concatenate([synth.sample_targets(3, w.n - 6000, 384), np.arange(w.n - 6000, w.n, 47)])
    ru, rJ = oracle.p2p(w.pos, w.strength, w.pos[idx], w.sigma)
    tol = TOL_COMP if compensated else TOL_PLAIN
    assert rel_l2(_rows(u, idx, 3), ru) <= tol
    assert rel_l2(_rows(g, idx, 9), rJ) <= tol
    # the segments of the blade below those filaments
    us, gs = api.segments_induce(to_dev(w.seg_a), to_dev(w.seg_b), P, w.seg_core, 2, compensated=compensated)
    torch.cuda.synchronize()
    rus, rJs = oracle.segments(w.seg_a, w.seg_b, w.pos[idx], w.seg_core, 2)
    assert rel_l2(_rows(us, idx, 3), rus) <= tol
    assert rel_l2(_rows(gs, idx, 9), rJs) <= tol


def test_multirotor_2m_induce_sampled(api):
    w = synth.make(5)
    P = to_dev(w.pos)
    u, g = api.induce(P, to_dev(w.strength), P, w.sigma, compensated=True)
    torch.cuda.synchronize()
    idx = synth.sample_targets(5, w.n, 256)
    ru, rJ = oracle.p2p(w.pos, w.strength, w.pos[idx], w.sigma)
    assert rel_l2(_rows(u, idx, 3), ru) <= TOL_COMP
    assert rel_l2(_rows(g, idx, 9), rJ) <= TOL_COMP


def test_multirotor_aic_1920_refined_to_1e12(api):
    w = synth.make(5, n=20000)
    u_ind = api.induce(to_dev(w.pos), to_dev(w.strength), to_dev(w.colloc), w.sigma, grad=False)
    A, b = api.aic_build(to_dev(w.rings), to_dev(w.colloc), to_dev(w.normal), w.seg_core, 2, v_rel=to_dev(w.v_rel),
                         w_ind=u_ind)
    x, it, be = api.aic_solve(A, b, tol=1e-12, max_iter=30)
    assert A.shape == (1920, 1920)
    assert be <= 1e-12
    Ah = A.cpu().numpy().astype(np.float64)
    bh = b.cpu().numpy()
    r = bh - Ah @ x.cpu().numpy()
    assert np.abs(r).max() / (np.abs(Ah).sum(axis=1).max() * np.abs(x.cpu().numpy()).max() + np.abs(bh).max()) <= 1e-12


def test_adjoint_200k_sampled(api):
    w = synth.make(4)
    rng = np.random.default_rng(4)
    nrm = w.normal[:, :3].astype(np.float64)
    P = to_dev(w.pos)
    S = to_dev(w.strength)
    C = to_dev(w.colloc)
    u = api.induce(P, S, C, w.sigma, grad=False)
    un = (u.double().cpu().numpy().T * nrm).sum(axis=1)
    g = (2 * un[:, None] * nrm).astype(np.float32)  # gradient of sum_k (u_k . n_k)^2
    dx, dG = api.induce_backward(P, S, C, w.sigma, to_dev(np.ascontiguousarray(g.T)))
    torch.cuda.synchronize()
    idx = synth.sample_targets(4, w.n, 4096)
    rx, rG = oracle.p2p_adjoint(w.pos[idx], w.strength[idx], w.colloc, w.sigma, g.astype(np.float64))
    assert rel_l2(_rows(dx, idx, 3), rx) <= 1e-5
    assert rel_l2(_rows(dG, idx, 3), rG) <= 1e-5
    del rng
