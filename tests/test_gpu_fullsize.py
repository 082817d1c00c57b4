"""GPU parity at the workloads' full sizes, in the launch configuration the benchmark
times, checked on sampled outputs that the FP64 oracle evaluates one by one."""
import numpy as np
import pytest

import oracle
from oracle import sampled
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


@pytest.mark.parametrize("compensated", [True, False])
def test_multirotor_2m_induce_sampled(api, compensated):
    w = synth.make(5)
    P = to_dev(w.pos)
    u, g = api.induce(P, to_dev(w.strength), P, w.sigma, compensated=compensated)
    torch.cuda.synchronize()
    idx = synth.sample_targets(5, w.n, 256)
    ru, rJ = oracle.p2p(w.pos, w.strength, w.pos[idx], w.sigma)
    tol = TOL_COMP if compensated else TOL_PLAIN
    assert rel_l2(_rows(u, idx, 3), ru) <= tol
    assert rel_l2(_rows(g, idx, 9), rJ) <= tol


def _rhs_both_forms(api, w, c_v=None):
    out = {}
    P, S, A, B = to_dev(w.pos), to_dev(w.strength), to_dev(w.seg_a), to_dev(w.seg_b)
    for comp in (True, False):
        prm = api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v if c_v is None else c_v, seg_core=w.seg_core,
                         u_inf=w.u_inf, compensated=comp)
        dx, dG, nut = api.rhs(P, S, A, B, prm)
        torch.cuda.synchronize()
        out[comp] = (dx, dG, nut)
    return out


def test_bvi_1m_rhs_sampled():
    """The right-hand side of Eq. 4-5 on the 1M forward-flight wake at 128 particles in
    runs of 16: four runs on the skewed helices, four on the straight filaments that
    pass 0.5, 1 and 2 sigma over blade 0's panels (stretching and exchange near the
    blade's segments)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11430_gb300 import api, build

    build.build()
    w = synth.make(3)
    n_hel = w.n - 6000
    fil = [n_hel + 2000 * f + 16 * q for f, q in ((0, 40), (0, 90), (1, 60), (2, 75))]  # 0.5, 0.5, 1, 2 sigma
    idx = np.sort(np.concatenate([synth.sample_runs(3, n_hel, 4, 16), *[np.arange(s, s + 16) for s in fil]]))
    rdx, rdG, rnut = sampled.rhs_at(w, idx)
    res = _rhs_both_forms(api, w)
    for comp, tol, tol_nu in ((True, TOL_COMP, 1e-5), (False, TOL_PLAIN, 1e-3)):
        dx, dG, nut = res[comp]
        assert rel_l2(_rows(dx, idx, 3), rdx) <= tol
        assert rel_l2(_rows(dG, idx, 3), rdG) <= tol
        assert rel_l2(nut[idx].double().cpu().numpy(), rnut) <= tol_nu


def test_multirotor_2m_rhs_sampled():
    """The right-hand side on the 2M two-rotor wake: dx/dt, nu_t and dGamma/dt without the
    eddy-viscosity exchange (c_V = 0: stretching + exchange at nu) at 128 random
    particles, and the full dGamma/dt (Vreman coupling in the exchange) at 32 particles
    in two runs of 16 (each of which needs the gradients of its ~2,000 neighbours)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11430_gb300 import api, build

    build.build()
    w = synth.make(5)
    idx = synth.sample_targets(55, w.n, 128)
    rdx, rdG0, rnut = sampled.rhs_at(w, idx, c_v=0.0)
    rnut = oracle.vreman(oracle.p2p(w.pos, w.strength, w.pos[idx], w.sigma)[1]
                         + oracle.segments(w.seg_a, w.seg_b, w.pos[idx], w.seg_core, w.vatistas_n)[1], w.sigma, w.c_v)
    idx_r = synth.sample_runs(56, w.n, 2, 16)
    _, rdG, _ = sampled.rhs_at(w, idx_r)
    full = _rhs_both_forms(api, w)
    cv0 = _rhs_both_forms(api, w, c_v=0.0)
    for comp, tol, tol_nu in ((True, TOL_COMP, 1e-5), (False, TOL_PLAIN, 1e-3)):
        dx, dG, nut = full[comp]
        assert rel_l2(_rows(dx, idx, 3), rdx) <= tol
        assert rel_l2(nut[idx].double().cpu().numpy(), rnut) <= tol_nu
        assert rel_l2(_rows(dG, idx_r, 3), rdG) <= tol
        assert rel_l2(_rows(cv0[comp][1], idx, 3), rdG0) <= tol


def test_hover_100k_first_stage_sampled():
    """One RK3 stage (k = 0) of the 100k hover wake through vpm_rk3_stage: the FP64
    increments of x and Gamma at sampled particles are dt/3 times the oracle's
    right-hand side there (the state is FP32-exact, so the stage reads it unrounded)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11430_gb300 import api, build

    build.build()
    w = synth.make(2)
    x0 = np.ascontiguousarray(w.pos[:, :3].astype(np.float64).T)
    G0 = np.ascontiguousarray(w.strength[:, :3].astype(np.float64).T)
    x, G = to_dev(x0), to_dev(G0)
    q = torch.full((6, w.n), float("nan"), dtype=torch.float64, device="cuda")  # stage 0 must not read q
    prm = api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core, u_inf=w.u_inf, compensated=True)
    api.rk3_stage(0, x, G, q, to_dev(w.pos[:, 3].copy()), to_dev(w.seg_a), to_dev(w.seg_b), prm, w.dt)
    torch.cuda.synchronize()
    idx = synth.sample_runs(21, w.n, 3, 16)
    rdx, rdG, _ = sampled.rhs_at(w, idx)
    dx = (x.cpu().numpy() - x0)[:, idx].T
    dG = (G.cpu().numpy() - G0)[:, idx].T
    assert rel_l2(dx, w.dt / 3.0 * rdx) <= TOL_COMP
    assert rel_l2(dG, w.dt / 3.0 * rdG) <= TOL_COMP
    assert rel_l2(q[:3, idx].cpu().numpy().T, w.dt * rdx) <= TOL_COMP
    assert rel_l2(q[3:, idx].cpu().numpy().T, w.dt * rdG) <= TOL_COMP


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
