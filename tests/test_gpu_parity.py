"""GPU parity: every entry point of libvpm against the FP64 oracle on identical
seeded FP32 inputs.  Relative L2 per output: compensated FP32 <= 2e-6, plain FP32
<= 1e-4 (the stated error budget); integer-valued properties bit-exact."""
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


def _check(api_u, api_g, ref_u, ref_J, tol, tag=""):
    eu = rel_l2(planar_to_rows(api_u, 3), ref_u)
    assert eu <= tol, f"{tag} u rel-L2 {eu:.3e} > {tol}"
    if api_g is not None:
        eg = rel_l2(grad_rows(api_g), ref_J)
        assert eg <= tol, f"{tag} grad rel-L2 {eg:.3e} > {tol}"
        return eu, eg
    return eu, None


@pytest.mark.parametrize("compensated", [True, False])
@pytest.mark.parametrize("n", [1, 37, 2000, 3001])
def test_induce_self_config1(api, n, compensated):
    """Targets = sources (self-exclusion), 2-blade hover wake; sizes span several tiles and a ragged tail."""
    w = synth.make(1, n=max(n, 2))
    pos, G = w.pos[:n], w.strength[:n]
    ru, rJ = oracle.p2p(pos, G, pos, w.sigma)
    u, g = api.induce(to_dev(pos), to_dev(G), to_dev(pos), w.sigma, compensated=compensated)
    torch.cuda.synchronize()
    if n == 1:
        assert np.all(u.cpu().numpy() == 0) and np.all(g.cpu().numpy() == 0)
        return
    _check(u, g, ru, rJ, TOL_COMP if compensated else TOL_PLAIN, f"n={n}")


@pytest.mark.parametrize("compensated", [True, False])
def test_induce_random_cloud_other_targets_velocity_only(api, compensated):
    pos, G = synth.random_cloud(5, 4099, sigma=0.05)
    tgt, _ = synth.random_cloud(6, 777, sigma=0.05)
    ru = oracle.p2p(pos, G, tgt, 0.05, grad=False)
    u = api.induce(to_dev(pos), to_dev(G), to_dev(tgt), 0.05, compensated=compensated, grad=False)
    torch.cuda.synchronize()
    _check(u, None, ru, None, TOL_COMP if compensated else TOL_PLAIN)


def test_induce_coincident_and_empty(api):
    pos = np.array([[0.1, 0.2, 0.3, 1e-3], [0.1, 0.2, 0.3, 1e-3], [0.4, 0.2, 0.3, 1e-3]], dtype=np.float32)
    G = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], dtype=np.float32)
    ru, rJ = oracle.p2p(pos, G, pos, 0.1)
    u, g = api.induce(to_dev(pos), to_dev(G), to_dev(pos), 0.1)
    torch.cuda.synchronize()
    _check(u, g, ru, rJ, TOL_COMP)
    u0, g0 = api.induce(to_dev(pos[:0]), to_dev(G[:0]), to_dev(pos), 0.1)
    torch.cuda.synchronize()
    assert np.all(u0.cpu().numpy() == 0) and np.all(g0.cpu().numpy() == 0)


@pytest.mark.parametrize("vn", [1, 2])
@pytest.mark.parametrize("compensated", [True, False])
def test_segments_config1(api, vn, compensated):
    w = synth.make(1)
    ru, rJ = oracle.segments(w.seg_a, w.seg_b, w.pos, w.seg_core, vn)
    u, g = api.segments_induce(to_dev(w.seg_a), to_dev(w.seg_b), to_dev(w.pos), w.seg_core, vn,
                               compensated=compensated)
    torch.cuda.synchronize()
    _check(u, g, ru, rJ, TOL_COMP if compensated else TOL_PLAIN, f"vn={vn}")


def test_segments_random_ragged_and_near(api):
    sa, sb = synth.random_segments(3, 301, length=0.2)
    tgt, _ = synth.random_cloud(4, 1029, sigma=0.05)
    # a few targets right next to segments (inside the core)
    tgt[:50, :3] = (0.5 * (sa[:50, :3] + sb[:50, :3]) + 1e-3).astype(np.float32)
    ru, rJ = oracle.segments(sa, sb, tgt, 0.02, 2)
    u, g = api.segments_induce(to_dev(sa), to_dev(sb), to_dev(tgt), 0.02, 2)
    torch.cuda.synchronize()
    _check(u, g, ru, rJ, TOL_COMP)


def test_segments_of_zero_length(api):
    """Zero-length segments (b = a) with a nonzero circulation induce nothing (the
    oracle's L = 0 case): mixed into tiles of ordinary segments, whose far targets take
    the guard-free path, and as a whole tile of them with targets exactly on their
    points."""
    sa, sb = synth.random_segments(5, 256, length=0.2)  # two full 128-segment tiles
    sb[10:30, :3] = sa[10:30, :3]  # 20 zero-length segments among the first tile
    pts = np.repeat(sa[:1, :3], 128, axis=0) + np.linspace(0.0, 0.1, 128, dtype=np.float32)[:, None]
    za = np.concatenate([pts, np.full((128, 1), 0.7, np.float32)], axis=1).astype(np.float32)
    sa = np.concatenate([sa, za]).astype(np.float32)  # a whole tile of zero-length segments
    sb = np.concatenate([sb, za]).astype(np.float32)
    tgt, _ = synth.random_cloud(6, 1000, sigma=0.05)
    tgt[:5, :3] = za[:5, :3]  # targets on the points of zero-length segments
    tgt[5:10, :3] = sa[10:15, :3]
    for core in (0.02, 0.0):
        ru, rJ = oracle.segments(sa, sb, tgt, core, 2)
        u, g = api.segments_induce(to_dev(sa), to_dev(sb), to_dev(tgt), core, 2)
        torch.cuda.synchronize()
        assert torch.isfinite(u).all() and torch.isfinite(g).all()
        _check(u, g, ru, rJ, TOL_COMP)


@pytest.mark.parametrize("vn", [1, 2])
def test_segments_closed_rings(api, vn):
    """Segment tiles made of closed four-sided rings are packed by corner (each corner
    shared by two sides).  They must match the oracle for targets far away, inside the
    core, on the sides, a few core radii from corners and exactly on corners (the
    end-point guard), including a ring with a zero-length side; and match the same
    segments taken one by one, which the library sees when the sides of every ring are
    listed in reverse order (the tile is then not a chain of closed rings).  (Targets
    much closer to a corner than the core radius lose the gradient to FP32 rounding in
    either form, 2e-4 at 1e-5 of 0.05-long sides, and are left out.)"""
    core = 0.02
    sa, sb = synth.random_rings(7, 50, box=0.6, size=0.12)  # 200 segments: 128 + 72, both tiles closed
    sb[20, :3] = sa[20, :3]  # ring 5, side 0 of zero length: corners 0 and 1 coincide
    sa[21, :3] = sa[20, :3]
    tgt, _ = synth.random_cloud(8, 1100, sigma=0.05)
    tgt[:8, :3] = sa[:8, :3]  # on corners
    tgt[8:16, :3] = 0.5 * (sa[8:16, :3] + sb[8:16, :3])  # mid-side
    tgt[16:24, :3] = sa[16:24, :3] + np.float32(2e-3)  # a few core radii from corners
    tgt[24:40, :3] = 0.3 * sa[24:40, :3] + 0.7 * sb[24:40, :3] + np.float32(3e-3)  # inside the core
    tgt[576:, 0] += np.float32(1.5)  # whole warps of targets clear of every tile: the guard-free form
    ru, rJ = oracle.segments(sa, sb, tgt, core, vn)
    u, g = api.segments_induce(to_dev(sa), to_dev(sb), to_dev(tgt), core, vn)
    torch.cuda.synchronize()
    assert torch.isfinite(u).all() and torch.isfinite(g).all()
    _check(u, g, ru, rJ, TOL_COMP, f"vn={vn}")
    rev = np.concatenate([np.arange(4 * r + 3, 4 * r - 1, -1) for r in range(50)])
    u2, g2 = api.segments_induce(to_dev(sa[rev]), to_dev(sb[rev]), to_dev(tgt), core, vn)
    torch.cuda.synchronize()
    for x, y in ((u, u2), (g, g2)):
        x, y = x.double().cpu().numpy(), y.double().cpu().numpy()
        assert np.linalg.norm(x - y) <= TOL_COMP * np.linalg.norm(y)


@pytest.mark.parametrize("classic", [False, True])
@pytest.mark.parametrize("compensated", [True, False])
def test_rhs_config1(api, classic, compensated):
    w = synth.make(1)
    rdx, rdG, rnut = oracle.rhs(w.pos, w.strength, w.seg_a, w.seg_b, w.sigma, nu=w.nu, c_v=w.c_v,
                                seg_core=w.seg_core, u_inf=w.u_inf, classic=classic)
    prm = api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core, u_inf=w.u_inf, compensated=compensated,
                     classic=classic)
    dx, dG, nut = api.rhs(to_dev(w.pos), to_dev(w.strength), to_dev(w.seg_a), to_dev(w.seg_b), prm)
    torch.cuda.synchronize()
    tol = TOL_COMP if compensated else TOL_PLAIN
    assert rel_l2(planar_to_rows(dx, 3), rdx) <= tol
    assert rel_l2(planar_to_rows(dG, 3), rdG) <= tol
    assert rel_l2(nut.cpu().numpy(), rnut) <= (1e-5 if compensated else 1e-3)


def test_rhs_conserves_total_vorticity_without_segments(api):
    """Transposed stretching + PSE cancel pairwise: sum_i dGamma_i/dt ~ 0 (up to FP32 rounding)."""
    w = synth.make(1)
    prm = api.Params(sigma=w.sigma, nu=1e-3, c_v=w.c_v)
    dx, dG, nut = api.rhs(to_dev(w.pos), to_dev(w.strength), None, None, prm)
    torch.cuda.synchronize()
    d = dG.double().cpu().numpy()
    assert np.abs(d.sum(axis=1)).max() <= 1e-5 * np.abs(d).sum(axis=1).max()


def test_step_config1(api):
    w = synth.make(1)
    x0 = w.pos[:, :3].astype(np.float64)
    G0 = w.strength[:, :3].astype(np.float64)
    vol = w.pos[:, 3].copy()
    dt = w.dt * 20  # a larger step makes the increment well above rounding
    rx, rG = oracle.step(x0, G0, vol, w.seg_a, w.seg_b, w.sigma, dt, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core,
                         u_inf=w.u_inf, cast_f32=True)
    X = to_dev(np.ascontiguousarray(x0.T))
    Gd = to_dev(np.ascontiguousarray(G0.T))
    prm = api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core, u_inf=w.u_inf, compensated=True)
    api.step(X, Gd, to_dev(vol), to_dev(w.seg_a), to_dev(w.seg_b), prm, dt)
    torch.cuda.synchronize()
    gx = X.cpu().numpy().T
    gG = Gd.cpu().numpy().T
    # compare the increments (the state itself is dominated by its unchanged part)
    assert rel_l2(gx - x0, rx - x0) <= 1e-5
    assert rel_l2(gG - G0, rG - G0) <= 1e-5


def test_rk3_stages_equal_one_step(api):
    """Three vpm_rk3_stage calls (k = 0, 1, 2, the register kept by the caller) give
    vpm_step's state bit for bit, and the staged step matches the oracle's step."""
    w = synth.make(1)
    x0 = np.ascontiguousarray(w.pos[:, :3].astype(np.float64).T)
    G0 = np.ascontiguousarray(w.strength[:, :3].astype(np.float64).T)
    vol, sa, sb = to_dev(w.pos[:, 3].copy()), to_dev(w.seg_a), to_dev(w.seg_b)
    dt = w.dt * 20
    prm = api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core, u_inf=w.u_inf, compensated=True)
    X1, G1 = to_dev(x0), to_dev(G0)
    api.step(X1, G1, vol, sa, sb, prm, dt)
    X2, G2 = to_dev(x0), to_dev(G0)
    q = torch.full((6, w.n), float("nan"), dtype=torch.float64, device="cuda")
    for k in range(3):
        api.rk3_stage(k, X2, G2, q, vol, sa, sb, prm, dt)
    torch.cuda.synchronize()
    assert torch.equal(X1, X2) and torch.equal(G1, G2)
    rx, rG = oracle.step(x0.T, G0.T, w.pos[:, 3].copy(), w.seg_a, w.seg_b, w.sigma, dt, nu=w.nu, c_v=w.c_v,
                         seg_core=w.seg_core, u_inf=w.u_inf, cast_f32=True)
    assert rel_l2(X2.cpu().numpy().T - x0.T, rx - x0.T) <= 1e-5
    assert rel_l2(G2.cpu().numpy().T - G0.T, rG - G0.T) <= 1e-5


def test_rk3_stage_rejects_bad_stage(api):
    from paper_2511_11430_gb300 import _lib

    x = torch.zeros((3, 4), dtype=torch.float64, device="cuda")
    q = torch.zeros((6, 4), dtype=torch.float64, device="cuda")
    vol = torch.ones(4, dtype=torch.float32, device="cuda")
    with pytest.raises(_lib.VpmError) as ei:
        api.rk3_stage(3, x, x.clone(), q, vol, None, None, api.Params(sigma=0.1), 1e-3)
    assert ei.value.status == _lib.VPM_ERR_INVALID_ARG


def test_aic_build_and_solve(api):
    w = synth.make(1)
    A_ref = oracle.aic_build(w.rings, w.colloc, w.normal, w.seg_core)
    u_ind = oracle.p2p(w.pos, w.strength, w.colloc, w.sigma, grad=False)
    b_ref = oracle.aic_rhs(w.v_rel, u_ind, w.normal)
    A, b = api.aic_build(to_dev(w.rings), to_dev(w.colloc), to_dev(w.normal), w.seg_core, 2, v_rel=to_dev(w.v_rel),
                         w_ind=to_dev(np.ascontiguousarray(u_ind.T.astype(np.float32))))
    torch.cuda.synchronize()
    assert rel_l2(A.cpu().numpy(), A_ref) <= 1e-5
    np.testing.assert_allclose(b.cpu().numpy(), b_ref, rtol=1e-6, atol=1e-6 * np.abs(b_ref).max())
    x, it, be = api.aic_solve(A, b, tol=1e-12, max_iter=30)
    assert be <= 1e-12
    # the FP64 solution of the FP32-stored system
    xr = oracle.lu_solve(A.cpu().numpy().astype(np.float64), b.cpu().numpy())
    assert rel_l2(x.cpu().numpy(), xr) <= 1e-9


def test_aic_solve_large_random_and_not_converged(api):
    rng = np.random.default_rng(1)
    n = 1283  # ragged with respect to the 32-column panels
    A = (rng.normal(size=(n, n)) + n ** 0.5 * np.eye(n)).astype(np.float32)
    b = rng.normal(size=n)
    x, it, be = api.aic_solve(to_dev(A), to_dev(b), tol=1e-13, max_iter=30)
    assert be <= 1e-13
    xr = np.linalg.solve(A.astype(np.float64), b)
    assert rel_l2(x.cpu().numpy(), xr) <= 1e-10
    with pytest.raises(Exception):
        api.aic_solve(to_dev(A), to_dev(b), tol=0.0, max_iter=1)
    Z = np.zeros((4, 4), dtype=np.float32)
    with pytest.raises(Exception):
        api.aic_solve(to_dev(Z), to_dev(np.ones(4)), tol=1e-12)


@pytest.mark.parametrize("n,kind", [(1, "gauss"), (31, "gauss"), (33, "perm"), (100, "gauss"), (257, "perm"),
                                    (1500, "gauss")])
def test_aic_solve_needs_pivoting(api, n, kind):
    """General matrices whose factorisation needs row exchanges: Gaussian entries, or a
    row-permuted near-identity (zero diagonal entries, so elimination without exchanges
    fails).  n = 1500 factors its first panels with the panel held in global memory."""
    rng = np.random.default_rng(n)
    if kind == "gauss":
        A = rng.normal(size=(n, n)).astype(np.float32)
    else:
        A = (rng.permutation(np.eye(n)) @ (np.eye(n) + 0.3 * rng.normal(size=(n, n)) / n ** 0.5)).astype(np.float32)
    b = rng.normal(size=n)
    x, it, be = api.aic_solve(to_dev(A), to_dev(b), tol=1e-12, max_iter=30)
    assert be <= 1e-12
    A64 = A.astype(np.float64)
    xr = np.linalg.solve(A64, b)
    cond = np.linalg.cond(A64)
    assert rel_l2(x.cpu().numpy(), xr) <= max(1e-10, 10 * cond * 1e-12)


@pytest.mark.parametrize("n", [1, 31, 33, 100, 257, 1280])
@pytest.mark.parametrize("dominant", [True, False])
def test_aic_solve_row_dominant_and_not(api, n, dominant):
    """A strictly row-dominant matrix is factored without row exchanges, any other with
    partial pivoting; both are refined to the FP64 solution of the FP32 matrix.  The
    non-dominant case is the dominant matrix with one row's diagonal made small."""
    rng = np.random.default_rng(1000 + n)
    A = rng.uniform(-1.0, 1.0, (n, n))
    A[np.arange(n), np.arange(n)] = (np.abs(A).sum(axis=1) + 0.05) * np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    if not dominant and n > 1:
        A[n // 2, n // 2] = 0.25
    A = A.astype(np.float32)
    b = rng.normal(size=n)
    x, it, be = api.aic_solve(to_dev(A), to_dev(b), tol=1e-12, max_iter=30)
    assert be <= 1e-12
    ref = oracle.lu_solve(A.astype(np.float64), b)
    np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_aic_solve_not_converged_returns_best_iterate(api):
    """With an unreachable tolerance the solve stops after max_iter corrections and
    returns the iterate of smallest backward error, whose error it reports."""
    rng = np.random.default_rng(5)
    n = 300
    A = rng.normal(size=(n, n)).astype(np.float32)
    b = rng.normal(size=n)
    x, it, be = api.aic_solve(to_dev(A), to_dev(b), tol=0.0, max_iter=3, raise_on_fail=False)
    assert it == 3
    xh = x.cpu().numpy()
    A64 = A.astype(np.float64)
    r = b - A64 @ xh
    berr = np.abs(r).max() / (np.abs(A64).sum(1).max() * np.abs(xh).max() + np.abs(b).max())
    # both errors sit at the rounding level of the FP64 residual, so compare their size only
    assert be < 1e-13 and berr < 1e-13


def test_aic_solve_zero_column_is_reported(api):
    rng = np.random.default_rng(3)
    A = rng.normal(size=(100, 100)).astype(np.float32)
    A[:, 40] = 0.0  # singular: the elimination meets an all-zero column at index 40
    with pytest.raises(Exception, match="singular"):
        api.aic_solve(to_dev(A), to_dev(rng.normal(size=100)), tol=1e-12)


@pytest.mark.parametrize("compensated", [True, False])
def test_backward_vs_oracle_adjoint(api, compensated):
    w = synth.make(4, n=5000)
    rng = np.random.default_rng(0)
    g = rng.normal(size=(w.n_ctrl, 3)).astype(np.float32)
    rx, rG = oracle.p2p_adjoint(w.pos, w.strength, w.colloc, w.sigma, g.astype(np.float64))
    dx, dG = api.induce_backward(to_dev(w.pos), to_dev(w.strength), to_dev(w.colloc), w.sigma,
                                 to_dev(np.ascontiguousarray(g.T)), compensated=compensated)
    torch.cuda.synchronize()
    tol = 1e-5 if compensated else 1e-3
    assert rel_l2(planar_to_rows(dx, 3), rx) <= tol
    assert rel_l2(planar_to_rows(dG, 3), rG) <= tol


def test_backward_near_field_targets(api):
    pos, G = synth.random_cloud(8, 1500, sigma=0.05, box=0.5)
    tgt = pos[:300].copy()
    tgt[:, :3] += np.float32(0.01)  # evaluation points inside the cores
    g = np.random.default_rng(2).normal(size=(300, 3)).astype(np.float32)
    rx, rG = oracle.p2p_adjoint(pos, G, tgt, 0.05, g.astype(np.float64))
    dx, dG = api.induce_backward(to_dev(pos), to_dev(G), to_dev(tgt), 0.05, to_dev(np.ascontiguousarray(g.T)))
    torch.cuda.synchronize()
    assert rel_l2(planar_to_rows(dx, 3), rx) <= 1e-5
    assert rel_l2(planar_to_rows(dG, 3), rG) <= 1e-5


def test_device_error_word_clean(api):
    assert api.device_error() == 0


@pytest.mark.parametrize("compensated", [True, False])
def test_rhs_shuffled_particle_order(api, compensated):
    """Results do not depend on the order of the particles (tile boxes, warp box
    splits and the near/far choice only change cost, never values)."""
    w = synth.make(1)
    perm = np.random.default_rng(5).permutation(w.n)
    pos, G = w.pos[perm], w.strength[perm]
    rdx, rdG, rnut = oracle.rhs(pos, G, w.seg_a, w.seg_b, w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core,
                                u_inf=w.u_inf)
    prm = api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core, u_inf=w.u_inf, compensated=compensated)
    dx, dG, nut = api.rhs(to_dev(pos), to_dev(G), to_dev(w.seg_a), to_dev(w.seg_b), prm)
    torch.cuda.synchronize()
    tol = TOL_COMP if compensated else TOL_PLAIN
    assert rel_l2(planar_to_rows(dx, 3), rdx) <= tol
    assert rel_l2(planar_to_rows(dG, 3), rdG) <= tol
