"""Pins of the oracle's time step (low-storage RK3, Sec. II.B), its LU solve and AIC
(Sec. II.A) and its adjoint of the particle -> point velocity."""
import numpy as np
import pytest

import oracle


def _poly3(M):
    I = np.eye(3)
    return I + M + M @ M / 2 + M @ M @ M / 6


def test_rk3_linear_stage_polynomial():
    """One particle held still (U_inf cancels the segments' velocity) sees a frozen velocity
    gradient J, so Eq. 5 is the linear ODE Gamma' = J^T Gamma and one third-order step must
    be the cubic Taylor polynomial of exp(dt J^T) exactly (Williamson's scheme)."""
    rng = np.random.default_rng(0)
    sa = np.array([[-1.0, 0.1, 0.2, 1.5], [0.3, -1.0, -0.1, -0.7], [0.2, 0.3, -1.0, 0.9]])
    sb = np.array([[1.0, -0.2, 0.1, 0.0], [-0.2, 1.0, 0.2, 0.0], [-0.1, 0.1, 1.0, 0.0]])
    x0 = np.array([[0.05, -0.03, 0.02]])
    u, J = oracle.segments(sa, sb, np.c_[x0, 0], 0.1, 2)
    G0 = rng.normal(size=(1, 3))
    dt = 0.05
    x1, G1 = oracle.step(x0, G0, np.array([1e-3]), sa, sb, sigma=0.05, dt=dt, seg_core=0.1, u_inf=-u[0],
                         cast_f32=False)
    np.testing.assert_array_equal(x1, x0)
    A = J[0].T
    np.testing.assert_allclose(G1[0], _poly3(dt * A) @ G0[0], rtol=1e-13)
    # and it is not the second-order polynomial (the third-order term matters here)
    I = np.eye(3)
    assert np.linalg.norm(G1[0] - (I + dt * A + (dt * A) @ (dt * A) / 2) @ G0[0]) > 1e-6 * np.linalg.norm(G0)


def _wavy_ring(n=120, R0=0.2, amp=0.03, gamma=2e-3):
    th = 2 * np.pi * (np.arange(n) + 0.5) / n
    r = R0 + amp * np.cos(3 * th)
    x = np.c_[r * np.cos(th), r * np.sin(th), 0.01 * np.sin(2 * th)]
    t = np.roll(x, -1, axis=0) - np.roll(x, 1, axis=0)
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    return x, gamma * t


def test_rk3_observed_temporal_order_is_three():
    """Step-halving on a perturbed vortex ring (the paper fits p = 2.83 for C_T, Eq. 11;
    the integrator alone must show order 3)."""
    x0, G0 = _wavy_ring()
    vol = np.full(len(x0), 0.02 ** 3)
    sigma = 0.03
    T = 0.2

    def run(nsteps):
        x, G = x0.copy(), G0.copy()
        for _ in range(nsteps):
            x, G = oracle.step(x, G, vol, None, None, sigma=sigma, dt=T / nsteps, nu=1e-4, cast_f32=False)
        return np.r_[x.ravel(), 1e2 * G.ravel()]

    ref = run(128)
    e = [np.linalg.norm(run(k) - ref) for k in (4, 8, 16)]
    p1, p2 = np.log2(e[0] / e[1]), np.log2(e[1] / e[2])
    assert 2.8 < p1 < 3.2 and 2.8 < p2 < 3.2, (e, p1, p2)


def test_lu_manufactured_solution_and_pivoting():
    rng = np.random.default_rng(3)
    n = 60
    A = rng.normal(size=(n, n))
    xt = rng.normal(size=n)
    b = A @ xt
    x = oracle.lu_solve(A, b)
    np.testing.assert_allclose(x, xt, rtol=0, atol=1e-11 * np.abs(xt).max())
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-11 * np.abs(xt).max())
    P = np.array([[0.0, 2.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 3.0]])  # needs row exchange
    np.testing.assert_allclose(oracle.lu_solve(P, [2.0, 1.0, 3.0]), [1.0, 1.0, 1.0], rtol=1e-15)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.lu_solve(np.zeros((2, 2)), [1.0, 1.0])


def _long_rings(n_chord, chord=1.0, far=1e4):
    """Flat-plate chordwise strip of rings on z = 0, flow along +x; the last ring's trailing
    segment is taken far downstream (steady wake) and the side segments far out."""
    dx = chord / n_chord
    rings, col = [], []
    for j in range(n_chord):
        x0 = j * dx + 0.25 * dx
        x1 = (j + 1) * dx + 0.25 * dx if j < n_chord - 1 else far
        rings.append([[x0, -far, 0], [x1, -far, 0], [x1, far, 0], [x0, far, 0]])
        col.append([j * dx + 0.75 * dx, 0.0, 0.0])
    return np.array(rings), np.array(col)


@pytest.mark.parametrize("n_chord", [1, 2, 4])
def test_aic_reproduces_thin_airfoil_lift(n_chord):
    """Vortex rings at the quarter chord of each panel and collocation at three quarters
    (Sec. II.A) give, for a 2-D flat plate, the thin-airfoil circulation pi c U sin(alpha)."""
    rings, col = _long_rings(n_chord)
    nrm = np.tile([0.0, 0.0, 1.0], (n_chord, 1))
    A = oracle.aic_build(rings, col, nrm, core=1e-9)
    U, alpha = 10.0, np.deg2rad(4.0)
    vrel = np.tile([U * np.cos(alpha), 0.0, U * np.sin(alpha)], (n_chord, 1))
    b = oracle.aic_rhs(vrel, None, nrm)
    G = oracle.lu_solve(A, b)
    total = G[-1]  # bound circulation of the last ring is the strip's total
    assert abs(total) == pytest.approx(np.pi * 1.0 * U * np.sin(alpha), rel=2e-4)


def test_aic_entry_is_ring_velocity_dot_normal():
    rng = np.random.default_rng(9)
    rings = rng.normal(size=(3, 4, 3))
    col = rng.normal(size=(3, 3))
    nrm = rng.normal(size=(3, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    A = oracle.aic_build(rings, col, nrm, core=0.01)
    for k in range(3):
        for l in range(3):
            c = rings[l]
            sa = np.c_[c, np.ones(4)]
            sb = np.c_[np.roll(c, -1, axis=0), np.zeros(4)]
            u = oracle.segments(sa, sb, np.r_[col[k], 0][None], 0.01, 2, grad=False)[0]
            assert A[k, l] == pytest.approx(u @ nrm[k], rel=1e-13, abs=1e-15)


def test_adjoint_matches_incremental_central_differences():
    """dL/dx_j and dL/dGamma_j of L = sum_k (u_k . n_k)^2 against central differences with
    h = 1e-6 (length unit R = 1), formed incrementally: moving particle j changes only its own
    contribution c_k, and L(+) - L(-) = sum_k (c+ - c-)(2 b_k + c+ + c-) with b_k the rest."""
    rng = np.random.default_rng(12)
    ns, nt, sigma = 150, 40, 0.05
    P = rng.uniform(-0.3, 0.3, size=(ns, 3))
    G = rng.normal(size=(ns, 3)) * 1e-3
    pos = np.c_[P, np.full(ns, sigma ** 3)]
    strn = np.c_[G, np.zeros(ns)]
    Y = rng.uniform(-0.3, 0.3, size=(nt, 3))
    Y[:5] = P[:5] + rng.normal(size=(5, 3)) * 0.3 * sigma  # some targets inside cores
    nrm = rng.normal(size=(nt, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    tgt = np.c_[Y, np.zeros(nt)]
    u = oracle.p2p(pos, strn, tgt, sigma, grad=False)
    un = np.sum(u * nrm, axis=1)
    g = 2 * un[:, None] * nrm
    dx, dG = oracle.p2p_adjoint(pos, strn, tgt, sigma, g)
    h = 1e-6
    for j in list(range(5)) + list(rng.choice(np.arange(5, ns), 11, replace=False)):
        cj = np.sum(oracle.p2p(pos[j:j + 1], strn[j:j + 1], tgt, sigma, grad=False) * nrm, axis=1)
        b = un - cj
        for d in range(3):
            for which, ref in (("x", dx), ("G", dG)):
                pp, sp = pos[j:j + 1].copy(), strn[j:j + 1].copy()
                pm, sm = pos[j:j + 1].copy(), strn[j:j + 1].copy()
                if which == "x":
                    pp[0, d] += h
                    pm[0, d] -= h
                else:
                    sp[0, d] += h
                    sm[0, d] -= h
                cp = np.sum(oracle.p2p(pp, sp, tgt, sigma, grad=False) * nrm, axis=1)
                cm = np.sum(oracle.p2p(pm, sm, tgt, sigma, grad=False) * nrm, axis=1)
                fd = np.sum((cp - cm) * (2 * b + cp + cm)) / (2 * h)
                scale = np.abs(ref[j]).max()
                assert abs(ref[j, d] - fd) <= 1e-7 * scale, (which, j, d, ref[j, d], fd)
