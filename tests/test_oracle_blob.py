"""Pins of the oracle's Gaussian-particle velocity and gradient (Eq. 2-4) against
mathematics that does not go through the oracle's own formulas: arbitrary-precision
evaluation of the blob's enclosed-vorticity function, direct numerical quadrature of
the Biot-Savart integral over the Gaussian vorticity of Eq. 3, the singular far field,
the solid-body near field, finite differences and symmetries."""
import numpy as np
import pytest
from scipy import integrate, stats

import oracle

SQ2PI = np.sqrt(2.0 / np.pi)


def test_enclosed_vorticity_matches_maxwell_cdf_and_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rho = np.concatenate([np.logspace(-5, 0, 40), np.linspace(1.0, 12.0, 45)])
    g, F = oracle.blob_gF(rho)
    for r, gi, Fi in zip(rho, g, F):
        R = mp.mpf(float(r))
        g_ref = mp.erf(R / mp.sqrt(2)) - mp.sqrt(2 / mp.pi) * R * mp.exp(-R * R / 2)
        F_ref = mp.sqrt(2 / mp.pi) * R ** 3 * mp.exp(-R * R / 2) - 3 * g_ref
        assert abs(gi - float(g_ref)) <= 1e-14 * abs(float(g_ref)) + 1e-300
        assert abs(Fi - float(F_ref)) <= 1e-13 * abs(float(F_ref)) + 1e-300
    # the same function is the Maxwell (chi, 3 dof) distribution's CDF
    np.testing.assert_allclose(g[rho > 1e-3], stats.maxwell.cdf(rho[rho > 1e-3]), rtol=1e-12)


def _blob_speed_quadrature(r, sigma):
    """|u| / |Gamma x r_hat| for one blob by 2-D quadrature of Biot-Savart over its vorticity.

    With the evaluation point on the polar axis at distance r and y = x - s n, the
    integrand of Biot-Savart over Gamma zeta(y) becomes Gamma x n zeta(|x - s n|)/(4 pi)
    ds dOmega; the azimuthal integral of n leaves 2 pi cos(theta) along the axis.
    """
    norm = (2 * np.pi * sigma ** 2) ** -1.5

    def inner(s, t):
        d2 = r * r - 2 * s * r * t + s * s
        return t * norm * np.exp(-0.5 * d2 / sigma ** 2)

    smax = r + 14 * sigma
    val, err = integrate.dblquad(inner, -1.0, 1.0, 0.0, smax, epsabs=1e-16, epsrel=1e-13)
    return 0.5 * val


@pytest.mark.parametrize("rho", [0.05, 0.4, 1.0, 1.7, 3.0, 5.5])
def test_single_blob_velocity_equals_biot_savart_quadrature(rho):
    sigma = 0.3
    r = rho * sigma
    ref = _blob_speed_quadrature(r, sigma)
    G = np.array([[0.0, 0.0, 2.0, 0.0]])
    tgt = np.array([[r, 0.0, 0.0, 0.0]])
    u = oracle.p2p(np.zeros((1, 4)), G, tgt, sigma, grad=False)
    # Gamma x r_hat = 2 z x x = (0, 2, 0)
    np.testing.assert_allclose(u[0], [0.0, 2.0 * ref, 0.0], rtol=2e-10, atol=1e-14 * abs(ref))


def test_far_field_is_singular_biot_savart():
    sigma = 0.01
    rng = np.random.default_rng(0)
    for _ in range(5):
        r = rng.normal(size=3)
        r *= 40 * sigma / np.linalg.norm(r)
        G = rng.normal(size=3)
        u, J = oracle.p2p(np.zeros((1, 4)), np.r_[G, 0][None], np.r_[r, 0][None], sigma)
        rr = np.linalg.norm(r)
        np.testing.assert_allclose(u[0], np.cross(G, r) / (4 * np.pi * rr ** 3), rtol=1e-14)
        # gradient of the point vortex: K' r / r with K = 1/(4 pi r^3)
        Jref = np.zeros((3, 3))
        eps = np.zeros((3, 3, 3))
        eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
        eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
        K = 1 / (4 * np.pi * rr ** 3)
        H = -3 / (4 * np.pi * rr ** 5)
        Jref = K * np.einsum("acb,c->ab", eps, G) + H * np.outer(np.cross(G, r), r)
        np.testing.assert_allclose(J[0], Jref, rtol=1e-13, atol=1e-13 * np.abs(Jref).max())


def test_near_field_is_solid_body_rotation():
    sigma = 0.05
    G = np.array([0.3, -0.2, 1.0])
    r = np.array([1.0, 2.0, -0.5]) * 1e-6 * sigma  # next series term is O(rho^2) ~ 1e-12
    u = oracle.p2p(np.zeros((1, 4)), np.r_[G, 0][None], np.r_[r, 0][None], sigma, grad=False)
    omega = SQ2PI / (12 * np.pi * sigma ** 3)
    np.testing.assert_allclose(u[0], omega * np.cross(G, r), rtol=1e-10)


def _fd_jacobian(pos, G, x, sigma, h):
    J = np.zeros((3, 3))
    for b in range(3):
        e = np.zeros(3)
        e[b] = h
        up = oracle.p2p(pos, G, np.r_[x + e, 0][None], sigma, grad=False)[0]
        um = oracle.p2p(pos, G, np.r_[x - e, 0][None], sigma, grad=False)[0]
        J[:, b] = (up - um) / (2 * h)
    return J


@pytest.mark.parametrize("rho", [0.02, 0.3, 0.99, 1.01, 2.5, 6.0, 15.0])
def test_gradient_matches_central_differences(rho):
    sigma = 0.1
    rng = np.random.default_rng(int(rho * 100))
    pos = np.zeros((1, 4))
    G = np.r_[rng.normal(size=3), 0][None]
    d = rng.normal(size=3)
    x = d / np.linalg.norm(d) * rho * sigma
    _, J = oracle.p2p(pos, G, np.r_[x, 0][None], sigma)
    Jfd = _fd_jacobian(pos, G, x, sigma, 1e-5 * sigma)
    np.testing.assert_allclose(J[0], Jfd, rtol=0, atol=2e-8 * np.abs(J[0]).max())
    # divergence-free velocity: trace vanishes
    assert abs(np.trace(J[0])) <= 1e-13 * np.abs(J[0]).max()


def test_pair_symmetry_odd_velocity_even_gradient():
    sigma = 0.2
    rng = np.random.default_rng(3)
    xj = rng.normal(size=3)
    G = rng.normal(size=3)
    for _ in range(4):
        r = rng.normal(size=3) * sigma * rng.uniform(0.1, 5)
        src = np.r_[xj, 1][None]
        up, Jp = oracle.p2p(src, np.r_[G, 0][None], np.r_[xj + r, 0][None], sigma)
        um, Jm = oracle.p2p(src, np.r_[G, 0][None], np.r_[xj - r, 0][None], sigma)
        np.testing.assert_allclose(up, -um, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(Jp, Jm, rtol=1e-12, atol=1e-13 * np.abs(Jp).max())


def test_brute_force_four_particles_and_no_self_induction():
    """u at each of 4 particles = sum over the other 3 of independent quadratures."""
    sigma = 0.25
    rng = np.random.default_rng(7)
    P = rng.normal(size=(4, 3)) * 0.3
    G = rng.normal(size=(4, 3))
    pos = np.c_[P, np.full(4, sigma ** 3)]
    strn = np.c_[G, np.zeros(4)]
    u = oracle.p2p(pos, strn, pos, sigma, grad=False)
    for i in range(4):
        ref = np.zeros(3)
        for j in range(4):
            if j == i:
                continue
            r = P[i] - P[j]
            rr = np.linalg.norm(r)
            ref += _blob_speed_quadrature(rr, sigma) * np.cross(G[j], r / rr)
        np.testing.assert_allclose(u[i], ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


def test_coincident_pair_contributes_nothing():
    sigma = 0.1
    pos = np.array([[0.1, 0.2, 0.3, 1e-3], [0.1, 0.2, 0.3, 1e-3], [0.5, 0.2, 0.3, 1e-3]])
    G = np.array([[1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, 1.0, 0]])
    u_all = oracle.p2p(pos, G, pos[:1], sigma, grad=False)
    u_far = oracle.p2p(pos[2:], G[2:], pos[:1], sigma, grad=False)
    np.testing.assert_array_equal(u_all, u_far)
