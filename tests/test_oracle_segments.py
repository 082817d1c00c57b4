"""Pins of the oracle's Vatistas-cored straight-segment velocity and gradient
(blade and wake vortex lines, Sec. II.A) against textbook closed forms, a direct
numerical line integral of the Biot-Savart law, finite differences, and the
particle discretisation of a segment by Eq. 6."""
import os

import numpy as np
import pytest
from scipy import integrate

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "segment_closed_forms.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, params, val = line.split()
        kv = dict(p.split("=") for p in params.split(","))
        out[name] = ({k: float(v) for k, v in kv.items()}, float(val))
    return out


def seg(a, b, gamma=1.0):
    return np.r_[a, gamma][None], np.r_[b, 0.0][None]


def u_at(sa, sb, x, core=0.0, n=2, grad=False):
    return oracle.segments(sa, sb, np.r_[x, 0][None], core, n, grad=grad)


def test_square_ring_centre():
    p, val = _golden()["square_ring_centre"]
    a = p["a"]
    c = np.array([[0, 0, 0], [a, 0, 0], [a, a, 0], [0, a, 0]], dtype=float)
    sa = np.c_[c, np.ones(4)]
    sb = np.c_[np.roll(c, -1, axis=0), np.zeros(4)]
    u = oracle.segments(sa, sb, np.array([[a / 2, a / 2, 0, 0]]), 0.0, 2, grad=False)
    np.testing.assert_allclose(u[0], [0, 0, val], rtol=1e-14, atol=1e-14)


def test_perpendicular_bisector():
    p, val = _golden()["bisector"]
    L, h = p["L"], p["h"]
    sa, sb = seg([-L / 2, 0, 0], [L / 2, 0, 0])
    u = u_at(sa, sb, [0, h, 0])
    np.testing.assert_allclose(u[0], [0, 0, val], rtol=1e-14)


def test_infinite_and_semi_infinite_line():
    p, val = _golden()["infinite_line"]
    h = p["h"]
    Lbig = 1e6
    sa, sb = seg([-Lbig, 0, 0], [Lbig, 0, 0])
    np.testing.assert_allclose(u_at(sa, sb, [0, 0, h])[0], [0, -val, 0], rtol=1e-10)
    sa, sb = seg([0, 0, 0], [Lbig, 0, 0])
    np.testing.assert_allclose(u_at(sa, sb, [0, 0, h])[0], [0, -val / 2, 0], rtol=1e-10)


@pytest.mark.parametrize("name,n", [("vatistas_n2", 2), ("vatistas_n1", 1)])
def test_vatistas_core_profile(name, n):
    p, val = _golden()[name]
    h, rc = p["h"], p["rc"]
    Lbig = 1e4
    sa, sb = seg([-Lbig, 0, 0], [Lbig, 0, 0])
    u = u_at(sa, sb, [0, h, 0], core=rc, n=n)
    np.testing.assert_allclose(u[0], [0, 0, val], rtol=1e-9)


def test_line_integral_of_biot_savart():
    """Away from the line the oracle equals the quadrature of Gamma/(4 pi) dl x (x-y)/|x-y|^3."""
    rng = np.random.default_rng(11)
    for _ in range(6):
        a, b = rng.normal(size=3), rng.normal(size=3)
        x = rng.normal(size=3) * 1.5
        g = rng.uniform(-2, 2)
        dl = b - a

        def comp(t, k):
            y = a + t * dl
            d = x - y
            return (np.cross(dl, d) / np.linalg.norm(d) ** 3)[k]

        ref = np.array([integrate.quad(comp, 0, 1, args=(k,), epsabs=1e-15, epsrel=1e-13)[0] for k in range(3)])
        ref *= g / (4 * np.pi)
        sa, sb = seg(a, b, g)
        np.testing.assert_allclose(u_at(sa, sb, x)[0], ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("n,core", [(2, 0.05), (1, 0.05), (2, 0.0)])
def test_gradient_matches_central_differences(n, core):
    rng = np.random.default_rng(5 + n)
    for _ in range(5):
        a, b = rng.normal(size=3) * 0.3, rng.normal(size=3) * 0.3
        x = rng.normal(size=3) * 0.3
        sa, sb = seg(a, b, rng.uniform(0.5, 2))
        u, J = u_at(sa, sb, x, core=core, n=n, grad=True)
        h = 1e-6
        Jfd = np.zeros((3, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            Jfd[:, k] = (u_at(sa, sb, x + e, core, n)[0] - u_at(sa, sb, x - e, core, n)[0]) / (2 * h)
        np.testing.assert_allclose(J[0], Jfd, rtol=0, atol=1e-7 * np.abs(J[0]).max())
        assert abs(np.trace(J[0])) <= 1e-12 * np.abs(J[0]).max()


def test_particle_chain_of_eq6_reproduces_segment_far_field():
    """A segment split into n Gaussian particles with Gamma_i = Gamma dl / n (Eq. 6) induces,
    far from the segment, the segment's own velocity; the midpoint-rule error falls as 1/n^2."""
    a, b, g = np.array([-0.5, 0.0, 0.0]), np.array([0.5, 0.1, 0.0]), 1.3
    sa, sb = seg(a, b, g)
    x = np.array([0.1, 0.6, 0.3])
    uref = u_at(sa, sb, x)[0]
    errs = []
    sigma = 0.01
    for n in (32, 128):
        t = (np.arange(n) + 0.5) / n
        P = a[None] + t[:, None] * (b - a)[None]
        Gi = np.repeat((g * (b - a) / n)[None], n, axis=0)
        up = oracle.p2p(np.c_[P, np.full(n, sigma ** 3)], np.c_[Gi, np.zeros(n)], np.r_[x, 0][None], sigma,
                        grad=False)[0]
        errs.append(np.linalg.norm(up - uref) / np.linalg.norm(uref))
    assert errs[1] < 1e-4
    assert 12 < errs[0] / errs[1] < 20  # second order: factor 16 for 4x more particles


def test_endpoint_and_axis_guards():
    sa, sb = seg([0, 0, 0], [1, 0, 0])
    assert np.all(u_at(sa, sb, [0, 0, 0], core=0.1, grad=True)[1] == 0)
    # on the axis beyond the segment with a core: zero velocity, finite gradient
    u, J = u_at(sa, sb, [2, 0, 0], core=0.1, grad=True)
    assert np.all(u == 0) and np.all(np.isfinite(J))
    # on the axis without core: guarded to zero
    u, J = u_at(sa, sb, [0.5, 0, 0], core=0.0, grad=True)
    assert np.all(u == 0) and np.all(J == 0)
