"""The adjoint behind torch.autograd (autograd.VPMInduce): gradients of the downwash
loss L = sum_k (u_k . n_k)^2 at the 1,280 control points of the 4-blade hover rotor
with respect to the particles' positions and strengths, through
torch.autograd.grad, against the FP64 oracle's adjoint and against FP64 central
differences of the oracle's own forward sum."""
import numpy as np
import pytest

import oracle
from paper_2511_11430_gb300 import synth
from tests._util import rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11430_gb300 import autograd, build

    build.build()
    return autograd


@pytest.fixture(scope="module")
def wake():
    return synth.make(4, n=5000)


def _loss_grads(ag, w, compensated):
    pos = to_dev(w.pos).requires_grad_(True)
    strn = to_dev(w.strength).requires_grad_(True)
    tgt = to_dev(w.colloc).requires_grad_(True)
    nrm = to_dev(np.ascontiguousarray(w.normal[:, :3].T))
    u = ag.induce(pos, strn, tgt, w.sigma, compensated=compensated)  # [3, K]
    L = ((u * nrm).sum(0) ** 2).sum()
    gp, gs, gt = torch.autograd.grad(L, [pos, strn, tgt], allow_unused=True)
    return gp, gs, gt


def _oracle_seed(w):
    """g_k = dL/du_k = 2 (u_k . n_k) n_k with the oracle's FP64 velocity."""
    u = oracle.p2p(w.pos, w.strength, w.colloc, w.sigma, grad=False)
    n = w.normal[:, :3].astype(np.float64)
    return 2.0 * (u * n).sum(axis=1, keepdims=True) * n, u, n


@pytest.mark.parametrize("compensated,tol", [(True, 1e-5), (False, 1e-3)])
def test_autograd_matches_oracle_adjoint(ag, wake, compensated, tol):
    w = wake
    gp, gs, gt = _loss_grads(ag, w, compensated)
    g, _, _ = _oracle_seed(w)
    rx, rG = oracle.p2p_adjoint(w.pos, w.strength, w.colloc, w.sigma, g)
    gp = gp.double().cpu().numpy()
    gs = gs.double().cpu().numpy()
    assert rel_l2(gp[:, :3], rx) <= tol
    assert rel_l2(gs[:, :3], rG) <= tol
    # the volume lane and the 4th strength lane receive nothing; the control points are
    # not differentiated (the adjoint returns no dL/dy)
    assert np.all(gp[:, 3] == 0.0) and np.all(gs[:, 3] == 0.0)
    assert gt is None


def test_autograd_matches_central_differences(ag, wake):
    """dL/dx_j and dL/dGamma_j on 64 random particles against FP64 central differences
    (h = 1e-6 R).  Perturbing particle j changes only its own terms c_jk, so the
    difference is formed as L(+) - L(-) = sum_k (a+_k - a-_k)(2 b_k + a+_k + a-_k) with
    a_k = c_jk . n_k and b_k the rest of u_k . n_k, free of cancellation."""
    w = wake
    gp, gs, _ = _loss_grads(ag, w, True)
    gp = gp.double().cpu().numpy()[:, :3]
    gs = gs.double().cpu().numpy()[:, :3]
    _, u, n = _oracle_seed(w)
    un = (u * n).sum(axis=1)
    h = 1e-6 * synth.R
    idx = synth.sample_targets(64, w.n, 64)
    fd_x = np.zeros((len(idx), 3))
    fd_G = np.zeros((len(idx), 3))

    def a_of(p, s):
        c = oracle.p2p(p[None, :], s[None, :], w.colloc, w.sigma, grad=False)
        return (c * n).sum(axis=1)

    for r, j in enumerate(idx):
        p0 = w.pos[j].astype(np.float64)
        s0 = w.strength[j].astype(np.float64)
        b = un - a_of(p0, s0)
        for c in range(3):
            for which, out in ((0, fd_x), (1, fd_G)):
                pp, pm, sp, sm = p0.copy(), p0.copy(), s0.copy(), s0.copy()
                if which == 0:
                    pp[c] += h
                    pm[c] -= h
                else:
                    sp[c] += h
                    sm[c] -= h
                ap, am = a_of(pp, sp), a_of(pm, sm)
                out[r, c] = ((ap - am) * (2.0 * b + ap + am)).sum() / (2.0 * h)
    assert rel_l2(gp[idx], fd_x) <= 1e-5
    assert rel_l2(gs[idx], fd_G) <= 1e-5
