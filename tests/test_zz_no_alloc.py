"""vpm_induce_noalloc: the velocity/gradient sweep for callers that cannot allocate
device memory for a workspace (for example a C or Fortran solver linked without a
CUDA memory manager, or a loop that must not allocate).  It runs on scratch the
library keeps in its own device memory, so it must give what the FP64 oracle and
vpm_induce with a caller workspace give, call after call (with and without the
gradient, on scratch the previous call left behind), up to its stated capacity,
and refuse problems too large for that scratch.  Collected last so that a run
stopping at the first failure has already run every other test; it also passes
alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2511_11430_gb300 import synth
from tests._util import TOL_COMP, TOL_PLAIN, rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11430_gb300 import _lib, build

    build.build()
    return _lib.load()


def _noalloc(lib, pos, G, tgt, sigma, grad=True, flags=1):
    n_src, n_tgt = pos.shape[0], tgt.shape[0]
    u = torch.full((3, n_tgt), float("nan"), dtype=torch.float32, device="cuda")
    g = torch.full((9, n_tgt), float("nan"), dtype=torch.float32, device="cuda") if grad else None
    st = lib.vpm_induce_noalloc(ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(G.data_ptr()), n_src,
                                ctypes.c_void_p(tgt.data_ptr()), n_tgt, ctypes.c_float(sigma), flags,
                                ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(g.data_ptr()) if grad else None,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, u, g


def _rows(t, idx):
    return t[:, idx].double().cpu().numpy().T


@pytest.mark.parametrize("compensated", [True, False])
def test_noalloc_matches_oracle_on_small_hover_wake(lib, compensated):
    w = synth.make(1)
    P, S = to_dev(w.pos), to_dev(w.strength)
    st, u, g = _noalloc(lib, P, S, P, w.sigma, flags=1 if compensated else 0)
    assert st == 0, lib.vpm_last_error()
    torch.cuda.synchronize()
    ru, rJ = oracle.p2p(w.pos, w.strength, w.pos, w.sigma)
    tol = TOL_COMP if compensated else TOL_PLAIN
    idx = np.arange(w.n)
    assert rel_l2(_rows(u, idx), ru) <= tol
    assert rel_l2(_rows(g, idx).reshape(-1, 3, 3), rJ) <= tol


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls(lib):
    from paper_2511_11430_gb300 import api

    w = synth.make(1)
    pos, G = synth.random_cloud(9, 3001, sigma=0.05)
    tgt, _ = synth.random_cloud(10, 517, sigma=0.05)
    # calls in a row on the one scratch array: sizes and layouts change from call to
    # call (the velocity-only sweep keeps 3 partial rows per target, the gradient 14),
    # so each call starts on what the previous one left behind
    cases = [(w.pos, w.strength, w.pos, w.sigma, True), (pos, G, tgt, 0.05, True),
             (pos, G, tgt, 0.05, False), (w.pos, w.strength, w.pos, w.sigma, False),
             (w.pos, w.strength, w.pos, w.sigma, True)]
    for pos_, G_, tgt_, sigma, grad in cases:
        P, S, Tg = to_dev(pos_), to_dev(G_), to_dev(tgt_)
        ref = api.induce(P, S, Tg, sigma, compensated=True, grad=grad)
        u_ref, g_ref = ref if grad else (ref, None)
        st, u, g = _noalloc(lib, P, S, Tg, sigma, grad=grad)
        assert st == 0, lib.vpm_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(u).all()
        assert rel_l2(u.double().cpu().numpy(), u_ref.double().cpu().numpy()) <= TOL_COMP
        if grad:
            assert torch.isfinite(g).all()
            assert rel_l2(g.double().cpu().numpy(), g_ref.double().cpu().numpy()) <= TOL_COMP


def test_noalloc_at_its_stated_capacity(lib):
    """250,000 particles of the hover wake onto themselves with the gradient, near the
    limit the header states for a 152-SM GB300, against the oracle on sampled targets."""
    w = synth.make(2, n=250_000)
    P, S = to_dev(w.pos), to_dev(w.strength)
    st, u, g = _noalloc(lib, P, S, P, w.sigma)
    assert st == 0, lib.vpm_last_error()
    torch.cuda.synchronize()
    idx = synth.sample_targets(8, w.n, 256)
    ru, rJ = oracle.p2p(w.pos, w.strength, w.pos[idx], w.sigma)
    assert rel_l2(_rows(u, idx), ru) <= TOL_COMP
    assert rel_l2(_rows(g, idx).reshape(-1, 3, 3), rJ) <= TOL_COMP


def test_noalloc_refuses_problems_beyond_its_scratch(lib):
    from paper_2511_11430_gb300 import _lib

    pos = to_dev(np.zeros((4, 4), dtype=np.float32))
    u = torch.zeros((3, 4), dtype=torch.float32, device="cuda")
    huge = 1 << 26  # far more sources than the fixed scratch can hold; nothing is launched
    st = lib.vpm_induce_noalloc(ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(pos.data_ptr()), huge,
                                ctypes.c_void_p(pos.data_ptr()), 4, ctypes.c_float(0.1), 1,
                                ctypes.c_void_p(u.data_ptr()), None, None)
    assert st == _lib.VPM_ERR_LIMIT
    assert b"scratch" in lib.vpm_last_error()
