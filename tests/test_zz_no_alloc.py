"""vpm_induce_noalloc: the velocity/gradient sweep for callers that cannot allocate
device memory for a workspace (for example a C or Fortran solver linked without a
CUDA memory manager, or a loop that must not allocate).  It runs on scratch the
library keeps in its own device memory, so it must give what vpm_induce gives
with a caller workspace, call after call, and refuse problems too large for that
scratch.  Collected last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2511_11430_gb300 import synth
from tests._util import TOL_COMP, rel_l2, to_dev

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


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls(lib):
    from paper_2511_11430_gb300 import api

    cases = []
    w = synth.make(1)
    cases.append((w.pos, w.strength, w.pos, w.sigma))
    pos, G = synth.random_cloud(9, 3001, sigma=0.05)
    tgt, _ = synth.random_cloud(10, 517, sigma=0.05)
    cases.append((pos, G, tgt, 0.05))
    for pos, G, tgt, sigma in cases:  # two calls in a row, different sizes
        P, S, Tg = to_dev(pos), to_dev(G), to_dev(tgt)
        u_ref, g_ref = api.induce(P, S, Tg, sigma, compensated=True)
        st, u, g = _noalloc(lib, P, S, Tg, sigma)
        assert st == 0, lib.vpm_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(u).all() and torch.isfinite(g).all()
        assert rel_l2(u.double().cpu().numpy(), u_ref.double().cpu().numpy()) <= TOL_COMP
        assert rel_l2(g.double().cpu().numpy(), g_ref.double().cpu().numpy()) <= TOL_COMP


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
