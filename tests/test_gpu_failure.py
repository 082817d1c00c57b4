"""Failure detection on the GPU without a fault: a bounded device wait on an mbarrier
phase that nothing completes must give up after its limit, latch the timeout in the
device error word (read and cleared by vpm_device_error) and leave the context usable."""
import ctypes
import time

import numpy as np
import pytest

import oracle
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


def test_bounded_wait_times_out_and_reports(lib):
    from paper_2511_11430_gb300 import _lib, api

    code = ctypes.c_int(-1)
    assert lib.vpm_device_error(ctypes.byref(code)) == 0  # start clean
    done = ctypes.c_int(-1)
    t0 = time.perf_counter()
    st = lib.vpm_selftest_wait(ctypes.c_double(20.0), ctypes.byref(done), None)
    dt = time.perf_counter() - t0
    assert st == 0, lib.vpm_last_error()
    assert done.value == 0  # the wait gave up
    assert 0.015 <= dt < 2.0
    assert lib.vpm_device_error(ctypes.byref(code)) == 0 and code.value == _lib.VPM_ERR_LIMIT
    assert lib.vpm_device_error(ctypes.byref(code)) == 0 and code.value == 0  # read once, cleared
    # the context is still usable
    pos, G = synth.random_cloud(3, 700, sigma=0.05)
    u, J = api.induce(to_dev(pos), to_dev(G), to_dev(pos), 0.05, compensated=True)
    ru, rJ = oracle.p2p(pos, G, pos, 0.05)
    assert rel_l2(u.double().cpu().numpy().T, ru) <= TOL_COMP
    assert lib.vpm_device_error(ctypes.byref(code)) == 0 and code.value == 0


def test_selftest_rejects_bad_limits(lib):
    from paper_2511_11430_gb300 import _lib

    done = ctypes.c_int(-1)
    assert lib.vpm_selftest_wait(ctypes.c_double(0.0), ctypes.byref(done), None) == _lib.VPM_ERR_INVALID_ARG
    assert lib.vpm_selftest_wait(ctypes.c_double(5000.0), ctypes.byref(done), None) == _lib.VPM_ERR_INVALID_ARG
    assert lib.vpm_selftest_wait(ctypes.c_double(10.0), None, None) == _lib.VPM_ERR_INVALID_ARG
