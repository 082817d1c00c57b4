"""The wake panel -> particle conversion (Sec. II.C, Eq. 6-8) through the C ABI
against the FP64 oracle.  Counts are integers decided in FP64 by the same correctly
rounded operations on both sides, and positions/strengths are the same sequence of
correctly rounded FP64 operations, so the comparison is exact."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2511_11430_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_11430_gb300 import api as a, build

    build.build()
    return a


def _d(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _random_edges(seed, m):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(m, 3))
    b = a + rng.normal(size=(m, 3)) * rng.uniform(0.01, 2.0, size=(m, 1))
    g = rng.normal(size=m)
    gnb = rng.normal(size=m)
    hn = (rng.uniform(size=m) < 0.5).astype(np.int32)
    tr = (rng.uniform(size=m) < 0.7).astype(np.int32)
    return a, b, g, gnb, hn, tr


@pytest.mark.parametrize("m,n_tip,n_shed", [(1, 1, 1), (37, 2, 1), (1000, 3, 2), (4099, 5, 3)])
def test_wake_convert_matches_oracle_exactly(api, m, n_tip, n_shed):
    a, b, g, gnb, hn, tr = _random_edges(m, m)
    ds_tip = 0.37
    xr, Gr, cr = oracle.wake_convert(a, b, g, gnb, hn, tr, ds_tip, n_tip, n_shed)
    x, G = api.wake_convert(_d(a), _d(b), _d(g), _d(tr, torch.int32), ds_tip, n_tip, n_shed, gamma_nb=_d(gnb),
                            has_nb=_d(hn, torch.int32))
    torch.cuda.synchronize()
    assert x.shape[1] == cr.sum()
    np.testing.assert_array_equal(x.cpu().numpy().T, xr)
    np.testing.assert_array_equal(G.cpu().numpy().T, Gr)


def test_wake_convert_large_and_without_neighbours(api):
    m = 100_000
    a, b, g, _, _, tr = _random_edges(7, m)
    xr, Gr, cr = oracle.wake_convert(a, b, g, None, None, tr, 0.11, 4, 2)
    x, G = api.wake_convert(_d(a), _d(b), _d(g), _d(tr, torch.int32), 0.11, 4, 2)
    torch.cuda.synchronize()
    assert x.shape[1] == cr.sum() > 10 * m
    np.testing.assert_array_equal(x.cpu().numpy().T, xr)
    np.testing.assert_array_equal(G.cpu().numpy().T, Gr)


def _hover_wake_row(S=40):
    """The oldest near-wake row of the hover rotor's blade 0: the trailing-edge node
    line, and the same line one time step (5 deg) earlier in azimuth, dropped by the
    inflow, so that the trailed edges grow with radius as in a rotor wake."""
    w = synth.make(1)
    r = np.linspace(0.15, 1.0, S + 1)
    dpsi = np.deg2rad(5.0)
    U = np.stack([np.zeros(S + 1), r, np.full(S + 1, -0.01)], 1)
    D = np.stack([r * np.sin(-dpsi), r * np.cos(-dpsi), np.full(S + 1, -0.02)], 1)
    rc = 0.5 * (r[1:] + r[:-1])
    gamma = 2.0 * rc * np.sqrt(1 - rc ** 2)
    return U, D, gamma, w


@pytest.mark.parametrize("n_tip", [1, 2, 4])
def test_wake_convert_row_matches_oracle(api, n_tip):
    U, D, gamma, _ = _hover_wake_row()
    ds_tip = float(np.sqrt(((D[-1] - U[-1]) ** 2).sum()))
    a, b, g, gnb, hn, tr = oracle.wake_row_edges(U, D, gamma)
    xr, Gr, cr = oracle.wake_convert(a, b, g, gnb, hn, tr, ds_tip, n_tip, 1)
    x, G = api.wake_convert_row(_d(U), _d(D), _d(gamma), ds_tip, n_tip, 1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.cpu().numpy().T, xr)
    np.testing.assert_array_equal(G.cpu().numpy().T, Gr)
    # Eq. 8 puts fewer particles on the short inboard trailed edges than the
    # conventional strategy that gives every trailed edge the tip's n_tip
    S = gamma.size
    if n_tip > 1:
        assert cr[:S + 1].sum() < n_tip * (S + 1)
    assert cr[S] == n_tip


def test_wake_convert_edge_cases(api):
    from paper_2511_11430_gb300 import _lib

    lib = _lib.load()
    # an empty edge list
    e = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    x, G = api.wake_convert(e, e, torch.zeros(0, dtype=torch.float64, device="cuda"),
                            torch.zeros(0, dtype=torch.int32, device="cuda"), 1.0, 2)
    assert x.shape == (3, 0)
    # a zero-length trailed edge keeps one particle of zero strength
    a = _d([[1.0, 2.0, 3.0]])
    x, G = api.wake_convert(a, a.clone(), _d([5.0]), _d([1], torch.int32), 1.0, 3)
    torch.cuda.synchronize()
    assert x.shape == (3, 1) and torch.all(G == 0) and torch.all(x[:, 0] == a[0])
    # too small a capacity: VPM_ERR_LIMIT, the needed count reported, nothing written
    b = _d([[1.0, 2.0, 13.0]])
    xo = torch.full((3, 4), 7.0, dtype=torch.float64, device="cuda")
    Go = xo.clone()
    ws = torch.empty(4096, dtype=torch.uint8, device="cuda")
    n_out = ctypes.c_int64(-1)
    tr = _d([1], torch.int32)
    g = _d([1.0])
    st = lib.vpm_wake_convert(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                              None, None, ctypes.c_void_p(tr.data_ptr()), 1, ctypes.c_double(1.0), 1, 1,
                              ctypes.c_void_p(xo.data_ptr()), ctypes.c_void_p(Go.data_ptr()), 4, ctypes.byref(n_out),
                              ctypes.c_void_p(ws.data_ptr()), 4096, None)
    torch.cuda.synchronize()
    assert st == _lib.VPM_ERR_LIMIT and n_out.value == 10 and torch.all(xo == 7.0)
    # invalid arguments: nothing launched
    st = lib.vpm_wake_convert(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                              None, None, ctypes.c_void_p(tr.data_ptr()), 1, ctypes.c_double(0.0), 1, 1,
                              ctypes.c_void_p(xo.data_ptr()), ctypes.c_void_p(Go.data_ptr()), 4, ctypes.byref(n_out),
                              ctypes.c_void_p(ws.data_ptr()), 4096, None)
    assert st == _lib.VPM_ERR_INVALID_ARG
