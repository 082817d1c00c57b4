"""FP64 CPU oracle of the vortex-particle hot path (test infrastructure only).

This package is the independent reference that the CUDA library is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the product package never does.  It shares no
code with the CUDA path: the arithmetic lives in ``vpm_oracle.c`` (plain double
loops written from the paper's Eq. 2-5, the Vatistas segment law, the Vreman
model, Williamson's RK3 and textbook LU), and this module only marshals numpy
arrays through ctypes.

Array conventions (all float64, C-contiguous, row-major):
  pos[n, 4] = (x, y, z, volume), str[n, 4] = (Gx, Gy, Gz, 0),
  tgt[n, 4] = (x, y, z, 0), seg_a[m, 4] = (ax, ay, az, circulation),
  seg_b[m, 4] = (bx, by, bz, 0); outputs u[n, 3] and J[n, 3, 3] with
  J[i, a, b] = d u_a / d x_b at target i.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vpm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math) into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # VPM_ORACLE_LIB points at another build of vpm_oracle.c (the mutation tests
            # use it to check that the pins catch planted mistakes).
            path = os.environ.get("VPM_ORACLE_LIB")
            if not path:
                build()
                path = _LIB_PATH
            lib = ctypes.CDLL(path)
            P = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            d = ctypes.c_double
            i = ctypes.c_int
            IP = ctypes.POINTER(ctypes.c_int)
            LP = ctypes.POINTER(ctypes.c_int64)
            sig = {
                "orc_blob_gF": [P, i64, P, P],
                "orc_p2p": [P, P, i64, P, i64, d, P, P],
                "orc_segments": [P, P, i64, P, i64, d, i, P, P],
                "orc_vreman": [P, i64, d, d, P],
                "orc_stretch": [P, P, i64, i, P],
                "orc_pse": [P, P, P, i64, d, d, P],
                "orc_pse_at": [P, P, P, i64, LP, i64, d, d, P],
                "orc_rhs": [P, P, i64, P, P, i64, d, d, d, d, i, P, i, P, P, P],
                "orc_step": [P, P, P, i64, P, P, i64, d, d, d, d, i, P, i, d, i],
                "orc_aic_build": [P, P, P, i64, d, i, P],
                "orc_aic_rhs": [P, P, P, i64, P],
                "orc_lu_solve": [P, P, i64, P],
                "orc_p2p_adjoint": [P, P, i64, P, i64, d, P, P, P],
                "orc_wake_convert": [P, P, P, P, IP, IP, i64, d, i, i, i64, P, P, LP],
                "orc_wake_row_edges": [P, P, P, i64, P, P, P, P, IP, IP],
                "orc_set_threads": [i],
                "orc_blade_loads": [P, P, i64, P, P, P, P, P, P, P, P, i64, d, d, P],
            }
            rtype = {"orc_lu_solve": ctypes.c_int, "orc_wake_convert": ctypes.c_int64}
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = rtype.get(name)
            _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, cols=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if cols is not None and a.shape[-1] != cols:
        pad = np.zeros(a.shape[:-1] + (cols,), dtype=np.float64)
        pad[..., : a.shape[-1]] = a
        a = pad
    return a


def set_threads(n: int | None) -> None:
    """Set the OpenMP thread count the oracle uses (None: leave the default)."""
    if n is not None:
        os.environ["OMP_NUM_THREADS"] = str(int(n))
        _load().orc_set_threads(int(n))


def blob_gF(rho):
    """g(rho) and F(rho) = rho g' - 3 g of the Gaussian blob (Eq. 3)."""
    rho = _f64(rho).ravel()
    g = np.empty_like(rho)
    F = np.empty_like(rho)
    _load().orc_blob_gF(_p(rho), rho.size, _p(g), _p(F))
    return g, F


def p2p(pos, strength, tgt, sigma, grad=True):
    """Velocity (and gradient) at targets induced by Gaussian particles."""
    pos, strength, tgt = _f64(pos, 4), _f64(strength, 4), _f64(tgt, 4)
    nt = tgt.shape[0]
    u = np.zeros((nt, 3))
    J = np.zeros((nt, 3, 3)) if grad else None
    _load().orc_p2p(_p(pos), _p(strength), pos.shape[0], _p(tgt), nt, float(sigma), _p(u), _p(J))
    return (u, J) if grad else u


def segments(seg_a, seg_b, tgt, core, vatistas_n=2, grad=True):
    """Velocity (and gradient) at targets induced by Vatistas-cored straight segments."""
    seg_a, seg_b, tgt = _f64(seg_a, 4), _f64(seg_b, 4), _f64(tgt, 4)
    nt = tgt.shape[0]
    u = np.zeros((nt, 3))
    J = np.zeros((nt, 3, 3)) if grad else None
    _load().orc_segments(_p(seg_a), _p(seg_b), seg_a.shape[0], _p(tgt), nt, float(core), int(vatistas_n), _p(u), _p(J))
    return (u, J) if grad else u


def vreman(J, delta, c_v=0.07):
    J = _f64(J).reshape(-1, 9)
    nu = np.zeros(J.shape[0])
    _load().orc_vreman(_p(J), J.shape[0], float(delta), float(c_v), _p(nu))
    return nu


def stretch(J, strength, classic=False):
    J = _f64(J).reshape(-1, 9)
    strength = _f64(strength, 4)
    s = np.zeros((J.shape[0], 3))
    _load().orc_stretch(_p(J), _p(strength), J.shape[0], int(bool(classic)), _p(s))
    return s


def pse(pos, strength, nu_t, sigma, nu):
    pos, strength = _f64(pos, 4), _f64(strength, 4)
    nt = None if nu_t is None else _f64(nu_t).ravel()
    p = np.zeros((pos.shape[0], 3))
    _load().orc_pse(_p(pos), _p(strength), _p(nt), pos.shape[0], float(sigma), float(nu), _p(p))
    return p


def pse_at(pos, strength, nu_t, sigma, nu, idx):
    """The exchange term of pse() at the particles idx only, each summed over all particles."""
    pos, strength = _f64(pos, 4), _f64(strength, 4)
    nt = None if nu_t is None else _f64(nu_t).ravel()
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    p = np.zeros((ix.size, 3))
    _load().orc_pse_at(_p(pos), _p(strength), _p(nt), pos.shape[0],
                       ix.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ix.size, float(sigma), float(nu), _p(p))
    return p


def _seg_arrays(seg_a, seg_b):
    if seg_a is None or len(seg_a) == 0:
        z = np.zeros((1, 4))
        return z, z, 0
    a, b = _f64(seg_a, 4), _f64(seg_b, 4)
    return a, b, a.shape[0]


def rhs(pos, strength, seg_a, seg_b, sigma, nu=1.5e-5, c_v=0.07, seg_core=None, vatistas_n=2,
        u_inf=(0.0, 0.0, 0.0), classic=False):
    """dx/dt, dGamma/dt and nu_t for every particle (Eq. 4-5)."""
    pos, strength = _f64(pos, 4), _f64(strength, 4)
    a, b, m = _seg_arrays(seg_a, seg_b)
    n = pos.shape[0]
    dxdt, dGdt, nut = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    ui = _f64(u_inf)
    _load().orc_rhs(_p(pos), _p(strength), n, _p(a), _p(b), m, float(sigma), float(nu), float(c_v),
                    float(sigma if seg_core is None else seg_core), int(vatistas_n), _p(ui), int(bool(classic)),
                    _p(dxdt), _p(dGdt), _p(nut))
    return dxdt, dGdt, nut


def step(x, G, vol, seg_a, seg_b, sigma, dt, nu=1.5e-5, c_v=0.07, seg_core=None, vatistas_n=2,
         u_inf=(0.0, 0.0, 0.0), classic=False, cast_f32=True):
    """One low-storage RK3 step; returns new (x, G) arrays of shape [n, 3]."""
    x = _f64(x).copy()
    G = _f64(G).copy()
    vol = _f64(vol).ravel()
    a, b, m = _seg_arrays(seg_a, seg_b)
    ui = _f64(u_inf)
    _load().orc_step(_p(x), _p(G), _p(vol), x.shape[0], _p(a), _p(b), m, float(sigma), float(nu), float(c_v),
                     float(sigma if seg_core is None else seg_core), int(vatistas_n), _p(ui), int(bool(classic)),
                     float(dt), int(bool(cast_f32)))
    return x, G


def aic_build(rings, colloc, normal, core, vatistas_n=2):
    rings = _f64(rings)
    if rings.shape[-1] == 3:
        rings = _f64(rings, 4)
    rings = np.ascontiguousarray(rings.reshape(-1, 4, 4))
    colloc, normal = _f64(colloc, 4), _f64(normal, 4)
    n = rings.shape[0]
    A = np.zeros((n, n))
    _load().orc_aic_build(_p(rings), _p(colloc), _p(normal), n, float(core), int(vatistas_n), _p(A))
    return A


def aic_rhs(v_rel, w_ind, normal):
    v_rel, normal = _f64(v_rel, 4), _f64(normal, 4)
    w = None if w_ind is None else _f64(w_ind)
    b = np.zeros(v_rel.shape[0])
    _load().orc_aic_rhs(_p(v_rel), _p(w), _p(normal), v_rel.shape[0], _p(b))
    return b


def lu_solve(A, b):
    A, b = _f64(A), _f64(b).ravel()
    x = np.zeros(b.size)
    rc = _load().orc_lu_solve(_p(A), _p(b), b.size, _p(x))
    if rc != 0:
        raise np.linalg.LinAlgError("zero pivot")
    return x


def p2p_adjoint(pos, strength, tgt, sigma, g):
    """dL/dx_j and dL/dGamma_j for a loss gradient g[k] = dL/du_k at the targets."""
    pos, strength, tgt, g = _f64(pos, 4), _f64(strength, 4), _f64(tgt, 4), _f64(g)
    ns = pos.shape[0]
    dx, dG = np.zeros((ns, 3)), np.zeros((ns, 3))
    _load().orc_p2p_adjoint(_p(pos), _p(strength), ns, _p(tgt), tgt.shape[0], float(sigma), _p(g), _p(dx), _p(dG))
    return dx, dG


def _ip(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def wake_convert(a, b, gamma, gamma_nb, has_nb, trailed, ds_tip, n_tip, n_shed=1):
    """Particles (x [n][3], G [n][3]) and per-edge counts from wake edges (Eq. 6-8)."""
    a, b = _f64(a).reshape(-1, 3), _f64(b).reshape(-1, 3)
    m = a.shape[0]
    g = _f64(gamma).ravel()
    gnb = _f64(np.zeros(m) if gamma_nb is None else gamma_nb).ravel()
    hn = np.ascontiguousarray(np.zeros(m) if has_nb is None else has_nb, dtype=np.int32)
    tr = np.ascontiguousarray(trailed, dtype=np.int32)
    counts = np.zeros(m, dtype=np.int64)
    lib = _load()
    cap = 0
    x = np.zeros((1, 3))
    G = np.zeros((1, 3))
    total = lib.orc_wake_convert(_p(a), _p(b), _p(g), _p(gnb), _ip(hn), _ip(tr), m, float(ds_tip), int(n_tip),
                                 int(n_shed), cap, _p(x), _p(G), counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if total == -2:
        raise ValueError("wake_convert: an edge's particle count is not finite or above 2^30")
    total = int(counts.sum())
    x = np.zeros((max(total, 1), 3))
    G = np.zeros((max(total, 1), 3))
    got = lib.orc_wake_convert(_p(a), _p(b), _p(g), _p(gnb), _ip(hn), _ip(tr), m, float(ds_tip), int(n_tip),
                               int(n_shed), total, _p(x), _p(G), counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    assert got == total
    return x[:total], G[:total], counts


def wake_row_edges(U, D, gamma):
    """Edges of one wake panel row (U, D node lines [S+1][3], panel circulations [S])."""
    U, D = _f64(U).reshape(-1, 3), _f64(D).reshape(-1, 3)
    g = _f64(gamma).ravel()
    S = g.size
    ne = 3 * S + 1
    a, b = np.zeros((ne, 3)), np.zeros((ne, 3))
    ge, gnb = np.zeros(ne), np.zeros(ne)
    hn = np.zeros(ne, dtype=np.int32)
    tr = np.zeros(ne, dtype=np.int32)
    _load().orc_wake_row_edges(_p(U), _p(D), _p(g), S, _p(a), _p(b), _p(ge), _p(gnb), _ip(hn), _ip(tr))
    return a, b, ge, gnb, hn, tr


def blade_loads(seg_a, seg_b, u_ind, omega, hub, u_inf, rings, normal, gamma, gamma_prev, dt, rho=1.225):
    """(force [3], moment about hub [3]) of the bound segments (Kutta-Joukowski) and of the
    panels' circulation change (unsteady Bernoulli); see orc_blade_loads."""
    sa, sb = _f64(seg_a, 4), _f64(seg_b, 4)
    u = _f64(u_ind).reshape(-1, 3)
    rings = _f64(rings)
    if rings.shape[-1] == 3:
        rings = _f64(rings, 4)
    rings = np.ascontiguousarray(rings.reshape(-1, 4, 4))
    nrm = _f64(normal, 4)
    g = _f64(gamma).ravel()
    gp = None if gamma_prev is None else _f64(gamma_prev).ravel()
    out = np.zeros(6)
    _load().orc_blade_loads(_p(sa), _p(sb), sa.shape[0], _p(u), _p(_f64(omega)), _p(_f64(hub)), _p(_f64(u_inf)),
                            _p(rings), _p(nrm), _p(g), _p(gp), g.size, float(dt), float(rho), _p(out))
    return out[:3], out[3:]
