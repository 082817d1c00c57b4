"""PyTorch-facing wrappers of the libvpm C ABI (argument marshalling only).

Every function takes CUDA tensors, checks dtype/shape/contiguity, allocates the
outputs and the scratch workspace through PyTorch's caching allocator, and calls
the C entry point of the same name on the current CUDA stream.  All arithmetic
runs in the library's kernels.

Layouts follow include/vpm.h: particles ``pos[n, 4] = (x, y, z, volume)`` and
``strength[n, 4] = (Gx, Gy, Gz, -)``, targets ``tgt[n, 4]``, segments
``seg_a[m, 4] = (ax, ay, az, circulation)``, ``seg_b[m, 4]``; velocity outputs are
planar ``u[3, n]`` and ``grad_u[9, n]`` with ``grad_u[3*a + b, i] = d u_a / d x_b``.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import VpmParams, check


def _void(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t, name, dtype, shape_tail=None, allow_none=False):
    if t is None:
        if allow_none:
            return
        raise ValueError(f"{name} is required")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} must have shape [n, {', '.join(map(str, shape_tail))}], got {tuple(t.shape)}")


def workspace_size(op: int, n_src: int = 0, n_tgt: int = 0, m_seg: int = 0, flags: int = 0) -> int:
    out = ctypes.c_size_t(0)
    check(_lib.load().vpm_workspace_size(op, n_src, n_tgt, m_seg, flags, ctypes.byref(out)))
    return int(out.value)


class Workspace:
    """A reusable device scratch buffer that grows on demand (one per stream of use)."""

    def __init__(self, device=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda")
        self.buf = None

    def get(self, nbytes: int):
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        return self.buf


def _ws(ws, nbytes, device):
    if isinstance(ws, Workspace):
        return ws.get(nbytes)
    if ws is not None:
        if ws.numel() * ws.element_size() < nbytes:
            raise ValueError(f"workspace of {ws.numel() * ws.element_size()} bytes, need {nbytes}")
        return ws
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _flags(compensated=False, classic=False, check_finite=False):
    return ((_lib.VPM_COMPENSATED if compensated else 0) | (_lib.VPM_STRETCH_CLASSIC if classic else 0)
            | (_lib.VPM_CHECK_FINITE if check_finite else 0))


def induce(src_pos, src_str, tgt, sigma: float, compensated: bool = True, grad: bool = True, ws=None,
           check_finite: bool = False):
    """Velocity (and gradient) at ``tgt`` induced by Gaussian particles (Eq. 2-4)."""
    _need(src_pos, "src_pos", torch.float32, (4,))
    _need(src_str, "src_str", torch.float32, (4,))
    _need(tgt, "tgt", torch.float32, (4,))
    n_src, n_tgt = src_pos.shape[0], tgt.shape[0]
    dev = tgt.device
    u = torch.empty((3, n_tgt), dtype=torch.float32, device=dev)
    g = torch.empty((9, n_tgt), dtype=torch.float32, device=dev) if grad else None
    flags = _flags(compensated, check_finite=check_finite)
    nb = workspace_size(_lib.VPM_OP_INDUCE, n_src, n_tgt, 0, flags)
    w = _ws(ws, nb, dev)
    check(_lib.load().vpm_induce(_void(src_pos), _void(src_str), n_src, _void(tgt), n_tgt, float(sigma), flags,
                                 _void(u), _void(g), _void(w), w.numel(), _stream()))
    return (u, g) if grad else u


def tree_induce(pos, strength, sigma: float, theta: float = 0.5, order: int = 4, grad: bool = True, ws=None):
    """Velocity (and gradient) at every particle from all the others by the treecode
    (vpm_tree_induce): far clusters by their Taylor expansion of order ``order``,
    near ones by the direct sum; theta = 0 gives the direct sum."""
    _need(pos, "pos", torch.float32, (4,))
    _need(strength, "strength", torch.float32, (4,))
    n = pos.shape[0]
    dev = pos.device
    u = torch.empty((3, n), dtype=torch.float32, device=dev)
    g = torch.empty((9, n), dtype=torch.float32, device=dev) if grad else None
    w = _ws(ws, workspace_size(_lib.VPM_OP_TREE, n), dev)
    check(_lib.load().vpm_tree_induce(_void(pos), _void(strength), n, float(sigma), float(theta), int(order),
                                      _void(u), _void(g), _void(w), w.numel(), _stream()))
    return (u, g) if grad else u


def segments_induce(seg_a, seg_b, tgt, core: float, vatistas_n: int = 2, compensated: bool = True,
                    grad: bool = True, ws=None):
    """Velocity (and gradient) at ``tgt`` induced by Vatistas-cored straight segments (Sec. II.A)."""
    _need(seg_a, "seg_a", torch.float32, (4,))
    _need(seg_b, "seg_b", torch.float32, (4,))
    _need(tgt, "tgt", torch.float32, (4,))
    m, n_tgt = seg_a.shape[0], tgt.shape[0]
    dev = tgt.device
    u = torch.empty((3, n_tgt), dtype=torch.float32, device=dev)
    g = torch.empty((9, n_tgt), dtype=torch.float32, device=dev) if grad else None
    flags = _flags(compensated)
    nb = workspace_size(_lib.VPM_OP_SEGMENTS, 0, n_tgt, m, flags)
    w = _ws(ws, nb, dev)
    check(_lib.load().vpm_segments_induce(_void(seg_a), _void(seg_b), m, _void(tgt), n_tgt, float(core),
                                          int(vatistas_n), flags, _void(u), _void(g), _void(w), w.numel(),
                                          _stream()))
    return (u, g) if grad else u


@dataclass
class Params:
    """Parameters of the right-hand side (vpm_params in include/vpm.h)."""
    sigma: float
    nu: float = 1.5e-5
    c_v: float = 0.07
    seg_core: float | None = None
    u_inf: tuple = (0.0, 0.0, 0.0)
    vatistas_n: int = 2
    compensated: bool = True
    classic: bool = False
    check_finite: bool = False

    def to_c(self) -> VpmParams:
        p = VpmParams()
        p.sigma = float(self.sigma)
        p.nu = float(self.nu)
        p.c_v = float(self.c_v)
        p.seg_core = float(self.sigma if self.seg_core is None else self.seg_core)
        for a in range(3):
            p.u_inf[a] = float(self.u_inf[a])
        p.vatistas_n = int(self.vatistas_n)
        p.flags = _flags(self.compensated, self.classic, self.check_finite)
        return p


def _segs(seg_a, seg_b):
    if seg_a is None or seg_a.shape[0] == 0:
        return None, None, 0
    _need(seg_a, "seg_a", torch.float32, (4,))
    _need(seg_b, "seg_b", torch.float32, (4,))
    return seg_a, seg_b, seg_a.shape[0]


def rhs(pos, strength, seg_a, seg_b, params: Params, ws=None):
    """dx/dt [3, n], dGamma/dt [3, n] and nu_t [n] of Eq. 4-5."""
    _need(pos, "pos", torch.float32, (4,))
    _need(strength, "strength", torch.float32, (4,))
    sa, sb, m = _segs(seg_a, seg_b)
    n = pos.shape[0]
    dev = pos.device
    dxdt = torch.empty((3, n), dtype=torch.float32, device=dev)
    dGdt = torch.empty((3, n), dtype=torch.float32, device=dev)
    nut = torch.empty((n,), dtype=torch.float32, device=dev)
    cp = params.to_c()
    nb = workspace_size(_lib.VPM_OP_RHS, n, 0, m, cp.flags)
    w = _ws(ws, nb, dev)
    check(_lib.load().vpm_rhs(_void(pos), _void(strength), n, _void(sa), _void(sb), m, ctypes.byref(cp),
                              _void(dxdt), _void(dGdt), _void(nut), _void(w), w.numel(), _stream()))
    return dxdt, dGdt, nut


def rhs_tree(pos, strength, seg_a, seg_b, params: Params, theta: float = 0.5, order: int = 4, ws=None):
    """As rhs, with the particle and segment u and grad u from the treecode (vpm_rhs_tree)."""
    _need(pos, "pos", torch.float32, (4,))
    _need(strength, "strength", torch.float32, (4,))
    sa, sb, m = _segs(seg_a, seg_b)
    n = pos.shape[0]
    dev = pos.device
    dxdt = torch.empty((3, n), dtype=torch.float32, device=dev)
    dGdt = torch.empty((3, n), dtype=torch.float32, device=dev)
    nut = torch.empty((n,), dtype=torch.float32, device=dev)
    cp = params.to_c()
    w = _ws(ws, workspace_size(_lib.VPM_OP_RHS_TREE, n, 0, m, cp.flags), dev)
    check(_lib.load().vpm_rhs_tree(_void(pos), _void(strength), n, _void(sa), _void(sb), m, ctypes.byref(cp),
                                   float(theta), int(order), _void(dxdt), _void(dGdt), _void(nut), _void(w),
                                   w.numel(), _stream()))
    return dxdt, dGdt, nut


def pack_state(x, G, vol, pos=None, strength=None):
    """FP32 packed particles pos [n, 4], strength [n, 4] from the FP64 state x, G [3, n] and vol [n]."""
    _need(x, "x", torch.float64)
    _need(G, "G", torch.float64)
    _need(vol, "vol", torch.float32)
    n = x.shape[1]
    if pos is None:
        pos = torch.empty((n, 4), dtype=torch.float32, device=x.device)
    if strength is None:
        strength = torch.empty((n, 4), dtype=torch.float32, device=x.device)
    check(_lib.load().vpm_pack_state(_void(x), _void(G), _void(vol), n, _void(pos), _void(strength), _stream()))
    return pos, strength


def step(x, G, vol, seg_a, seg_b, params: Params, dt: float, ws=None):
    """One low-storage RK3 step, in place on x [3, n] and G [3, n] (float64)."""
    _need(x, "x", torch.float64)
    _need(G, "G", torch.float64)
    _need(vol, "vol", torch.float32)
    if x.dim() != 2 or x.shape[0] != 3 or G.shape != x.shape or vol.shape != (x.shape[1],):
        raise ValueError("x and G must be [3, n] and vol [n]")
    sa, sb, m = _segs(seg_a, seg_b)
    n = x.shape[1]
    cp = params.to_c()
    nb = workspace_size(_lib.VPM_OP_STEP, n, 0, m, cp.flags)
    w = _ws(ws, nb, x.device)
    check(_lib.load().vpm_step(_void(x), _void(G), _void(vol), n, _void(sa), _void(sb), m, ctypes.byref(cp),
                               float(dt), _void(w), w.numel(), _stream()))
    return x, G


def rk3_stage(k: int, x, G, q, vol, seg_a, seg_b, params: Params, dt: float, ws=None):
    """Stage k (0, 1, 2) of the low-storage RK3 step, in place on x, G [3, n] and the
    register q [6, n] (float64, kept by the caller between stages)."""
    _need(x, "x", torch.float64)
    _need(G, "G", torch.float64)
    _need(q, "q", torch.float64)
    _need(vol, "vol", torch.float32)
    if x.dim() != 2 or x.shape[0] != 3 or G.shape != x.shape or vol.shape != (x.shape[1],):
        raise ValueError("x and G must be [3, n] and vol [n]")
    if tuple(q.shape) != (6, x.shape[1]):
        raise ValueError("q must be [6, n]")
    sa, sb, m = _segs(seg_a, seg_b)
    n = x.shape[1]
    cp = params.to_c()
    w = _ws(ws, workspace_size(_lib.VPM_OP_STAGE, n, 0, m, cp.flags), x.device)
    check(_lib.load().vpm_rk3_stage(int(k), _void(x), _void(G), _void(q), _void(vol), n, _void(sa), _void(sb), m,
                                    ctypes.byref(cp), float(dt), _void(w), w.numel(), _stream()))
    return x, G


def step_tree(x, G, vol, seg_a, seg_b, params: Params, dt: float, theta: float = 0.5, order: int = 4, ws=None):
    """As step, with the treecode right-hand side (vpm_step_tree)."""
    _need(x, "x", torch.float64)
    _need(G, "G", torch.float64)
    _need(vol, "vol", torch.float32)
    if x.dim() != 2 or x.shape[0] != 3 or G.shape != x.shape or vol.shape != (x.shape[1],):
        raise ValueError("x and G must be [3, n] and vol [n]")
    sa, sb, m = _segs(seg_a, seg_b)
    n = x.shape[1]
    cp = params.to_c()
    w = _ws(ws, workspace_size(_lib.VPM_OP_STEP_TREE, n, 0, m, cp.flags), x.device)
    check(_lib.load().vpm_step_tree(_void(x), _void(G), _void(vol), n, _void(sa), _void(sb), m, ctypes.byref(cp),
                                    float(theta), int(order), float(dt), _void(w), w.numel(), _stream()))
    return x, G


def aic_build(rings, colloc, normal, core: float, vatistas_n: int = 2, v_rel=None, w_ind=None, rhs: bool = True):
    """AIC matrix A [n, n] (float32) and, when v_rel is given, the Neumann right-hand side b [n] (float64)."""
    _need(rings, "rings", torch.float32, (4, 4))
    _need(colloc, "colloc", torch.float32, (4,))
    _need(normal, "normal", torch.float32, (4,))
    n = rings.shape[0]
    dev = rings.device
    A = torch.empty((n, n), dtype=torch.float32, device=dev)
    b = None
    if rhs and v_rel is not None:
        _need(v_rel, "v_rel", torch.float32, (4,))
        if w_ind is not None:
            _need(w_ind, "w_ind", torch.float32)
        b = torch.empty((n,), dtype=torch.float64, device=dev)
    check(_lib.load().aic_build(_void(rings), _void(colloc), _void(normal), n, float(core), int(vatistas_n),
                                _void(v_rel), _void(w_ind), _void(A), _void(b), _stream()))
    return A, b


def ring_segments(rings, gamma, seg_a=None, seg_b=None):
    """The 4 n segments c0->c1->c2->c3->c0 of n blade rings [n, 4, 4] carrying the
    circulations gamma [n] (float64): seg_a, seg_b [4 n, 4] (float32, a.w = circulation)."""
    _need(rings, "rings", torch.float32, (4, 4))
    _need(gamma, "gamma", torch.float64)
    n = rings.shape[0]
    if seg_a is None:
        seg_a = torch.empty((4 * n, 4), dtype=torch.float32, device=rings.device)
    if seg_b is None:
        seg_b = torch.empty((4 * n, 4), dtype=torch.float32, device=rings.device)
    check(_lib.load().vpm_ring_segments(_void(rings), _void(gamma), n, _void(seg_a), _void(seg_b), _stream()))
    return seg_a, seg_b


def aic_solve(A, b, tol: float = 1e-12, max_iter: int = 30, ws=None, raise_on_fail: bool = True):
    """x [n] float64 with A factored in FP32 and FP64 iterative refinement; returns (x, iters, backward_error)."""
    _need(A, "A", torch.float32)
    _need(b, "b", torch.float64)
    n = b.shape[0]
    x = torch.empty((n,), dtype=torch.float64, device=b.device)
    nb = workspace_size(_lib.VPM_OP_AIC_SOLVE, 0, n, 0, 0)
    w = _ws(ws, nb, b.device)
    it = ctypes.c_int(0)
    be = ctypes.c_double(0.0)
    st = _lib.load().aic_solve(_void(A), _void(b), _void(x), n, float(tol), int(max_iter), ctypes.byref(it),
                               ctypes.byref(be), _void(w), w.numel(), _stream())
    if raise_on_fail or st not in (_lib.VPM_OK, _lib.VPM_ERR_NOT_CONVERGED):
        check(st)
    return x, int(it.value), float(be.value)


def induce_backward(src_pos, src_str, tgt, sigma: float, grad_out, compensated: bool = True, ws=None):
    """dL/dx [3, n_src] and dL/dGamma [3, n_src] for grad_out = dL/du [3, n_tgt]."""
    _need(src_pos, "src_pos", torch.float32, (4,))
    _need(src_str, "src_str", torch.float32, (4,))
    _need(tgt, "tgt", torch.float32, (4,))
    _need(grad_out, "grad_out", torch.float32)
    n_src, n_tgt = src_pos.shape[0], tgt.shape[0]
    if tuple(grad_out.shape) != (3, n_tgt):
        raise ValueError("grad_out must be [3, n_tgt]")
    dev = src_pos.device
    dx = torch.empty((3, n_src), dtype=torch.float32, device=dev)
    dG = torch.empty((3, n_src), dtype=torch.float32, device=dev)
    flags = _flags(compensated)
    nb = workspace_size(_lib.VPM_OP_BACKWARD, n_src, n_tgt, 0, flags)
    w = _ws(ws, nb, dev)
    check(_lib.load().vpm_induce_backward(_void(src_pos), _void(src_str), n_src, _void(tgt), n_tgt, float(sigma),
                                          flags, _void(grad_out), _void(dx), _void(dG), _void(w), w.numel(),
                                          _stream()))
    return dx, dG


def trace_enable(timing: bool = True) -> None:
    check(_lib.load().vpm_trace_enable(1 if timing else 0))


def trace_reset() -> None:
    check(_lib.load().vpm_trace_reset())


def trace_read(kind: int):
    """(launches, total_ms) of a trace kind (VPM_TRACE_*); synchronises on the recorded events."""
    n = ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    check(_lib.load().vpm_trace_read(int(kind), ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def device_error() -> int:
    """Reads and clears the library's device error word (synchronises the device)."""
    code = ctypes.c_int(0)
    check(_lib.load().vpm_device_error(ctypes.byref(code)))
    return int(code.value)


def _wake_out(ld, device):
    x = torch.empty((3, max(ld, 1)), dtype=torch.float64, device=device)
    return x, torch.empty_like(x)


def wake_convert(edge_a, edge_b, gamma, trailed, ds_tip: float, n_tip: int, n_shed: int = 1, gamma_nb=None,
                 has_nb=None, capacity: int | None = None, ws=None):
    """Particles from wake edges (Sec. II.C, Eq. 6-8): returns x [3, n] and Gamma [3, n]
    (float64, planar).  ``capacity`` bounds n (default: enough for every edge's count)."""
    _need(edge_a, "edge_a", torch.float64, (3,))
    _need(edge_b, "edge_b", torch.float64, (3,))
    _need(gamma, "gamma", torch.float64)
    _need(trailed, "trailed", torch.int32)
    if has_nb is not None:
        _need(has_nb, "has_nb", torch.int32)
        _need(gamma_nb, "gamma_nb", torch.float64)
    m = edge_a.shape[0]
    lib = _lib.load()
    w = _ws(ws, workspace_size(_lib.VPM_OP_WAKE_CONVERT, m, 0, 0, 0), edge_a.device)
    n_out = ctypes.c_int64(0)
    cap = capacity
    if cap is None:  # ask for the count first (nothing is written when it does not fit)
        st = lib.vpm_wake_convert(_void(edge_a), _void(edge_b), _void(gamma), _void(gamma_nb), _void(has_nb),
                                  _void(trailed), m, float(ds_tip), int(n_tip), int(n_shed), None, None, 0,
                                  ctypes.byref(n_out), _void(w), w.numel(), _stream())
        if st not in (_lib.VPM_OK, _lib.VPM_ERR_LIMIT):
            check(st)
        cap = int(n_out.value)
    x, G = _wake_out(cap, edge_a.device)
    st = lib.vpm_wake_convert(_void(edge_a), _void(edge_b), _void(gamma), _void(gamma_nb), _void(has_nb),
                              _void(trailed), m, float(ds_tip), int(n_tip), int(n_shed), _void(x), _void(G), cap,
                              ctypes.byref(n_out), _void(w), w.numel(), _stream())
    check(st)
    n = int(n_out.value)
    return x[:, :n], G[:, :n]


def wake_convert_row(U, D, gamma, ds_tip: float, n_tip: int, n_shed: int = 1, capacity: int | None = None, ws=None):
    """Particles from one wake panel row (node lines U, D [S+1, 3], circulations [S])."""
    _need(U, "U", torch.float64, (3,))
    _need(D, "D", torch.float64, (3,))
    _need(gamma, "gamma", torch.float64)
    S = gamma.shape[0]
    lib = _lib.load()
    w = _ws(ws, workspace_size(_lib.VPM_OP_WAKE_ROW, S, 0, 0, 0), U.device)
    n_out = ctypes.c_int64(0)
    cap = capacity
    if cap is None:
        st = lib.vpm_wake_convert_row(_void(U), _void(D), _void(gamma), S, float(ds_tip), int(n_tip), int(n_shed),
                                      None, None, 0, ctypes.byref(n_out), _void(w), w.numel(), _stream())
        if st not in (_lib.VPM_OK, _lib.VPM_ERR_LIMIT):
            check(st)
        cap = int(n_out.value)
    x, G = _wake_out(cap, U.device)
    st = lib.vpm_wake_convert_row(_void(U), _void(D), _void(gamma), S, float(ds_tip), int(n_tip), int(n_shed),
                                  _void(x), _void(G), cap, ctypes.byref(n_out), _void(w), w.numel(), _stream())
    check(st)
    n = int(n_out.value)
    return x[:, :n], G[:, :n]
