#!/usr/bin/env python3
"""Throughput of the vortex-particle hot path on GB300.

One step = one pass of the whole hot path over a synthetic rotor wake:
  pack the FP64 particle state to FP32, the particles' velocity at the blade control
  points, the AIC build and its FP32-LU / FP64-refined solve, the blade rings'
  segments with the solved circulations, one stage of the low-storage RK3 time
  update (its right-hand side: the particle + segment u + grad u sweep, Vreman,
  stretching, PSE; then the FP64 stage update), and the adjoint of the downwash
  loss at the control points.  The stage index cycles 0, 1, 2, so three
  consecutive steps are one full RK3 time step.
Default workload: two counter-rotating 3-blade rotors (2,000,000 particles, 7,680
segments, 1,920 control points) -- the largest single-GPU configuration.
Metric: particle-particle u + grad u pair interactions per second (N (N - 1) per
step), compensated FP32.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config 1..5]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "VPM pair interactions/s (u+∇u), compensated FP32 vs FP64 form at stated error"
UNIT = "pair-interactions/s"
FLOPS_P2P = 54   # u + grad u, far-field operation tree, FFMA = 2 flops
FLOPS_SEG = 120  # Vatistas segment u + grad u, same counting convention
L2_FLUSH_BYTES = 256 << 20
TOL = {"compensated": 2e-6, "plain": 1e-4, "nu_t": {"compensated": 1e-5, "plain": 1e-3}}
# DRAM bytes (read + write) of one sweep_kernel<grad, compensated, stretch> launch over the
# particle tiles, from one ncu capture of that launch per workload (profiles/sweep_kernel_*.md), keyed by
# (particles, segments); valid only while the kernel's sources hash to SWEEP_SRC_SHA256,
# else the bench reports traffic null.
SWEEP_TRAFFIC_BYTES = {(2_000_000, 7_680): 142_549_244_000 + 355_496_960}
SWEEP_SRC_SHA256 = "554c12209b1a3bebcca23b4f0ce95552fb9362a866002d2d20a1288ac8c463fe"
SWEEP_SRC = ["paper_2511_11430_gb300/csrc/vpm_sweep.cu", "paper_2511_11430_gb300/csrc/vpm_kernel.cuh",
             "paper_2511_11430_gb300/csrc/vpm_common.cuh"]


def sweep_src_hash():
    import hashlib

    h = hashlib.sha256()
    for f in SWEEP_SRC:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def sweep_traffic(n, m):
    """The captured DRAM traffic of one sweep launch, if a capture matches the sources
    and the workload."""
    if sweep_src_hash() != SWEEP_SRC_SHA256:
        return None
    return SWEEP_TRAFFIC_BYTES.get((n, m))


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=5)
    ap.add_argument("--particles", type=int, default=None, help="override the particle count (testing only)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the informative extras (segment/particle parts, treecode, wake conversion, "
                         "the hover-wake line)")
    ap.add_argument("--cpu-seconds", type=float, default=None,
                    help="reference arm: seconds of oracle work per step (default: 60 s over all steps)")
    ap.add_argument("--error-targets", type=int, default=1024)
    ap.add_argument("--part", choices=["aic", "wake", "tree", "rotor", "rhs"], default=None,
                    help="time one component alone (for profiling; prints a text line, not the JSON contract)")
    return ap.parse_args(argv)


def run_rotor(args):
    """The AH-1G rotor in forward flight (Eq. 12 pitch and flapping, advance ratio 0.19)
    through the near-wake driver: shedding, conversion, RK3 particles, AIC and loads each
    step, for --steps revolutions at 10 deg per step (after --warmup revolutions, whose
    loads are reported too).  Prints the thrust and torque coefficients averaged per
    revolution, the particle count and the wall time per step."""
    import torch

    from paper_2511_11430_gb300 import build, synth, wake

    build.build()
    kin = synth.AH1G
    dpsi = 10.0
    per_rev = int(round(360.0 / dpsi))
    # sigma 0.075 R: about 1.3 times the particle spacing on the tip's trailed edge
    # (Omega R dt / n_tip), the overlap the particle method needs
    g = wake.RotorWake(n_blades=2, n_span=24, n_chord=4, max_rows=2, n_tip=3, kin=kin,
                       dt=np.deg2rad(dpsi) / kin.omega, sigma=0.075 * kin.radius, seg_core=0.02 * kin.radius)
    revs = args.warmup + args.steps
    t0 = time.perf_counter()
    for _ in range(revs * per_rev):
        g.step()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    h = np.array(g.history)
    rows = []
    for r in range(revs):
        seg = h[r * per_rev:(r + 1) * per_rev]
        rows.append({"revolution": r + 1, "C_T": float(seg[:, 1].mean()), "C_Q": float(seg[:, 2].mean())})
    print(json.dumps({"part": "rotor", "case": "AH-1G forward flight, mu 0.19, 2 blades x 24 x 4 panels, 10 deg steps",
                      "revolutions": rows, "particles": g.n, "ms_per_step": 1e3 * wall / (revs * per_rev),
                      "paper_C_T": {"NL-UVLM-VPM": 0.00478, "experiment": 0.00464}}), flush=True)


def run_part(args):
    """One component, repeated --steps times after --warmup: the AIC build + solve of the
    blade lattice, the conversion of 2,000 hover wake rows, the treecode (theta 0.5,
    order 4) on the 1,000,000-particle BVI wake (--particles to shrink it), or the
    direct right-hand side (vpm_rhs, compensated: the particle and segment sweeps, Vreman,
    stretching, PSE) of the --config workload."""
    import torch

    from paper_2511_11430_gb300 import api, build, synth

    build.build()

    def T(a, dt=None):
        t = torch.from_numpy(np.ascontiguousarray(a))
        return (t if dt is None else t.to(dt)).cuda()
    if args.part == "aic":
        w = synth.make(args.config, n=1000)
        rings, colloc, normal, vrel = T(w.rings), T(w.colloc), T(w.normal), T(w.v_rel)
        wsb = api.Workspace()

        def once():
            A, b = api.aic_build(rings, colloc, normal, w.seg_core, 2, v_rel=vrel)
            return api.aic_solve(A, b, tol=1e-12, max_iter=30, ws=wsb)
        what = f"aic_build + aic_solve, n = {w.n_ctrl}"
    elif args.part == "tree":
        w = synth.make(3, n=args.particles)
        P, S = T(w.pos), T(w.strength)
        wsb = api.Workspace()

        def once():
            return api.tree_induce(P, S, w.sigma, theta=0.5, order=4, ws=wsb)
        what = f"tree_induce (theta 0.5, order 4), {w.n:,} particles"
    elif args.part == "rhs":
        w = synth.make(args.config) if args.particles is None else synth.make(args.config, n=args.particles)
        P, S, A, B = T(w.pos), T(w.strength), T(w.seg_a), T(w.seg_b)
        prm = api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core, u_inf=w.u_inf, compensated=True)
        wsb = api.Workspace()

        def once():
            return api.rhs(P, S, A, B, prm, ws=wsb)
        what = f"rhs (compensated), {w.name}: {w.n:,} particles, {w.m:,} segments"
    else:
        ea, eb, eg, egn, ehn, etr, ds_tip = synth.rotor_wake_edges(5, 2000)
        wa, wb, wg, wgn = (T(q, torch.float64) for q in (ea, eb, eg, egn))
        whn, wtr = T(ehn, torch.int32), T(etr, torch.int32)
        wsb = api.Workspace()
        npart = int(api.wake_convert(wa, wb, wg, wtr, ds_tip, 4, 1, gamma_nb=wgn, has_nb=whn, ws=wsb)[0].shape[1])

        def once():
            return api.wake_convert(wa, wb, wg, wtr, ds_tip, 4, 1, gamma_nb=wgn, has_nb=whn, capacity=npart, ws=wsb)
        what = f"wake_convert, {len(ea)} edges -> {npart} particles"
    for _ in range(args.warmup):
        once()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        once()
    e1.record()
    e1.synchronize()
    print(f"{what}: {e0.elapsed_time(e1) / max(args.steps, 1):.3f} ms per call", flush=True)


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_desc(w):
    rot = w.meta.get("rotors")
    head = f"{rot} x {w.meta.get('blades')}-blade rotors" if rot else f"{w.meta.get('blades')}-blade rotor"
    return (f"{w.name}: {head}, {w.n:,} Gaussian particles (sigma {w.sigma:g} R), "
            f"{w.m:,} Vatistas blade segments, {w.n_ctrl:,} control points")


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores (CPU baseline, reference values, reference arm)
# ---------------------------------------------------------------------------
def oracle_rate(w, seconds, cores):
    """P2P u + grad u pair interactions/s of the FP64 oracle on a bounded sample of
    targets against all sources (sized to take about `seconds`)."""
    import oracle
    from paper_2511_11430_gb300 import synth

    oracle.build()
    oracle.set_threads(cores)
    n = w.n
    k = 64
    while True:
        idx = synth.sample_targets(7, n, k)
        t0 = time.perf_counter()
        oracle.p2p(w.pos, w.strength, w.pos[idx], w.sigma)
        dt = time.perf_counter() - t0
        if dt >= seconds * 0.5 or k >= n:
            rate = k * (n - 1) / dt
            return rate, k, dt
        k = min(n, int(k * max(2.0, seconds / max(dt, 1e-3) * 0.6)))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def error_samples(w, k):
    """Sampled particles of the error report: k random ones (u, grad u, dx/dt, nu_t and
    dGamma/dt without the eddy viscosity's exchange coupling) and runs of consecutive
    particles for the full right-hand side (all particles of a small wake)."""
    from paper_2511_11430_gb300 import synth

    idx_u = synth.sample_targets(11, w.n, k)
    idx_r = np.arange(w.n) if w.n <= 4000 else synth.sample_runs(12, w.n, 2, 16)
    return idx_u, idx_r


def oracle_reference(w, idx_u, idx_r, cores):
    """The FP64 oracle's values at the sampled particles, and its timed rate (the
    cpu_baseline leg: u + grad u at idx_u against every particle)."""
    import oracle
    from oracle import sampled

    oracle.build()
    oracle.set_threads(cores)
    t0 = time.perf_counter()
    u, J = oracle.p2p(w.pos, w.strength, w.pos[idx_u], w.sigma)
    dt = time.perf_counter() - t0
    rate = len(idx_u) * (w.n - 1) / dt
    us, Js = oracle.segments(w.seg_a, w.seg_b, w.pos[idx_u], w.seg_core, w.vatistas_n)
    Jt = J + Js
    ref = {"u": u, "grad_u": J, "dxdt": u + us + np.asarray(w.u_inf), "nu_t": oracle.vreman(Jt, w.sigma, w.c_v),
           "dGdt_cv0": oracle.stretch(Jt, w.strength[idx_u]) + oracle.pse_at(w.pos, w.strength, None, w.sigma, w.nu,
                                                                             idx_u)}
    rdx, rdG, rnut = sampled.rhs_at(w, idx_r)
    ref.update({"dxdt_r": rdx, "dGdt": rdG, "nu_t_r": rnut})
    # one core, on a sample of about 3 s
    k1 = max(8, int(len(idx_u) * 3.0 / max(dt * cores, 1e-3)))
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.p2p(w.pos, w.strength, w.pos[idx_u[:k1]], w.sigma)
    d1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{len(idx_u)} sampled targets x all {w.n:,} sources, P2P u + grad u in FP64 ({dt:.1f} s)",
           "single_thread": {"value": min(k1, len(idx_u)) * (w.n - 1) / d1, "unit": UNIT,
                             "sample": f"{min(k1, len(idx_u))} sampled targets x all {w.n:,} sources ({d1:.1f} s)"}}
    return ref, cpu


def max_over_ranks(dist, ms, device):
    """The slowest rank's time: every rank's timed region ends when the last one does."""
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world_size, units_per_rank_step, steps, total_ms):
    """Units that all ranks processed (each rank runs its own replica) per second."""
    return world_size * units_per_rank_step * steps / (total_ms * 1e-3)


def run_reference(args):
    ws, rank, local = dist_info()
    if ws > 1 and rank != 0:
        return  # the oracle runs once, on rank 0's host cores; the other ranks exit without work
    from paper_2511_11430_gb300 import synth

    w = synth.make(args.config) if args.particles is None else synth.make(args.config, n=args.particles)
    cores = host_cores()
    per_step = args.cpu_seconds if args.cpu_seconds is not None else max(2.0, 60.0 / max(1, args.steps + args.warmup))
    rates = []
    for i in range(args.warmup + args.steps):
        r, k, dt = oracle_rate(w, per_step, cores)
        if i >= args.warmup:
            rates.append((r, k, dt))
    value = float(np.mean([r for r, _, _ in rates]))
    k = rates[-1][1]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean([d for _, _, d in rates]) * 1e3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(w), "reference": "FP64 CPU oracle (plain direct sum) on host cores",
                   "sample": f"{k} targets x {w.n - 1:,} sources per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{k} sampled targets x all {w.n:,} sources, P2P u + grad u in FP64"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
class HotPath:
    """The benchmark step on one workload, through the public API."""

    def __init__(self, w, dev):
        import torch

        from paper_2511_11430_gb300 import api

        self.api, self.w, self.dev = api, w, dev
        T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        self.n, self.m, self.K = w.n, w.m, w.n_ctrl
        self.x0 = np.ascontiguousarray(w.pos[:, :3].astype(np.float64).T)
        self.G0 = np.ascontiguousarray(w.strength[:, :3].astype(np.float64).T)
        self.vol = T(w.pos[:, 3].copy())
        self.rings, self.colloc, self.normal, self.vrel = T(w.rings), T(w.colloc), T(w.normal), T(w.v_rel)
        self.nrm = self.normal[:, :3].t().contiguous()
        self.T = T

    def params(self, compensated):
        w = self.w
        return self.api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core, u_inf=w.u_inf,
                               compensated=compensated)

    def new_state(self):
        import torch

        return {"x": self.T(self.x0), "G": self.T(self.G0),
                "q": torch.zeros((6, self.n), dtype=torch.float64, device=self.dev), "k": 0}

    def new_bufs(self):
        import torch

        n, dev = self.n, self.dev
        return {"ws": self.api.Workspace(dev), "ws_aic": self.api.Workspace(dev), "ws_adj": self.api.Workspace(dev),
                "pos": torch.empty((n, 4), dtype=torch.float32, device=dev),
                "str": torch.empty((n, 4), dtype=torch.float32, device=dev),
                "sa": torch.empty((4 * self.K, 4), dtype=torch.float32, device=dev),
                "sb": torch.empty((4 * self.K, 4), dtype=torch.float32, device=dev)}

    def step(self, st, prm, b, x=None, G=None, q=None, vol=None):
        """One pass of the hot path: one RK3 stage of the particles with the blade
        circulation solved for the current wake.  Returns (Gamma_b, dL/dx, dL/dGamma)."""
        api, w = self.api, self.w
        x = st["x"] if x is None else x
        G = st["G"] if G is None else G
        q = st["q"] if q is None else q
        vol = self.vol if vol is None else vol
        pos, strn = api.pack_state(x, G, vol, b["pos"], b["str"])
        u_c = api.induce(pos, strn, self.colloc, w.sigma, compensated=prm.compensated, grad=False, ws=b["ws"])
        A, rhs = api.aic_build(self.rings, self.colloc, self.normal, w.seg_core, 2, v_rel=self.vrel, w_ind=u_c)
        gam, _, _ = api.aic_solve(A, rhs, tol=1e-12, max_iter=30, ws=b["ws_aic"])
        sa, sb = api.ring_segments(self.rings, gam, b["sa"], b["sb"])
        api.rk3_stage(st["k"], x, G, q, vol, sa, sb, prm, w.dt, ws=b["ws"])
        st["k"] = (st["k"] + 1) % 3
        g = 2.0 * (u_c * self.nrm).sum(0, keepdim=True) * self.nrm  # d/du of sum_k (u_k . n_k)^2
        dx, dG = api.induce_backward(pos, strn, self.colloc, w.sigma, g.contiguous(), compensated=prm.compensated,
                                     ws=b["ws_adj"])
        return gam, dx, dG


def timed_loop(hp, prm, steps, warmup, flush, dist, trace=False):
    """W untimed steps, then K steps, each bracketed by CUDA events on the launching
    stream after an L2 flush outside the events.  Returns (total ms, trace)."""
    import torch

    from paper_2511_11430_gb300 import _lib

    api = hp.api
    st = hp.new_state()
    b = hp.new_bufs()
    for _ in range(warmup):
        hp.step(st, prm, b)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    if trace:
        api.trace_enable(True)
        api.trace_reset()
    s = torch.cuda.current_stream()
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        hp.step(st, prm, b)
        e1.record(s)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    tr = None
    if trace:
        tr = {k: api.trace_read(k) for k in (_lib.VPM_TRACE_ALL, _lib.VPM_TRACE_SWEEP, _lib.VPM_TRACE_ADJOINT,
                                             _lib.VPM_TRACE_PSE, _lib.VPM_TRACE_SWEEP_VEL,
                                             _lib.VPM_TRACE_SEGMENTS)}
        api.trace_enable(False)
    return total, tr


def e2e_loop(hp, prm, steps, warmup, flush, dist):
    """The same step end to end through the public API from pinned host buffers: each
    timed step copies its inputs (FP64 state and RK register, volumes, blade geometry)
    host -> device, runs, and copies its results (state, register, blade circulation,
    adjoint) back, all inside the step's events (the L2 flush stays outside)."""
    import torch

    n, K = hp.n, hp.K
    w = hp.w
    dev = hp.dev
    xh = torch.from_numpy(hp.x0).pin_memory()
    Gh = torch.from_numpy(hp.G0).pin_memory()
    qh = torch.zeros((6, n), dtype=torch.float64).pin_memory()
    volh = torch.from_numpy(w.pos[:, 3].copy()).pin_memory()
    geo_h = [torch.from_numpy(a).pin_memory() for a in (w.rings, w.colloc, w.normal, w.v_rel)]
    xo, Go, qo = torch.empty_like(xh).pin_memory(), torch.empty_like(Gh).pin_memory(), torch.empty_like(qh).pin_memory()
    gho = torch.empty((K,), dtype=torch.float64).pin_memory()
    dxo = torch.empty((3, n), dtype=torch.float32).pin_memory()
    dGo = torch.empty((3, n), dtype=torch.float32).pin_memory()
    x_d, G_d, q_d = (torch.empty_like(t, device=dev) for t in (xh, Gh, qh))
    vol_d = torch.empty_like(volh, device=dev)
    geo_d = [torch.empty_like(h, device=dev) for h in geo_h]
    b = hp.new_bufs()
    st = {"k": 0}

    def one():
        x_d.copy_(xh, non_blocking=True)
        G_d.copy_(Gh, non_blocking=True)
        q_d.copy_(qh, non_blocking=True)
        vol_d.copy_(volh, non_blocking=True)
        for d_, h_ in zip(geo_d, geo_h):
            d_.copy_(h_, non_blocking=True)
        hp.rings, hp.colloc, hp.normal, hp.vrel = geo_d
        hp.nrm = hp.normal[:, :3].t().contiguous()
        gam, dx, dG = hp.step(st, prm, b, x=x_d, G=G_d, q=q_d, vol=vol_d)
        xo.copy_(x_d, non_blocking=True)
        Go.copy_(G_d, non_blocking=True)
        qo.copy_(q_d, non_blocking=True)
        gho.copy_(gam, non_blocking=True)
        dxo.copy_(dx, non_blocking=True)
        dGo.copy_(dG, non_blocking=True)

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    s = torch.cuda.current_stream()
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        one()
        e1.record(s)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    h2d = (xh.numel() + Gh.numel() + qh.numel()) * 8 + volh.numel() * 4 + sum(h.numel() * 4 for h in geo_h)
    d2h = (xo.numel() + Go.numel() + qo.numel() + gho.numel()) * 8 + (dxo.numel() + dGo.numel()) * 4
    return total, int(h2d), int(d2h)


def gpu_error_values(hp, idx_u, idx_r):
    """The GPU's outputs at the sampled particles, both precision forms, from full-size
    launches on the initial state: vpm_induce (u, grad u), vpm_rhs with the workload's
    Vreman coefficient (dx/dt, nu_t, dGamma/dt) and with c_V = 0 (dGamma/dt without
    the eddy viscosity)."""
    import torch

    api, w = hp.api, hp.w
    P, S = hp.T(w.pos), hp.T(w.strength)
    sa, sb = hp.T(w.seg_a), hp.T(w.seg_b)
    ws = api.Workspace(hp.dev)
    rows = lambda t, ix: t[:, ix].double().cpu().numpy().T
    out = {}
    for form, comp in (("compensated", True), ("plain", False)):
        u, g = api.induce(P, S, P, w.sigma, compensated=comp, ws=ws)
        prm = hp.params(comp)
        dx, dG, nut = api.rhs(P, S, sa, sb, prm, ws=ws)
        prm0 = hp.params(comp)
        prm0.c_v = 0.0
        _, dG0, _ = api.rhs(P, S, sa, sb, prm0, ws=ws)
        torch.cuda.synchronize()
        out[form] = {"u": rows(u, idx_u), "grad_u": rows(g, idx_u).reshape(-1, 3, 3), "dxdt": rows(dx, idx_u),
                     "nu_t": nut[idx_u].double().cpu().numpy(), "dGdt_cv0": rows(dG0, idx_u),
                     "dGdt": rows(dG, idx_r), "dxdt_r": rows(dx, idx_r)}
    return out


def error_report(gpu, ref, idx_u, idx_r):
    rel = lambda a_, b_: float(np.linalg.norm(a_ - b_) / np.linalg.norm(b_))
    rep = {"sample_targets": len(idx_u), "rhs_sample_targets": len(idx_r),
           "rhs_sample": ("all particles" if len(idx_r) > 32 else
                          f"{len(idx_r)} particles in runs of 16 consecutive ones (shared exchange neighbourhoods)"),
           "tolerance": TOL}
    for form in ("compensated", "plain"):
        g = gpu[form]
        rep[form] = {"u": rel(g["u"], ref["u"]), "grad_u": rel(g["grad_u"], ref["grad_u"]),
                     "dxdt": rel(g["dxdt"], ref["dxdt"]), "nu_t": rel(g["nu_t"], ref["nu_t"]),
                     "dGdt_cv0": rel(g["dGdt_cv0"], ref["dGdt_cv0"]), "dGdt": rel(g["dGdt"], ref["dGdt"])}
    rep["keys"] = ("u, grad_u, dxdt, nu_t, dGdt_cv0 (stretching + exchange at nu, c_V = 0) on sample_targets random "
                   "particles; dGdt (the full right-hand side with the Vreman exchange coupling) on "
                   "rhs_sample_targets")
    return rep


def roofline(tr, n, m, sms, clk):
    from paper_2511_11430_gb300 import _lib

    sm_max = 2070.0
    peak = sms * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 lanes x FFMA x max SM clock, TFLOP/s
    nl, sms_ms = tr[_lib.VPM_TRACE_SWEEP]
    avg_ms = sms_ms / max(nl, 1)
    ns_, seg_ms = tr.get(_lib.VPM_TRACE_SEGMENTS, (0, 0.0))
    # a small problem sweeps its segment tiles in the particle launch (no segment launch)
    flops_launch = FLOPS_P2P * n * (n - 1) + (FLOPS_SEG * n * m if not ns_ else 0)
    achieved = flops_launch / (avg_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": sweep_traffic(n, m), "kernel": "sweep_kernel<grad, compensated, stretch, particle tiles>",
            "launches": nl, "avg_launch_ms": avg_ms, "flops_per_launch": flops_launch,
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 (FFMA) x {sm_max:.0f} MHz max SM clock (derived)"}
    if ns_ and m:
        seg_avg = seg_ms / ns_
        seg_t = FLOPS_SEG * n * m / (seg_avg * 1e-3) / 1e12
        roof["segment_launch"] = {"kernel": "sweep_kernel<grad, compensated, stretch, segment tiles>",
                                  "launches": ns_, "avg_launch_ms": seg_avg, "flops_per_launch": FLOPS_SEG * n * m,
                                  "achieved": seg_t, "frac": seg_t / peak}
    if clk and clk.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / (sms * 128 * 2 * clk["sm_mhz"] * 1e6 / 1e12)
    return roof


def extras(hp, args, flush, rank):
    """Informative figures outside the timed step: the particle and segment parts of the
    sweep alone, the treecode on the 1M BVI wake, the wake conversion, and (when the
    main workload is another one) the hover wake's step rate."""
    import torch

    from paper_2511_11430_gb300 import api, synth

    out = {}
    dev = hp.dev
    s = torch.cuda.current_stream()

    def ms_of(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            fn()
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    w = hp.w
    n, m = w.n, w.m
    try:
        P, S = hp.T(w.pos), hp.T(w.strength)
        sa, sb = hp.T(w.seg_a), hp.T(w.seg_b)
        pws = api.Workspace(dev)
        reps = 1 if n >= 1_000_000 else 3
        p_ms = ms_of(lambda: api.induce(P, S, P, w.sigma, compensated=True, ws=pws), reps)
        pp_ms = ms_of(lambda: api.induce(P, S, P, w.sigma, compensated=False, ws=pws), reps)
        from paper_2511_11430_gb300 import _lib

        api.trace_reset()
        api.trace_enable(True)
        s_ms = ms_of(lambda: api.segments_induce(sa, sb, P, w.seg_core, 2, compensated=True, ws=pws), 3)
        nls, tls = api.trace_read(_lib.VPM_TRACE_SEGMENTS)
        api.trace_enable(False)
        pp, sp_ = n * (n - 1), n * m
        out["sweep_parts"] = {
            "p2p": {"pairs": pp, "ms": p_ms, "pairs_per_s": pp / (p_ms * 1e-3),
                    "tflops": pp * FLOPS_P2P / (p_ms * 1e-3) / 1e12},
            "p2p_plain": {"pairs": pp, "ms": pp_ms, "pairs_per_s": pp / (pp_ms * 1e-3),
                          "tflops": pp * FLOPS_P2P / (pp_ms * 1e-3) / 1e12},
            "segments": {"pairs": sp_, "ms": s_ms, "pairs_per_s": sp_ / (s_ms * 1e-3),
                         "tflops": sp_ * FLOPS_SEG / (s_ms * 1e-3) / 1e12,
                         "launch_ms": tls / max(nls, 1),
                         "launch_tflops": sp_ * FLOPS_SEG / (tls / max(nls, 1) * 1e-3) / 1e12 if nls else None},
            "note": "vpm_induce (particles onto themselves) and vpm_segments_induce (segments onto the particles) "
                    "alone, u + grad u; includes each call's packing and epilogue"}
        del P, S, pws
    except Exception as ex:  # informative, never fatal
        out["sweep_parts"] = {"unavailable": str(ex)[:200]}

    if args.config != 2:
        try:
            h2 = HotPath(synth.make(2), dev)
            tot, tr2 = timed_loop(h2, h2.params(True), max(args.steps, 6), max(args.warmup, 3), flush, None, True)
            k2 = max(args.steps, 6)
            from paper_2511_11430_gb300 import _lib

            nl, sw = tr2[_lib.VPM_TRACE_SWEEP]
            out["hover4_100k"] = {"value": h2.n * (h2.n - 1) * k2 / (tot * 1e-3), "unit": UNIT, "steps": k2,
                                  "ms_per_step": tot / k2, "sweep_launch_ms": sw / max(nl, 1),
                                  "workload": workload_desc(h2.w)}
        except Exception as ex:
            out["hover4_100k"] = {"unavailable": str(ex)[:200]}

    try:
        wt = synth.make(3)
        Pt = torch.from_numpy(wt.pos).to(dev)
        St = torch.from_numpy(wt.strength).to(dev)
        tws = api.Workspace(dev)
        tms = ms_of(lambda: api.tree_induce(Pt, St, wt.sigma, theta=0.5, order=4, ws=tws), 3)
        prm_t = api.Params(sigma=wt.sigma, nu=wt.nu, c_v=wt.c_v, seg_core=wt.seg_core, u_inf=wt.u_inf,
                           compensated=False)
        At, Bt = torch.from_numpy(wt.seg_a).to(dev), torch.from_numpy(wt.seg_b).to(dev)
        rms = ms_of(lambda: api.rhs_tree(Pt, St, At, Bt, prm_t, theta=0.5, order=4, ws=tws), 2)
        out["treecode"] = {"particles": wt.n, "theta": 0.5, "order": 4, "ms": tms, "rhs_ms": rms,
                           "note": "O(n log n) variant on the 1M BVI wake (informative)"}
        del Pt, St, At, Bt, tws
    except Exception as ex:
        out["treecode"] = {"unavailable": str(ex)[:200]}

    try:
        ea, eb, eg, egn, ehn, etr, ds_tip = synth.rotor_wake_edges(5, 2000)
        Td = lambda a_, dt_: torch.from_numpy(np.ascontiguousarray(a_)).to(dt_).to(dev)
        wa, wb, wg, wgn = (Td(q, torch.float64) for q in (ea, eb, eg, egn))
        whn, wtr = Td(ehn, torch.int32), Td(etr, torch.int32)
        wws = api.Workspace(dev)
        xw, _ = api.wake_convert(wa, wb, wg, wtr, ds_tip, 4, 1, gamma_nb=wgn, has_nb=whn, ws=wws)
        npart = int(xw.shape[1])
        wms = ms_of(lambda: api.wake_convert(wa, wb, wg, wtr, ds_tip, 4, 1, gamma_nb=wgn, has_nb=whn,
                                             capacity=npart, ws=wws), 5)
        m_e = len(ea)
        algo = 72 * m_e + 16 * m_e + 48 * npart
        out["wake_convert"] = {"edges": m_e, "particles": npart, "ms": wms, "particles_per_s": npart / (wms * 1e-3),
                               "algorithmic_bytes": algo, "achieved_gbs": algo / (wms * 1e-3) / 1e9,
                               "note": "device time of one vpm_wake_convert call incl. its one host sync"}
    except Exception as ex:
        out["wake_convert"] = {"unavailable": str(ex)[:200]}
    return out


def run_ours(args):
    import torch

    ws_n, rank, local = dist_info()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if ws_n > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    from paper_2511_11430_gb300 import _lib, api, build, synth

    build.build()
    w = synth.make(args.config) if args.particles is None else synth.make(args.config, n=args.particles)
    hp = HotPath(w, dev)
    n, m, K = w.n, w.m, w.n_ctrl
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    pairs_step = n * (n - 1)
    side = max(3, args.steps // 6)  # steps of the plain and end-to-end legs

    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    total_ms, tr = timed_loop(hp, hp.params(True), args.steps, args.warmup, flush, dist, trace=True)
    clk = clocks.stop() if clocks else None
    total_ms = max_over_ranks(dist, total_ms, dev)
    value = whole_job_rate(ws_n, pairs_step, args.steps, total_ms)

    plain = None
    if not args.no_plain:
        pm, _ = timed_loop(hp, hp.params(False), side, 1, flush, dist)
        pm = max_over_ranks(dist, pm, dev)
        plain = {"value": whole_job_rate(ws_n, pairs_step, side, pm), "unit": UNIT, "steps": side,
                 "ms_per_step": pm / side, "dtype": "f32 (plain accumulation)"}

    e2e = None
    if not args.no_e2e:
        em, h2d, d2h = e2e_loop(hp, hp.params(True), side, 1, flush, dist)
        em = max_over_ranks(dist, em, dev)
        e2e = {"value": whole_job_rate(ws_n, pairs_step, side, em), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": side, "ms_per_step": em / side,
               "note": "per step: L2 flush outside the events; H2D of the inputs, the step, D2H of the results "
                       "inside them (as the device-timed loop)"}

    props = torch.cuda.get_device_properties(dev)
    roof = roofline(tr, n, m, props.multi_processor_count, clk)

    err = {"unavailable": "the FP64 reference values come from the cpu_baseline leg (skipped)"}
    cpu = None
    ext = {}
    if rank == 0:
        with_ref = ws_n == 1 and not args.no_cpu_baseline
        idx_u, idx_r = error_samples(w, args.error_targets)
        gpu_vals = None
        if with_ref:  # the GPU side of the error report (its reference comes from the oracle leg)
            try:
                gpu_vals = gpu_error_values(hp, idx_u, idx_r)
            except Exception as ex:  # the error report is informative, never fatal
                gpu_vals = str(ex)[:200]
        if not args.no_extras:
            ext = extras(hp, args, flush, rank)
        if with_ref:
            try:
                ref, cpu = oracle_reference(w, idx_u, idx_r, host_cores())
                err = (error_report(gpu_vals, ref, idx_u, idx_r) if isinstance(gpu_vals, dict)
                       else {"unavailable": gpu_vals})
            except Exception as ex:
                err = {"unavailable": str(ex)[:200]}

    if dist is not None:
        dist.barrier()
    if rank == 0:
        launches_total = tr[_lib.VPM_TRACE_ALL][0]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_n, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(w), "particles": n, "segments": m, "control_points": K,
                       "pairs_per_step": pairs_step, "segment_pairs_per_step": n * m,
                       "step": "one RK3 stage of the particles with the AIC solve, control-point velocity and "
                               "adjoint (stages cycle 0, 1, 2)",
                       "precision": "compensated FP32 pair sums, FP64 state/refinement",
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MB write)",
                       "parallelism": "replicas" if ws_n > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches_total),
            "clocks": clk, "plain": plain, "error": err,
            "kernel_ms": {"sweep_grad": list(tr[_lib.VPM_TRACE_SWEEP]), "adjoint": list(tr[_lib.VPM_TRACE_ADJOINT]),
                          "pse": list(tr[_lib.VPM_TRACE_PSE]), "sweep_vel": list(tr[_lib.VPM_TRACE_SWEEP_VEL]),
                          "segments": list(tr[_lib.VPM_TRACE_SEGMENTS])},
        }
        line.update(ext)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.part == "rotor":
        run_rotor(args)
    elif args.part is not None:
        run_part(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
