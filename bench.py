#!/usr/bin/env python3
"""Throughput of the vortex-particle hot path on GB300.

One step = one pass of the whole hot path over the 4-blade hover wake
(100,000 particles, 5,120 blade segments, 1,280 control points, sigma = 0.01 R):
  pack the FP64 state to FP32, induced velocity at the control points, AIC build
  and FP32-LU/FP64-refined solve, one low-storage RK3 step (three right-hand
  sides, each a particle + segment u + grad u sweep, Vreman, stretching, PSE,
  stage update), and the adjoint of the downwash loss at the control points.
Metric: particle-particle u + grad u pair interactions per second (3 N (N - 1) per
step), compensated FP32.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
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
# DRAM bytes (read + write) of one sweep_kernel<grad, compensated, stretch> launch on the
# hover wake (100,000 particles, 5,120 segments), from one ncu capture of that launch
# (profiles/sweep_kernel_hover4_100k.md); valid only while the kernel's sources hash to
# SWEEP_SRC_SHA256, else the bench reports traffic null.
SWEEP_TRAFFIC_BYTES = 11_791_872 + 3_584
SWEEP_SRC_SHA256 = "8310509dd5e9d952b30014f01a599cda4f59934a5e8bc295c4982abcda745572"
SWEEP_SRC = ["paper_2511_11430_gb300/csrc/vpm_sweep.cu", "paper_2511_11430_gb300/csrc/vpm_kernel.cuh",
             "paper_2511_11430_gb300/csrc/vpm_common.cuh"]


def sweep_traffic(n, m):
    """The captured DRAM traffic of the sweep launch, if the capture matches the sources
    and the workload (hover, 100,000 particles, 5,120 segments)."""
    import hashlib

    h = hashlib.sha256()
    root = os.path.dirname(os.path.abspath(__file__))
    for f in SWEEP_SRC:
        with open(os.path.join(root, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != SWEEP_SRC_SHA256 or n != 100_000 or m != 5_120:
        return None
    return SWEEP_TRAFFIC_BYTES


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--particles", type=int, default=None, help="override the particle count (testing only)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=None,
                    help="seconds of oracle work per CPU-baseline sample (default 12; reference arm: 60 s over all steps)")
    ap.add_argument("--no-tree", action="store_true", help="skip the informative treecode timing")
    ap.add_argument("--part", choices=["aic", "wake", "tree", "rotor"], default=None,
                    help="time one component alone (for profiling; prints a text line, not the JSON contract)")
    return ap.parse_args()


def run_rotor(args):
    """The AH-1G rotor in forward flight (Eq. 12 pitch and flapping, advance ratio 0.19)
    through the near-wake driver: shedding, conversion, RK3 particles, AIC and loads each
    step, for --steps revolutions at 10 deg per step (after --warmup revolutions, whose
    loads are reported too).  Prints the thrust and torque coefficients averaged per
    revolution, the particle count and the wall time per step."""
    import time

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
    hover blade lattice, the conversion of 2,000 hover wake rows, or the treecode
    (theta 0.5, order 4) on the 1,000,000-particle BVI wake (--particles to shrink it)."""
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
    return (f"{w.name}: {w.meta.get('blades')}-blade rotor wake, {w.n:,} Gaussian particles (sigma {w.sigma:g} R), "
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
# the FP64 oracle on the host cores (CPU baseline and reference arm)
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


def oracle_values(w, idx):
    """The FP64 oracle's u and grad u at the sampled particles idx (cpu_baseline leg)."""
    import oracle

    return oracle.p2p(w.pos, w.strength, w.pos[idx], w.sigma)


def oracle_threads_default(cores):
    import oracle

    oracle.set_threads(cores)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


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
def run_ours(args):
    import torch

    from paper_2511_11430_gb300 import _lib, api, build, synth

    ws_n, rank, local = dist_info()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if ws_n > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    build.build()
    w = synth.make(args.config) if args.particles is None else synth.make(args.config, n=args.particles)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    n, m, K = w.n, w.m, w.n_ctrl
    x0 = np.ascontiguousarray(w.pos[:, :3].astype(np.float64).T)
    G0 = np.ascontiguousarray(w.strength[:, :3].astype(np.float64).T)
    vol = T(w.pos[:, 3].copy())
    sa, sb = T(w.seg_a), T(w.seg_b)
    rings, colloc, normal, vrel = T(w.rings), T(w.colloc), T(w.normal), T(w.v_rel)
    nrm = normal[:, :3].t().contiguous()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def make_state():
        return T(x0), T(G0)

    def hot_path_step(state, prm, wsb):
        x, G = state
        pos, strn = api.pack_state(x, G, vol, wsb["pos"], wsb["str"])
        u_c = api.induce(pos, strn, colloc, w.sigma, compensated=prm.compensated, grad=False, ws=wsb["ws"])
        A, b = api.aic_build(rings, colloc, normal, w.seg_core, 2, v_rel=vrel, w_ind=u_c)
        gam, it, be = api.aic_solve(A, b, tol=1e-12, max_iter=30, ws=wsb["ws"])
        api.step(x, G, vol, sa, sb, prm, w.dt, ws=wsb["ws"])
        g = 2.0 * (u_c * nrm).sum(0, keepdim=True) * nrm  # d/du of sum_k (u_k . n_k)^2
        dx, dG = api.induce_backward(pos, strn, colloc, w.sigma, g.contiguous(), compensated=prm.compensated,
                                     ws=wsb["ws"])
        return gam, dx, dG

    def new_bufs():
        return {"ws": api.Workspace(dev), "pos": torch.empty((n, 4), dtype=torch.float32, device=dev),
                "str": torch.empty((n, 4), dtype=torch.float32, device=dev)}

    def timed(prm, steps, warmup, trace=False):
        state = make_state()
        bufs = new_bufs()
        for _ in range(warmup):
            hot_path_step(state, prm, bufs)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        if trace:
            api.trace_enable(True)
            api.trace_reset()
        st = torch.cuda.current_stream()
        total = 0.0
        for _ in range(steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            hot_path_step(state, prm, bufs)
            e1.record(st)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        tr = None
        if trace:
            tr = {k: api.trace_read(k) for k in (_lib.VPM_TRACE_ALL, _lib.VPM_TRACE_SWEEP, _lib.VPM_TRACE_ADJOINT,
                                                 _lib.VPM_TRACE_PSE, _lib.VPM_TRACE_SWEEP_VEL)}
            api.trace_enable(False)
        return max_over_ranks(dist, total, dev), tr

    prm_c = api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core, u_inf=w.u_inf, compensated=True)
    prm_p = api.Params(sigma=w.sigma, nu=w.nu, c_v=w.c_v, seg_core=w.seg_core, u_inf=w.u_inf, compensated=False)
    pairs_step = 3 * n * (n - 1)
    seg_pairs_step = 3 * n * m

    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    total_ms, tr = timed(prm_c, args.steps, args.warmup, trace=True)
    clk = clocks.stop() if clocks else None
    ms_step = total_ms / args.steps
    value = whole_job_rate(ws_n, pairs_step, args.steps, total_ms)

    plain = None
    if not args.no_plain:
        pm, _ = timed(prm_p, max(3, args.steps // 2), 1)
        plain = {"value": whole_job_rate(ws_n, pairs_step, max(3, args.steps // 2), pm), "unit": UNIT,
                 "ms_per_step": pm / max(3, args.steps // 2), "dtype": "f32 (plain accumulation)"}

    # roofline of the dominant kernel: the particle + segment u + grad u sweep
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = 2070.0
    peak = sms * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 lanes x FFMA x max SM clock, TFLOP/s
    nl, sms_ms = tr[_lib.VPM_TRACE_SWEEP]
    avg_ms = sms_ms / max(nl, 1)
    flops_launch = FLOPS_P2P * n * (n - 1) + FLOPS_SEG * n * m
    achieved = flops_launch / (avg_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": sweep_traffic(n, m), "kernel": "sweep_kernel<grad, compensated>", "launches": nl,
            "avg_launch_ms": avg_ms, "flops_per_launch": flops_launch,
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 (FFMA) x {sm_max:.0f} MHz (fallback-free derivation)"}
    if clk and clk.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / (sms * 128 * 2 * clk["sm_mhz"] * 1e6 / 1e12)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x0).pin_memory()
        Gh = torch.from_numpy(G0).pin_memory()
        xo = torch.empty_like(xh).pin_memory()
        Go = torch.empty_like(Gh).pin_memory()
        gho = torch.empty((K,), dtype=torch.float64).pin_memory()
        dxo = torch.empty((3, n), dtype=torch.float32).pin_memory()
        dGo = torch.empty((3, n), dtype=torch.float32).pin_memory()
        volh = torch.from_numpy(w.pos[:, 3].copy()).pin_memory()
        host_in = [torch.from_numpy(a).pin_memory() for a in (w.seg_a, w.seg_b, w.rings, w.colloc, w.normal,
                                                              w.v_rel)]
        bufs = new_bufs()
        x_d, G_d = torch.empty_like(xh, device=dev), torch.empty_like(Gh, device=dev)
        dev_in = [torch.empty_like(h, device=dev) for h in host_in]
        vol_d = torch.empty_like(volh, device=dev)

        def e2e_step():
            x_d.copy_(xh, non_blocking=True)
            G_d.copy_(Gh, non_blocking=True)
            vol_d.copy_(volh, non_blocking=True)
            for d_, h_ in zip(dev_in, host_in):
                d_.copy_(h_, non_blocking=True)
            gam, dx, dG = hot_path_step((x_d, G_d), prm_c, bufs)
            xo.copy_(x_d, non_blocking=True)
            Go.copy_(G_d, non_blocking=True)
            gho.copy_(gam, non_blocking=True)
            dxo.copy_(dx, non_blocking=True)
            dGo.copy_(dG, non_blocking=True)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ksteps = max(2, args.steps // 2)
        e0.record(st)
        for _ in range(ksteps):
            e2e_step()
        e1.record(st)
        e1.synchronize()
        e2e_ms = max_over_ranks(dist, e0.elapsed_time(e1), dev)
        h2d = (xh.numel() + Gh.numel()) * 8 + volh.numel() * 4 + sum(h.numel() * 4 for h in host_in)
        d2h = (xo.numel() + Go.numel() + gho.numel()) * 8 + (dxo.numel() + dGo.numel()) * 4
        e2e = {"value": whole_job_rate(ws_n, pairs_step, ksteps, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": e2e_ms / ksteps}

    # error at the stated tolerance, on a sample (outside every timed region): the GPU
    # side here, the FP64 reference values in the cpu_baseline leg below
    err_gpu = None
    err_idx = synth.sample_targets(11, n, 96)
    if rank == 0:
        try:
            pos, strn = api.pack_state(*make_state(), vol)
            u, gr = api.induce(pos, strn, pos, w.sigma, compensated=True)
            up, gp = api.induce(pos, strn, pos, w.sigma, compensated=False)
            U = lambda t: t[:, err_idx].double().cpu().numpy().T
            Jm = lambda t: t[:, err_idx].double().cpu().numpy().T.reshape(-1, 3, 3)
            err_gpu = (U(u), Jm(gr), U(up), Jm(gp))
        except Exception as ex:  # the error report is informative, never fatal
            err_gpu = str(ex)[:200]

    # the wake panel -> particle conversion (Eq. 6-8), outside the timed step: the edges of
    # 2,000 wake panel rows of the 4-blade hover rotor, n_tip = 4 (informative)
    wake = None
    if rank == 0:
        try:
            ea, eb, eg, egn, ehn, etr, ds_tip = synth.rotor_wake_edges(5, 2000)
            Td = lambda a_, dt_: torch.from_numpy(np.ascontiguousarray(a_)).to(dt_).to(dev)
            wa, wb, wg, wgn = (Td(q, torch.float64) for q in (ea, eb, eg, egn))
            whn, wtr = Td(ehn, torch.int32), Td(etr, torch.int32)
            wws = api.Workspace(dev)
            xw, Gw = api.wake_convert(wa, wb, wg, wtr, ds_tip, 4, 1, gamma_nb=wgn, has_nb=whn, ws=wws)
            npart = int(xw.shape[1])
            reps = 5
            torch.cuda.synchronize()
            st = torch.cuda.current_stream()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                api.wake_convert(wa, wb, wg, wtr, ds_tip, 4, 1, gamma_nb=wgn, has_nb=whn, capacity=npart, ws=wws)
            e1.record(st)
            e1.synchronize()
            wms = e0.elapsed_time(e1) / reps
            m_e = len(ea)
            algo = 72 * m_e + 16 * m_e + 48 * npart  # edges in, counts/offsets out, particles out
            wake = {"edges": m_e, "particles": npart, "ms": wms, "particles_per_s": npart / (wms * 1e-3),
                    "algorithmic_bytes": algo, "achieved_gbs": algo / (wms * 1e-3) / 1e9,
                    "note": "device time of one vpm_wake_convert call incl. its one host sync"}
        except Exception as ex:  # informative, never fatal
            wake = {"unavailable": str(ex)[:200]}

    # the particle-particle and the segment-particle parts of the right-hand side sweep,
    # each alone (compensated, with the gradient), so that the two pair rates are reported
    # apart (informative, outside the timed step)
    parts = None
    if rank == 0:
        try:
            pos, strn = api.pack_state(*make_state(), vol)
            pws = api.Workspace(dev)
            st = torch.cuda.current_stream()

            def sweep_ms(fn, reps=3):
                fn()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for _ in range(reps):
                    fn()
                e1.record(st)
                e1.synchronize()
                return e0.elapsed_time(e1) / reps

            p_ms = sweep_ms(lambda: api.induce(pos, strn, pos, w.sigma, compensated=True, ws=pws))
            s_ms = sweep_ms(lambda: api.segments_induce(sa, sb, pos, w.seg_core, 2, compensated=True, ws=pws))
            pp, sp_ = n * (n - 1), n * m
            parts = {
                "p2p": {"pairs": pp, "ms": p_ms, "pairs_per_s": pp / (p_ms * 1e-3),
                        "tflops": pp * FLOPS_P2P / (p_ms * 1e-3) / 1e12},
                "segments": {"pairs": sp_, "ms": s_ms, "pairs_per_s": sp_ / (s_ms * 1e-3),
                             "tflops": sp_ * FLOPS_SEG / (s_ms * 1e-3) / 1e12},
                "note": "vpm_induce (particles onto themselves) and vpm_segments_induce (segments onto the "
                        "particles) alone, compensated, u + grad u; includes each call's packing and epilogue",
            }
        except Exception as ex:  # informative, never fatal
            parts = {"unavailable": str(ex)[:200]}

    # the treecode (the O(n log n) variant, outside the timed step) on the 1,000,000-particle
    # BVI wake against the direct plain sum of the same wake (informative)
    tree = None
    wt = tree_idx = tree_gpu = None
    if rank == 0 and not args.no_tree:
        try:
            wt = synth.make(3)
            Pt = torch.from_numpy(wt.pos).to(dev)
            St = torch.from_numpy(wt.strength).to(dev)
            tws = api.Workspace(dev)
            st = torch.cuda.current_stream()

            def timed(fn, reps):
                fn()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for _ in range(reps):
                    fn()
                e1.record(st)
                e1.synchronize()
                return e0.elapsed_time(e1) / reps

            out = {}
            tms = timed(lambda: out.__setitem__("t", api.tree_induce(Pt, St, wt.sigma, theta=0.5, order=4, ws=tws)), 3)
            dms = timed(lambda: api.induce(Pt, St, Pt, wt.sigma, compensated=False, ws=tws), 1)
            # the whole right-hand side (segments, Vreman, stretching, PSE) with the treecode
            # against the direct one
            prm_t = api.Params(sigma=wt.sigma, nu=wt.nu, c_v=wt.c_v, seg_core=wt.seg_core, u_inf=wt.u_inf,
                               compensated=False)
            At = torch.from_numpy(wt.seg_a).to(dev)
            Bt = torch.from_numpy(wt.seg_b).to(dev)
            rms = timed(lambda: api.rhs_tree(Pt, St, At, Bt, prm_t, theta=0.5, order=4, ws=tws), 2)
            rdms = timed(lambda: api.rhs(Pt, St, At, Bt, prm_t, ws=tws), 1)
            ut, gt = out["t"]
            tree_idx = synth.sample_targets(11, wt.n, 32)
            tree_gpu = (ut.cpu().numpy().T[tree_idx].astype(np.float64),
                        gt.cpu().numpy().T[tree_idx].reshape(-1, 3, 3).astype(np.float64))
            tree = {"particles": wt.n, "theta": 0.5, "order": 4, "ms": tms, "direct_plain_ms": dms,
                    "speedup": dms / tms, "rhs_ms": rms, "rhs_direct_plain_ms": rdms}
            del Pt, St, At, Bt, tws, out, ut, gt
        except Exception as ex:  # informative, never fatal
            tree = {"unavailable": str(ex)[:200]}

    # the cpu_baseline leg: the FP64 oracle on the host cores, timed, and the same oracle's
    # values at the sampled targets of the error reports (the only place the main arm
    # runs it)
    cpu = None
    err = {"unavailable": "the FP64 reference values come from the cpu_baseline leg (skipped)"}
    rel = lambda a_, b_: float(np.linalg.norm(a_ - b_) / np.linalg.norm(b_))
    if rank == 0 and ws_n == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        rate, k, dt = oracle_rate(w, 12.0 if args.cpu_seconds is None else args.cpu_seconds, cores)
        rate1, k1, dt1 = oracle_rate(w, 3.0, 1)
        oracle_threads_default(cores)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{k} sampled targets x all {n:,} sources, P2P u + grad u in FP64 ({dt:.1f} s)",
               "single_thread": {"value": rate1, "unit": UNIT,
                                 "sample": f"{k1} sampled targets x all {n:,} sources ({dt1:.1f} s)"}}
        try:
            ru, rJ = oracle_values(w, err_idx)
            if isinstance(err_gpu, tuple):
                cu, cg, pu, pg = err_gpu
                err = {"sample_targets": len(err_idx), "compensated": {"u": rel(cu, ru), "grad_u": rel(cg, rJ)},
                       "plain": {"u": rel(pu, ru), "grad_u": rel(pg, rJ)},
                       "tolerance": {"compensated": 2e-6, "plain": 1e-4}}
            else:
                err = {"unavailable": str(err_gpu)}
            if tree_gpu is not None and "unavailable" not in tree:
                tu, tJ = oracle_values(wt, tree_idx)
                tree["error_vs_oracle"] = {"sample_targets": len(tree_idx), "u": rel(tree_gpu[0], tu),
                                           "grad_u": rel(tree_gpu[1], tJ)}
        except Exception as ex:  # informative, never fatal
            err = {"unavailable": str(ex)[:200]}

    if dist is not None:
        dist.barrier()
    if rank == 0:
        launches_total = tr[_lib.VPM_TRACE_ALL][0]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_n, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(w), "particles": n, "segments": m, "control_points": K,
                       "pairs_per_step": pairs_step, "segment_pairs_per_step": seg_pairs_step,
                       "precision": "compensated FP32 pair sums, FP64 state/refinement",
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MB write)",
                       "parallelism": "replicas" if ws_n > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches_total),
            "clocks": clk, "plain": plain, "error": err, "wake_convert": wake, "sweep_parts": parts, "treecode": tree,
            "kernel_ms": {"sweep_grad": [nl, sms_ms], "adjoint": list(tr[_lib.VPM_TRACE_ADJOINT]),
                          "pse": list(tr[_lib.VPM_TRACE_PSE]), "sweep_vel": list(tr[_lib.VPM_TRACE_SWEEP_VEL])},
        }
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
