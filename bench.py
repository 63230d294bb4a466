#!/usr/bin/env python3
"""Throughput benchmark of the discrete-PML RK4 step (grid-point updates per second).

One "step" = one RK4 step of the whole periodic box (interior + layer) of the 2D
workload with an 8192^2 physical domain and a 32-cell quadratic layer on every side
(T = 8256^2 vertices), 16 seeded Gaussian pulses, dt = 0.5 h.  The headline runs the
FP32 path; FP64 and the adjoint step are reported beside it.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With --gpus N > 1 launch under torchrun: every rank runs an independent replica of the
workload on its own GPU (the method has no exchange step on one box), the timed region
is bracketed by barriers and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "grid-point updates/s (GPts/s) and % HBM roofline, FP32 vs FP64, fwd and adjoint"
UNIT = "GPts/s"
# algorithmic flops of one point-update (one RK4 step of one vertex): 4 stages x (a 5-point
# difference, 6 flop, plus 4 fused stage / accumulate operations, 8 flop)
FLOP_PER_UPDATE_2D = 56
# flops the FP64 interior kernel executes per vertex (the RK4 polynomial in closed form):
# four 5-point differences (5 flop each) and two outputs of four FMAs and an add (9 flop each)
FP64_KERNEL_FLOP_PER_POINT = 38


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measure_fp_peaks(local, target_s=0.15):
    """FP64 and FP32 FMA throughput of this GPU from the library's own kernel
    (pml_fma_peak), with the clocks sampled while it runs."""
    import torch
    from paper_1804_01390_gb300 import _lib
    st = torch.cuda.current_stream().cuda_stream
    out = {}
    clk = ClockSampler(local)
    clk.start()
    for prec in (64, 32):
        iters = 1024
        tf, ms = _lib.pml_fma_peak(prec, st, iters)
        iters = max(1024, int(iters * target_s * 1e3 / max(ms, 1e-3)) // 16 * 16)
        tf, ms = _lib.pml_fma_peak(prec, st, iters)
        out["fp%d_tflops" % prec] = tf
        out["fp%d_ms" % prec] = ms
        out["fp%d_iters" % prec] = iters
    clk.stop()
    out["clocks"] = clk.summary()
    out["method"] = ("pml_fma_peak: 4 x 512 threads per SM, 8 independent FMA chains per thread, one "
                     "timed launch of ~%.0f ms per precision (CUDA events), 2 flop per FMA" % (target_s * 1e3))
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms in the background; start()
    returns once the first sample has arrived, so the samples cover the timed region that
    follows."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.perf_counter()
        while not self.rows and time.perf_counter() - t0 < 3.0:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ------------------------------------------------------------------------------------
# distributed plumbing (replicas)
# ------------------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, device=None):
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------
# measurements
# ------------------------------------------------------------------------------------

def _workload(n=None):
    from paper_1804_01390_gb300 import workloads as wk
    return wk.cfg2() if n is None else wk.cfg2(N=n)


def timed_steps(solver, steps, warmup, ws, profile=False):
    """Device time (ms) of `steps` RK4 steps on the solver's stream, after warm-up."""
    import torch
    from paper_1804_01390_gb300 import _lib
    solver.step(warmup)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    if profile:
        _lib.pml_profile_enable(solver.ctx, 1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(solver.stream)
    solver.step(steps)
    e1.record(solver.stream)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = None
    if profile:
        prof = _lib.pml_profile_read(solver.ctx)
        _lib.pml_profile_enable(solver.ctx, 0)
    return ms, prof


def _errs(got, want, scale_peak=None, scale_l2=None):
    import numpy as np
    d = got - want
    peak = float(np.abs(want).max()) if scale_peak is None else scale_peak
    nrm = float(np.linalg.norm(want)) if scale_l2 is None else scale_l2
    mx = float(np.abs(d).max())
    return {"max_abs": mx, "max_abs_rel_peak": mx / peak if peak > 0 else None,
            "rel_l2": float(np.linalg.norm(d)) / nrm if nrm > 0 else None}


def accuracy_section(wl, u0, variant, one_step, dev, steps=100):
    """FP32 against FP64 on the headline workload after `steps` steps (the FP64 path is the
    one the oracle pins element by element in the parity tests), and the truncation error of
    32- and 64-cell layers against a 1024^2 box whose boundary is never reached (128^2
    window, 1000 steps; the paper's check of the layer, Sec. 1.1.4), in both precisions."""
    import numpy as np
    import torch
    from paper_1804_01390_gb300 import autotune
    from paper_1804_01390_gb300 import workloads as wk
    from paper_1804_01390_gb300.solver import PMLSolver
    res = {}
    fields = {}
    for prec in (64, 32):
        s = PMLSolver(wl.N, wl.w, dt=wl.dt, precision=prec, device=dev)
        if prec == 32:
            autotune.select(s.ctx, variant, one_step)
        s.set_initial(torch.from_numpy(u0.astype(np.float64 if prec == 64 else np.float32)).to(dev))
        s.step(steps)
        fields[prec] = [s.read(f).double().cpu().numpy() for f in (0, 1)]
        s.close()
        del s
        torch.cuda.empty_cache()
    res["fp32_vs_fp64"] = {"steps": steps, "workload": "headline workload, the FP32 kernel shape of the headline",
                           "U": _errs(fields[32][0], fields[64][0]), "V": _errs(fields[32][1], fields[64][1])}
    del fields

    def window_u(wlx, prec, M=None, n=1000):
        if M is None:
            s = PMLSolver(wlx.N, wlx.w, dt=wlx.dt, precision=prec, device=dev)
            s.set_initial(torch.from_numpy(wk.initial_field(wlx)).to(dev))
            lo = (wlx.w, wlx.w)
        else:
            big, offs = wk.reference_box(wlx, M)
            s = PMLSolver(big.N, 0, dt=wlx.dt, precision=prec, device=dev)
            s.set_initial(torch.from_numpy(wk.reference_initial_field(wlx, M)).to(dev))
            lo = offs
        s.step(n)
        u = s.read(0).double().cpu().numpy()[lo[1]:lo[1] + wlx.N[1], lo[0]:lo[0] + wlx.N[0]]
        s.close()
        return u

    ref_wl = wk.cfg1(w=64)
    b64 = window_u(ref_wl, 64, M=1024)
    u_init = wk.initial_field(ref_wl)
    peak0, n0 = float(np.abs(u_init).max()), float(np.linalg.norm(u_init))
    trunc = {"reference": "1024^2 box without layer, FP64, same masked initial data, 1000 steps; errors "
                          "relative to the initial field's peak and norm",
             "fp32_floor": _errs(window_u(ref_wl, 32, M=1024), b64, peak0, n0)}
    for w in (16, 32, 64):
        wlx = wk.cfg1(w=w)
        trunc["w%d" % w] = {"fp64": _errs(window_u(wlx, 64), b64, peak0, n0),
                            "fp32": _errs(window_u(wlx, 32), b64, peak0, n0)}
    res["truncation_vs_big_domain"] = trunc
    return res


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch
    from paper_1804_01390_gb300 import workloads as wk
    from paper_1804_01390_gb300.solver import PMLSolver

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = _workload(args.n)
    pts = wl.points
    u0 = wk.initial_field(wl, dtype=np.float32)
    K, W = args.steps, args.warmup
    hbm_peak, peak_kind = _peaks()
    # bytes one point-update must move (each step reads and writes U, V once, plus
    # Phi_a, Psi_a on their 2w - 1 active cells per axis): 4 + 4 sum_a (2w - 1) / T_a words
    words_per_update = 4.0 + 4.0 * sum((2 * wl.w - 1) / t for t in wl.T)

    def step_roofline(gpts, esz):
        b = words_per_update * esz
        return {"bytes_per_update": b, "achieved_gbs": gpts * b, "peak": hbm_peak, "unit": "GB/s",
                "frac": gpts * b / hbm_peak, "peak_kind": peak_kind,
                "definition": "point-updates/s x algorithmic bytes per point-update / measured copy bandwidth"}

    # ---- FP32 headline: inputs resident in HBM ------------------------------------
    from paper_1804_01390_gb300 import autotune
    s = PMLSolver(wl.N, wl.w, dt=wl.dt, precision=32, device=dev)
    u_dev = torch.from_numpy(u0).to(dev)
    s.set_initial(u_dev)
    if args.variant is None:
        variant, tune_table = autotune.tune(s, steps=20, use_cache=not args.retune)
        one_step = s.one_step_variant
    else:   # a fixed variant (profiling): no tuning launches
        variant, tune_table, one_step = args.variant, None, None
        autotune.select(s.ctx, variant)
    from paper_1804_01390_gb300 import _lib as _l
    tb = _l.pml_get_time_block(s.ctx)
    s.set_initial(u_dev)
    clk = ClockSampler(local)
    clk.start()
    # headline: no events between the kernels (the interior kernel may overlap the layer
    # kernel of the same step); then the same K steps again with every kernel bracketed by
    # events for the per-kernel durations of the roofline
    ms, _ = timed_steps(s, K, W, ws, profile=False)
    clk.stop()
    ms_max = max_over_ranks(ms, ws, dev)
    value = pts * K * ws / (ms_max / 1e3) / 1e9
    ms_prof, prof = timed_steps(s, K, 0, ws, profile=True)
    (ms_k, n_k) = prof
    # vertices one interior launch advances: the layer-free run (n - 2 per axis), shrunk
    # by 2 at both ends for the two-step kernel, which advances them two steps per launch
    interior_pts = int(np.prod([n - 2 - (4 if tb == 2 else 0) for n in wl.N]))
    bytes_per_launch = interior_pts * 4 * 4               # U, V read + written once per launch, FP32
    avg_launch_s = ms_k[0] / max(n_k[0], 1) / 1e3
    achieved = bytes_per_launch / avg_launch_s / 1e9
    # the same launch counted per point-update at the one-step figure (16 B per update)
    effective = bytes_per_launch * tb / avg_launch_s / 1e9
    # DRAM traffic of the dominant kernel from an ncu capture of this very kernel shape
    # (variant 6, k_interior2d_tb2<float, false, 4, 3, 6, 2, 128>) on the 6144^2 case: 335.3 MB
    # read + 256.8 MB written per launch over 6134^2 vertices, scaled by the vertices per launch
    traffic = None
    if tb == 2 and variant == 6:
        traffic = (335.3e6 + 256.8e6) * interior_pts / 6134.0 ** 2
    launches = int(n_k.sum())
    layer_share = float(ms_k[1] / max(ms_k.sum(), 1e-30))

    # ---- FP32 end to end through the C ABI with host buffers ------------------------
    s.close()
    del s
    torch.cuda.synchronize()
    e2e = None
    if not args.no_e2e:
        from paper_1804_01390_gb300 import _lib
        s = PMLSolver(wl.N, wl.w, dt=wl.dt, precision=32, device=dev)
        autotune.select(s.ctx, variant, one_step)
        u_host = torch.from_numpy(u0).pin_memory()
        out_host = torch.empty_like(u_host).pin_memory()
        s.set_initial(u_host)
        s.step(W)
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        _lib.pml_set_initial(s.ctx, u_host.data_ptr(), None, 0)
        _lib.pml_step(s.ctx, K)
        _lib.pml_read_field(s.ctx, 0, out_host.data_ptr(), 0)
        t1 = time.perf_counter()
        barrier(ws)
        e_ms = max_over_ranks((t1 - t0) * 1e3, ws, dev)
        nb = u_host.numel() * 4
        e2e = {"value": pts * K * ws / (e_ms / 1e3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": nb / K,
               "d2h_bytes_per_step": nb / K, "ms": e_ms,
               "how": "pml_set_initial(host pinned U0) + pml_step(K) + pml_read_field(host U), wall clock"}
        s.close()
        del s

    # ---- FP64: the paper's precision, bound by the FP64 pipe ---------------------------
    fp64 = None
    peaks = None
    if not args.no_fp64:
        peaks = measure_fp_peaks(local)
        fp64_peak = peaks["fp64_tflops"]
        K64 = max(K // 10, 10)
        s = PMLSolver(wl.N, wl.w, dt=wl.dt, precision=64, device=dev)
        autotune.tune(s, steps=5, use_cache=not args.retune)
        u64 = u0.astype(np.float64)
        s.set_initial(torch.from_numpy(u64).to(dev))
        clk64 = ClockSampler(local)
        clk64.start()
        ms64, _ = timed_steps(s, K64, min(W, 3), ws, profile=False)
        clk64.stop()
        ms64 = max_over_ranks(ms64, ws, dev)
        v64 = pts * K64 * ws / (ms64 / 1e3) / 1e9
        _, prof64 = timed_steps(s, K64, 0, ws, profile=True)
        m64, n64 = prof64
        t_int = m64[0] / max(n64[0], 1) / 1e3
        int64_pts = int(np.prod([n - 2 for n in wl.N]))
        kernel_tflops = int64_pts * FP64_KERNEL_FLOP_PER_POINT / t_int / 1e12
        step_tflops = v64 / ws * FLOP_PER_UPDATE_2D / 1e3
        # end to end through the C ABI with host buffers, as for the FP32 headline
        e2e64 = None
        if not args.no_e2e:
            from paper_1804_01390_gb300 import _lib
            u_host64 = torch.from_numpy(u64).pin_memory()
            out_host64 = torch.empty_like(u_host64).pin_memory()
            torch.cuda.synchronize()
            barrier(ws)
            t0 = time.perf_counter()
            _lib.pml_set_initial(s.ctx, u_host64.data_ptr(), None, 0)
            _lib.pml_step(s.ctx, K64)
            _lib.pml_read_field(s.ctx, 0, out_host64.data_ptr(), 0)
            t1 = time.perf_counter()
            barrier(ws)
            e_ms64 = max_over_ranks((t1 - t0) * 1e3, ws, dev)
            nb64 = u_host64.numel() * 8
            e2e64 = {"value": pts * K64 * ws / (e_ms64 / 1e3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": nb64 / K64,
                     "d2h_bytes_per_step": nb64 / K64, "ms": e_ms64,
                     "how": "pml_set_initial(host pinned U0) + pml_step(K) + pml_read_field(host U), wall clock"}
        fp64 = {"metric": METRIC, "value": v64, "unit": UNIT, "dtype": "f64", "steps": K64, "warmup": min(W, 3),
                "ms_per_step": ms64 / K64, "workload": "the headline workload in FP64",
                "roofline": {"bound": "alu", "achieved": step_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                             "frac": step_tflops / fp64_peak, "peak_kind": "measured",
                             "peak_method": peaks["method"], "flop_per_update": FLOP_PER_UPDATE_2D,
                             "definition": "point-updates/s x 56 algorithmic flop per point-update / measured "
                                           "FP64 FMA throughput",
                             "traffic": None},
                "kernel_roofline": {"kernel": "k_interior2d<double>", "bound": "alu",
                                    "flop_per_vertex": FP64_KERNEL_FLOP_PER_POINT, "achieved": kernel_tflops,
                                    "peak": fp64_peak, "unit": "TFLOP/s", "frac": kernel_tflops / fp64_peak,
                                    "avg_launch_ms": t_int * 1e3,
                                    "note": "flops the closed-form interior kernel executes per vertex"},
                "hbm_roofline": step_roofline(v64 / ws, 8),
                "e2e": e2e64, "clocks": clk64.summary(),
                "cpu_baseline": "see the top-level cpu_baseline (the FP64 oracle on the same layer)"}
        s.close()
        del s

    # ---- accuracy of the FP32 path: against the FP64 path, and truncation vs a big box ----
    accuracy = None
    if not args.no_accuracy:
        accuracy = accuracy_section(wl, u0, variant, one_step, dev)

    # ---- adjoint (FP32) --------------------------------------------------------------
    adj = None
    if not args.no_adjoint:
        import torch as _t
        from paper_1804_01390_gb300 import _lib
        s = PMLSolver(wl.N, wl.w, dt=wl.dt, precision=32, device=dev, adjoint=True)
        autotune.select(s.ctx, variant, one_step)
        s.set_initial(_t.from_numpy(u0).to(dev))
        s.adjoint_reset()
        Ka = max(K // 2, 10)
        _lib.pml_adjoint_step(s.ctx, min(W, 3), None, None, None)
        _t.cuda.synchronize()
        barrier(ws)
        e0 = _t.cuda.Event(enable_timing=True)
        e1 = _t.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        _lib.pml_adjoint_step(s.ctx, Ka, None, None, None)
        e1.record(s.stream)
        _t.cuda.synchronize()
        barrier(ws)
        msa = max_over_ranks(e0.elapsed_time(e1), ws, dev)
        va = pts * Ka * ws / (msa / 1e3) / 1e9
        adj = {"value": va, "unit": UNIT, "steps": Ka, "ms_per_step": msa / Ka, "dtype": "f32",
               "hbm_roofline": step_roofline(va / ws, 4)}
        s.close()
        del s

    # ---- 3D (512^3 + 24-cell layer, FP32, 8 Ricker sources) ---------------------------
    d3 = None
    if not args.no_3d:
        wl3 = wk.cfg3() if args.n3 is None else wk.cfg3(N=args.n3)
        K3 = max(K // 20, 10)
        s = PMLSolver(wl3.N, wl3.w, dt=wl3.dt, precision=32, device=dev)
        if args.variant3 is None:   # frame kernel: tile kernel, level passes or slab tiles
            var3, tune3 = autotune.tune(s, steps=5, use_cache=not args.retune)
        else:                       # a fixed frame kernel (profiling): no tuning launches
            var3, tune3 = args.variant3, None
            autotune.select(s.ctx, var3)
        u3 = torch.from_numpy(wk.initial_field(wl3, dtype=np.float32)).to(dev)
        s.set_initial(u3)
        src = wl3.sources
        s.set_sources(src["coords"], src["amp"], src["f_peak"], src["t_delay"])
        ms3, _ = timed_steps(s, K3, min(W, 3), ws, profile=False)
        ms3 = max_over_ranks(ms3, ws, dev)
        ms3p, prof3 = timed_steps(s, K3, 0, ws, profile=True)
        m3, n3 = prof3
        pts3 = wl3.points
        int3 = int(np.prod([n - 2 for n in wl3.N]))
        t_int3 = m3[0] / max(n3[0], 1) / 1e3
        ach3 = int3 * 16 / t_int3 / 1e9
        d3 = {"workload": "3D %d^3 interior + %d-cell quadratic PML (T = %d^3), Gaussian s=6 + 8 Ricker sources, FP32"
                          % (wl3.N[0], wl3.w, wl3.T[0]),
              "value": pts3 * K3 * ws / (ms3 / 1e3) / 1e9, "unit": UNIT, "steps": K3, "ms_per_step": ms3 / K3,
              "layer_variant": {0: "z-streaming tile kernel", 1: "level passes", 2: "slab tiles"}.get(var3, var3),
              "autotune_ms_per_step": tune3,
              "roofline": {"bound": "hbm", "kernel": "k_interior3d_rows<float> (FP32 layer-free kernel)", "achieved": ach3, "peak": hbm_peak,
                           "unit": "GB/s", "frac": ach3 / hbm_peak, "avg_launch_ms": t_int3 * 1e3,
                           "bytes_per_launch": int3 * 16},
              "kernel_ms_per_step": {"interior": m3[0] / max(n3[0], 1), "layer": m3[1] / max(n3[0], 1),
                                     "points": m3[2] / max(n3[0], 1)}}
        s.close()
        del s, u3

    # ---- batched: 96 grids of uneven sizes, one launch pair per step, graph replay ------
    d4 = None
    if not args.no_batch:
        from paper_1804_01390_gb300.solver import PMLBatch
        wls = wk.cfg4() if args.n4 is None else wk.cfg4(hi=args.n4, lo=min(256, args.n4))
        K4 = 32 * max(K // 64, 2)
        solvers = []
        for wl4 in wls:
            s4 = PMLSolver(wl4.N, wl4.w, dt=wl4.dt, precision=32, device=dev)
            solvers.append(s4)
        inits4 = [torch.from_numpy(wk.initial_field(wl4, dtype=np.float32)).to(dev) for wl4 in wls]
        for s4, u4 in zip(solvers, inits4):
            s4.set_initial(u4)
        b4 = PMLBatch(solvers)
        var4, tune4 = b4.autotune(32)
        for s4, u4 in zip(solvers, inits4):
            s4.set_initial(u4)
        stream4 = solvers[0].stream
        b4.step(max(W, 3))
        torch.cuda.synchronize()
        barrier(ws)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream4)
        b4.step(K4)
        e1.record(stream4)
        torch.cuda.synchronize()
        barrier(ws)
        ms4 = max_over_ranks(e0.elapsed_time(e1), ws, dev)
        b4.profile(True)
        b4.step(64)
        m4, n4 = b4.profile_read()
        b4.profile(False)
        pts4 = sum(wl4.points for wl4 in wls)
        tb4 = b4.time_block()
        int4 = 0   # vertices one interior launch advances (the run shrunk by 2 for two steps)
        for s4 in solvers:
            runs = []
            for a in range(2):
                r = int(s4.layout(a)[2].sum())
                runs.append(max(r - 4, 0) if (tb4 == 2 and r < s4.T[a]) else r)
            int4 += int(np.prod(runs))
        t_int4 = m4[0] / max(n4[0], 1) / 1e3
        ach4 = int4 * 16 / t_int4 / 1e9
        ngrid, items4, tiles4, ctas4 = b4.info()
        d4 = {"workload": "96 independent 2D grids, sides uniform in [%d, %d], quadratic PML 16..32 cells, "
                          "one Gaussian s=4 each, FP32" % (min(min(w.N) for w in wls), max(max(w.N) for w in wls)),
              "value": pts4 * K4 * ws / (ms4 / 1e3) / 1e9, "unit": UNIT, "steps": K4, "ms_per_step": ms4 / K4,
              "points": pts4, "interior_points": int4, "variant": var4, "autotune_ms_per_step": list(tune4),
              "work_items": items4, "layer_tiles": tiles4, "interior_ctas": ctas4,
              "steps_per_pass": tb4,
              "launch": ("CUDA graph of 32 steps: 16 pairs of two layer passes + one two-step interior launch "
                         "over all grids" if tb4 == 2 else
                         "CUDA graph of 32 steps (one layer + one interior launch per step over all grids)"),
              "roofline": {"bound": "hbm",
                           "kernel": "k_interior2d_tb2_batch<float>" if tb4 == 2 else "k_interior2d_batch<float>",
                           "achieved": ach4, "peak": hbm_peak, "steps_per_launch": tb4,
                           "unit": "GB/s", "frac": ach4 / hbm_peak, "avg_launch_ms": t_int4 * 1e3,
                           "bytes_per_launch": int4 * 16},
              "kernel_ms_per_step": {"interior": m4[0] / 64, "layer": m4[1] / 64}}
        b4.close()
        for s4 in solvers:
            s4.close()
        del solvers, inits4, b4
        torch.cuda.synchronize()

    # ---- the paper's stress workload: random sigma per edge, white noise in a disk -------
    stress = None
    if not args.no_stress:
        Ns, ws_w = 4096, 20
        Ts = Ns + 2 * ws_w
        rng_s = np.random.default_rng(91)
        e_s = np.arange(Ts)
        layer_s = (e_s <= ws_w - 2) | (e_s >= ws_w + Ns)
        sig_s = [np.where(layer_s, 2.0 * rng_s.random(Ts), 0.0) for _ in range(2)]
        s = PMLSolver((Ns, Ns), ws_w, sigma="user", user_sigma=sig_s, precision=32, device=dev)
        from paper_1804_01390_gb300 import _lib
        _lib.pml_set_variant(s.ctx, variant)
        u_s = wk.white_noise_disk((Ts, Ts), (Ts / 2.0, Ts / 2.0), 512.0, 0.25, seed=92,
                                  window=((ws_w, ws_w), (ws_w + Ns - 1, ws_w + Ns - 1)))
        s.set_initial(torch.from_numpy(u_s.astype(np.float32)).to(dev))
        Kst = max(K // 4, 50)
        ms_s, _ = timed_steps(s, Kst, min(W, 3), ws, profile=False)
        ms_s = max_over_ranks(ms_s, ws, dev)
        stress = {"workload": "2D %d^2 interior + %d-cell layer, sigma ~ U[0,2/h) per edge (user path), white noise "
                              "of variance 1/4 in a disk of radius 512, FP32" % (Ns, ws_w),
                  "value": Ts * Ts * Kst * ws / (ms_s / 1e3) / 1e9, "unit": UNIT, "steps": Kst,
                  "ms_per_step": ms_s / Kst}
        s.close()
        del s

    # ---- layer backed by a reflecting wall (the headline workload with walls, FP32) ------
    dwall = None
    if not args.no_wall:
        from paper_1804_01390_gb300 import _lib
        s = PMLSolver(wl.N, wl.w, dt=wl.dt, precision=32, device=dev, wall=True)
        _lib.pml_set_variant(s.ctx, variant)
        s.set_initial(torch.from_numpy(u0).to(dev))
        Kw = max(K // 4, 50)
        msw, _ = timed_steps(s, Kw, min(W, 3), ws, profile=False)
        msw = max_over_ranks(msw, ws, dev)
        dwall = {"workload": "2D %d^2 interior + 32-cell quadratic PML backed by reflecting walls, FP32" % wl.N[0],
                 "value": pts * Kw * ws / (msw / 1e3) / 1e9, "unit": UNIT, "steps": Kw, "ms_per_step": msw / Kw}
        s.close()
        del s

    # ---- damping gradient with sqrt(n) checkpoints (2048^2 + 32 adjoint workload, FP32,
    #      its full 10^4 steps) ---------------------------------------------------------
    gsig = None
    if not args.no_grad_sigma:
        from paper_1804_01390_gb300 import _lib
        wl5 = wk.cfg5()
        n5 = wl5.steps if args.n5 is None else args.n5
        s = PMLSolver(wl5.N, wl5.w, dt=wl5.dt, precision=32, device=dev, adjoint=True)
        u5 = torch.from_numpy(wk.initial_field(wl5, dtype=np.float32)).to(dev)
        src5 = wl5.sources
        s.set_sources(src5["coords"], src5["amp"], src5["f_peak"], src5["t_delay"])
        for nn in (min(n5, 100), n5):   # the first (short) call is the warm-up
            tgt5 = torch.zeros((nn, len(wl5.receivers)), dtype=torch.float32, device=dev)
            s.set_initial(u5)
            s.set_receivers(wl5.receivers, nn)
            scratch = _lib.pml_sigma_gradient_bytes(s.ctx, nn, 0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            J5, _, _ = s.sigma_gradient(nn, tgt5)
            t1 = time.perf_counter()
        pts5 = wl5.points
        K5 = int(np.ceil(np.sqrt(n5)))
        gsig = {"workload": "2D 2048^2 interior + 32-cell quadratic PML, 16 Ricker sources, 64 receivers, FP32: "
                            "%d forward steps with checkpoints every %d, then the adjoint with the damping "
                            "gradient" % (n5, K5),
                "steps": n5, "seconds": t1 - t0, "ms_per_step": (t1 - t0) * 1e3 / n5,
                "value": pts5 * n5 / (t1 - t0) / 1e9, "unit": "GPts/s (forward + adjoint + gradient per step)",
                "scratch_gb": scratch / 1e9,
                "scratch_note": "device memory the call allocates for its duration (pml_sigma_gradient_bytes): "
                                "%d checkpoints, %d states of one segment and 7 more states; storing every "
                                "state would take %.0f GB" % ((n5 + K5 - 1) // K5, K5,
                                                               (n5 + 1) * scratch / ((n5 + K5 - 1) // K5 + K5 + 7) / 1e9),
                "misfit": J5}
        s.close()
        del s, u5

    # ---- misfit gradient w.r.t. U0 and the source amplitudes (2048^2 + 32, 10^4 steps) ---
    mgrad = None
    if not args.no_misfit:
        from paper_1804_01390_gb300.autograd import traces
        wl5 = wk.cfg5()
        n5 = wl5.steps if args.n5 is None else args.n5
        src5 = wl5.sources
        s = PMLSolver(wl5.N, wl5.w, dt=wl5.dt, precision=32, device=dev, adjoint=True)
        # target traces: the seeded "true" model (another pulse, other amplitudes)
        g_t, a_t = wk.cfg5_target(wl5)
        wl_t = wk.Workload("cfg5-target", 2, wl5.N, wl5.w, dt=wl5.dt, steps=n5, gaussians=g_t,
                           sources=src5, receivers=wl5.receivers, seed=6)
        u_t = torch.from_numpy(wk.initial_field(wl_t, dtype=np.float32)).to(dev)
        d5 = traces(s, u_t, torch.tensor(a_t, dtype=torch.float64), n5, src5["coords"], wl5.receivers,
                    src5["f_peak"], src5["t_delay"]).detach().clone()
        u5 = torch.from_numpy(wk.initial_field(wl5, dtype=np.float32)).to(dev).requires_grad_(True)
        a5 = torch.tensor(src5["amp"], dtype=torch.float64, requires_grad=True)
        # warm-up: 20 steps forward and back
        trw = traces(s, u5, a5, 20, src5["coords"], wl5.receivers, src5["f_peak"], src5["t_delay"])
        (0.5 * (trw.double() ** 2).sum()).backward()
        u5.grad = None
        a5.grad = None
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        tr5 = traces(s, u5, a5, n5, src5["coords"], wl5.receivers, src5["f_peak"], src5["t_delay"])
        J5 = 0.5 * ((tr5.double() - d5.double()) ** 2).sum()
        J5.backward()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sec = max_over_ranks(t1 - t0, ws, dev)
        mgrad = {"workload": "2D 2048^2 interior + 32-cell quadratic PML, Gaussian s=8, 16 Ricker sources, 64 "
                             "receivers on a line, FP32: L2 misfit of the traces against a seeded target model, "
                             "gradient w.r.t. U0 and the 16 amplitudes through torch.autograd (forward with "
                             "traces, then the transposed steps with the residual injected)",
                 "steps": n5, "seconds": sec, "ms_per_step": sec * 1e3 / n5,
                 "value": 2 * wl5.points * n5 * ws / sec / 1e9,
                 "unit": "GPts/s (forward and transposed point-updates)",
                 "misfit": float(J5.item()), "grad_u0_l2": float(u5.grad.double().norm().item()),
                 "grad_amp": [float(x) for x in a5.grad.tolist()],
                 "checkpoints": "none needed: the traces are linear in U0 and the amplitudes, so the "
                                "adjoint needs no forward states"}
        s.close()
        del s, u5, u_t, d5

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)

    if fp64 is not None and cpu is not None:
        fp64["cpu_baseline"] = cpu   # the oracle is FP64: the same baseline serves both lines
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "2D %d^2 interior + 32-cell quadratic PML (T = %d^2), 16 seeded "
                                   "Gaussian pulses, RK4 dt = 0.5h" % (wl.N[0], wl.T[0]), "grid": list(wl.T),
                       "pml_width": wl.w, "interior_variant": variant, "steps_per_pass": tb,
                       "autotune_ms_per_step": tune_table,
                       "l2": "inputs larger than L2 (U and V are 272 MB each; 1.09 GB state read + written "
                             "per pass, one pass per %d step%s)" % (tb, "s" if tb > 1 else ""), "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": traffic, "peak_kind": peak_kind,
                         "traffic_note": ("ncu dram bytes read + written of the same kernel shape on the 6144^2 case, "
                                          "scaled by vertices per launch" if traffic else
                                          "no capture of the chosen kernel shape"),
                         "kernel": "k_interior2d_tb2<float>" if tb == 2 else "k_interior2d<float>",
                         "steps_per_launch": tb, "bytes_per_launch": bytes_per_launch,
                         "bytes_rule": "16 B per vertex per launch (U, V read and written once)",
                         "effective_gbs_per_update": effective,
                         "avg_launch_ms": avg_launch_s * 1e3, "layer_time_share": layer_share,
                         "timing": "per-kernel CUDA events on the solver stream over a second pass of the "
                                   "same K steps (%.3f ms/step with events)" % (ms_prof / K)},
            "hbm_roofline": step_roofline(value / ws, 4),
            "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(), "fp64": fp64,
            "fp_peaks": peaks, "accuracy": accuracy, "adjoint": adj,
            "cfg3": d3, "batched": d4, "stress": stress, "grad_sigma": gsig, "wall": dwall,
            "misfit_gradient": mgrad,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ------------------------------------------------------------------------------------

def _oracle_sample(N=1024, w=32):
    """A bounded sample of the workload: the same layer (w = 32, quadratic, sigma_max 2)
    around a 1024^2 physical domain, Gaussian pulses from the same recipe."""
    import oracle
    from paper_1804_01390_gb300 import workloads as wk
    wl = wk.cfg2(N=N, w=w, npulses=4)
    sig = [oracle.sigma_profile(n, w, oracle.KIND_POWER, 2.0, 2.0) for n in wl.N]
    g = oracle.Grid(wl.T, 1.0, sig)
    y = g.zeros_state()
    y[0] = wk.initial_field(wl).reshape(-1)
    return oracle, g, y, wl


def cpu_baseline(seconds=10.0):
    oracle, g, y, wl = _oracle_sample()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    oracle.rk4(g, y, 1, wl.dt, openmp=True)   # warm-up (page-in, thread pool)
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds and steps < 1000:
        y, _ = oracle.rk4(g, y, 1, wl.dt, step0=steps, openmp=True)
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": g.n * steps / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d RK4 steps of the FP64 C oracle (OpenMP build) on a %dx%d box: the same "
                      "32-cell quadratic layer around a 1024^2 domain" % (steps, g.T[0], g.T[1]),
            "seconds": dt}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    oracle, g, y, wl = _oracle_sample()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    for k in range(args.warmup):
        y, _ = oracle.rk4(g, y, 1, wl.dt, step0=k, openmp=True)
    t0 = time.perf_counter()
    for k in range(args.steps):
        y, _ = oracle.rk4(g, y, 1, wl.dt, step0=args.warmup + k, openmp=True)
    dt = time.perf_counter() - t0
    value = g.n * args.steps / dt / 1e9
    sample = ("each step: one RK4 step of the FP64 C oracle (OpenMP build) on a %dx%d box, the same "
              "32-cell quadratic layer around a 1024^2 domain" % (g.T[0], g.T[1]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "2D 8192^2 interior + 32-cell quadratic PML (T = 8256^2), 16 seeded "
                                   "Gaussian pulses, RK4 dt = 0.5h", "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--n3", type=int, default=None, help="3D physical side (default 512)")
    ap.add_argument("--variant3", type=int, default=None,
                    help="use this 3D frame kernel (0 tile kernel, 1 level passes, 2 slab tiles) instead of "
                         "the autotuned one (profiling)")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-stress", action="store_true")
    ap.add_argument("--no-grad-sigma", action="store_true")
    ap.add_argument("--no-wall", action="store_true")
    ap.add_argument("--no-misfit", action="store_true")
    ap.add_argument("--n5", type=int, default=None, help="steps of the misfit-gradient workload (default 10^4)")
    ap.add_argument("--n4", type=int, default=None, help="largest side of the batched grids (default 2048)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--retune", action="store_true", help="ignore the autotune cache")
    ap.add_argument("--variant", type=int, default=None,
                    help="use this 2D FP32 kernel variant instead of the autotuned one (profiling)")
    ap.add_argument("--n", type=int, default=None,
                    help="physical domain side (default 8192); smaller values are for profiling runs")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if args.steps is None:
        args.steps = 20 if args.impl == "reference" else 2000
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    try:
        run_ours(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
