"""Benchmark of the operator hot path on the throughput workload stress1024.

One step = one pass of the A / A^T pair behind the reconstruction-loss
gradient for a batch of 8 histories: y = A x (forward) followed by
g = A^T y (adjoint), on the Kerr a = 0.94, i = 75 deg geometry with a
1024 x 1024 image, a 256 x 512 source grid, 256 hats and 1024 frames (FP32
tables and accumulation), x ~ U(0, 1) per coefficient.  Ray tables come from
the library's own GPU tracer (rtt_trace_rays), the operator from
rtt_build_operator.  The same JSON line carries the batch sweep 1-64 of that
workload, the kerr256 step (a = 0.5, i = 50 deg, 256 x 256 with 2 x 2 ring
sub-rays, 64 x 128 nodes, 64 hats, 256 frames), the 12-geometry rank audit
against the plain FP64 path, and the FP64 CPU oracle timed on the host.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).  Under torchrun each rank runs an
independent replica (weak scaling; the operator has no exchange step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "A+A^T applies/s"
UNIT = "history-applies/s"
BATCH = 8
SWEEP_BATCHES = (1, 2, 4, 8, 16, 32, 64)
L2_FLUSH_BYTES = 256 << 20


WORKLOAD = ("stress1024: Kerr a=0.94 i=75deg 1024x1024, 256x512 source, 256 hats, 1024 frames, "
            "resolved n=0..2, FP32")
WORKLOAD_KERR256 = ("kerr256: Kerr a=0.5 i=50deg 256x256 (2x2 ring sub-rays), 64x128 source, "
                    "64 hats, 256 frames, resolved n=0..2")


def measured_peaks(kind: str = "hbm"):
    """(peak, "measured" | "fallback"): HBM copy GB/s, or (kind="tensor") the
    burst dense BF16 TFLOP/s."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops" if kind == "tensor" else "hbm_gbs"]), "measured"
    return (1800.0 if kind == "tensor" else 6400.0), "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,clocks.mem")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons, power, mem = [], [], set(), [], []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for v, dst in ((f[3], power), (f[9] if len(f) > 9 else "", mem)):
                    try:
                        dst.append(float(v))
                    except ValueError:
                        pass
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "sm_min_mhz": min(sm),
               "reasons": sorted(reasons), "samples": len(sm)}
        if power:
            out["power_w_max"] = max(power)
        if mem:
            out["mem_mhz"] = statistics.median(mem)
            out["mem_min_mhz"] = min(mem)
        return out


def build_workload(device, w, batch, seed0: int = 1, tune: bool = True):
    """Trace, build and (optionally) autotune an operator; x ~ U(0, 1) per
    coefficient from the seeded generator (seeds seed0 .. seed0 + batch - 1)."""
    import torch

    from paper_2609_05528_b300 import build, rtt
    from paper_2609_05528_b300 import inputs as I
    build.build()
    s = I.screen_samples(w)
    torch.cuda.synchronize(device)
    tab = rtt.rtt_trace_rays(w.geometry.spin, w.geometry.incl_deg, w.grid, s)
    op = rtt.Operator(w, tab)
    x = torch.from_numpy(I.uniform_batch(w, range(seed0, seed0 + batch)).astype(np.float32)).to(device)
    op.tune = op.autotune(batch) if tune else None  # kernel variants (setup, untimed)
    return tab, op, x


def kernel_source_hash() -> str:
    """Hash of the apply kernels' source: ncu DRAM traffic recorded in
    profiles/ is used only while this hash is unchanged."""
    import hashlib
    h = hashlib.sha256()
    for name in ("apply.cu", "adjoint.cu", "kern_common.cuh", "rtt_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2609_05528_b300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str = "kerr256", variant=None):
    """DRAM bytes per launch of `kernel` (the apply A or AT) from the committed
    ncu record of `workload` at batch 8, or None when the record is missing,
    was taken on other kernel sources, or (variant given) on another kernel
    variant of the apply."""
    p = os.path.join(ROOT, "profiles", f"traffic_{workload}_b8.json")
    try:
        with open(p) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return None
    if variant is not None and "variant" in rec:
        keys = ("fwd_kernel", "fwd_bc", "fwd_half", "fwd_order", "fwd_cols") if kernel == "A" else \
               ("adj_kernel", "adj_cols")
        if any(int(rec["variant"].get(k, -1)) != int(variant.get(k, -2)) for k in keys):
            return None
    return rec.get("traffic_bytes", {}).get(kernel)


def algorithmic_bytes(op, B, elem=4, weight_bytes=16):
    """Bytes the method must move per launch: y once, x once, plus tables
    (weight_bytes: the four corner weights of a ray, 16 in FP32, 8 in BF16)."""
    E = int(op.info.n_rays)
    R = int(op.info.n_rows)
    S = int(op.info.n_nodes)
    y = R * op.n_frames * B * elem
    x = S * op.n_hats * B * elem
    table_fwd = E * (16 + weight_bytes) + (R + 1) * 4
    # adjoint: the cell-ordered ray table (row, column, hat base and fraction,
    # four corner weights) and the gather table (four record indices per node)
    table_adj = E * (16 + weight_bytes) + S * 16
    return {"A": y + x + table_fwd, "AT": y + x + table_adj, "y": y, "x": x}


def time_loop(stream, fn, n, flush=None):
    """Per-call device times (ms) of fn on `stream`, CUDA events around each
    call, optional L2 flush before each (outside the events)."""
    import torch
    out = []
    for _ in range(n):
        if flush is not None:
            flush.zero_()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        fn()
        a1.record(stream)
        a1.synchronize()
        out.append(a0.elapsed_time(a1))
    return out


def roofline_of(op, B, mA, mAT, traffic_key=None):
    """traffic_key: the workload name of the committed ncu traffic record
    (used when it was taken on the variants op runs at batch B)."""
    ab = algorithmic_bytes(op, B)
    dom, dom_ms = ("A", mA) if mA >= mAT else ("AT", mAT)
    peak, peak_kind = measured_peaks()
    achieved = ab[dom] / (dom_ms * 1e-3) / 1e9
    return ab, {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_traffic(dom, traffic_key, op.get_variant(B)) if traffic_key else None,
                "traffic_other": recorded_traffic("AT" if dom == "A" else "A", traffic_key, op.get_variant(B))
                if traffic_key else None,
                "algorithmic_bytes": ab[dom], "source_hash": kernel_source_hash(),
                "A_frac": ab["A"] / (mA * 1e-3) / 1e9 / peak,
                "AT_frac": ab["AT"] / (mAT * 1e-3) / 1e9 / peak}


def run_ours(args, rank, world, device):
    import torch

    from paper_2609_05528_b300 import inputs as I
    from paper_2609_05528_b300 import rtt
    torch.cuda.set_device(device)
    w = I.stress1024(0.94)
    tab, op, x = build_workload(device, w, BATCH)
    stream = torch.cuda.current_stream(device)
    R = op.arm_rows(7)
    y = torch.empty((R, op.n_frames, BATCH), dtype=torch.float32, device=device)
    g = torch.empty_like(x)

    def step():
        op.apply_A(x, y)
        op.apply_AT(y, g)

    # y (12.4 GB) and x (1.07 GB) are far larger than L2: no flush needed
    with ClockSampler(device.index if device.index is not None else 0) as clk:
        n_warm = max(args.warmup, 3)
        for _ in range(n_warm - 1):
            step()
        torch.cuda.synchronize(device)
        ranks_barrier(world)
        step()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("bench_timed")
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize(device)
        ranks_barrier(world)
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, device)
    clocks = clk.summary()
    # the split between the two applies, each timed alone (events around one call)
    t_A = time_loop(stream, lambda: op.apply_A(x, y), args.steps)
    t_AT = time_loop(stream, lambda: op.apply_AT(y, g), args.steps)
    mA, mAT = float(np.median(t_A)), float(np.median(t_AT))
    ab, roof = roofline_of(op, BATCH, mA, mAT, traffic_key="stress1024")

    # the BF16-weight table variant of the same step (rtt_set_weight_precision):
    # the applies read 8-byte corner weights; y's change against the FP32
    # weights on every 101st row
    try:
        y_ref = y[::101].clone()  # y of the last FP32-weight forward above
        op.set_weight_precision(rtt.WEIGHTS_BF16)
        tune16 = op.autotune(BATCH)  # the variants for these tables (bit-neutral)
        op.apply_A(x, y)
        op.apply_AT(y, g)
        mA16 = float(np.median(time_loop(stream, lambda: op.apply_A(x, y), args.steps)))
        mAT16 = float(np.median(time_loop(stream, lambda: op.apply_AT(y, g), args.steps)))
        op.apply_A(x, y)
        rel = float(torch.linalg.vector_norm(y[::101] - y_ref) / torch.linalg.vector_norm(y_ref))
        op.set_weight_precision(rtt.WEIGHTS_FP32)
        op.tune = op.autotune(BATCH)  # back to the FP32 tables' variants
        ab16 = algorithmic_bytes(op, BATCH, weight_bytes=8)
        peak16, _ = measured_peaks()
        bf16 = {"ms_per_step": mA16 + mAT16, "value": job_value(world, BATCH, mA16 + mAT16),
                "A_ms": mA16, "AT_ms": mAT16,
                "variant": [tune16["fwd_kernel"], tune16["fwd_bc"], tune16["adj_kernel"]],
                "A_frac": ab16["A"] / (mA16 * 1e-3) / 1e9 / peak16,
                "AT_frac": ab16["AT"] / (mAT16 * 1e-3) / 1e9 / peak16,
                "y_rel_l2_vs_fp32_weights": rel, "rows_compared": int(y_ref.shape[0])}
        del y_ref
    except Exception as exc:  # a measurement extra; report why it failed
        bf16 = {"error": str(exc)[:200]}

    # the same step replayed from a captured CUDA graph
    graph = None
    try:
        graph_obj = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device)
        cap.wait_stream(stream)
        with torch.cuda.stream(cap):
            step()
        torch.cuda.synchronize(device)
        with torch.cuda.graph(graph_obj, stream=cap):
            step()
        torch.cuda.synchronize(device)
        for _ in range(3):
            graph_obj.replay()
        gm = max_over_ranks(float(np.mean(time_loop(stream, graph_obj.replay, args.steps))), world,
                            device)
        graph = {"ms_per_step": gm, "value": job_value(world, BATCH, gm)}
    except Exception as exc:  # capture is a measurement extra; report why it failed
        graph = {"error": str(exc)[:200]}

    # end-to-end through the C ABI with host buffers: x from pinned host
    # memory to the device, A, A^T, the gradient back to pinned host memory
    xh = x.cpu().pin_memory()
    gh = torch.empty(g.shape, dtype=g.dtype).pin_memory()
    xd = torch.empty_like(x)

    def e2e_step():
        xd.copy_(xh, non_blocking=True)
        op.apply_A(xd, y)
        op.apply_AT(y, g)
        gh.copy_(g, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize(device)
    e2e_serial_ms = max_over_ranks(float(np.mean(time_loop(stream, e2e_step, max(3, args.steps // 4)))),
                                   world, device)
    # pipelined over steps as a user streaming histories would run it: each
    # step still copies its x in and its gradient out, overlapping the
    # kernels of its neighbours (copy-in, compute, copy-out streams, two
    # buffer sets, event dependencies)
    s_in, s_cmp, s_out = (torch.cuda.Stream(device) for _ in range(3))
    xds = [torch.empty_like(x) for _ in range(2)]
    gds = [torch.empty_like(x) for _ in range(2)]
    ghs = [torch.empty(g.shape, dtype=g.dtype).pin_memory() for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_cmp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def pipeline(n):
        for i in range(n):
            b = i % 2
            if i >= 2:
                s_in.wait_event(ev_cmp[b])  # x buffer b was read by step i - 2
            with torch.cuda.stream(s_in):
                xds[b].copy_(xh, non_blocking=True)
            ev_in[b].record(s_in)
            s_cmp.wait_event(ev_in[b])
            if i >= 2:
                s_cmp.wait_event(ev_out[b])  # gradient buffer b was copied out by step i - 2
            op.apply_A(xds[b], y, stream=s_cmp)
            op.apply_AT(y, gds[b], stream=s_cmp)
            ev_cmp[b].record(s_cmp)
            s_out.wait_event(ev_cmp[b])
            with torch.cuda.stream(s_out):
                ghs[b].copy_(gds[b], non_blocking=True)
            ev_out[b].record(s_out)

    pipeline(3)
    torch.cuda.synchronize(device)
    n_pipe = max(4, args.steps // 2)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(s_in)
    s_cmp.wait_event(p0)
    s_out.wait_event(p0)
    pipeline(n_pipe)
    p1.record(s_out)
    p1.synchronize()
    torch.cuda.synchronize(device)
    e2e_ms = max_over_ranks(p0.elapsed_time(p1) / n_pipe, world, device)
    del xds, gds, ghs, xd

    # plain FP64 GPU path (the same kernels in double) for comparison
    fp64 = None
    try:
        x64 = x.double()
        y64 = torch.empty((R, op.n_frames, BATCH), dtype=torch.float64, device=device)
        g64 = torch.empty_like(x64)
        op.apply_A(x64, y64)
        op.apply_AT(y64, g64)
        torch.cuda.synchronize(device)
        f_ms = time_loop(stream, lambda: (op.apply_A(x64, y64), op.apply_AT(y64, g64)), 3)
        fp64_ms = max_over_ranks(float(np.mean(f_ms)), world, device)
        fp64 = {"value": job_value(world, BATCH, fp64_ms), "ms_per_step": fp64_ms}
        del x64, y64, g64
    except Exception as exc:  # a measurement extra; report why it failed
        fp64 = {"error": str(exc)[:200]}
    del y, g
    torch.cuda.empty_cache()

    # kerr256, batch 8 (the autograd reconstruction step's workload), before
    # the long sweep, with its own clock record
    with ClockSampler(device.index if device.index is not None else 0) as clk_k:
        k256 = run_kerr256(args, world, device)
    k256["clocks"] = clk_k.summary()

    # batch sweep of the same workload (A and A^T GB/s against HBM, FP32 and
    # BF16-weight tables), each batch size autotuned first; y >= 1.5 GB per
    # history, far above L2
    sweep = []
    peak, _ = measured_peaks()
    clk_s = ClockSampler(device.index if device.index is not None else 0)
    clk_s.__enter__()
    for B in (() if args.no_sweep else SWEEP_BATCHES):
        try:
            tune = op.autotune(B)
            xb = torch.from_numpy(I.uniform_batch(w, range(1, 1 + B)).astype(np.float32)).to(device)
            yb = torch.empty((R, op.n_frames, B), dtype=torch.float32, device=device)
            gb = torch.empty_like(xb)
            op.apply_A(xb, yb)
            op.apply_AT(yb, gb)
            reps = 5 if B <= 16 else 3
            tA = float(np.median(time_loop(stream, lambda: op.apply_A(xb, yb), reps)))
            tT = float(np.median(time_loop(stream, lambda: op.apply_AT(yb, gb), reps)))
            abb = algorithmic_bytes(op, B)
            row = {"batch": B, "A_ms": tA, "AT_ms": tT,
                   "A_gbs": abb["A"] / (tA * 1e-3) / 1e9, "AT_gbs": abb["AT"] / (tT * 1e-3) / 1e9,
                   "A_frac": abb["A"] / (tA * 1e-3) / 1e9 / peak,
                   "AT_frac": abb["AT"] / (tT * 1e-3) / 1e9 / peak,
                   "history_applies_per_s": B / ((tA + tT) * 1e-3),
                   "variant": {k: tune[k] for k in ("fwd_kernel", "fwd_bc", "fwd_order", "adj_kernel")}}
            # the BF16-weight table variant beside the FP32 one, tuned for its tables
            op.set_weight_precision(rtt.WEIGHTS_BF16)
            tune16 = op.autotune(B)
            op.apply_A(xb, yb)
            op.apply_AT(yb, gb)
            tA16 = float(np.median(time_loop(stream, lambda: op.apply_A(xb, yb), reps)))
            tT16 = float(np.median(time_loop(stream, lambda: op.apply_AT(yb, gb), reps)))
            op.set_weight_precision(rtt.WEIGHTS_FP32)
            ab16 = algorithmic_bytes(op, B, weight_bytes=8)
            row["bf16_weights"] = {"A_ms": tA16, "AT_ms": tT16,
                                   "variant": [tune16["fwd_kernel"], tune16["fwd_bc"], tune16["adj_kernel"]],
                                   "A_frac": ab16["A"] / (tA16 * 1e-3) / 1e9 / peak,
                                   "AT_frac": ab16["AT"] / (tT16 * 1e-3) / 1e9 / peak,
                                   "history_applies_per_s": B / ((tA16 + tT16) * 1e-3)}
            sweep.append(row)
            del xb, yb, gb
            torch.cuda.empty_cache()
        except Exception as exc:
            sweep.append({"batch": B, "error": str(exc)[:200]})
    clk_s.__exit__(None, None, None)
    sweep_clocks = clk_s.summary() if sweep else None
    n_rays, n_nodes = int(op.info.n_rays), op.n_nodes
    op.close()

    value = job_value(world, BATCH, ms_step)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch": BATCH, "rows": R, "rays": n_rays,
                   "nodes": n_nodes, "hats": w.time.n_hats, "frames": w.time.n_frames,
                   "x": "U(0,1) per coefficient, seeds 1..8",
                   "l2": "inputs larger than L2 (y 12.4 GB per step), no flush",
                   "parallelism": f"replicas x{world}", "autotune": op.tune},
        "hbm_gbs": (ab["A"] + ab["AT"]) / (ms_step * 1e-3) / 1e9,
        "kernels_ms": {"A": mA, "AT": mAT},
        "roofline": roof,
        "e2e": {"value": job_value(world, BATCH, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
                "pipelined": "copy-in / compute / copy-out streams over steps",
                "serial_ms_per_step": e2e_serial_ms,
                "h2d_bytes_per_step": int(xh.numel() * 4), "d2h_bytes_per_step": int(gh.numel() * 4)},
        "fp64_path": fp64,
        "bf16_weights": bf16,
        "cuda_graph": graph,
        "sweep": sweep,
        "sweep_clocks": sweep_clocks,
        "kerr256": k256,
        "clocks": clocks,
        "gpu_launches": launches_per_step(BATCH) * args.steps,
    }
    return out


def run_kerr256(args, world, device):
    """kerr256 at batch 8: the A + A^T step (L2 flushed between steps), its
    split, the order mixing of its y (Eq. 4) and a CUDA-graph replay."""
    import torch

    from paper_2609_05528_b300 import inputs as I
    from paper_2609_05528_b300 import rtt
    w = I.kerr256()
    _, op, x = build_workload(device, w, BATCH, seed0=100)
    stream = torch.cuda.current_stream(device)
    R = op.arm_rows(7)
    y = torch.empty((R, op.n_frames, BATCH), dtype=torch.float32, device=device)
    g = torch.empty_like(x)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def step():
        op.apply_A(x, y)
        op.apply_AT(y, g)

    for _ in range(3):
        flush.zero_()
        step()
    torch.cuda.synchronize(device)
    ms = float(np.mean(time_loop(stream, step, args.steps, flush)))
    mA = float(np.median(time_loop(stream, lambda: op.apply_A(x, y), args.steps, flush)))
    mAT = float(np.median(time_loop(stream, lambda: op.apply_AT(y, g), args.steps, flush)))
    _, roof = roofline_of(op, BATCH, mA, mAT, traffic_key="kerr256")
    mix = {}
    try:
        peak_m, _ = measured_peaks()
        for name, mode in (("unresolved", rtt.MIX_UNRESOLVED), ("total_flux", rtt.MIX_TOTAL_FLUX)):
            yl = op.mix_rows(y, mode)
            mm = float(np.mean(time_loop(stream, lambda: op.mix_rows(y, mode, out=yl), args.steps,
                                         flush)))
            nbytes = (y.numel() + yl.numel()) * 4
            mix[name] = {"ms": mm, "rows_out": int(yl.shape[0]), "algorithmic_bytes": int(nbytes),
                         "GB/s": nbytes / (mm * 1e-3) / 1e9, "frac": nbytes / (mm * 1e-3) / 1e9 / peak_m}
    except Exception as exc:  # a measurement extra; report why it failed
        mix = {"error": str(exc)[:200]}
    out = {"workload": WORKLOAD_KERR256, "batch": BATCH, "ms_per_step": ms,
           "value": job_value(world, BATCH, ms), "kernels_ms": {"A": mA, "AT": mAT},
           "roofline": roof, "order_mix": mix, "autotune": op.tune,
           "l2": "flushed between timed steps (256 MiB write)"}
    op.close()
    return out


def run_gemm(args, device):
    """The tensor-core FP64 contraction C = A^T B on N(0, 1) inputs: CUDA-event
    time per call (after --warmup calls; --steps timed calls), its FP64 and
    digit-product rates, cuBLAS DGEMM on the same operands, and the largest
    error relative to sum_k |A_ki| |B_kj|."""
    import torch

    from paper_2609_05528_b300 import rtt
    k, m, n = args.gemm
    g = torch.Generator(device=device).manual_seed(1)
    A = torch.randn((k, m), dtype=torch.float64, device=device, generator=g)
    B = torch.randn((k, n), dtype=torch.float64, device=device, generator=g)
    stream = torch.cuda.current_stream(device)
    for _ in range(max(args.warmup, 1)):
        C = rtt.gemm_tn(A, B)
    torch.cuda.synchronize(device)
    t = float(np.median(time_loop(stream, lambda: rtt.gemm_tn(A, B), max(args.steps, 1))))
    td = float(np.median(time_loop(stream, lambda: A.T @ B, 2)))
    ref = A.T @ B
    err = float(((C - ref).abs() / (A.abs().T @ B.abs())).max())
    peak = measured_peaks(kind="tensor")[0]
    return {"k": k, "m": m, "n": n, "ms": t, "dgemm_ms": td, "fp64_tflops": 2 * k * m * n / t / 1e9,
            "digit_product_tflops": 56 * k * m * n / t / 1e9,
            "frac_of_bf16_peak": 56 * k * m * n / t / 1e9 / peak, "max_err_over_abs_bound": err}


def run_profile_case(args, device):
    """The step alone, for profiling: the workload at batch args.batch
    (default 8) with its autotuned variants, max(warmup, 3) untimed steps,
    then args.steps steps inside the NVTX range bench_timed
    (ncu --nvtx-include "bench_timed/")."""
    import torch

    from paper_2609_05528_b300 import inputs as I
    w = I.stress1024(0.94) if args.profile == "stress1024" else I.kerr256()
    B = args.batch
    # --variant pins the kernel variant (the one an autotuned run without the
    # profiler printed): a tuner timing its candidates under a profiler could
    # choose differently
    _, op, x = build_workload(device, w, B, seed0=100, tune=not args.variant)
    if args.variant:
        fk, bc, half, ak, order, fcols, acols = (int(v) for v in args.variant.split(","))
        op.set_variant(B, fk, bc, half, ak, fwd_order=order, fwd_cols=fcols, adj_cols=acols)
    y = torch.empty((op.arm_rows(7), op.n_frames, B), dtype=torch.float32, device=device)
    g = torch.empty_like(x)
    for _ in range(max(args.warmup, 3)):
        op.apply_A(x, y)
        op.apply_AT(y, g)
    torch.cuda.synchronize(device)
    torch.cuda.nvtx.range_push("bench_timed")
    for _ in range(args.steps):
        op.apply_A(x, y)
        op.apply_AT(y, g)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(device)
    out = {"workload": w.name, "batch": B, "steps": args.steps, "variant": op.get_variant(B),
           "algorithmic_bytes": algorithmic_bytes(op, B), "source_hash": kernel_source_hash(),
           "status": op.status()}
    op.close()
    return out


def ranks_barrier(world: int):
    """Barrier across the replicas (no-op on one process)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The job's time for a timed region: the slowest replica's."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, batch: int, ms: float) -> float:
    """Whole-job throughput: every replica applies A + A^T to its own batch
    (weak scaling), so the job moves world * batch histories per step."""
    return world * batch / (ms * 1e-3)


def launches_per_step(B: int) -> int:
    """Kernel launches of one A + A^T pair: one forward launch; per batch pass
    of the adjoint (32 columns, 64 at batches of whole 64-column passes) one
    cell kernel and one gather launch."""
    pc = 64 if B % 64 == 0 else 32
    return 1 + 2 * ((B + pc - 1) // pc)


def run_sweep(device, batches=(1, 2, 4, 8, 16, 32, 64), reps: int = 5):
    """Throughput sweep on the stress1024 workloads (i=75 deg, 1024x1024,
    256x512 nodes, 256 hats, 1024 frames; Schwarzschild and Kerr a=0.94):
    A and A^T achieved GB/s (algorithmic bytes / event time) per batch size,
    and on the Kerr workload the BF16-weight table variant beside it.
    y is >= 1.5 GB per history, far above L2, so no flush is needed."""
    import torch

    from paper_2609_05528_b300 import inputs as I
    from paper_2609_05528_b300 import rtt
    peak, peak_kind = measured_peaks()
    stream = torch.cuda.current_stream(device)
    lines = []
    for spin in (0.94, 0.0):
        bf16 = spin == 0.94
        w = I.stress1024(spin)
        tab = rtt.rtt_trace_rays(w.geometry.spin, w.geometry.incl_deg, w.grid, I.screen_samples(w))
        op = rtt.Operator(w, tab)
        R = op.arm_rows(7)
        gen = torch.Generator(device=device).manual_seed(1)
        res = []
        for B in batches:
            tune = op.autotune(B)
            x = torch.rand((op.n_nodes, op.n_hats, B), generator=gen, device=device)
            y = torch.empty((R, op.n_frames, B), dtype=torch.float32, device=device)
            g = torch.empty_like(x)
            for _ in range(2):
                op.apply_A(x, y)
                op.apply_AT(y, g)
            torch.cuda.synchronize(device)
            ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(reps)]
            for e0, e1, e2 in ev:
                e0.record(stream)
                op.apply_A(x, y)
                e1.record(stream)
                op.apply_AT(y, g)
                e2.record(stream)
            torch.cuda.synchronize(device)
            tA = float(np.mean([a.elapsed_time(b) for a, b, _ in ev]))
            tT = float(np.mean([b.elapsed_time(c) for _, b, c in ev]))
            ab = algorithmic_bytes(op, B)
            row = {"batch": B, "A_ms": tA, "AT_ms": tT,
                   "variant": [tune["fwd_kernel"], tune["fwd_bc"], tune["adj_kernel"]],
                   "rule_ms": [tune["fwd_ms_rule"], tune["adj_ms_rule"]],
                   "A_gbs": ab["A"] / (tA * 1e-3) / 1e9, "AT_gbs": ab["AT"] / (tT * 1e-3) / 1e9,
                   "A_frac": ab["A"] / (tA * 1e-3) / 1e9 / peak,
                   "AT_frac": ab["AT"] / (tT * 1e-3) / 1e9 / peak}
            if bf16:  # the BF16-weight table variant beside the FP32 one
                op.set_weight_precision(rtt.WEIGHTS_BF16)
                op.apply_A(x, y)
                op.apply_AT(y, g)
                tA16 = float(np.median(time_loop(stream, lambda: op.apply_A(x, y), reps)))
                tT16 = float(np.median(time_loop(stream, lambda: op.apply_AT(y, g), reps)))
                op.set_weight_precision(rtt.WEIGHTS_FP32)
                ab16 = algorithmic_bytes(op, B, weight_bytes=8)
                row["bf16_weights"] = {"A_ms": tA16, "AT_ms": tT16,
                                       "A_frac": ab16["A"] / (tA16 * 1e-3) / 1e9 / peak,
                                       "AT_frac": ab16["AT"] / (tT16 * 1e-3) / 1e9 / peak}
            res.append(row)
            del x, y, g
            torch.cuda.empty_cache()
        lines.append({"sweep": f"stress1024 a={spin:g} i=75deg", "rows": R,
                      "rays": int(op.info.n_rays), "peak_gbs": peak, "peak_kind": peak_kind,
                      "results": res})
        op.close()
    return lines


def run_audit(device):
    """The 12-geometry rank audit (Sec. 6.2-6.3): spins {0, .5, .75, .94} x
    inclinations {20, 50, 75} deg at kerr256 sizes, S224 class, direct and
    resolved arms.  Times the audit with the FP64 class Gram (separable S224,
    no P) against the normal-operator Gram and the plain FP64 path (Gram over
    data samples)."""
    import torch

    from paper_2609_05528_b300 import inputs as I
    from paper_2609_05528_b300 import rtt
    t0 = time.perf_counter()
    ops, Qs, cells = [], [], []
    for w in I.audit12():
        tab = rtt.rtt_trace_rays(w.geometry.spin, w.geometry.incl_deg, w.grid, I.screen_samples(w))
        op = rtt.Operator(w, tab)
        cells.append((w, tab))
        ops.append(op)
        Qs.append(rtt.synth_class(op, rtt.CLASS_S224))
    torch.cuda.synchronize(device)
    t_build = time.perf_counter() - t0
    out = {"workload": "12 geometries: spins {0,0.5,0.75,0.94} x incl {20,50,75} deg, kerr256 sizes, "
                       "S224 class, arms direct/resolved, SNR0=100, rho=1",
           "trace_and_build_s": t_build}
    runs = {}
    for name, mode in (("class", rtt.GRAM_CLASS_S224), ("normal", rtt.GRAM_NORMAL),
                       ("data", rtt.GRAM_DATA)):
        torch.cuda.synchronize(device)
        t = time.perf_counter()
        recs, sig = rtt.rank_audit(ops, Qs, (1, 7), mode=mode)
        torch.cuda.synchronize(device)
        runs[name] = (time.perf_counter() - t, recs)
    tn, rn = runs["class"]
    td, rd = runs["data"]
    # the class audit is one batched plan over the 24 (geometry, arm) jobs:
    # create (tables, A_{0,0.999}, buffers), a run (one launch per stage, no
    # host synchronisation) and the results; a second run and a run replayed
    # from a captured CUDA graph reuse the plan
    torch.cuda.synchronize(device)
    t = time.perf_counter()
    plan = rtt.AuditPlan(ops, (1, 7))
    torch.cuda.synchronize(device)
    t_create = time.perf_counter() - t
    runs_s = []
    for _ in range(2):
        t = time.perf_counter()
        plan.run()
        recs_p, _ = plan.results()
        runs_s.append(time.perf_counter() - t)
    s = torch.cuda.Stream(device)
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize(device)
    with torch.cuda.stream(s):
        graph.capture_begin()
        plan.run(stream=s)
        graph.capture_end()
    torch.cuda.synchronize(device)
    t = time.perf_counter()
    with torch.cuda.stream(s):
        graph.replay()
    recs_g, _ = plan.results(stream=s)
    t_graph = time.perf_counter() - t
    out["plan"] = {"jobs": len(ops) * 2, "create_s": round(t_create, 4),
                   "run_and_results_s": [round(v, 4) for v in runs_s],
                   "graph_replay_and_results_s": round(t_graph, 4),
                   "stage_s": {k: round(sum(getattr(r[i], "seconds_" + k) for r in recs_p for i in range(2)), 4)
                               for k in ("probe", "gram", "eig")},
                   "graph_records_identical": all(
                       a[i].rank == b[i].rank and a[i].reach.J_old == b[i].reach.J_old
                       and a[i].sigma_max == b[i].sigma_max
                       for a, b in zip(recs_p, recs_g) for i in range(2))}
    plan.close()
    out["seconds"] = tn
    out["normal_operator_gram_seconds"] = runs["normal"][0]
    out["fp64_data_path_seconds"] = td
    out["speedup_vs_fp64_data_path"] = td / tn
    out["max_rel_sigma_diff_class_vs_data"] = max(
        float(np.max(np.abs(np.array([a[i].sigma_max for i in range(2)]) -
                            np.array([b[i].sigma_max for i in range(2)])) /
                     np.array([b[i].sigma_max for i in range(2)])))
        for a, b in zip(rn, rd))
    out["rank_direct"] = [r[0].rank for r in rn]
    out["rank_resolved"] = [r[1].rank for r in rn]
    out["L_anchor_direct"] = [r[0].reach.L_anchor for r in rn]
    out["L_anchor_resolved"] = [r[1].reach.L_anchor for r in rn]
    out["J_old_direct"] = [round(r[0].reach.J_old, 3) for r in rn]
    out["J_old_resolved"] = [round(r[1].reach.J_old, 3) for r in rn]
    out["min_rank_margin"] = min(min(r[0].margin, r[1].margin) for r in rn)
    out["sigma_max_range"] = [min(min(r[0].sigma_max, r[1].sigma_max) for r in rn),
                              max(max(r[0].sigma_max, r[1].sigma_max) for r in rn)]
    out["sigma_min_range"] = [min(min(r[0].sigma_min_pos, r[1].sigma_min_pos) for r in rn),
                              max(max(r[0].sigma_min_pos, r[1].sigma_min_pos) for r in rn)]
    out["seconds_per_record"] = [round(r[i].seconds, 4) for r in rn for i in range(2)]
    out["seconds_split"] = {k: round(sum(getattr(r[i], "seconds_" + k) for r in rn for i in range(2)), 3)
                            for k in ("probe", "gram", "eig")}
    out["ranks_agree_between_paths"] = all(a[i].rank == b[i].rank and a[i].rank == c[i].rank
                                           for a, b, c in zip(rn, rd, runs["normal"][1])
                                           for i in range(2))
    # mechanism arms (Sec. 6.4): the unresolved image and the total-flux
    # readout of the resolved stack as whitened collapses with propagated
    # noise (Eq. 4); restricted Gram through the normal operator with the
    # collapse between the applies, FP64 eigenvalues, rank = #{sigma >= rho}
    mech = {}
    for name, mode in (("unresolved", rtt.MIX_UNRESOLVED), ("total_flux", rtt.MIX_TOTAL_FLUX)):
        torch.cuda.synchronize(device)
        t = time.perf_counter()
        Gs = torch.stack([rtt.gram_normal_mix(op, Q, mode) for op, Q in zip(ops, Qs)])
        ev = rtt.eigvals_sym_batched(Gs)
        torch.cuda.synchronize(device)
        sig = np.sqrt(np.maximum(ev, 0.0))
        ranks = [int(np.count_nonzero(sv >= 1.0)) for sv in sig]  # rho = 1
        # probe information of the mixed arm, then its reach and J_old (the
        # footprints of the summed orders; A_{0,0.999} of the direct order)
        rr = []
        for op in ops:
            info = rtt.probe_info_mix(op, mode, 7)
            rr.append(rtt.reach(op, info, 7, a0q=rtt.direct_age_quantile(op))[0])
        torch.cuda.synchronize(device)
        mech[name] = {"rank": ranks, "median_rank": float(np.median(ranks)),
                      "sigma_max_range": [float(sig[:, -1].min()), float(sig[:, -1].max())],
                      "L_anchor": [r.L_anchor for r in rr],
                      "J_old": [round(r.J_old, 3) for r in rr],
                      "median_J_old": float(np.median([r.J_old for r in rr])),
                      "seconds": round(time.perf_counter() - t, 3)}
    mech["resolved_median_rank"] = float(np.median(out["rank_resolved"]))
    mech["resolved_median_J_old"] = float(np.median(out["J_old_resolved"]))
    mech["direct_median_J_old"] = float(np.median(out["J_old_direct"]))
    mech["direct_median_rank"] = float(np.median(out["rank_direct"]))
    mech["never_above_resolved"] = all(u <= r and f <= r for u, f, r in zip(
        mech["unresolved"]["rank"], mech["total_flux"]["rank"], out["rank_resolved"]))
    # pairing-destroyed control (Sec. 6.4): each cell's delays permuted within
    # each order (seeded), the same rays, weights and source points; the
    # resolved arm's rank, reach and J_old through the class-Gram audit
    torch.cuda.synchronize(device)
    t = time.perf_counter()
    pdr = []
    for i, (w, tab) in enumerate(cells):
        n_e = int(np.asarray(tab["r"]).shape[0])
        op_pd = rtt.Operator(w, rtt.arm_table(tab, rtt.ARM_PAIRING_DESTROYED,
                                              I.uniforms(1000 + i, n_e)))
        recs, _ = rtt.rank_audit([op_pd], [None], (7,), mode=rtt.GRAM_CLASS_S224)
        pdr.append(recs[0][0])
        op_pd.close()
    mech["pairing_destroyed"] = {"rank": [r.rank for r in pdr],
                                 "L_anchor": [r.reach.L_anchor for r in pdr],
                                 "J_old": [round(r.reach.J_old, 3) for r in pdr],
                                 "median_J_old": float(np.median([r.reach.J_old for r in pdr])),
                                 "seconds_with_build": round(time.perf_counter() - t, 3)}
    # delay-only and spatial-only arms (Sec. 6.4): the rings keep their delays
    # with their source points moved to the direct quantile partners', or keep
    # their source points with the partners' delays; the resolved arm's rank,
    # reach and J_old through the class-Gram audit
    for name, kind in (("delay_only", rtt.ARM_DELAY_ONLY), ("spatial_only", rtt.ARM_SPATIAL_ONLY)):
        try:
            torch.cuda.synchronize(device)
            t = time.perf_counter()
            arm = []
            for w, tab in cells:
                op_a = rtt.Operator(w, rtt.arm_table(tab, kind))
                recs, _ = rtt.rank_audit([op_a], [None], (7,), mode=rtt.GRAM_CLASS_S224)
                arm.append(recs[0][0])
                op_a.close()
            mech[name] = {"rank": [r.rank for r in arm],
                          "L_anchor": [r.reach.L_anchor for r in arm],
                          "J_old": [round(r.reach.J_old, 3) for r in arm],
                          "median_J_old": float(np.median([r.reach.J_old for r in arm])),
                          "median_rank": float(np.median([r.rank for r in arm])),
                          "seconds_with_build": round(time.perf_counter() - t, 3)}
            if name == "delay_only":  # the scalar probe ignores the source point
                mech[name]["J_old_equals_resolved"] = mech[name]["J_old"] == out["J_old_resolved"]
        except Exception as exc:  # a measurement extra; report why it failed
            mech[name] = {"error": f"{type(exc).__name__}: {exc}"}
    out["mechanism_arms"] = mech
    # threshold sweep at the reconstruction geometry a = 0.5, i = 50 deg (Sec.
    # 3.3, Table 2): detectability depends on rho / SNR_0 only, so a threshold
    # rho at SNR_0 = 100 is rho = 1 on I(a) / rho^2; anchor-connected spans
    sweep = []
    for (w, _), op in zip(cells, ops):
        if abs(w.geometry.spin - 0.5) < 1e-9 and abs(w.geometry.incl_deg - 50.0) < 1e-9:
            inf = {m: rtt.probe_info(op, m) for m in (1, 7)}
            for rho in (10.0 / 3.0, 1.0, 1.0 / 3.0):
                sweep.append({"rho": round(rho, 3), "equivalent_snr0": round(100.0 / rho, 1),
                              "direct_span": rtt.reach(op, inf[1] / rho ** 2, 1)[0].L_anchor,
                              "resolved_span": rtt.reach(op, inf[7] / rho ** 2, 7)[0].L_anchor})
    out["threshold_sweep_a0.5_i50"] = sweep
    # localized directional reach (Sec. 3.3 Eq. 14) at the same geometry: the
    # oldest age at which one of the 28 normalised directions passes (rho = 1)
    loc = {}
    for (w, _), op in zip(cells, ops):
        if abs(w.geometry.spin - 0.5) < 1e-9 and abs(w.geometry.incl_deg - 50.0) < 1e-9:
            t = time.perf_counter()
            for name, m in (("direct", 1), ("resolved", 7)):
                il = rtt.probe_info_local(op, m)
                ok = np.nonzero(np.any(il >= 1.0, axis=1))[0]
                loc[name] = float(rtt.AGES[ok[-1]]) if ok.size else None
            loc["seconds"] = round(time.perf_counter() - t, 3)
    out["localized_reach_a0.5_i50"] = loc
    for op in ops:
        op.close()
    return out


def run_ladder(device):
    """The class ladder of Sec. 7-8 (Eq. 43, Tables 4-5): at the reconstruction
    geometry (kerr256: a = 0.5, i = 50 deg) and on schw32 (whose history is
    older than the direct footprint, so Theorem 4.1's zero columns appear),
    per class: dimension, exactly-zero direct columns (zero diagonal of the
    direct Gram), operational rank sigma >= 1 for the direct and resolved
    arms, the spectrum's extremes; FP64 normal-operator Gram, FP64
    eigenvalues."""
    import torch

    from paper_2609_05528_b300 import build, rtt
    from paper_2609_05528_b300 import inputs as I
    build.build()
    kinds = [("S224", rtt.CLASS_S224), ("S448T", rtt.CLASS_S448T), ("S528S", rtt.CLASS_S528S),
             ("S1056ST", rtt.CLASS_S1056ST), ("L224", rtt.CLASS_L224), ("L448", rtt.CLASS_L448),
             ("L1056", rtt.CLASS_L1056)]
    out = {"ladder": "Sec. 7-8 class ladder (Eq. 43)", "rho": 1.0, "snr0": 100.0, "workloads": []}
    for w in (I.kerr256(), I.schw32()):
        tab = rtt.rtt_trace_rays(w.geometry.spin, w.geometry.incl_deg, w.grid, I.screen_samples(w))
        op = rtt.Operator(w, tab)
        rows = []
        for name, kind in kinds:
            torch.cuda.synchronize(device)
            t = time.perf_counter()
            Q = rtt.synth_class(op, kind)
            rec = {"class": name, "dim": int(Q.shape[2])}
            for arm, tag in ((1, "direct"), (7, "resolved")):
                torch.cuda.synchronize(device)
                tg = time.perf_counter()
                G = rtt.gram(op, Q, arm, mode=rtt.GRAM_NORMAL)
                diag_zero = int((torch.diagonal(G) == 0).sum())
                ev = rtt.eigvals_sym_batched(G[None])[0]
                sig = np.sqrt(np.maximum(ev, 0.0))
                rec[tag + "_gram_and_eig_s"] = round(time.perf_counter() - tg, 3)
                rec[tag + "_rank"] = int(np.count_nonzero(sig >= 1.0))
                rec[tag + "_zero_columns"] = diag_zero
                rec[tag + "_sigma_max"] = float(sig[-1])
                rec[tag + "_sigma_min_at_or_above_rho"] = float(sig[sig >= 1.0].min()) if (sig >= 1.0).any() else None
                del G
            # the adaptive randomized range finder (blocks of 256 seeded
            # Gaussian vectors, FP64 Ritz values) on the resolved arm
            d = int(Q.shape[2])
            nbk = (d + 255) // 256 + 1
            omega = I.normals(7000 + d, d * 256 * nbk).reshape(d, 256 * nbk)
            torch.cuda.synchronize(device)
            tr = time.perf_counter()
            sig_rf, rank_rf, blocks = rtt.range_finder(op, Q, omega, 7, 256, 1.0)
            rec["range_finder_resolved"] = {"rank": rank_rf, "blocks": blocks, "basis": int(sig_rf.shape[0]),
                                            "seconds": round(time.perf_counter() - tr, 3)}
            del Q
            torch.cuda.synchronize(device)
            rec["seconds"] = round(time.perf_counter() - t, 3)
            rows.append(rec)
        # old-structure subspace (Sec. 7, Eq. 41): the compact classes'
        # temporal functions with exactly zero direct response in every
        # spatial column, and, within each, the spatial coefficients
        # orthogonal to the constant level (the four radial functions with
        # the constant azimuthal mode sum to psi = 1); ranks of the direct,
        # resolved and order-summed (unresolved image) arms on it
        old = []
        for name, kind in kinds:
            if not name.startswith("L"):
                continue
            Q = rtt.synth_class(op, kind)
            d = int(Q.shape[2])
            nr, na = (4, 7) if d in (224, 448) else (6, 11)
            nt = d // (nr * na)
            Gd = rtt.gram(op, Q, 1, mode=rtt.GRAM_NORMAL).cpu().numpy()
            Gr = rtt.gram(op, Q, 7, mode=rtt.GRAM_NORMAL).cpu().numpy()
            Gu = rtt.gram_normal_mix(op, Q, rtt.MIX_UNRESOLVED, 7).cpu().numpy()
            del Q
            zero = np.diag(Gd) == 0.0
            old_m = [m for m in range(nt) if all(zero[sp * nt + m] for sp in range(nr * na))]
            if not old_m:
                old.append({"class": name, "old_temporal_functions": 0})
                continue
            lev = np.zeros(nr * na)
            lev[[i * na for i in range(nr)]] = 1.0
            lev /= np.linalg.norm(lev)
            B = np.linalg.svd(np.eye(nr * na) - np.outer(lev, lev))[0][:, :nr * na - 1]
            C = np.zeros((d, len(old_m) * (nr * na - 1)))
            for j, m in enumerate(old_m):
                for sp in range(nr * na):
                    C[sp * nt + m, j * (nr * na - 1):(j + 1) * (nr * na - 1)] = B[sp]
            Gs = torch.from_numpy(np.stack([C.T @ G @ C for G in (Gd, Gr, Gu)])).to(device)
            ev = rtt.eigvals_sym_batched(Gs)
            sig = np.sqrt(np.maximum(ev, 0.0))
            old.append({"class": name, "old_temporal_functions": len(old_m),
                        "dim": int(C.shape[1]),
                        "direct_rank": int(np.count_nonzero(sig[0] >= 1.0)),
                        "direct_sigma_max": float(sig[0][-1]),
                        "resolved_rank": int(np.count_nonzero(sig[1] >= 1.0)),
                        "order_summed_rank": int(np.count_nonzero(sig[2] >= 1.0))})
        out["workloads"].append({"workload": w.name, "spin": w.geometry.spin,
                                 "incl_deg": w.geometry.incl_deg, "classes": rows,
                                 "old_structure": old})
        op.close()
    return out


def run_recovery(device, n_test: int = 60, n_val: int = 20, max_iter: int = 400,
                 tol: float = 1e-6):
    """Held-out recovery (Sec. 9) on Kerr a=0.94, i=50 deg at kerr256 sizes:
    60 test and 20 validation histories (1-4 flaring hot spots plus a
    log-normal level), data = scale A x_true + N(0, 1) whitened noise, the
    direct-only arm using the n=0 rows of the same draw.  Ridge by batched CG
    on A^T A + lambda I for 8 lambdas (validation-selected), and TSVD in S224
    at the operational rank.  Error = ||x_hat - x_true|| / ||x_true|| on the
    grid x hat coefficients."""
    import torch

    from paper_2609_05528_b300 import inputs as I
    from paper_2609_05528_b300 import rtt
    lambdas = 10.0 ** np.arange(-3, 5)
    L = len(lambdas)
    w = I.recovery()
    tab = rtt.rtt_trace_rays(w.geometry.spin, w.geometry.incl_deg, w.grid, I.screen_samples(w))
    op = rtt.Operator(w, tab)
    R0 = int(op.info.rows_per_order[0])
    sets = {}
    for name, seeds, nseed in (("test", range(1000, 1000 + n_test), 11),
                               ("val", range(2000, 2000 + n_val), 12)):
        xt = torch.from_numpy(I.recovery_batch(w, seeds).astype(np.float32)).to(device)
        d = op.apply_A(xt)
        d += torch.from_numpy(I.noise(tuple(d.shape), nseed).astype(np.float32)).to(device)
        sets[name] = (xt, d)

    def errors(xh, xt, per):
        n = xt.shape[2]
        xh = xh.reshape(xt.shape[0], xt.shape[1], n, per).double()
        diff = xh - xt.double()[..., None]
        return (diff.pow(2).sum((0, 1)).sqrt() / xt.double().pow(2).sum((0, 1)).sqrt()[:, None]).cpu().numpy()

    out = {"workload": "recovery: Kerr a=0.94 i=50deg, kerr256 sizes, 60 test + 20 validation "
                       "histories, SNR0=100 whitened noise, lambdas 1e-3..1e4",
           "arms": {}}
    Q = rtt.synth_class(op, rtt.CLASS_S224)
    err = {}
    for arm in (1, 7):
        rec = {}
        for name in ("val", "test"):
            xt, d = sets[name]
            data = (d[:R0] if arm == 1 else d).contiguous()
            torch.cuda.synchronize(device)
            t = time.perf_counter()
            xh, it, rel = rtt.solve_ridge(op, data, lambdas, arm, max_iter=max_iter, tol=tol,
                                          refresh_every=25, raise_on_stall=False)
            torch.cuda.synchronize(device)
            rec[name] = {"seconds": time.perf_counter() - t, "iterations": it,
                         "max_relres": float(np.max(rel)), "columns": int(xh.shape[2]),
                         "err": errors(xh, xt, L)}
            del xh
        li = int(np.argmin(np.median(rec["val"]["err"], axis=0)))
        # TSVD in S224 at the operational rank of this arm
        t = time.perf_counter()
        G = rtt.gram(op, Q, arm, rtt.GRAM_NORMAL)
        ev, V, _ = rtt.eig_sym(G)
        sig = np.sqrt(np.maximum(ev, 0.0))
        rank = int(np.count_nonzero(sig >= 1.0))  # rho = 1 (Eq. 31)
        xt, d = sets["test"]
        data64 = (d[:R0] if arm == 1 else d).double().contiguous()
        xts = rtt.solve_tsvd(op, Q, V, ev, rank, data64, arm)
        torch.cuda.synchronize(device)
        t_tsvd = time.perf_counter() - t
        e_tsvd = errors(xts, xt, 1)[:, 0]
        err[arm] = rec["test"]["err"][:, li]
        out["arms"]["direct" if arm == 1 else "resolved"] = {
            "lambda": float(lambdas[li]),
            "ridge_median_err": float(np.median(err[arm])),
            "ridge_median_err_per_lambda": [round(float(v), 4) for v in np.median(rec["test"]["err"], axis=0)],
            "ridge_seconds_test": round(rec["test"]["seconds"], 3),
            "ridge_seconds_val": round(rec["val"]["seconds"], 3),
            "ridge_iterations": rec["test"]["iterations"],
            "ridge_max_fp64_relres": rec["test"]["max_relres"],
            "ridge_columns": rec["test"]["columns"],
            "tsvd_rank": rank, "tsvd_median_err": float(np.median(e_tsvd)),
            "tsvd_seconds": round(t_tsvd, 3)}
    red = 1.0 - err[7] / err[1]
    out["median_paired_reduction"] = float(np.median(red))
    out["histories_improved"] = int(np.count_nonzero(red > 0))
    op.close()
    return out


_ORACLE_TABLES = {}


def oracle_sample(w, row_block: int = 4, every: int = 8):
    """The oracle's ray table on a bounded, stratified sample of the screen:
    every `every`-th block of `row_block` pixel rows (1 / every of the
    screen).  Built once per workload (untimed)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O

    from paper_2609_05528_b300 import inputs as I
    key = (w.name, row_block, every)
    if key not in _ORACLE_TABLES:
        s = I.screen_samples(w)
        iy = s.pixel // w.geometry.nx
        m = (iy // row_block) % every == 0
        sub = I.ScreenSamples(s.alpha[m], s.beta[m], s.pixel[m], s.n_sub[m], s.d_omega_pixel)
        _ORACLE_TABLES[key] = O.build_table(w, sub)
    return _ORACLE_TABLES[key], every


def oracle_pairs_per_s(w, budget_s: float = 12.0, threads: int | None = None):
    """Time the FP64 CPU oracle (as it stands) on A + A^T for one history on
    the stratified screen sample of `oracle_sample`, on all host cores or on
    `threads` of them.  Returns (history-applies/s scaled to the whole
    screen, threads used, pairs timed, sample description)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O

    from paper_2609_05528_b300 import inputs as I
    tab, every = oracle_sample(w)
    scl = O.scale(tab)
    x = I.uniform_batch(w, [1])
    all_cores = O.max_threads()
    if threads:
        O.set_threads(threads)
    try:
        cores = O.max_threads()
        n = 0
        t0 = time.perf_counter()
        while True:
            yv = O.apply_A(w, tab, x, scl)
            O.apply_AT(w, tab, yv, scl)
            n += 1
            if time.perf_counter() - t0 > budget_s:
                break
        dt = time.perf_counter() - t0
    finally:
        O.set_threads(all_cores)
    sample = (f"{n} x (A + A^T) on 1 history, FP64 oracle, on every {every}th block of 4 pixel "
              f"rows ({tab.n_rows} data rows, 1/{every} of the screen); value scaled by 1/{every}")
    return n / dt / every, cores, n, sample


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-audit", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the batch sweep leg")
    ap.add_argument("--sweep", action="store_true",
                    help="print the stress1024 batch sweep (one JSON line per geometry) and exit")
    ap.add_argument("--recovery", action="store_true",
                    help="print the held-out recovery leg (ridge + TSVD) as one JSON line and exit")
    ap.add_argument("--ladder", action="store_true",
                    help="print the class-ladder audit (Sec. 7-8) as one JSON line and exit")
    ap.add_argument("--audit", action="store_true",
                    help="print the 12-geometry audit leg as one JSON line and exit")
    ap.add_argument("--gemm", type=int, nargs=3, metavar=("K", "M", "N"),
                    help="time rtt_gemm_tn_f64 (C = A^T B, A: K x M, B: K x N, N(0,1) FP64) against "
                         "cuBLAS DGEMM, print one JSON line and exit")
    ap.add_argument("--batch", type=int, default=8, help="history batch of the --profile step")
    ap.add_argument("--variant", default="",
                    help="--profile: fwd_kernel,fwd_bc,fwd_half,adj_kernel,fwd_order,fwd_cols,adj_cols "
                         "instead of autotuning")
    ap.add_argument("--profile", choices=["stress1024", "kerr256"],
                    help="for ncu: build the workload at batch 8, autotune, warm up, run --steps "
                         "A + A^T steps inside the NVTX range bench_timed, and exit")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_2609_05528_b300 import inputs as I

    if args.impl == "reference":
        # the reference arm is the FP64 CPU oracle, timed on the host cores
        if rank != 0:
            return
        w = I.stress1024(0.94)
        vals = []
        for _ in range(max(1, args.steps)):
            v, cores, n, sample = oracle_pairs_per_s(w, budget_s=10.0)
            vals.append(v)
            if len(vals) >= 2:
                break
        v = float(np.mean(vals))
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
                          "n_gpus": 1, "steps": len(vals), "warmup": 0,
                          "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": WORKLOAD, "batch": 1,
                                     "sample": "one history per pass on a stratified 1/8 of the "
                                               "screen (the unit is per history, so the batch does "
                                               "not change it)",
                                     "parallelism": f"host cores x{cores}"},
                          "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores,
                                           "kind": "oracle", "sample": sample},
                          "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = torch.device("cuda", local)
    if args.sweep:
        if rank == 0:
            torch.cuda.set_device(device)
            for line in run_sweep(device):
                print(json.dumps(line))
        return
    if args.recovery:
        if rank == 0:
            torch.cuda.set_device(device)
            print(json.dumps(run_recovery(device)))
        return
    if args.ladder:
        if rank == 0:
            torch.cuda.set_device(device)
            print(json.dumps(run_ladder(device)))
        return
    if args.audit:
        if rank == 0:
            torch.cuda.set_device(device)
            print(json.dumps(run_audit(device)))
        return
    if args.gemm:
        if rank == 0:
            torch.cuda.set_device(device)
            print(json.dumps(run_gemm(args, device)))
        return
    if args.profile:
        if rank == 0:
            torch.cuda.set_device(device)
            print(json.dumps(run_profile_case(args, device)))
        return
    out = run_ours(args, rank, world, device)
    if rank == 0 and world == 1 and not args.no_audit:
        out["audit"] = run_audit(device)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            w5 = I.stress1024(0.94)
            v, cores, n, sample = oracle_pairs_per_s(w5)
            v1, _, n1, sample1 = oracle_pairs_per_s(w5, budget_s=6.0, threads=1)
            out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                   "sample": sample + ", ~12 s",
                                   "single_core": {"value": v1, "unit": UNIT, "cores": 1,
                                                   "sample": sample1 + ", ~6 s"}}
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
