"""Benchmark: immersed-boundary steps/s on the 256^3 + ~1M-marker synthetic cochlea.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]

One JSON line on rank 0.  A step is one full IB time step (forces, bin sort,
spread, FFT fluid solve with projection, interpolation and move) of the
FP32 path (FP32 fields, FFTs and forces; FP64 reference positions plus FP32
displacements).  `value` is device-timed with CUDA events on the library's
stream, inputs resident in HBM; the working set (~1.1 GB) exceeds the 129 MB
L2, so no flush is needed between steps.  `e2e` drives the same steps through
the C ABI with host buffers: per step the marker positions go host->device
(ib_set_state), one step runs, and the new positions come back (ib_get_state).
`roofline` is the top single-kernel stage's algorithmic bytes over its mean
event time; `step_roofline` is every stage's algorithmic bytes over the
timed step.

Multi-GPU: the step does not shard (one periodic FFT grid); N > 1 runs N
independent replicas, one per GPU (weak scaling), no collective on the data
path.  `--impl reference` times the FP64 CPU oracle on the host's cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IB steps/s @256^3+1M markers (FP32 vs FP64 GPU), adjoint/fwd ratio, %HBM peak"
WORKLOAD = ("cochlea256: 256^3 periodic grid (h = 1/256 cm), 993,216 markers = 2048x192 helicoidal membrane "
            "+ 600,000 tethered wall markers, 20,000 fibers, 4 kHz body-force tone, dt = 30 ns")


def workload_config(p, world: int) -> dict:
    """The `config` object of both arms' JSON lines: the workload and how it is run."""
    return {"workload": WORKLOAD, "grid": [int(v) for v in p.grid.n], "markers": int(p.structure.m),
            "springs": int(len(p.structure.spring_k)),
            "l2": "working set ~1.1 GB > 129 MB L2; no flush between steps",
            "parallelism": f"{world} independent replica(s), one per GPU"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clocks not sampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# Stages that are one kernel launch each (their event time is the kernel's).
SINGLE_KERNEL_STAGES = {"fft_x_fwd": "k_xfwd", "fft_x_inv": "k_xinv", "fft_z_proj": "k_zproj",
                        "fft_y_fwd": "k_ypass", "fft_y_inv": "k_ypass", "records": "k_records",
                        "keys": "k_keys_state"}

# DRAM bytes (read + write) per launch from one ncu capture of the kernel as
# it stands, with the capture it came from; drop an entry when its kernel
# changes (the line then reports traffic null).
DRAM_TRAFFIC = {"k_xfwd": (266313728 + 162198272,
                           "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_xfwd<float, 256, 4> on this "
                           "workload (bench.py --steps 5), the kernel as built loading only the upwind x and z "
                           "neighbours, the body-force factor converted once per warp"),
                "k_zproj": (203452928 + 144030208,
                            "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_zproj<float, 256, 8> on this "
                            "workload (bench.py --steps 5), the kernel as built loading and storing in FFT order"),
                "k_xinv": (202931968 + 149302528,
                           "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_xinv<float, 256, 4> on this "
                           "workload (bench.py --steps 5), the kernel as built with per-thread fixed lines"),
                "k_records": (80161024 + 26139648,
                              "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_records on this workload "
                              "(bench.py --steps 5)")}


def stage_bytes(name: str, G: int, n: int, m: int, touched_tiles: int) -> float:
    """Algorithmic HBM bytes of one stage at FP32 (each array read or written once)."""
    S = 8 * (n * n) * (n // 2 + 1)            # one complex half spectrum incl. the kx = n/2 plane
    touched_cells = touched_tiles * 512
    ntiles = G // 512
    passes = max(1, math.ceil((math.ceil(math.log2(G)) - 9) / 8))   # 8-bit radix passes over the tile bits
    chunks = -(-m // 1024)                                            # radix blocks of 1024 keys
    return {
        "keys": m * (12 + 12 + 12 + 4 + 4 + 12),             # cell0, r0, d in; key, tile count, rfrac out
        # per pass: digit counts read the keys, the scatter reads keys + ids and
        # writes them (the first pass has no ids to read); the digit-count scans
        # (write, read, write); the bin plan over the tiles and the work items
        "sort": passes * 20 * m - 4 * m + passes * 3 * 4 * 256 * chunks + 16 * ntiles + 8 * (ntiles + -(-m // 512)),
        "records": m * (4 + 12 + 12 + 64) + 24 * m,           # perm, rfrac, d, record out; links (~2/marker)
        "spread": m * 64 + 12 * touched_cells,                # records once, F on touched tiles
        "fft_x_fwd": 3 * 4 * G + 3 * S + 12 * touched_cells,  # u in, spectrum out, F in on touched tiles
        "fft_y_fwd": 3 * 2 * S,
        "fft_z_proj": 3 * 2 * S,
        "fft_y_inv": 3 * 2 * S,
        "fft_x_inv": 3 * S + 3 * 4 * G,
        "interp": m * (64 + 4 + 4 + 48) + 12 * touched_cells,  # record, key, perm, d = hi + lo r+w; u on touched cells
    }[name]


def replica_throughput(ms_local: float, steps: int, dist=None, device=None):
    """Whole-job steps/s of independent replicas: every rank ran `steps` steps
    in ms_local ms; the job time is the slowest rank's (max over ranks)."""
    import torch
    world = dist.get_world_size() if dist else 1
    t = torch.tensor([float(ms_local)], device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return world * steps / (ms / 1e3), ms


def run_gpu(args):
    import numpy as np
    import torch

    from paper_math_0301321_gb300 import synth
    from paper_math_0301321_gb300.binding import Context

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()

    p = synth.cochlea256()
    n = p.grid.n[0]
    G, m = p.grid.G, p.structure.m
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = Context(p.grid, prec="fp32", stream=stream)
        ctx.set_structure(p.structure)
        ctx.set_state(p.u, p.X, 0.0)
        ctx.step(args.warmup)
        ctx.sync()  # raises on non-finite marker velocities
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            t_wall = time.perf_counter()
            e0.record(stream)
            ctx.step(args.steps)
            e1.record(stream)
            e1.synchronize()
            t_wall = time.perf_counter() - t_wall
        ctx.sync()
        barrier()
        torch.cuda.synchronize()
        value, ms = replica_throughput(e0.elapsed_time(e1), args.steps, dist, "cuda")
        ms_per_step = ms / args.steps
        gpu_launches = args.steps * kernels_per_step(n)

        # per-stage device times (eager launches, events on the same stream)
        nprof = max(3, min(args.steps, 20))
        stage_ms, tiles = ctx.profile(nprof)
        u_chk, X_chk, t_chk = ctx.get_state()
        finite = bool(torch.isfinite(u_chk).all().item() and torch.isfinite(X_chk).all().item())

        # end to end through the C ABI with pinned host buffers
        X_host = X_chk.cpu().numpy().astype(np.float64)
        X_pin = torch.from_numpy(X_host).pin_memory()
        X_out = torch.empty_like(X_pin).pin_memory()
        from paper_math_0301321_gb300 import binding
        import ctypes as C
        ne2e = max(3, min(args.steps, 20))
        ctx_h = Context(p.grid, prec="fp32", device=False, stream=stream)
        ctx_h.set_structure(p.structure)
        ctx_h.set_state(p.u, p.X, 0.0)
        ctx_h.step(1)
        ctx_h.sync()
        tt = C.c_double()
        lib = ctx_h.lib
        t0 = time.perf_counter()
        for i in range(ne2e):
            binding._check(lib.ib_set_state(ctx_h.h, None, C.c_void_p(X_pin.data_ptr()), float(i) * p.grid.dt))
            binding._check(lib.ib_step(ctx_h.h, 1))
            binding._check(lib.ib_get_state(ctx_h.h, None, C.c_void_p(X_out.data_ptr()), C.byref(tt)))
        e2e_s = time.perf_counter() - t0
        ctx_h.close()
        e2e_value = world * ne2e / e2e_s

        # the reverse step on this workload: one ib_adjoint_step about the
        # current state with u^{n+1} given (device buffers), against the step
        adj256 = None
        if not args.skip_adjoint:
            snap = ctx.new_snapshot()
            ctx.snapshot_save(snap)
            ctx.step(1)
            nxt = ctx.new_snapshot()
            ctx.snapshot_save(nxt)
            ctx.snapshot_load(snap)
            lam_u = torch.randn((3,) + ctx.n[::-1], dtype=torch.float32, device="cuda")
            lam_D = torch.randn((3, m), dtype=torch.float64, device="cuda")
            gb = torch.zeros(len(p.structure.bend_b), dtype=torch.float64, device="cuda")
            outs = (torch.empty_like(lam_u), torch.empty_like(lam_D))
            u1 = ctx.snapshot_velocity(nxt)
            for _ in range(3):
                ctx.adjoint_step(lam_u, lam_D, u_np1=u1, grad_b=gb, out=outs)
            ka = 10
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(ka):
                ctx.adjoint_step(lam_u, lam_D, u_np1=u1, grad_b=gb, out=outs)
            e1.record(stream)
            e1.synchronize()
            adj_ms = e0.elapsed_time(e1) / ka
            adj256 = {"adjoint_step_ms": round(adj_ms, 4), "fwd_step_ms": round(ms_per_step, 4),
                      "ratio": round(adj_ms / ms_per_step, 3),
                      "how": "ib_adjoint_step with u^{n+1} given, device buffers, CUDA events; "
                             "forward = the timed graph step above"}
            del snap, nxt, lam_u, lam_D, outs, u1

        # one FP32 step of this workload from a perturbed state, kept for the
        # per-field error against the oracle's step (cpu_baseline)
        D1, u1s, t1 = perturbed_state(p)
        ctx.set_state(u1s, None, t1)
        ctx.set_displacement(D1)
        ctx.step(1)
        ug1, _, _ = ctx.get_state()
        fp32_one = (ug1.cpu().numpy().astype(np.float64), ctx.get_displacement().cpu().numpy())
        cufft = cufft_crosscheck(p, stream, stage_ms)

        # the tensor-core y passes (IB_FP32_TCFFT) on the same workload: steps/s
        # and one step from the perturbed state for the per-field error
        tc = None
        if not args.skip_tc:
            ctx.close()
            torch.cuda.empty_cache()
            ctx = Context(p.grid, prec="fp32_tcfft", stream=stream)
            ctx.set_structure(p.structure)
            ctx.set_state(p.u, p.X, 0.0)
            ctx.step(args.warmup)
            ctx.sync()
            ktc = max(20, min(args.steps, 200))
            e0.record(stream)
            ctx.step(ktc)
            e1.record(stream)
            e1.synchronize()
            ctx.sync()
            tc_ms = e0.elapsed_time(e1) / ktc
            tc_stages, _ = ctx.profile(nprof)
            ctx.set_state(u1s, None, t1)
            ctx.set_displacement(D1)
            ctx.step(1)
            ug1, _, _ = ctx.get_state()
            tc_one = (ug1.cpu().numpy().astype(np.float64), ctx.get_displacement().cpu().numpy())
            tc = {"value": round(1e3 / tc_ms, 2), "unit": "IB steps/s", "ms_per_step": round(tc_ms, 4),
                  "steps": ktc, "fft_y_fwd_ms": round(tc_stages["fft_y_fwd"], 4),
                  "fft_y_inv_ms": round(tc_stages["fft_y_inv"], 4),
                  "how": "IB_FP32_TCFFT: the y passes as radix-16 DFT products on tcgen05 (split BF16, FP32 "
                         "accumulation in tensor memory), every other stage as the FP32 step"}

        # the plain FP64 GPU step on the same inputs
        fp64 = None
        if not args.skip_fp64:
            ctx.close()
            torch.cuda.empty_cache()
            c64 = Context(p.grid, prec="fp64", stream=stream)
            c64.set_structure(p.structure)
            c64.set_state(p.u, p.X, 0.0)
            c64.step(2)
            c64.sync()
            k64 = 20
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            c64.step(k64)
            f1.record(stream)
            f1.synchronize()
            c64.sync()
            fp64 = {"value": world * k64 / (f0.elapsed_time(f1) / 1e3), "steps": k64}
            c64.close()

        # the widened model (half-cube grid, windows, probe)
        nxt = None
        if not args.skip_next:
            torch.cuda.empty_cache()
            nxt = next_leg(500)

        # the tone-sweep batch
        batch = None
        if not args.skip_batch:
            torch.cuda.empty_cache()
            batch = batch_leg(200)

        # the reverse step: its own workload (the adjoint's), FP32
        adjoint = None
        if not args.skip_adjoint:
            torch.cuda.empty_cache()
            adjoint = adjoint_leg(stream)

    pk, src = peaks()
    tot = sum(stage_ms.values())
    # the dominant kernel: the longest stage that is a single kernel launch
    dom = max(SINGLE_KERNEL_STAGES, key=lambda k: stage_ms[k])
    kern = SINGLE_KERNEL_STAGES[dom]
    achieved = stage_bytes(dom, G, n, m, tiles) / (stage_ms[dom] / 1e3) / 1e9
    stages = {k: {"ms": round(v, 4), "share": round(v / tot, 4),
                  "gbs": round(stage_bytes(k, G, n, m, tiles) / (v / 1e3) / 1e9, 1),
                  "frac": round(stage_bytes(k, G, n, m, tiles) / (v / 1e3) / 1e9 / pk["hbm_gbs"], 4)}
              for k, v in stage_ms.items()}
    step_bytes = sum(stage_bytes(k, G, n, m, tiles) for k in stage_ms)
    out = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "IB steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded generator, no datasets)",
        "config": workload_config(p, world),
        "precision": "FP32 fields/forces/FFTs, FP64 reference positions + FP32 displacements",
        "roofline": {"bound": "hbm", "kernel": kern, "stage": dom, "achieved": round(achieved, 1),
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / pk["hbm_gbs"], 4),
                     "peak_source": f"{src} hbm_gbs (burst copy)",
                     "algorithmic_bytes": stage_bytes(dom, G, n, m, tiles),
                     "traffic": DRAM_TRAFFIC.get(kern, (None, None))[0],
                     "traffic_source": DRAM_TRAFFIC.get(kern, (None, "no capture of the current kernel"))[1]},
        "stages": stages,
        # the whole step: every stage's algorithmic bytes over the timed (graph) step time
        "step_roofline": {"algorithmic_bytes": round(step_bytes), "achieved": round(step_bytes / ms_per_step / 1e6, 1),
                          "peak": pk["hbm_gbs"], "unit": "GB/s",
                          "frac": round(step_bytes / ms_per_step / 1e6 / pk["hbm_gbs"], 4)},
        "active_tiles": tiles,
        "gpu_launches": gpu_launches,
        "e2e": {"value": round(e2e_value, 2), "unit": "IB steps/s", "h2d_bytes_per_step": 24 * m + 8,
                "d2h_bytes_per_step": 24 * m + 8 + 4,
                "how": "per step: ib_set_state(X host->device) + ib_step(1) + ib_get_state(X device->host), "
                       "pinned host buffers, wall clock"},
        "fp64_gpu": fp64,
        "adjoint": {"cochlea256": adj256, "gradient_workload": adjoint},
        "batch": batch,
        "next": nxt,
        "finite": finite,
        "clocks": clk.summary(),
    }
    out["cufft_crosscheck"] = cufft
    out["tcfft"] = tc
    if rank == 0 and world == 1 and not args.skip_cpu:
        out["cpu_baseline"], (Do, uo) = cpu_baseline(p)
        D1, u1s, _ = perturbed_state(p)

        def rel(a, b):
            return float(np.linalg.norm(a - b) / np.linalg.norm(b))

        def mrel(a, b):
            return float(np.abs(a - b).max() / np.abs(b).max())
        if tc is not None:
            ug, Dg = tc_one
            tc["error_vs_oracle"] = {"u": rel(ug, uo), "dX": rel(Dg - D1, Do - D1), "u_max_elem": mrel(ug, uo),
                                     "dX_max_elem": mrel(Dg - D1, Do - D1)}
        ug, Dg = fp32_one
        out["error_vs_oracle"] = {
            "u": rel(ug, uo), "dX": rel(Dg - D1, Do - D1), "u_max_elem": mrel(ug, uo), "dX_max_elem": mrel(Dg - D1, Do - D1),
            "how": "one FP32 GPU step vs one FP64 oracle step from the same state (membrane bump 1e-7 cm + "
                   "2e-8 cm noise, smooth 0.1 cm/s velocity): norm-wise relative error of u^{n+1} and of the "
                   "displacement increment X^{n+1} - X^n, and the largest element error over the largest element"}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def kernels_per_step(n: int) -> int:
    """Kernels the library launches per step (all its own), for the launch count claim."""
    G = n ** 3
    bits = max(1, (G - 1).bit_length()) - 9          # tile bits of the cell key (8^3 tiles)
    passes = 1 if bits <= 0 else (bits + 7) // 8     # 8-bit LSD radix passes
    keys = 1
    sort = passes * (1 + 2 + 1)                      # hist, 2-kernel scan, scatter
    bins = 2                                         # bin sums, fill
    records = 1
    spread = 3                                       # touched tiles, scatter, gather
    fluid = 5                                        # x-fwd, y, z + projection, y inverse, x inverse
    interp = 2                                       # interp, move
    return keys + sort + bins + records + spread + fluid + interp


def next_leg(steps: int):
    """The widened model: steps/s of the 256x256x128 half-cube cochlea and of
    the 128^3 cochlea with its windows and stapes load (FP32, graph steps,
    CUDA events), and the cost of recording the centre line every 10th step."""
    import numpy as np
    import torch

    from paper_math_0301321_gb300 import synth
    from paper_math_0301321_gb300.binding import Context

    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(ctx, k):
        ctx.step(5)
        torch.cuda.synchronize()
        e0.record(s)
        ctx.step(k)
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    out = {}
    for name, p in (("halfcube", synth.cochlea_halfcube()), ("windows128", synth.cochlea_windows())):
        ctx = Context(p.grid, prec="fp32")
        ctx.set_structure(p.structure)
        ctx.set_state(p.u, None, 0.0)
        ms = timed(ctx, steps)
        row = {"grid": list(p.grid.n), "markers": p.structure.m, "ms_per_step": round(ms, 4),
               "steps_per_s": round(1e3 / ms, 2)}
        if name == "windows128":
            cl = p.structure.centerline
            ctx.set_probe(cl, p.structure.normal0[:, cl], every=10, capacity=max(1, steps // 10 + 10))
            ms_p = timed(ctx, steps)
            ctx.read_probe()
            row["probe_every10_ms_per_step"] = round(ms_p, 4)
            row["probe_overhead"] = round(ms_p / ms - 1.0, 4)
        ctx.sync()
        ctx.close()
        out[name] = row
    return out


def batch_leg(steps: int):
    """The tone sweep: 48 independent FP32 instances (grids from {64, 96,
    128}^3, membranes 256x24 or 512x48, 200k wall markers each, 200 Hz -
    12 kHz) advanced by one graph launch per step (ib_batch), tile shapes
    from ib_batch_autotune; against the same instances stepped one after
    another (each its own graph)."""
    import torch

    from paper_math_0301321_gb300 import synth
    from paper_math_0301321_gb300.binding import Batch, Context

    probs = synth.tone_sweep()
    ctxs = []
    for p in probs:
        c = Context(p.grid, prec="fp32")
        c.set_structure(p.structure)
        c.set_state(p.u, None, 0.0)
        ctxs.append(c)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # one after another
    for c in ctxs:
        c.step(2)
    torch.cuda.synchronize()
    k_seq = max(5, steps // 4)
    e0.record(s)
    for c in ctxs:
        c.step(k_seq)
    e1.record(s)
    e1.synchronize()
    seq_ms = e0.elapsed_time(e1) / k_seq
    # batched
    b = Batch(ctxs, steps_per_launch=1)
    t0 = time.perf_counter()
    b.autotune(reps=3)
    tune_s = time.perf_counter() - t0
    b.step(3)
    b.sync()
    e0.record(s)
    b.step(steps)
    e1.record(s)
    e1.synchronize()
    b.sync()
    ms = e0.elapsed_time(e1) / steps
    points = sum(p.grid.G for p in probs)
    markers = sum(p.structure.m for p in probs)
    tuning = ctxs[0].get_tuning()
    b.close()
    for c in ctxs:
        c.close()
    n = len(probs)
    return {
        "workload": f"tone sweep: {n} instances, grids from {{64,96,128}}^3, membranes 256x24 / 512x48, "
                    f"200k wall markers each ({markers} markers, {points} grid points in all), "
                    "200 Hz - 12 kHz, dt = 30 ns, FP32",
        "steps": steps,
        "ms_per_batch_step": round(ms, 4),
        "instance_steps_per_s": round(n / (ms / 1e3), 1),
        "grid_point_updates_per_s": round(points / (ms / 1e3), 1),
        "sequential_ms_per_step": round(seq_ms, 4),
        "speedup_vs_sequential": round(seq_ms / ms, 3),
        "tuning": tuning,
        "autotune_s": round(tune_s, 2),
        "how": "one CUDA graph launch per step holds every instance's step as a parallel branch; "
               "sequential = each instance's own step graph launched in turn; CUDA events",
    }


def adjoint_leg(stream):
    """Cost of the reverse step against the forward step.

    (1) The gradient workload (128^3, 512x48 membrane in 64 stiffness
    segments, 200k wall markers, FP32): one forward step (graph) and one
    ib_adjoint_step (u^{n+1} given, and recomputed), CUDA events on the
    library's stream; then the full 800-step checkpointed sweep (snapshots
    every 40 steps, misfit over the last 200 steps) through the autograd
    Function, wall clock around forward and backward."""
    import torch

    from paper_math_0301321_gb300 import synth
    from paper_math_0301321_gb300.adjoint import MembraneRun, membrane_response, misfit

    p = synth.cochlea128_adjoint()
    run = MembraneRun(p, prec="fp32", n_steps=800, window=200, ckpt_every=40)
    ctx = run.ctx
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s = torch.cuda.current_stream()

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(k):
            fn()
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    ctx.step(20)
    fwd_ms = timed(lambda: ctx.step(1), 50)
    snap = ctx.new_snapshot()
    ctx.snapshot_save(snap)
    ctx.step(1)
    nxt = ctx.new_snapshot()
    ctx.snapshot_save(nxt)
    ctx.snapshot_load(snap)
    lam_u = torch.randn((3,) + ctx.n[::-1], dtype=ctx.dtype_t, device="cuda")
    lam_D = torch.randn((3, ctx.m), dtype=torch.float64, device="cuda")
    gb = torch.zeros(run.nseg, dtype=torch.float64, device="cuda")
    out = (torch.empty_like(lam_u), torch.empty_like(lam_D))
    u1 = ctx.snapshot_velocity(nxt)
    adj_ms = timed(lambda: ctx.adjoint_step(lam_u, lam_D, u_np1=u1, grad_b=gb, out=out), 20)
    adj_rc_ms = timed(lambda: ctx.adjoint_step(lam_u, lam_D, grad_b=gb, out=out), 20)

    b0 = torch.tensor(p.structure.bend_b, dtype=torch.float64)
    with torch.no_grad():
        eta_t = run.forward(b0)
    # one untimed sweep (forward, misfit, backward) through the timed code
    # path: the first use of a kernel in a process may load or compile it
    # (seconds on a cold start), which is not the sweep's cost
    theta_w = torch.tensor(synth.perturbed_stiffness(p, 6), dtype=torch.float64, requires_grad=True)
    misfit(membrane_response(theta_w, run), eta_t).backward()
    theta = torch.tensor(synth.perturbed_stiffness(p, 5), dtype=torch.float64, requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eta = membrane_response(theta, run)
    loss = misfit(eta, eta_t)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    grad_finite = bool(torch.isfinite(theta.grad).all().item())
    run.close()
    grad_check = gradient_check()
    return {
        "workload": f"cochlea128_adjoint: 128^3 grid, {p.structure.m:,} markers (512x48 membrane in 64 stiffness "
                    "segments + 200,000 tethered wall markers), 1 kHz tone, dt = 30 ns, FP32",
        "fwd_step_ms": round(fwd_ms, 4),
        "adjoint_step_ms": round(adj_ms, 4),
        "ratio": round(adj_ms / fwd_ms, 3),
        "adjoint_step_recompute_ms": round(adj_rc_ms, 4),
        "ratio_recompute": round(adj_rc_ms / fwd_ms, 3),
        "sweep": {"steps": 800, "ckpt_every": 40, "window": 200,
                  "forward_s": round(t1 - t0, 4), "backward_s": round(t2 - t1, 4),
                  "backward_ms_per_step": round((t2 - t1) / 800 * 1e3, 4),
                  "backward_over_fwd_step": round((t2 - t1) / 800 * 1e3 / fwd_ms, 3),
                  "how": "after one untimed sweep (forward, misfit, backward) through the same path; "
                         "forward: 800 graph steps + snapshot every 40 + membrane eta read at the last 200; "
                         "backward: replay each 40-step segment from its snapshot keeping every state, "
                         "then 40 ib_adjoint_step calls (u^{n+1} given); wall clock"},
        "grad_finite": grad_finite,
        "grad_check": grad_check,
    }


def gradient_check():
    """The FP32 and FP64 gradients of the 128^3 gradient workload's misfit
    (started from a membrane bump with 1e4 x the graded bending stiffness, the
    configuration in which the stiffness moves the response above FP64
    rounding) on 2 seeded stiffness parameters, each against FP64 central
    differences (h = 1e-4 relative): the relative error per parameter."""
    import numpy as np
    import torch

    from paper_math_0301321_gb300 import synth
    from paper_math_0301321_gb300.adjoint import MembraneRun, membrane_response, misfit

    p = synth.with_bend_scale(synth.cochlea128_adjoint(), 1e4)
    D0 = synth.membrane_bump(p, 1e-4, 3)
    b0 = np.asarray(p.structure.bend_b)
    b = synth.perturbed_stiffness(p, 5)
    idx = [int(i) for i in np.sort(np.minimum((synth.uniform(5, 81, 2) * len(b)).astype(int), len(b) - 1))]
    grads, fd = {}, []
    for prec in ("fp64", "fp32"):
        run = MembraneRun(p, prec=prec, n_steps=800, window=200, ckpt_every=40, D0=D0)
        with torch.no_grad():
            eta_t = run.forward(torch.tensor(b0))
        theta = torch.tensor(b, requires_grad=True)
        misfit(membrane_response(theta, run), eta_t).backward()
        grads[prec] = theta.grad.numpy()[idx]
        if prec == "fp64":
            for s_ in idx:
                h = 1e-4 * b[s_]
                bp, bm = b.copy(), b.copy()
                bp[s_] += h
                bm[s_] -= h
                with torch.no_grad():
                    lp = float(misfit(run.forward(torch.tensor(bp)), eta_t))
                    lm = float(misfit(run.forward(torch.tensor(bm)), eta_t))
                fd.append((lp - lm) / (2 * h))
        run.close()
    fd = np.array(fd)
    return {"params": idx, "fd": fd.tolist(),
            "fp64_rel_err": (np.abs(grads["fp64"] - fd) / np.abs(fd)).tolist(),
            "fp32_rel_err": (np.abs(grads["fp32"] - fd) / np.abs(fd)).tolist(),
            "target": 1e-4,
            "how": "800-step checkpointed sweep (snapshots every 40, misfit over the last 200) through the "
                   "autograd Function; FP64 central differences of the FP64 forward, h = 1e-4 relative"}


def perturbed_state(p):
    """A state of the workload in which every force law and both upwind
    branches act: a membrane bump of 1e-7 cm plus 2e-8 cm of seeded noise on
    every marker, and a smooth seeded velocity of 0.1 cm/s (all values
    representable in FP32, so both precisions start from the same state)."""
    import numpy as np

    from paper_math_0301321_gb300 import synth
    D = synth.membrane_bump(p, 1e-7, 3) + 2e-8 * synth.normal(17, 61, 3 * p.structure.m).reshape(3, -1)
    u = synth.random_velocity(17, p.grid.n, amp=0.1, modes=8)
    return (np.asarray(D, np.float32).astype(np.float64), np.asarray(u, np.float32).astype(np.float64), 2.0e-5)


def cpu_baseline(p):
    """The FP64 oracle, as it stands, timed for one step of the same workload
    (from the perturbed state); returns the timing and the oracle's state."""
    import oracle
    st = oracle.Structure(p.structure)
    D, u, t = perturbed_state(p)
    t0 = time.perf_counter()
    Do, uo, _ = oracle.step(p.grid, st, D, u, t, 1)
    dt = time.perf_counter() - t0
    return ({"value": round(1.0 / dt, 5), "unit": "IB steps/s", "cores": 1, "kind": "oracle",
             "sample": f"1 full FP64 oracle step of the same 256^3 + {p.structure.m}-marker workload "
                       f"({dt:.1f} s, single thread)"}, (Do, uo))


def cufft_crosscheck(p, stream, stage_ms):
    """cuFFT (through torch.fft) on the same transforms as the fluid solve's
    FFT passes: a 3-D real-to-complex transform of the three FP32 velocity
    components and the complex-to-real inverse, CUDA events on `stream`.  A
    timed library yardstick only; the hand-written passes also fuse the
    right-hand side, the projection and the Helmholtz factor."""
    import torch
    n = tuple(p.grid.n[::-1])
    with torch.cuda.stream(stream):
        x = torch.randn((3,) + n, dtype=torch.float32, device="cuda")
        X = torch.fft.rfftn(x, dim=(1, 2, 3))
        y = torch.fft.irfftn(X, s=n, dim=(1, 2, 3))
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        k = 20
        for _ in range(3):
            X = torch.fft.rfftn(x, dim=(1, 2, 3))
            y = torch.fft.irfftn(X, s=n, dim=(1, 2, 3))
        e[0].record(stream)
        for _ in range(k):
            X = torch.fft.rfftn(x, dim=(1, 2, 3))
        e[1].record(stream)
        for _ in range(k):
            y = torch.fft.irfftn(X, s=n, dim=(1, 2, 3))
        e[2].record(stream)
        e[2].synchronize()
    fwd, inv = e[0].elapsed_time(e[1]) / k, e[1].elapsed_time(e[2]) / k
    ours_fwd = stage_ms["fft_x_fwd"] + stage_ms["fft_y_fwd"] + stage_ms["fft_z_proj"] / 2
    ours_inv = stage_ms["fft_z_proj"] / 2 + stage_ms["fft_y_inv"] + stage_ms["fft_x_inv"]
    del x, X, y
    return {"cufft_r2c_ms": round(fwd, 4), "cufft_c2r_ms": round(inv, 4), "cufft_total_ms": round(fwd + inv, 4),
            "passes_total_ms": round(ours_fwd + ours_inv, 4),
            "how": "torch.fft.rfftn / irfftn (cuFFT) of 3 FP32 components on the same grid, 20 calls each, CUDA "
                   "events; passes_total_ms = the five hand-written passes, which also form the right-hand side "
                   "(upwind advection, force, body force) and apply the projection and Helmholtz factor"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the same workload (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_math_0301321_gb300 import synth
    p = synth.cochlea256()
    st = oracle.Structure(p.structure)
    D, u, t = np.zeros_like(p.X), p.u, 0.0
    # untimed warm-up steps (at most 60 s of them), then timed steps (at most
    # 150 s), so that the arm ends within a few minutes
    warm = 0
    start = time.perf_counter()
    while warm < args.warmup and time.perf_counter() - start < 60.0:
        D, u, t = oracle.step(p.grid, st, D, u, t, 1)
        warm += 1
    budget = 150.0
    times = []
    start = time.perf_counter()
    while len(times) < max(1, args.steps):
        t0 = time.perf_counter()
        D, u, t = oracle.step(p.grid, st, D, u, t, 1)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - start + times[-1] > budget:
            break
    per = sum(times) / len(times)
    val = 1.0 / per
    sample = (f"{len(times)} full FP64 oracle step(s) of the 256^3 + {p.structure.m}-marker workload, "
              f"single thread, after {warm} warm-up step(s); capped at {budget:.0f} s of timed stepping")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(val, 5), "unit": "IB steps/s", "n_gpus": 1,
        "steps": len(times), "warmup": warm, "ms_per_step": round(per * 1e3, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
        "config": workload_config(p, int(os.environ.get("WORLD_SIZE", "1"))),
        "precision": "FP64 throughout (the CPU oracle)",
        "cpu_baseline": {"value": round(val, 5), "unit": "IB steps/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(val, 5), "unit": "IB steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--skip-cpu", action="store_true", help="omit the CPU oracle baseline")
    ap.add_argument("--skip-fp64", action="store_true", help="omit the FP64 GPU step")
    ap.add_argument("--skip-adjoint", action="store_true", help="omit the reverse-step timing")
    ap.add_argument("--skip-batch", action="store_true", help="omit the tone-sweep batch timing")
    ap.add_argument("--skip-next", action="store_true", help="omit the half-cube / windows / probe timing")
    ap.add_argument("--skip-tc", action="store_true", help="omit the tensor-core FFT leg")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_math_0301321_gb300 import build
        build.build()
        run_gpu(args)


if __name__ == "__main__":
    main()
