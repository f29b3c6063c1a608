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

Multi-GPU: the step does not shard (one periodic FFT grid); N > 1 runs N
independent replicas, one per GPU (weak scaling), no collective on the data
path.  `--impl reference` times the FP64 CPU oracle on the machine's host cores.
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


def stage_bytes(name: str, G: int, n: int, m: int, touched_tiles: int) -> float:
    """Algorithmic HBM bytes of one stage at FP32 (each array read or written once)."""
    S = 8 * (n * n) * (n // 2 + 1)            # one complex half spectrum incl. the kx = n/2 plane
    touched_cells = touched_tiles * 512
    return {
        "keys": m * (12 + 12 + 12 + 4 + 4 + 12),             # cell0, r0, d in; key, bucket count, rfrac out
        "sort": m * (3 * 16 + 3 * 4) + 3 * 4 * (G // 8),      # 3 radix passes (k,v r+w) + hist; bucket scan
        "records": m * (4 + 12 + 12 + 64) + 24 * m,           # perm, rfrac, d, record out; links (~2/marker)
        "spread": m * 64 + 12 * touched_cells,                # records once, F on touched tiles
        "fft_x_fwd": 3 * 4 * G + 3 * S + 12 * touched_cells,  # u in, spectrum out, F in on touched tiles
        "fft_y_fwd": 3 * 2 * S,
        "fft_z_proj": 3 * 2 * S,
        "fft_y_inv": 3 * 2 * S,
        "fft_x_inv": 3 * S + 3 * 4 * G,
        "interp": m * (64 + 4 + 4 + 24) + 12 * touched_cells,  # record, key, perm, d r+w; u on touched cells
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
            k64 = max(2, min(args.steps // 10, 10))
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            c64.step(k64)
            f1.record(stream)
            f1.synchronize()
            c64.sync()
            fp64 = {"value": world * k64 / (f0.elapsed_time(f1) / 1e3), "steps": k64}
            c64.close()

    pk, src = peaks()
    tot = sum(stage_ms.values())
    dom = max(stage_ms, key=stage_ms.get)
    achieved = stage_bytes(dom, G, n, m, tiles) / (stage_ms[dom] / 1e3) / 1e9
    stages = {k: {"ms": round(v, 4), "share": round(v / tot, 4),
                  "gbs": round(stage_bytes(k, G, n, m, tiles) / (v / 1e3) / 1e9, 1)} for k, v in stage_ms.items()}
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
        "config": {"workload": WORKLOAD, "grid": [n, n, n], "markers": m, "springs": int(len(p.structure.spring_k)),
                   "precision": "FP32 fields/forces/FFTs, FP64 reference positions + FP32 displacements",
                   "l2": "working set ~1.1 GB > 129 MB L2; no flush between steps",
                   "parallelism": f"{world} independent replica(s), one per GPU"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1),
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / pk["hbm_gbs"], 4),
                     "peak_source": f"{src} hbm_gbs", "traffic": None},
        "stages": stages,
        "active_tiles": tiles,
        "gpu_launches": gpu_launches,
        "e2e": {"value": round(e2e_value, 2), "unit": "IB steps/s", "h2d_bytes_per_step": 24 * m + 8,
                "d2h_bytes_per_step": 24 * m + 8 + 4,
                "how": "per step: ib_set_state(X host->device) + ib_step(1) + ib_get_state(X device->host), "
                       "pinned host buffers, wall clock"},
        "fp64_gpu": fp64,
        "finite": finite,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.skip_cpu:
        out["cpu_baseline"] = cpu_baseline(p)
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def kernels_per_step(n: int) -> int:
    """Kernels the library launches per step (all its own), for the launch count claim."""
    passes = 3 if n > 32 else 2                      # radix passes for this grid's key width
    keys = 1
    sort = passes * (1 + 3 + 1)                      # hist, 3-kernel scan, scatter
    bucket = 3
    records = 1
    spread = 2                                       # tile list + persistent spread
    fluid = 1 + 2 + 2 + 2 + 1                        # x-fwd, y cols+rows, z main+nyq, y inv, x-inv
    interp = 1
    return keys + sort + bucket + records + spread + fluid + interp


def cpu_baseline(p):
    """The FP64 oracle, as it stands, timed for one step of the same workload."""
    import numpy as np

    import oracle
    st = oracle.Structure(p.structure)
    D = np.zeros_like(p.X)
    t0 = time.perf_counter()
    oracle.step(p.grid, st, D, p.u, 0.0, 1)
    dt = time.perf_counter() - t0
    return {"value": round(1.0 / dt, 5), "unit": "IB steps/s", "cores": 1, "kind": "oracle",
            "sample": f"1 full FP64 oracle step of the same 256^3 + {p.structure.m}-marker workload "
                      f"({dt:.1f} s, single thread)"}


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
              f"single thread, no warm-up (CPU code); capped at {budget:.0f} s of stepping")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(val, 5), "unit": "IB steps/s", "n_gpus": 1,
        "steps": len(times), "warmup": 0, "ms_per_step": round(per * 1e3, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
        "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": round(val, 5), "unit": "IB steps/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(val, 5), "unit": "IB steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--skip-cpu", action="store_true", help="omit the CPU oracle baseline")
    ap.add_argument("--skip-fp64", action="store_true", help="omit the FP64 GPU step")
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
