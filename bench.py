"""Benchmark of the hybrid light-transport loop (one step = one full render).

Workload: the hash-grid scene of the paper-shaped benchmark (800x800, 1 spp,
16-level hash grid with 2^19 FP16 entries per level, MLP 32-64-64-4, 128^3
occupancy, 10,240-triangle glass sphere, mirror cube, diffuse floor, one
point light, up to 8 segments per path, fixed step sqrt(3)/1024).  Inputs are
synthetic and seeded.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp16|bf16]
    python bench.py --impl reference    # the FP64 CPU oracle on the host cores

Under torchrun (N > 1) every rank renders its own copy of the workload
(replicas: pixels are independent, there is no data exchange); rank 0 prints.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray-segments/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP32_FLOP_PER_SAMPLE = 2 * (32 * 64 + 64 * 64 + 64 * 4)  # MLP multiply-adds x 2
SM_COUNT, FP32_LANES_PER_SM = 152, 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--engine", default="auto", choices=["auto", "megakernel", "wavefront"])
    ap.add_argument("--width", type=int, default=800)
    ap.add_argument("--height", type=int, default=800)
    ap.add_argument("--cpu-stride", type=int, default=4, help="oracle sample: every n-th row and column")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                r = subprocess.run(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                    "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if r.returncode == 0 and r.stdout.strip():
                    self.rows.append([x.strip() for x in r.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if len(r) > 5 + k and r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def workload(args):
    from paper_2309_04581_gb300 import scenes as S
    sc = S.config2(args.width, args.height)
    name = f"hash-grid field + glass/mirror/diffuse meshes, {args.width}x{args.height}, 1 spp, 8 bounces"
    return sc, name


def cpu_baseline(sc, stride: int):
    """The FP64 oracle, as it stands, on a strided pixel sample of the workload."""
    import oracle
    from paper_2309_04581_gb300 import scenes as S
    oracle.build()
    ids = S.strided_pixels(sc.camera.width, sc.camera.height, stride)
    t = time.perf_counter()
    res = oracle.render(sc, ids, records=False)
    dt = time.perf_counter() - t
    seg = res["counts"]["segments"]
    return {"value": seg / dt, "unit": METRIC, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"every {stride}th row and column ({len(ids)} of {sc.n_rays} pixels), {seg} segments in {dt:.1f} s",
            "samples_per_s": res["counts"]["samples_supported"] / dt}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc, name = workload(args)
    cb = None
    vals = []
    for _ in range(args.warmup):
        pass
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(sc, max(args.cpu_stride, 8))
        vals.append(cb["value"])
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "precision": "fp64", "l2": "inputs resident; oracle on host"},
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"], "value": v,
                             "unit": METRIC},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2309_04581_gb300 import build as cuda_build
    import paper_2309_04581_gb300.mrf as M

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        cuda_build.build()
    if world > 1:
        dist.barrier()
    sc, name = workload(args)
    prec = {"fp32": M.MRF_PREC_FP32, "fp16": M.MRF_PREC_FP16, "bf16": M.MRF_PREC_BF16}[args.precision]
    engine = {"auto": M.MRF_ENGINE_AUTO, "megakernel": M.MRF_ENGINE_MEGAKERNEL,
              "wavefront": M.MRF_ENGINE_WAVEFRONT}[args.engine]
    r = M.Renderer(sc, device=local, precision=prec)
    stream = torch.cuda.Stream(local)
    out = torch.empty((sc.n_rays, 4), dtype=torch.float32, device=f"cuda:{local}")
    # one untimed run for the deterministic work counts
    with torch.cuda.stream(stream):
        _, st = r.render(out=out, engine=engine, stats=True, stream=stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")  # 256 MB > L2
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            r.render(out=out, engine=engine, stream=stream.cuda_stream)
    stream.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with sampler:
        t0 = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
                evs[k][0].record(stream)
                r.render(out=out, engine=engine, stream=stream.cuda_stream)
                evs[k][1].record(stream)
        stream.synchronize()
        wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        t = torch.tensor([ms], device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    segs = st["segments"]
    samples = st["samples_evaluated"] + st["shadow_samples_evaluated"]
    value = world * segs / (ms / 1e3)
    # end to end through the C ABI: host output buffer, device->host copy inside the call
    host_out = torch.empty((sc.n_rays, 4), dtype=torch.float32).pin_memory()
    e2e_ms = []
    for k in range(max(3, args.steps // 2)):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t = time.perf_counter()
        r.render(out=host_out, engine=engine, stream=stream.cuda_stream)
        e2e_ms.append((time.perf_counter() - t) * 1e3)
    e2e = world * segs / (statistics.median(e2e_ms) / 1e3)
    pk, pk_kind = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    if args.precision == "fp32":
        flop = FP32_FLOP_PER_SAMPLE * samples
        peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flop / (ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": (flop / (ms / 1e3) / 1e12) / peak, "traffic": None,
                "kernel": "render_megakernel", "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}
    else:
        flop = FP32_FLOP_PER_SAMPLE * samples
        peak = pk["bf16_tflops"]
        roof = {"bound": "tensor", "achieved": flop / (ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": (flop / (ms / 1e3) / 1e12) / peak, "traffic": None, "kernel": "render",
                "peak_kind": pk_kind}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "fp16": "f16", "bf16": "bf16"}[args.precision],
            "data": "synthetic",
            "config": {"workload": name, "precision": args.precision, "engine": args.engine,
                       "l2": "256 MB buffer written between timed steps", "parallelism": f"replicas x{world}"},
            "field_samples_per_s": world * samples / (ms / 1e3),
            "work_per_step": {"segments": segs, "samples_evaluated": st["samples_evaluated"],
                              "shadow_samples_evaluated": st["shadow_samples_evaluated"],
                              "samples_nominal": st["samples_nominal"], "shadow_rays": st["shadow_rays"],
                              "paths": st["paths"], "fp64_retests": st["fp64_retests"]},
            "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
            "wall_s_timed_region": wall,
            "roofline": roof,
            "e2e": {"value": e2e, "unit": METRIC, "h2d_bytes_per_step": 48,
                    "d2h_bytes_per_step": sc.n_rays * 16, "ms_per_step": statistics.median(e2e_ms)},
            "gpu_launches": args.steps,
            "clocks": sampler.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc, args.cpu_stride)
    if rank == 0:
        print(json.dumps(line), flush=True)
    r.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
