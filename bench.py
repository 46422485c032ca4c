#!/usr/bin/env python3
"""Benchmark of the GB300 tensor-core beamformer.

Default workload (the radio-astronomy block): 512 independent products
(256 frequency channels x 2 polarisations, both polarisations of a channel
sharing its weights), each 1024 beams x 288 receivers x 4096 samples,
FP16 inputs, FP32 accumulation.  One step is one pass of the hot path over
one block of samples that is already resident in HBM:
    tcbf_transpose_pack(X)  (interleaved complex FP16 -> packed planes)
    tcbf_beamform_fp16      (all 512 products in one persistent launch)
The weights are computed once from geometry beforehand (they are constant
over many blocks) and timed separately.

Metric: TeraOps/s with 8 useful operations per complex multiply-accumulate
(8 * batch * M * N * K per step).  Prints ONE JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Beamforming TeraOps/s (8 ops/cMAC), % tensor peak; served p50/p99 latency"
UNIT = "TeraOps/s"

WORKLOADS = {
    "radio": dict(
        B=512, M=1024, N=4096, K=288, w_batches=256, near_field=False,
        desc="radio-astronomy FP16 block: 256 channels x 2 pols = 512 products of "
             "1024 beams x 288 receivers x 4096 samples, weights from geometry "
             "(110-190 MHz, 3 km disk, beams within 5 deg of zenith)"),
    "ultrasound": dict(
        B=1, M=65536, N=256, K=16384, w_batches=1, near_field=True,
        desc="computational ultrasound FP16: 65536 voxels x 16384 (128 elements x 128 "
             "frequency bins) x 256 frames, near-field model matrix"),
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="radio")
    ap.add_argument("--config", type=int, default=None, help="kernel configuration (tile shape)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batches", type=int, default=None,
                    help="override the number of products (small profiling cases)")
    return ap.parse_args()


def ops_per_step(w):
    return 8.0 * w["B"] * w["M"] * w["N"] * w["K"]


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return dict(hbm_gbs=float(d["hbm_gbs"]), bf16_tflops=float(d["bf16_tflops"]),
                    bf16_tflops_sustained=float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                    source="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0,
                    source="fallback")


def kernel_sources_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, only if the
    kernel's sources are unchanged since that capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)[kernel]
    except Exception:
        return None
    if rec.get("workload") != workload:
        return None
    if rec.get("sources_sha") != kernel_sources_sha(rec.get("sources", [])):
        return None
    return rec.get("bytes_per_launch")


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_median": statistics.median(power) if power else None}


# -------------------------------------------------------------- CPU oracle
def cpu_baseline(w, seconds, seed=0):
    """Time the FP64 oracle on a bounded sample of the same workload: the
    first `nb` products (their weights computed by the oracle itself)."""
    import numpy as np
    import oracle
    import tcbf_inputs as ti
    geom = ti.radio_geometry(seed, w["M"], w["K"], w["B"] // 2) if not w["near_field"] \
        else ti.ultrasound_geometry()
    per_w = w["B"] // w["w_batches"]

    def sample(nb):
        nw = (nb + per_w - 1) // per_w
        Wf = oracle.weights_fp16(geom.rx_pos, geom.targets, geom.freqs[:nw], geom.near_field, geom.c)
        if w["near_field"]:
            X = ti.ultrasound_frames(seed + 1, w["K"], w["N"])[:nb]
        else:
            X = np.stack([ti.radio_x_batch(seed + 1, b, w["K"], w["N"]) for b in range(nb)])
        return Wf, X

    if w["near_field"]:
        # one product is the whole workload: time a block of its voxel rows
        X = ti.ultrasound_frames(seed + 1, w["K"], w["N"])

        def rows_w(rows):
            return oracle.weights_fp16(geom.rx_pos, geom.targets[:rows], geom.freqs[:1],
                                       True, geom.c)
        rows = 16
        Wf = rows_w(rows)
        t0 = time.perf_counter()
        oracle.cgemm(Wf, X)
        dt = time.perf_counter() - t0
        rows = max(16, min(w["M"], int(rows * seconds / max(dt, 1e-3))))
        Wf = rows_w(rows)
        t0 = time.perf_counter()
        oracle.cgemm(Wf, X)
        dt = time.perf_counter() - t0
        ops = 8.0 * rows * w["N"] * w["K"]
        desc = f"{rows} of {w['M']} voxel rows of the one product"
    else:
        Wf, X = sample(per_w)
        t0 = time.perf_counter()
        oracle.cgemm(Wf[:1], X[:per_w])
        dt1 = (time.perf_counter() - t0) / per_w
        nb = max(per_w, min(w["B"], int(seconds / max(dt1, 1e-3)) // per_w * per_w))
        Wf, X = sample(nb)
        t0 = time.perf_counter()
        oracle.cgemm(Wf, X)
        dt = time.perf_counter() - t0
        ops = 8.0 * nb * w["M"] * w["N"] * w["K"]
        desc = f"{nb} of {w['B']} products (whole products, FP64 triple loop)"
    return {"value": ops / dt / 1e12, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "sample": desc, "seconds": round(dt, 3),
            "host_cpus": os.cpu_count()}


def reference_arm(args, w):
    """The oracle as the reference arm: each step one bounded sample."""
    import numpy as np
    import oracle
    import tcbf_inputs as ti
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    geom = ti.radio_geometry(0, w["M"], w["K"], w["B"] // 2) if not w["near_field"] \
        else ti.ultrasound_geometry()
    Wf = oracle.weights_fp16(geom.rx_pos, geom.targets, geom.freqs[:1], geom.near_field, geom.c)
    if w["near_field"]:
        rows = 16
        Wf = Wf[:, :rows]
        X = ti.ultrasound_frames(1, w["K"], w["N"])
        ops = 8.0 * rows * w["N"] * w["K"]
        desc = f"{rows} voxel rows of the product per step"
    else:
        X = ti.radio_x_batch(1, 0, w["K"], w["N"])[None]
        ops = 8.0 * w["M"] * w["N"] * w["K"]
        desc = "1 of 512 products per step"
    for _ in range(args.warmup):
        oracle.cgemm(Wf, X)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.cgemm(Wf, X)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = ops * len(times) / tot / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": w["desc"], "batch": w["B"], "M": w["M"], "N": w["N"], "K": w["K"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- GPU
def main():
    args = parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.batches is not None and args.workload == "radio":
        w["B"] = args.batches
        w["w_batches"] = max(1, args.batches // 2)
        w["desc"] = w["desc"].replace("256 channels x 2 pols = 512", f"{args.batches}")
    if args.impl == "reference":
        reference_arm(args, w)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2505_03269_gb300 as tcbf
    import tcbf_inputs as ti
    from paper_2505_03269_gb300 import build as tcbf_build

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        tcbf_build.build()
    if world > 1:
        dist.barrier()
    tcbf.load()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    B, M, N, K, Bw = w["B"], w["M"], w["N"], w["K"], w["w_batches"]
    # ---- inputs: geometry and samples (host), then resident on the device
    if w["near_field"]:
        geom = ti.ultrasound_geometry()
        Xh = ti.ultrasound_frames(1, K, N)
    else:
        geom = ti.radio_geometry(0, M, K, B // 2)
        Xh = ti.radio_x(1, B, K, N)
    Xd = torch.from_numpy(Xh).cuda()
    plan = tcbf.Plan(B, M, N, K, tcbf.MODE_FP16, w_batches=Bw, device=local)
    if args.config is not None:
        plan.set_config(args.config)
    Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
    Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
    Y = torch.empty((B, M, N, 2), dtype=torch.float32, device="cuda")
    rx = torch.from_numpy(geom.rx_pos).cuda()
    tg = torch.from_numpy(geom.targets).cuda()
    fr = torch.from_numpy(np.ascontiguousarray(geom.freqs[:Bw])).cuda()
    stream = torch.cuda.current_stream()

    # weights: once, timed on their own
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plan.weights_from_geometry(rx, tg, w["near_field"], fr, geom.c, Wp)
    e0.record()
    plan.weights_from_geometry(rx, tg, w["near_field"], fr, geom.c, Wp)
    e1.record()
    torch.cuda.synchronize()
    weights_ms = e0.elapsed_time(e1)

    def step():
        plan.transpose_pack(1, Xd, Xp)
        plan.beamform_fp16(Wp, Xp, Y)

    for _ in range(max(args.warmup, 3)):
        step()
    barrier()
    assert plan.last_device_error() == 0

    # ---- timed region: K steps, events around each kernel on the launch stream
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    for i in range(args.steps):
        ev[i][0].record(stream)
        plan.transpose_pack(1, Xd, Xp)
        ev[i][1].record(stream)
        plan.beamform_fp16(Wp, Xp, Y)
        ev[i][2].record(stream)
    barrier()
    clocks = sampler.stop()
    status = plan.last_device_error()
    total_ms = ev[0][0].elapsed_time(ev[-1][2])
    pack_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    gemm_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * ops_per_step(w) / (ms_per_step * 1e-3) / 1e12

    # ---- parity on sampled outputs (full size, the launch configuration timed above)
    import oracle
    g = np.random.default_rng(123)
    npts = 128
    pts = np.stack([g.integers(0, B, npts), g.integers(0, M, npts), g.integers(0, N, npts)], 1)
    ref = np.empty(npts, np.complex128)
    for i, (b, m, n) in enumerate(pts):
        bw = b // (B // Bw)
        Wrow = oracle.weights_fp16(geom.rx_pos, geom.targets[m:m + 1], geom.freqs[bw:bw + 1],
                                   geom.near_field, geom.c)
        ref[i] = oracle.cgemm_points(Wrow, Xh[b:b + 1], np.array([[0, 0, n]]))[0]
    ti_ = torch.from_numpy(pts).cuda()
    Yh = Y[ti_[:, 0], ti_[:, 1], ti_[:, 2]].double().cpu().numpy()
    got = Yh[:, 0] + 1j * Yh[:, 1]
    parity = {"points": npts, "rel_err": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
              "reference": "FP64 oracle, its own weights from the same geometry"}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        Xhost = torch.from_numpy(Xh).pin_memory()
        Yhost = torch.empty((B, M, N, 2), dtype=torch.float32, pin_memory=True)
        for _ in range(1):
            Xd.copy_(Xhost, non_blocking=True)
            step()
            Yhost.copy_(Y, non_blocking=True)
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.e2e_steps):
            Xd.copy_(Xhost, non_blocking=True)
            step()
            Yhost.copy_(Y, non_blocking=True)
        b.record()
        barrier()
        e2e_ms = a.elapsed_time(b) / args.e2e_steps
        te = torch.tensor([e2e_ms], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": world * ops_per_step(w) / (float(te.item()) * 1e-3) / 1e12, "unit": UNIT,
               "h2d_bytes_per_step": int(Xh.nbytes), "d2h_bytes_per_step": int(Y.numel() * 4),
               "ms_per_step": float(te.item()),
               "how": "pinned host X -> device, pack, beamform, Y -> pinned host, one stream"}
        del Xhost, Yhost

    # ---- roofline of the dominant kernel (the GEMM)
    peaks = load_peaks()
    gemm_bytes = plan.packed_size(0) + plan.packed_size(1) + B * M * N * 8
    pack_bytes = 2 * plan.packed_size(1)
    ai = ops_per_step(w) / gemm_bytes
    ridge = peaks["bf16_tflops"] * 1e12 / (peaks["hbm_gbs"] * 1e9)
    gemm_tops = ops_per_step(w) / (gemm_ms * 1e-3) / 1e12
    gemm_gbs = gemm_bytes / (gemm_ms * 1e-3) / 1e9
    gemm_sources = ["paper_2505_03269_gb300/csrc/gemm_f16.cu", "paper_2505_03269_gb300/csrc/ptx.cuh"]
    if ai < ridge:
        roof = {"bound": "hbm", "achieved": gemm_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": gemm_gbs / peaks["hbm_gbs"]}
    else:
        roof = {"bound": "tensor", "achieved": gemm_tops, "peak": peaks["bf16_tflops"],
                "unit": "TFLOP/s", "frac": gemm_tops / peaks["bf16_tflops"]}
    roof["traffic"] = recorded_traffic("gemm_f16", args.workload)
    roof["kernel"] = "cgemm_f16_kernel"
    roof["algorithmic_bytes"] = gemm_bytes
    roof["peak_source"] = peaks["source"]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": w["desc"], "batch": B, "M": M, "N": N, "K": K, "w_batches": Bw,
                   "step": "transpose_pack(X) + beamform_fp16 (weights resident)",
                   "l2": "inputs larger than L2 (X %.2f GB, Y %.1f GB per step)"
                         % (Xh.nbytes / 1e9, B * M * N * 8 / 1e9),
                   "kernel_config": plan.config_name(plan.get_config()),
                   "parallelism": f"{world} independent replica(s), no collective"},
        "gpu_launches": 2 * args.steps,
        "roofline": roof,
        "kernels": {"gemm_ms": gemm_ms, "pack_ms": pack_ms, "weights_ms_once": weights_ms,
                    "gemm_tops": gemm_tops,
                    "gemm_frac_of_bf16_peak": gemm_tops / peaks["bf16_tflops"],
                    "gemm_ai_ops_per_byte": ai,
                    "pack_gbs": pack_bytes / (pack_ms * 1e-3) / 1e9,
                    "pack_frac_of_hbm": pack_bytes / (pack_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]},
        "clocks": clocks,
        "device_status": status,
        "parity_sampled": parity,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
