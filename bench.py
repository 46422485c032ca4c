#!/usr/bin/env python3
"""Benchmark of the GB300 tensor-core beamformer.

Default workload (the radio-astronomy block): 512 independent products
(256 frequency channels x 2 polarisations, both polarisations of a channel
sharing its weights), each 1024 beams x 288 receivers x 4096 samples,
FP16 inputs, FP32 accumulation.  One step is one pass of the hot path over
one block of samples that is already resident in HBM: the plan reads X in
its interleaved complex layout (TCBF_FLAG_INTERLEAVED_X), so the step is
    tcbf_beamform_fp16      (all 512 products in one persistent launch,
                             no transpose/pack pass over X)
The planar path (tcbf_transpose_pack(X) into planes + the planar GEMM) is
timed beside it (`planar_step`).  The weights are computed once from
geometry beforehand (they are constant over many blocks) and timed
separately.

The same JSON line carries the other configured workloads as sub-records
(`workloads`): the ultrasound block (65536 voxels x 16384 x 256 frames) in
FP16, split-FP8 (E4M3 hi+lo, three products) and plain FP8, the 1-bit radio
block (64 channels x 2048 beams x 1024 receivers x 8192 samples, exact
int32), and the serving stream (continuous batching, p50/p99 latency beside
the one-request-per-launch FP16 baseline); each with its GEMM time, roofline
and clocks, the FP8 ones with their error against the FP16 path on the same
inputs.  --workload runs one of them as the headline instead, --no-subs skips
the sub-records.  Parity with the oracle is the tests' job (the full-size
tests sample these workloads in the launch configurations timed here); the
oracle runs here only as the CPU baseline and the reference arm.

Metric: TeraOps/s with 8 useful operations per complex multiply-accumulate
(8 * batch * M * N * K per step).  Prints ONE JSON line.  One GPU only:
--gpus other than 1 exits with an error before any CUDA call.

  python bench.py [--gpus 1] [--steps K] [--warmup W] [--impl ours|reference]
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
FP8_OVER_BF16 = 4.5 / 2.25     # nominal dense-rate ratio used to scale the measured bf16 peak
TF32_OVER_BF16 = 1.1 / 2.25    # the same for TF32
FP4_OVER_BF16 = 13.5 / 2.25    # and for the dense 4-bit (E2M1) rate

WORKLOADS = {
    "radio": dict(
        mode="fp16", B=512, M=1024, N=4096, K=288, w_batches=256, geometry="radio",
        layout="interleaved",
        desc="radio-astronomy FP16 block: 256 channels x 2 pols = 512 products of "
             "1024 beams x 288 receivers x 4096 samples, weights from geometry "
             "(110-190 MHz, 3 km disk, beams within 5 deg of zenith)"),
    "ultrasound": dict(
        mode="fp16", B=1, M=65536, N=256, K=16384, w_batches=1, geometry="ultrasound",
        stacked=True,
        desc="computational ultrasound FP16: 65536 voxels x 16384 (128 elements x 128 "
             "frequency bins) x 256 frames, near-field model matrix"),
    "onebit": dict(
        mode="1bit", B=64, M=2048, N=8192, K=1024, w_batches=64, geometry="radio",
        desc="radio-astronomy 1-bit block: 64 channels x 2048 beams x 1024 receivers x "
             "8192 samples, W = signs of the steering weights from geometry (110-190 MHz, "
             "3 km disk, beams within 5 deg of zenith), X = signs of complex Gaussian "
             "samples, +-1+-i values, exact int32 output"),
    # the paper's kernel-tuning shapes (Sec. IV, Table III), for comparison with its
    # TeraOps/s and TeraOps/J; the 1-bit one with K cut from 524288 so a step takes seconds
    "paper_fp16": dict(
        mode="fp16", B=1, M=8192, N=8192, K=8192, w_batches=1, geometry="random", stacked=True,
        desc="paper tuning shape FP16: M = N = K = 8192, W = exp(i phi) random phases, "
             "X complex Gaussian"),
    "paper_int1": dict(
        mode="1bit", B=1, M=32768, N=8192, K=65536, w_batches=1, geometry=None, x_phase=True,
        desc="paper tuning shape 1-bit with K reduced: 32768 x 8192 x 65536 (the paper's K is "
             "524288), +-1+-i values, exact int32 output"),
    # the paper's small roofline shapes (Sec. IV-A, Fig. 3), memory-bound
    "paper_fp16_batched": dict(
        mode="fp16", B=256, M=1024, N=1024, K=64, w_batches=256, geometry="random",
        layout="interleaved",
        desc="paper roofline shape FP16: 256 products of 1024 x 1024 x 64, W = exp(i phi) "
             "random phases per product, X complex Gaussian, read as it lies"),
    "paper_int1_batched": dict(
        mode="1bit", B=256, M=1024, N=1024, K=256, w_batches=256, geometry=None,
        desc="paper roofline shape 1-bit: 256 products of 1024 x 1024 x 256, random sign "
             "weights per product, X = signs of complex Gaussian samples, exact int32 output"),
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
    ap.add_argument("--no-energy", action="store_true", help="skip the power-sampled loops")
    ap.add_argument("--e2e-chunk", type=int, default=0,
                    help="batches per chunk of the end-to-end host pipeline (0: about batch / 16)")
    ap.add_argument("--mode", choices=["fp16", "fp8split", "fp8", "tf32"], default=None,
                    help="arithmetic of the FP workloads (default fp16); fp8split: E4M3 hi+lo, "
                         "three products; fp8: the plain E4M3 product (hi only)")
    ap.add_argument("--fp8-scales", choices=["row", "block"], default="row",
                    help="FP8 scales: per row / sample, or per 32 k of each (block-scaled MMAs)")
    ap.add_argument("--layout", choices=["interleaved", "planar", "stacked"], default=None,
                    help="FP16 X layout: interleaved (no pack, the radio default), planar, stacked")
    ap.add_argument("--no-subs", action="store_true", help="skip the sub-workload records")
    ap.add_argument("--sub-steps", type=int, default=10)
    ap.add_argument("--serving-requests", type=int, default=400)
    ap.add_argument("--batches", type=int, default=None,
                    help="override the number of products (small profiling cases)")
    ap.add_argument("--m-rows", type=int, default=None,
                    help="override the beams / voxels per product (small profiling cases)")
    return ap.parse_args()


def workload(args):
    w = dict(WORKLOADS[args.workload])
    if args.mode is not None and w["mode"] != "1bit":
        w["mode"] = args.mode
        if args.mode == "fp8split":
            w["desc"] = w["desc"].replace("FP16", "split-FP8 (E4M3 hi+lo)")
        elif args.mode == "tf32":
            w["desc"] = w["desc"].replace("FP16", "TF32 (FP32 data)")
        elif args.mode == "fp8":
            w["desc"] = w["desc"].replace("FP16", "FP8 (E4M3, per-row scales)")
    if args.batches is not None:
        w["B"] = args.batches
        if args.workload == "radio":
            w["w_batches"] = max(1, args.batches // 2)
        else:
            w["w_batches"] = min(w["w_batches"], args.batches)
        w["desc"] += f" [{args.batches} products]"
    if getattr(args, "m_rows", None) is not None:
        w["M"] = args.m_rows
        w["desc"] += f" [{args.m_rows} rows]"
    if getattr(args, "fp8_scales", "row") == "block" and w["mode"] in ("fp8split", "fp8"):
        w["fp8_block"] = True
        w["desc"] = w["desc"].replace("per-row scales", "block scales").replace(
            "(E4M3 hi+lo)", "(E4M3 hi+lo, block scales)")
        if "block scales" not in w["desc"]:
            w["desc"] += " [a scale per 32 k of each row and sample]"
    if getattr(args, "layout", None) is not None and w["mode"] == "fp16":
        w["layout"] = args.layout
        w["stacked"] = args.layout == "stacked"
    return w


def layout_of(w):
    """FP16 X layout of the workload: interleaved (read as it lies), stacked
    planes, or the default planar planes."""
    if w["mode"] != "fp16":
        return "planar"
    if w.get("stacked"):
        return "stacked"
    return w.get("layout", "planar")


def is_fp8(w):
    """Either E4M3 form: the hi+lo split (three products) or plain (hi only)."""
    return w["mode"] in ("fp8split", "fp8")


def fp8_products(w):
    return 1 if w["mode"] == "fp8" else 3


def ops_per_step(w):
    return 8.0 * w["B"] * w["M"] * w["N"] * w["K"]


def tops(ops, ms):
    """TeraOps/s of `ops` useful operations done in `ms` milliseconds."""
    return ops / (ms * 1e-3) / 1e12


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


def recorded_traffic(kernel, workload_name, config_name):
    """DRAM bytes per launch from a committed ncu summary of this kernel, this
    workload and this tile configuration, only if the kernel's sources are
    unchanged since that capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            records = json.load(fh)["records"]
    except Exception:
        return None
    for rec in records:
        if (rec.get("kernel"), rec.get("workload"), rec.get("config")) != (
                kernel, workload_name, config_name):
            continue
        if rec.get("sources_sha") != kernel_sources_sha(rec.get("sources", [])):
            return None
        return rec.get("bytes_per_launch")
    return None


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

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_median": statistics.median(power) if power else None}


# ----------------------------------------------------------------- inputs
def geometry_of(w):
    import numpy as np
    import tcbf_inputs as ti
    if w["geometry"] == "random":
        return None
    if w["geometry"] == "radio":     # one channel per weight batch
        return ti.radio_geometry(0, w["M"], w["K"], w["w_batches"])
    if w["geometry"] == "ultrasound":
        g = ti.ultrasound_geometry()
        if w["M"] < len(g.targets):          # reduced profiling case: the first M voxels
            g = ti.Geometry(g.rx_pos, np.ascontiguousarray(g.targets[: w["M"]]), g.freqs,
                            g.near_field, g.c)
        return g
    return None


def host_x(w):
    import tcbf_inputs as ti
    if w.get("x_phase"):       # unit-magnitude random phases, drawn in parallel (large K)
        return ti.random_phase_rows(1, w["K"], w["N"])
    if w["geometry"] == "random":
        return ti.complex_gaussian_fp16(ti.rng(1), (w["B"], w["K"], w["N"]))
    if w["geometry"] == "ultrasound":
        return ti.ultrasound_frames(1, w["K"], w["N"])
    return ti.radio_x(1, w["B"], w["K"], w["N"])


def onebit_weights(w):
    import tcbf_inputs as ti
    return ti.random_sign_words(ti.rng(0), (w["w_batches"], 2, w["M"], ti.words_per_row(w["K"])))


# -------------------------------------------------------------- CPU oracle
def oracle_sample(w, seconds_target):
    """The oracle on a bounded sample of the workload; returns (ops, seconds, text)."""
    import numpy as np
    import oracle
    import tcbf_inputs as ti

    if w["mode"] == "1bit":
        if w["geometry"] == "radio":    # signs of the first channel's steering weights
            geom = geometry_of(w)
            wc = oracle.weights(geom.rx_pos, geom.targets, geom.freqs[:1], False, geom.c)
            Wb = oracle.pack_signs_f64(wc, ti.words_per_row(w["K"]))
        else:
            Wb = onebit_weights(w)[:1]
        X = host_x(w) if w.get("x_phase") else ti.radio_x_batch(1, 0, w["K"], w["N"])[None]
        Xb = oracle.pack_signs(X, k_is_row=True, Kw=Wb.shape[-1])

        def run(rows):
            t0 = time.perf_counter()
            oracle.bgemm(Wb[:, :, :rows], Xb, w["K"])
            return time.perf_counter() - t0
        rows = 8
        dt = run(rows)
        rows = max(8, min(w["M"], int(rows * seconds_target / max(dt, 1e-3))))
        dt = run(rows)
        return 8.0 * rows * w["N"] * w["K"], dt, \
            f"{rows} of {w['M']} beam rows of one product (int64 loops)"

    geom = geometry_of(w)
    if w["geometry"] == "random":
        X = host_x(w)[:1]
        Wr = ti.random_phase_rows(0, min(256, w["M"]), w["K"])

        def run(rows):
            t0 = time.perf_counter()
            oracle.cgemm(Wr[:, :rows], X)
            return time.perf_counter() - t0
        rows = 4
        dt = run(rows)
        rows = max(4, min(Wr.shape[1], int(rows * seconds_target / max(dt, 1e-3))))
        dt = run(rows)
        return 8.0 * rows * w["N"] * w["K"], dt, f"{rows} of {w['M']} beam rows of one product"
    if w["geometry"] == "ultrasound":
        X = host_x(w)

        def run(rows):
            Wf = oracle.weights_fp16(geom.rx_pos, geom.targets[:rows], geom.freqs[:1], True, geom.c)
            t0 = time.perf_counter()
            oracle.cgemm(Wf, X)
            return time.perf_counter() - t0
        rows = 16
        dt = run(rows)
        rows = max(16, min(w["M"], int(rows * seconds_target / max(dt, 1e-3))))
        dt = run(rows)
        return 8.0 * rows * w["N"] * w["K"], dt, f"{rows} of {w['M']} voxel rows of the product"

    per_w = w["B"] // w["w_batches"]

    def sample(nb):
        nw = (nb + per_w - 1) // per_w
        Wf = oracle.weights_fp16(geom.rx_pos, geom.targets, geom.freqs[:nw], False, geom.c)
        X = np.stack([ti.radio_x_batch(1, b, w["K"], w["N"]) for b in range(nb)])
        return Wf, X
    Wf, X = sample(per_w)
    t0 = time.perf_counter()
    oracle.cgemm(Wf[:1], X[:per_w])
    dt1 = (time.perf_counter() - t0) / per_w
    nb = max(per_w, min(w["B"], int(seconds_target / max(dt1, 1e-3)) // per_w * per_w))
    Wf, X = sample(nb)
    t0 = time.perf_counter()
    oracle.cgemm(Wf, X)
    dt = time.perf_counter() - t0
    return 8.0 * nb * w["M"] * w["N"] * w["K"], dt, \
        f"{nb} of {w['B']} products (whole products, FP64 loops)"


def cpu_baseline(w, seconds):
    import oracle
    ops, dt, desc = oracle_sample(w, seconds)
    return {"value": ops / dt / 1e12, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "sample": desc, "seconds": round(dt, 3),
            "host_cpus": os.cpu_count()}


def reference_arm(args, w):
    """The oracle as the reference arm: each step one bounded sample."""
    import oracle
    target = 0.4      # seconds of oracle work per step
    _, _, desc = oracle_sample(w, target)
    for _ in range(args.warmup):
        oracle_sample(w, target)
    samples = [oracle_sample(w, target) for _ in range(args.steps)]
    tot_ops = sum(s[0] for s in samples)
    tot = sum(s[1] for s in samples)
    value = tot_ops / tot / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(samples),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64" if w["mode"] == "1bit" else "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": w["desc"], "batch": w["B"], "M": w["M"], "N": w["N"], "K": w["K"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": desc + " per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- GPU
class GpuWorkload:
    """Device-resident inputs and the step of one workload."""

    def __init__(self, w, local, config, xh=None):
        import numpy as np
        import torch
        import paper_2505_03269_gb300 as tcbf
        self.w = w
        B, M, N, K, Bw = w["B"], w["M"], w["N"], w["K"], w["w_batches"]
        self.Xh = host_x(w) if xh is None else xh
        if w["mode"] == "tf32":              # the TF32 path is for data that arrives in FP32
            self.Xh = self.Xh.astype(np.float32)
        self.src_type = tcbf.SRC_CF32 if self.Xh.dtype == np.float32 else tcbf.SRC_CF16
        self.Xd = torch.from_numpy(self.Xh).cuda()
        mode = (tcbf.MODE_1BIT if w["mode"] == "1bit" else
                tcbf.MODE_FP8SPLIT if is_fp8(w) else
                tcbf.MODE_TF32 if w["mode"] == "tf32" else tcbf.MODE_FP16)
        # compute-bound FP16 shapes pack X with a third, negated plane (two N = 256
        # MMAs per K step); the radio block reads X as it lies (no pack)
        lay = layout_of(w)
        flags = (tcbf.FLAG_STACKED_X if lay == "stacked" else
                 tcbf.FLAG_INTERLEAVED_X if lay == "interleaved" else 0)
        if w["mode"] == "fp8":
            flags = tcbf.FLAG_FP8_HI_ONLY
        if w.get("fp8_block"):
            flags |= tcbf.FLAG_FP8_BLOCK_SCALES
        self.layout = lay
        self.plan = tcbf.Plan(B, M, N, K, mode, w_batches=Bw, device=local, flags=flags)
        if config is not None:
            self.plan.set_config(config)
        self.Wp = torch.empty(self.plan.packed_size(0), dtype=torch.uint8, device="cuda")
        # interleaved X: the GEMM reads the resident samples themselves
        self.Xp = (self.Xd if lay == "interleaved" else
                   torch.empty(self.plan.packed_size(1), dtype=torch.uint8, device="cuda"))
        ydt = torch.int32 if w["mode"] == "1bit" else torch.float32
        self.Y = torch.empty((B, M, N, 2), dtype=ydt, device="cuda")
        self.weights_ms = None
        if w["mode"] == "1bit" and w["geometry"] is None:
            self.Wbits = onebit_weights(w)
            self.Wp.copy_(torch.from_numpy(self.Wbits.view(np.uint8).ravel()).cuda())
        elif w["geometry"] == "random":
            import tcbf_inputs as ti
            self.Wh = ti.random_phase_rows(0, Bw * M, K).reshape(Bw, M, K, 2)
            self.plan.transpose_pack(0, torch.from_numpy(self.Wh).cuda(), self.Wp)
        else:
            self.geom = geometry_of(w)
            rx = torch.from_numpy(self.geom.rx_pos).cuda()
            tg = torch.from_numpy(self.geom.targets).cuda()
            fr = torch.from_numpy(np.ascontiguousarray(self.geom.freqs[:Bw])).cuda()
            args = (rx, tg, self.geom.near_field, fr, self.geom.c, self.Wp)
            self.plan.weights_from_geometry(*args)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            self.plan.weights_from_geometry(*args)
            e1.record()
            torch.cuda.synchronize()
            self.weights_ms = e0.elapsed_time(e1)

    def fp4(self):
        """1-bit plan on the 4-bit tensor path: W is expanded to E2M1 once
        (weights fixed over the block, as they are packed once on the FP16
        path), and each step packs X straight into its E2M1 planes
        (tcbf_transpose_pack_expanded) before the GEMM."""
        return (self.w["mode"] == "1bit" and
                self.plan.config_name(self.plan.get_config()).startswith("1bit->e2m1"))

    def prepare_weights(self):
        if self.fp4():
            self.plan.expand_1bit(0, self.Wp)

    def pack(self):
        if self.fp4():                       # samples -> E2M1 planes in one pass
            self.plan.transpose_pack_expanded(1, self.Xd, self.src_type)
        elif self.layout != "interleaved":   # interleaved X needs no pack
            self.plan.transpose_pack(1, self.Xd, self.Xp, self.src_type)

    def prep(self):
        pass

    def gemm(self):
        if self.fp4():
            self.plan.beamform_1bit_expanded(self.Y)
        elif self.w["mode"] == "1bit":
            self.plan.beamform_1bit(self.Wp, self.Xp, self.Y)
        elif is_fp8(self.w):
            self.plan.beamform_fp8split(self.Wp, self.Xp, self.Y)
        elif self.w["mode"] == "tf32":
            self.plan.beamform_tf32(self.Wp, self.Xp, self.Y)
        else:
            self.plan.beamform_fp16(self.Wp, self.Xp, self.Y)

    def step(self):
        self.pack()
        self.prep()
        self.gemm()

    def gemm_bytes(self):
        """Algorithmic bytes of the GEMM: its operands in the method's own
        encoding (packed FP16 / FP8 / TF32 planes or the interleaved samples;
        for 1-bit the packed sign bits, 2 bits per complex value) read once,
        and Y written once.  FP16 and TF32 planes count K elements per row:
        their rows are padded to K rounded up to 64 (whole 128-byte lines),
        and the pad is zeros of the layout, not data."""
        w_bytes, x_bytes = self.plan.packed_size(0), self.plan.packed_size(1)
        if self.w["mode"] in ("fp16", "tf32"):
            K, Kp = self.w["K"], self.plan.Kp
            w_bytes = w_bytes * K // Kp
            if self.layout != "interleaved":
                x_bytes = x_bytes * K // Kp
        return w_bytes + x_bytes + self.Y.numel() * 4

    def fp4_plane_bytes(self):
        """Bytes the 4-bit 1-bit GEMM actually reads: its E2M1 planes (W: Wr,
        Wi; X: -Xi, Xr, Xi; 16 bytes per word of bits, rows of whole 128-byte
        lines) and Y."""
        w, kq = self.w, (self.plan.Kw + 7) // 8 * 8
        return (w["w_batches"] * 2 * w["M"] + w["B"] * 3 * w["N"]) * kq * 16 + self.Y.numel() * 4


def stacked_split_launches(gw):
    """1 when the stacked SM-pair GEMM splits its last wave (FP16, stacked X,
    configuration 0, K > 4096 in chunks of 2048, a partial last wave of r
    pair tiles with min(chunks, pairs // r) >= 2, N even, the chunk
    workspace within 64 MiB): a second kernel then adds the later chunks."""
    import torch
    w = gw.w
    if w["mode"] != "fp16" or gw.layout != "stacked" or gw.plan.get_config() != 0:
        return 0
    if w["K"] <= 4096 or w["N"] % 2:
        return 0
    pairs = torch.cuda.get_device_properties(0).multi_processor_count // 2
    tiles = -(-w["M"] // 256) * -(-w["N"] // 128) * w["B"]
    chunks, r = -(-w["K"] // 2048), tiles % pairs
    if r == 0 or min(chunks, pairs // r) < 2 or r * (chunks - 1) * 256 * 1024 > 64 << 20:
        return 0
    return 1


def fp8_error_vs_fp16(gw):
    """Accuracy of an FP8 step: the relative Frobenius distance of its Y
    from the FP16 path's Y for the same samples and geometry, computed on the
    device in FP64.  The FP16 GEMM is within 2e-5 of the exact product of
    its FP16 inputs (the tests' parity bar against the oracle), well below
    the E4M3 errors this measures."""
    import torch
    w16 = dict(gw.w, mode="fp16")
    w16.pop("fp8_block", None)
    g16 = GpuWorkload(w16, 0, None, xh=gw.Xh)
    try:
        g16.step()
        torch.cuda.synchronize()
        num = den = 0.0
        for b in range(gw.Y.shape[0]):
            r = g16.Y[b].double()
            num += float(torch.sum((gw.Y[b].double() - r) ** 2))
            den += float(torch.sum(r * r))
        return {"rel_err": (num / den) ** 0.5,
                "reference": "the FP16 path (" + g16.plan.config_name(g16.plan.get_config()) +
                             ") on the same samples and geometry, whole output, FP64 on the "
                             "device"}
    finally:
        g16.plan.close()
        del g16
        torch.cuda.empty_cache()


def roofline_of(gw, peaks, gemm_ms):
    """Roofline of the step's dominant kernel (the GEMM): bound, achieved,
    peak, fraction, with the algorithmic bytes / flops it is measured on."""
    w = gw.w
    ops = ops_per_step(w)
    gbytes = gw.gemm_bytes()
    mma_factor = 1.0
    if gw.fp4():
        tensor_peak = peaks["bf16_tflops"] * FP4_OVER_BF16
        peak_note = ("dense E2M1 tensor peak = measured bf16 burst x nominal fp4/bf16 ratio "
                     "13.5/2.25; the GEMM alone (the expansion of X is timed beside it)")
        kname = "cgemm_1bit_fp4_pair_kernel"
    elif w["mode"] == "1bit":
        tensor_peak = peaks["bf16_tflops"] * FP8_OVER_BF16
        peak_note = "E4M3 tensor peak = measured bf16 burst x nominal fp8/bf16 ratio 2"
        kname = "cgemm_1bit_kernel"
    elif w["mode"] == "tf32":
        tensor_peak = peaks["bf16_tflops"] * TF32_OVER_BF16
        peak_note = "TF32 tensor peak = measured bf16 burst x nominal tf32/bf16 ratio 1.1/2.25"
        kname = "cgemm_tc_kernel<tf32>"
    elif is_fp8(w):
        tensor_peak = peaks["bf16_tflops"] * FP8_OVER_BF16
        mma_factor = float(fp8_products(w))
        peak_note = ("E4M3 tensor peak = measured bf16 burst x nominal fp8/bf16 ratio 2; "
                     + ("algorithmic flops = 3 x useful (Wh Xh + Wh Xl + Wl Xh)"
                        if fp8_products(w) == 3 else "algorithmic flops = useful (Wh Xh)"))
        kname = "cgemm_tc_kernel<split-block>" if w.get("fp8_block") else "cgemm_tc_kernel<split>"
    else:
        tensor_peak = peaks["bf16_tflops"]
        peak_note = "FP16 tensor peak = measured bf16 burst (same dense rate)"
        kname = {"stacked": "cgemm_stacked_pair_kernel", "interleaved": "cgemm_ix_kernel"}.get(
            gw.layout, "cgemm_tc_kernel")
    ai = mma_factor * ops / gbytes
    ridge = tensor_peak * 1e12 / (peaks["hbm_gbs"] * 1e9)
    gemm_tops = mma_factor * ops / (gemm_ms * 1e-3) / 1e12
    gemm_gbs = gbytes / (gemm_ms * 1e-3) / 1e9
    if ai < ridge:
        roof = {"bound": "hbm", "achieved": gemm_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": gemm_gbs / peaks["hbm_gbs"]}
    else:
        roof = {"bound": "tensor", "achieved": gemm_tops, "peak": tensor_peak,
                "unit": "TFLOP/s", "frac": gemm_tops / tensor_peak}
    roof.update({"kernel": kname, "algorithmic_bytes": gbytes, "peak_source": peaks["source"],
                 "tensor_peak_note": peak_note,
                 "ceiling_tops": min(tensor_peak, ai * peaks["hbm_gbs"] / 1e3),
                 "algorithmic_flops_per_useful_op": mma_factor,
                 "gemm_tops": gemm_tops, "gemm_frac_of_tensor_peak": gemm_tops / tensor_peak})
    if gw.fp4():
        fb = gw.fp4_plane_bytes()
        roof["kernel_plane_bytes"] = fb
        roof["kernel_plane_gbs"] = fb / (gemm_ms * 1e-3) / 1e9
        roof["algorithmic_bytes_note"] = ("packed sign bits of W and X (2 bits per complex "
                                          "value) + int32 Y; the E2M1 planes the kernel reads "
                                          "are an intermediate of this design (kernel_plane_bytes)")
    if roof["bound"] == "hbm":
        # the same read and write bytes streamed alone: what this byte mix allows
        from paper_2505_03269_gb300 import peaks as tcbf_peaks
        wbytes = gw.Y.numel() * 4
        kbytes = roof.get("kernel_plane_bytes") or gbytes
        try:
            st = tcbf_peaks.stream((kbytes - wbytes) / 1e9, wbytes / 1e9)
        except Exception as exc:      # e.g. no room for the two buffers beside the workload
            roof["byte_mix_ceiling"] = {"unavailable": str(exc)}
            return roof
        ceil_gbs = max(v["gbs"] for k, v in st.items() if k.startswith("blocks_per_sm"))
        kgbs = kbytes / (gemm_ms * 1e-3) / 1e9
        roof["byte_mix_ceiling"] = {
            "read_bytes": st["read_bytes"], "write_bytes": st["write_bytes"], "gbs": ceil_gbs,
            "kernel_gbs": kgbs, "frac": kgbs / ceil_gbs,
            "how": "tcbf_peak_stream: the GEMM's read bytes with 16-byte loads, then its write "
                   "bytes with 16-byte stores, fastest of 4, 8 and 16 blocks per SM"}
    return roof


class Stepper:
    """Timed steps of one GpuWorkload: events around each kernel on the
    launch stream (pack, the 4-bit path's expansion of X, the GEMM)."""

    def __init__(self, gw):
        import torch
        self.gw = gw
        self.stream = torch.cuda.current_stream()

    def run(self, nsteps, sample_clocks=False):
        import torch
        gw, stream = self.gw, self.stream
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(nsteps)]
        sampler = ClockSampler(0) if sample_clocks else None
        if sampler:
            sampler.start()
        torch.cuda.synchronize()
        for i in range(nsteps):
            ev[i][0].record(stream)
            gw.pack()
            ev[i][1].record(stream)
            gw.prep()
            ev[i][2].record(stream)
            gw.gemm()
            ev[i][3].record(stream)
        torch.cuda.synchronize()
        clk = sampler.stop() if sampler else None
        return {"total_ms": ev[0][0].elapsed_time(ev[-1][3]),
                "pack_ms": statistics.mean(e[0].elapsed_time(e[1]) for e in ev),
                "prep_ms": statistics.mean(e[1].elapsed_time(e[2]) for e in ev),
                "gemm_ms": statistics.mean(e[2].elapsed_time(e[3]) for e in ev),
                "clocks": clk}


def measure_sub(name, w, args, peaks, traffic_key=None):
    """A configured workload as a sub-record: default configuration,
    args.sub_steps timed steps, roofline and clocks (FP8: error against the
    FP16 path)."""
    import torch
    gw = GpuWorkload(w, 0, None)
    try:
        gw.prepare_weights()
        st = Stepper(gw)
        for _ in range(3):
            gw.step()
        torch.cuda.synchronize()
        r = st.run(args.sub_steps, sample_clocks=True)
        status = gw.plan.last_device_error()
        ms = r["total_ms"] / args.sub_steps
        out = {"workload": w["desc"], "batch": w["B"], "M": w["M"], "N": w["N"], "K": w["K"],
               "value": tops(ops_per_step(w), ms), "unit": UNIT, "ms_per_step": ms,
               "steps": args.sub_steps,
               "dtype": ("e2m1" if gw.fp4() else
                         {"1bit": "u1", "fp8split": "e4m3x2", "fp8": "e4m3"}.get(w["mode"], "f16")),
               "fp8_scales": ("block (UE8M0 per 32 k)" if w.get("fp8_block") else
                              "row" if is_fp8(w) else None),
               "kernel_config": gw.plan.config_name(gw.plan.get_config()),
               "kernels": {"gemm_ms": r["gemm_ms"], "pack_ms": r["pack_ms"],
                           "pack_note": ("X packed straight into the E2M1 planes" if gw.fp4()
                                         else None),
                           "gemm_useful_tops": tops(ops_per_step(w), r["gemm_ms"])},
               "roofline": roofline_of(gw, peaks, r["gemm_ms"]),
               "clocks": r["clocks"], "device_status": status}
        if traffic_key:
            out["roofline"]["traffic"] = recorded_traffic(
                out["roofline"]["kernel"], traffic_key, out["kernel_config"])
        if is_fp8(w):
            out["error_vs_fp16_path"] = fp8_error_vs_fp16(gw)
        return out
    finally:
        gw.plan.close()
        del gw
        torch.cuda.empty_cache()


def measure_serving(args):
    """Configured serving stream: the continuous-batching server against the
    one-request-per-launch FP16 baseline at offered loads 0.8 and 0.95 of
    the baseline's capacity."""
    from paper_2505_03269_gb300 import serve
    t0 = time.perf_counter()
    r = serve.measure(n_requests=args.serving_requests, loads=(0.8, 0.95))
    r["seconds"] = time.perf_counter() - t0
    r["p99_ms_at_0.95"] = r["loads"][-1]["continuous_batching"]["p99_ms"]
    r["p50_ms_at_0.95"] = r["loads"][-1]["continuous_batching"]["p50_ms"]
    return r


def main():
    args = parse_args()
    if args.gpus != 1:
        # every product fits one GB300; the library and this benchmark are one-GPU only
        sys.exit(f"bench.py: --gpus {args.gpus} is not supported: this benchmark runs on one GPU")
    w = workload(args)
    if args.impl == "reference":
        reference_arm(args, w)
        return

    import numpy as np
    import torch

    import paper_2505_03269_gb300 as tcbf
    from paper_2505_03269_gb300 import build as tcbf_build

    torch.cuda.set_device(0)
    tcbf_build.build()
    tcbf.load()
    peaks = load_peaks()

    gw = GpuWorkload(w, 0, args.config)
    plan = gw.plan
    gw.prepare_weights()
    stream = torch.cuda.current_stream()
    st = Stepper(gw)
    warmup = max(args.warmup, 3)
    for _ in range(warmup):
        gw.step()
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0

    # ---- the fixed default configuration against the autotuned one
    tuning = None
    if args.config is None:
        d = st.run(max(3, args.steps // 4))
        default_name = plan.config_name(plan.get_config())
        from paper_2505_03269_gb300 import tuner
        entry = tuner.tune(plan, gw.Wp, gw.Xp, gw.Y, reps=3, store=False)
        tuning = {"default": {"config": default_name, "gemm_ms": d["gemm_ms"]},
                  "tuned": {"config": entry["name"]}, "ms_per_config": entry["ms"],
                  "how": "every configuration's whole beamform call (4-bit 1-bit path: "
                         "both expansions and the GEMM), timed round-robin"}
        gw.prepare_weights()
        for _ in range(2):
            gw.step()

    # ---- timed region: K steps (tuned configuration), clocks sampled
    r = st.run(args.steps, sample_clocks=True)
    total_ms, pack_ms, gemm_ms, clocks = r["total_ms"], r["pack_ms"], r["gemm_ms"], r["clocks"]
    status = plan.last_device_error()
    ms_per_step = total_ms / args.steps
    value = tops(ops_per_step(w), ms_per_step)
    if tuning is not None:
        tuning["tuned"]["gemm_ms"] = gemm_ms
        tuning["speedup_gemm"] = tuning["default"]["gemm_ms"] / gemm_ms

    # ---- the same step replayed as one captured CUDA graph
    plan.graph_capture(gw.Xd if gw.layout != "interleaved" else None, gw.Xp, gw.Wp, gw.Y,
                       gw.src_type)
    plan.graph_launch()
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        plan.graph_launch()
    g1.record(stream)
    torch.cuda.synchronize()
    graph_ms = g0.elapsed_time(g1) / args.steps

    fp8_error = fp8_error_vs_fp16(gw) if is_fp8(w) else None

    # ---- energy efficiency (Sec. IV: useful TeraOps/s over the GPU's mean power while the
    # kernels run): the step, then the GEMM alone, each looped for about a second and a
    # half with the board power sampled by nvidia-smi every 100 ms
    energy = None
    if not args.no_energy:
        def power_loop(unit, unit_ms):
            n = max(3, int(1500.0 / max(unit_ms, 1e-3)))
            sampler = ClockSampler(0)
            sampler.start()
            p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p0.record(stream)
            for _ in range(n):
                unit()
            p1.record(stream)
            torch.cuda.synchronize()
            clk = sampler.stop()
            ms = p0.elapsed_time(p1) / n
            t = tops(ops_per_step(w), ms)
            pw = clk["power_w_median"] if clk else None
            return {"tops": t, "ms": ms, "iterations": n,
                    "power_w_median": pw, "samples": clk["samples"] if clk else 0,
                    "sm_mhz": clk["sm_mhz"] if clk else None,
                    "reasons": clk["reasons"] if clk else None,
                    "tops_per_joule": t / pw if pw else None}
        energy = {"step": power_loop(gw.step, ms_per_step),
                  "gemm": power_loop(gw.gemm, gemm_ms),
                  "unit": "TeraOps/J",
                  "how": "useful TeraOps/s of a ~1.5 s loop divided by the median board power "
                         "nvidia-smi reports during it (every 100 ms); a sustained rate under "
                         "the board's power limit, below the short timed region's"}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        Xhost = torch.from_numpy(gw.Xh).pin_memory()
        Yhost = torch.empty(gw.Y.shape, dtype=gw.Y.dtype, pin_memory=True)
        src_type = 1 if gw.Xh.dtype == np.float32 else 0

        def e2e_step():
            gw.plan.beamform_host(Xhost, gw.Wp, Yhost, chunk=args.e2e_chunk, src_type=src_type,
                                  stream=stream)
        e2e_step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        # the host link's own device-to-host rate (one plain copy of up to 4 GiB of Y),
        # the floor the step's Y copy-out cannot beat
        nl = min(gw.Y.numel(), 1 << 30)
        ysrc, ydst = gw.Y.view(-1)[:nl], Yhost.view(-1)[:nl]
        ydst.copy_(ysrc, non_blocking=True)
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        ydst.copy_(ysrc, non_blocking=True)
        l1.record(stream)
        torch.cuda.synchronize()
        link_gbs = nl * 4 / (l0.elapsed_time(l1) * 1e-3) / 1e9
        te_ms = a.elapsed_time(b) / args.e2e_steps
        floor_ms = gw.Y.numel() * 4 / link_gbs / 1e6
        e2e = {"value": tops(ops_per_step(w), te_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(gw.Xh.nbytes), "d2h_bytes_per_step": int(gw.Y.numel() * 4),
               "ms_per_step": te_ms,
               "how": "tcbf_beamform_host on pinned host X and Y: "
                      + ("ranges of W rows of the one product (X in and packed once), "
                         "beamform of one range overlapped with the device-to-host copy of "
                         "the previous on separate streams" if w["B"] == 1 else
                         "chunks of batches, host-to-device copy, "
                         + ("beamform of the copied samples as they lie" if gw.layout == "interleaved"
                            else "pack + beamform")
                         + " and device-to-host copy of neighbouring chunks overlapped on "
                           "separate streams"),
               "chunk": ("about M / 4 rows, whole waves of 128-row tiles" if w["B"] == 1
                         else args.e2e_chunk or "auto (about batch / 16)"),
               "d2h_link_gbs": link_gbs, "d2h_floor_ms": floor_ms,
               "frac_of_d2h_floor": floor_ms / te_ms,
               # the larger of the two limits: the device-resident step and the Y copy-out
               "floor_ms": max(ms_per_step, floor_ms),
               "frac_of_floor": max(ms_per_step, floor_ms) / te_ms}
        del Xhost, Yhost

    # ---- roofline of the dominant kernel (the GEMM)
    roof = roofline_of(gw, peaks, gemm_ms)
    kname = roof["kernel"]
    fp4_micro = None
    if gw.fp4():
        # the 4-bit rate measured on chip by the library's microbenchmark
        # (kind::mxf4, operands in shared memory), beside the nominal-ratio peak
        from paper_2505_03269_gb300 import peaks as tcbf_peaks
        fp4_micro = tcbf_peaks.measure(7, 0)
    full_size = args.batches is None and args.m_rows is None
    traffic_key = f"{args.workload}/{w['mode']}" if full_size else None
    roof["traffic"] = recorded_traffic(kname, traffic_key, plan.config_name(plan.get_config()))
    gemm_tops = roof["gemm_tops"]
    pack_bytes = gw.Xh.nbytes + plan.packed_size(1)
    ops = ops_per_step(w)
    step_desc = ("transpose_pack_expanded(X) (sign-quantised straight into E2M1 planes) + "
                 "beamform_1bit_expanded (weights expanded once, resident)" if gw.fp4() else
                 "beamform_fp16 reading the resident interleaved samples (no transpose/pack "
                 "pass; weights resident)" if gw.layout == "interleaved" else
                 "transpose_pack(X) + beamform (weights resident)")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("e2m1" if gw.fp4() else
                  {"1bit": "u1", "fp8split": "e4m3x2", "fp8": "e4m3", "tf32": "tf32"}.get(
                      w["mode"], "f16")),
        "data": "synthetic",
        "config": {"workload": w["desc"], "batch": w["B"], "M": w["M"], "N": w["N"], "K": w["K"],
                   "w_batches": w["w_batches"], "step": step_desc, "x_layout": gw.layout,
                   "l2": "inputs larger than L2 (X %.2f GB, Y %.1f GB per step)"
                         % (gw.Xh.nbytes / 1e9, gw.Y.numel() * 4 / 1e9),
                   "kernel_config": plan.config_name(plan.get_config()),
                   "parallelism": "one GPU"},
        # kernels per step: the GEMM, plus pack(X) unless X is read interleaved
        # (the 4-bit 1-bit path packs X straight into its E2M1 planes); split-FP8
        # packs X in three kernels (column maxima, pack, exponents) after a memset
        "gpu_launches": ((4 if is_fp8(w) else 2 if gw.fp4() else
                          1 if gw.layout == "interleaved" else 2 + stacked_split_launches(gw))
                         * args.steps),
        "roofline": roof,
        "kernels": {"gemm_ms": gemm_ms, "pack_ms": pack_ms if gw.layout != "interleaved" else 0.0,
                    "weights_ms_once": gw.weights_ms,
                    "pack_x_into_e2m1_ms": pack_ms if gw.fp4() else None,
                    "gemm_useful_tops": ops / (gemm_ms * 1e-3) / 1e12,
                    "gemm_tops": gemm_tops, "gemm_frac_of_tensor_peak": roof["gemm_frac_of_tensor_peak"],
                    "fp4_microbench_tops": fp4_micro,
                    "gemm_frac_of_fp4_microbench": gemm_tops / fp4_micro if fp4_micro else None,
                    "gemm_gbs": gw.gemm_bytes() / (gemm_ms * 1e-3) / 1e9,
                    "gemm_ai_ops_per_byte": ops / gw.gemm_bytes()},
        "clocks": clocks,
        "autotune": tuning,
        "graph_step": {"ms_per_step": graph_ms, "value": tops(ops, graph_ms),
                       "how": "tcbf_graph_capture of the step, replayed K times (4-bit 1-bit "
                              "path: the captured call also expands W)"},
        "device_status": status,
        "error_vs_fp16_path": fp8_error,
        "e2e": e2e,
        "energy": energy,
    }
    if gw.layout != "interleaved" and not gw.fp4() and w["mode"] != "1bit":
        line["kernels"]["pack_gbs"] = pack_bytes / (pack_ms * 1e-3) / 1e9
        line["kernels"]["pack_frac_of_hbm"] = line["kernels"]["pack_gbs"] / peaks["hbm_gbs"]
    Xh_keep = gw.Xh
    plan.close()
    del gw, plan, st
    torch.cuda.empty_cache()

    # ---- the planar path of the same workload: transpose/pack X + planar GEMM
    if w.get("layout") == "interleaved" and args.config is None:
        wp = dict(w, layout="planar")
        gp = GpuWorkload(wp, 0, None, xh=Xh_keep)
        try:
            for _ in range(3):
                gp.step()
            torch.cuda.synchronize()
            from paper_2505_03269_gb300 import tuner
            tuner.tune(gp.plan, gp.Wp, gp.Xp, gp.Y, reps=2, store=False)
            rp = Stepper(gp).run(max(5, args.steps // 2))
            pms = rp["total_ms"] / max(5, args.steps // 2)
            line["planar_step"] = {
                "ms_per_step": pms, "value": tops(ops, pms), "pack_ms": rp["pack_ms"],
                "gemm_ms": rp["gemm_ms"],
                "pack_gbs": (gp.Xh.nbytes + gp.plan.packed_size(1)) / (rp["pack_ms"] * 1e-3) / 1e9,
                "kernel_config": gp.plan.config_name(gp.plan.get_config()),
                "how": "the same block through tcbf_transpose_pack into planes and the tuned "
                       "planar four-MMA GEMM, for comparison with the interleaved step"}
        finally:
            gp.plan.close()
            del gp
            torch.cuda.empty_cache()

    # ---- the other configured workloads, as sub-records
    if not args.no_subs and args.workload == "radio" and args.batches is None:
        subs = {}
        for key, wname, mode, scales in (("ultrasound_fp16", "ultrasound", None, "row"),
                                         ("ultrasound_fp8split", "ultrasound", "fp8split", "row"),
                                         ("ultrasound_fp8", "ultrasound", "fp8", "row"),
                                         ("ultrasound_fp8split_block", "ultrasound", "fp8split", "block"),
                                         ("ultrasound_fp8_block", "ultrasound", "fp8", "block"),
                                         ("onebit", "onebit", None, "row")):
            sa = argparse.Namespace(**vars(args))
            sa.workload, sa.mode, sa.layout, sa.batches, sa.m_rows = wname, mode, None, None, None
            sa.fp8_scales = scales
            try:
                ws = workload(sa)
                subs[key] = measure_sub(key, ws, args, peaks,
                                        traffic_key=f"{wname}/{ws['mode']}")
            except Exception as exc:      # reported, never silently dropped
                subs[key] = {"error": f"{type(exc).__name__}: {exc}"}
        try:
            subs["serving"] = measure_serving(args)
        except Exception as exc:
            subs["serving"] = {"error": f"{type(exc).__name__}: {exc}"}
        line["workloads"] = subs
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
