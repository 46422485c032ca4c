"""Size sweep of the complex GEMM (the paper's benchmark over matrix sizes,
Sec. IV-B, Fig. 4): batch 1, M = N = K = S for a grid of sizes that are and
are not multiples of the 128-row tile, FP16 and 1-bit, with the fixed
default configuration and the autotuned one.  In the paper the sizes that
are not a multiple of the work per thread block are padded, which shows as a
sawtooth; here the TMA loads fill the out-of-range part of a tile with zeros
and the stores clip it, so only the partial tile's MMA work is extra.

  python -m paper_2505_03269_gb300.sweep [--sizes 256,1000,...] [--modes fp16,1bit]

Prints one markdown table row per (mode, size).  Inputs are seeded random
values drawn on the device (timing only; parity is the tests' job).
"""
from __future__ import annotations

import argparse

DEFAULT_SIZES = [256, 512, 1000, 1024, 1500, 2000, 2048, 3000, 4096, 4100, 6144, 8192]


def _time(fn, reps):
    import torch
    s = torch.cuda.current_stream()
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_size(mode: str, S: int, seed: int = 0):
    import torch
    import paper_2505_03269_gb300 as tcbf
    m = tcbf.MODE_1BIT if mode == "1bit" else tcbf.MODE_FP16
    g = torch.Generator(device="cuda").manual_seed(seed + S)
    W = torch.randn((1, S, S, 2), generator=g, device="cuda").half()
    X = torch.randn((1, S, S, 2), generator=g, device="cuda").half()
    ops = 8.0 * S * S * S
    with tcbf.Plan(1, S, S, S, m) as plan:
        Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
        plan.transpose_pack(0, W, Wp)
        plan.transpose_pack(1, X, Xp)
        Y = torch.empty((1, S, S, 2), dtype=torch.int32 if mode == "1bit" else torch.float32,
                        device="cuda")
        gemm = plan.beamform_1bit if mode == "1bit" else plan.beamform_fp16
        reps = max(5, min(200, int(2e13 / ops)))

        def one():
            gemm(Wp, Xp, Y)
        default_ms = _time(one, reps)
        best, _ = plan.autotune(Wp, Xp, Y, reps=3)
        tuned_ms = _time(one, reps)
        status = plan.last_device_error()
        return {"mode": mode, "S": S, "default_ms": default_ms,
                "default_tops": ops / (default_ms * 1e-3) / 1e12,
                "tuned": plan.config_name(best), "tuned_ms": tuned_ms,
                "tuned_tops": ops / (tuned_ms * 1e-3) / 1e12, "status": status}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default=",".join(str(s) for s in DEFAULT_SIZES))
    ap.add_argument("--modes", default="fp16,1bit")
    args = ap.parse_args()
    print("| mode | S | default ms | default TeraOps/s | tuned TeraOps/s | tuned configuration |")
    print("|---|---|---|---|---|---|")
    for mode in args.modes.split(","):
        for S in (int(x) for x in args.sizes.split(",")):
            r = run_size(mode, S)
            assert r["status"] == 0, r
            print(f"| {mode} | {S} | {r['default_ms']:.4f} | {r['default_tops']:.0f} | "
                  f"{r['tuned_tops']:.0f} | {r['tuned']} |", flush=True)


if __name__ == "__main__":
    main()
