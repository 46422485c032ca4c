"""Size sweep of the complex GEMM (the paper's benchmark over matrix sizes,
Sec. IV-B, Fig. 4): batch 1, M = N = K = S for a grid of sizes that are and
are not multiples of the 128-row tile, FP16 and 1-bit, with the plan's
default layout and configuration and the autotuned ones.  In the paper the sizes that
are not a multiple of the work per thread block are padded, which shows as a
sawtooth; here the TMA loads fill the out-of-range part of a tile with zeros
and the stores clip it, so only the partial tile's MMA work is extra.

  python -m paper_2505_03269_gb300.sweep [--sizes 256,1000,...] [--modes fp16,1bit]
      [--layouts auto,planar,stacked,interleaved]

Prints one markdown table row per (mode, FP16 X layout, size): "auto" lets
the plan choose the layout (TCBF_FLAG_AUTO_LAYOUT), the others fix it.  Inputs are seeded random
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


LAYOUT_FLAGS = {"planar": 0, "stacked": 1, "interleaved": 8, "auto": 32}


def run_size(mode: str, S: int, layout: str = "auto", seed: int = 0, rounds: int = 3):
    """One size: a plan as created ("default": the create-time layout and
    configuration) and a tuned one (FP16 "auto": tcbf_autotune_layout over
    the planar and stacked layouts; otherwise tcbf_autotune), timed in
    alternating rounds so that a drift of the clocks affects both alike;
    each keeps its fastest round."""
    import torch
    import paper_2505_03269_gb300 as tcbf
    m = tcbf.MODE_1BIT if mode == "1bit" else tcbf.MODE_FP16
    flags = LAYOUT_FLAGS[layout] if m == tcbf.MODE_FP16 else 0
    g = torch.Generator(device="cuda").manual_seed(seed + S)
    W = torch.randn((1, S, S, 2), generator=g, device="cuda").half()
    X = torch.randn((1, S, S, 2), generator=g, device="cuda").half()
    ops = 8.0 * S * S * S
    Y = torch.empty((1, S, S, 2), dtype=torch.int32 if mode == "1bit" else torch.float32,
                    device="cuda")
    with tcbf.Plan(1, S, S, S, m, flags=flags) as dplan, tcbf.Plan(1, S, S, S, m, flags=flags) as tplan:
        Wp = torch.empty(dplan.packed_size(0), dtype=torch.uint8, device="cuda")
        dplan.transpose_pack(0, W, Wp)
        default_layout = layout_name(dplan.flags) if m == tcbf.MODE_FP16 else "1-bit"
        layout_ms = None
        if flags == LAYOUT_FLAGS["auto"]:
            _, layout_ms = tplan.autotune_layout(Wp, X, Y, reps=3)
        plans = []
        for plan in (dplan, tplan):
            Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
            plan.transpose_pack(1, X, Xp)
            plans.append((plan, Xp))
        if flags != LAYOUT_FLAGS["auto"]:
            tplan.autotune(Wp, plans[1][1], Y, reps=3)
        reps = max(5, min(200, int(2e13 / ops)))
        best = [float("inf"), float("inf")]
        for _ in range(rounds):
            for i, (plan, Xp) in enumerate(plans):
                gemm = plan.beamform_1bit if mode == "1bit" else plan.beamform_fp16
                best[i] = min(best[i], _time(lambda: gemm(Wp, Xp, Y), reps))
        status = dplan.last_device_error() or tplan.last_device_error()
        return {"mode": mode, "S": S, "layout": default_layout,
                "tuned_layout": layout_name(tplan.flags) if m == tcbf.MODE_FP16 else "1-bit",
                "default_ms": best[0], "default_tops": ops / (best[0] * 1e-3) / 1e12,
                "tuned": tplan.config_name(tplan.get_config()), "tuned_ms": best[1],
                "tuned_tops": ops / (best[1] * 1e-3) / 1e12, "layout_ms": layout_ms,
                "status": status}


def layout_name(flags: int) -> str:
    if flags & LAYOUT_FLAGS["stacked"]:
        return "stacked"
    if flags & LAYOUT_FLAGS["interleaved"]:
        return "interleaved"
    return "planar"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default=",".join(str(s) for s in DEFAULT_SIZES))
    ap.add_argument("--modes", default="fp16,1bit")
    ap.add_argument("--layouts", default="auto",
                    help="FP16 X layouts: any of auto, planar, stacked, interleaved")
    args = ap.parse_args()
    print("| mode | layout | S | default ms | default TeraOps/s | tuned TeraOps/s | "
          "tuned layout | tuned configuration |")
    print("|---|---|---|---|---|---|---|---|")
    for mode in args.modes.split(","):
        layouts = args.layouts.split(",") if mode == "fp16" else ["planar"]
        for layout in layouts:
            for S in (int(x) for x in args.sizes.split(",")):
                r = run_size(mode, S, layout)
                assert r["status"] == 0, r
                print(f"| {mode} | {r['layout']} | {S} | {r['default_ms']:.4f} | "
                      f"{r['default_tops']:.0f} | {r['tuned_tops']:.0f} | {r['tuned_layout']} | "
                      f"{r['tuned']} |", flush=True)


if __name__ == "__main__":
    main()
