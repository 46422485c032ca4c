"""Run the library's on-chip peak microbenchmarks (include/tcbf_peak.h) and
print one JSON object: TeraOps/s per kind, with the SM clock seen.

  python -m paper_2505_03269_gb300.peaks [--device D] [--scale S]
  python -m paper_2505_03269_gb300.peaks --stream READ_GB WRITE_GB [--device D]

--stream times an HBM stream with that read/write mix instead (the
ceiling of a memory-bound step's byte mix) for 4, 8 and 16 blocks per SM.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import subprocess

from . import binding
from . import build as tcbf_build

KINDS = {
    0: ("tcgen05_f16_m128n256k16", 40000),
    1: ("tcgen05_f8f6f4_e4m3_m128n256k32", 40000),
    2: ("tcgen05_i8", 1),
    3: ("mma_sync_f16_m16n8k16", 20000),
    4: ("mma_sync_b1_and_m16n8k256", 20000),
    5: ("cuda_core_popc_xor32", 20000),
    6: ("tcgen05_f16_m128n128k16", 80000),
    7: ("tcgen05_mxf4_e2m1_m128n256k64", 40000),
    8: ("tcgen05_mxf4nvf4_ue4m3x16_m128n256k64", 40000),
    9: ("tcgen05_mxf4nvf4_ue8m0x32_m128n256k64", 40000),
}


def sm_clock(device: int):
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(device), "--query-gpu=clocks.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=10).stdout.strip()
        return float(out)
    except Exception:
        return None


def _peak_fn():
    lib = binding.load()
    f = lib.tcbf_peak_run
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                  ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    return f


def measure(kind: int, device: int = 0) -> float:
    """TeraOps/s of one microbenchmark kind (raises on a failed run)."""
    sec, ops = ctypes.c_double(), ctypes.c_double()
    st = _peak_fn()(kind, device, KINDS[kind][1], ctypes.byref(sec), ctypes.byref(ops))
    if st != 0:
        raise binding.TcbfError(st, f"tcbf_peak_run({kind})")
    return ops.value / sec.value / 1e12


def stream(read_gb: float, write_gb: float, device: int = 0) -> dict:
    """GB/s of tcbf_peak_stream for the given read and write volumes."""
    tcbf_build.build()
    lib = binding.load()
    f = lib.tcbf_peak_stream
    f.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                  ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    rb = int(read_gb * 1e9) // 16 * 16
    wb = int(write_gb * 1e9) // 16 * 16
    res = {"read_bytes": rb, "write_bytes": wb}
    for per_sm in (4, 8, 16):
        sec = ctypes.c_double()
        st = f(device, rb, wb, per_sm, ctypes.byref(sec))
        if st != 0:
            raise binding.TcbfError(st, "tcbf_peak_stream")
        res[f"blocks_per_sm_{per_sm}"] = {"ms": sec.value * 1e3,
                                          "gbs": (rb + wb) / sec.value / 1e9}
    return res


def run(device: int = 0, scale: float = 1.0) -> dict:
    tcbf_build.build()
    f = _peak_fn()
    res = {}
    for kind, (name, iters) in KINDS.items():
        sec, ops = ctypes.c_double(), ctypes.c_double()
        st = f(kind, device, max(1, int(iters * scale)), ctypes.byref(sec), ctypes.byref(ops))
        if st != 0:
            res[name] = {"status": binding.STATUS_NAMES.get(st, st)}
            continue
        res[name] = {"tops": ops.value / sec.value / 1e12, "seconds": sec.value,
                     "sm_mhz_after": sm_clock(device)}
    return res


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--stream", type=float, nargs=2, metavar=("READ_GB", "WRITE_GB"))
    a = ap.parse_args()
    if a.stream:
        print(json.dumps(stream(a.stream[0], a.stream[1], a.device)))
    else:
        print(json.dumps(run(a.device, a.scale)))
