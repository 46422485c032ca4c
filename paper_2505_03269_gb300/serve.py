"""Continuous-batching beamforming server: ctypes shim of include/tcbf_server.h
and the serving-stream measurement.

The server itself (admission by HBM budget, multi-stream overlap, resident
weight sets, completion tracking) is native code in libtcbf.so; this module
marshals arguments and computes latency percentiles from its per-request
timestamps.

Serving stream (stand-in for live beamforming requests): 32 resident weight
sets with beams in [64, 4096] and receivers in [64, 2048] drawn log-uniform
once; requests with samples in [256, 8192] log-uniform, modes 70% FP16,
20% split-FP8, 10% 1-bit, Poisson arrivals at a chosen fraction of the
capacity of the one-request-per-launch FP16 baseline.

  python -m paper_2505_03269_gb300.serve [--requests 600] [--load 0.8]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math

import numpy as np

from . import binding
from .binding import MODE_1BIT, MODE_FP8SPLIT, MODE_FP16, SRC_CF16, Plan, _check

SERVER_SYMBOLS = ["tcbf_server_create", "tcbf_server_register_weights", "tcbf_server_submit",
                  "tcbf_server_start", "tcbf_server_wait_all", "tcbf_server_result",
                  "tcbf_server_stats", "tcbf_server_destroy"]


class Request(ctypes.Structure):
    _fields_ = [("set_id", ctypes.c_int32), ("mode", ctypes.c_int32), ("N", ctypes.c_int64),
                ("src_type", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("host_x", ctypes.c_void_p), ("host_y", ctypes.c_void_p),
                ("arrival_s", ctypes.c_double)]


class RequestResult(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("stream", ctypes.c_int32),
                ("status", ctypes.c_int32), ("ops", ctypes.c_double)]


class Counters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("pending", ctypes.c_uint64),
                ("inflight", ctypes.c_uint64), ("peak_inflight", ctypes.c_int64),
                ("arena_bytes", ctypes.c_uint64), ("peak_arena_bytes", ctypes.c_uint64)]


def _lib():
    lib = binding.load()
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    sig = {
        "tcbf_server_create": [ctypes.POINTER(vp), i32, ctypes.c_size_t, i32, i32],
        "tcbf_server_register_weights": [vp, i32, i32, i64, i64, vp],
        "tcbf_server_submit": [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)],
        "tcbf_server_start": [vp],
        "tcbf_server_wait_all": [vp, ctypes.c_double],
        "tcbf_server_result": [vp, ctypes.c_uint64, ctypes.POINTER(RequestResult)],
        "tcbf_server_stats": [vp, ctypes.POINTER(Counters)],
        "tcbf_server_destroy": [vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    return lib


class Server:
    def __init__(self, arena_bytes: int, num_streams: int = 4, max_inflight: int = 0, device=0):
        self.lib = _lib()
        h = ctypes.c_void_p()
        _check(self.lib.tcbf_server_create(ctypes.byref(h), device, int(arena_bytes),
                                           num_streams, max_inflight), "tcbf_server_create")
        self.h = h

    def register_weights(self, set_id, mode, M, K, Wp):
        _check(self.lib.tcbf_server_register_weights(self.h, set_id, mode, M, K,
                                                     ctypes.c_void_p(Wp.data_ptr())),
               "tcbf_server_register_weights")

    def submit(self, set_id, mode, N, host_x, host_y=None, arrival_s=0.0, src_type=SRC_CF16):
        r = Request(set_id, mode, N, src_type, 0, ctypes.c_void_p(host_x.data_ptr()),
                    ctypes.c_void_p(host_y.data_ptr()) if host_y is not None else None,
                    float(arrival_s))
        t = ctypes.c_uint64()
        _check(self.lib.tcbf_server_submit(self.h, ctypes.byref(r), ctypes.byref(t)),
               "tcbf_server_submit")
        return t.value

    def start(self):
        _check(self.lib.tcbf_server_start(self.h), "tcbf_server_start")

    def wait_all(self, timeout_s=600.0):
        _check(self.lib.tcbf_server_wait_all(self.h, float(timeout_s)), "tcbf_server_wait_all")

    def result(self, ticket) -> RequestResult:
        out = RequestResult()
        _check(self.lib.tcbf_server_result(self.h, ticket, ctypes.byref(out)), "tcbf_server_result")
        return out

    def counters(self) -> Counters:
        out = Counters()
        _check(self.lib.tcbf_server_stats(self.h, ctypes.byref(out)), "tcbf_server_stats")
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.tcbf_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------ request stream
def log_uniform_int(g, lo, hi, size=None):
    return np.floor(np.exp(g.uniform(math.log(lo), math.log(hi + 1), size))).astype(np.int64)


def make_weight_sets(seed=0, n_sets=32, beams=(64, 4096), receivers=(64, 2048)):
    g = np.random.Generator(np.random.PCG64(seed))
    M = log_uniform_int(g, *beams, n_sets)
    K = log_uniform_int(g, *receivers, n_sets)
    return [(int(m), int(k)) for m, k in zip(M, K)]


def make_stream(seed=1, n_requests=600, n_sets=32, samples=(256, 8192),
                mix=((MODE_FP16, 0.7), (MODE_FP8SPLIT, 0.2), (MODE_1BIT, 0.1))):
    """Requests (set, mode, N) in arrival order; arrival times are assigned
    separately for a chosen rate (unit-rate exponential gaps returned)."""
    g = np.random.Generator(np.random.PCG64(seed))
    sets = g.integers(0, n_sets, n_requests)
    modes = g.choice([m for m, _ in mix], n_requests, p=[p for _, p in mix])
    N = log_uniform_int(g, *samples, n_requests)
    gaps = g.exponential(1.0, n_requests)
    return [dict(set_id=int(s), mode=int(m), N=int(n), gap=float(t))
            for s, m, n, t in zip(sets, modes, N, gaps)]


def setup_weights(server, sets, modes, seed=2):
    """Pack each resident weight set (random unit-phase W) for each mode."""
    import torch
    import tcbf_inputs as ti
    keep = []
    for sid, (M, K) in enumerate(sets):
        W, _ = ti.small_fp16(seed=seed + sid, M=M, K=K, N=1)
        Wd = torch.from_numpy(W).cuda()
        for mode in modes:
            with Plan(1, M, 1, K, mode) as plan:
                Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
                plan.transpose_pack(0, Wd, Wp)
            server.register_weights(sid, mode, M, K, Wp)
            keep.append(Wp)
    torch.cuda.synchronize()
    return keep


def run_stream(reqs, sets, rate, arena_bytes, num_streams, max_inflight, force_mode=None,
               host_x=None, host_y=None):
    """Serve `reqs` with Poisson arrivals at `rate` requests/s (rate None:
    all at t = 0).  Returns per-request (arrival, admit, done, ops)."""
    modes = sorted({force_mode if force_mode is not None else r["mode"] for r in reqs})
    with Server(arena_bytes, num_streams, max_inflight) as srv:
        keep = setup_weights(srv, sets, modes)
        t = 0.0
        tickets = []
        for r in reqs:
            if rate is not None:
                t += r["gap"] / rate
            mode = force_mode if force_mode is not None else r["mode"]
            tickets.append(srv.submit(r["set_id"], mode, r["N"], host_x, host_y,
                                      arrival_s=t if rate is not None else 0.0))
        srv.start()
        srv.wait_all()
        res = [srv.result(tk) for tk in tickets]
        cnt = srv.counters()
        del keep
    arr = np.array([[x.arrival_s, x.admit_s, x.done_s, x.ops, x.status] for x in res])
    return arr, cnt


def summarize(arr, cnt=None):
    lat = (arr[:, 2] - arr[:, 0]) * 1e3
    span = arr[:, 2].max() - arr[:, 0].min()
    out = {"requests": int(len(arr)), "failed": int(np.sum(arr[:, 4] != 0)),
           "throughput_tops": float(arr[:, 3].sum() / span / 1e12),
           "requests_per_s": float(len(arr) / span),
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "mean_ms": float(lat.mean()), "makespan_s": float(span)}
    if cnt is not None:
        out["peak_inflight"] = int(cnt.peak_inflight)
        out["peak_arena_gb"] = cnt.peak_arena_bytes / 1e9
    return out


def measure(n_requests=600, loads=(0.5, 0.8, 0.95, 1.5, 3.0), arena_gb=120.0, num_streams=8,
            seed=1):
    """Capacity of the serial FP16 baseline (all requests at t = 0, one at a
    time, one stream), then the same request stream with Poisson arrivals at
    each load (x that capacity) through the continuous-batching server (mixed
    modes) and through the serial FP16 baseline."""
    import torch
    sets = make_weight_sets()
    reqs = make_stream(seed=seed, n_requests=n_requests)
    Kmax = max(k for _, k in sets)
    Mmax = max(m for m, _ in sets)
    Nmax = max(r["N"] for r in reqs)
    g = np.random.default_rng(3)
    host_x = torch.from_numpy(
        g.standard_normal((Kmax, Nmax, 2)).astype(np.float16)).pin_memory()
    host_y = torch.empty((Mmax, Nmax, 2), dtype=torch.float32, pin_memory=True)
    arena = int(arena_gb * 1e9)
    base, _ = run_stream(reqs, sets, None, arena, 1, 1, MODE_FP16, host_x, host_y)
    capacity = len(reqs) / (base[:, 2].max() - base[:, 0].min())
    sat, sc = run_stream(reqs, sets, None, arena, num_streams, 0, None, host_x, host_y)
    out = {"stream": {"requests": n_requests, "weight_sets": len(sets),
                      "modes": "70% FP16 / 20% split-FP8 / 10% 1-bit", "arena_gb": arena_gb,
                      "streams": num_streams, "baseline_capacity_per_s": capacity,
                      "host_y": "one shared pinned sink (results discarded)"},
           "all_at_once": {"continuous_batching": summarize(sat, sc),
                           "serial_fp16_one_per_launch": summarize(base)},
           "loads": []}
    for load in loads:
        rate = load * capacity
        cont, cc = run_stream(reqs, sets, rate, arena, num_streams, 0, None, host_x, host_y)
        serial, scc = run_stream(reqs, sets, rate, arena, 1, 1, MODE_FP16, host_x, host_y)
        out["loads"].append({"load": load, "rate_per_s": rate,
                             "continuous_batching": summarize(cont, cc),
                             "serial_fp16_one_per_launch": summarize(serial, scc)})
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=600)
    ap.add_argument("--loads", type=str, default="0.5,0.8,0.95,1.5,3.0")
    ap.add_argument("--arena-gb", type=float, default=120.0)
    ap.add_argument("--streams", type=int, default=8)
    a = ap.parse_args()
    loads = tuple(float(x) for x in a.loads.split(","))
    print(json.dumps(measure(a.requests, loads, a.arena_gb, a.streams)))
