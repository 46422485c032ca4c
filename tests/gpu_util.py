"""Helpers for the GPU parity tests: build/load the library and run the
CUDA path on numpy inputs.  Every computation goes through libtcbf.so."""
from __future__ import annotations

import numpy as np
import torch

import paper_2505_03269_gb300 as tcbf
from paper_2505_03269_gb300 import build as tcbf_build


def ensure_lib():
    tcbf_build.build()
    return tcbf.load()


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def empty_bytes(n: int) -> torch.Tensor:
    return torch.empty(max(n, 16), dtype=torch.uint8, device="cuda")


def run_fp16(W: np.ndarray, X: np.ndarray, config: int | None = None, src_type=tcbf.SRC_CF16,
             flags: int = 0, rows=None):
    """W [Bw,M,K,2], X [B,K,N,2] (fp16 or fp32 pairs) -> Y complex128 [B,M,N] via the GPU.
    flags: plan flags (e.g. FLAG_INTERLEAVED_X); rows: per-batch beam counts."""
    Bw, M, K, _ = W.shape
    B, _, N, _ = X.shape
    with tcbf.Plan(B, M, N, K, tcbf.MODE_FP16, w_batches=Bw, flags=flags) as plan:
        if config is not None:
            plan.set_config(config)
        if rows is not None:
            plan.set_batch_rows(rows)
        Wd, Xd = dev(W), dev(X)
        Wp = empty_bytes(plan.packed_size(0))
        Xp = empty_bytes(plan.packed_size(1))
        Y = torch.empty((B, M, N, 2), dtype=torch.float32, device="cuda")
        plan.transpose_pack(0, Wd, Wp, src_type)
        plan.transpose_pack(1, Xd, Xp, src_type)
        plan.beamform_fp16(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        Yh = Y.cpu().numpy().astype(np.float64)
    return Yh[..., 0] + 1j * Yh[..., 1]
