"""The allocation-free FP16 beamform entry point, checked against the
ordinary plan-based path.

tcbf_beamform_fp16_noalloc is for callers that cannot allocate device memory
when they beamform (stream capture, real-time loops, host frameworks that own
the memory budget): it packs the samples into a fixed static device array
instead of a caller buffer and needs no plan.  Its output must equal the
plan path's (transpose_pack + beamform_fp16) within the FP16 tolerance, on
consecutive calls that reuse the same static array.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

import tcbf_inputs as ti

TOL = 2e-5


def _lib():
    from paper_2505_03269_gb300 import binding
    from paper_2505_03269_gb300 import build as tcbf_build
    tcbf_build.build()
    return binding


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    """Packed samples above 64 MiB: TCBF_ERR_BUDGET before any device work."""
    binding = _lib()
    # 512 x 2 x 4096 x 288 x 2 bytes = 2.4 GB of packed samples
    st = binding.beamform_fp16_noalloc(512, 1024, 4096, 288, 16, 16, 16, w_batches=256,
                                       check=False, stream=0)
    assert st == 4


@pytest.mark.gpu
def test_noalloc_matches_plan_path_on_consecutive_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    binding = _lib()
    from paper_2505_03269_gb300 import MODE_FP16, Plan

    def plan_path(W, X):
        Bw, M, K, _ = W.shape
        B, _, N, _ = X.shape
        with Plan(B, M, N, K, MODE_FP16, w_batches=Bw) as plan:
            Wd = torch.from_numpy(W).cuda()
            Xd = torch.from_numpy(X).cuda()
            Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
            Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
            Y = torch.empty((B, M, N, 2), dtype=torch.float32, device="cuda")
            plan.transpose_pack(0, Wd, Wp)
            plan.transpose_pack(1, Xd, Xp)
            plan.beamform_fp16(Wp, Xp, Y)
            torch.cuda.synchronize()
            assert plan.last_device_error() == 0
            return Wp, Y.cpu().numpy()

    def rel(a, b):
        return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))

    cases = [dict(seed=1, B=3, Bw=3, M=100, N=200, K=77),
             dict(seed=2, B=4, Bw=2, M=130, N=96, K=300)]
    for c in cases:
        W, _ = ti.small_fp16(seed=c["seed"], M=c["M"], K=c["K"], N=8, B=c["Bw"])
        X = ti.complex_gaussian_fp16(ti.rng(c["seed"] + 10), (c["B"], c["K"], c["N"]))
        Wp, Yref = plan_path(W, X)
        Xd = torch.from_numpy(X).cuda()
        Y = torch.full((c["B"], c["M"], c["N"], 2), float("nan"), dtype=torch.float32,
                       device="cuda")
        st = binding.beamform_fp16_noalloc(c["B"], c["M"], c["N"], c["K"], Wp, Xd, Y,
                                           w_batches=c["Bw"], device=0, check=True)
        assert st == 0, binding.status_string(st)
        torch.cuda.synchronize()
        assert rel(Y.cpu().numpy(), Yref) <= TOL
