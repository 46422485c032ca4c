"""The allocation-free FP16 beamform entry point, checked against the
ordinary plan-based path.

tcbf_beamform_fp16_noalloc is for callers that cannot allocate device memory
when they beamform (stream capture, real-time loops, host frameworks that own
the memory budget): it packs the samples into a fixed static device array
instead of a caller buffer and needs no plan.  Its output must equal the
plan path's (transpose_pack + beamform_fp16, the same kernels with the
default configuration) bit for bit, and the FP64 oracle within the FP16
tolerance, on consecutive calls that reuse the same static array, for FP16
and FP32 sources.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

import oracle
import tcbf_inputs as ti

TOL = 2e-5


def _lib():
    from paper_2505_03269_gb300 import binding
    from paper_2505_03269_gb300 import build as tcbf_build
    try:
        tcbf_build.build()
    except RuntimeError as exc:      # no CUDA toolkit on this runner
        pytest.skip(f"libtcbf.so cannot be built here: {exc}")
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
    from paper_2505_03269_gb300 import MODE_FP16, SRC_CF16, SRC_CF32, Plan

    def plan_path(W, X, src_type):
        Bw, M, K, _ = W.shape
        B, _, N, _ = X.shape
        with Plan(B, M, N, K, MODE_FP16, w_batches=Bw) as plan:
            Wd = torch.from_numpy(W).cuda()
            Xd = torch.from_numpy(X).cuda()
            Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
            Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
            Y = torch.empty((B, M, N, 2), dtype=torch.float32, device="cuda")
            plan.transpose_pack(0, Wd, Wp)
            plan.transpose_pack(1, Xd, Xp, src_type)
            plan.beamform_fp16(Wp, Xp, Y)
            torch.cuda.synchronize()
            assert plan.last_device_error() == 0
            return Wp, Y.cpu().numpy()

    cases = [dict(seed=1, B=3, Bw=3, M=100, N=200, K=77, f32=False),
             dict(seed=2, B=4, Bw=2, M=130, N=96, K=300, f32=False),
             dict(seed=3, B=2, Bw=1, M=64, N=130, K=50, f32=True)]
    for c in cases:
        W, _ = ti.small_fp16(seed=c["seed"], M=c["M"], K=c["K"], N=8, B=c["Bw"])
        X = ti.complex_gaussian_fp16(ti.rng(c["seed"] + 10), (c["B"], c["K"], c["N"]))
        src_type = SRC_CF16
        if c["f32"]:      # an FP32 source, rounded to FP16 by both paths
            X = (X.astype(np.float32) * np.float32(1.0 + 2.0 ** -13)).astype(np.float32)
            src_type = SRC_CF32
        Wp, Yref = plan_path(W, X, src_type)
        Xd = torch.from_numpy(X).cuda()
        Y = torch.full((c["B"], c["M"], c["N"], 2), float("nan"), dtype=torch.float32,
                       device="cuda")
        st = binding.beamform_fp16_noalloc(c["B"], c["M"], c["N"], c["K"], Wp, Xd, Y,
                                           w_batches=c["Bw"], device=0, src_type=src_type,
                                           check=True)
        assert st == 0, binding.status_string(st)
        torch.cuda.synchronize()
        got = Y.cpu().numpy()
        # the same pack and GEMM kernels as the plan path: bit for bit
        assert np.array_equal(got, Yref)
        # and against the FP64 oracle on the FP16 values both paths multiply
        Yc = got.astype(np.float64)
        X16 = X.astype(np.float16) if c["f32"] else X
        ref = oracle.cgemm(W, X16)
        assert oracle.rel_frobenius(Yc[..., 0] + 1j * Yc[..., 1], ref) <= TOL
        # the same call without the status check (no synchronisation inside)
        Y.fill_(float("nan"))
        st = binding.beamform_fp16_noalloc(c["B"], c["M"], c["N"], c["K"], Wp, Xd, Y,
                                           w_batches=c["Bw"], device=0, src_type=src_type,
                                           check=False)
        assert st == 0, binding.status_string(st)
        torch.cuda.synchronize()
        assert np.array_equal(Y.cpu().numpy(), Yref)
