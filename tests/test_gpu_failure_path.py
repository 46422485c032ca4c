"""The device-side failure path, tested without a fault: every wait in the
GEMM kernels gives up after 2 s and records it in the plan's status word.
The test hook tcbf_debug_drop_fill leaves one operand load of the first CTA
out, so its MMA issuer, producer and epilogue waits run out; the kernel
releases its tensor memory and returns, tcbf_last_device_error reports
TCBF_ERR_TIMEOUT, and the same plan then computes correct results."""
import time

import numpy as np
import pytest

import oracle
import tcbf_inputs as ti

pytestmark = pytest.mark.gpu

TCBF_ERR_TIMEOUT = 6


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import ensure_lib
    return ensure_lib()


# 4 x 512 x 1280 outputs in 128 x 128 tiles = 160 tiles, so the first CTA of the
# 152-CTA grid holds two: fill 0 is the first tile's first stage, fill 5 lies in its
# second tile (FP16: 4 stages of 64 K per tile; plain FP8: 2 stages of 128 K)
@pytest.mark.parametrize("mode,fill", [("fp16", 0), ("fp16", 5), ("fp8", 3)])
def test_dropped_load_times_out_and_plan_recovers(mode, fill):
    import torch
    from gpu_util import dev, empty_bytes
    from paper_2505_03269_gb300 import FLAG_FP8_HI_ONLY, MODE_FP16, MODE_FP8SPLIT, Plan
    B, M, K, N = 4, 512, 256, 1280
    W, X = ti.small_fp16(seed=77, M=M, K=K, N=N, B=B)
    fp8 = mode == "fp8"
    with Plan(B, M, N, K, MODE_FP8SPLIT if fp8 else MODE_FP16,
              flags=FLAG_FP8_HI_ONLY if fp8 else 0) as plan:
        plan.set_config(0)
        Wp = empty_bytes(plan.packed_size(0))
        Xp = empty_bytes(plan.packed_size(1))
        plan.transpose_pack(0, dev(W), Wp)
        plan.transpose_pack(1, dev(X), Xp)
        Y = torch.zeros((B, M, N, 2), dtype=torch.float32, device="cuda")
        run = plan.beamform_fp8split if fp8 else plan.beamform_fp16
        torch.cuda.synchronize()
        plan.debug_drop_fill(fill)
        t0 = time.monotonic()
        run(Wp, Xp, Y)
        torch.cuda.synchronize()
        dt = time.monotonic() - t0
        assert plan.last_device_error() == TCBF_ERR_TIMEOUT
        assert 1.5 < dt < 30.0
        # the hook applied to that call only: the same plan is correct again
        Y.fill_(float("nan"))
        run(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        Yh = Y.cpu().numpy().astype(np.float64)
    got = Yh[..., 0] + 1j * Yh[..., 1]
    ref = oracle.cgemm_split(W, X, products=1) if fp8 else oracle.cgemm(W, X)
    assert oracle.rel_frobenius(got, ref) <= 2e-5


def test_drop_fill_rejected_where_unsupported():
    from paper_2505_03269_gb300 import (FLAG_STACKED_X, MODE_1BIT, MODE_FP16, Plan,
                                        TcbfError)
    with Plan(1, 256, 256, 64, MODE_FP16) as plan:
        plan.set_config(6)                      # cluster configuration
        with pytest.raises(TcbfError):
            plan.debug_drop_fill(0)
        plan.debug_drop_fill(-1)                # clearing is always accepted
    with Plan(1, 256, 256, 64, MODE_FP16, flags=FLAG_STACKED_X) as plan:
        with pytest.raises(TcbfError):
            plan.debug_drop_fill(0)
    with Plan(1, 256, 256, 64, MODE_1BIT) as plan:
        with pytest.raises(TcbfError):
            plan.debug_drop_fill(0)
