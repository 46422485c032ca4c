"""tcbf_beamform_host: the step for host-resident X and Y, chunked over the
batches (a single batch: over ranges of W rows) with the copies overlapped
with the kernels.

Bars: bit-exact against the device-buffer path of the same plan (the same
kernels on the same batches; only the data movement differs) for every
mode, including a ragged last chunk, weight sharing across batches inside
and across chunks (split-FP8's per-row W exponents of a sub-range), both
source types, repeated calls and a staging that grows; FP16 also within
the 2e-5 parity bar of the FP64 oracle."""
import numpy as np
import pytest

import oracle
import tcbf_inputs as ti

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import ensure_lib
    return ensure_lib()


def _pinned(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def _device_path(plan, mode, Wd, Xd, src_type, B, M, N):
    """Wp (packed, on the device) and Y of the device-buffer calls."""
    import torch
    from gpu_util import empty_bytes
    from paper_2505_03269_gb300 import MODE_1BIT, MODE_FP16
    Wp = empty_bytes(plan.packed_size(0))
    Xp = empty_bytes(plan.packed_size(1))
    plan.transpose_pack(0, Wd, Wp, src_type)
    plan.transpose_pack(1, Xd, Xp, src_type)
    dt = torch.int32 if mode == MODE_1BIT else torch.float32
    Y = torch.empty((B, M, N, 2), dtype=dt, device="cuda")
    if mode == MODE_FP16:
        plan.beamform_fp16(Wp, Xp, Y)
    elif mode == 3:
        plan.beamform_tf32(Wp, Xp, Y)
    elif mode == MODE_1BIT:
        plan.beamform_1bit(Wp, Xp, Y)
    else:
        plan.beamform_fp8split(Wp, Xp, Y)
    torch.cuda.synchronize()
    assert plan.last_device_error() == 0
    return Wp, Y.cpu()


def _host_path(plan, Wp, X_host, Y_like, chunk, src_type, calls=1):
    import torch
    Yh = torch.full(Y_like.shape, -3, dtype=Y_like.dtype).pin_memory()
    s = torch.cuda.Stream()
    for _ in range(calls):
        plan.beamform_host(X_host, Wp, Yh, chunk=chunk, src_type=src_type, stream=s)
    s.synchronize()
    assert plan.last_device_error() == 0
    return Yh


def _inputs(seed, Bw, B, M, N, K, src_type):
    W, X = ti.small_fp16(seed=seed, M=M, K=K, N=N, B=B)
    W = np.ascontiguousarray(W[:Bw])
    if src_type == 1:
        W, X = W.astype(np.float32), X.astype(np.float32)
    return W, X


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("B,Bw,M,N,K,chunk", [(6, 3, 130, 300, 200, 4), (4, 2, 64, 256, 96, 2),
                                              (5, 5, 200, 136, 72, 0), (3, 1, 96, 64, 40, 3)])
def test_host_path_equals_device_path(mode, B, Bw, M, N, K, chunk):
    from gpu_util import dev
    from paper_2505_03269_gb300 import Plan
    src_type = 0
    W, X = _inputs(M + N + K, Bw, B, M, N, K, src_type)
    with Plan(B, M, N, K, mode, w_batches=Bw) as plan:
        Wp, Yref = _device_path(plan, mode, dev(W), dev(X), src_type, B, M, N)
        Yh = _host_path(plan, Wp, _pinned(X), Yref, chunk, src_type)
    assert np.array_equal(Yh.numpy(), Yref.numpy())


@pytest.mark.parametrize("src_type", [0, 1])
def test_fp16_host_path_against_oracle(src_type):
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_FP16, Plan
    B, Bw, M, N, K = 6, 2, 160, 384, 160
    W, X = _inputs(11, Bw, B, M, N, K, src_type)
    with Plan(B, M, N, K, MODE_FP16, w_batches=Bw) as plan:
        Wp, Yref = _device_path(plan, MODE_FP16, dev(W), dev(X), src_type, B, M, N)
        Yh = _host_path(plan, Wp, _pinned(X), Yref, 3 if Bw == 2 else 0, src_type).numpy()
    Y = Yh[..., 0].astype(np.float64) + 1j * Yh[..., 1]
    W16 = W.astype(np.float16) if src_type == 1 else W
    X16 = X.astype(np.float16) if src_type == 1 else X
    assert oracle.rel_frobenius(Y, oracle.cgemm(W16, X16)) <= TOL


def test_repeated_calls_and_growing_staging():
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_FP16, Plan
    B, Bw, M, N, K = 8, 4, 128, 256, 64
    W, X = _inputs(3, Bw, B, M, N, K, 0)
    with Plan(B, M, N, K, MODE_FP16, w_batches=Bw) as plan:
        Wp, Yref = _device_path(plan, MODE_FP16, dev(W), dev(X), 0, B, M, N)
        for chunk, calls in [(2, 3), (6, 2), (4, 1), (8, 1)]:
            Yh = _host_path(plan, Wp, _pinned(X), Yref, chunk, 0, calls=calls)
            assert np.array_equal(Yh.numpy(), Yref.numpy()), chunk


def test_invalid_arguments():
    import torch
    from paper_2505_03269_gb300 import MODE_FP16, Plan, TcbfError
    with Plan(4, 64, 64, 32, MODE_FP16, w_batches=2) as plan:
        Wp = torch.zeros(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        Xh = torch.zeros((4, 32, 64, 2), dtype=torch.float16).pin_memory()
        Yh = torch.zeros((4, 64, 64, 2), dtype=torch.float32).pin_memory()
        with pytest.raises(TcbfError, match="INVALID_ARG"):
            plan.beamform_host(Xh, Wp, Yh, chunk=1)          # not a multiple of batch / w_batches
        with pytest.raises(TcbfError, match="INVALID_ARG"):
            plan.beamform_host(Xh, Wp, Yh, chunk=2, src_type=7)
        plan.set_batch_rows([64, 10, 64, 1])
        with pytest.raises(TcbfError, match="UNSUPPORTED"):
            plan.beamform_host(Xh, Wp, Yh, chunk=2)


# One batch: X in and packed once, then ranges of W rows, each copied out while the
# next computes.  M = 20000 with N = 300 gives ranges of 6400 rows (whole waves of
# 128-row tiles on 152 SMs) and a ragged last range of 800; M = 100 is one range.
@pytest.mark.parametrize("mode,flags", [(0, 0), (0, 1), (1, 0), (1, 2), (2, 0)])
@pytest.mark.parametrize("M", [20000, 100])
def test_single_batch_row_ranges_equal_device_path(mode, flags, M):
    from gpu_util import dev
    from paper_2505_03269_gb300 import Plan
    N, K = 300, 64
    W, X = _inputs(M + flags, 1, 1, M, N, K, 0)
    with Plan(1, M, N, K, mode, flags=flags) as plan:
        Wp, Yref = _device_path(plan, mode, dev(W), dev(X), 0, 1, M, N)
        Yh = _host_path(plan, Wp, _pinned(X), Yref, 0, 0, calls=2)
    assert np.array_equal(Yh.numpy(), Yref.numpy())


# The 4-bit tensor path of the 1-bit mode expands W and X into plan-owned
# scratch; the batch chunks and the row ranges of one batch (sub-plans that
# share it, one after another on one stream) equal the device path.
@pytest.mark.parametrize("config", [5, 6, 7])
@pytest.mark.parametrize("B,Bw,M,N,K,chunk", [(6, 3, 130, 300, 200, 2), (1, 1, 20000, 300, 64, 0)])
def test_1bit_fp4_host_path_equals_device_path(config, B, Bw, M, N, K, chunk):
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_1BIT, Plan
    W, X = _inputs(M + config, Bw, B, M, N, K, 0)
    with Plan(B, M, N, K, MODE_1BIT, w_batches=Bw) as plan:
        plan.set_config(config)
        Wp, Yref = _device_path(plan, MODE_1BIT, dev(W), dev(X), 0, B, M, N)
        Yh = _host_path(plan, Wp, _pinned(X), Yref, chunk, 0, calls=2)
    assert np.array_equal(Yh.numpy(), Yref.numpy())


def test_single_batch_fp32_source_against_oracle():
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_FP16, Plan
    M, N, K = 13000, 256, 96
    W, X = _inputs(5, 1, 1, M, N, K, 1)
    with Plan(1, M, N, K, MODE_FP16) as plan:
        Wp, Yref = _device_path(plan, MODE_FP16, dev(W), dev(X), 1, 1, M, N)
        Yh = _host_path(plan, Wp, _pinned(X), Yref, 0, 1).numpy()
    assert np.array_equal(Yh, Yref.numpy())
    rows = np.arange(0, M, 37)
    Y = Yh[0, rows, :, 0].astype(np.float64) + 1j * Yh[0, rows, :, 1]
    ref = oracle.cgemm(np.ascontiguousarray(W[:, rows].astype(np.float16)), X.astype(np.float16))[0]
    assert oracle.rel_frobenius(Y, ref) <= TOL
