"""TF32 mode on the GPU: FP32 data rounded once to TF32 (10 mantissa bits,
FP32's exponent range) and multiplied with kind::tf32 MMAs.

Bars: the packed planes equal the oracle's TF32 rounding bit for bit (FP32
sources, ties and subnormals included; FP16 sources convert exactly); the
product is within the 16-bit mode's 2e-5 of the FP64 oracle on the rounded
inputs, for ragged shapes, every tile configuration and promoted long K;
integer inputs are exact; values far outside FP16's range keep that bar."""
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


def _run(W, X, config=None, src_type=1):
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_TF32, Plan
    Bw, M, K, _ = W.shape
    B, _, N, _ = X.shape
    with Plan(B, M, N, K, MODE_TF32, w_batches=Bw) as plan:
        if config is not None:
            plan.set_config(config)
        Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
        Y = torch.full((B, M, N, 2), float("nan"), dtype=torch.float32, device="cuda")
        plan.transpose_pack(0, dev(W), Wp, src_type)
        plan.transpose_pack(1, dev(X), Xp, src_type)
        plan.beamform_tf32(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        Yh = Y.cpu().numpy().astype(np.float64)
        return Yh[..., 0] + 1j * Yh[..., 1], Wp.cpu().numpy(), Xp.cpu().numpy(), plan.Kp


def _f32(seed, shape, scale=1.0):
    g = ti.rng(seed)
    return (g.standard_normal(shape) * scale).astype(np.float32)


def _ref(W, X):
    return oracle.cgemm(oracle.round_tf32(W), oracle.round_tf32(X))


@pytest.mark.parametrize("B,M,N,K", [(1, 3, 5, 7), (2, 70, 130, 100), (1, 40, 66, 33)])
def test_tf32_pack_matches_oracle_rounding(B, M, N, K):
    W = _f32(M, (B, M, K, 2))
    X = _f32(N, (B, K, N, 2))
    # ties, values just off a tie, a subnormal and values beyond FP16's range
    X.reshape(-1)[:6] = np.array([1 + 2 ** -11, 1 + 3 * 2 ** -11, 1 + 2 ** -11 + 2 ** -23,
                                  3e-39, 1e30, -7e-20], np.float32)
    _, Wraw, Xraw, Kp = _run(W, X)
    Wp = Wraw.view(np.float32).reshape(B, 2, M, Kp).astype(np.float64)
    Xp = Xraw.view(np.float32).reshape(B, 2, N, Kp).astype(np.float64)
    rW, rX = oracle.round_tf32(W), oracle.round_tf32(X)
    for p in range(2):
        assert np.array_equal(Wp[:, p, :, :K], rW[..., p])
        assert np.array_equal(Xp[:, p, :, :K], rX[..., p].transpose(0, 2, 1))
    assert not Wp[..., K:].any() and not Xp[..., K:].any()


def test_tf32_fp16_source_converts_exactly():
    W, X = ti.small_fp16(seed=3, M=50, K=60, N=70, B=2)
    Y, Wraw, _, Kp = _run(W, X, src_type=0)
    Wp = Wraw.view(np.float32).reshape(2, 2, 50, Kp)[..., :60]
    assert np.array_equal(Wp.transpose(0, 2, 3, 1), W.astype(np.float32))
    assert oracle.rel_frobenius(Y, oracle.cgemm(W, X)) <= TOL


@pytest.mark.parametrize("config", [0, 1, 3, 6, 8])
@pytest.mark.parametrize("B,Bw,M,N,K", [(1, 1, 5, 7, 3), (4, 2, 130, 300, 200), (1, 1, 64, 1024, 128),
                                        (2, 1, 129, 257, 129)])
def test_tf32_gemm_matches_oracle(config, B, Bw, M, N, K):
    W = _f32(B * M + K, (Bw, M, K, 2))
    X = _f32(N + K, (B, K, N, 2))
    Y, _, _, _ = _run(W, X, config)
    assert oracle.rel_frobenius(Y, _ref(W, X)) <= TOL


@pytest.mark.parametrize("config", [0, 8])
def test_tf32_long_k_promoted(config):
    W = _f32(40, (1, 256, 5000, 2))
    X = _f32(41, (1, 5000, 128, 2))
    Y, _, _, _ = _run(W, X, config)
    assert oracle.rel_frobenius(Y, _ref(W, X)) <= TOL


def test_tf32_integer_inputs_exact():
    g = ti.rng(6)
    W = g.integers(-8, 9, (1, 100, 200, 2)).astype(np.float32)
    X = g.integers(-8, 9, (2, 200, 96, 2)).astype(np.float32)
    Y, _, _, _ = _run(W, X)
    assert np.array_equal(Y, oracle.cgemm(W.astype(np.float64), X.astype(np.float64)))


def test_tf32_keeps_fp32_range():
    """Weights near 1e-6 and samples near 1e6 (outside FP16's normal range):
    TF32 keeps them, within the same bar."""
    W = _f32(7, (1, 64, 96, 2), scale=1e-6)
    X = _f32(8, (1, 96, 80, 2), scale=1e6)
    Y, _, _, _ = _run(W, X)
    assert oracle.rel_frobenius(Y, _ref(W, X)) <= TOL
    assert np.abs(Y).max() > 1.0


def test_tf32_weights_from_geometry():
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_TF32, Plan
    geom = ti.ultrasound_geometry(n_elements=32, n_bins=16, grid=(8, 8, 4))
    M, K = geom.targets.shape[0], geom.rx_pos.shape[0]
    with Plan(1, M, 8, K, MODE_TF32) as plan:
        Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        plan.weights_from_geometry(dev(geom.rx_pos), dev(geom.targets), True,
                                   dev(np.ascontiguousarray(geom.freqs)), geom.c, Wp)
        torch.cuda.synchronize()
        got = Wp.cpu().numpy().view(np.float32).reshape(1, 2, M, plan.Kp)[..., :K]
    w = oracle.weights(geom.rx_pos, geom.targets, geom.freqs, True, geom.c)
    for p, part in enumerate((w.real, w.imag)):
        ref = oracle.round_tf32(part.astype(np.float32))
        g32 = got[:, p].astype(np.float64)
        ulp = np.ldexp(1.0, np.frexp(np.maximum(np.abs(ref), 1e-30))[1] - 11)
        assert np.all(np.abs(g32 - ref) <= ulp)
        assert np.mean(g32 == ref) >= 0.999
