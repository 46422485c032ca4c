"""FP16 beamforming on the GPU against the FP64 CPU oracle.

Tolerance: relative Frobenius error <= 2e-5 over re and im jointly (the
target stated for the 16-bit mode); integer-valued and identity inputs,
whose FP32 partial sums are all exact, must match bit for bit."""
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


def _run(*a, **k):
    from gpu_util import run_fp16
    return run_fp16(*a, **k)


def test_small_fp16_workload():
    """64 beams x 128 receivers x 1024 samples, batch 1, seed 0."""
    W, X = ti.small_fp16(seed=0)
    Y = _run(W, X)
    Yref = oracle.cgemm(W, X)
    assert oracle.rel_frobenius(Y, Yref) <= TOL


@pytest.mark.parametrize("config", [0, 1, 2, 6, 7, 8])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (3, 5, 7), (17, 33, 127), (129, 130, 288),
                                   (127, 257, 129), (200, 96, 64), (64, 1024, 200)])
def test_ragged_shapes(config, M, N, K):
    W, X = ti.small_fp16(seed=M * 7 + N + K, M=M, K=K, N=N, B=2)
    Y = _run(W, X, config=config)
    Yref = oracle.cgemm(W, X)
    assert oracle.rel_frobenius(Y, Yref) <= TOL


@pytest.mark.parametrize("config", [0, 1, 2, 6, 7, 8])
def test_integer_inputs_bit_exact(config):
    g = ti.rng(1)
    W = ti.integer_complex_fp16(g, (2, 150, 300))
    X = ti.integer_complex_fp16(g, (4, 300, 270))
    Y = _run(W, X, config=config)
    Yref = oracle.cgemm(W, X)
    assert np.array_equal(Y, Yref)


def test_identity_weights_bit_exact():
    K, N = 160, 300
    W = np.zeros((1, K, K, 2), np.float16)
    W[0, np.arange(K), np.arange(K), 0] = 1.0
    _, X = ti.small_fp16(seed=2, M=1, K=K, N=N)
    Y = _run(W, X)
    Xc = X[..., 0].astype(np.float64) + 1j * X[..., 1].astype(np.float64)
    assert np.array_equal(Y, Xc)


def test_imaginary_identity_weights():
    """W = i I maps X to i X: checks the negated term of the real part."""
    K, N = 96, 64
    W = np.zeros((1, K, K, 2), np.float16)
    W[0, np.arange(K), np.arange(K), 1] = 1.0
    _, X = ti.small_fp16(seed=5, M=1, K=K, N=N)
    Y = _run(W, X)
    Xc = X[..., 0].astype(np.float64) + 1j * X[..., 1].astype(np.float64)
    assert np.array_equal(Y, 1j * Xc)


def test_shared_weights_across_batches():
    g = ti.rng(6)
    W, _ = ti.small_fp16(seed=6, M=100, K=72, N=8, B=3)
    X = ti.complex_gaussian_fp16(g, (6, 72, 150))
    Y = _run(W, X)
    Yref = oracle.cgemm(W, X)
    assert oracle.rel_frobenius(Y, Yref) <= TOL


def test_fp32_source_rounds_to_nearest():
    g = ti.rng(8)
    W32 = g.standard_normal((1, 40, 56, 2)).astype(np.float32)
    X32 = g.standard_normal((2, 56, 48, 2)).astype(np.float32)
    from paper_2505_03269_gb300 import SRC_CF32
    Y = _run(W32, X32, src_type=SRC_CF32)
    Yref = oracle.cgemm(W32.astype(np.float16), X32.astype(np.float16))
    assert oracle.rel_frobenius(Y, Yref) <= TOL


@pytest.mark.parametrize("config", [0, 2, 7, 8])
@pytest.mark.parametrize("K", [4100, 8192, 16384])
def test_long_k_within_tolerance(config, K):
    """Above K = 4096 the partial sums are promoted to FP32 every 2048 K;
    the error must stay within the FP16 tolerance at any K."""
    W, _ = ti.small_fp16(seed=K, M=256, K=K, N=8)
    X = ti.complex_gaussian_fp16(ti.rng(K + 1), (1, K, 192))
    Y = _run(W, X, config=config)
    Yref = oracle.cgemm(W, X)
    assert oracle.rel_frobenius(Y, Yref) <= TOL


def test_long_k_integer_inputs_bit_exact():
    """Integer partial sums stay exact through the promotion."""
    g = ti.rng(12)
    W = ti.integer_complex_fp16(g, (1, 130, 9000), lo=-2, hi=2)
    X = ti.integer_complex_fp16(g, (1, 9000, 70), lo=-2, hi=2)
    Y = _run(W, X)
    assert np.array_equal(Y, oracle.cgemm(W, X))


def test_wide_tile_rejected_for_long_k():
    from paper_2505_03269_gb300 import MODE_FP16, Plan, TcbfError
    with Plan(1, 128, 128, 8192, MODE_FP16) as plan:
        with pytest.raises(TcbfError):
            plan.set_config(1)
