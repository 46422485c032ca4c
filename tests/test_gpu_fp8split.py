"""Split-FP8 mode on the GPU (and its plain E4M3 form, TCBF_FLAG_FP8_HI_ONLY,
which packs one byte per element).

Two references: the oracle's own split arithmetic (E4M3 hi+lo with per-row
power-of-two scales, Y = 2^-(eW+eX)(Wh Xh + Wh Xl + Wl Xh) in FP64), which
the GPU must match within the FP32-accumulation tolerance of the 16-bit
mode (2e-5), and the plain FP64 product of the FP16 inputs, whose distance
is the method's accuracy (stated, not a parity bar: ~1e-3)."""
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


def _plan(B, M, N, K, Bw=0, flags=0):
    from paper_2505_03269_gb300 import MODE_FP8SPLIT, Plan
    return Plan(B, M, N, K, MODE_FP8SPLIT, w_batches=Bw, flags=flags)


def _decode_split(raw, nb, rows, K, hi_only=False):
    """Packed split bytes -> (hi, lo) [nb, 2, rows, K] doubles and exps [nb, rows]
    (hi-only rows: lo is None)."""
    import torch
    parts = 1 if hi_only else 2
    Kb2 = parts * ((K + 63) // 64 * 64)
    assert raw.size == nb * 2 * rows * Kb2 + 4 * nb * rows
    data = raw[: nb * 2 * rows * Kb2].reshape(nb, 2, rows, Kb2 // (64 * parts), parts, 64)
    vals = torch.from_numpy(np.ascontiguousarray(data)).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    hi = vals[..., 0, :].reshape(nb, 2, rows, -1)[..., :K]
    lo = None if hi_only else vals[..., 1, :].reshape(nb, 2, rows, -1)[..., :K]
    ex = raw[nb * 2 * rows * Kb2:].view(np.int32).reshape(nb, rows)
    return hi, lo, ex


def _run(W, X, config=None, src_type=0, flags=0):
    import torch
    from gpu_util import dev
    Bw, M, K, _ = W.shape
    B, _, N, _ = X.shape
    with _plan(B, M, N, K, Bw, flags) as plan:
        if config is not None:
            plan.set_config(config)
        Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
        Y = torch.empty((B, M, N, 2), dtype=torch.float32, device="cuda")
        plan.transpose_pack(0, dev(W), Wp, src_type)
        plan.transpose_pack(1, dev(X), Xp, src_type)
        plan.beamform_fp8split(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        Yh = Y.cpu().numpy().astype(np.float64)
        return Yh[..., 0] + 1j * Yh[..., 1], Wp.cpu().numpy(), Xp.cpu().numpy()


# K <= 320 packs X in one on-chip pass, longer K in two; N % 4 picks 16-byte loads
@pytest.mark.parametrize("B,M,N,K,src", [(1, 3, 5, 7, 0), (2, 70, 130, 100, 0), (2, 128, 256, 288, 0),
                                         (2, 40, 96, 320, 0), (1, 64, 68, 400, 0),
                                         (2, 33, 72, 150, 1), (1, 20, 66, 77, 1)])
def test_split_pack_matches_oracle_exactly(B, M, N, K, src):
    W, X = ti.small_fp16(seed=M + K, M=M, K=K, N=N, B=B)
    X[0, 0, :3, 0] = np.array([0.0, -0.0, 6e-8], np.float16)
    if src == 1:            # FP32 sources holding FP16 values: the same packed bytes
        _, Wraw, Xraw = _run(W.astype(np.float32), X.astype(np.float32), src_type=1)
    else:
        _, Wraw, Xraw = _run(W, X)
    (Wh, Wl, eW), (Xh, Xl, eX) = oracle.split_operands(W, X)
    hi, lo, ex = _decode_split(Wraw, B, M, K)
    assert np.array_equal(ex, eW)
    assert np.array_equal(hi, Wh.transpose(0, 3, 1, 2)) and np.array_equal(lo, Wl.transpose(0, 3, 1, 2))
    hi, lo, ex = _decode_split(Xraw, B, N, K)
    assert np.array_equal(ex, eX)
    assert np.array_equal(hi, Xh.transpose(0, 3, 2, 1)) and np.array_equal(lo, Xl.transpose(0, 3, 2, 1))


@pytest.mark.parametrize("config", [0, 1, 3])
@pytest.mark.parametrize("B,Bw,M,N,K", [(1, 1, 64, 1024, 128), (4, 2, 130, 300, 200),
                                        (1, 1, 5, 7, 3)])
def test_split_gemm_matches_split_oracle(config, B, Bw, M, N, K):
    W, _ = ti.small_fp16(seed=B * M + K, M=M, K=K, N=8, B=Bw)
    X = ti.complex_gaussian_fp16(ti.rng(N + K), (B, K, N))
    Y, _, _ = _run(W, X, config)
    assert oracle.rel_frobenius(Y, oracle.cgemm_split(W, X)) <= TOL
    err = oracle.rel_frobenius(Y, oracle.cgemm(W, X))
    assert err < 5e-3          # the method's own accuracy (about 1e-3)


def test_split_long_k_promoted():
    W, _ = ti.small_fp16(seed=40, M=256, K=5000, N=8)
    X = ti.complex_gaussian_fp16(ti.rng(41), (1, 5000, 128))
    Y, _, _ = _run(W, X)
    assert oracle.rel_frobenius(Y, oracle.cgemm_split(W, X)) <= TOL


def test_split_weights_from_geometry():
    """Split weights straight from geometry against the oracle's FP16 weights
    split by the oracle (entries whose FP16 weight differs by an ulp may differ)."""
    import torch
    from gpu_util import dev
    geom = ti.ultrasound_geometry(n_elements=32, n_bins=16, grid=(8, 8, 4))
    M, K = geom.targets.shape[0], geom.rx_pos.shape[0]
    with _plan(1, M, 8, K) as plan:
        Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        plan.weights_from_geometry(dev(geom.rx_pos), dev(geom.targets), True,
                                   dev(np.ascontiguousarray(geom.freqs)), geom.c, Wp)
        torch.cuda.synchronize()
        raw = Wp.cpu().numpy()
    hi, lo, ex = _decode_split(raw, 1, M, K)
    W16 = oracle.weights_fp16(geom.rx_pos, geom.targets, geom.freqs, True, geom.c)
    Wh, Wl, eW = oracle.split_rows(W16.reshape(M, K, 2))
    assert np.mean(ex[0] == eW) >= 0.99
    same = (hi[0].transpose(1, 2, 0) == Wh) & (lo[0].transpose(1, 2, 0) == Wl)
    assert np.mean(same) >= 0.999


# products per complex K step: 1 = plain E4M3 (TCBF_FLAG_FP8_HI_ONLY), 3 = hi+lo split,
# 4 = split with Wl Xl (TCBF_FLAG_FP8_FOUR_PRODUCTS)
@pytest.mark.parametrize("products,flags,ceiling", [(1, 2, 1e-1), (3, 0, 5e-3), (4, 4, 5e-3)])
@pytest.mark.parametrize("config", [0, 8])
def test_split_product_count_matches_oracle(products, flags, ceiling, config):
    W, _ = ti.small_fp16(seed=50 + products, M=130, K=300, N=8, B=2)
    X = ti.complex_gaussian_fp16(ti.rng(51), (4, 300, 260))
    Y, _, _ = _run(W, X, config, flags=flags)
    assert oracle.rel_frobenius(Y, oracle.cgemm_split(W, X, products=products)) <= TOL
    assert oracle.rel_frobenius(Y, oracle.cgemm(W, X)) < ceiling


def test_plain_fp8_exact_on_four_bit_integers():
    g = ti.rng(52)
    W = ti.integer_complex_fp16(g, (1, 100, 200))
    X = ti.integer_complex_fp16(g, (2, 200, 96))
    Y, _, _ = _run(W, X, flags=2)
    assert np.array_equal(Y, oracle.cgemm(W, X))


# The plain E4M3 form packs the hi bytes alone: K <= 320 in one pass, longer K tiled,
# FP32 sources, ragged K around the 64-element blocks
@pytest.mark.parametrize("B,M,N,K,src", [(1, 3, 5, 7, 0), (2, 70, 130, 100, 0), (2, 128, 256, 288, 0),
                                         (1, 64, 68, 400, 0), (2, 33, 72, 150, 1), (1, 20, 66, 129, 1)])
def test_hi_only_pack_matches_oracle_exactly(B, M, N, K, src):
    W, X = ti.small_fp16(seed=M + K + 1, M=M, K=K, N=N, B=B)
    if src == 1:
        _, Wraw, Xraw = _run(W.astype(np.float32), X.astype(np.float32), src_type=1, flags=2)
    else:
        _, Wraw, Xraw = _run(W, X, flags=2)
    (Wh, _, eW), (Xh, _, eX) = oracle.split_operands(W, X)
    hi, lo, ex = _decode_split(Wraw, B, M, K, hi_only=True)
    assert np.array_equal(ex, eW) and np.array_equal(hi, Wh.transpose(0, 3, 1, 2))
    hi, lo, ex = _decode_split(Xraw, B, N, K, hi_only=True)
    assert np.array_equal(ex, eX) and np.array_equal(hi, Xh.transpose(0, 3, 2, 1))
    # the pad bytes of every row are zero
    Kb = (K + 63) // 64 * 64
    rows = Wraw[: B * 2 * M * Kb].reshape(-1, Kb)
    assert not rows[:, K:].any()


_HI_SHAPES = [(1, 1, 5, 7, 3), (4, 2, 130, 300, 200), (1, 1, 64, 1024, 128), (2, 1, 129, 257, 129)]


# configuration 1 (128 x 256 tiles) has no TMEM room for promoted sums, so K > 4096
# runs on the others
@pytest.mark.parametrize("config,B,Bw,M,N,K",
                         [(c,) + s for c in (0, 1, 3, 6, 8) for s in _HI_SHAPES]
                         + [(c, 1, 1, 256, 128, 5000) for c in (0, 3, 6, 8)])
def test_hi_only_gemm_matches_oracle(config, B, Bw, M, N, K):
    """Stages of 128 K per 128-byte row: K = 3, 128, 129 and 200 end mid-stage or on
    its edge; K = 5000 crosses the 2048-K promotion chunks."""
    W, _ = ti.small_fp16(seed=B * M + K + 2, M=M, K=K, N=8, B=Bw)
    X = ti.complex_gaussian_fp16(ti.rng(N + K + 2), (B, K, N))
    Y, _, _ = _run(W, X, config, flags=2)
    assert oracle.rel_frobenius(Y, oracle.cgemm_split(W, X, products=1)) <= TOL


def test_hi_only_weights_from_geometry():
    import torch
    from gpu_util import dev
    geom = ti.ultrasound_geometry(n_elements=32, n_bins=16, grid=(8, 8, 4))
    M, K = geom.targets.shape[0], geom.rx_pos.shape[0]
    with _plan(1, M, 8, K, flags=2) as plan:
        Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        plan.weights_from_geometry(dev(geom.rx_pos), dev(geom.targets), True,
                                   dev(np.ascontiguousarray(geom.freqs)), geom.c, Wp)
        torch.cuda.synchronize()
        raw = Wp.cpu().numpy()
    hi, _, ex = _decode_split(raw, 1, M, K, hi_only=True)
    W16 = oracle.weights_fp16(geom.rx_pos, geom.targets, geom.freqs, True, geom.c)
    Wh, _, eW = oracle.split_rows(W16.reshape(M, K, 2))
    assert np.mean(ex[0] == eW) >= 0.99
    assert np.mean(hi[0].transpose(1, 2, 0) == Wh) >= 0.999
