"""Block-scaled FP8 on the GPU (TCBF_FLAG_FP8_BLOCK_SCALES): a UE8M0 scale
per 32 k of each W row and X sample, applied by the tensor cores' block-scaled
E4M3 MMAs.

References: the oracle's block-scaled split (oracle.split_blocks for the
packed bytes and codes, bit for bit; oracle.cgemm_split_blocks for the
product, within the 16-bit mode's FP32-accumulation tolerance 2e-5), and the
FP64 product of the FP16 inputs for the method's own accuracy (stated, with
a loose ceiling).  Integer-valued inputs are exact in E4M3 after block
scaling, so their products must be bit exact."""
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


def _flags(products):
    import paper_2505_03269_gb300 as tcbf
    f = tcbf.FLAG_FP8_BLOCK_SCALES
    if products == 1:
        f |= tcbf.FLAG_FP8_HI_ONLY
    if products == 4:
        f |= tcbf.FLAG_FP8_FOUR_PRODUCTS
    return f


def _run(W, X, products=3, config=None, src_type=0):
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_FP8SPLIT, Plan
    Bw, M, K, _ = W.shape
    B, _, N, _ = X.shape
    with Plan(B, M, N, K, MODE_FP8SPLIT, w_batches=Bw, flags=_flags(products)) as plan:
        if config is not None:
            plan.set_config(config)
        Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
        Y = torch.full((B, M, N, 2), float("nan"), dtype=torch.float32, device="cuda")
        plan.transpose_pack(0, dev(W), Wp, src_type)
        plan.transpose_pack(1, dev(X), Xp, src_type)
        plan.beamform_fp8split(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        Yh = Y.cpu().numpy().astype(np.float64)
        return Yh[..., 0] + 1j * Yh[..., 1], Wp.cpu().numpy(), Xp.cpu().numpy()


def _decode(raw, nb, rows, K, per_tile, hi_only):
    """Packed block-scaled bytes -> hi, lo [nb, 2, rows, K] doubles (lo None
    for hi-only rows) and the scale codes [nb, rows, 2 * stages] in stage
    order (hi codes of the stage's blocks, then lo codes)."""
    import torch
    parts = 1 if hi_only else 2
    Kb2 = parts * ((K + 63) // 64 * 64)
    data_n = nb * 2 * rows * Kb2
    data = raw[:data_n].reshape(nb, 2, rows, Kb2 // (64 * parts), parts, 64)
    vals = torch.from_numpy(np.ascontiguousarray(data)).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    hi = vals[..., 0, :].reshape(nb, 2, rows, -1)[..., :K]
    lo = None if hi_only else vals[..., 1, :].reshape(nb, 2, rows, -1)[..., :K]
    sk = 128 if hi_only else 64
    stages = (K + sk - 1) // sk
    tiles = (rows + per_tile - 1) // per_tile
    sf = raw[data_n:].reshape(nb, tiles, stages, 32, 4, 4)
    assert raw.size == data_n + nb * tiles * stages * 512
    codes = np.empty((nb, rows, stages, 4), np.int64)
    for r in range(rows):
        t, rr = divmod(r, per_tile)
        codes[:, r] = sf[:, t, :, rr % 32, rr // 32, :]
    return hi, lo, codes


@pytest.mark.parametrize("products", [3, 1])
@pytest.mark.parametrize("B,M,N,K,src", [(1, 3, 5, 7, 0), (2, 70, 130, 100, 0), (1, 130, 70, 300, 0),
                                         (2, 33, 72, 150, 1)])
def test_block_pack_matches_oracle_exactly(products, B, M, N, K, src):
    """Bytes and scale codes of W (rows) and X (samples) equal the oracle's
    block split: hi codes 127 - e, lo codes 123 - e (lo 16 times larger)."""
    g = ti.rng(M + K)
    W = (ti.complex_gaussian_fp16(g, (B, M, K)).astype(np.float64) *
         np.exp2(g.integers(-9, 9, (B, M, K, 1)))).astype(np.float16)
    X = ti.complex_gaussian_fp16(g, (B, K, N))
    X[0, 0, :3, 0] = np.array([0.0, -0.0, 6e-8], np.float16)
    args = (W.astype(np.float32), X.astype(np.float32)) if src else (W, X)
    _, Wraw, Xraw = _run(*args, products=products, src_type=src)
    hi_only = products == 1
    for raw, V, nb, rows, per in ((Wraw, W.reshape(B * M, K, 2), B, M, 128),
                                  (Xraw, np.ascontiguousarray(X.transpose(0, 2, 1, 3)).reshape(B * N, K, 2),
                                   B, N, 64)):
        h, l, codes = _decode(raw, nb, rows, K, per, hi_only)
        oh, ol, oe = oracle.split_blocks(V)
        oh = oh.reshape(nb, rows, K, 2).transpose(0, 3, 1, 2)
        ol = ol.reshape(nb, rows, K, 2).transpose(0, 3, 1, 2)
        oe = oe.reshape(nb, rows, -1)
        assert np.array_equal(h, oh)
        if not hi_only:
            assert np.array_equal(l, ol)
        nblk = oe.shape[-1]
        if hi_only:
            got = codes.reshape(nb, rows, -1)[..., :nblk]
            assert np.array_equal(got, 127 - oe)
        else:
            got_hi = codes[..., :2].reshape(nb, rows, -1)[..., :nblk]
            got_lo = codes[..., 2:].reshape(nb, rows, -1)[..., :nblk]
            assert np.array_equal(got_hi, 127 - oe)
            assert np.array_equal(got_lo, 123 - oe)


@pytest.mark.parametrize("config", [0, 1])
@pytest.mark.parametrize("products", [1, 3, 4])
@pytest.mark.parametrize("B,Bw,M,N,K", [(1, 1, 64, 1024, 128), (4, 2, 130, 300, 200),
                                        (1, 1, 5, 7, 3), (2, 2, 200, 70, 333)])
def test_block_gemm_matches_oracle(config, products, B, Bw, M, N, K):
    g = ti.rng(B * M + K + products)
    W = (ti.complex_gaussian_fp16(g, (Bw, M, K)).astype(np.float64) *
         np.exp2(g.integers(-6, 6, (Bw, M, K, 1)))).astype(np.float16)
    X = ti.complex_gaussian_fp16(g, (B, K, N))
    Y, _, _ = _run(W, X, products=products, config=config)
    assert oracle.rel_frobenius(Y, oracle.cgemm_split_blocks(W, X, products)) <= TOL
    err = oracle.rel_frobenius(Y, oracle.cgemm(W, X))
    assert err < (1e-1 if products == 1 else 5e-3)


@pytest.mark.parametrize("products", [1, 3])
def test_block_integer_inputs_bit_exact(products):
    """Integers of magnitude <= 8 are E4M3 numbers after any block scaling,
    so every product is exact: the GPU must equal the FP64 product."""
    g = ti.rng(7)
    W = ti.integer_complex_fp16(g, (2, 150, 300))
    X = ti.integer_complex_fp16(g, (4, 300, 130))
    Y, _, _ = _run(W, X, products=products)
    assert np.array_equal(Y, oracle.cgemm(W, X))


def test_block_imaginary_identity():
    """W = i I (block scales of zero blocks and of ones): Y = i X exactly
    when X holds E4M3-exact values (the negated Wi Xi term of Re)."""
    K, N = 96, 64
    W = np.zeros((1, K, K, 2), np.float16)
    W[0, np.arange(K), np.arange(K), 1] = 1.0
    X = ti.integer_complex_fp16(ti.rng(8), (1, K, N))
    Y, _, _ = _run(W, X)
    Xc = X[..., 0].astype(np.float64) + 1j * X[..., 1].astype(np.float64)
    assert np.array_equal(Y, 1j * Xc)


def test_block_long_k_promoted():
    W, _ = ti.small_fp16(seed=40, M=256, K=5000, N=8)
    X = ti.complex_gaussian_fp16(ti.rng(41), (1, 5000, 128))
    for products in (1, 3):
        Y, _, _ = _run(W, X, products=products)
        assert oracle.rel_frobenius(Y, oracle.cgemm_split_blocks(W, X, products)) <= TOL


def test_block_weights_from_geometry_then_gemm():
    """Block-scaled weights straight from the near-field geometry: bytes
    and codes against the oracle's block split of its own FP16 weights
    (entries whose FP16 weight differs by an ulp may differ), then the
    GEMM of those GPU weights against the FP64 product."""
    import torch
    from gpu_util import dev
    import paper_2505_03269_gb300 as tcbf
    geom = ti.ultrasound_geometry(n_elements=32, n_bins=16, grid=(8, 8, 4))
    M, K = geom.targets.shape[0], geom.rx_pos.shape[0]
    N = 96
    X = ti.complex_gaussian_fp16(ti.rng(9), (1, K, N))
    with tcbf.Plan(1, M, N, K, tcbf.MODE_FP8SPLIT, flags=_flags(3)) as plan:
        Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
        plan.weights_from_geometry(dev(geom.rx_pos), dev(geom.targets), True,
                                   dev(np.ascontiguousarray(geom.freqs)), geom.c, Wp)
        plan.transpose_pack(1, dev(X), Xp)
        Y = torch.empty((1, M, N, 2), dtype=torch.float32, device="cuda")
        plan.beamform_fp8split(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        raw = Wp.cpu().numpy()
        Yh = Y.cpu().numpy().astype(np.float64)
    h, l, codes = _decode(raw, 1, M, K, 128, False)
    W16 = oracle.weights_fp16(geom.rx_pos, geom.targets, geom.freqs, True, geom.c)
    oh, ol, oe = oracle.split_blocks(W16.reshape(M, K, 2))
    same = (h[0].transpose(1, 2, 0) == oh) & (l[0].transpose(1, 2, 0) == ol)
    assert np.mean(same) >= 0.999
    assert np.mean(codes[0][..., :2].reshape(M, -1)[:, : oe.shape[1]] == 127 - oe) >= 0.99
    err = oracle.rel_frobenius(Yh[..., 0] + 1j * Yh[..., 1], oracle.cgemm(W16, X))
    assert err < 5e-3
