"""1-bit complex beamforming on the GPU against the exact int64 oracle.

Bar: bit-exact int32 output, on both arithmetic paths: bits expanded on
chip to E4M3 (configurations 0-4) and the 4-bit tensor path (5-7: E2M1
planes in the plan's scratch, block-scaled MMAs on SM pairs, the default),
including its expand-once entry points.  Inputs are iid fair bits,
including random bits beyond K in the last word (they must be ignored),
ragged shapes that leave partial tiles and partial stages, weight sharing
across batches, the matched-conjugate closed form, and the full-size 1-bit
radio block on sampled outputs."""
import numpy as np
import pytest

import oracle
import tcbf_inputs as ti

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import ensure_lib
    return ensure_lib()


def run_1bit(Wb, Xb, K, config=None):
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_1BIT, Plan
    Bw, _, M, kw = Wb.shape
    B, _, N, _ = Xb.shape
    with Plan(B, M, N, K, MODE_1BIT, w_batches=Bw) as plan:
        assert plan.Kw == kw
        if config is not None:
            plan.set_config(config)
        Y = torch.full((B, M, N, 2), -7, dtype=torch.int32, device="cuda")
        plan.beamform_1bit(dev(Wb), dev(Xb), Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        return Y.cpu().numpy().astype(np.int64)


# 5-7: the 4-bit tensor path (bits expanded to E2M1 planes in the plan's
# scratch, block-scaled MMAs on SM pairs)
@pytest.mark.parametrize("config", [0, 1, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("B,M,N,K", [(1, 1, 1, 1), (2, 3, 5, 7), (2, 33, 70, 45),
                                     (1, 128, 256, 1024), (3, 130, 300, 200),
                                     (2, 200, 64, 129), (1, 64, 1000, 640)])
def test_random_bits_bit_exact(config, B, M, N, K):
    Wb, Xb = ti.onebit_block(seed=M + N + K, B=B, M=M, K=K, N=N)
    Y = run_1bit(Wb, Xb, K, config)
    assert np.array_equal(Y, oracle.bgemm(Wb, Xb, K))


@pytest.mark.parametrize("config", [0, 4, 5, 6, 7, 8])
def test_shared_weights_bit_exact(config):
    g = ti.rng(4)
    K = 300
    Wb = ti.random_sign_words(g, (2, 2, 96, ti.words_per_row(K)))
    Xb = ti.random_sign_words(g, (6, 2, 150, ti.words_per_row(K)))
    Y = run_1bit(Wb, Xb, K, config)
    assert np.array_equal(Y, oracle.bgemm(Wb, Xb, K))


def test_matched_conjugate_gives_2K():
    K = 1000
    g = ti.rng(5)
    Xb = ti.random_sign_words(g, (1, 2, 256, ti.words_per_row(K)))
    Wb = Xb[:, :, :128].copy()
    Wb[:, 1] = ~Wb[:, 1]
    Y = run_1bit(Wb, Xb, K)
    d = np.arange(128)
    assert np.all(Y[0, d, d, 0] == 2 * K) and np.all(Y[0, d, d, 1] == 0)


def test_pack_then_gemm_pipeline():
    """Sign-pack FP16 values on the GPU, then the 1-bit GEMM, against the
    oracle's own sign packing and int64 product."""
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_1BIT, Plan
    B, M, N, K = 3, 100, 200, 333
    W, X = ti.small_fp16(seed=11, M=M, K=K, N=N, B=B)
    with Plan(B, M, N, K, MODE_1BIT) as plan:
        Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
        Y = torch.empty((B, M, N, 2), dtype=torch.int32, device="cuda")
        plan.transpose_pack(0, dev(W), Wp)
        plan.transpose_pack(1, dev(X), Xp)
        plan.beamform_1bit(Wp, Xp, Y)
        torch.cuda.synchronize()
        kw = plan.Kw
        Yg = Y.cpu().numpy().astype(np.int64)
    Wb = oracle.pack_signs(W, k_is_row=False, Kw=kw)
    Xb = oracle.pack_signs(X, k_is_row=True, Kw=kw)
    assert np.array_equal(Yg, oracle.bgemm(Wb, Xb, K))


@pytest.mark.parametrize("config", [0, 5, 6, 7, 8])
def test_full_size_radio_1bit_sampled(config):
    """64 channels x 2048 beams x 1024 receivers x 8192 samples: the whole
    launch as timed, checked bit-exact on sampled row/column blocks."""
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_1BIT, Plan
    B, M, K, N = 64, 2048, 1024, 8192
    Wb, Xb = ti.onebit_block(seed=0, B=B, M=M, K=K, N=N)
    with Plan(B, M, N, K, MODE_1BIT) as plan:
        plan.set_config(config)
        Y = torch.empty((B, M, N, 2), dtype=torch.int32, device="cuda")
        plan.beamform_1bit(dev(Wb), dev(Xb), Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        g = np.random.default_rng(0)
        for _ in range(6):
            b = int(g.integers(B))
            ms = np.sort(g.choice(M, 16, replace=False))
            ns = np.sort(g.choice(N, 16, replace=False))
            ref = oracle.bgemm(Wb[b:b + 1][:, :, ms], Xb[b:b + 1][:, :, ns], K)[0]
            got = Y[b][torch.from_numpy(ms).cuda()][:, torch.from_numpy(ns).cuda()]
            assert np.array_equal(got.cpu().numpy().astype(np.int64), ref)


def test_all_configurations_bit_identical():
    """Every 1-bit configuration, including stacked planes, gives the same
    exact integers on a ragged shape (partial tiles, a partial last K stage)."""
    Wb, Xb = ti.onebit_block(seed=31, B=3, M=389, K=333, N=270)
    ref = oracle.bgemm(Wb, Xb, 333)
    from paper_2505_03269_gb300 import MODE_1BIT, Plan
    with Plan(3, 389, 270, 333, MODE_1BIT) as plan:
        n = plan.num_configs()
    for c in range(n):
        assert np.array_equal(run_1bit(Wb, Xb, 333, c), ref), c


def test_default_configuration_is_the_4bit_path():
    from paper_2505_03269_gb300 import MODE_1BIT, Plan
    with Plan(2, 300, 200, 500, MODE_1BIT) as plan:
        assert plan.config_name(plan.get_config()).startswith("1bit->e2m1")


def test_default_configuration_threshold_in_k():
    """K <= 6144 starts on the 256 x 112 two-accumulator tiles (configuration
    8), larger K on the 256 x 128 one-accumulator tiles (configuration 5)."""
    from paper_2505_03269_gb300 import MODE_1BIT, Plan
    with Plan(1, 256, 256, 6144, MODE_1BIT) as plan:
        assert plan.get_config() == 8, plan.config_name(plan.get_config())
    with Plan(1, 256, 256, 6145, MODE_1BIT) as plan:
        assert plan.get_config() == 5, plan.config_name(plan.get_config())


def test_expand_once_then_gemm_per_block():
    """W expanded once, then X blocks expanded and multiplied in turn: each
    block exact, and equal to the one-call path."""
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_1BIT, Plan
    B, M, N, K = 2, 260, 190, 700
    g = ti.rng(41)
    Wb = ti.random_sign_words(g, (1, 2, M, ti.words_per_row(K)))
    with Plan(B, M, N, K, MODE_1BIT, w_batches=1) as plan:
        for config in (5, 6, 7):
            plan.set_config(config)
            plan.expand_1bit(0, dev(Wb))
            for blk in range(3):
                Xb = ti.random_sign_words(g, (B, 2, N, ti.words_per_row(K)))
                Y = torch.full((B, M, N, 2), -7, dtype=torch.int32, device="cuda")
                plan.expand_1bit(1, dev(Xb))
                plan.beamform_1bit_expanded(Y)
                Y1 = torch.full_like(Y, -9)
                plan.beamform_1bit(dev(Wb), dev(Xb), Y1)
                torch.cuda.synchronize()
                assert plan.last_device_error() == 0
                got = Y.cpu().numpy().astype(np.int64)
                assert np.array_equal(got, oracle.bgemm(Wb, Xb, K)), (config, blk)
                assert np.array_equal(got, Y1.cpu().numpy().astype(np.int64))


def test_expand_needs_the_4bit_path():
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_1BIT, Plan, TcbfError
    K = 64
    Wb = ti.random_sign_words(ti.rng(42), (1, 2, 8, ti.words_per_row(K)))
    with Plan(1, 8, 8, K, MODE_1BIT) as plan:
        plan.set_config(0)
        with pytest.raises(TcbfError, match="UNSUPPORTED"):
            plan.expand_1bit(0, dev(Wb))
        Y = torch.zeros((1, 8, 8, 2), dtype=torch.int32, device="cuda")
        with pytest.raises(TcbfError, match="UNSUPPORTED"):
            plan.beamform_1bit_expanded(Y)
        plan.set_config(5)
        with pytest.raises(TcbfError, match="INVALID_ARG"):
            plan.expand_1bit(2, dev(Wb))
        plan.set_batch_rows([3])          # uneven rows: not on the 4-bit path
        with pytest.raises(TcbfError, match="UNSUPPORTED"):
            plan.expand_1bit(0, dev(Wb))


def test_radio_signs_from_geometry_exact():
    """The configured 1-bit radio recipe on a reduced block: W = signs of the
    steering weights computed by the GPU's weights kernel on a 1-bit plan,
    X = signs of complex Gaussian samples packed by the GPU; the oracle takes
    the signs of its own FP64 weights of the same geometry and its own sign
    packing of the same samples.  Exact int32 output on every element."""
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_1BIT, Plan
    B, M, K, N = 4, 256, 1024, 512
    geom = ti.radio_geometry(seed=0, n_beams=M, n_stations=K, n_channels=B)
    X = ti.radio_x(1, B, K, N)
    with Plan(B, M, N, K, MODE_1BIT) as plan:
        Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
        plan.weights_from_geometry(dev(geom.rx_pos), dev(geom.targets), geom.near_field,
                                   dev(geom.freqs), geom.c, Wp)
        plan.transpose_pack(1, dev(X), Xp)
        Y = torch.full((B, M, N, 2), -7, dtype=torch.int32, device="cuda")
        plan.beamform_1bit(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        got = Y.cpu().numpy().astype(np.int64)
        kw = plan.Kw
        wbits_gpu = Wp.cpu().numpy().view(np.uint32).reshape(B, 2, M, kw)
    wc = oracle.weights(geom.rx_pos, geom.targets, geom.freqs, geom.near_field, geom.c)
    Wb = oracle.pack_signs_f64(wc, kw)
    assert np.array_equal(wbits_gpu, Wb)
    Xb = oracle.pack_signs(X, k_is_row=True, Kw=kw)
    assert np.array_equal(got, oracle.bgemm(Wb, Xb, K))


@pytest.mark.parametrize("config", [5, 6, 7, 8])
@pytest.mark.parametrize("B,M,N,K,f32", [(2, 300, 200, 333, False), (3, 130, 70, 64, False),
                                         (1, 257, 129, 1025, True), (2, 64, 33, 31, True)])
def test_pack_straight_into_e2m1_planes(config, B, M, N, K, f32):
    """tcbf_transpose_pack_expanded (complex values -> E2M1 planes in one
    pass) gives exactly the oracle's product of the sign-quantised values,
    on ragged K (a partial word pair) and with -0 and NaN components (-0 is
    +1, NaN is -1), for FP16 and FP32 sources."""
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_1BIT, SRC_CF16, SRC_CF32, Plan
    g = ti.rng(B * 1000 + K)
    W = ti.complex_gaussian_fp16(g, (B, M, K))
    X = ti.complex_gaussian_fp16(g, (B, K, N))
    W.reshape(-1)[::17] = np.float16(-0.0)
    X.reshape(-1)[::13] = np.float16(-0.0)
    X.reshape(-1)[5::29] = np.float16(np.nan)
    src_type = SRC_CF32 if f32 else SRC_CF16
    Ws, Xs = (W.astype(np.float32), X.astype(np.float32)) if f32 else (W, X)
    with Plan(B, M, N, K, MODE_1BIT) as plan:
        plan.set_config(config)
        plan.transpose_pack_expanded(0, dev(Ws), src_type)
        plan.transpose_pack_expanded(1, dev(Xs), src_type)
        Y = torch.full((B, M, N, 2), -7, dtype=torch.int32, device="cuda")
        plan.beamform_1bit_expanded(Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        got = Y.cpu().numpy().astype(np.int64)
        kw = plan.Kw
    Wb = oracle.pack_signs(W, k_is_row=False, Kw=kw)
    Xb = oracle.pack_signs(X, k_is_row=True, Kw=kw)
    assert np.array_equal(got, oracle.bgemm(Wb, Xb, K))
