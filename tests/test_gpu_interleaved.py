"""FP16 beamforming on interleaved complex samples (plans with
TCBF_FLAG_INTERLEAVED_X: the GEMM reads X as the caller holds it, with no
transpose/pack pass) against the FP64 CPU oracle.

The kernel forms Wr X and Wi X side by side from an MN-major operand and
combines them into Re and Im in FP32, so its rounding differs from the planar
kernels': results are held to the oracle at the FP16 tolerance (relative
Frobenius error <= 2e-5), and integer-valued or identity inputs, whose FP32
partial sums are all exact, bit for bit.  Shapes span several tiles and
ragged edges in M, N and K, and both operand-load forms (W in one 5-D box
when M % 8 == 0, else per 8-beam group; X in one 4-D box when N % 32 == 0,
else per 64 columns); N % 4 != 0 and uneven batch rows take the
pack-and-planar fallback inside the same call."""
import numpy as np
import pytest

import oracle
import tcbf_inputs as ti

pytestmark = pytest.mark.gpu

TOL = 2e-5
# resident W (4 stages of 128 K, K <= 320), SM pairs with 128-K / 64-K stages, one SM,
# resident W (3 stages, K <= 384; 5 stages of 96 K and 8 of 64 K, K <= 320)
CONFIGS = [0, 1, 2, 3, 4, 5, 6]
LONG_K_CONFIGS = [1, 2, 3]


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_util import ensure_lib
    return ensure_lib()


def _run(W, X, **k):
    import paper_2505_03269_gb300 as tcbf
    from gpu_util import run_fp16
    return run_fp16(W, X, flags=tcbf.FLAG_INTERLEAVED_X, **k)


@pytest.mark.parametrize("config", CONFIGS)
def test_small_fp16_workload(config):
    """64 beams x 128 receivers x 1024 samples, batch 1, seed 0."""
    W, X = ti.small_fp16(seed=0)
    Y = _run(W, X, config=config)
    assert oracle.rel_frobenius(Y, oracle.cgemm(W, X)) <= TOL


@pytest.mark.parametrize("config", CONFIGS)
@pytest.mark.parametrize("M,N,K", [(1, 4, 1), (3, 8, 7), (17, 36, 127), (129, 132, 288),
                                   (127, 260, 129), (200, 96, 64), (64, 1024, 200),
                                   (300, 388, 45), (1024, 512, 288), (136, 100, 72),
                                   (130, 64, 300)])
def test_ragged_shapes(config, M, N, K):
    W, X = ti.small_fp16(seed=M * 7 + N + K, M=M, K=K, N=N, B=2)
    Y = _run(W, X, config=config)
    assert oracle.rel_frobenius(Y, oracle.cgemm(W, X)) <= TOL


@pytest.mark.parametrize("M,N,K", [(5, 1, 3), (33, 7, 70), (130, 258, 100), (64, 1021, 288)])
def test_sample_counts_not_multiple_of_four(M, N, K):
    """Rows of X that TMA cannot address (4N bytes not a multiple of 16) go
    through the plan's packed planes and the planar kernel."""
    W, X = ti.small_fp16(seed=N + K, M=M, K=K, N=N, B=3)
    Y = _run(W, X)
    assert oracle.rel_frobenius(Y, oracle.cgemm(W, X)) <= TOL


@pytest.mark.parametrize("config", CONFIGS)
def test_integer_inputs_bit_exact(config):
    g = ti.rng(1)
    W = ti.integer_complex_fp16(g, (2, 150, 300))
    X = ti.integer_complex_fp16(g, (4, 300, 272))
    Y = _run(W, X, config=config)
    assert np.array_equal(Y, oracle.cgemm(W, X))


@pytest.mark.parametrize("config", CONFIGS)
def test_identity_weights_bit_exact(config):
    K, N = 160, 300
    W = np.zeros((1, K, K, 2), np.float16)
    W[0, np.arange(K), np.arange(K), 0] = 1.0
    _, X = ti.small_fp16(seed=2, M=1, K=K, N=N)
    Y = _run(W, X, config=config)
    Xc = X[..., 0].astype(np.float64) + 1j * X[..., 1].astype(np.float64)
    assert np.array_equal(Y, Xc)


@pytest.mark.parametrize("config", CONFIGS)
def test_imaginary_identity_weights(config):
    """W = i I maps X to i X: Re takes -Wi Xi from the partner lane, Im +Wi Xr."""
    K, N = 96, 64
    W = np.zeros((1, K, K, 2), np.float16)
    W[0, np.arange(K), np.arange(K), 1] = 1.0
    _, X = ti.small_fp16(seed=5, M=1, K=K, N=N)
    Y = _run(W, X, config=config)
    Xc = X[..., 0].astype(np.float64) + 1j * X[..., 1].astype(np.float64)
    assert np.array_equal(Y, 1j * Xc)


@pytest.mark.parametrize("config", CONFIGS)
def test_one_nonzero_weight_per_beam(config):
    """Beam m reads receiver (3 m) mod K with weight (m % 5 - 2) + (m % 3 - 1) i:
    every output is one exact complex product, so a lane or column
    misplaced anywhere in the tile shows up as a wrong value."""
    M, K, N = 200, 77, 136
    W = np.zeros((1, M, K, 2), np.float16)
    m = np.arange(M)
    W[0, m, (3 * m) % K, 0] = (m % 5) - 2
    W[0, m, (3 * m) % K, 1] = (m % 3) - 1
    X = ti.integer_complex_fp16(ti.rng(3), (2, K, N))
    Y = _run(W, X, config=config)
    assert np.array_equal(Y, oracle.cgemm(W, X))


def test_shared_weights_across_batches():
    g = ti.rng(6)
    W, _ = ti.small_fp16(seed=6, M=100, K=72, N=8, B=3)
    X = ti.complex_gaussian_fp16(g, (6, 72, 152))
    Y = _run(W, X)
    assert oracle.rel_frobenius(Y, oracle.cgemm(W, X)) <= TOL


def test_fp32_source_rounds_to_nearest():
    g = ti.rng(8)
    W32 = g.standard_normal((1, 40, 56, 2)).astype(np.float32)
    X32 = g.standard_normal((2, 56, 48, 2)).astype(np.float32)
    from paper_2505_03269_gb300 import SRC_CF32
    Y = _run(W32, X32, src_type=SRC_CF32)
    Yref = oracle.cgemm(W32.astype(np.float16), X32.astype(np.float16))
    assert oracle.rel_frobenius(Y, Yref) <= TOL


@pytest.mark.parametrize("config", LONG_K_CONFIGS)
@pytest.mark.parametrize("K", [4100, 8192, 16384])
def test_long_k_within_tolerance(config, K):
    """Above K = 4096 the partial sums are promoted to FP32 every 2048 K."""
    W, _ = ti.small_fp16(seed=K, M=256, K=K, N=8)
    X = ti.complex_gaussian_fp16(ti.rng(K + 1), (1, K, 192))
    Y = _run(W, X, config=config)
    assert oracle.rel_frobenius(Y, oracle.cgemm(W, X)) <= TOL


def test_long_k_integer_inputs_bit_exact():
    g = ti.rng(12)
    W = ti.integer_complex_fp16(g, (1, 130, 9000), lo=-2, hi=2)
    X = ti.integer_complex_fp16(g, (1, 9000, 72), lo=-2, hi=2)
    Y = _run(W, X)
    assert np.array_equal(Y, oracle.cgemm(W, X))


def test_uneven_batch_rows():
    """Per-batch beam counts take the planar fallback; rows below rows[b]
    must match the oracle."""
    rows = [1, 130, 64, 200]
    g = ti.rng(9)
    W, _ = ti.small_fp16(seed=9, M=200, K=96, N=8, B=4)
    X = ti.complex_gaussian_fp16(g, (4, 96, 136))
    Y = _run(W, X, rows=rows)
    ref = oracle.cgemm(W, X)
    for b, r in enumerate(rows):
        assert oracle.rel_frobenius(Y[b, :r], ref[b, :r]) <= TOL


def test_packed_size_and_plain_copy():
    """X of an interleaved plan is the caller's layout: packed_size(1) is
    batch*K*N*4 bytes and transpose_pack copies it unchanged."""
    import torch
    import paper_2505_03269_gb300 as tcbf
    from gpu_util import dev
    B, M, N, K = 3, 40, 20, 30
    _, X = ti.small_fp16(seed=4, M=M, K=K, N=N, B=B)
    with tcbf.Plan(B, M, N, K, tcbf.MODE_FP16, flags=tcbf.FLAG_INTERLEAVED_X) as plan:
        assert plan.packed_size(1) == B * K * N * 4
        Xd = dev(X)
        Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
        plan.transpose_pack(1, Xd, Xp)
        torch.cuda.synchronize()
        assert np.array_equal(Xp.cpu().numpy(), X.view(np.uint8).ravel())


def test_autotune_and_graph_replay():
    import torch
    import paper_2505_03269_gb300 as tcbf
    from gpu_util import dev, empty_bytes
    W, X = ti.small_fp16(seed=21, M=256, K=288, N=512, B=4)
    B, K, N = X.shape[0], X.shape[1], X.shape[2]
    M = W.shape[1]
    with tcbf.Plan(B, M, N, K, tcbf.MODE_FP16, w_batches=4, flags=tcbf.FLAG_INTERLEAVED_X) as plan:
        assert plan.num_configs() == 7
        Wp = empty_bytes(plan.packed_size(0))
        Xd = dev(X)
        plan.transpose_pack(0, dev(W), Wp)
        Y = torch.empty((B, M, N, 2), dtype=torch.float32, device="cuda")
        best, ms = plan.autotune(Wp, Xd, Y, reps=2)
        assert best in range(7) and all(v > 0 for v in ms)
        Y.zero_()
        plan.beamform_fp16(Wp, Xd, Y)
        torch.cuda.synchronize()
        direct = Y.cpu().numpy()
        Y.zero_()
        plan.graph_capture(None, Xd, Wp, Y)
        plan.graph_launch()
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        assert np.array_equal(Y.cpu().numpy(), direct)
    Yc = direct.astype(np.float64)
    assert oracle.rel_frobenius(Yc[..., 0] + 1j * Yc[..., 1], oracle.cgemm(W, X)) <= TOL


def test_host_pipeline():
    """tcbf_beamform_host on an interleaved plan: X copied in goes straight
    to the GEMM (no pack)."""
    import torch
    import paper_2505_03269_gb300 as tcbf
    from gpu_util import dev, empty_bytes
    W, X = ti.small_fp16(seed=31, M=96, K=64, N=256, B=8)
    B, K, N, M = X.shape[0], X.shape[1], X.shape[2], W.shape[1]
    with tcbf.Plan(B, M, N, K, tcbf.MODE_FP16, w_batches=8, flags=tcbf.FLAG_INTERLEAVED_X) as plan:
        Wp = empty_bytes(plan.packed_size(0))
        plan.transpose_pack(0, dev(W), Wp)
        Xh = torch.from_numpy(X).pin_memory()
        Yh = torch.empty((B, M, N, 2), dtype=torch.float32, pin_memory=True)
        plan.beamform_host(Xh, Wp, Yh, chunk=2)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        Y = Yh.numpy().astype(np.float64)
    assert oracle.rel_frobenius(Y[..., 0] + 1j * Y[..., 1], oracle.cgemm(W, X)) <= TOL


def test_resident_weights_limited_to_short_k():
    """Configurations 0, 5 and 6 keep W in shared memory beside four, five
    or eight X stages and need K <= 320, configuration 4 (three stages)
    K <= 384: up to 320 the plan starts on whichever of 0 and 5 keeps more
    K rows in flight (5 at K = 288), on 4 up to 384, and on the streaming
    pair tiles above; each resident form is refused above its K."""
    import paper_2505_03269_gb300 as tcbf
    for K, default, refused in ((288, 5, []), (256, 0, []), (64, 5, []), (320, 0, []),
                                (321, 4, [0, 5, 6]), (384, 4, [0, 5, 6]), (385, 1, [0, 4, 5, 6])):
        with tcbf.Plan(1, 8, 8, K, tcbf.MODE_FP16, flags=tcbf.FLAG_INTERLEAVED_X) as plan:
            assert plan.get_config() == default, K
            for c in refused:
                with pytest.raises(tcbf.TcbfError):
                    plan.set_config(c)


@pytest.mark.parametrize("config,K", [(0, 1), (0, 64), (0, 129), (0, 288), (0, 319), (0, 320),
                                      (4, 1), (4, 129), (4, 288), (4, 383), (4, 384),
                                      (5, 1), (5, 95), (5, 97), (5, 288), (5, 320),
                                      (6, 1), (6, 65), (6, 288), (6, 320)])
def test_resident_weights_across_k(config, K):
    """Every resident-W block count (1-5 or 1-6 blocks of 64 K, ragged last
    block) with several units per pair (uneven unit counts over the pairs)."""
    W, X = ti.small_fp16(seed=K, M=300, K=K, N=520, B=3)
    Y = _run(W, X, config=config)
    assert oracle.rel_frobenius(Y, oracle.cgemm(W, X)) <= TOL


def test_flag_rules():
    import paper_2505_03269_gb300 as tcbf
    with pytest.raises(tcbf.TcbfError):      # FP16 only
        tcbf.Plan(1, 8, 8, 8, tcbf.MODE_1BIT, flags=tcbf.FLAG_INTERLEAVED_X)
    with pytest.raises(tcbf.TcbfError):      # not with stacked planes
        tcbf.Plan(1, 8, 8, 8, tcbf.MODE_FP16,
                  flags=tcbf.FLAG_INTERLEAVED_X | tcbf.FLAG_STACKED_X)
    with tcbf.Plan(1, 8, 8, 8, tcbf.MODE_FP16, flags=tcbf.FLAG_INTERLEAVED_X) as plan:
        with pytest.raises(tcbf.TcbfError):  # the failure-path hook is one-SM planar only
            plan.debug_drop_fill(0)


@pytest.mark.parametrize("config", [0, 4, 5, 6])
@pytest.mark.parametrize("B,Bw,M,N", [(6, 2, 300, 520), (6, 1, 300, 520), (5, 5, 300, 520),
                                      (152, 76, 100, 64), (304, 76, 100, 36)])
def test_resident_weights_shared_by_several_products(config, B, Bw, M, N):
    """Products that share a weight batch run back to back on one resident
    W (one W load per weight batch and 128 beams) when that fills the last
    wave of SM pairs as well: 152 and 304 products of one 128-beam row on
    76 pairs take groups of 2 and 4; the ragged cases keep one product per
    unit.  Every product against the oracle."""
    W, _ = ti.small_fp16(seed=B * 10 + Bw, M=M, K=288, N=8, B=Bw)
    X = ti.complex_gaussian_fp16(ti.rng(B + Bw), (B, 288, N))
    Y = _run(W, X, config=config)
    assert oracle.rel_frobenius(Y, oracle.cgemm(W, X)) <= TOL
