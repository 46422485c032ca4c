"""Transpose/pack and weights-from-geometry kernels against the oracle.

Packing only moves data (and rounds FP32 to FP16, or keeps a sign), so it
must match bit for bit.  Weights are computed with an FP64 phase reduction
and FP32 sin/cos, then rounded to FP16: they must lie within one FP16 ulp
of the oracle's FP64 weights rounded once, and equal them for >= 99.9 % of
entries."""
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


def _plan(B, M, N, K, mode, Bw=0):
    from paper_2505_03269_gb300 import Plan
    return Plan(B, M, N, K, mode, w_batches=Bw)


def _packed(plan, which, src, src_type=0):
    import torch
    from gpu_util import dev
    dst = torch.zeros(plan.packed_size(which), dtype=torch.uint8, device="cuda")
    plan.transpose_pack(which, dev(src), dst, src_type)
    torch.cuda.synchronize()
    return dst.cpu().numpy()


def _expected_planes(V16, k_axis_last):
    """Planar layout of interleaved complex FP16: [nb][2][rows][Kp] with zero pad."""
    if not k_axis_last:                     # X [B][K][N][2] -> rows are N
        V16 = np.ascontiguousarray(V16.transpose(0, 2, 1, 3))
    nb, rows, K, _ = V16.shape
    Kp = (K + 63) // 64 * 64
    out = np.zeros((nb, 2, rows, Kp), np.float16)
    out[:, 0, :, :K] = V16[..., 0]
    out[:, 1, :, :K] = V16[..., 1]
    return out


@pytest.mark.parametrize("B,M,N,K", [(1, 5, 7, 3), (3, 70, 130, 77), (2, 64, 256, 288),
                                     (2, 40, 132, 77), (1, 16, 4096, 288)])
def test_pack_fp16_layout_bit_exact(B, M, N, K):
    from paper_2505_03269_gb300 import MODE_FP16
    W, X = ti.small_fp16(seed=B + M, M=M, K=K, N=N, B=B)
    with _plan(B, M, N, K, MODE_FP16) as plan:
        Wp = _packed(plan, 0, W).view(np.float16)
        Xp = _packed(plan, 1, X).view(np.float16)
    assert np.array_equal(Wp.view(np.uint16), _expected_planes(W, True).ravel().view(np.uint16))
    assert np.array_equal(Xp.view(np.uint16), _expected_planes(X, False).ravel().view(np.uint16))


@pytest.mark.parametrize("N", [66, 68])          # row starts unaligned / 16-byte aligned
def test_pack_fp32_source_rounds_to_nearest_even(N):
    from paper_2505_03269_gb300 import MODE_FP16, SRC_CF32
    g = np.random.default_rng(3)
    X32 = (g.standard_normal((2, 40, N, 2)) * 1000).astype(np.float32)
    # values exactly between two FP16 numbers must round to even
    X32[0, 0, :4, 0] = np.array([1 + 2**-11, 1 + 3 * 2**-11, -(1 + 2**-11), 2049.0], np.float32)
    with _plan(2, 4, N, 40, MODE_FP16) as plan:
        Xp = _packed(plan, 1, X32, SRC_CF32).view(np.float16)
    assert np.array_equal(Xp.view(np.uint16),
                          _expected_planes(X32.astype(np.float16), False).ravel().view(np.uint16))


@pytest.mark.parametrize("B,M,N,K", [(1, 3, 5, 1), (2, 33, 70, 45), (2, 64, 96, 300)])
def test_pack_1bit_signs_bit_exact(B, M, N, K):
    from paper_2505_03269_gb300 import MODE_1BIT
    W, X = ti.small_fp16(seed=K, M=M, K=K, N=N, B=B)
    # special values: signed zeros, tiny and huge magnitudes
    flat = X.reshape(-1)
    flat[:6] = np.array([0.0, -0.0, 6e-8, -6e-8, 65504, -65504], np.float16)
    with _plan(B, M, N, K, MODE_1BIT) as plan:
        Wb = _packed(plan, 0, W).view(np.uint32)
        Xb = _packed(plan, 1, X).view(np.uint32)
        kw = plan.Kw
    assert np.array_equal(Wb, oracle.pack_signs(W, k_is_row=False, Kw=kw).ravel())
    assert np.array_equal(Xb, oracle.pack_signs(X, k_is_row=True, Kw=kw).ravel())


def _ulp_key(h16):
    u = h16.view(np.uint16).astype(np.int32)
    mag = u & 0x7FFF
    return np.where(u & 0x8000, -mag, mag)


def _gpu_weights(geom, Bw, mode):
    import torch
    from gpu_util import dev
    M, K = geom.targets.shape[0], geom.rx_pos.shape[0]
    with _plan(Bw, M, 8, K, mode) as plan:
        Wp = torch.zeros(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        plan.weights_from_geometry(dev(geom.rx_pos), dev(geom.targets), geom.near_field,
                                   dev(np.ascontiguousarray(geom.freqs[:Bw])), geom.c, Wp)
        torch.cuda.synchronize()
        return Wp.cpu().numpy(), plan.Kp, plan.Kw


@pytest.mark.parametrize("which", ["radio", "ultrasound"])
def test_weights_fp16_within_one_ulp(which):
    from paper_2505_03269_gb300 import MODE_FP16
    if which == "radio":
        geom = ti.radio_geometry(seed=0, n_beams=512, n_stations=288, n_channels=4)
        Bw = 4
    else:
        geom = ti.ultrasound_geometry(grid=(16, 8, 8))      # 1024 voxels x 16384 columns
        Bw = 1
    raw, Kp, _ = _gpu_weights(geom, Bw, MODE_FP16)
    M, K = geom.targets.shape[0], geom.rx_pos.shape[0]
    got = raw.view(np.float16).reshape(Bw, 2, M, Kp)
    ref = oracle.weights_fp16(geom.rx_pos, geom.targets, geom.freqs[:Bw], geom.near_field, geom.c)
    for p in range(2):
        a = _ulp_key(np.ascontiguousarray(got[:, p, :, :K]))
        b = _ulp_key(np.ascontiguousarray(ref[..., p]))
        d = np.abs(a - b)
        assert d.max() <= 1
        assert np.mean(d == 0) >= 0.999
    assert np.all(got[:, :, :, K:] == 0)


def test_weights_1bit_signs():
    """Sign bits of the weights; components within 1e-6 of zero may go either way."""
    from paper_2505_03269_gb300 import MODE_1BIT
    geom = ti.radio_geometry(seed=1, n_beams=256, n_stations=300, n_channels=2)
    raw, _, kw = _gpu_weights(geom, 2, MODE_1BIT)
    M, K = 256, 300
    got = raw.view(np.uint32).reshape(2, 2, M, kw)
    w = oracle.weights(geom.rx_pos, geom.targets, geom.freqs[:2], False, geom.c)
    k = np.arange(K)
    bits = (got[..., k // 32] >> (k % 32).astype(np.uint32)) & 1          # [2, 2, M, K]
    for p, comp in ((0, w.real), (1, w.imag)):
        sure = np.abs(comp) > 1e-6
        assert np.array_equal(bits[:, p][sure], (comp >= 0)[sure].astype(np.uint32))
    # pad bits beyond K are zero
    assert np.all((got[..., K // 32] >> np.uint32(K % 32)) == 0)


def test_weights_then_gemm_pipeline():
    """GPU weights -> GPU GEMM against oracle weights -> oracle GEMM."""
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_FP16, Plan
    geom = ti.radio_geometry(seed=0, n_beams=256, n_stations=288, n_channels=4)
    B, Bw, M, K, N = 8, 4, 256, 288, 512
    X = ti.radio_x(1, B, K, N)
    with Plan(B, M, N, K, MODE_FP16, w_batches=Bw) as plan:
        Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
        Y = torch.empty((B, M, N, 2), dtype=torch.float32, device="cuda")
        plan.weights_from_geometry(dev(geom.rx_pos), dev(geom.targets), False,
                                   dev(np.ascontiguousarray(geom.freqs[:Bw])), geom.c, Wp)
        plan.transpose_pack(1, dev(X), Xp)
        plan.beamform_fp16(Wp, Xp, Y)
        torch.cuda.synchronize()
        Yh = Y.cpu().numpy().astype(np.float64)
    Yg = Yh[..., 0] + 1j * Yh[..., 1]
    Wref = oracle.weights_fp16(geom.rx_pos, geom.targets, geom.freqs[:Bw], False, geom.c)
    assert oracle.rel_frobenius(Yg, oracle.cgemm(Wref, X)) <= 2e-5


@pytest.mark.parametrize("which,dst_type", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("B,M,N,K", [(1, 3, 5, 1), (2, 33, 70, 45), (2, 64, 96, 300)])
def test_unpack_1bit_inverts_pack_exactly(which, dst_type, B, M, N, K):
    """tcbf_unpack_bits on the GPU's own packed signs gives back sign(v) as +-1,
    and on random words (junk beyond K included) equals the oracle's unpacking."""
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_1BIT
    W, X = ti.small_fp16(seed=K + 3, M=M, K=K, N=N, B=B)
    X.reshape(-1)[:2] = np.array([0.0, -0.0], np.float16)
    V = W if which == 0 else X
    rows = M if which == 0 else N
    dt = torch.float16 if dst_type == 0 else torch.float32
    with _plan(B, M, N, K, MODE_1BIT) as plan:
        kw = plan.Kw
        packed = _packed(plan, which, V).view(np.uint32).reshape(B, 2, rows, kw)
        words = ti.random_sign_words(ti.rng(K + 4), (B, 2, rows, kw))
        outs = []
        for src in (packed, words):
            out = torch.full(V.shape, 7.0, dtype=dt, device="cuda")
            plan.unpack_bits(which, dev(np.ascontiguousarray(src)), out, dst_type)
            torch.cuda.synchronize()
            assert plan.last_device_error() == 0
            outs.append(out.cpu().numpy().astype(np.float64))
    assert np.array_equal(outs[0], np.where(V.astype(np.float64) >= 0, 1.0, -1.0))
    assert np.array_equal(outs[1], oracle.unpack_signs(words, K, k_is_row=(which == 1)))
