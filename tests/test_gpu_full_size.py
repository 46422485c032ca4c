"""Full-size FP16 blocks through the path the benchmark times, checked on
sampled outputs against the FP64 oracle.

  radio block:      512 products (256 channels x 2 polarisations) of
                    1024 beams x 288 receivers x 4096 samples, weights from
                    the station geometry on the GPU, one persistent launch
  ultrasound block: 65536 voxels x 16384 (128 elements x 128 bins) x 256
                    frames, near-field model matrix from geometry, stacked
                    sample planes
  both blocks also through the interleaved-X kernel (the GEMM reads X as
  it lies, no transpose/pack pass)

The oracle computes its own weights from the same geometry (FP64, rounded
once to FP16) and the complex sum at each sampled output.  Bar: relative
Frobenius error over the samples <= 2e-5."""
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


def _sampled_error(Y, Xh, geom, B, Bw, M, N, npts=96, seed=7):
    import torch
    g = np.random.default_rng(seed)
    pts = np.stack([g.integers(0, B, npts), g.integers(0, M, npts), g.integers(0, N, npts)], 1)
    ref = np.empty(npts, np.complex128)
    for i, (b, m, n) in enumerate(pts):
        bw = b // (B // Bw)
        Wrow = oracle.weights_fp16(geom.rx_pos, geom.targets[m:m + 1], geom.freqs[bw:bw + 1],
                                   geom.near_field, geom.c)
        ref[i] = oracle.cgemm_points(Wrow, Xh[b:b + 1], np.array([[0, 0, n]]))[0]
    t = torch.from_numpy(pts).cuda()
    Yh = Y[t[:, 0], t[:, 1], t[:, 2]].double().cpu().numpy()
    got = Yh[:, 0] + 1j * Yh[:, 1]
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def _run_block(B, Bw, M, N, K, geom, Xh, flags=0, configs=(None,)):
    import torch
    from gpu_util import empty_bytes
    from paper_2505_03269_gb300 import MODE_FP16, Plan
    errs = []
    with Plan(B, M, N, K, MODE_FP16, w_batches=Bw, flags=flags) as plan:
        Wp = empty_bytes(plan.packed_size(0))
        Xp = empty_bytes(plan.packed_size(1))
        rx = torch.from_numpy(geom.rx_pos).cuda()
        tg = torch.from_numpy(geom.targets).cuda()
        fr = torch.from_numpy(np.ascontiguousarray(geom.freqs[:Bw])).cuda()
        plan.weights_from_geometry(rx, tg, geom.near_field, fr, geom.c, Wp)
        Xd = torch.from_numpy(Xh).cuda()
        plan.transpose_pack(1, Xd, Xp)
        del Xd
        Y = torch.empty((B, M, N, 2), dtype=torch.float32, device="cuda")
        for c in configs:
            if c is not None:
                plan.set_config(c)
            Y.fill_(float("nan"))
            plan.beamform_fp16(Wp, Xp, Y)
            torch.cuda.synchronize()
            assert plan.last_device_error() == 0
            assert not torch.isnan(Y).any()
            errs.append(_sampled_error(Y, Xh, geom, B, Bw, M, N))
        del Y
    torch.cuda.empty_cache()
    return errs


def test_full_size_radio_block_sampled():
    B, Bw, M, K, N = 512, 256, 1024, 288, 4096
    geom = ti.radio_geometry(0, M, K, Bw)
    Xh = ti.radio_x(1, B, K, N)
    # the default tile shape and the cluster-multicast shape the autotuner picks most often
    for err in _run_block(B, Bw, M, N, K, geom, Xh, configs=(0, 6)):
        assert err <= TOL


def test_full_size_radio_block_interleaved_x_sampled():
    """The radio block through the interleaved-X kernel (no pack of X): every
    configuration (resident W with four or three stages, streamed W on SM
    pairs or one SM), sampled against the oracle."""
    from paper_2505_03269_gb300 import FLAG_INTERLEAVED_X
    B, Bw, M, K, N = 512, 256, 1024, 288, 4096
    geom = ti.radio_geometry(0, M, K, Bw)
    Xh = ti.radio_x(1, B, K, N)
    for err in _run_block(B, Bw, M, N, K, geom, Xh, flags=FLAG_INTERLEAVED_X,
                          configs=(0, 1, 2, 3, 4, 5, 6)):
        assert err <= TOL


def test_full_size_ultrasound_interleaved_x_sampled():
    from paper_2505_03269_gb300 import FLAG_INTERLEAVED_X
    M, K, N = 65536, 16384, 256
    geom = ti.ultrasound_geometry()
    Xh = ti.ultrasound_frames(1, K, N)
    for err in _run_block(1, 1, M, N, K, geom, Xh, flags=FLAG_INTERLEAVED_X, configs=(1,)):
        assert err <= TOL


def test_full_size_ultrasound_block_sampled():
    from paper_2505_03269_gb300 import FLAG_STACKED_X
    M, K, N = 65536, 16384, 256
    geom = ti.ultrasound_geometry()
    Xh = ti.ultrasound_frames(1, K, N)
    for err in _run_block(1, 1, M, N, K, geom, Xh, flags=FLAG_STACKED_X, configs=(0, 1, 2)):
        assert err <= TOL


def test_full_size_ultrasound_split_fp8_sampled():
    """Split-FP8 on the full ultrasound block: the GPU splits the weights it
    computes from geometry and the frames it packs; the oracle splits its own
    FP16 weights and frames.  Parity bar 2e-5 against the oracle's split
    arithmetic; the method's accuracy against the exact product (about 1e-3)
    is stated, with a loose ceiling."""
    import torch
    from gpu_util import empty_bytes
    from paper_2505_03269_gb300 import MODE_FP8SPLIT, Plan
    M, K, N = 65536, 16384, 256
    geom = ti.ultrasound_geometry()
    Xh = ti.ultrasound_frames(1, K, N)
    with Plan(1, M, N, K, MODE_FP8SPLIT) as plan:
        Wp = empty_bytes(plan.packed_size(0))
        Xp = empty_bytes(plan.packed_size(1))
        rx = torch.from_numpy(geom.rx_pos).cuda()
        tg = torch.from_numpy(geom.targets).cuda()
        fr = torch.from_numpy(np.ascontiguousarray(geom.freqs[:1])).cuda()
        plan.weights_from_geometry(rx, tg, geom.near_field, fr, geom.c, Wp)
        plan.transpose_pack(1, torch.from_numpy(Xh).cuda(), Xp)
        Y = torch.full((1, M, N, 2), float("nan"), dtype=torch.float32, device="cuda")
        plan.beamform_fp8split(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        g = np.random.default_rng(11)
        ms, ns = g.integers(0, M, 48), g.integers(0, N, 48)
        got = np.empty(48, np.complex128)
        ref_split = np.empty(48, np.complex128)
        ref = np.empty(48, np.complex128)
        for i, (m, n) in enumerate(zip(ms, ns)):
            Wrow = oracle.weights_fp16(geom.rx_pos, geom.targets[m:m + 1], geom.freqs[:1],
                                       geom.near_field, geom.c)
            Xcol = np.ascontiguousarray(Xh[:, :, n:n + 1])
            ref_split[i] = oracle.cgemm_split(Wrow, Xcol)[0, 0, 0]
            ref[i] = oracle.cgemm(Wrow, Xcol)[0, 0, 0]
            v = Y[0, int(m), int(n)].double().cpu().numpy()
            got[i] = v[0] + 1j * v[1]
    assert np.linalg.norm(got - ref_split) / np.linalg.norm(ref_split) <= TOL
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 5e-3


def test_full_size_ultrasound_plain_fp8_sampled():
    """Plain E4M3 (one byte per element, hi product only) on the full ultrasound
    shape.  W is drawn on the host (unit-magnitude random phases, FP16) so both
    sides see the same FP16 values: the GPU packs and multiplies them, the
    oracle splits the same rows and takes the one-product sum.  Parity bar 2e-5;
    the method's accuracy against the exact product (a few percent) is stated
    with a loose ceiling."""
    import torch
    from gpu_util import empty_bytes
    from paper_2505_03269_gb300 import FLAG_FP8_HI_ONLY, MODE_FP8SPLIT, Plan
    M, K, N = 65536, 16384, 256
    W = ti.random_phase_rows(3, M, K)
    Xh = ti.ultrasound_frames(1, K, N)
    with Plan(1, M, N, K, MODE_FP8SPLIT, flags=FLAG_FP8_HI_ONLY) as plan:
        Wp = empty_bytes(plan.packed_size(0))
        Xp = empty_bytes(plan.packed_size(1))
        Wd = torch.from_numpy(W).cuda()
        plan.transpose_pack(0, Wd, Wp)
        del Wd
        plan.transpose_pack(1, torch.from_numpy(Xh).cuda(), Xp)
        Y = torch.full((1, M, N, 2), float("nan"), dtype=torch.float32, device="cuda")
        plan.beamform_fp8split(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        g = np.random.default_rng(13)
        ms, ns = g.integers(0, M, 48), g.integers(0, N, 48)
        got = np.empty(48, np.complex128)
        ref_fp8 = np.empty(48, np.complex128)
        ref = np.empty(48, np.complex128)
        for i, (m, n) in enumerate(zip(ms, ns)):
            Wrow = np.ascontiguousarray(W[:, m:m + 1])
            Xcol = np.ascontiguousarray(Xh[:, :, n:n + 1])
            ref_fp8[i] = oracle.cgemm_split(Wrow, Xcol, products=1)[0, 0, 0]
            ref[i] = oracle.cgemm(Wrow, Xcol)[0, 0, 0]
            v = Y[0, int(m), int(n)].double().cpu().numpy()
            got[i] = v[0] + 1j * v[1]
        del Y
    torch.cuda.empty_cache()
    assert np.linalg.norm(got - ref_fp8) / np.linalg.norm(ref_fp8) <= TOL
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-1


@pytest.mark.parametrize("products", [3, 1])
def test_full_size_ultrasound_block_scaled_fp8_sampled(products):
    """Block-scaled FP8 (a scale per 32 k) on the full ultrasound shape.  Three
    products: W from the near-field geometry on the GPU, against the
    oracle's block split of its own FP16 weights.  One product: W drawn on
    the host (unit-magnitude random phases in FP16) so both sides split the
    same FP16 values (with one product a weight one FP16 unit apart can
    land on the neighbouring E4M3 value).  Parity bar 2e-5 against the
    oracle's block-scaled arithmetic; accuracy against the exact product
    stated with a loose ceiling."""
    import torch
    from gpu_util import empty_bytes
    from paper_2505_03269_gb300 import (FLAG_FP8_BLOCK_SCALES, FLAG_FP8_HI_ONLY, MODE_FP8SPLIT,
                                        Plan)
    M, K, N = 65536, 16384, 256
    geom = ti.ultrasound_geometry()
    Xh = ti.ultrasound_frames(1, K, N)
    Wh = ti.random_phase_rows(3, M, K) if products == 1 else None
    flags = FLAG_FP8_BLOCK_SCALES | (FLAG_FP8_HI_ONLY if products == 1 else 0)
    with Plan(1, M, N, K, MODE_FP8SPLIT, flags=flags) as plan:
        Wp = empty_bytes(plan.packed_size(0))
        Xp = empty_bytes(plan.packed_size(1))
        if Wh is None:
            rx = torch.from_numpy(geom.rx_pos).cuda()
            tg = torch.from_numpy(geom.targets).cuda()
            fr = torch.from_numpy(np.ascontiguousarray(geom.freqs[:1])).cuda()
            plan.weights_from_geometry(rx, tg, geom.near_field, fr, geom.c, Wp)
        else:
            Wd = torch.from_numpy(Wh).cuda()
            plan.transpose_pack(0, Wd, Wp)
            del Wd
        plan.transpose_pack(1, torch.from_numpy(Xh).cuda(), Xp)
        Y = torch.full((1, M, N, 2), float("nan"), dtype=torch.float32, device="cuda")
        plan.beamform_fp8split(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        g = np.random.default_rng(17)
        ms, ns = g.integers(0, M, 48), g.integers(0, N, 48)
        got = np.empty(48, np.complex128)
        ref_blk = np.empty(48, np.complex128)
        ref = np.empty(48, np.complex128)
        for i, (m, n) in enumerate(zip(ms, ns)):
            if Wh is None:
                Wrow = oracle.weights_fp16(geom.rx_pos, geom.targets[m:m + 1], geom.freqs[:1],
                                           geom.near_field, geom.c)
            else:
                Wrow = np.ascontiguousarray(Wh[:, m:m + 1])
            Xcol = np.ascontiguousarray(Xh[:, :, n:n + 1])
            ref_blk[i] = oracle.cgemm_split_blocks(Wrow, Xcol, products=products)[0, 0, 0]
            ref[i] = oracle.cgemm(Wrow, Xcol)[0, 0, 0]
            v = Y[0, int(m), int(n)].double().cpu().numpy()
            got[i] = v[0] + 1j * v[1]
        del Y
    torch.cuda.empty_cache()
    assert np.linalg.norm(got - ref_blk) / np.linalg.norm(ref_blk) <= TOL
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < (5e-3 if products > 1 else 1e-1)
