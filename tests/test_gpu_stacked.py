"""FP16 plans with stacked sample planes (TCBF_FLAG_STACKED_X).

The packed X holds [-Xi, Xr, Xi]; the GEMM issues Wr [Xr; Xi] + Wi [-Xi; Xr]
as two N = 256 MMAs per K step, on one SM (configurations 1-4) or on SM
pairs with M = 256 (configuration 0, the default).  Bars: the packed bytes are the plain
planes plus the sign-flipped imaginary plane, bit for bit; the product is
within the FP16 parity bar of the FP64 oracle; and because every output
element is summed in the same order as in the four-MMA kernel (Wr Xr then
-Wi Xi, Wr Xi then Wi Xr, promoted every 2048 K in both), the two paths
agree bit for bit."""
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


def _run(W, X, stacked=True, config=None, src_type=0, rows=None, packed=False):
    import torch
    from gpu_util import dev, empty_bytes
    from paper_2505_03269_gb300 import FLAG_STACKED_X, MODE_FP16, Plan
    Bw, M, K, _ = W.shape
    B, _, N, _ = X.shape
    with Plan(B, M, N, K, MODE_FP16, w_batches=Bw, flags=FLAG_STACKED_X if stacked else 0) as plan:
        if config is not None:
            plan.set_config(config)
        if rows is not None:
            plan.set_batch_rows(rows)
        Wp = empty_bytes(plan.packed_size(0))
        Xp = empty_bytes(plan.packed_size(1))
        Y = torch.full((B, M, N, 2), float("nan"), dtype=torch.float32, device="cuda")
        plan.transpose_pack(0, dev(W), Wp, src_type)
        plan.transpose_pack(1, dev(X), Xp, src_type)
        plan.beamform_fp16(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        Yh = Y.cpu().numpy().astype(np.float64)
        out = Yh[..., 0] + 1j * Yh[..., 1]
        if packed:
            return out, Xp.cpu().numpy(), (K + 63) // 64 * 64
        return out


@pytest.mark.parametrize("B,N,K,src", [(2, 130, 77, 0), (1, 256, 288, 0), (2, 68, 40, 1),
                                       (1, 7, 3, 0)])
def test_stacked_pack_layout_bit_exact(B, N, K, src):
    W, X = ti.small_fp16(seed=N + K, M=16, K=K, N=N, B=B)
    if src == 1:
        _, Xp, Kp = _run(W.astype(np.float32), X.astype(np.float32), src_type=1, packed=True)
    else:
        _, Xp, Kp = _run(W, X, packed=True)
    Xp = Xp[: B * 3 * N * Kp * 2].view(np.uint16).reshape(B, 3, N, Kp)
    Xt = np.ascontiguousarray(X.transpose(0, 2, 1, 3))          # [B][N][K][2]
    want = np.zeros((B, 3, N, Kp), np.uint16)
    want[:, 1, :, :K] = Xt[..., 0].view(np.uint16)
    want[:, 2, :, :K] = Xt[..., 1].view(np.uint16)
    want[:, 0] = want[:, 2] ^ 0x8000     # -Xi: every sign bit flipped, zero pad included
    assert np.array_equal(Xp, want)


@pytest.mark.parametrize("config", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (3, 5, 7), (129, 130, 288), (127, 257, 129),
                                   (200, 96, 64), (64, 1024, 200), (300, 260, 70)])
def test_stacked_ragged_shapes(config, M, N, K):
    W, X = ti.small_fp16(seed=M * 7 + N + K, M=M, K=K, N=N, B=2)
    Y = _run(W, X, config=config)
    assert oracle.rel_frobenius(Y, oracle.cgemm(W, X)) <= TOL


@pytest.mark.parametrize("config", [0, 1])
@pytest.mark.parametrize("K,N", [(300, 300), (5000, 300), (5000, 301)])
def test_stacked_equals_four_mma_kernel_bit_for_bit(K, N, config):
    """Odd N stores Y from registers (no TMA store, so no split of the last
    wave); promoted long K then runs on the alternating accumulators alone."""
    W, _ = ti.small_fp16(seed=K, M=260, K=K, N=8, B=2)
    X = ti.complex_gaussian_fp16(ti.rng(K + 1), (4, K, N))
    Ys = _run(W, X, stacked=True, config=config)
    Y0 = _run(W, X, stacked=False)
    assert np.array_equal(Ys, Y0)
    assert oracle.rel_frobenius(Ys, oracle.cgemm(W, X)) <= TOL


@pytest.mark.parametrize("config", [0, 1])
def test_stacked_integer_inputs_bit_exact(config):
    g = ti.rng(1)
    W = ti.integer_complex_fp16(g, (2, 150, 300))
    X = ti.integer_complex_fp16(g, (4, 300, 270))
    assert np.array_equal(_run(W, X, config=config), oracle.cgemm(W, X))


def test_stacked_identity_and_imaginary_identity():
    K, N = 96, 200
    _, X = ti.small_fp16(seed=5, M=1, K=K, N=N)
    Xc = X[..., 0].astype(np.float64) + 1j * X[..., 1].astype(np.float64)
    for part, factor in ((0, 1.0), (1, 1j)):
        W = np.zeros((1, K, K, 2), np.float16)
        W[0, np.arange(K), np.arange(K), part] = 1.0
        assert np.array_equal(_run(W, X), factor * Xc)


@pytest.mark.parametrize("config", [0, 1])
@pytest.mark.parametrize("K", [8192, 16384])
def test_stacked_long_k_within_tolerance(K, config):
    W, _ = ti.small_fp16(seed=K, M=256, K=K, N=8)
    X = ti.complex_gaussian_fp16(ti.rng(K), (1, K, 256))
    assert oracle.rel_frobenius(_run(W, X, config=config), oracle.cgemm(W, X)) <= TOL


def _pair_split(B, M, N, K, pairs=76):
    """The SM-pair kernel's split of its last wave (host rule, for the test
    shapes below): (tail tiles, parts per tail tile) or None.  K above 4096 is
    summed in chunks of 2048; the r tiles of a partial last wave run as
    min(chunks, pairs // r) units of whole chunks each."""
    tiles = (M + 255) // 256 * ((N + 127) // 128) * B
    chunks = (K + 2047) // 2048 if K > 4096 else 1
    r = tiles % pairs
    if chunks < 2 or r == 0 or min(chunks, pairs // r) < 2:
        return None
    return r, min(chunks, pairs // r)


@pytest.mark.parametrize("B,M,N,K", [(1, 1024, 1024, 8192), (3, 300, 200, 5000),
                                     (1, 2052, 2052, 4100)])
def test_stacked_pair_split_last_wave_bit_for_bit(B, M, N, K):
    """Tiles of a partial last wave run as parts of whole accumulation chunks
    on the idle SM pairs, the later chunks added by a second kernel in chunk
    order: the same bits as the one-SM kernel (which runs every tile whole),
    the same bits on a second call, and within the bar of the oracle at
    points of the split tiles."""
    import torch
    from gpu_util import dev, empty_bytes
    from paper_2505_03269_gb300 import FLAG_STACKED_X, MODE_FP16, Plan
    props = torch.cuda.get_device_properties(0)
    if props.multi_processor_count == 152:
        assert _pair_split(B, M, N, K) is not None
    W, _ = ti.small_fp16(seed=K + M, M=M, K=K, N=8)
    X = ti.complex_gaussian_fp16(ti.rng(K + N), (B, K, N))
    with Plan(B, M, N, K, MODE_FP16, w_batches=1, flags=FLAG_STACKED_X) as plan:
        Wp = empty_bytes(plan.packed_size(0))
        Xp = empty_bytes(plan.packed_size(1))
        plan.transpose_pack(0, dev(W), Wp)
        plan.transpose_pack(1, dev(X), Xp)
        outs = []
        for config in (0, 0, 1):
            plan.set_config(config)
            Y = torch.full((B, M, N, 2), float("nan"), dtype=torch.float32, device="cuda")
            plan.beamform_fp16(Wp, Xp, Y)
            torch.cuda.synchronize()
            assert plan.last_device_error() == 0
            outs.append(Y.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])
    # points in the last tiles of the tile order (the last batch's last
    # sample tiles and rows), against the FP64 oracle
    g = ti.rng(5)
    pts = np.stack([np.full(64, B - 1), g.integers(max(0, M - 300), M, 64),
                    g.integers(max(0, N - 256), N, 64)], axis=1)
    Yc = outs[0][..., 0].astype(np.float64) + 1j * outs[0][..., 1].astype(np.float64)
    got = Yc[pts[:, 0], pts[:, 1], pts[:, 2]]
    want = oracle.cgemm_points(W, X, pts)
    assert np.linalg.norm(got - want) <= TOL * np.linalg.norm(want)


def test_stacked_pair_split_in_a_captured_step():
    """A captured step (pack + split GEMM + the chunk sums) replays to the
    direct launches' bits."""
    import torch
    from gpu_util import dev, empty_bytes
    from paper_2505_03269_gb300 import FLAG_STACKED_X, MODE_FP16, Plan
    B, M, N, K = 1, 1024, 1024, 8192
    W, _ = ti.small_fp16(seed=3, M=M, K=K, N=8)
    X = ti.complex_gaussian_fp16(ti.rng(4), (B, K, N))
    with Plan(B, M, N, K, MODE_FP16, w_batches=1, flags=FLAG_STACKED_X) as plan:
        Wp = empty_bytes(plan.packed_size(0))
        Xp = empty_bytes(plan.packed_size(1))
        Xd = dev(X)
        plan.transpose_pack(0, dev(W), Wp)
        Y = torch.empty((B, M, N, 2), dtype=torch.float32, device="cuda")
        plan.graph_capture(Xd, Xp, Wp, Y)
        plan.graph_launch()
        torch.cuda.synchronize()
        Yg = Y.cpu().numpy().copy()
        plan.transpose_pack(1, Xd, Xp)
        Y.fill_(float("nan"))
        plan.beamform_fp16(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        assert np.array_equal(Y.cpu().numpy(), Yg)


@pytest.mark.parametrize("K", [100, 5000])
def test_stacked_uneven_beam_counts(K):
    """Uneven beam counts run the one-SM stacked tiles (per-batch m-tiles),
    K = 5000 with its promoted chunks on the alternating accumulators."""
    rows = [300, 1, 129]
    W, _ = ti.small_fp16(seed=21, M=300, K=K, N=8, B=3)
    X = ti.complex_gaussian_fp16(ti.rng(22), (3, K, 200))
    Y = _run(W, X, rows=rows)
    Yref = oracle.cgemm(W, X)
    for b, r in enumerate(rows):
        assert oracle.rel_frobenius(Y[b, :r], Yref[b, :r]) <= TOL


def test_stacked_host_pipeline():
    import torch
    from gpu_util import dev, empty_bytes
    from paper_2505_03269_gb300 import FLAG_STACKED_X, MODE_FP16, Plan
    W, X = ti.small_fp16(seed=9, M=130, K=150, N=260, B=6)
    W = np.ascontiguousarray(W[:3])
    Yd = _run(W, X)
    with Plan(6, 130, 260, 150, MODE_FP16, w_batches=3, flags=FLAG_STACKED_X) as plan:
        Wp = empty_bytes(plan.packed_size(0))
        plan.transpose_pack(0, dev(W), Wp)
        Xh = torch.from_numpy(X).pin_memory()
        Yh = torch.empty((6, 130, 260, 2), dtype=torch.float32).pin_memory()
        s = torch.cuda.Stream()
        plan.beamform_host(Xh, Wp, Yh, chunk=2, stream=s)
        s.synchronize()
        assert plan.last_device_error() == 0
    Yn = Yh.numpy().astype(np.float64)
    assert np.array_equal(Yn[..., 0] + 1j * Yn[..., 1], Yd)


@pytest.mark.parametrize("B,M,N,K", [(1, 600, 300, 5000), (4, 300, 260, 4500)])
def test_stacked_host_pipeline_long_k(B, M, N, K):
    """tcbf_beamform_host with promoted long K on stacked planes: its
    sub-plans (row ranges of W, or chunks of batches) may split their last
    wave with the plan's chunk workspace, one after the other on one
    stream; the result equals the device-resident call bit for bit."""
    import torch
    from gpu_util import dev, empty_bytes
    from paper_2505_03269_gb300 import FLAG_STACKED_X, MODE_FP16, Plan
    W, _ = ti.small_fp16(seed=M + K, M=M, K=K, N=8)
    X = ti.complex_gaussian_fp16(ti.rng(N + K), (B, K, N))
    Yd = _run(W, X)
    with Plan(B, M, N, K, MODE_FP16, w_batches=1, flags=FLAG_STACKED_X) as plan:
        Wp = empty_bytes(plan.packed_size(0))
        plan.transpose_pack(0, dev(W), Wp)
        Xh = torch.from_numpy(X).pin_memory()
        Yh = torch.empty((B, M, N, 2), dtype=torch.float32).pin_memory()
        s = torch.cuda.Stream()
        plan.beamform_host(Xh, Wp, Yh, stream=s)
        s.synchronize()
        assert plan.last_device_error() == 0
    Yn = Yh.numpy().astype(np.float64)
    assert np.array_equal(Yn[..., 0] + 1j * Yn[..., 1], Yd)


def _auto_threshold():
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "tcbf.h")).read()
    return float(re.search(r"#define TCBF_AUTO_STACKED_MIN_INTENSITY (\d+)", hdr).group(1))


def _intensity(B, Bw, M, N, K):
    """8 B M N K operations over the bytes of the stacked layout: packed W
    (2 planes), packed X (3 planes), both padded to K rounded up to 64, and
    the complex64 output."""
    Kp = (K + 63) // 64 * 64
    return 8.0 * B * M * N * K / (2 * 2 * Bw * M * Kp + 3 * 2 * B * N * Kp + 8 * B * M * N)


@pytest.mark.parametrize("B,Bw,M,N,K", [(1, 1, 4096, 4096, 4096), (1, 1, 8192, 8192, 8192),
                                        (512, 256, 1024, 4096, 288), (1, 1, 256, 256, 256),
                                        (1, 1, 1024, 1024, 4096), (1, 1, 1024, 1024, 2048),
                                        (64, 64, 65536 // 64, 128, 16384)])
def test_auto_layout_follows_the_intensity(B, Bw, M, N, K):
    """TCBF_FLAG_AUTO_LAYOUT resolves to the stacked layout exactly when the
    shape's operations per byte reach the documented threshold."""
    from paper_2505_03269_gb300 import FLAG_AUTO_LAYOUT, FLAG_STACKED_X, MODE_FP16, Plan
    with Plan(B, M, N, K, MODE_FP16, w_batches=Bw, flags=FLAG_AUTO_LAYOUT) as plan:
        want = FLAG_STACKED_X if _intensity(B, Bw, M, N, K) >= _auto_threshold() else 0
        assert plan.flags == want
        Kp = (K + 63) // 64 * 64
        assert plan.packed_size(1) == (3 if want else 2) * B * N * Kp * 2


def test_auto_layout_plan_computes_the_stacked_product():
    """An auto-layout plan on a compute-bound shape packs and multiplies as
    the stacked plan does (bit for bit), and matches the oracle."""
    import torch
    from gpu_util import dev, empty_bytes
    from paper_2505_03269_gb300 import FLAG_AUTO_LAYOUT, FLAG_STACKED_X, MODE_FP16, Plan
    M, N, K = 1024, 1024, 4096
    assert _intensity(1, 1, M, N, K) >= _auto_threshold()
    W, X = ti.small_fp16(seed=77, M=M, K=K, N=N, B=1)
    with Plan(1, M, N, K, MODE_FP16, flags=FLAG_AUTO_LAYOUT) as plan:
        assert plan.flags == FLAG_STACKED_X
        Wp = empty_bytes(plan.packed_size(0))
        Xp = empty_bytes(plan.packed_size(1))
        Y = torch.full((1, M, N, 2), float("nan"), dtype=torch.float32, device="cuda")
        plan.transpose_pack(0, dev(W), Wp)
        plan.transpose_pack(1, dev(X), Xp)
        plan.beamform_fp16(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        Yh = Y.cpu().numpy().astype(np.float64)
    got = Yh[..., 0] + 1j * Yh[..., 1]
    assert np.array_equal(got, _run(W, X, stacked=True))
    rows = slice(0, 96)
    ref = oracle.cgemm(W[:, rows], X)
    assert oracle.rel_frobenius(got[:, rows], ref) <= TOL


def test_autotune_layout_picks_a_timed_layout_and_stays_correct():
    """tcbf_autotune_layout times the planar, stacked and interleaved steps
    and keeps the fastest with its tuned configuration; it refuses plans made
    without the auto flag, and after repacking X for the chosen layout the
    plan's product is within the FP16 bar of the oracle."""
    import torch
    from gpu_util import dev, empty_bytes
    from paper_2505_03269_gb300 import (FLAG_AUTO_LAYOUT, FLAG_INTERLEAVED_X, FLAG_STACKED_X,
                                        MODE_FP16, Plan, TcbfError)
    B, M, N, K = 2, 384, 320, 1000
    W, X = ti.small_fp16(seed=5, M=M, K=K, N=N, B=B)
    Wd, Xd = dev(W), dev(X)
    with Plan(B, M, N, K, MODE_FP16, flags=0) as fixed:
        Wp = empty_bytes(fixed.packed_size(0))
        Y = torch.empty((B, M, N, 2), dtype=torch.float32, device="cuda")
        fixed.transpose_pack(0, Wd, Wp)
        with pytest.raises(TcbfError):          # not an auto-layout plan
            fixed.autotune_layout(Wp, Xd, Y)
    with Plan(B, M, N, K, MODE_FP16, flags=FLAG_AUTO_LAYOUT) as plan:
        flags, ms = plan.autotune_layout(Wp, Xd, Y, reps=2)
        layouts = (0, FLAG_STACKED_X, FLAG_INTERLEAVED_X)
        assert flags in layouts and plan.flags == flags
        assert all(t > 0 for t in ms)
        assert flags == layouts[int(np.argmin(ms))]
        Xp = empty_bytes(plan.packed_size(1))
        plan.transpose_pack(1, Xd, Xp)
        Y.fill_(float("nan"))
        plan.beamform_fp16(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        Yh = Y.cpu().numpy().astype(np.float64)
    got = Yh[..., 0] + 1j * Yh[..., 1]
    assert oracle.rel_frobenius(got, oracle.cgemm(W, X)) <= TOL


def test_autotune_layout_skips_interleaved_when_n_is_not_a_multiple_of_four():
    """Rows of 4N bytes that are not 16-byte multiples: the fused
    interleaved kernel cannot read X, so only planar and stacked are timed."""
    import torch
    from gpu_util import dev, empty_bytes
    from paper_2505_03269_gb300 import FLAG_AUTO_LAYOUT, FLAG_STACKED_X, MODE_FP16, Plan
    W, X = ti.small_fp16(seed=8, M=128, K=64, N=130, B=1)
    with Plan(1, 128, 130, 64, MODE_FP16, flags=FLAG_AUTO_LAYOUT) as plan:
        Wp = empty_bytes(plan.packed_size(0))
        plan.transpose_pack(0, dev(W), Wp)
        Y = torch.empty((1, 128, 130, 2), dtype=torch.float32, device="cuda")
        flags, ms = plan.autotune_layout(Wp, dev(X), Y, reps=1)
        assert ms[2] == -1 and ms[0] > 0 and ms[1] > 0
        assert flags in (0, FLAG_STACKED_X)


def test_autotune_layout_then_host_pipeline():
    """A layout change releases the plan's host-pipeline staging (sized for
    the old layout): the end-to-end call made before and after the tuner
    both match the oracle."""
    import torch
    from gpu_util import dev, empty_bytes
    from paper_2505_03269_gb300 import FLAG_AUTO_LAYOUT, MODE_FP16, Plan
    B, M, N, K = 4, 200, 256, 288
    W, X = ti.small_fp16(seed=31, M=M, K=K, N=N, B=B)
    ref = oracle.cgemm(W, X)
    with Plan(B, M, N, K, MODE_FP16, flags=FLAG_AUTO_LAYOUT) as plan:
        Wp = empty_bytes(plan.packed_size(0))
        plan.transpose_pack(0, dev(W), Wp)
        Xh = torch.from_numpy(X).pin_memory()
        for tune in (False, True):
            if tune:
                Y = torch.empty((B, M, N, 2), dtype=torch.float32, device="cuda")
                plan.autotune_layout(Wp, dev(X), Y, reps=1)
            Yh = torch.full((B, M, N, 2), float("nan"), dtype=torch.float32).pin_memory()
            plan.beamform_host(Xh, Wp, Yh, chunk=2)
            torch.cuda.synchronize()
            assert plan.last_device_error() == 0
            y = Yh.numpy().astype(np.float64)
            assert oracle.rel_frobenius(y[..., 0] + 1j * y[..., 1], ref) <= TOL
