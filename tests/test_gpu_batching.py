"""Persistent batched launch: uneven beam counts per batch in one launch,
bit-identical results across tile configurations, the autotuner and its
cache, and CUDA-graph capture of a whole step."""
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


def _setup_fp16(W, X):
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_FP16, Plan
    Bw, M, K, _ = W.shape
    B, _, N, _ = X.shape
    plan = Plan(B, M, N, K, MODE_FP16, w_batches=Bw)
    Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
    Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
    Xd = dev(X)
    plan.transpose_pack(0, dev(W), Wp)
    plan.transpose_pack(1, Xd, Xp)
    Y = torch.full((B, M, N, 2), float("nan"), dtype=torch.float32, device="cuda")
    return plan, Wp, Xd, Xp, Y


def _c(Y):
    Yh = Y.cpu().numpy().astype(np.float64)
    return Yh[..., 0] + 1j * Yh[..., 1]


@pytest.mark.parametrize("K", [100, 5000])
@pytest.mark.parametrize("config", [0, 3])
def test_uneven_beam_counts_one_launch(config, K):
    import torch
    rows = [300, 1, 129, 128, 257]
    B, M, N = len(rows), max(rows), 200
    W, _ = ti.small_fp16(seed=21, M=M, K=K, N=8, B=B)
    X = ti.complex_gaussian_fp16(ti.rng(22), (B, K, N))
    plan, Wp, Xd, Xp, Y = _setup_fp16(W, X)
    with plan:
        plan.set_config(config)
        plan.set_batch_rows(rows)
        plan.beamform_fp16(Wp, Xp, Y)
        torch.cuda.synchronize()
        assert plan.last_device_error() == 0
        Yg = _c(Y)
    Yref = oracle.cgemm(W, X)
    for b, r in enumerate(rows):
        assert oracle.rel_frobenius(Yg[b, :r], Yref[b, :r]) <= TOL
        untouched = Yg[b, (r + 127) // 128 * 128:]
        assert np.all(np.isnan(untouched.real))


# config 5 (4-bit tensor path) cannot walk uneven batches and runs config 0
@pytest.mark.parametrize("config", [0, 4, 5])
def test_uneven_beam_counts_1bit(config):
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_1BIT, Plan
    rows = [5, 256, 130]
    B, M, N, K = 3, 256, 300, 200
    Wb, Xb = ti.onebit_block(seed=23, B=B, M=M, K=K, N=N)
    with Plan(B, M, N, K, MODE_1BIT) as plan:
        plan.set_config(config)
        plan.set_batch_rows(rows)
        Y = torch.full((B, M, N, 2), -999, dtype=torch.int32, device="cuda")
        plan.beamform_1bit(dev(Wb), dev(Xb), Y)
        torch.cuda.synchronize()
        Yg = Y.cpu().numpy().astype(np.int64)
    Yref = oracle.bgemm(Wb, Xb, K)
    for b, r in enumerate(rows):
        assert np.array_equal(Yg[b, :r], Yref[b, :r])
        assert np.all(Yg[b, (r + 127) // 128 * 128:] == -999)


def test_all_configurations_bit_identical():
    """Every tile configuration accumulates each output over K in the same
    order, so the FP16 results agree bit for bit (the same holds for 1-bit)."""
    import torch
    W, X = ti.small_fp16(seed=24, M=300, K=350, N=520, B=2)
    plan, Wp, Xd, Xp, Y = _setup_fp16(W, X)
    outs = []
    with plan:
        for c in range(plan.num_configs()):
            plan.set_config(c)
            plan.beamform_fp16(Wp, Xp, Y)
            torch.cuda.synchronize()
            outs.append(Y.cpu().numpy().copy())
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))
    assert oracle.rel_frobenius(_c(torch.from_numpy(outs[0])), oracle.cgemm(W, X)) <= TOL


def test_autotune_and_cache(tmp_path):
    import torch
    from paper_2505_03269_gb300 import tuner
    W, X = ti.small_fp16(seed=25, M=256, K=5000, N=256, B=1)
    plan, Wp, Xd, Xp, Y = _setup_fp16(W, X)
    with plan:
        best, ms = plan.autotune(Wp, Xp, Y, reps=2)
        assert plan.get_config() == best
        assert ms[best] > 0 and ms[best] == min(t for t in ms if t > 0)
        assert ms[1] == -1.0 and ms[4] == -1.0       # BN=256 tiles are not valid at K > 4096
        torch.cuda.synchronize()
        assert oracle.rel_frobenius(_c(Y), oracle.cgemm(W, X)) <= TOL
        path = str(tmp_path / "tuning.json")
        entry = tuner.tune(plan, Wp, Xp, Y, reps=1, path=path)
        plan.set_config(0 if entry["config"] != 0 else 2)
        again = tuner.tune_or_load(plan, Wp, Xp, Y, path=path)
        assert again["cached"] and plan.get_config() == entry["config"]


def test_graph_capture_replays_the_step():
    import torch
    W, X = ti.small_fp16(seed=26, M=256, K=288, N=1024, B=4)
    plan, Wp, Xd, Xp, Y = _setup_fp16(W, X)
    with plan:
        plan.graph_capture(Xd, Xp, Wp, Y)
        plan.graph_launch()
        torch.cuda.synchronize()
        Y1 = Y.cpu().numpy().copy()
        assert oracle.rel_frobenius(_c(torch.from_numpy(Y1)), oracle.cgemm(W, X)) <= TOL
        # new samples in the same buffer: the replay packs and beamforms them
        X2 = ti.complex_gaussian_fp16(ti.rng(27), X.shape[:3])
        Xd.copy_(torch.from_numpy(X2).cuda())
        plan.graph_launch()
        torch.cuda.synchronize()
        assert oracle.rel_frobenius(_c(Y), oracle.cgemm(W, X2)) <= TOL
        # and equals the direct launches bit for bit
        plan.transpose_pack(1, Xd, Xp)
        Yd = torch.empty_like(Y)
        plan.beamform_fp16(Wp, Xp, Yd)
        torch.cuda.synchronize()
        assert torch.equal(Y.view(torch.int32), Yd.view(torch.int32))
