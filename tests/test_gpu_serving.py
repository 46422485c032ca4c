"""Continuous-batching server: every request's result is the same alone and
in the mix (bit for bit: each runs the same kernels and tile configuration),
admission respects the HBM budget and arrival times, oversize requests are
rejected, and a served FP16 result matches the FP64 oracle."""
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


SETS = [(100, 64), (300, 200), (257, 129), (64, 300)]


def _alone(mode, W, X):
    """The same request through a plan: pack X, beamform."""
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_1BIT, MODE_FP8SPLIT, Plan
    _, M, K, _ = W.shape
    _, _, N, _ = X.shape
    with Plan(1, M, N, K, mode) as plan:
        Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
        Xp = torch.empty(plan.packed_size(1), dtype=torch.uint8, device="cuda")
        plan.transpose_pack(0, dev(W), Wp)
        plan.transpose_pack(1, dev(X), Xp)
        Y = torch.empty((1, M, N, 2), dtype=torch.int32 if mode == MODE_1BIT else torch.float32,
                        device="cuda")
        {MODE_1BIT: plan.beamform_1bit, MODE_FP8SPLIT: plan.beamform_fp8split}.get(
            mode, plan.beamform_fp16)(Wp, Xp, Y)
        torch.cuda.synchronize()
        return Y.cpu().numpy()[0].view(np.uint32)


def test_alone_equals_in_mix_and_budget_respected():
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_1BIT, MODE_FP8SPLIT, MODE_FP16, Plan
    from paper_2505_03269_gb300.serve import Server
    modes = [MODE_FP16, MODE_FP8SPLIT, MODE_1BIT]
    Ws = [ti.small_fp16(seed=50 + i, M=m, K=k, N=1)[0] for i, (m, k) in enumerate(SETS)]
    g = np.random.default_rng(5)
    reqs = []
    for i in range(18):
        sid = int(g.integers(len(SETS)))
        mode = modes[i % 3]
        N = int(g.integers(100, 2000))
        X = ti.complex_gaussian_fp16(ti.rng(100 + i), (1, SETS[sid][1], N))
        reqs.append((sid, mode, N, X))
    arena = 24 << 20          # small: forces queueing
    keep = []
    with Server(arena, num_streams=4) as srv:
        for sid, (M, K) in enumerate(SETS):
            for mode in modes:
                with Plan(1, M, 1, K, mode) as plan:
                    Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
                    plan.transpose_pack(0, dev(Ws[sid]), Wp)
                srv.register_weights(sid, mode, M, K, Wp)
                keep.append(Wp)
        torch.cuda.synchronize()
        outs, tickets = [], []
        for sid, mode, N, X in reqs:
            hx = torch.from_numpy(X[0]).pin_memory()
            hy = torch.zeros((SETS[sid][0], N, 2), dtype=torch.float32).pin_memory()
            outs.append((hx, hy))
            tickets.append(srv.submit(sid, mode, N, hx, hy))
        srv.start()
        srv.wait_all(120)
        res = [srv.result(t) for t in tickets]
        cnt = srv.counters()
    assert all(r.status == 0 for r in res)
    assert cnt.peak_arena_bytes <= arena and cnt.peak_inflight >= 2
    for (sid, mode, N, X), (hx, hy) in zip(reqs, outs):
        served = hy.numpy().view(np.uint32)
        assert np.array_equal(served, _alone(mode, Ws[sid], X))
        if mode == MODE_FP16:
            Y = hy.numpy().astype(np.float64)
            ref = oracle.cgemm(Ws[sid], X)[0]
            assert oracle.rel_frobenius(Y[..., 0] + 1j * Y[..., 1], ref) <= 2e-5


def test_arrivals_respected_and_oversize_rejected():
    import torch
    from gpu_util import dev
    from paper_2505_03269_gb300 import MODE_FP16, Plan, TcbfError
    from paper_2505_03269_gb300.serve import Server
    M, K, N = 128, 64, 512
    W = ti.small_fp16(seed=7, M=M, K=K, N=1)[0]
    X = ti.complex_gaussian_fp16(ti.rng(8), (K, N))
    with Server(8 << 20, num_streams=2) as srv:
        with Plan(1, M, 1, K, MODE_FP16) as plan:
            Wp = torch.empty(plan.packed_size(0), dtype=torch.uint8, device="cuda")
            plan.transpose_pack(0, dev(W), Wp)
        srv.register_weights(0, MODE_FP16, M, K, Wp)
        torch.cuda.synchronize()
        hx = torch.from_numpy(X).pin_memory()
        with pytest.raises(TcbfError):               # buffers larger than the whole arena
            srv.submit(0, MODE_FP16, 200000, hx)
        with pytest.raises(TcbfError):               # unknown weight set
            srv.submit(3, MODE_FP16, N, hx)
        ts = [srv.submit(0, MODE_FP16, N, hx, arrival_s=0.02 * i) for i in range(6)]
        srv.start()
        srv.wait_all(60)
        for t in ts:
            r = srv.result(t)
            assert r.status == 0 and r.admit_s >= r.arrival_s and r.done_s >= r.admit_s
