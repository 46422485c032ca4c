"""Host-side logic of the serving stream (no GPU): the seeded weight-set and
request generators follow the stated distributions and mix."""
import numpy as np

from paper_2505_03269_gb300 import MODE_1BIT, MODE_FP8SPLIT, MODE_FP16
from paper_2505_03269_gb300 import serve


def test_weight_sets_log_uniform_bounds_and_seeded():
    a = serve.make_weight_sets(seed=0)
    assert a == serve.make_weight_sets(seed=0) and len(a) == 32
    assert all(64 <= m <= 4096 and 64 <= k <= 2048 for m, k in a)


def test_request_stream_distribution():
    reqs = serve.make_stream(seed=1, n_requests=20000)
    N = np.array([r["N"] for r in reqs])
    assert N.min() >= 256 and N.max() <= 8192
    # log-uniform: the median sits near the geometric mean of the bounds
    assert abs(np.log(np.median(N)) - 0.5 * (np.log(256) + np.log(8193))) < 0.05
    modes = np.array([r["mode"] for r in reqs])
    for m, p in ((MODE_FP16, 0.7), (MODE_FP8SPLIT, 0.2), (MODE_1BIT, 0.1)):
        assert abs(np.mean(modes == m) - p) < 0.015
    gaps = np.array([r["gap"] for r in reqs])
    assert abs(gaps.mean() - 1.0) < 0.03          # unit-rate exponential gaps
    assert reqs[:5] == serve.make_stream(seed=1, n_requests=20000)[:5]
