"""Pins for the CPU oracle, against facts that do not come from the oracle.

Each test checks the oracle against something fixed by the paper or by
mathematics: brute force on tiny inputs, a library routine on a special
case, closed forms (identity weights, integer inputs, plane-wave coherent
gain, matched 1-bit conjugate), the paper's worked example (Table II) and
its popcount identities (Eq. 4-6), exhaustive 1-bit enumeration, and
IEEE binary16 decoding against numpy over all 65536 patterns.
"""
import cmath
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from oracle import onebit
import tcbf_inputs as ti

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- binary16
def test_half_decode_exhaustive_against_numpy():
    h = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    mine = oracle.half_to_double(h)
    ref = h.view(np.float16).astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(mine), nan)
    assert np.array_equal(mine[~nan], ref[~nan])
    # signed zero keeps its sign
    assert math.copysign(1.0, mine[0x8000]) == -1.0


# ----------------------------------------------------------- complex GEMM
def _brute(W, X):
    """Eq. 3 with Python complex numbers, no arrays."""
    Bw, M, K = W.shape
    B, _, N = X.shape
    Y = np.zeros((B, M, N), complex)
    for b in range(B):
        for m in range(M):
            for n in range(N):
                s = 0j
                for k in range(K):
                    s += complex(W[b // (B // Bw), m, k]) * complex(X[b, k, n])
                Y[b, m, n] = s
    return Y


@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_cgemm_brute_force_tiny(K):
    g = np.random.default_rng(K)
    B, Bw, M, N = 4, 2, 3, 5
    W = g.standard_normal((Bw, M, K)) + 1j * g.standard_normal((Bw, M, K))
    X = g.standard_normal((B, K, N)) + 1j * g.standard_normal((B, K, N))
    Y = oracle.cgemm(W, X)
    Yb = _brute(W, X)
    assert np.allclose(Y, Yb, rtol=1e-14, atol=1e-14)


def test_cgemm_matches_library_matmul():
    g = np.random.default_rng(7)
    B, M, K, N = 3, 17, 33, 29
    W = g.standard_normal((B, M, K)) + 1j * g.standard_normal((B, M, K))
    X = g.standard_normal((B, K, N)) + 1j * g.standard_normal((B, K, N))
    Y = oracle.cgemm(W, X)
    assert np.allclose(Y, W @ X, rtol=1e-12, atol=1e-12)


def test_cgemm_fp16_path_equals_decoded_fp64_path():
    W, X = ti.small_fp16(seed=3, M=9, K=21, N=13, B=2)
    Y16 = oracle.cgemm(W, X)
    Y64 = oracle.cgemm(W.astype(np.float64), X.astype(np.float64))
    assert np.array_equal(Y16, Y64)


def test_cgemm_points_equal_full():
    W, X = ti.small_fp16(seed=4, M=11, K=37, N=19, B=3)
    Y = oracle.cgemm(W, X)
    g = np.random.default_rng(0)
    pts = np.stack([g.integers(0, 3, 50), g.integers(0, 11, 50), g.integers(0, 19, 50)], 1)
    P = oracle.cgemm_points(W, X, pts)
    assert np.array_equal(P, Y[pts[:, 0], pts[:, 1], pts[:, 2]])


def test_identity_weights_return_x_exactly():
    K, N = 24, 40
    W = np.zeros((1, K, K, 2), np.float16)
    W[0, np.arange(K), np.arange(K), 0] = 1.0
    _, X = ti.small_fp16(seed=1, M=1, K=K, N=N)
    Y = oracle.cgemm(W, X)
    Xc = X[..., 0].astype(np.float64) + 1j * X[..., 1].astype(np.float64)
    assert np.array_equal(Y, Xc)


def test_integer_inputs_exact():
    g = ti.rng(5)
    W = ti.integer_complex_fp16(g, (2, 6, 50))
    X = ti.integer_complex_fp16(g, (2, 50, 7))
    Y = oracle.cgemm(W, X)
    wi = W.astype(np.int64)
    xi = X.astype(np.int64)
    re = wi[..., 0] @ xi[..., 0] - wi[..., 1] @ xi[..., 1]
    im = wi[..., 0] @ xi[..., 1] + wi[..., 1] @ xi[..., 0]
    assert np.array_equal(Y.real, re.astype(np.float64))
    assert np.array_equal(Y.imag, im.astype(np.float64))


def test_batch_weight_sharing():
    g = np.random.default_rng(9)
    B, Bw, M, K, N = 6, 3, 4, 5, 7
    W = g.standard_normal((Bw, M, K)) + 1j * g.standard_normal((Bw, M, K))
    X = g.standard_normal((B, K, N)) + 1j * g.standard_normal((B, K, N))
    Y = oracle.cgemm(W, X)
    for b in range(B):
        assert np.allclose(Y[b], W[b // 2] @ X[b], rtol=1e-13, atol=1e-13)


def test_conjugation_symmetry_and_linearity():
    g = np.random.default_rng(11)
    W = g.standard_normal((1, 5, 6)) + 1j * g.standard_normal((1, 5, 6))
    X = g.standard_normal((1, 6, 4)) + 1j * g.standard_normal((1, 6, 4))
    X2 = g.standard_normal((1, 6, 4)) + 1j * g.standard_normal((1, 6, 4))
    Y = oracle.cgemm(W, X)
    assert np.allclose(oracle.cgemm(W.conj(), X.conj()), Y.conj(), rtol=1e-14, atol=1e-14)
    a = 0.3 - 1.7j
    assert np.allclose(oracle.cgemm(W, a * X + X2), a * Y + oracle.cgemm(W, X2),
                       rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- weights
def test_plane_wave_on_axis_gives_coherent_gain_K():
    """x_k = exp(+2 pi i f tau_k) s; steering the beam at the source gives y = K s."""
    K, f, c = 96, 150e6, ti.SPEED_OF_LIGHT
    g = np.random.default_rng(3)
    pos = np.zeros((K, 3))
    pos[:, 0] = g.uniform(-1000, 1000, K)
    pos[:, 1] = g.uniform(-1000, 1000, K)
    theta = 0.2
    s_dir = np.array([[math.sin(theta), 0.0, math.cos(theta)]])
    w = oracle.weights(pos, s_dir, np.full((1, K), f), False, c)        # [1,1,K]
    tau = pos @ s_dir[0] / c
    s = 0.7 - 0.2j
    x = (np.exp(2j * np.pi * f * tau) * s).reshape(1, K, 1)
    y = oracle.cgemm(w, x)[0, 0, 0]
    assert abs(y - K * s) <= 1e-11 * K


def test_weights_unit_modulus_and_zero_delay():
    geom = ti.radio_geometry(seed=0, n_beams=16, n_stations=12, n_channels=3)
    w = oracle.weights(geom.rx_pos, geom.targets, geom.freqs, False, geom.c)
    assert np.allclose(np.abs(w), 1.0, atol=1e-14)
    # a receiver at the reference point has zero delay: w = 1
    pos = geom.rx_pos.copy()
    pos[0] = 0.0
    w0 = oracle.weights(pos, geom.targets, geom.freqs, False, geom.c)
    assert np.all(w0[:, :, 0] == 1.0)


def test_weights_match_library_exp():
    geom = ti.ultrasound_geometry(n_elements=8, n_bins=4, grid=(3, 2, 4))
    w = oracle.weights(geom.rx_pos, geom.targets, geom.freqs, True, geom.c)
    d = np.linalg.norm(geom.targets[:, None, :] - geom.rx_pos[None, :, :], axis=2)
    ref = np.exp(-2j * np.pi * geom.freqs[0][None, :] * d / geom.c) / d
    assert np.allclose(w[0], ref, rtol=1e-12, atol=0)
    assert np.allclose(np.abs(w[0]), 1.0 / d, rtol=1e-14)


def test_weights_quarter_cycle_large_phase():
    """f tau = n + 1/4 with n ~ 1e6 gives w = -i exactly after FP16 rounding."""
    pos = np.array([[1.0, 0.0, 0.0]])
    tgt = np.array([[1.0, 0.0, 0.0]])
    f = np.array([[1_000_000.25]])
    w16 = oracle.weights_fp16(pos, tgt, f, False, 1.0)
    assert float(w16[0, 0, 0, 0]) == 0.0 and float(w16[0, 0, 0, 1]) == -1.0
    f = np.array([[1_000_000.5]])      # half cycle: w = -1
    w16 = oracle.weights_fp16(pos, tgt, f, False, 1.0)
    assert float(w16[0, 0, 0, 0]) == -1.0 and float(w16[0, 0, 0, 1]) == 0.0


# ----------------------------------------------------------------- 1-bit
def _read_table2():
    rows, scal = [], {}
    with open(os.path.join(GOLDEN, "table2_1bit_dot.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            t = line.split()
            if t[0].isdigit():
                rows.append([int(v) for v in t])
            else:
                scal[t[0]] = int(t[1])
    return rows, scal


def test_table2_worked_example():
    rows, scal = _read_table2()
    K = len(rows)
    a = sum(r[4] << r[0] for r in rows)
    b = sum(r[5] << r[0] for r in rows)
    assert onebit.values(a, K) == [r[1] for r in rows]
    assert onebit.values(b, K) == [r[2] for r in rows]
    assert onebit.popc(a ^ b) == scal["popc"]
    assert onebit.dot_xor(a, b, K) == scal["eq4"] == scal["dot"]
    assert onebit.dot_and(a, b, K) == scal["dot"]
    # through the int64 oracle: imaginary planes all +1 gives
    # Re = A.B - K and Im = sum A + sum B (Sec. III-B product)
    Wb = np.zeros((1, 2, 1, 4), np.uint32)
    Xb = np.zeros((1, 2, 1, 4), np.uint32)
    Wb[0, 0, 0, 0], Wb[0, 1, 0, 0] = a, 0xF
    Xb[0, 0, 0, 0], Xb[0, 1, 0, 0] = b, 0xF
    Y = oracle.bgemm(Wb, Xb, K)
    assert Y[0, 0, 0, 0] == scal["dot"] - K
    assert Y[0, 0, 0, 1] == sum(r[1] for r in rows) + sum(r[2] for r in rows)


def test_eq4_equals_eq6_random():
    g = np.random.default_rng(1)
    for _ in range(2000):
        K = int(g.integers(1, 300))
        a = int(g.integers(0, 2**62)) | (int(g.integers(0, 2**62)) << 62)
        b = int(g.integers(0, 2**62)) | (int(g.integers(0, 2**62)) << 62)
        v = sum(x * y for x, y in zip(onebit.values(a, K), onebit.values(b, K)))
        assert onebit.dot_xor(a, b, K) == v == onebit.dot_and(a, b, K)


@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_bgemm_exhaustive_small_K(K):
    """All 4^K complex 1-bit vectors against all 4^K: the int64 oracle equals
    explicit +-1 complex arithmetic and the paper's Eq. 5 for several pads."""
    n = 4 ** K
    vecs = list(itertools.product(range(1 << K), repeat=2))          # (re bits, im bits)
    Wb = np.zeros((1, 2, n, 4), np.uint32)
    Xb = np.zeros((1, 2, n, 4), np.uint32)
    for i, (r, im) in enumerate(vecs):
        Wb[0, 0, i, 0], Wb[0, 1, i, 0] = r, im
        Xb[0, 0, i, 0], Xb[0, 1, i, 0] = r, im
    Y = oracle.bgemm(Wb, Xb, K)
    vals = [np.array(onebit.values(r, K)) + 1j * np.array(onebit.values(im, K)) for r, im in vecs]
    V = np.array(vals)                                               # [n, K] complex
    ref = V @ V.T                                                    # W rows times X columns
    assert np.array_equal(Y[0, :, :, 0], ref.real.astype(np.int64))
    assert np.array_equal(Y[0, :, :, 1], ref.imag.astype(np.int64))
    g = np.random.default_rng(K)
    for _ in range(300):
        i, j = int(g.integers(n)), int(g.integers(n))
        (ar, ai), (br, bi) = vecs[i], vecs[j]
        for pad in (0, 1, 5, 32 - K, 128 - K):
            assert onebit.complex_dot_padded(ar, ai, br, bi, K, pad) == tuple(Y[0, i, j])


def test_bgemm_matched_conjugate_gives_2K():
    K = 77
    g = ti.rng(2)
    Xb = ti.random_sign_words(g, (1, 2, 5, ti.words_per_row(K)))
    Wb = Xb.copy()
    Wb[:, 1] = ~Wb[:, 1]                 # conj: same real bits, flipped imaginary bits
    Y = oracle.bgemm(Wb, Xb, K)
    assert np.all(np.diagonal(Y[0, :, :, 0]) == 2 * K)
    assert np.all(np.diagonal(Y[0, :, :, 1]) == 0)


def test_bgemm_ignores_bits_beyond_K():
    K = 45
    g = ti.rng(3)
    Wb, Xb = ti.onebit_block(seed=3, B=2, M=6, K=K, N=7)
    Y = oracle.bgemm(Wb, Xb, K)
    kw = Wb.shape[-1]
    keep = np.zeros(kw, np.uint32)
    keep[0] = 0xFFFFFFFF
    keep[1] = (1 << (K - 32)) - 1
    Y2 = oracle.bgemm(Wb & keep, Xb & keep, K)
    assert np.array_equal(Y, Y2)
    # and it equals Python complex arithmetic on the unpacked values
    def unpack(row):
        return np.array([(1 if (int(row[k // 32]) >> (k % 32)) & 1 else -1) for k in range(K)])
    for b in range(2):
        for m in range(6):
            w = unpack(Wb[b, 0, m]) + 1j * unpack(Wb[b, 1, m])
            for n in range(7):
                x = unpack(Xb[b, 0, n]) + 1j * unpack(Xb[b, 1, n])
                y = np.sum(w * x)
                assert (Y[b, m, n, 0], Y[b, m, n, 1]) == (int(y.real), int(y.imag))


def test_pack_signs_definition():
    """Sign convention: +0 and -0 both give +1 (bit 1); any negative value,
    however small, gives -1 (bit 0). Expected bits are tabulated by hand."""
    table = [(0.0, 1), (-0.0, 1), (6e-8, 1), (-6e-8, 0), (65504.0, 1), (-65504.0, 0),
             (np.inf, 1), (-np.inf, 0), (0.5, 1), (-0.5, 0), (3.0, 1), (-2.0, 0)]
    K = 40
    g = np.random.default_rng(4)
    idx = g.integers(0, len(table), (1, 3, K, 2))
    V = np.empty((1, 3, K, 2), np.float16)
    bit = np.empty((1, 3, K, 2), np.int64)
    for i, (v, bt) in enumerate(table):
        V[idx == i] = v
        bit[idx == i] = bt
    Kw = ti.words_per_row(K)
    P = oracle.pack_signs(V, k_is_row=False, Kw=Kw)
    for r in range(3):
        for p in range(2):
            want = [0] * Kw
            for k in range(K):
                want[k // 32] |= int(bit[0, r, k, p]) << (k % 32)
            assert [int(v) for v in P[0, p, r]] == want
    # transposed packing equals packing of the explicit transpose
    T = oracle.pack_signs(np.ascontiguousarray(V.transpose(0, 2, 1, 3)), k_is_row=True, Kw=Kw)
    assert np.array_equal(T, P)


def test_pack_signs_f64_definition():
    """FP64 sign packing: the hand table of bits (values far below the FP16
    range keep their sign: -1e-30 gives bit 0, where rounding to FP16 first
    would give -0 and bit 1), pads beyond K zero, and equality with the FP16
    packer wherever the values are FP16 numbers."""
    table = [(0.0, 1), (-0.0, 1), (1e-30, 1), (-1e-30, 0), (-6e-8, 0), (2.5, 1), (-7.0, 0)]
    K = 70
    g = np.random.default_rng(5)
    idx = g.integers(0, len(table), (2, 3, K, 2))
    vals = np.array([v for v, _ in table])
    bits = np.array([b for _, b in table])
    V = vals[idx[..., 0]] + 1j * vals[idx[..., 1]]
    Kw = ti.words_per_row(K)
    P = oracle.pack_signs_f64(V, Kw)
    assert P.shape == (2, 2, 3, Kw) and P.dtype == np.uint32
    for b in range(2):
        for r in range(3):
            for p in range(2):
                want = [0] * Kw
                for k in range(K):
                    want[k // 32] |= int(bits[idx[b, r, k, p]]) << (k % 32)
                assert [int(v) for v in P[b, p, r]] == want
    # FP16-representable values: the same planes as the FP16 packer
    W16, _ = ti.small_fp16(seed=3, M=5, K=K, N=1, B=2)
    Wc = W16[..., 0].astype(np.float64) + 1j * W16[..., 1].astype(np.float64)
    assert np.array_equal(oracle.pack_signs_f64(Wc, Kw), oracle.pack_signs(W16, False, Kw))


# ----------------------------------------------- block-scaled split FP8 oracle
def test_split_blocks_exponents_are_per_block_maxima():
    """Each 32-k block of a row gets the largest e with amax 2^e <= 448, amax
    over that block's k and both planes only (the last block may be short)."""
    g = np.random.default_rng(11)
    K = 100
    V = (g.standard_normal((3, K, 2)) * np.exp2(g.integers(-6, 7, (3, K, 1)))).astype(np.float16)
    hi, lo, ex = oracle.split_blocks(V)
    assert ex.shape == (3, 4)
    for r in range(3):
        for j in range(4):
            blk = np.abs(V[r, 32 * j: 32 * j + 32].astype(np.float64))
            amax = blk.max()
            e = int(ex[r, j])
            assert amax * 2.0 ** e <= 448.0 < amax * 2.0 ** (e + 1)


def test_split_blocks_exact_for_short_significands():
    """Values with at most 8 significant bits, all within a factor 8 of their
    block's largest (so no part falls into E4M3's subnormal range), split
    exactly: hi + lo / 16 = v 2^e, and the four-product block-scaled GEMM
    equals the FP64 product; with three products the dropped Wl Xl term
    is the only difference."""
    g = np.random.default_rng(12)

    def short(shape):
        m = g.integers(128, 256, shape).astype(np.float64)        # 8-bit significands
        sign = np.where(g.random(shape) < 0.5, -1.0, 1.0)
        ex = g.integers(-2, 1, shape)                              # within a factor 8
        blk = np.repeat(g.integers(-8, 4, shape[:-2] + (shape[-2] // 32 + 1,)), 32, axis=-1)
        blk = blk[..., : shape[-2]][..., None]                     # per-32-k block magnitude
        return (sign * m * np.exp2(ex + blk - 8)).astype(np.float16)
    W = short((2, 5, 70, 2))
    XT = short((4, 9, 70, 2))
    X = np.ascontiguousarray(XT.transpose(0, 2, 1, 3))
    hi, lo, ex = oracle.split_blocks(W.reshape(10, 70, 2))
    e = np.repeat(ex, 32, axis=1)[:, :70][..., None]
    assert np.array_equal(hi + lo / 16.0, W.reshape(10, 70, 2).astype(np.float64) * np.exp2(e))
    exact = oracle.cgemm(W, X)
    assert oracle.rel_frobenius(oracle.cgemm_split_blocks(W, X, products=4), exact) < 1e-15
    Wh, Wl = oracle.unscaled_blocks(W.reshape(10, 70, 2))
    XTh, XTl = oracle.unscaled_blocks(XT.reshape(36, 70, 2))
    Xl = np.ascontiguousarray(XTl.reshape(4, 9, 70, 2).transpose(0, 2, 1, 3))
    three = oracle.cgemm_split_blocks(W, X, products=3)
    assert oracle.rel_frobenius(three + oracle.cgemm(Wl.reshape(2, 5, 70, 2), Xl), exact) < 1e-15


def test_split_blocks_scale_one_block_alone():
    """Scaling one 32-k block of one W row by 2^s changes only that block's
    exponent (by -s), leaves its hi and lo bytes as they were, and scales
    that block's contribution to the product by exactly 2^s."""
    W, X = ti.small_fp16(seed=13, M=4, K=96, N=6, B=1)
    W2 = W.copy()
    W2[0, 2, 32:64] = (W2[0, 2, 32:64].astype(np.float64) * 8.0).astype(np.float16)
    h1, l1, e1 = oracle.split_blocks(W[0])
    h2, l2, e2 = oracle.split_blocks(W2[0])
    assert e2[2, 1] == e1[2, 1] - 3
    mask = np.ones_like(e1, bool)
    mask[2, 1] = False
    assert np.array_equal(e1[mask], e2[mask])
    assert np.array_equal(h1, h2) and np.array_equal(l1, l2)
    Y1 = oracle.cgemm_split_blocks(W, X, products=3)
    Y2 = oracle.cgemm_split_blocks(W2, X, products=3)
    # the block's own contribution, from the same split restricted to k in [32, 64)
    Wb = np.zeros_like(W)
    Wb[0, 2, 32:64] = W[0, 2, 32:64]
    Xb = np.zeros_like(X)
    Xb[:, 32:64] = X[:, 32:64]
    blk = oracle.cgemm_split_blocks(Wb, X, products=3)
    assert np.allclose(Y2, Y1 + 7.0 * blk, rtol=0, atol=1e-12 * np.abs(Y1).max())


def test_split_blocks_single_block_rows_match_row_scales():
    """For K <= 32 a row is one block, so the block exponent equals the
    per-row exponent of the per-row split and the hi parts are the same."""
    W, _ = ti.small_fp16(seed=14, M=7, K=29, N=1, B=1)
    hb, _, eb = oracle.split_blocks(W[0])
    hr, _, er = oracle.split_rows(W[0])
    assert np.array_equal(eb[:, 0], er)
    assert np.array_equal(hb, hr)


# ----------------------------------------------------------- split FP8 oracle
def test_e4m3_rounding_matches_library_cast():
    """Against torch's float8_e4m3fn conversion (round to nearest even) on a
    dense set of values inside the finite range, including every E4M3 value
    and every midpoint between neighbours."""
    torch = pytest.importorskip("torch")
    codes = torch.arange(256, dtype=torch.int32).to(torch.uint8).view(torch.float8_e4m3fn)
    vals = codes.to(torch.float64).numpy()
    vals = np.unique(vals[np.isfinite(vals)])
    mids = (vals[1:] + vals[:-1]) / 2
    g = np.random.default_rng(0)
    rnd = g.uniform(-448, 448, 20000) * np.exp(g.uniform(-12, 0, 20000))
    x = np.concatenate([vals, mids, mids + 1e-9, mids - 1e-9, rnd])
    x = x[np.abs(x) <= 448]
    ref = torch.from_numpy(x).to(torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    # the float32 step may move values within 1e-9 of a midpoint; keep exact ones
    exact = torch.from_numpy(x).to(torch.float32).to(torch.float64).numpy() == x
    assert np.array_equal(oracle.e4m3_round(x[exact]), ref[exact])
    assert oracle.e4m3_round(np.array([449.0, -1e6]))[0] == 448.0


def test_split_exponent_definition():
    for amax in [1e-7, 0.001, 0.99, 1.0, 3.5, 447.9, 448.0, 448.1, 65504.0]:
        e = oracle.split_exponent(amax)
        assert amax * 2.0 ** e <= 448.0 < amax * 2.0 ** (e + 1)
    assert oracle.split_exponent(0.0) == 0


def test_split_is_exact_for_short_significands():
    """Values with at most 8 significant bits (after scaling) are hi + lo exactly."""
    g = np.random.default_rng(1)
    mant = g.integers(128, 256, (3, 40, 2)) * g.choice([-1, 1], (3, 40, 2))
    V = (mant * np.ldexp(1.0, g.integers(-12, -2, (3, 40, 2)))).astype(np.float16)
    hi, lo, e = oracle.split_rows(V)
    back = (hi + lo) * np.ldexp(1.0, -e)[:, None, None]
    assert np.array_equal(back, V.astype(np.float64))


def test_split_four_products_equal_product_of_reconstructions():
    """(Wh + Wl)(Xh + Xl) = WhXh + WhXl + WlXh + WlXl, scaled back."""
    W, X = ti.small_fp16(seed=31, M=7, K=33, N=9, B=2)
    (Wh, Wl, eW), (Xh, Xl, eX) = oracle.split_operands(W, X)
    Wr = (Wh + Wl) * np.ldexp(1.0, -eW)[..., None, None]
    Xr = (Xh + Xl) * np.ldexp(1.0, -eX)[:, None, :, None]
    ref = oracle.cgemm(Wr, Xr)
    Y4 = oracle.cgemm_split(W, X, products=4)
    assert np.allclose(Y4, ref, rtol=1e-13, atol=1e-13)
    # the three-product form differs from it by exactly the dropped Wl Xl term
    Y3 = oracle.cgemm_split(W, X, products=3)
    drop = oracle.cgemm(Wl, Xl) * np.ldexp(1.0, -(eW[:, :, None] + eX[:, None, :]))
    assert np.allclose(Y3 + drop, Y4, rtol=1e-13, atol=1e-13)


def test_split_error_level_on_gaussian_data():
    """Characterises the method's accuracy (no paper value exists): the
    three-product hi+lo split of FP16 data lands near 1e-3 relative."""
    W, X = ti.small_fp16(seed=32, M=32, K=256, N=64)
    err = oracle.rel_frobenius(oracle.cgemm_split(W, X), oracle.cgemm(W, X))
    assert 1e-4 < err < 5e-3


def test_plain_fp8_product_exact_on_four_bit_integers():
    """Integers in [-8, 8] have at most four significant bits, so after the
    per-row power-of-two scale they are exact E4M3 values: the lo parts are
    zero and the one-product (plain FP8) form equals the exact product."""
    g = ti.rng(33)
    W = ti.integer_complex_fp16(g, (2, 12, 40))
    X = ti.integer_complex_fp16(g, (2, 40, 10))
    (_, Wl, _), (_, Xl, _) = oracle.split_operands(W, X)
    assert not Wl.any() and not Xl.any()
    exact = oracle.cgemm(W, X)
    for products in (1, 3, 4):
        assert np.array_equal(oracle.cgemm_split(W, X, products=products), exact)


def test_plain_fp8_error_level_on_gaussian_data():
    """The one-product form keeps E4M3's 3 fraction bits per operand: on
    Gaussian data its error sits at the few-percent level, well above the
    three-product split's (no paper value exists for either)."""
    W, X = ti.small_fp16(seed=34, M=32, K=256, N=64)
    exact = oracle.cgemm(W, X)
    e1 = oracle.rel_frobenius(oracle.cgemm_split(W, X, products=1), exact)
    e3 = oracle.rel_frobenius(oracle.cgemm_split(W, X, products=3), exact)
    assert 5e-3 < e1 < 1e-1
    assert e3 < e1 / 5
    with pytest.raises(ValueError):
        oracle.cgemm_split(W, X, products=2)


def test_unpack_signs_table2_and_round_trip():
    """Unpacking follows Fig. 1: Table II's binary columns read back as its
    decimal columns; and unpack(pack(v)) is the sign quantisation of v
    (v >= 0 -> +1, so -0 -> +1), for ragged K on both layouts."""
    rows, _ = _read_table2()
    a_bits = sum(int(r[4]) << i for i, r in enumerate(rows))
    b_bits = sum(int(r[5]) << i for i, r in enumerate(rows))
    P = np.array([a_bits, b_bits], np.uint32).reshape(1, 2, 1, 1)     # re plane = A, im plane = B
    U = oracle.unpack_signs(np.concatenate([P, np.zeros((1, 2, 1, 3), np.uint32)], -1), 4, False)
    assert U[0, 0, :, 0].tolist() == [float(r[1]) for r in rows]
    assert U[0, 0, :, 1].tolist() == [float(r[2]) for r in rows]
    g = ti.rng(8)
    for K in (1, 31, 33, 130):
        V = ti.complex_gaussian_fp16(g, (2, 5, K))
        V.reshape(-1)[:2] = np.array([0.0, -0.0], np.float16)
        want = np.where(V.astype(np.float64) >= 0, 1.0, -1.0)
        kw = ti.words_per_row(K)
        assert np.array_equal(oracle.unpack_signs(oracle.pack_signs(V, False, kw), K, False), want)
        X = ti.complex_gaussian_fp16(g, (2, K, 7))
        wantx = np.where(X.astype(np.float64) >= 0, 1.0, -1.0)
        assert np.array_equal(oracle.unpack_signs(oracle.pack_signs(X, True, kw), K, True), wantx)


def _tf32_exact(v: float) -> float:
    """Brute force with exact rationals: the TF32 neighbours of v (the grid of
    11 significant bits, subnormal step 2^-136) and the nearer one, ties to the
    even significand, overflow past the largest TF32 value to infinity."""
    from fractions import Fraction
    import math
    if not math.isfinite(v) or v == 0.0:
        return v
    f = Fraction(v)
    a = abs(f)
    e = math.floor(math.log2(a))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    q = Fraction(2) ** (max(e, -126) - 10)
    lo = (a // q) * q
    hi = lo + q
    if a - lo < hi - a:
        r = lo
    elif hi - a < a - lo:
        r = hi
    else:
        r = lo if (lo / q) % 2 == 0 else hi
    if r > Fraction(oracle.TF32_MAX):
        return math.copysign(math.inf, v)
    return math.copysign(float(r), v)


def test_round_tf32_against_exact_rationals():
    g = np.random.default_rng(12)
    bits = g.integers(0, 2 ** 32, 3000, dtype=np.uint64).astype(np.uint32)
    # ties (dropped bits exactly 0x1000) with both kept-bit parities, values just
    # off the tie, subnormals, the largest finite values and zero
    ties = (g.integers(0, 2 ** 19, 200, dtype=np.uint64).astype(np.uint32) << 13) | 0x1000
    near = ties ^ 1
    sub = g.integers(1, 2 ** 23, 100, dtype=np.uint64).astype(np.uint32)
    big = np.array([0x7f7fffff, 0x7f7ff000, 0x7f7fefff, 0xff7fffff, 0x00000000, 0x80000000],
                   np.uint32)
    x = np.concatenate([bits, ties, near, sub, big]).view(np.float32)
    x = x[np.isfinite(x)]
    got = oracle.round_tf32(x)
    want = np.array([_tf32_exact(float(v)) for v in x.astype(np.float64)])
    assert np.array_equal(got, want)
    # every result is representable: its FP32 pattern has the 13 low bits zero
    fin = np.isfinite(got)
    assert not np.any(got[fin].astype(np.float32).view(np.uint32) & 0x1fff)
    # FP16 values are TF32 values
    h = g.standard_normal(1000).astype(np.float16).astype(np.float32)
    assert np.array_equal(oracle.round_tf32(h), h.astype(np.float64))
    assert oracle.round_tf32(np.array([np.inf, -np.inf], np.float32)).tolist() == [np.inf, -np.inf]
