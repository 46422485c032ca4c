"""CPU oracle for the tensor-core beamformer (arXiv 2505.03269).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the library.  It shares
no code with the CUDA path.  The arithmetic lives in ``tcbf_oracle.c``
(FP64 / int64 loops, compiled with gcc); this module only builds, loads and
marshals it, plus the paper's 1-bit popcount identities in ``onebit.py``.

Functions and the passages they follow:
  cgemm(W, X)            Eq. 3 with the complex product of Sec. III-B, FP64
  cgemm_points(W, X, p)  Eq. 3 at chosen output points
  bgemm(Wb, Xb, K)       Eq. 3 over 1-bit values of Fig. 1, exact int64
  pack_signs(V, ...)     1-bit sign quantisation, Sec. III-D / Sec. V-A
  pack_signs_f64(V, Kw)  the same quantisation of FP64 values (weights' signs)
  cgemm_split(W, X, p)   split-FP8 product, per-row scales (8-bit floats: Sec. VI)
  cgemm_split_blocks     the same with a scale per 32 K per row / sample
  weights(geom)          w = A exp(-2 pi i f tau), Eq. 1-2
  half_to_double(h)      IEEE binary16 decoding (the FP16 storage format)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tcbf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile tcbf_oracle.c with gcc (OpenMP, no fast-math: IEEE FP64)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_num_threads.argtypes = []
        lib.oracle_half_to_double.restype = ctypes.c_double
        lib.oracle_half_to_double.argtypes = [ctypes.c_uint16]
        lib.oracle_cgemm_f64.argtypes = [i64, i64, i64, i64, i64, p, p, p]
        lib.oracle_cgemm_f16.argtypes = [i64, i64, i64, i64, i64, p, p, p, p, p]
        lib.oracle_cgemm_f16_points.argtypes = [i64, i64, i64, i64, i64, p, p, i64, p, p]
        lib.oracle_bgemm.argtypes = [i64, i64, i64, i64, i64, i64, p, p, p]
        lib.oracle_pack_signs_f16.argtypes = [i64, i64, i64, ctypes.c_int, i64, p, p]
        lib.oracle_weights.argtypes = [i64, i64, i64, p, p, ctypes.c_int, p, ctypes.c_double, p]
        for f in ("oracle_cgemm_f64", "oracle_cgemm_f16", "oracle_cgemm_f16_points",
                  "oracle_bgemm", "oracle_pack_signs_f16", "oracle_weights"):
            getattr(lib, f).restype = None
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def num_threads() -> int:
    """Threads the oracle's OpenMP loops run on."""
    return int(_load().oracle_num_threads())


def half_to_double(h: np.ndarray) -> np.ndarray:
    """Decode binary16 bit patterns (uint16) one by one."""
    lib = _load()
    flat = np.ascontiguousarray(h, dtype=np.uint16).ravel()
    return np.array([lib.oracle_half_to_double(int(v)) for v in flat]).reshape(h.shape)


def _as_complex_pairs_f64(A: np.ndarray) -> np.ndarray:
    if np.iscomplexobj(A):
        out = np.empty(A.shape + (2,), dtype=np.float64)
        out[..., 0] = A.real
        out[..., 1] = A.imag
        return out
    return np.ascontiguousarray(A, dtype=np.float64)


def _to_complex(P: np.ndarray) -> np.ndarray:
    return P[..., 0] + 1j * P[..., 1]


def cgemm(W: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Y[b] = W[b'] X[b] (Eq. 3), FP64, returned as complex128 [B, M, N].

    W: [Bw, M, K, 2] and X: [B, K, N, 2] interleaved pairs, either float16
    (decoded exactly to FP64) or float64; complex arrays are accepted too.
    Batch b uses weight matrix b // (B // Bw)."""
    lib = _load()
    if W.dtype == np.float16 and X.dtype == np.float16:
        Bw, M, K, _ = W.shape
        B, K2, N, _ = X.shape
        assert K == K2 and B % Bw == 0
        Y = np.empty((B, M, N, 2), np.float64)
        wd = np.empty(M * K * 2, np.float64)
        xd = np.empty(K * N * 2, np.float64)
        Wc = np.ascontiguousarray(W).view(np.uint16)
        Xc = np.ascontiguousarray(X).view(np.uint16)
        lib.oracle_cgemm_f16(B, M, N, K, Bw, _ptr(Wc), _ptr(Xc), _ptr(Y), _ptr(wd), _ptr(xd))
        return _to_complex(Y)
    Wd = _as_complex_pairs_f64(W)
    Xd = _as_complex_pairs_f64(X)
    Bw, M, K, _ = Wd.shape
    B, K2, N, _ = Xd.shape
    assert K == K2 and B % Bw == 0
    Y = np.empty((B, M, N, 2), np.float64)
    lib.oracle_cgemm_f64(B, M, N, K, Bw, _ptr(Wd), _ptr(Xd), _ptr(Y))
    return _to_complex(Y)


def cgemm_points(W: np.ndarray, X: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Eq. 3 evaluated only at output points pts [P, 3] = (b, m, n); FP16 inputs."""
    lib = _load()
    assert W.dtype == np.float16 and X.dtype == np.float16
    Bw, M, K, _ = W.shape
    B, _, N, _ = X.shape
    pts = np.ascontiguousarray(pts, dtype=np.int64)
    out = np.empty((len(pts), 2), np.float64)
    Wc = np.ascontiguousarray(W).view(np.uint16)
    Xc = np.ascontiguousarray(X).view(np.uint16)
    lib.oracle_cgemm_f16_points(B, M, N, K, Bw, _ptr(Wc), _ptr(Xc), len(pts), _ptr(pts), _ptr(out))
    return _to_complex(out)


def bgemm(Wb: np.ndarray, Xb: np.ndarray, K: int) -> np.ndarray:
    """Exact 1-bit complex product (Fig. 1 values, Eq. 3), int64 [B, M, N, 2].

    Wb: [Bw, 2, M, Kw] and Xb: [B, 2, N, Kw] uint32 packed planes."""
    lib = _load()
    Bw, _, M, Kw = Wb.shape
    B, _, N, Kw2 = Xb.shape
    assert Kw == Kw2 and B % Bw == 0 and K <= 32 * Kw
    Y = np.empty((B, M, N, 2), np.int64)
    Wc = np.ascontiguousarray(Wb, dtype=np.uint32)
    Xc = np.ascontiguousarray(Xb, dtype=np.uint32)
    lib.oracle_bgemm(B, M, N, K, Bw, Kw, _ptr(Wc), _ptr(Xc), _ptr(Y))
    return Y


def pack_signs(V: np.ndarray, k_is_row: bool, Kw: int) -> np.ndarray:
    """Sign-quantise interleaved complex FP16 V [B, R, C, 2] into packed
    planes [B, 2, rows, Kw].  k_is_row=False packs along C (weights, rows =
    beams); k_is_row=True packs along R and transposes (data, rows = samples)."""
    lib = _load()
    assert V.dtype == np.float16
    B, R, C, _ = V.shape
    rows = C if k_is_row else R
    out = np.empty((B, 2, rows, Kw), np.uint32)
    Vc = np.ascontiguousarray(V).view(np.uint16)
    lib.oracle_pack_signs_f16(B, R, C, int(k_is_row), Kw, _ptr(Vc), _ptr(out))
    return out


def pack_signs_f64(V: np.ndarray, Kw: int) -> np.ndarray:
    """Sign-quantise complex FP64 values V [B, rows, K] (e.g. the steering
    weights of ``weights``) into packed planes [B, 2, rows, Kw] without
    rounding them to FP16 first: bit 1 iff the component is >= 0 (so -0.0
    gives +1), element k in bit k % 32 of word k / 32, zero bits for k >= K
    (Fig. 1; Sec. III-D)."""
    V = np.asarray(V, np.complex128)
    B, rows, K = V.shape
    out = np.zeros((B, 2, rows, Kw * 32), np.uint8)
    out[:, 0, :, :K] = V.real >= 0
    out[:, 1, :, :K] = V.imag >= 0
    packed = np.packbits(out, axis=-1, bitorder="little")          # 4 bytes per word
    return np.ascontiguousarray(packed).view("<u4").reshape(B, 2, rows, Kw)


TF32_MAX = (2.0 - 2.0 ** -10) * 2.0 ** 127


def round_tf32(x: np.ndarray) -> np.ndarray:
    """FP32 values rounded to TF32 (an implicit bit and 10 stored mantissa
    bits over FP32's exponent range): to nearest, ties to the even
    neighbour; beyond the largest TF32 value to +-inf.  Float64 result.
    A value with leading bit 2^e (e >= -126, else the subnormal step) has
    the quantum 2^(e - 10); x / quantum is exact in FP64 and rint rounds it
    half to even."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    out = x.copy()
    fin = np.isfinite(x) & (x != 0)
    _, e2 = np.frexp(x[fin])                    # x = f 2^e2, 0.5 <= |f| < 1
    q = np.ldexp(1.0, np.maximum(e2 - 1, -126) - 10)
    r = np.rint(x[fin] / q) * q
    r = np.where(np.abs(r) > TF32_MAX, np.copysign(np.inf, r), r)
    out[fin] = r
    return out


def unpack_signs(P: np.ndarray, K: int, k_is_row: bool) -> np.ndarray:
    """Packed planes [B, 2, rows, Kw] back to interleaved complex +-1 values
    (Fig. 1: bit 1 is +1, bit 0 is -1; element k is bit k % 32 of word
    k / 32): [B, rows, K, 2] (weights), or transposed to [B, K, rows, 2]
    when k_is_row (data, rows = samples).  Float64."""
    P = np.ascontiguousarray(P, dtype=np.uint32)
    k = np.arange(K)
    bits = (P[..., k // 32] >> (k % 32).astype(np.uint32)) & 1          # [B, 2, rows, K]
    vals = np.where(bits == 1, 1.0, -1.0)
    out = np.moveaxis(vals, 1, -1)                                       # [B, rows, K, 2]
    if k_is_row:
        out = out.transpose(0, 2, 1, 3)
    return np.ascontiguousarray(out)


def weights(rx_pos, targets, freqs, near_field: bool, c: float) -> np.ndarray:
    """w[b,m,k] = A exp(-2 pi i f[b,k] tau[m,k]) in FP64 -> complex128 [Bw, M, K]."""
    lib = _load()
    rx = np.ascontiguousarray(rx_pos, dtype=np.float64)
    tg = np.ascontiguousarray(targets, dtype=np.float64)
    fr = np.ascontiguousarray(freqs, dtype=np.float64)
    K = rx.shape[0]
    M = tg.shape[0]
    Bw = fr.shape[0]
    assert fr.shape[1] == K
    out = np.empty((Bw, M, K, 2), np.float64)
    lib.oracle_weights(Bw, M, K, _ptr(rx), _ptr(tg), int(near_field), _ptr(fr), float(c), _ptr(out))
    return _to_complex(out)


def weights_fp16(rx_pos, targets, freqs, near_field: bool, c: float) -> np.ndarray:
    """The FP64 weights rounded once to FP16 (round-to-nearest-even),
    interleaved [Bw, M, K, 2] — the expected output of the weights kernel."""
    w = weights(rx_pos, targets, freqs, near_field, c)
    out = np.empty(w.shape + (2,), np.float16)
    out[..., 0] = w.real
    out[..., 1] = w.imag
    return out


def rel_frobenius(Y: np.ndarray, Yref: np.ndarray) -> float:
    """||Y - Yref||_F / ||Yref||_F over real and imaginary parts, FP64."""
    d = np.asarray(Y, np.complex128) - np.asarray(Yref, np.complex128)
    return float(np.sqrt(np.sum(np.abs(d) ** 2)) / np.sqrt(np.sum(np.abs(Yref) ** 2)))


# ---------------------------------------------------------------- split FP8
def e4m3_round(v: np.ndarray) -> np.ndarray:
    """Round doubles to E4M3 (nearest, ties to even fraction, saturating at 448)."""
    lib = _load()
    f = lib.oracle_e4m3_round
    f.restype = ctypes.c_double
    f.argtypes = [ctypes.c_double]
    flat = np.asarray(v, np.float64).ravel()
    return np.array([f(float(x)) for x in flat]).reshape(np.shape(v))


def split_exponent(amax: float) -> int:
    lib = _load()
    f = lib.oracle_split_exponent
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_double]
    return int(f(float(amax)))


def split_rows(V16: np.ndarray):
    """V16 [R, K, 2] FP16 rows -> (hi, lo) [R, K, 2] doubles of the scaled
    values and exps [R]: v = (hi + lo) 2^-e approximately."""
    lib = _load()
    f = lib.oracle_split_rows
    f.restype = None
    f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    R, K, _ = V16.shape
    src = np.ascontiguousarray(V16).view(np.uint16)
    hi = np.empty((R, K, 2), np.float64)
    lo = np.empty((R, K, 2), np.float64)
    ex = np.empty(R, np.int32)
    f(R, K, _ptr(src), _ptr(hi), _ptr(lo), _ptr(ex))
    return hi, lo, ex


def split_operands(W16: np.ndarray, X16: np.ndarray):
    """Split W rows (per beam) and X columns (per sample) of FP16 operands.
    Returns (Wh, Wl, eW) with W* [Bw, M, K, 2], eW [Bw, M], and
    (Xh, Xl, eX) with X* [B, K, N, 2], eX [B, N]."""
    Bw, M, K, _ = W16.shape
    B, _, N, _ = X16.shape
    Wh, Wl, eW = split_rows(W16.reshape(Bw * M, K, 2))
    XT = np.ascontiguousarray(X16.transpose(0, 2, 1, 3)).reshape(B * N, K, 2)
    Xh, Xl, eX = split_rows(XT)
    def back(A):
        return np.ascontiguousarray(A.reshape(B, N, K, 2).transpose(0, 2, 1, 3))
    return ((Wh.reshape(Bw, M, K, 2), Wl.reshape(Bw, M, K, 2), eW.reshape(Bw, M)),
            (back(Xh), back(Xl), eX.reshape(B, N)))


def split_blocks(V16: np.ndarray):
    """V16 [R, K, 2] FP16 rows -> (hi, lo, exps): per row and 32-K block the
    exponent e (exps [R, ceil(K/32)]), hi = RN_e4m3(v 2^e) and lo =
    RN_e4m3(16 (v 2^e - hi)) as doubles [R, K, 2], so v ~ (hi + lo / 16) 2^-e."""
    lib = _load()
    f = lib.oracle_split_blocks
    f.restype = None
    f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    R, K, _ = V16.shape
    src = np.ascontiguousarray(V16).view(np.uint16)
    hi = np.empty((R, K, 2), np.float64)
    lo = np.empty((R, K, 2), np.float64)
    ex = np.empty((R, (K + 31) // 32), np.int32)
    f(R, K, _ptr(src), _ptr(hi), _ptr(lo), _ptr(ex))
    return hi, lo, ex


def unscaled_blocks(V16: np.ndarray):
    """The hi and lo parts of split_blocks in their true magnitudes: rows
    [R, K, 2] of hi 2^-e and lo 2^-(e+4), each element with its block's e
    (exact power-of-two scalings of E4M3 values)."""
    hi, lo, ex = split_blocks(V16)
    e = np.repeat(ex, 32, axis=1)[:, : V16.shape[1]][..., None].astype(np.float64)
    return np.ldexp(hi, -e.astype(np.int64)), np.ldexp(lo, -(e + 4).astype(np.int64))


def cgemm_split_blocks(W16: np.ndarray, X16: np.ndarray, products: int = 3) -> np.ndarray:
    """Split-FP8 beamforming with a scale per 32 consecutive k of each W row
    (beam) and each X column (sample) in FP64: with every part taken at its
    true magnitude (Wh, Wl from W's blocks, Xh, Xl from X's),
    Y = Wh Xh + Wh Xl + Wl Xh (products=3), + Wl Xl (4), or Wh Xh alone (the
    plain block-scaled E4M3 product, 1); complex128 [B, M, N]."""
    if products not in (1, 3, 4):
        raise ValueError("products must be 1, 3 or 4")
    Bw, M, K, _ = W16.shape
    B, _, N, _ = X16.shape
    Wh, Wl = unscaled_blocks(W16.reshape(Bw * M, K, 2))
    XT = np.ascontiguousarray(X16.transpose(0, 2, 1, 3)).reshape(B * N, K, 2)
    Xh, Xl = unscaled_blocks(XT)

    def w(A):
        return A.reshape(Bw, M, K, 2)

    def x(A):
        return np.ascontiguousarray(A.reshape(B, N, K, 2).transpose(0, 2, 1, 3))
    Y = cgemm(w(Wh), x(Xh))
    if products >= 3:
        Y = Y + cgemm(w(Wh), x(Xl)) + cgemm(w(Wl), x(Xh))
    if products == 4:
        Y = Y + cgemm(w(Wl), x(Xl))
    return Y


def cgemm_split(W16: np.ndarray, X16: np.ndarray, products: int = 3) -> np.ndarray:
    """Split-FP8 beamforming in FP64: Y = 2^-(eW+eX) (Wh Xh + Wh Xl + Wl Xh)
    (products=3), with Wl Xl added (products=4), or the plain per-row-scaled
    E4M3 product Y = 2^-(eW+eX) Wh Xh (products=1); complex128 [B, M, N]."""
    if products not in (1, 3, 4):
        raise ValueError("products must be 1, 3 or 4")
    (Wh, Wl, eW), (Xh, Xl, eX) = split_operands(W16, X16)
    Y = cgemm(Wh, Xh)
    if products >= 3:
        Y = Y + cgemm(Wh, Xl) + cgemm(Wl, Xh)
    if products == 4:
        Y = Y + cgemm(Wl, Xl)
    B = X16.shape[0]
    per_w = B // W16.shape[0]
    scale_w = np.repeat(eW, per_w, axis=0)                     # [B, M]
    return Y * np.ldexp(1.0, -(scale_w[:, :, None] + eX[:, None, :]))
