"""Seeded synthetic inputs for the tensor-core beamformer.

This module is shared by the CPU oracle, the tests and the benchmark.  It
holds no beamforming arithmetic: only random draws (numpy PCG64), array
geometry for the workloads of the paper's applications (Sec. V), and the
storage formats the library accepts (interleaved complex FP16, packed sign
words).  Weights that the method derives from geometry (Eq. 1-2) are NOT made
here; geometry is returned and each side computes its own weights.

Draw order inside every generator is fixed (real parts, imaginary parts, then
phases / positions / directions) so a seed names one input set exactly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SPEED_OF_LIGHT = 299_792_458.0   # m/s, radio workloads
SPEED_OF_SOUND_TISSUE = 1540.0   # m/s, ultrasound workload


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def interleave_fp16(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Round re/im to IEEE binary16 (round-to-nearest-even) and interleave
    them as (..., 2) — the library's input format for complex FP16."""
    out = np.empty(re.shape + (2,), dtype=np.float16)
    out[..., 0] = re
    out[..., 1] = im
    return out


def complex_gaussian_fp16(g: np.random.Generator, shape) -> np.ndarray:
    """iid N(0,1) real and imaginary parts, drawn real-first, as FP16 pairs."""
    re = g.standard_normal(shape, dtype=np.float32)
    im = g.standard_normal(shape, dtype=np.float32)
    return interleave_fp16(re, im)


def integer_complex_fp16(g: np.random.Generator, shape, lo=-8, hi=8) -> np.ndarray:
    """Small integer-valued complex entries; every partial sum of a product
    of two such matrices is an exact integer in FP32 while K*2*hi*hi < 2**24."""
    re = g.integers(lo, hi + 1, size=shape)
    im = g.integers(lo, hi + 1, size=shape)
    return interleave_fp16(re.astype(np.float64), im.astype(np.float64))


def random_sign_words(g: np.random.Generator, shape) -> np.ndarray:
    """iid fair bits, 32 per uint32 word (1-bit complex planes, Fig. 1)."""
    return g.integers(0, 2**32, size=shape, dtype=np.uint32)


def words_per_row(K: int) -> int:
    """Packed 1-bit row length in 32-bit words: K rounded up to 128 bits
    so every row starts on a 16-byte boundary."""
    return ((K + 127) // 128) * 4


# ---------------------------------------------------------------------------
# Workload 1: plain FP16 beamform, batch 1, W 64x128, X 128x1024.
# ---------------------------------------------------------------------------
def small_fp16(seed=0, M=64, K=128, N=1024, B=1):
    """X re/im iid N(0,1) -> FP16; W = exp(i phi), phi ~ U[0, 2 pi) -> FP16.
    Returns (W [B,M,K,2] fp16, X [B,K,N,2] fp16)."""
    g = rng(seed)
    xr = g.standard_normal((B, K, N))
    xi = g.standard_normal((B, K, N))
    phi = g.uniform(0.0, 2.0 * math.pi, size=(B, M, K))
    X = interleave_fp16(xr, xi)
    W = interleave_fp16(np.cos(phi), np.sin(phi))
    return W, X


def random_phase_rows(seed, M, K, block_rows=1024, threads=None):
    """W = exp(i phi), phi ~ U[0, 2 pi) -> FP16, [1, M, K, 2], drawn in
    blocks of rows from independent streams in parallel (full-size model
    matrices with the value distribution of the small FP16 workload)."""
    import concurrent.futures as cf
    import os
    out = np.empty((1, M, K, 2), np.float16)

    def one(blk):
        r0 = blk * block_rows
        r1 = min(M, r0 + block_rows)
        phi = batch_rng(seed, blk).uniform(0.0, 2.0 * math.pi, size=(r1 - r0, K))
        out[0, r0:r1, :, 0] = np.cos(phi)
        out[0, r0:r1, :, 1] = np.sin(phi)

    with cf.ThreadPoolExecutor(threads or min(32, os.cpu_count() or 4)) as ex:
        list(ex.map(one, range((M + block_rows - 1) // block_rows)))
    return out


# ---------------------------------------------------------------------------
# Radio-astronomy geometry (Sec. V-B): stations in a disk, beams near zenith.
# ---------------------------------------------------------------------------
@dataclass
class Geometry:
    rx_pos: np.ndarray     # [K,3] float64 receiver positions (m)
    targets: np.ndarray    # [M,3] float64: unit directions (far field) or voxel positions (m)
    freqs: np.ndarray      # [Bw,K] float64 frequency seen by column k of weight batch b (Hz)
    near_field: bool
    c: float


def station_disk(g, K, radius_m=1500.0):
    """K positions uniform in area over a disk of the given radius, z = 0."""
    u = g.random(K)
    v = g.random(K)
    r = radius_m * np.sqrt(u)
    a = 2.0 * math.pi * v
    return np.stack([r * np.cos(a), r * np.sin(a), np.zeros(K)], axis=1)


def beams_near_zenith(g, M, max_zenith_deg=5.0):
    """M unit vectors uniform over the spherical cap theta <= max_zenith."""
    cmin = math.cos(math.radians(max_zenith_deg))
    cz = g.uniform(cmin, 1.0, size=M)
    az = g.uniform(0.0, 2.0 * math.pi, size=M)
    s = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return np.stack([s * np.cos(az), s * np.sin(az), cz], axis=1)


def channel_freqs(n_channels=256, f_lo=110e6, f_hi=190e6):
    """Channel centres f_c = f_lo + (c + 1/2) (f_hi - f_lo) / n_channels."""
    c = np.arange(n_channels, dtype=np.float64)
    return f_lo + (c + 0.5) * (f_hi - f_lo) / n_channels


def radio_geometry(seed=0, n_beams=1024, n_stations=288, n_channels=256):
    """Positions drawn first, then directions (fixed draw order)."""
    g = rng(seed)
    pos = station_disk(g, n_stations)
    dirs = beams_near_zenith(g, n_beams)
    f = channel_freqs(n_channels)
    freqs = np.repeat(f[:, None], n_stations, axis=1)
    return Geometry(pos, dirs, freqs, False, SPEED_OF_LIGHT)


def batch_rng(seed: int, b: int) -> np.random.Generator:
    """Independent stream for batch b (so any subset of batches can be
    regenerated alone, and batches can be drawn in parallel)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, b])))


def radio_x_batch(seed, b, n_stations=288, n_samples=4096):
    """Samples of batch b: complex Gaussian FP16 [K, N, 2]."""
    return complex_gaussian_fp16(batch_rng(seed, b), (n_stations, n_samples))


def radio_x(seed=1, batches=512, n_stations=288, n_samples=4096, out=None, threads=None):
    """X for all batches, [B, K, N, 2] FP16, drawn batch by batch in parallel."""
    import concurrent.futures as cf
    import os
    if out is None:
        out = np.empty((batches, n_stations, n_samples, 2), np.float16)

    def one(b):
        out[b] = radio_x_batch(seed, b, n_stations, n_samples)

    with cf.ThreadPoolExecutor(threads or min(32, os.cpu_count() or 4)) as ex:
        list(ex.map(one, range(batches)))
    return out


def radio_block(seed=0, n_beams=1024, n_stations=288, n_samples=4096,
                n_channels=256, n_pols=2, make_x=True):
    """Batched radio block: batch index b = 2*channel + pol; both
    polarisations of a channel share that channel's weights.  X is
    complex Gaussian FP16 [B, K, N, 2] with B = channels * pols."""
    geom = radio_geometry(seed, n_beams, n_stations, n_channels)
    X = radio_x(seed + 1, n_channels * n_pols, n_stations, n_samples) if make_x else None
    return geom, X


# ---------------------------------------------------------------------------
# Computational ultrasound geometry (Sec. V-A).
# ---------------------------------------------------------------------------
def ultrasound_geometry(n_elements=128, pitch_m=0.3e-3, n_bins=128,
                        f_lo=10e6, f_hi=20e6, grid=(32, 32, 64),
                        xy_half_m=20e-3, z_range_m=(5e-3, 45e-3)):
    """Linear array along x (centred, z = 0); column k = element * n_bins + bin;
    voxel centres on a regular grid, flattened x-fastest: m = (iz*ny + iy)*nx + ix."""
    e = (np.arange(n_elements) - (n_elements - 1) / 2.0) * pitch_m
    elem = np.stack([e, np.zeros(n_elements), np.zeros(n_elements)], axis=1)
    bins = f_lo + np.arange(n_bins) * (f_hi - f_lo) / n_bins
    rx_pos = np.repeat(elem, n_bins, axis=0)                # [K,3]
    freqs = np.tile(bins, n_elements)[None, :]              # [1,K]
    nx, ny, nz = grid
    xs = -xy_half_m + (np.arange(nx) + 0.5) * (2 * xy_half_m / nx)
    ys = -xy_half_m + (np.arange(ny) + 0.5) * (2 * xy_half_m / ny)
    z0, z1 = z_range_m
    zs = z0 + (np.arange(nz) + 0.5) * ((z1 - z0) / nz)
    Z, Y, Xg = np.meshgrid(zs, ys, xs, indexing="ij")
    targets = np.stack([Xg.ravel(), Y.ravel(), Z.ravel()], axis=1)
    return Geometry(rx_pos, targets, freqs, True, SPEED_OF_SOUND_TISSUE)


def ultrasound_frames(seed=0, K=16384, n_frames=256):
    """Complex Gaussian echoes, FP16 [1, K, n_frames, 2]."""
    return complex_gaussian_fp16(rng(seed), (1, K, n_frames))


# ---------------------------------------------------------------------------
# 1-bit radio block: packed sign planes [B, 2, rows, Kw] (re plane, im plane).
# ---------------------------------------------------------------------------
def onebit_block(seed=0, B=64, M=2048, K=1024, N=8192):
    g = rng(seed)
    kw = words_per_row(K)
    Xb = random_sign_words(g, (B, 2, N, kw))
    Wb = random_sign_words(g, (B, 2, M, kw))
    return Wb, Xb
