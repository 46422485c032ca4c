// weights.cu — steering weights from geometry (Eq. 1-2).
//
// For weight batch b, beam/voxel m and receiver k:
//   far field : tau = (p_k . s_m) / c,        A = 1
//   near field: d = |t_m - p_k|, tau = d / c, A = 1 / d
//   w = A exp(-2 pi i f[b,k] tau)
// The phase phi = f tau (cycles) is formed in FP64 and reduced exactly to
// r = phi - rint(phi) in [-1/2, 1/2] (Sterbenz: the subtraction is exact),
// the only FP64 step; sin/cos of 2 pi r come from CUDA's sincospif in FP32.
// Output goes straight into the GEMM's packed W layout, so W needs no
// separate transpose/pack pass:
//   FP16 mode : planes [Bw][2][M][Kp], one thread per 8 consecutive k
//   TF32 mode : FP32 planes [Bw][2][M][Kp] rounded to TF32, 4 k per thread
//   1-bit mode: sign planes [Bw][2][M][Kw], one warp per 32 consecutive k
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "tcbf_internal.h"

namespace tcbf {
namespace {

struct Geo {
    const double *rx;
    const double *tg;
    const double *freqs;
    double c;
    int near_field;
    int64_t M;
    int K;
};

// Weight as FP32 (re, im).
__device__ __forceinline__ void weight(const Geo &g, int64_t bw, int64_t m, int k, float &re,
                                       float &im) {
    const double px = g.rx[3 * k], py = g.rx[3 * k + 1], pz = g.rx[3 * k + 2];
    const double tx = g.tg[3 * m], ty = g.tg[3 * m + 1], tz = g.tg[3 * m + 2];
    double tau, amp;
    if (g.near_field) {
        const double dx = tx - px, dy = ty - py, dz = tz - pz;
        const double d = sqrt(dx * dx + dy * dy + dz * dz);
        tau = d / g.c;
        amp = 1.0 / d;
    } else {
        tau = (px * tx + py * ty + pz * tz) / g.c;
        amp = 1.0;
    }
    const double phi = g.freqs[bw * g.K + k] * tau;
    const double t = 2.0 * (phi - rint(phi));         // half-turns in [-1, 1], exact
    // The FP32 argument t_hi drops up to 2^-25 half-turns; that residual is
    // added back to first order, sin(pi(h + l)) ~ sin(pi h) + pi l cos(pi h)
    // and cos(pi(h + l)) ~ cos(pi h) - pi l sin(pi h), so components near
    // zero keep their relative accuracy (|pi l| < 1e-7, the square ~1e-14).
    const float t_hi = static_cast<float>(t);
    const float pl = 3.14159265358979f * static_cast<float>(t - static_cast<double>(t_hi));
    float s0, c0;
    sincospif(t_hi, &s0, &c0);
    const float s = fmaf(c0, pl, s0);
    const float co = fmaf(-s0, pl, c0);
    const float a = static_cast<float>(amp);
    re = a * co;
    im = -a * s;
}

__global__ void weights_f16_kernel(Geo g, __half *__restrict__ dst, int64_t Bw, int Kp) {
    const int64_t chunks = Kp / 8;
    const int64_t total = Bw * g.M * chunks;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int k0 = static_cast<int>(i % chunks) * 8;
        const int64_t r = i / chunks;
        const int64_t m = r % g.M, bw = r / g.M;
        __align__(16) __half re[8], im[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float wr = 0.f, wi = 0.f;
            if (k0 + j < g.K) weight(g, bw, m, k0 + j, wr, wi);
            re[j] = __float2half_rn(wr);
            im[j] = __float2half_rn(wi);
        }
        *reinterpret_cast<uint4 *>(dst + (static_cast<size_t>(bw * 2 + 0) * g.M + m) * Kp + k0) =
            *reinterpret_cast<const uint4 *>(re);
        *reinterpret_cast<uint4 *>(dst + (static_cast<size_t>(bw * 2 + 1) * g.M + m) * Kp + k0) =
            *reinterpret_cast<const uint4 *>(im);
    }
}

// TF32: the FP32 weight rounded to TF32 (nearest, ties to even; see the
// pack kernels), one thread per 4 consecutive k.
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    u += 0x0fffu + ((u >> 13) & 1u);
    return __uint_as_float(u & 0xffffe000u);
}

__global__ void weights_tf32_kernel(Geo g, float *__restrict__ dst, int64_t Bw, int Kp) {
    const int64_t chunks = Kp / 4;
    const int64_t total = Bw * g.M * chunks;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int k0 = static_cast<int>(i % chunks) * 4;
        const int64_t r = i / chunks;
        const int64_t m = r % g.M, bw = r / g.M;
        float re[4], im[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            re[j] = im[j] = 0.f;
            if (k0 + j < g.K) weight(g, bw, m, k0 + j, re[j], im[j]);
        }
        *reinterpret_cast<float4 *>(dst + (static_cast<size_t>(bw * 2 + 0) * g.M + m) * Kp + k0) =
            make_float4(to_tf32(re[0]), to_tf32(re[1]), to_tf32(re[2]), to_tf32(re[3]));
        *reinterpret_cast<float4 *>(dst + (static_cast<size_t>(bw * 2 + 1) * g.M + m) * Kp + k0) =
            make_float4(to_tf32(im[0]), to_tf32(im[1]), to_tf32(im[2]), to_tf32(im[3]));
    }
}

__global__ void weights_bits_kernel(Geo g, uint32_t *__restrict__ dst, int64_t Bw, int Kw) {
    const int lane = threadIdx.x & 31;
    const int64_t total = Bw * g.M * Kw;
    const int64_t warps_total = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; i < total;
         i += warps_total) {
        const int w = static_cast<int>(i % Kw);
        const int64_t r = i / Kw;
        const int64_t m = r % g.M, bw = r / g.M;
        const int k = 32 * w + lane;
        float wr = -1.f, wi = -1.f;
        if (k < g.K) weight(g, bw, m, k, wr, wi);
        const uint32_t br = __ballot_sync(0xffffffffu, k < g.K && wr >= 0.f);
        const uint32_t bi = __ballot_sync(0xffffffffu, k < g.K && wi >= 0.f);
        if (lane == 0) {
            dst[(static_cast<size_t>(bw * 2 + 0) * g.M + m) * Kw + w] = br;
            dst[(static_cast<size_t>(bw * 2 + 1) * g.M + m) * Kw + w] = bi;
        }
    }
}

// Split-FP8: one warp per (weight batch, beam) row; the weights are computed
// twice, first for the row's largest magnitude (the scale exponent), then
// for the hi/lo bytes, in the packed layout of the transpose/pack kernel
// (HI: the hi bytes only, for plans that keep the hi product alone).
__device__ __forceinline__ void split_bytes(float v, uint8_t &hi, uint8_t &lo) {
    hi = static_cast<uint8_t>(__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3));
    const float h = __half2float(__half(__nv_cvt_fp8_to_halfraw(hi, __NV_E4M3)));
    lo = static_cast<uint8_t>(__nv_cvt_float_to_fp8(v - h, __NV_SATFINITE, __NV_E4M3));
}

template <bool HI>
__global__ void weights_split8_kernel(Geo g, uint8_t *__restrict__ dst, int32_t *__restrict__ exps,
                                      int64_t Bw, int Kb2) {
    const int lane = threadIdx.x & 31;
    const int64_t rows = Bw * g.M;
    const int64_t warps_total = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t r = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; r < rows;
         r += warps_total) {
        const int64_t m = r % g.M, bw = r / g.M;
        float amax = 0.f;
        for (int k = lane; k < g.K; k += 32) {
            float wr, wi;
            weight(g, bw, m, k, wr, wi);
            // the FP16 value the other modes would see
            wr = __half2float(__float2half_rn(wr));
            wi = __half2float(__float2half_rn(wi));
            amax = fmaxf(amax, fmaxf(fabsf(wr), fabsf(wi)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        int e = 0;
        if (amax > 0.f) {
            int q;
            const float f = frexpf(amax, &q);
            e = max(-100, min(100, (f <= 0.875f) ? 9 - q : 8 - q));
        }
        const float s = __int_as_float((127 + e) << 23);
        uint8_t *row_re = dst + (static_cast<size_t>(bw * 2 + 0) * g.M + m) * Kb2;
        uint8_t *row_im = dst + (static_cast<size_t>(bw * 2 + 1) * g.M + m) * Kb2;
        constexpr int kBlk = HI ? 64 : 128;
        for (int j = 0; j < Kb2 / kBlk; ++j) {
            uint8_t h[2][2], l[2][2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int k = 64 * j + 2 * lane + q;
                float wr = 0.f, wi = 0.f;
                if (k < g.K) {
                    weight(g, bw, m, k, wr, wi);
                    wr = __half2float(__float2half_rn(wr));
                    wi = __half2float(__float2half_rn(wi));
                }
                split_bytes(wr * s, h[0][q], l[0][q]);
                split_bytes(wi * s, h[1][q], l[1][q]);
            }
            *reinterpret_cast<uint16_t *>(row_re + kBlk * j + 2 * lane) = h[0][0] | (h[0][1] << 8);
            *reinterpret_cast<uint16_t *>(row_im + kBlk * j + 2 * lane) = h[1][0] | (h[1][1] << 8);
            if (!HI) {
                *reinterpret_cast<uint16_t *>(row_re + kBlk * j + 64 + 2 * lane) = l[0][0] | (l[0][1] << 8);
                *reinterpret_cast<uint16_t *>(row_im + kBlk * j + 64 + 2 * lane) = l[1][0] | (l[1][1] << 8);
            }
        }
        if (lane == 0) exps[r] = e;
    }
}

// Block-scaled split-FP8 (TCBF_FLAG_FP8_BLOCK_SCALES): one warp per row; per
// 64-k block lanes 0-15 hold k 0-31 and lanes 16-31 k 32-63, each half
// taking its 32-k block's exponent from its own largest magnitude; bytes as
// the transpose/pack kernel writes them (lo kept 16 times larger), the
// scale codes into the 512-byte tiles of 128 rows per stage.
template <bool HI>
__global__ void weights_split8_blk_kernel(Geo g, uint8_t *__restrict__ dst, uint8_t *__restrict__ sf,
                                          int64_t Bw, int Kb2, int stages) {
    const int lane = threadIdx.x & 31;
    const int64_t rows = Bw * g.M;
    const int64_t warps_total = int64_t(gridDim.x) * (blockDim.x >> 5);
    const int64_t tiles = (g.M + kFp8BlkRowsW - 1) / kFp8BlkRowsW;
    for (int64_t r = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; r < rows;
         r += warps_total) {
        const int64_t m = r % g.M, bw = r / g.M;
        uint8_t *row_re = dst + (static_cast<size_t>(bw * 2 + 0) * g.M + m) * Kb2;
        uint8_t *row_im = dst + (static_cast<size_t>(bw * 2 + 1) * g.M + m) * Kb2;
        uint8_t *tile_base = sf + static_cast<size_t>(bw * tiles + m / kFp8BlkRowsW) * stages * kFp8BlkTile;
        const int rr = static_cast<int>(m % kFp8BlkRowsW);
        const int tl = (rr & 31) * 16 + (rr >> 5) * 4;     // this row's entry in a tile
        constexpr int kBlk = HI ? 64 : 128;
        for (int jj = 0; jj < Kb2 / kBlk; ++jj) {
            float wr[2], wi[2];
            float amax = 0.f;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int k = 64 * jj + 2 * lane + q;
                wr[q] = wi[q] = 0.f;
                if (k < g.K) {
                    weight(g, bw, m, k, wr[q], wi[q]);
                    // the FP16 value the other modes would see
                    wr[q] = __half2float(__float2half_rn(wr[q]));
                    wi[q] = __half2float(__float2half_rn(wi[q]));
                }
                amax = fmaxf(amax, fmaxf(fabsf(wr[q]), fabsf(wi[q])));
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            int e = 0;
            if (amax > 0.f) {
                int q;
                const float f = frexpf(amax, &q);
                e = max(-100, min(100, (f <= 0.875f) ? 9 - q : 8 - q));
            }
            const float sc = __int_as_float((127 + e) << 23);
            uint8_t h[2][2], l[2][2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const float v = (p == 0 ? wr[q] : wi[q]) * sc;
                    h[p][q] = static_cast<uint8_t>(__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3));
                    const float hb = __half2float(__half(__nv_cvt_fp8_to_halfraw(h[p][q], __NV_E4M3)));
                    l[p][q] = static_cast<uint8_t>(
                        __nv_cvt_float_to_fp8(16.f * (v - hb), __NV_SATFINITE, __NV_E4M3));
                }
            }
            *reinterpret_cast<uint16_t *>(row_re + kBlk * jj + 2 * lane) = h[0][0] | (h[0][1] << 8);
            *reinterpret_cast<uint16_t *>(row_im + kBlk * jj + 2 * lane) = h[1][0] | (h[1][1] << 8);
            if (!HI) {
                *reinterpret_cast<uint16_t *>(row_re + kBlk * jj + 64 + 2 * lane) = l[0][0] | (l[0][1] << 8);
                *reinterpret_cast<uint16_t *>(row_im + kBlk * jj + 64 + 2 * lane) = l[1][0] | (l[1][1] << 8);
            }
            if ((lane & 15) == 0) {
                const int b2 = lane >> 4;
                if (HI) {
                    tile_base[static_cast<size_t>(jj / 2) * kFp8BlkTile + tl + 2 * (jj & 1) + b2] =
                        static_cast<uint8_t>(127 - e);
                } else {
                    tile_base[static_cast<size_t>(jj) * kFp8BlkTile + tl + b2] = static_cast<uint8_t>(127 - e);
                    tile_base[static_cast<size_t>(jj) * kFp8BlkTile + tl + 2 + b2] =
                        static_cast<uint8_t>(123 - e);
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_weights(const tcbf_plan_s &pl, const double *rx, const double *tg,
                           int near_field, const double *freqs, double c, void *Wp,
                           cudaStream_t s) {
    Geo g;
    g.rx = rx;
    g.tg = tg;
    g.freqs = freqs;
    g.c = c;
    g.near_field = near_field;
    g.M = pl.p.M;
    g.K = static_cast<int>(pl.p.K);
    const int64_t Bw = pl.p.w_batches;
    if (pl.p.mode == TCBF_MODE_1BIT) {
        const int64_t work = Bw * pl.p.M * pl.Kw * 32;
        const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, int64_t(pl.num_sms) * 32)));
        weights_bits_kernel<<<grid, 256, 0, s>>>(g, static_cast<uint32_t *>(Wp), Bw, int(pl.Kw));
    } else if (pl.p.mode == TCBF_MODE_TF32) {
        const int64_t work = Bw * pl.p.M * (pl.Kp / 4);
        const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, int64_t(pl.num_sms) * 32)));
        weights_tf32_kernel<<<grid, 256, 0, s>>>(g, static_cast<float *>(Wp), Bw, int(pl.Kp));
    } else if (pl.p.mode == TCBF_MODE_FP16) {
        const int64_t work = Bw * pl.p.M * (pl.Kp / 8);
        const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, int64_t(pl.num_sms) * 32)));
        weights_f16_kernel<<<grid, 256, 0, s>>>(g, static_cast<__half *>(Wp), Bw, int(pl.Kp));
    } else if (fp8_block_scaled(pl.p.flags)) {
        const int64_t rows = Bw * pl.p.M;
        const int Kb2 = static_cast<int>(pl.Kb2);
        auto *d = static_cast<uint8_t *>(Wp);
        uint8_t *sf = d + rows * 2 * Kb2;
        const int64_t sfb = fp8blk_sf_bytes(Bw, pl.p.M, pl.p.K, pl.p.flags, 0);
        cudaError_t e = cudaMemsetAsync(sf, 127, static_cast<size_t>(sfb), s);
        if (e != cudaSuccess) return e;
        const int st = static_cast<int>(fp8blk_stages(pl.p.K, pl.p.flags));
        const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((rows * 32 + 255) / 256, int64_t(pl.num_sms) * 32)));
        if (fp8_hi_only(pl.p.flags))
            weights_split8_blk_kernel<true><<<grid, 256, 0, s>>>(g, d, sf, Bw, Kb2, st);
        else
            weights_split8_blk_kernel<false><<<grid, 256, 0, s>>>(g, d, sf, Bw, Kb2, st);
    } else {
        const int64_t rows = Bw * pl.p.M;
        const int Kb2 = static_cast<int>(pl.Kb2);
        auto *d = static_cast<uint8_t *>(Wp);
        auto *ex = reinterpret_cast<int32_t *>(d + rows * 2 * Kb2);
        const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((rows * 32 + 255) / 256, int64_t(pl.num_sms) * 32)));
        if (fp8_hi_only(pl.p.flags))
            weights_split8_kernel<true><<<grid, 256, 0, s>>>(g, d, ex, Bw, Kb2);
        else
            weights_split8_kernel<false><<<grid, 256, 0, s>>>(g, d, ex, Bw, Kb2);
    }
    return cudaGetLastError();
}

}  // namespace tcbf
