// pack.cu — transpose / pack kernels (Sec. III: the GEMM needs its inputs
// split into real and imaginary planes and tiled in device memory; 1-bit
// inputs are packed 32 samples per 32-bit word).  Memory-bound: every byte
// is read once and written once, with coalesced accesses on both sides.
//
//   W (weights) [Bw][M][K] complex  -> [Bw][2][M][Kp] planes (no transpose)
//   X (samples) [B][K][N] complex   -> [B][2][N][Kp] planes (transposed so K
//                                      is contiguous for the GEMM's TMA)
//   1-bit: the same two shapes, keeping only the sign of each component,
//   32 signs per uint32 along K (bit k % 32 of word k / 32, 1 = +1).
//   TF32: the FP16 shapes with FP32 storage, each value rounded to TF32.
#include <cuda_fp16.h>

#include <algorithm>

#include "tcbf_internal.h"

namespace tcbf {
namespace {

struct CF16 {
    using raw = __half2;
    static __device__ __forceinline__ void load(const void *src, size_t i, float &re, float &im) {
        const __half2 v = reinterpret_cast<const __half2 *>(src)[i];
        re = __low2float(v);
        im = __high2float(v);
    }
    static __device__ __forceinline__ void load_h(const void *src, size_t i, __half &re,
                                                  __half &im) {
        const __half2 v = reinterpret_cast<const __half2 *>(src)[i];
        re = __low2half(v);
        im = __high2half(v);
    }
    // value i as one word: re in the low half, im in the high half
    static __device__ __forceinline__ uint32_t load_word(const void *src, size_t i) {
        return reinterpret_cast<const uint32_t *>(src)[i];
    }
    // values i .. i + 3 (i a multiple of 4, 16-byte aligned)
    static __device__ __forceinline__ void load4(const void *src, size_t i, uint32_t (&w)[4]) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(src) + i / 4);
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
    }
};

struct CF32 {
    static __device__ __forceinline__ void load(const void *src, size_t i, float &re, float &im) {
        const float2 v = reinterpret_cast<const float2 *>(src)[i];
        re = v.x;
        im = v.y;
    }
    static __device__ __forceinline__ void load_h(const void *src, size_t i, __half &re,
                                                  __half &im) {
        const float2 v = reinterpret_cast<const float2 *>(src)[i];
        re = __float2half_rn(v.x);
        im = __float2half_rn(v.y);
    }
    static __device__ __forceinline__ uint32_t to_word(float re, float im) {
        const __half2 h = __halves2half2(__float2half_rn(re), __float2half_rn(im));
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    static __device__ __forceinline__ uint32_t load_word(const void *src, size_t i) {
        const float2 v = reinterpret_cast<const float2 *>(src)[i];
        return to_word(v.x, v.y);
    }
    // values i .. i + 3 (i a multiple of 4, 32-byte aligned)
    static __device__ __forceinline__ void load4(const void *src, size_t i, uint32_t (&w)[4]) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(src) + i / 2);
        const float4 c = __ldg(reinterpret_cast<const float4 *>(src) + i / 2 + 1);
        w[0] = to_word(a.x, a.y);
        w[1] = to_word(a.z, a.w);
        w[2] = to_word(c.x, c.y);
        w[3] = to_word(c.z, c.w);
    }
};

int grid_for(int64_t work, int threads, int num_sms) {
    const int64_t blocks = (work + threads - 1) / threads;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(blocks, int64_t(num_sms) * 16)));
}

// ------------------------------------------------ interleaved FP16 samples
// X of plans that keep the caller's interleaved layout: FP32 values rounded
// to FP16 in place of the layout, four complex values per thread.
__global__ void round_cf32_to_cf16_kernel(const float4 *__restrict__ src, uint2 *__restrict__ dst,
                                          int64_t n2) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n2;
         i += int64_t(gridDim.x) * blockDim.x) {
        const float4 v = __ldg(src + i);     // two complex values
        uint2 o;
        o.x = CF32::to_word(v.x, v.y);
        o.y = CF32::to_word(v.z, v.w);
        dst[i] = o;
    }
}

__global__ void round_tail_kernel(const float2 *__restrict__ src, uint32_t *__restrict__ dst) {
    const float2 v = *src;
    *dst = CF32::to_word(v.x, v.y);
}

// ------------------------------------------------------------ FP16 planes
// W: one thread writes 8 consecutive K elements (16 bytes) of both planes.
template <typename S>
__global__ void pack_f16_w_kernel(const void *__restrict__ src, __half *__restrict__ dst,
                                  int64_t rows, int64_t M, int K, int Kp) {
    const int64_t chunks = Kp / 8;
    const int64_t total = rows * chunks;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = i / chunks;
        const int k0 = static_cast<int>(i % chunks) * 8;
        const int64_t bw = r / M, m = r % M;
        __align__(16) __half re[8], im[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = k0 + j;
            if (k < K) {
                S::load_h(src, static_cast<size_t>(r) * K + k, re[j], im[j]);
            } else {
                re[j] = __float2half_rn(0.f);
                im[j] = __float2half_rn(0.f);
            }
        }
        const size_t o_re = (static_cast<size_t>(bw * 2 + 0) * M + m) * Kp + k0;
        const size_t o_im = (static_cast<size_t>(bw * 2 + 1) * M + m) * Kp + k0;
        *reinterpret_cast<uint4 *>(dst + o_re) = *reinterpret_cast<const uint4 *>(re);
        *reinterpret_cast<uint4 *>(dst + o_im) = *reinterpret_cast<const uint4 *>(im);
    }
}

// X: 64 (k) x 64 (n) tiles through shared memory, one 32-bit word (re, im
// halves) per complex value.  Loads read rows of X (n contiguous), four
// values per thread as one 16-byte access (FP16 source; FP32 sources are
// rounded while loading); stores write rows of the packed planes (k
// contiguous), eight threads per 128-byte row, each splitting 8 words into
// 8 re and 8 im halves with byte permutes.  The word of (k, n) sits at
// column n ^ 4 (k / 8) of row k: the 16-byte row writes stay contiguous and
// the column reads of a warp (4 n x 8 k-chunks) hit 32 distinct banks.
constexpr int TT = 64;
constexpr int TPITCH = TT + 2;   // halves; odd word pitch spreads banks (split-FP8 X pack)

// PL = 3 writes the stacked layout: planes -Xi, Xr, Xi (the sign bits of
// the imaginary halves flipped for the first).
template <typename S, bool VEC, int PL>
__global__ void __launch_bounds__(256) pack_f16_x_kernel(const void *__restrict__ src,
                                                        __half *__restrict__ dst, int K, int N,
                                                        int Kp, int k_tiles, int n_tiles) {
    __shared__ __align__(16) uint32_t tile[TT * TT];
    const int tid = threadIdx.x;
    const int64_t tiles_per_b = int64_t(k_tiles) * n_tiles;
    const int64_t b = blockIdx.y;
    for (int64_t t = blockIdx.x; t < tiles_per_b; t += gridDim.x) {
        const int kt = static_cast<int>(t / n_tiles);
        const int nt = static_cast<int>(t % n_tiles);
        const int k0 = kt * TT, n0 = nt * TT;
        // load: thread (ty, tx) takes n = 4 tx .. 4 tx + 3 of rows ty + 16 i
        const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int kk = ty + 16 * i;
            const int k = k0 + kk;
            const int n = n0 + 4 * tx;
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (k < K) {
                const size_t e = (static_cast<size_t>(b) * K + k) * N + n;
                if (VEC && n + 3 < N) {
                    S::load4(src, e, w);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (n + q < N) w[q] = S::load_word(src, e + q);
                }
            }
            const int col = (4 * tx) ^ (4 * (kk >> 3));
            *reinterpret_cast<uint4 *>(&tile[kk * TT + col]) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        __syncthreads();
        // store: thread -> (row n, k-chunk c of 8); two rows per thread
        const int c = tid & 7;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int nn = (tid >> 3) + 32 * h;
            const int n = n0 + nn;
            const int k = k0 + 8 * c;
            if (n < N && k < Kp) {
                uint32_t v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = tile[(8 * c + j) * TT + (nn ^ (4 * c))];
                uint4 re, im;
                re.x = __byte_perm(v[0], v[1], 0x5410);
                re.y = __byte_perm(v[2], v[3], 0x5410);
                re.z = __byte_perm(v[4], v[5], 0x5410);
                re.w = __byte_perm(v[6], v[7], 0x5410);
                im.x = __byte_perm(v[0], v[1], 0x7632);
                im.y = __byte_perm(v[2], v[3], 0x7632);
                im.z = __byte_perm(v[4], v[5], 0x7632);
                im.w = __byte_perm(v[6], v[7], 0x7632);
                const size_t o_re = (static_cast<size_t>(b * PL + PL - 2) * N + n) * Kp + k;
                const size_t o_im = (static_cast<size_t>(b * PL + PL - 1) * N + n) * Kp + k;
                *reinterpret_cast<uint4 *>(dst + o_re) = re;
                *reinterpret_cast<uint4 *>(dst + o_im) = im;
                if (PL == 3) {
                    const size_t o_neg = (static_cast<size_t>(b * PL) * N + n) * Kp + k;
                    *reinterpret_cast<uint4 *>(dst + o_neg) =
                        make_uint4(im.x ^ 0x80008000u, im.y ^ 0x80008000u, im.z ^ 0x80008000u,
                                   im.w ^ 0x80008000u);
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ TF32 planes
// Rounding to TF32 (10 stored mantissa bits) to nearest, ties to even, kept
// in FP32 storage with the 13 low bits zero: adding 0xFFF plus the lowest
// kept bit and clearing the dropped bits rounds the magnitude (a carry into
// the exponent is the correct step to the next binade, or to infinity).
// Infinities pass unchanged; NaNs stay NaN (quiet bit set).
__device__ __forceinline__ float tf32_rne(float x) {
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) == 0x7f800000u)
        return __uint_as_float((u & 0x007fffffu) ? ((u | 0x00400000u) & 0xffffe000u) : u);
    u += 0x0fffu + ((u >> 13) & 1u);
    return __uint_as_float(u & 0xffffe000u);
}

// W: one thread writes 4 consecutive K elements (16 bytes) of both planes.
template <typename S>
__global__ void pack_tf32_w_kernel(const void *__restrict__ src, float *__restrict__ dst,
                                   int64_t rows, int64_t M, int K, int Kp) {
    const int64_t chunks = Kp / 4;
    const int64_t total = rows * chunks;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = i / chunks;
        const int k0 = static_cast<int>(i % chunks) * 4;
        const int64_t bw = r / M, m = r % M;
        float re[4], im[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            re[j] = im[j] = 0.f;
            if (k0 + j < K) S::load(src, static_cast<size_t>(r) * K + k0 + j, re[j], im[j]);
        }
        *reinterpret_cast<float4 *>(dst + (static_cast<size_t>(bw * 2 + 0) * M + m) * Kp + k0) =
            make_float4(tf32_rne(re[0]), tf32_rne(re[1]), tf32_rne(re[2]), tf32_rne(re[3]));
        *reinterpret_cast<float4 *>(dst + (static_cast<size_t>(bw * 2 + 1) * M + m) * Kp + k0) =
            make_float4(tf32_rne(im[0]), tf32_rne(im[1]), tf32_rne(im[2]), tf32_rne(im[3]));
    }
}

// X: 32 (k) x 32 (n) tiles through shared memory: warps read rows of X (n
// contiguous) and write rows of the packed planes (k contiguous).
template <typename S>
__global__ void __launch_bounds__(256) pack_tf32_x_kernel(const void *__restrict__ src,
                                                         float *__restrict__ dst, int K, int N,
                                                         int Kp, int k_tiles, int n_tiles) {
    __shared__ float2 tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t b = blockIdx.y;
    const int64_t tiles_per_b = int64_t(k_tiles) * n_tiles;
    for (int64_t t = blockIdx.x; t < tiles_per_b; t += gridDim.x) {
        const int k0 = static_cast<int>(t / n_tiles) * 32;
        const int n0 = static_cast<int>(t % n_tiles) * 32;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int kk = ty + 8 * i;
            float re = 0.f, im = 0.f;
            if (k0 + kk < K && n0 + tx < N)
                S::load(src, (static_cast<size_t>(b) * K + k0 + kk) * N + n0 + tx, re, im);
            tile[kk][tx] = make_float2(tf32_rne(re), tf32_rne(im));
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int nn = ty + 8 * i;
            const int n = n0 + nn, k = k0 + tx;
            if (n < N && k < Kp) {
                const float2 v = tile[tx][nn];
                dst[(static_cast<size_t>(b * 2 + 0) * N + n) * Kp + k] = v.x;
                dst[(static_cast<size_t>(b * 2 + 1) * N + n) * Kp + k] = v.y;
            }
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------- sign bits
// Sign of one component: v >= 0 gives bit 1 (+1), so -0 gives +1; negative
// values and NaN give bit 0 (-1).
__device__ __forceinline__ uint32_t sign_bit(float v) { return v >= 0.f ? 1u : 0u; }

// W: one warp per (row, word); lane l holds element 32 w + l, a ballot
// assembles the word with lane l at bit l.
template <typename S>
__global__ void pack_bits_w_kernel(const void *__restrict__ src, uint32_t *__restrict__ dst,
                                   int64_t rows, int64_t M, int K, int Kw) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = int64_t(gridDim.x) * (blockDim.x >> 5);
    const int64_t total = rows * Kw;
    for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; i < total;
         i += warps_total) {
        const int64_t r = i / Kw;
        const int w = static_cast<int>(i % Kw);
        const int k = 32 * w + lane;
        float re = -1.f, im = -1.f;
        if (k < K) S::load(src, static_cast<size_t>(r) * K + k, re, im);
        const uint32_t wr = __ballot_sync(0xffffffffu, k < K && sign_bit(re));
        const uint32_t wi = __ballot_sync(0xffffffffu, k < K && sign_bit(im));
        if (lane == 0) {
            const int64_t bw = r / M, m = r % M;
            dst[(static_cast<size_t>(bw * 2 + 0) * M + m) * Kw + w] = wr;
            dst[(static_cast<size_t>(bw * 2 + 1) * M + m) * Kw + w] = wi;
        }
    }
}

// X: lane l owns column n0 + l and walks the 32 rows k of one word, so each
// load instruction reads 32 consecutive samples of one row.
template <typename S>
__global__ void pack_bits_x_kernel(const void *__restrict__ src, uint32_t *__restrict__ dst,
                                   int K, int N, int Kw, int n_groups) {
    const int lane = threadIdx.x & 31;
    const int64_t b = blockIdx.y;
    const int64_t total = int64_t(Kw) * n_groups;
    const int64_t warps_total = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; i < total;
         i += warps_total) {
        const int w = static_cast<int>(i / n_groups);
        const int n = static_cast<int>(i % n_groups) * 32 + lane;
        uint32_t wr = 0, wi = 0;
        if (n < N) {
            const int kend = min(32, K - 32 * w);
            for (int j = 0; j < kend; ++j) {
                float re, im;
                S::load(src, (static_cast<size_t>(b) * K + 32 * w + j) * N + n, re, im);
                wr |= sign_bit(re) << j;
                wi |= sign_bit(im) << j;
            }
            dst[(static_cast<size_t>(b * 2 + 0) * N + n) * Kw + w] = wr;
            dst[(static_cast<size_t>(b * 2 + 1) * N + n) * Kw + w] = wi;
        }
    }
}

// Unpacking (the inverse of the two kernels above): bits back to interleaved
// complex +-1 values (Fig. 1: bit 1 is +1, bit 0 is -1), one (re, im) pair
// per store.  W: one warp per (row, word), lane l writes element 32 w + l.
// X: lane l owns column n0 + l of one word and walks its 32 rows k, so each
// store instruction writes 32 consecutive samples of one row.
__device__ __forceinline__ void store_pm1(__half *p, uint32_t re, uint32_t im) {
    *reinterpret_cast<__half2 *>(p) = __halves2half2(__float2half_rn(re ? 1.f : -1.f),
                                                     __float2half_rn(im ? 1.f : -1.f));
}
__device__ __forceinline__ void store_pm1(float *p, uint32_t re, uint32_t im) {
    *reinterpret_cast<float2 *>(p) = make_float2(re ? 1.f : -1.f, im ? 1.f : -1.f);
}

template <typename T>
__global__ void unpack_bits_w_kernel(const uint32_t *__restrict__ src, T *__restrict__ dst,
                                     int64_t rows, int64_t M, int K, int Kw) {
    const int lane = threadIdx.x & 31;
    const int words = (K + 31) / 32;
    const int64_t warps_total = int64_t(gridDim.x) * (blockDim.x >> 5);
    const int64_t total = rows * words;
    for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; i < total;
         i += warps_total) {
        const int64_t r = i / words;
        const int w = static_cast<int>(i % words);
        const int k = 32 * w + lane;
        const int64_t bw = r / M, m = r % M;
        const uint32_t wr = __ldg(src + (static_cast<size_t>(bw * 2 + 0) * M + m) * Kw + w);
        const uint32_t wi = __ldg(src + (static_cast<size_t>(bw * 2 + 1) * M + m) * Kw + w);
        if (k < K) store_pm1(dst + (static_cast<size_t>(r) * K + k) * 2, (wr >> lane) & 1u, (wi >> lane) & 1u);
    }
}

template <typename T>
__global__ void unpack_bits_x_kernel(const uint32_t *__restrict__ src, T *__restrict__ dst,
                                     int K, int N, int Kw, int n_groups) {
    const int lane = threadIdx.x & 31;
    const int64_t b = blockIdx.y;
    const int words = (K + 31) / 32;
    const int64_t total = int64_t(words) * n_groups;
    const int64_t warps_total = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; i < total;
         i += warps_total) {
        const int w = static_cast<int>(i / n_groups);
        const int n = static_cast<int>(i % n_groups) * 32 + lane;
        if (n >= N) continue;
        const uint32_t wr = __ldg(src + (static_cast<size_t>(b * 2 + 0) * N + n) * Kw + w);
        const uint32_t wi = __ldg(src + (static_cast<size_t>(b * 2 + 1) * N + n) * Kw + w);
        const int kend = min(32, K - 32 * w);
        for (int j = 0; j < kend; ++j)
            store_pm1(dst + ((static_cast<size_t>(b) * K + 32 * w + j) * N + n) * 2, (wr >> j) & 1u,
                      (wi >> j) & 1u);
    }
}

}  // namespace

cudaError_t launch_unpack_bits(const tcbf_plan_s &pl, int which, const uint32_t *src, int dst_type,
                               void *dst, cudaStream_t s) {
    const int K = static_cast<int>(pl.p.K), Kw = static_cast<int>(pl.Kw);
    const int words = (K + 31) / 32;
    if (which == 0) {
        const int64_t rows = pl.p.w_batches * pl.p.M;
        const int grid = grid_for(rows * words * 32, 256, pl.num_sms);
        if (dst_type == TCBF_SRC_CF16)
            unpack_bits_w_kernel<__half><<<grid, 256, 0, s>>>(src, static_cast<__half *>(dst), rows,
                                                               pl.p.M, K, Kw);
        else
            unpack_bits_w_kernel<float><<<grid, 256, 0, s>>>(src, static_cast<float *>(dst), rows,
                                                              pl.p.M, K, Kw);
    } else {
        const int n_groups = static_cast<int>(ceil_div(pl.p.N, 32));
        const int64_t per_b = int64_t(words) * n_groups * 32;
        const int bx = std::max(1, std::min(grid_for(per_b, 256, pl.num_sms), 4096));
        dim3 grid(bx, static_cast<unsigned>(pl.p.batch));
        if (dst_type == TCBF_SRC_CF16)
            unpack_bits_x_kernel<__half><<<grid, 256, 0, s>>>(src, static_cast<__half *>(dst), K,
                                                               int(pl.p.N), Kw, n_groups);
        else
            unpack_bits_x_kernel<float><<<grid, 256, 0, s>>>(src, static_cast<float *>(dst), K,
                                                              int(pl.p.N), Kw, n_groups);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_f16_w(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                              cudaStream_t s) {
    const int64_t rows = pl.p.w_batches * pl.p.M;
    const int grid = grid_for(rows * (pl.Kp / 8), 256, pl.num_sms);
    auto *d = static_cast<__half *>(dst);
    if (src_type == TCBF_SRC_CF16)
        pack_f16_w_kernel<CF16><<<grid, 256, 0, s>>>(src, d, rows, pl.p.M, int(pl.p.K), int(pl.Kp));
    else
        pack_f16_w_kernel<CF32><<<grid, 256, 0, s>>>(src, d, rows, pl.p.M, int(pl.p.K), int(pl.Kp));
    return cudaGetLastError();
}

cudaError_t launch_pack_f16_x(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                              cudaStream_t s) {
    const int k_tiles = static_cast<int>(ceil_div(pl.Kp, TT));
    const int n_tiles = static_cast<int>(ceil_div(pl.p.N, TT));
    const int64_t per_b = int64_t(k_tiles) * n_tiles;
    const int bx = static_cast<int>(std::min<int64_t>(per_b, std::max<int64_t>(1, int64_t(pl.num_sms) * 8 / std::max<int64_t>(1, std::min<int64_t>(pl.p.batch, 8)))));
    dim3 grid(bx, static_cast<unsigned>(pl.p.batch));
    auto *d = static_cast<__half *>(dst);
    // 16-byte loads of four values need every row of X to start 16-byte aligned
    const bool vec = pl.p.N % 4 == 0;
    const int K = int(pl.p.K), N = int(pl.p.N), Kp = int(pl.Kp);
    auto run = [&](auto kern) { kern<<<grid, 256, 0, s>>>(src, d, K, N, Kp, k_tiles, n_tiles); };
    const bool stacked = x_planes(pl) == 3;
    if (src_type == TCBF_SRC_CF16) {
        if (stacked)
            vec ? run(pack_f16_x_kernel<CF16, true, 3>) : run(pack_f16_x_kernel<CF16, false, 3>);
        else
            vec ? run(pack_f16_x_kernel<CF16, true, 2>) : run(pack_f16_x_kernel<CF16, false, 2>);
    } else {
        if (stacked)
            vec ? run(pack_f16_x_kernel<CF32, true, 3>) : run(pack_f16_x_kernel<CF32, false, 3>);
        else
            vec ? run(pack_f16_x_kernel<CF32, true, 2>) : run(pack_f16_x_kernel<CF32, false, 2>);
    }
    return cudaGetLastError();
}

cudaError_t launch_copy_x_cf16(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                               cudaStream_t s) {
    const int64_t values = pl.p.batch * pl.p.K * pl.p.N;
    if (src_type == TCBF_SRC_CF16) {
        if (src == dst) return cudaSuccess;
        return cudaMemcpyAsync(dst, src, static_cast<size_t>(values * 4), cudaMemcpyDeviceToDevice, s);
    }
    // values is even when N is; an odd count leaves one value for a second pass
    const int64_t n2 = values / 2;
    if (n2 > 0)
        round_cf32_to_cf16_kernel<<<grid_for(n2, 256, pl.num_sms), 256, 0, s>>>(
            static_cast<const float4 *>(src), static_cast<uint2 *>(dst), n2);
    if (values & 1) {
        const float2 *tail = static_cast<const float2 *>(src) + (values - 1);
        round_tail_kernel<<<1, 1, 0, s>>>(tail, static_cast<uint32_t *>(dst) + (values - 1));
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_tf32_w(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                               cudaStream_t s) {
    const int64_t rows = pl.p.w_batches * pl.p.M;
    const int grid = grid_for(rows * (pl.Kp / 4), 256, pl.num_sms);
    auto *d = static_cast<float *>(dst);
    if (src_type == TCBF_SRC_CF16)
        pack_tf32_w_kernel<CF16><<<grid, 256, 0, s>>>(src, d, rows, pl.p.M, int(pl.p.K), int(pl.Kp));
    else
        pack_tf32_w_kernel<CF32><<<grid, 256, 0, s>>>(src, d, rows, pl.p.M, int(pl.p.K), int(pl.Kp));
    return cudaGetLastError();
}

cudaError_t launch_pack_tf32_x(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                               cudaStream_t s) {
    const int k_tiles = static_cast<int>(ceil_div(pl.Kp, 32));
    const int n_tiles = static_cast<int>(ceil_div(pl.p.N, 32));
    const int64_t per_b = int64_t(k_tiles) * n_tiles;
    const int bx = static_cast<int>(std::min<int64_t>(per_b, std::max<int64_t>(1, int64_t(pl.num_sms) * 8 / std::max<int64_t>(1, std::min<int64_t>(pl.p.batch, 8)))));
    dim3 grid(bx, static_cast<unsigned>(pl.p.batch));
    auto *d = static_cast<float *>(dst);
    const int K = int(pl.p.K), N = int(pl.p.N), Kp = int(pl.Kp);
    if (src_type == TCBF_SRC_CF16)
        pack_tf32_x_kernel<CF16><<<grid, 256, 0, s>>>(src, d, K, N, Kp, k_tiles, n_tiles);
    else
        pack_tf32_x_kernel<CF32><<<grid, 256, 0, s>>>(src, d, K, N, Kp, k_tiles, n_tiles);
    return cudaGetLastError();
}

cudaError_t launch_pack_bits_w(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                               cudaStream_t s) {
    const int64_t rows = pl.p.w_batches * pl.p.M;
    const int grid = grid_for(rows * pl.Kw * 32, 256, pl.num_sms);
    auto *d = static_cast<uint32_t *>(dst);
    if (src_type == TCBF_SRC_CF16)
        pack_bits_w_kernel<CF16><<<grid, 256, 0, s>>>(src, d, rows, pl.p.M, int(pl.p.K), int(pl.Kw));
    else
        pack_bits_w_kernel<CF32><<<grid, 256, 0, s>>>(src, d, rows, pl.p.M, int(pl.p.K), int(pl.Kw));
    return cudaGetLastError();
}

cudaError_t launch_pack_bits_x(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                               cudaStream_t s) {
    const int n_groups = static_cast<int>(ceil_div(pl.p.N, 32));
    const int64_t per_b = int64_t(pl.Kw) * n_groups * 32;
    const int bx = std::max(1, std::min(grid_for(per_b, 256, pl.num_sms), 4096));
    dim3 grid(bx, static_cast<unsigned>(pl.p.batch));
    auto *d = static_cast<uint32_t *>(dst);
    if (src_type == TCBF_SRC_CF16)
        pack_bits_x_kernel<CF16><<<grid, 256, 0, s>>>(src, d, int(pl.p.K), int(pl.p.N), int(pl.Kw), n_groups);
    else
        pack_bits_x_kernel<CF32><<<grid, 256, 0, s>>>(src, d, int(pl.p.K), int(pl.p.N), int(pl.Kw), n_groups);
    return cudaGetLastError();
}

}  // namespace tcbf

// ===========================================================================
// Split-FP8 packing.  Each packed row (one beam of W, one sample of X, one
// plane) holds K in 64-element blocks of 64 E4M3 "hi" bytes then 64 E4M3
// "lo" bytes (HI: hi bytes only, 64 per block, for plans that keep the hi
// product alone); int32 scale exponents follow the data, one per row (shared
// by both planes).  With e the largest integer such that amax * 2^e <= 448
// (amax over the row's K elements and both planes), hi = RN(v 2^e) and
// lo = RN(v 2^e - hi), both saturating.  FP32 sources are first rounded to
// FP16, so every mode sees the same input values.
// ===========================================================================
#include <cuda_fp8.h>

namespace tcbf {
namespace {

__device__ __forceinline__ int split_exponent(float amax) {
    if (!(amax > 0.f)) return 0;
    int q;
    const float f = frexpf(amax, &q);          // amax = f 2^q, f in [0.5, 1)
    int e = (f <= 0.875f) ? 9 - q : 8 - q;     // 448 = 0.875 * 2^9
    return max(-100, min(100, e));
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ uint8_t e4m3(float x) {
    return static_cast<uint8_t>(__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3));
}

__device__ __forceinline__ float e4m3_to_float(uint8_t b) {
    return __half2float(__half(__nv_cvt_fp8_to_halfraw(b, __NV_E4M3)));
}

// hi and lo bytes of one value already scaled by 2^e
__device__ __forceinline__ void split_value(float v, uint8_t &hi, uint8_t &lo) {
    hi = e4m3(v);
    lo = e4m3(v - e4m3_to_float(hi));
}

// The same for two values at once (paired conversions): hi and lo hold
// the bytes of (a, b) in their low and high byte.
__device__ __forceinline__ void split_pair(float a, float b, uint16_t &hi, uint16_t &lo) {
    const __nv_fp8x2_storage_t h = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const __half2 hb = __half2(__nv_cvt_fp8x2_to_halfraw2(h, __NV_E4M3));
    const float2 back = __half22float2(hb);
    hi = h;
    lo = __nv_cvt_float2_to_fp8x2(make_float2(a - back.x, b - back.y), __NV_SATFINITE, __NV_E4M3);
}

template <typename S>
__device__ __forceinline__ float2 load_f16_value(const void *src, size_t i) {
    __half re, im;
    S::load_h(src, i, re, im);
    return make_float2(__half2float(re), __half2float(im));
}

// W rows (no transpose): one warp per row.
template <typename S, bool HI>
__global__ void split8_rows_kernel(const void *__restrict__ src, uint8_t *__restrict__ dst,
                                   int32_t *__restrict__ exps, int64_t rows, int64_t M, int K,
                                   int Kb2) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t r = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; r < rows;
         r += warps_total) {
        float amax = 0.f;
        for (int k = lane; k < K; k += 32) {
            const float2 v = load_f16_value<S>(src, static_cast<size_t>(r) * K + k);
            amax = fmaxf(amax, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        const int e = split_exponent(amax);
        const float s = pow2f(e);
        const int64_t bw = r / M, m = r % M;
        uint8_t *row_re = dst + (static_cast<size_t>(bw * 2 + 0) * M + m) * Kb2;
        uint8_t *row_im = dst + (static_cast<size_t>(bw * 2 + 1) * M + m) * Kb2;
        constexpr int kBlk = HI ? 64 : 128;
        for (int j = 0; j < Kb2 / kBlk; ++j) {
            uint8_t h[2][2], l[2][2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int k = 64 * j + 2 * lane + q;
                float2 v = make_float2(0.f, 0.f);
                if (k < K) v = load_f16_value<S>(src, static_cast<size_t>(r) * K + k);
                split_value(v.x * s, h[0][q], l[0][q]);
                split_value(v.y * s, h[1][q], l[1][q]);
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

// ------------------------------------------------ block-scaled split FP8
// One value v scaled by 2^e: hi = RN(v 2^e), lo = RN(16 (v 2^e - hi)) (the
// lo part kept 16 times larger, its scale 2^-(e + 4)).
__device__ __forceinline__ void split_value_blk(float v, uint8_t &hi, uint8_t &lo) {
    hi = e4m3(v);
    lo = e4m3(16.f * (v - e4m3_to_float(hi)));
}

// UE8M0 code of the scale 2^-e of a block with exponent e.
__device__ __forceinline__ uint8_t ue8m0_code(int e) { return static_cast<uint8_t>(127 - e); }

// Byte of scale tile entry (row r of the tile's 128 or 64, byte j):
// [l][g][j] with r = 32 g + l.
__device__ __forceinline__ int sf_entry(int r, int j) { return (r & 31) * 16 + (r >> 5) * 4 + j; }

// W rows, block-scaled: one warp per row; per 64-k block of the row lanes
// 0-15 hold k 0-31 and lanes 16-31 k 32-63 (two values each), each half
// reducing its own 32-k block's largest magnitude over both planes.
template <typename S, bool HI>
__global__ void split8_rows_blk_kernel(const void *__restrict__ src, uint8_t *__restrict__ dst,
                                       uint8_t *__restrict__ sf, int64_t rows, int64_t M, int K,
                                       int Kb2, int stages) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = int64_t(gridDim.x) * (blockDim.x >> 5);
    const int64_t tiles = (M + kFp8BlkRowsW - 1) / kFp8BlkRowsW;
    for (int64_t r = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; r < rows;
         r += warps_total) {
        const int64_t bw = r / M, m = r % M;
        uint8_t *row_re = dst + (static_cast<size_t>(bw * 2 + 0) * M + m) * Kb2;
        uint8_t *row_im = dst + (static_cast<size_t>(bw * 2 + 1) * M + m) * Kb2;
        uint8_t *tile_base = sf + static_cast<size_t>(bw * tiles + m / kFp8BlkRowsW) * stages * kFp8BlkTile;
        const int rr = static_cast<int>(m % kFp8BlkRowsW);
        constexpr int kBlk = HI ? 64 : 128;
        for (int jj = 0; jj < Kb2 / kBlk; ++jj) {
            float2 v[2];
            float amax = 0.f;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int k = 64 * jj + 2 * lane + q;
                v[q] = make_float2(0.f, 0.f);
                if (k < K) v[q] = load_f16_value<S>(src, static_cast<size_t>(r) * K + k);
                amax = fmaxf(amax, fmaxf(fabsf(v[q].x), fabsf(v[q].y)));
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            const int e = split_exponent(amax);
            const float sc = pow2f(e);
            uint8_t h[2][2], l[2][2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                split_value_blk(v[q].x * sc, h[0][q], l[0][q]);
                split_value_blk(v[q].y * sc, h[1][q], l[1][q]);
            }
            *reinterpret_cast<uint16_t *>(row_re + kBlk * jj + 2 * lane) = h[0][0] | (h[0][1] << 8);
            *reinterpret_cast<uint16_t *>(row_im + kBlk * jj + 2 * lane) = h[1][0] | (h[1][1] << 8);
            if (!HI) {
                *reinterpret_cast<uint16_t *>(row_re + kBlk * jj + 64 + 2 * lane) = l[0][0] | (l[0][1] << 8);
                *reinterpret_cast<uint16_t *>(row_im + kBlk * jj + 64 + 2 * lane) = l[1][0] | (l[1][1] << 8);
            }
            if ((lane & 15) == 0) {
                const int b2 = lane >> 4;                  // 32-k block within the 64
                if (HI) {                                  // stages of 128 k: 4 hi codes
                    uint8_t *t = tile_base + static_cast<size_t>(jj / 2) * kFp8BlkTile;
                    t[sf_entry(rr, 2 * (jj & 1) + b2)] = ue8m0_code(e);
                } else {                                   // stages of 64 k: 2 hi, 2 lo codes
                    uint8_t *t = tile_base + static_cast<size_t>(jj) * kFp8BlkTile;
                    t[sf_entry(rr, b2)] = ue8m0_code(e);
                    t[sf_entry(rr, 2 + b2)] = ue8m0_code(e + 4);
                }
            }
        }
    }
}

// X transpose + block-scaled split: 64 (k) x 64 (n) tiles as in
// split8_pack_x_kernel, with each (sample, 32-k block) exponent taken from
// the tile itself; the tile's 64 samples are one X scale group.
template <typename S, bool HI>
__global__ void __launch_bounds__(256) split8_pack_x_blk_kernel(const void *__restrict__ src,
                                                               uint8_t *__restrict__ dst,
                                                               uint8_t *__restrict__ sf, int K,
                                                               int N, int Kb2, int k_tiles,
                                                               int n_tiles, int stages) {
    __shared__ __half sre[TT][TPITCH];
    __shared__ __half sim[TT][TPITCH];
    __shared__ int es[TT][2];
    const int tid = threadIdx.x;
    const int64_t b = blockIdx.y;
    const int64_t tiles_per_b = int64_t(k_tiles) * n_tiles;
    for (int64_t t = blockIdx.x; t < tiles_per_b; t += gridDim.x) {
        const int kt = static_cast<int>(t / n_tiles);
        const int nt = static_cast<int>(t % n_tiles);
        const int k0 = kt * TT, n0 = nt * TT;
        const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int kk = ty + 16 * i;
            const int k = k0 + kk;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int nn = tx * 4 + q;
                const int n = n0 + nn;
                __half re = __float2half_rn(0.f), im = __float2half_rn(0.f);
                if (k < K && n < N) S::load_h(src, (static_cast<size_t>(b) * K + k) * N + n, re, im);
                sre[nn][kk] = re;
                sim[nn][kk] = im;
            }
        }
        __syncthreads();
        // exponents of the tile's (sample, 32-k block) pairs, and their codes
        if (tid < 2 * TT) {
            const int nn = tid >> 1, b2 = tid & 1;
            float amax = 0.f;
            for (int j = 0; j < 32; ++j) {
                amax = fmaxf(amax, fabsf(__half2float(sre[nn][32 * b2 + j])));
                amax = fmaxf(amax, fabsf(__half2float(sim[nn][32 * b2 + j])));
            }
            const int e = split_exponent(amax);
            es[nn][b2] = e;
            if (n0 + nn < N) {
                uint8_t *tile = sf + (static_cast<size_t>(b) * n_tiles + nt) * stages * kFp8BlkTile;
                if (HI) {
                    tile[static_cast<size_t>(kt / 2) * kFp8BlkTile + sf_entry(nn, 2 * (kt & 1) + b2)] =
                        ue8m0_code(e);
                } else {
                    tile[static_cast<size_t>(kt) * kFp8BlkTile + sf_entry(nn, b2)] = ue8m0_code(e);
                    tile[static_cast<size_t>(kt) * kFp8BlkTile + sf_entry(nn, 2 + b2)] = ue8m0_code(e + 4);
                }
            }
        }
        __syncthreads();
        // thread -> (row nn, 16-byte chunk c of 8: 4 hi chunks then 4 lo chunks)
        const int c = tid & 7;
        constexpr int kBlk = HI ? 64 : 128;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int nn = (tid >> 3) + 32 * h;
            const int n = n0 + nn;
            if (n < N && !(HI && c >= 4)) {
                const int kc = 16 * (c & 3);
                const float sc = pow2f(es[nn][kc >> 5]);
                const bool want_lo = c >= 4;
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    __align__(16) uint8_t out[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float v = __half2float(p == 0 ? sre[nn][kc + j] : sim[nn][kc + j]) * sc;
                        uint8_t hi, lo;
                        split_value_blk(v, hi, lo);
                        out[j] = want_lo ? lo : hi;
                    }
                    uint8_t *row = dst + (static_cast<size_t>(b * 2 + p) * N + n) * Kb2 + kt * kBlk;
                    *reinterpret_cast<uint4 *>(row + 16 * c) = *reinterpret_cast<const uint4 *>(out);
                }
            }
        }
        __syncthreads();
    }
}

// X columns: the largest magnitude per (batch, sample) over K, reduced in
// parallel: each thread scans 256 rows of one sample (consecutive threads
// read consecutive samples of a row of X) and folds its maximum into the
// exponent slot with an integer atomic max (valid for non-negative floats),
// which holds the float's bits until split8_exps_kernel converts it.
template <typename S>
__global__ void split8_amax_x_kernel(const void *__restrict__ src, int32_t *__restrict__ slot,
                                     int64_t B, int K, int N, int k_chunks) {
    const int64_t total = B * N * k_chunks;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t n = i % N;
        const int64_t rest = i / N;
        const int kc = static_cast<int>(rest % k_chunks);
        const int64_t b = rest / k_chunks;
        float amax = 0.f;
        const int k1 = min(K, (kc + 1) * 256);
        for (int k = kc * 256; k < k1; ++k) {
            const float2 v = load_f16_value<S>(src, (static_cast<size_t>(b) * K + k) * N + n);
            amax = fmaxf(amax, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
        atomicMax(slot + b * N + n, __float_as_int(amax));
    }
}

__global__ void split8_exps_kernel(int32_t *__restrict__ slot, int64_t rows) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < rows;
         i += int64_t(gridDim.x) * blockDim.x)
        slot[i] = split_exponent(__int_as_float(slot[i]));
}

// X transpose + split: 64 (k) x 64 (n) tiles; each output row of a tile is
// one K block: 64 hi bytes and 64 lo bytes per plane (HI: 64 hi bytes).
template <typename S, bool HI>
__global__ void __launch_bounds__(256) split8_pack_x_kernel(const void *__restrict__ src,
                                                           uint8_t *__restrict__ dst,
                                                           const int32_t *__restrict__ exps,
                                                           int K, int N, int Kb2, int k_tiles,
                                                           int n_tiles) {
    __shared__ __half sre[TT][TPITCH];
    __shared__ __half sim[TT][TPITCH];
    const int tid = threadIdx.x;
    const int64_t b = blockIdx.y;
    const int64_t tiles_per_b = int64_t(k_tiles) * n_tiles;
    for (int64_t t = blockIdx.x; t < tiles_per_b; t += gridDim.x) {
        const int kt = static_cast<int>(t / n_tiles);
        const int nt = static_cast<int>(t % n_tiles);
        const int k0 = kt * TT, n0 = nt * TT;
        const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int kk = ty + 16 * i;
            const int k = k0 + kk;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int nn = tx * 4 + q;
                const int n = n0 + nn;
                __half re = __float2half_rn(0.f), im = __float2half_rn(0.f);
                if (k < K && n < N) S::load_h(src, (static_cast<size_t>(b) * K + k) * N + n, re, im);
                sre[nn][kk] = re;
                sim[nn][kk] = im;
            }
        }
        __syncthreads();
        // thread -> (row nn, 16-byte chunk c of 8: 4 hi chunks then 4 lo chunks)
        const int c = tid & 7;
        constexpr int kBlk = HI ? 64 : 128;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int nn = (tid >> 3) + 32 * h;
            const int n = n0 + nn;
            if (n < N && !(HI && c >= 4)) {
                const float s = pow2f(split_exponent(__int_as_float(exps[b * N + n])));
                const int kc = 16 * (c & 3);
                const bool want_lo = c >= 4;
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    __align__(16) uint8_t out[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float v = __half2float(p == 0 ? sre[nn][kc + j] : sim[nn][kc + j]) * s;
                        uint8_t hi, lo;
                        split_value(v, hi, lo);
                        out[j] = want_lo ? lo : hi;
                    }
                    uint8_t *row = dst + (static_cast<size_t>(b * 2 + p) * N + n) * Kb2 + kt * kBlk;
                    *reinterpret_cast<uint4 *>(row + 16 * c) = *reinterpret_cast<const uint4 *>(out);
                }
            }
        }
        __syncthreads();
    }
}

// X transpose + split in one pass when all of K fits on chip (K <= 320):
// a CTA of 8 TN threads takes TN samples of one batch, loads every K row of
// them (16-byte loads of four values into a word tile, column
// n ^ 4 ((k / 8) % (TN / 4))), takes each sample's largest magnitude over K
// and both planes, splits every value once into its hi and lo bytes into a
// staged output tile (rows of 2 x Kb2 bytes, padded by 16 so the row writes
// of a warp hit distinct banks), and writes the packed rows out
// contiguously.  Small tiles keep several CTAs per SM, so one CTA's loads
// overlap another's split and stores.
constexpr int kSplitFusedMaxK = 320;

template <int TN>
struct SplitFusedSmem {
    static __host__ __device__ int rows(int K) { return (K + 63) / 64 * 64; }
    static __host__ __device__ int out_pitch(int Kb2) { return 2 * Kb2 + 16; }
    static __host__ __device__ int bytes(int K, int Kb2) {
        return rows(K) * TN * 4 + TN * out_pitch(Kb2) + 8 * TN * 4 + TN * 4;
    }
};

template <typename S, bool VEC, int TN, bool HI>
__global__ void __launch_bounds__(8 * TN) split8_pack_x_fused_kernel(const void *__restrict__ src,
                                                                     uint8_t *__restrict__ dst,
                                                                     int32_t *__restrict__ exps,
                                                                     int64_t B, int K, int N,
                                                                     int Kb2) {
    using L = SplitFusedSmem<TN>;
    constexpr int SW = TN / 4 - 1;                        // column swizzle mask (in 4-word units)
    extern __shared__ __align__(16) uint8_t sm[];
    const int R = L::rows(K);                             // K rows incl. zero pad to 64
    const int pitch = L::out_pitch(Kb2);
    uint32_t *tile = reinterpret_cast<uint32_t *>(sm);                 // [R][TN] words
    uint8_t *out = sm + R * TN * 4;                                     // [TN][pitch]
    float *red = reinterpret_cast<float *>(out + TN * pitch);           // [8][TN]
    int *es = reinterpret_cast<int *>(red + 8 * TN);                    // [TN]
    const int tid = threadIdx.x;
    const int n_tiles = (N + TN - 1) / TN;
    const int64_t total = B * n_tiles;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const int64_t b = t / n_tiles;
        const int n0 = static_cast<int>(t % n_tiles) * TN;
        // load: TN / 4 threads per row, 32 rows per round
        const int q = tid % (TN / 4);
        for (int k = tid / (TN / 4); k < R; k += 32) {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            const int n = n0 + 4 * q;
            if (k < K) {
                const size_t e = (static_cast<size_t>(b) * K + k) * N + n;
                if (VEC && n + 3 < N) {
                    S::load4(src, e, w);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (n + j < N) w[j] = S::load_word(src, e + j);
                }
            }
            const int col = (4 * q) ^ (4 * ((k >> 3) & SW));
            *reinterpret_cast<uint4 *>(&tile[k * TN + col]) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        __syncthreads();
        // largest magnitude per sample: 8 threads per sample, then combined
        {
            const int n = tid % TN, part = tid / TN;
            float amax = 0.f;
            for (int k = part; k < R; k += 8) {
                const uint32_t v = tile[k * TN + (n ^ (4 * ((k >> 3) & SW)))];
                const __half2 h = *reinterpret_cast<const __half2 *>(&v);
                amax = fmaxf(amax, fmaxf(fabsf(__low2float(h)), fabsf(__high2float(h))));
            }
            red[part * TN + n] = amax;
        }
        __syncthreads();
        if (tid < TN) {
            float amax = 0.f;
#pragma unroll
            for (int p = 0; p < 8; ++p) amax = fmaxf(amax, red[p * TN + tid]);
            const int e = split_exponent(amax);
            es[tid] = e;
            if (n0 + tid < N) exps[b * N + n0 + tid] = e;
        }
        __syncthreads();
        // split: item -> (sample n fastest, plane, 16-element chunk c); hi and lo of
        // every value once
        const int chunks = R / 16;
        for (int i = tid; i < TN * 2 * chunks; i += 8 * TN) {
            const int n = i % TN;
            const int p = (i / TN) & 1;
            const int c = i / (2 * TN);
            const float s = pow2f(es[n]);
            __align__(16) uint16_t hi[8], lo[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = 16 * c + 2 * j;
                const uint32_t v0 = tile[k * TN + (n ^ (4 * ((k >> 3) & SW)))];
                const uint32_t v1 = tile[(k + 1) * TN + (n ^ (4 * (((k + 1) >> 3) & SW)))];
                const __half2 h0 = *reinterpret_cast<const __half2 *>(&v0);
                const __half2 h1 = *reinterpret_cast<const __half2 *>(&v1);
                const float a = (p == 0 ? __low2float(h0) : __high2float(h0)) * s;
                const float b = (p == 0 ? __low2float(h1) : __high2float(h1)) * s;
                split_pair(a, b, hi[j], lo[j]);
            }
            uint8_t *row = out + n * pitch + p * Kb2 + (c >> 2) * (HI ? 64 : 128) + (c & 3) * 16;
            *reinterpret_cast<uint4 *>(row) = *reinterpret_cast<const uint4 *>(hi);
            if (!HI) *reinterpret_cast<uint4 *>(row + 64) = *reinterpret_cast<const uint4 *>(lo);
        }
        __syncthreads();
        // write the packed rows: 16-byte chunks, consecutive threads along a row
        const int row_chunks = Kb2 / 16;
        for (int i = tid; i < TN * 2 * row_chunks; i += 8 * TN) {
            const int j = i % row_chunks;
            const int rp = i / row_chunks;               // sample-major: (n, p)
            const int n = rp >> 1, p = rp & 1;
            if (n0 + n < N) {
                uint8_t *grow = dst + (static_cast<size_t>(b * 2 + p) * N + n0 + n) * Kb2;
                *reinterpret_cast<uint4 *>(grow + 16 * j) =
                    *reinterpret_cast<const uint4 *>(out + n * pitch + p * Kb2 + 16 * j);
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_pack_split8_w(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                                 cudaStream_t s) {
    const int64_t rows = pl.p.w_batches * pl.p.M;
    const int Kb2 = static_cast<int>(pl.Kb2);
    auto *d = static_cast<uint8_t *>(dst);
    if (fp8_block_scaled(pl.p.flags)) {
        // scale tiles: 127 (2^0) everywhere first, so rows beyond M hold a valid code
        uint8_t *sf = d + rows * 2 * Kb2;
        const int64_t sfb = fp8blk_sf_bytes(pl.p.w_batches, pl.p.M, pl.p.K, pl.p.flags, 0);
        cudaError_t e = cudaMemsetAsync(sf, 127, static_cast<size_t>(sfb), s);
        if (e != cudaSuccess) return e;
        const int grid = grid_for(rows * 32, 256, pl.num_sms);
        const int st = static_cast<int>(fp8blk_stages(pl.p.K, pl.p.flags));
        const int K = static_cast<int>(pl.p.K);
        auto run = [&](auto kern) { kern<<<grid, 256, 0, s>>>(src, d, sf, rows, pl.p.M, K, Kb2, st); };
        const bool hi = fp8_hi_only(pl.p.flags);
        if (src_type == TCBF_SRC_CF16)
            hi ? run(split8_rows_blk_kernel<CF16, true>) : run(split8_rows_blk_kernel<CF16, false>);
        else
            hi ? run(split8_rows_blk_kernel<CF32, true>) : run(split8_rows_blk_kernel<CF32, false>);
        return cudaGetLastError();
    }
    auto *ex = reinterpret_cast<int32_t *>(d + rows * 2 * Kb2);
    const int grid = grid_for(rows * 32, 256, pl.num_sms);
    const bool hi = fp8_hi_only(pl.p.flags);
    const int K = static_cast<int>(pl.p.K);
    if (src_type == TCBF_SRC_CF16) {
        if (hi) split8_rows_kernel<CF16, true><<<grid, 256, 0, s>>>(src, d, ex, rows, pl.p.M, K, Kb2);
        else split8_rows_kernel<CF16, false><<<grid, 256, 0, s>>>(src, d, ex, rows, pl.p.M, K, Kb2);
    } else {
        if (hi) split8_rows_kernel<CF32, true><<<grid, 256, 0, s>>>(src, d, ex, rows, pl.p.M, K, Kb2);
        else split8_rows_kernel<CF32, false><<<grid, 256, 0, s>>>(src, d, ex, rows, pl.p.M, K, Kb2);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_split8_x(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                                 cudaStream_t s) {
    const int64_t B = pl.p.batch, N = pl.p.N;
    const int Kb2 = static_cast<int>(pl.Kb2);
    auto *d = static_cast<uint8_t *>(dst);
    if (fp8_block_scaled(pl.p.flags)) {
        uint8_t *sf = d + B * 2 * N * Kb2;
        const int64_t sfb = fp8blk_sf_bytes(B, N, pl.p.K, pl.p.flags, 1);
        cudaError_t e = cudaMemsetAsync(sf, 127, static_cast<size_t>(sfb), s);
        if (e != cudaSuccess) return e;
        static_assert(TT == kFp8BlkRowsX, "one transpose tile of samples per X scale group");
        const int k_tiles = static_cast<int>(ceil_div(pl.p.K, TT));
        const int n_tiles = static_cast<int>(ceil_div(N, TT));
        const int64_t per_b = int64_t(k_tiles) * n_tiles;
        const int bx = static_cast<int>(std::min<int64_t>(per_b, std::max<int64_t>(1, int64_t(pl.num_sms) * 8 / std::max<int64_t>(1, std::min<int64_t>(B, 8)))));
        dim3 grid(bx, static_cast<unsigned>(B));
        const int st = static_cast<int>(fp8blk_stages(pl.p.K, pl.p.flags));
        const int K = static_cast<int>(pl.p.K), Ni = static_cast<int>(N);
        auto run = [&](auto kern) {
            kern<<<grid, 256, 0, s>>>(src, d, sf, K, Ni, Kb2, k_tiles, n_tiles, st);
        };
        const bool hi = fp8_hi_only(pl.p.flags);
        if (src_type == TCBF_SRC_CF16)
            hi ? run(split8_pack_x_blk_kernel<CF16, true>) : run(split8_pack_x_blk_kernel<CF16, false>);
        else
            hi ? run(split8_pack_x_blk_kernel<CF32, true>) : run(split8_pack_x_blk_kernel<CF32, false>);
        return cudaGetLastError();
    }
    auto *ex = reinterpret_cast<int32_t *>(d + B * 2 * N * Kb2);
    const int g1 = grid_for(B * N, 256, pl.num_sms);
    const bool hi = fp8_hi_only(pl.p.flags);
    const int k_tiles = static_cast<int>(ceil_div(pl.p.K, 64));
    const int n_tiles = static_cast<int>(ceil_div(N, TT));
    const int64_t per_b = int64_t(k_tiles) * n_tiles;
    const int bx = static_cast<int>(std::min<int64_t>(per_b, std::max<int64_t>(1, int64_t(pl.num_sms) * 8 / std::max<int64_t>(1, std::min<int64_t>(B, 8)))));
    dim3 grid(bx, static_cast<unsigned>(B));
    const int k_chunks = static_cast<int>(ceil_div(pl.p.K, 256));
    const int g_amax = grid_for(B * N * k_chunks, 256, pl.num_sms);
    if (pl.p.K <= kSplitFusedMaxK) {
        constexpr int TN = 16;
        const int smem = SplitFusedSmem<TN>::bytes(int(pl.p.K), Kb2);
        const bool vec = N % 4 == 0;
        const int K = int(pl.p.K), Ni = int(N);
        auto launch = [&](auto kern) -> cudaError_t {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 8 * TN, smem);
            if (e != cudaSuccess) return e;
            const int64_t tiles = B * ceil_div(N, TN);
            const int g = static_cast<int>(std::min<int64_t>(tiles, int64_t(pl.num_sms) * std::max(1, per_sm)));
            kern<<<g, 8 * TN, smem, s>>>(src, d, ex, B, K, Ni, Kb2);
            return cudaGetLastError();
        };
        if (src_type == TCBF_SRC_CF16) {
            if (hi)
                return vec ? launch(split8_pack_x_fused_kernel<CF16, true, TN, true>)
                           : launch(split8_pack_x_fused_kernel<CF16, false, TN, true>);
            return vec ? launch(split8_pack_x_fused_kernel<CF16, true, TN, false>)
                       : launch(split8_pack_x_fused_kernel<CF16, false, TN, false>);
        }
        if (hi)
            return vec ? launch(split8_pack_x_fused_kernel<CF32, true, TN, true>)
                       : launch(split8_pack_x_fused_kernel<CF32, false, TN, true>);
        return vec ? launch(split8_pack_x_fused_kernel<CF32, true, TN, false>)
                   : launch(split8_pack_x_fused_kernel<CF32, false, TN, false>);
    }
    cudaError_t e = cudaMemsetAsync(ex, 0, sizeof(int32_t) * B * N, s);
    if (e != cudaSuccess) return e;
    const int K = static_cast<int>(pl.p.K), Ni = static_cast<int>(N);
    if (src_type == TCBF_SRC_CF16) {
        split8_amax_x_kernel<CF16><<<g_amax, 256, 0, s>>>(src, ex, B, K, Ni, k_chunks);
        if (hi) split8_pack_x_kernel<CF16, true><<<grid, 256, 0, s>>>(src, d, ex, K, Ni, Kb2, k_tiles, n_tiles);
        else split8_pack_x_kernel<CF16, false><<<grid, 256, 0, s>>>(src, d, ex, K, Ni, Kb2, k_tiles, n_tiles);
    } else {
        split8_amax_x_kernel<CF32><<<g_amax, 256, 0, s>>>(src, ex, B, K, Ni, k_chunks);
        if (hi) split8_pack_x_kernel<CF32, true><<<grid, 256, 0, s>>>(src, d, ex, K, Ni, Kb2, k_tiles, n_tiles);
        else split8_pack_x_kernel<CF32, false><<<grid, 256, 0, s>>>(src, d, ex, K, Ni, Kb2, k_tiles, n_tiles);
    }
    split8_exps_kernel<<<g1, 256, 0, s>>>(ex, B * N);
    return cudaGetLastError();
}

}  // namespace tcbf
