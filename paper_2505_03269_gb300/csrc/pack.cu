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
};

int grid_for(int64_t work, int threads, int num_sms) {
    const int64_t blocks = (work + threads - 1) / threads;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(blocks, int64_t(num_sms) * 16)));
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

// X: 64 (k) x 64 (n) tiles through shared memory.  Loads read rows of X
// (n contiguous); stores write rows of the packed planes (k contiguous),
// eight threads per 128-byte row.
constexpr int TT = 64;
constexpr int TPITCH = TT + 2;   // halves; odd word pitch spreads banks

template <typename S>
__global__ void __launch_bounds__(256) pack_f16_x_kernel(const void *__restrict__ src,
                                                        __half *__restrict__ dst, int K, int N,
                                                        int Kp, int k_tiles, int n_tiles) {
    __shared__ __half sre[TT][TPITCH];
    __shared__ __half sim[TT][TPITCH];
    const int tid = threadIdx.x;
    const int64_t tiles_per_b = int64_t(k_tiles) * n_tiles;
    const int64_t b = blockIdx.y;
    for (int64_t t = blockIdx.x; t < tiles_per_b; t += gridDim.x) {
        const int kt = static_cast<int>(t / n_tiles);
        const int nt = static_cast<int>(t % n_tiles);
        const int k0 = kt * TT, n0 = nt * TT;
        // load: thread (ty, tx) reads 4 consecutive n at rows ty + 16 i
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
        // store: thread -> (row n, 16-byte chunk c); two rows per thread
        const int c = tid & 7;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int nn = (tid >> 3) + 32 * h;
            const int n = n0 + nn;
            const int k = k0 + 8 * c;
            if (n < N && k < Kp) {
                __align__(16) __half re[8], im[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    re[j] = sre[nn][8 * c + j];
                    im[j] = sim[nn][8 * c + j];
                }
                const size_t o_re = (static_cast<size_t>(b * 2 + 0) * N + n) * Kp + k;
                const size_t o_im = (static_cast<size_t>(b * 2 + 1) * N + n) * Kp + k;
                *reinterpret_cast<uint4 *>(dst + o_re) = *reinterpret_cast<const uint4 *>(re);
                *reinterpret_cast<uint4 *>(dst + o_im) = *reinterpret_cast<const uint4 *>(im);
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

}  // namespace

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
    if (src_type == TCBF_SRC_CF16)
        pack_f16_x_kernel<CF16><<<grid, 256, 0, s>>>(src, d, int(pl.p.K), int(pl.p.N), int(pl.Kp), k_tiles, n_tiles);
    else
        pack_f16_x_kernel<CF32><<<grid, 256, 0, s>>>(src, d, int(pl.p.K), int(pl.p.N), int(pl.Kp), k_tiles, n_tiles);
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
