// gemm_1bit_fp4.cu — exact 1-bit complex GEMM on the 4-bit tensor path.
//
// The +-1 +-i values of the 1-bit mode (Fig. 1: bit 1 = +1, bit 0 = -1) are
// exact in E2M1 (+1 = 0x2, -1 = 0xA, and 0x0 for k >= K, so no padding
// correction as in Eq. 5 is needed), and the block-scaled 4-bit MMAs
// (kind::mxf4, every UE8M0 scale 2^0) run at a multiple of the FP8 rate.
// Each call expands the packed bits into E2M1 planes in plan-owned device
// memory (one pass over the packed words, writing four times their bytes),
// then multiplies them on SM pairs with stacked sample planes, as the
// stacked FP16 kernel does: W planes Wr, Wi; X planes -Xi, Xr, Xi;
//     Wr [Xr; Xi] + Wi [-Xi; Xr] = [Re | Im]
// two M = 256, N = 2 SBN MMAs per 64-K step.  kind::mxf4 has no negate bit,
// so the sign sits in the -Xi plane.  Every partial sum is an integer of
// magnitude <= 2K, exact in FP32 for K <= 2^23, so Y equals K - 2 Hamming
// (Eq. 4) exactly, as with the E4M3 kernel.
//
// Warp roles (192 threads per CTA, clusters of two CTAs on two SMs):
//   warp 0      TMA producer, both CTAs: this CTA's 128 rows of Wr and Wi
//               and its half of each B operand (even CTA Xr and -Xi, odd CTA
//               Xi and Xr), 128 bytes (256 K) of each row per stage, all
//               completing on the even CTA's full barrier
//   warp 1      TMEM owner; in the even CTA the single-thread MMA issuer
//   warps 2-5   scale-factor fill at start, then the epilogue: TMEM ->
//               int32 pairs -> staged TMA stores (two buffers per warp),
//               releasing an accumulator on the even CTA's barrier
// Tensor memory: the accumulators from column 0 (two of them at columns 0
// and a multiple of 64), the scale factors in the columns above them up to
// 512 (from 256, 384 for two 192-column accumulators, 480 for two of 224
// columns at 0 and 256), every byte UE8M0 127, so any scale layout the MMA
// reads returns 1.0.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cstring>

#include "ptx.cuh"
#include "tcbf_internal.h"

namespace tcbf {
namespace {

using namespace dev;

constexpr int kRowBytes = 128;     // bytes of each row per stage: 256 E2M1 values
constexpr int kStageK = 256;
constexpr int64_t kMaxExactK = int64_t(1) << 23;
// Tile order: groups of kGroupM pair rows (256 W rows each), samples
// fastest within a group, so the clusters running at one time share both
// their W rows and their X columns in L2 (with samples fastest over all
// rows, a long-K product streams all of X from memory once per pair row).
constexpr int kGroupM = 8;

// 8 sign bits -> 8 E2M1 nibbles, element j in nibble j (low nibble first):
// bit 1 -> 0x2 (+1), bit 0 -> 0xA (-1), NEG swaps the two; elements at or
// beyond `valid` (of this byte) are 0.  The three masked shifts move bit j
// to bit 4j.
template <bool NEG>
__device__ __forceinline__ uint32_t e2m1_byte(uint32_t byte, int valid) {
    uint32_t x = byte & 0xFFu;
    x = (x | (x << 12)) & 0x000F000Fu;
    x = (x | (x << 6)) & 0x03030303u;
    x = (x | (x << 3)) & 0x11111111u;
    uint32_t v = (NEG ? 0x22222222u : 0xAAAAAAAAu) ^ (x << 3);
    if (valid < 8) v &= valid <= 0 ? 0u : (0xFFFFFFFFu >> (32 - 4 * valid));
    return v;
}

// One packed word (32 elements, element j at bit j) -> 16 bytes of E2M1.
template <bool NEG>
__device__ __forceinline__ uint4 e2m1_word(uint32_t w, int valid) {
    return make_uint4(e2m1_byte<NEG>(w, valid), e2m1_byte<NEG>(w >> 8, valid - 8),
                      e2m1_byte<NEG>(w >> 16, valid - 16), e2m1_byte<NEG>(w >> 24, valid - 24));
}

// E2M1 rows hold Kq = Kw rounded up to 8 words (16 bytes each), so every row
// starts on a 128-byte line: each 128-byte box row of the GEMM's tensor loads
// is then one whole line.  Words at or beyond Kw (k >= K) are 0.

// W bits [w_batches][2][w_rows][Kw] -> E2M1 [w_batches][2][M][Kq x 16 bytes].
__global__ void expand_w_fp4_kernel(const uint32_t *__restrict__ Wb, uint4 *__restrict__ Wq,
                                    int64_t rows, int M, int64_t w_rows, int Kw, int Kq, int K) {
    const int64_t total = rows * Kq;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = i / Kq;
        const int w = static_cast<int>(i - r * Kq);
        const int64_t plane = r / M;
        const int64_t m = r - plane * M;
        const uint32_t bits = w < Kw ? __ldg(Wb + (plane * w_rows + m) * Kw + w) : 0u;
        Wq[i] = e2m1_word<false>(bits, K - 32 * w);
    }
}

// X bits [batch][2][N][Kw] -> E2M1 planes [batch][3][N][Kq x 16 bytes]:
// -Xi, Xr, Xi.
__global__ void expand_x_fp4_kernel(const uint32_t *__restrict__ Xb, uint4 *__restrict__ Xq,
                                    int64_t batch, int64_t N, int Kw, int Kq, int K) {
    const int64_t total = batch * N * Kq;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = i / Kq;            // b * N + n
        const int w = static_cast<int>(i - r * Kq);
        const int64_t b = r / N;
        const int64_t n = r - b * N;
        const uint32_t xr = w < Kw ? __ldg(Xb + ((b * 2) * N + n) * Kw + w) : 0u;
        const uint32_t xi = w < Kw ? __ldg(Xb + ((b * 2 + 1) * N + n) * Kw + w) : 0u;
        const int valid = K - 32 * w;
        Xq[((b * 3) * N + n) * Kq + w] = e2m1_word<true>(xi, valid);
        Xq[((b * 3 + 1) * N + n) * Kq + w] = e2m1_word<false>(xr, valid);
        Xq[((b * 3 + 2) * N + n) * Kq + w] = e2m1_word<false>(xi, valid);
    }
}

// Sign of one source component as the 1-bit pack takes it: v >= 0 gives
// +1 (so -0 gives +1), anything else (negative, NaN) -1.
__device__ __forceinline__ uint32_t sign_of(float v) { return v >= 0.f ? 1u : 0u; }

__device__ __forceinline__ void load_cf(const void *src, size_t i, bool f32, float &re, float &im) {
    if (f32) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(src) + i);
        re = v.x;
        im = v.y;
    } else {
        const __half2 v = __ldg(reinterpret_cast<const __half2 *>(src) + i);
        re = __low2float(v);
        im = __high2float(v);
    }
}

// Interleaved complex X [batch][K][N] -> E2M1 planes [batch][3][N][Kq x 16
// bytes] (-Xi, Xr, Xi) in one pass, without the packed bits.  A block of
// 256 threads takes 128 samples x 256 k (8 words): warp w reads the 32 rows
// of word w, lane l samples n0 + 4l .. n0 + 4l + 3 (one 16-byte load of FP16
// values per row when N % 4 == 0, so a warp reads 512 contiguous bytes of a
// row; else one value at a time); the sign words go through shared memory,
// and the block writes each sample's 8 words as 128 contiguous bytes per
// plane.
constexpr int kPackSamples = 128;
constexpr int kPackWords = 8;

template <bool F32, bool VEC>
__global__ void __launch_bounds__(256) pack_x_fp4_kernel(const void *__restrict__ src,
                                                         uint8_t *__restrict__ Xq, int K, int N,
                                                         int Kw, int Kq, int n_tiles, int w_tiles) {
    __shared__ uint32_t bits[2][kPackSamples][kPackWords + 1];   // [re/im][sample][word]
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t b = blockIdx.y;
    const size_t row = static_cast<size_t>(Kq) * 16;
    for (int t = blockIdx.x; t < n_tiles * w_tiles; t += gridDim.x) {
        const int n0 = (t % n_tiles) * kPackSamples;
        const int w0 = (t / n_tiles) * kPackWords;
        const int w = w0 + warp;                       // this warp's word
        const int k0 = 32 * w;
        const int kend = w < Kw ? max(0, min(32, K - k0)) : 0;
        const int nl = n0 + 4 * lane;                  // this lane's first sample
        uint32_t wr[4] = {0u, 0u, 0u, 0u}, wi[4] = {0u, 0u, 0u, 0u};
        if (VEC && nl + 4 <= N) {
#pragma unroll 4
            for (int j = 0; j < kend; ++j) {
                const size_t i = (static_cast<size_t>(b) * K + k0 + j) * N + nl;
                float v[8];
                if (F32) {
                    const float4 p = __ldg(reinterpret_cast<const float4 *>(src) + i / 2);
                    const float4 q = __ldg(reinterpret_cast<const float4 *>(src) + i / 2 + 1);
                    v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w;
                    v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
                } else {
                    const uint4 p = __ldg(reinterpret_cast<const uint4 *>(src) + i / 4);
                    const uint32_t u[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const __half2 h = *reinterpret_cast<const __half2 *>(&u[q]);
                        v[2 * q] = __low2float(h);
                        v[2 * q + 1] = __high2float(h);
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    wr[q] |= sign_of(v[2 * q]) << j;
                    wi[q] |= sign_of(v[2 * q + 1]) << j;
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (nl + q >= N) break;
                for (int j = 0; j < kend; ++j) {
                    float re, im;
                    load_cf(src, (static_cast<size_t>(b) * K + k0 + j) * N + nl + q, F32, re, im);
                    wr[q] |= sign_of(re) << j;
                    wi[q] |= sign_of(im) << j;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            bits[0][4 * lane + q][warp] = wr[q];
            bits[1][4 * lane + q][warp] = wi[q];
        }
        __syncthreads();
        // 3 planes x 128 samples x 8 words of 16 bytes; 8 consecutive threads
        // write one sample's 128 bytes of a plane
        for (int c = threadIdx.x; c < 3 * kPackSamples * kPackWords; c += 256) {
            const int plane = c / (kPackSamples * kPackWords);
            const int sr = (c / kPackWords) % kPackSamples;
            const int wd = c % kPackWords;
            const int n = n0 + sr, ww = w0 + wd;
            if (n >= N || ww >= Kq) continue;
            const int valid = K - 32 * ww;
            // planes -Xi (0), Xr (1), Xi (2)
            const uint32_t v = bits[plane == 1 ? 0 : 1][sr][wd];
            const uint4 q = plane == 0 ? e2m1_word<true>(v, valid) : e2m1_word<false>(v, valid);
            *reinterpret_cast<uint4 *>(Xq + ((static_cast<size_t>(b) * 3 + plane) * N + n) * row +
                                       16 * static_cast<size_t>(ww)) = q;
        }
        __syncthreads();
    }
}

// Interleaved complex W [w_batches][M][K] -> E2M1 planes [w_batches][2][M]
// [Kq x 16 bytes] (Wr, Wi): one warp per row and word, lane l reads k = 32 w
// + l, a ballot forms each plane's word and two lanes write its 16 bytes.
template <bool F32>
__global__ void pack_w_fp4_kernel(const void *__restrict__ src, uint4 *__restrict__ Wq,
                                  int64_t rows, int64_t M, int K, int Kq) {
    const int lane = threadIdx.x & 31;
    const int64_t warps_total = int64_t(gridDim.x) * (blockDim.x >> 5);
    const int64_t total = rows * Kq;
    for (int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; i < total;
         i += warps_total) {
        const int64_t r = i / Kq;
        const int w = static_cast<int>(i % Kq);
        const int k = 32 * w + lane;
        float re = -1.f, im = -1.f;
        if (k < K) load_cf(src, static_cast<size_t>(r) * K + k, F32, re, im);
        const uint32_t br = __ballot_sync(0xffffffffu, k < K && sign_of(re));
        const uint32_t bi = __ballot_sync(0xffffffffu, k < K && sign_of(im));
        const int64_t bw = r / M, m = r % M;
        const int valid = K - 32 * w;
        if (lane < 2) {
            const uint4 v = e2m1_word<false>(lane == 0 ? br : bi, valid);
            Wq[(static_cast<size_t>(bw * 2 + lane) * M + m) * Kq + w] = v;
        }
    }
}

struct Fp4Args {
    int32_t *Y;
    uint32_t *status;
    int tma_store;
    int M, N, K;
    int per_w;
    int m_pairs, n_tiles;     // 256-row pair tiles per batch, SBN-sample tiles
    int num_kb;               // 256-K stages
    int total_tiles;
};

// (batch, pair row, sample tile) of tile t: within a batch, groups of
// kGroupM pair rows (the last one possibly shorter), pair rows fastest
// inside a group, then sample tiles.
__device__ __forceinline__ void fp4_decode(int t, const Fp4Args &a, int &b, int &mp, int &nt) {
    const int per_b = a.m_pairs * a.n_tiles;
    b = t / per_b;
    const int local = t - b * per_b;
    const int group = local / (kGroupM * a.n_tiles);
    const int first = group * kGroupM;
    const int gm = min(kGroupM, a.m_pairs - first);
    const int in = local - group * kGroupM * a.n_tiles;
    mp = first + in % gm;
    nt = in / gm;
}

constexpr int kFp4Threads = 192;

template <int SBN, int STAGES>
struct CfgFp4 {
    static constexpr int W_PLANE = 128 * kRowBytes;            // 16 KB
    static constexpr int X_PLANE = SBN * kRowBytes;
    static constexpr int W_BYTES = 2 * W_PLANE;                 // Wr, Wi (this CTA's rows)
    static constexpr int STAGE_BYTES = W_BYTES + 2 * X_PLANE;  // + this CTA's halves of B1, B2
    static constexpr int ACC_COLS = 2 * SBN;                    // [Re | Im]
    // accumulators start at multiples of 64 columns
    static constexpr int ACC_STRIDE = (ACC_COLS + 63) / 64 * 64;
    static constexpr int TMEM_COLS = 512;
    // two accumulators when they leave at least 32 columns for the scales
    static constexpr int ACC_BUFS = ACC_STRIDE + ACC_COLS + 32 <= TMEM_COLS ? 2 : 1;
    // scale factors: A from SF_COL, B from the middle of the rest (the MMA
    // reads at most 4 columns of A's and 8 of B's; all of them hold 2^0)
    static constexpr int SF_COL = ((ACC_BUFS - 1) * ACC_STRIDE + ACC_COLS + 31) / 32 * 32;
    static constexpr int SFB_COL = SF_COL + (TMEM_COLS - SF_COL) / 2;
    // two 32 x 128-byte output buffers per epilogue warp: one store in
    // flight while the next block is staged (the output stream of short-K
    // products is bound by the stores a warp keeps in flight)
    static constexpr int STAGING_BYTES = 4 * 2 * 4096;
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + STAGING_BYTES + 256 + 1024;
    static_assert(SF_COL + 32 <= TMEM_COLS, "room for the scale columns");
    static_assert(SBN % 16 == 0 && SBN >= 32 && 2 * SBN <= 256, "pair N");
    static_assert(X_PLANE % 1024 == 0, "swizzle atoms");
    static_assert(SMEM_BYTES <= 232448, "shared memory");
};

__device__ __forceinline__ void st_shared_i4(uint32_t addr, int a, int b, int c, int d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
                 "r"(d)
                 : "memory");
}

template <int SBN, int STAGES>
__global__ void __launch_bounds__(kFp4Threads, 1)
    cgemm_1bit_fp4_pair_kernel(const __grid_constant__ CUtensorMap tmW,
                               const __grid_constant__ CUtensorMap tmX,
                               const __grid_constant__ CUtensorMap tmY, const Fp4Args args) {
    using C = CfgFp4<SBN, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
    const uint32_t s0 = smem_u32(smem);
    const uint32_t staging0 = s0 + STAGES * C::STAGE_BYTES;
    const uint32_t bar0 = staging0 + C::STAGING_BYTES;
    const uint32_t full0 = bar0;
    const uint32_t empty0 = full0 + 8 * STAGES;
    const uint32_t tfull0 = empty0 + 8 * STAGES;
    const uint32_t tempty0 = tfull0 + 16;
    const uint32_t done_bar = tempty0 + 16;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + STAGES * C::STAGE_BYTES +
                                                       C::STAGING_BYTES + 16 * STAGES + 40);
    volatile uint32_t *abort_flag = tmem_slot + 1;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int rank = static_cast<int>(cluster_ctarank());
    const bool leader = rank == 0;
    const int t_first = static_cast<int>(cluster_id_x());
    const int t_step = static_cast<int>(nclusters_x());
    constexpr uint16_t kBoth = 3;
    // packed planes -Xi (0), Xr (1), Xi (2): this CTA's rows of B1 and of B2
    const int plane_b1 = leader ? 1 : 2;
    const int plane_b2 = leader ? 0 : 1;
    auto decode = [&](int t, int &b, int &mp, int &nt) { fp4_decode(t, args, b, mp, nt); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);          // used in the even CTA
            mbar_init(empty0 + 8 * s, 1);         // the even CTA's commit, both CTAs
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, 8);        // 4 epilogue warps x 2 CTAs (even CTA)
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
        tma_prefetch_desc(&tmW);
        tma_prefetch_desc(&tmX);
        if (args.tma_store) tma_prefetch_desc(&tmY);
    }
    if (warp == 1) {
        tmem_alloc_pair(smem_u32(tmem_slot), C::TMEM_COLS);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // scale factors of A and B: every byte of columns [SF_COL, 512) is 2^0
    if (warp >= 2) {
        const uint32_t lane_off = static_cast<uint32_t>((warp & 3) * 32) << 16;
#pragma unroll 1
        for (int c = C::SF_COL; c < C::TMEM_COLS; c += 4)
            tmem_st_fill4(tmem_base + lane_off + c, 0x7F7F7F7Fu);
        tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();                       // both CTAs' scale columns are written
    tc_fence_after();
    const uint32_t full0_lead = mapa_shared(full0, 0);
    const uint32_t tempty0_lead = mapa_shared(tempty0, 0);

    if (warp == 0) {
        // --------------------------------------------- TMA producer, both CTAs
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued = 0;
            bool ok = true;
            for (int t = t_first; t < args.total_tiles && ok; t += t_step) {
                int b, mp, nt;
                decode(t, b, mp, nt);
                const int bw = b / args.per_w;
                for (int kb = 0; kb < args.num_kb; ++kb) {
                    if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = full0_lead + 8 * stage;
                    if (leader) mbar_arrive_expect_tx(full0 + 8 * stage, 2 * C::STAGE_BYTES);
                    const uint32_t dst = s0 + stage * C::STAGE_BYTES;
                    const int x = kb * kRowBytes;
                    tma_load_3d_pair(dst, &tmW, fb, x, mp * 256 + 128 * rank, 2 * bw);
                    tma_load_3d_pair(dst + C::W_BYTES, &tmX, fb, x, nt * SBN, 3 * b + plane_b1);
                    tma_load_3d_pair(dst + C::W_BYTES + C::X_PLANE, &tmX, fb, x, nt * SBN,
                                     3 * b + plane_b2);
                    ++issued;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                atomicOr(args.status, kErrTimeoutProducer);
                *abort_flag = 1;
                if (leader) {
                    for (int s = 0; s < STAGES; ++s) {
                        if (issued > static_cast<uint32_t>(s)) {
                            const uint32_t count = (issued - s + STAGES - 1) / STAGES;
                            if (!mbar_wait(full0 + 8 * s, (count - 1) & 1u))
                                atomicOr(args.status, kErrTimeoutDrain);
                        }
                    }
                }
            } else {
                // the even CTA's release of every slot this CTA filled has arrived
                for (int s = 0; s < STAGES; ++s) {
                    if (issued > static_cast<uint32_t>(s)) {
                        const uint32_t count = (issued - s + STAGES - 1) / STAGES;
                        if (!mbar_wait(empty0 + 8 * s, (count - 1) & 1u))
                            atomicOr(args.status, kErrTimeoutDrain);
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------ MMA issuer, even CTA only
        if (lane == 0 && leader) {
            constexpr uint32_t kIdesc = idesc_mxf4(256, 2 * SBN);
            const uint32_t sfa = tmem_base + C::SF_COL;
            const uint32_t sfb = tmem_base + C::SFB_COL;
            int stage = 0;
            uint32_t phase = 0;
            int ev = 0;
            bool ok = true;
            for (int t = t_first; t < args.total_tiles && ok; t += t_step, ++ev) {
                const int acc = ev % C::ACC_BUFS;
                const uint32_t aphase = (ev / C::ACC_BUFS) & 1;
                if (!mbar_wait(tempty0 + 8 * acc, aphase ^ 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + acc * C::ACC_STRIDE;
                for (int kb = 0; kb < args.num_kb; ++kb) {
                    if (!mbar_wait(full0 + 8 * stage, phase) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = s0 + stage * C::STAGE_BYTES;   // Wr, Wi
                    const uint32_t x = a + C::W_BYTES;                 // B1 half, B2 half
                    // 32 bytes (64 K) per MMA; K beyond the last value is 0
                    const int ksteps = min(kRowBytes / 32, (args.K - kb * kStageK + 63) / 64);
                    for (int j = 0; j < ksteps; ++j) {
                        const uint32_t accum = (kb > 0 || j > 0) ? 1u : 0u;
                        // Wr [Xr; Xi] -> [Wr Xr | Wr Xi]
                        mma_mxf4_pair(d, sdesc_kmajor_sw128(a + 32 * j),
                                      sdesc_kmajor_sw128(x + 32 * j), kIdesc, sfa, sfb, accum);
                        // Wi [-Xi; Xr] -> [-Wi Xi | Wi Xr]
                        mma_mxf4_pair(d, sdesc_kmajor_sw128(a + C::W_PLANE + 32 * j),
                                      sdesc_kmajor_sw128(x + C::X_PLANE + 32 * j), kIdesc, sfa,
                                      sfb, 1u);
                    }
                    mma_commit_pair(empty0 + 8 * stage, kBoth);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit_pair(tfull0 + 8 * acc, kBoth);
            }
            if (!ok) {
                atomicOr(args.status, kErrTimeoutMma);
                *abort_flag = 1;
            }
            mma_commit_pair(done_bar, 1);
            if (!mbar_wait(done_bar, 0)) atomicOr(args.status, kErrTimeoutDrain);
        }
    } else {
        // ------------------------------------------------- epilogue, both CTAs
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t stage_buf = staging0 + (warp - 2) * 8192;
        const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
        int ev = 0;
        int chunk_count = 0;
        bool ok = true;
        for (int t = t_first; t < args.total_tiles && ok; t += t_step, ++ev) {
            int b, mp, nt;
            decode(t, b, mp, nt);
            const int mrow0 = mp * 256 + 128 * rank;           // this CTA's first row
            const int m = mrow0 + row;
            int32_t *yrow = args.Y + (static_cast<size_t>(b) * args.M + m) * args.N * 2;
            const int acc = ev % C::ACC_BUFS;
            const uint32_t aphase = (ev / C::ACC_BUFS) & 1;
            if (!mbar_wait(tfull0 + 8 * acc, aphase) || *abort_flag) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t tP = tmem_base + lane_off + acc * C::ACC_STRIDE;
#pragma unroll 1
            for (int c = 0; c < SBN / 16; ++c) {
                float re[16], im[16];
                tmem_ld_2x16(tP + c * 16, tP + SBN + c * 16, re, im);
                const int n0 = nt * SBN + c * 16;
                if (args.tma_store) {
                    if (n0 < args.N) {
                        const uint32_t buf = stage_buf + (chunk_count & 1) * 4096;
                        if (lane == 0) bulk_wait_read<1>();   // the buffer's last store has read it
                        __syncwarp();
                        const uint32_t rbase = buf + lane * 128;
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            st_shared_i4(rbase + ((j ^ (lane & 7)) << 4), __float2int_rn(re[2 * j]),
                                         __float2int_rn(im[2 * j]), __float2int_rn(re[2 * j + 1]),
                                         __float2int_rn(im[2 * j + 1]));
                        fence_async_smem();
                        __syncwarp();
                        if (lane == 0) {
                            tma_store_3d(&tmY, buf, 2 * n0, mrow0 + quarter * 32, b);
                            bulk_commit();
                        }
                        ++chunk_count;
                    }
                } else if (m < args.M && n0 < args.N) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (n0 + i < args.N) {
                            yrow[2 * (n0 + i)] = __float2int_rn(re[i]);
                            yrow[2 * (n0 + i) + 1] = __float2int_rn(im[i]);
                        }
                }
            }
            // this warp is done with the accumulator (its values are in registers):
            // release it on the even CTA at CTA scope
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_remote(tempty0_lead + 8 * acc);
        }
        if (args.tma_store && lane == 0) bulk_wait<0>();
        __syncwarp();
        if (!ok && lane == 0) {
            atomicOr(args.status, kErrTimeoutEpilogue);
            *abort_flag = 1;
        }
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync();                       // no CTA leaves while its peer may signal it
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, C::TMEM_COLS);
    }
}

// E2M1 row length in 16-byte words: Kw rounded up to 8 (128-byte rows)
int64_t fp4_words(const tcbf_plan_s &pl) { return round_up(pl.Kw, 8); }
int64_t fp4_row_bytes(const tcbf_plan_s &pl) { return fp4_words(pl) * 16; }

size_t fp4_w_bytes(const tcbf_plan_s &pl) {
    return static_cast<size_t>(pl.p.w_batches) * 2 * pl.p.M * fp4_row_bytes(pl);
}

size_t fp4_x_bytes(const tcbf_plan_s &pl) {
    return static_cast<size_t>(pl.p.batch) * 3 * pl.p.N * fp4_row_bytes(pl);
}

int expand_grid(int64_t total, int num_sms) {
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256),
                                                                   int64_t(num_sms) * 16)));
}

// Packed bits of W (which 0) or X (which 1) into the plan's E2M1 planes.
cudaError_t launch_expand(const tcbf_plan_s &pl, int which, const uint32_t *bits, cudaStream_t s) {
    const tcbf_problem &p = pl.p;
    uint8_t *Wq = static_cast<uint8_t *>(pl.fp4_buf);
    if (which == 0) {
        const int64_t rows = p.w_batches * 2 * p.M;
        expand_w_fp4_kernel<<<expand_grid(rows * fp4_words(pl), pl.num_sms), 256, 0, s>>>(
            bits, reinterpret_cast<uint4 *>(Wq), rows, static_cast<int>(p.M), w_plane_rows(pl),
            static_cast<int>(pl.Kw), static_cast<int>(fp4_words(pl)), static_cast<int>(p.K));
    } else {
        expand_x_fp4_kernel<<<expand_grid(p.batch * p.N * fp4_words(pl), pl.num_sms), 256, 0, s>>>(
            bits, reinterpret_cast<uint4 *>(Wq + fp4_w_bytes(pl)), p.batch, p.N,
            static_cast<int>(pl.Kw), static_cast<int>(fp4_words(pl)), static_cast<int>(p.K));
    }
    return cudaGetLastError();
}

// Interleaved complex W (which 0) or X (which 1) of type src_type straight
// into the plan's E2M1 planes.
cudaError_t launch_pack_fp4(const tcbf_plan_s &pl, int which, int src_type, const void *src,
                            cudaStream_t s) {
    const tcbf_problem &p = pl.p;
    uint8_t *Wq = static_cast<uint8_t *>(pl.fp4_buf);
    const bool f32 = src_type == TCBF_SRC_CF32;
    if (which == 0) {
        const int64_t rows = p.w_batches * p.M;
        const int Kq = static_cast<int>(fp4_words(pl));
        const int grid = expand_grid(rows * Kq * 32, pl.num_sms);
        auto *dst = reinterpret_cast<uint4 *>(Wq);
        if (f32)
            pack_w_fp4_kernel<true><<<grid, 256, 0, s>>>(src, dst, rows, p.M, int(p.K), Kq);
        else
            pack_w_fp4_kernel<false><<<grid, 256, 0, s>>>(src, dst, rows, p.M, int(p.K), Kq);
    } else {
        const int n_tiles = static_cast<int>(ceil_div(p.N, kPackSamples));
        const int w_tiles = static_cast<int>(fp4_words(pl) / kPackWords);
        // blocks per batch: enough for every SM to hold several across the batches
        const int64_t per_b = int64_t(n_tiles) * w_tiles;
        const int bx = static_cast<int>(std::max<int64_t>(
            1, std::min<int64_t>(per_b, ceil_div(int64_t(pl.num_sms) * 16, p.batch))));
        dim3 grid(bx, static_cast<unsigned>(p.batch));
        uint8_t *dst = Wq + fp4_w_bytes(pl);
        // 16-byte loads need every row of X to start 16-byte aligned (N % 4 == 0)
        const bool vec = p.N % 4 == 0;
        auto run = [&](auto kern) {
            kern<<<grid, 256, 0, s>>>(src, dst, int(p.K), int(p.N), int(pl.Kw), int(fp4_words(pl)),
                                      n_tiles, w_tiles);
        };
        if (f32)
            vec ? run(pack_x_fp4_kernel<true, true>) : run(pack_x_fp4_kernel<true, false>);
        else
            vec ? run(pack_x_fp4_kernel<false, true>) : run(pack_x_fp4_kernel<false, false>);
    }
    return cudaGetLastError();
}

// The GEMM on the plan's E2M1 planes.
template <int SBN, int STAGES>
cudaError_t launch_fp4_pair(const tcbf_plan_s &pl, int32_t *Y, cudaStream_t s) {
    using C = CfgFp4<SBN, STAGES>;
    const tcbf_problem &p = pl.p;
    uint8_t *Wq = static_cast<uint8_t *>(pl.fp4_buf);
    uint8_t *Xq = Wq + fp4_w_bytes(pl);
    const int64_t R = fp4_row_bytes(pl);
    CUtensorMap tmW, tmX, tmY;
    {
        const uint64_t dims[3] = {static_cast<uint64_t>(R), static_cast<uint64_t>(p.M),
                                  static_cast<uint64_t>(2 * p.w_batches)};
        const uint64_t strides[2] = {static_cast<uint64_t>(R), static_cast<uint64_t>(p.M * R)};
        const uint32_t box[3] = {kRowBytes, 128, 2};
        if (encode_tiled(&tmW, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, Wq, dims, strides, box,
                         CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const uint64_t dims[3] = {static_cast<uint64_t>(R), static_cast<uint64_t>(p.N),
                                  static_cast<uint64_t>(3 * p.batch)};
        const uint64_t strides[2] = {static_cast<uint64_t>(R), static_cast<uint64_t>(p.N * R)};
        const uint32_t box[3] = {kRowBytes, SBN, 1};       // one plane of SBN samples
        if (encode_tiled(&tmX, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, Xq, dims, strides, box,
                         CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const int tma_store = (p.N % 2 == 0) ? 1 : 0;
    if (tma_store) {
        const uint64_t dims[3] = {static_cast<uint64_t>(2 * p.N), static_cast<uint64_t>(p.M),
                                  static_cast<uint64_t>(p.batch)};
        const uint64_t strides[2] = {static_cast<uint64_t>(p.N * 8),
                                     static_cast<uint64_t>(p.M * p.N * 8)};
        const uint32_t box[3] = {32, 32, 1};
        if (encode_tiled(&tmY, CU_TENSOR_MAP_DATA_TYPE_INT32, 3, Y, dims, strides, box,
                         CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    } else {
        memset(&tmY, 0, sizeof(tmY));
    }
    Fp4Args a;
    a.Y = Y;
    a.status = pl.status;
    a.tma_store = tma_store;
    a.M = static_cast<int>(p.M);
    a.N = static_cast<int>(p.N);
    a.K = static_cast<int>(p.K);
    a.per_w = static_cast<int>(pl.per_w);
    a.m_pairs = static_cast<int>(ceil_div(p.M, 256));
    a.n_tiles = static_cast<int>(ceil_div(p.N, SBN));
    a.num_kb = static_cast<int>(ceil_div(R, kRowBytes));
    const int64_t total = int64_t(a.m_pairs) * p.batch * a.n_tiles;
    if (total > 0x7fffffff) return cudaErrorInvalidValue;
    a.total_tiles = static_cast<int>(total);
    auto kern = cgemm_1bit_fp4_pair_kernel<SBN, STAGES>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kFp4Threads);
    cfg.dynamicSmemBytes = C::SMEM_BYTES;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // resident pairs per device, measured once (benign if two threads both measure)
    static std::atomic<int> max_clusters[64];
    int mc = max_clusters[pl.device & 63].load(std::memory_order_relaxed);
    if (mc == 0) {
        cfg.gridDim = dim3(pl.num_sms / 2 * 2);
        e = cudaOccupancyMaxActiveClusters(&mc, kern, &cfg);
        if (e != cudaSuccess) return e;
        if (mc < 1) return cudaErrorInvalidConfiguration;
        max_clusters[pl.device & 63].store(mc, std::memory_order_relaxed);
    }
    cfg.gridDim = dim3(static_cast<unsigned>(std::min<int64_t>(total, mc)) * 2);
    e = cudaLaunchKernelEx(&cfg, kern, tmW, tmX, tmY, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

size_t gemm_1bit_fp4_scratch_bytes(const tcbf_plan_s &pl) { return fp4_w_bytes(pl) + fp4_x_bytes(pl); }

cudaError_t gemm_1bit_fp4_reserve(tcbf_plan_s &pl) {
    const size_t need = gemm_1bit_fp4_scratch_bytes(pl);
    if (pl.fp4_buf && pl.fp4_bytes >= need) return cudaSuccess;
    if (pl.fp4_buf) cudaFree(pl.fp4_buf);
    pl.fp4_buf = nullptr;
    pl.fp4_bytes = 0;
    void *buf = nullptr;
    const cudaError_t e = cudaMalloc(&buf, need);
    if (e != cudaSuccess) {
        cudaGetLastError();   // the failed allocation is not sticky; clear it
        return e;
    }
    pl.fp4_buf = buf;
    pl.fp4_bytes = need;
    return cudaSuccess;
}

void gemm_1bit_fp4_release(tcbf_plan_s &pl) {
    if (pl.fp4_buf) cudaFree(pl.fp4_buf);
    pl.fp4_buf = nullptr;
    pl.fp4_bytes = 0;
}

bool gemm_1bit_fp4_usable(const tcbf_plan_s &pl) {
    return pl.p.mode == TCBF_MODE_1BIT && !pl.m_prefix && pl.p.K <= kMaxExactK && pl.fp4_buf &&
           pl.fp4_bytes >= gemm_1bit_fp4_scratch_bytes(pl);
}

cudaError_t launch_expand_1bit_fp4(const tcbf_plan_s &pl, int which, const uint32_t *bits,
                                   cudaStream_t s) {
    if (!gemm_1bit_fp4_usable(pl)) return cudaErrorNotSupported;
    return launch_expand(pl, which, bits, s);
}

cudaError_t launch_pack_1bit_fp4(const tcbf_plan_s &pl, int which, int src_type, const void *src,
                                 cudaStream_t s) {
    if (!gemm_1bit_fp4_usable(pl)) return cudaErrorNotSupported;
    return launch_pack_fp4(pl, which, src_type, src, s);
}

cudaError_t launch_gemm_1bit_fp4_expanded(const tcbf_plan_s &pl, int32_t *Y, cudaStream_t s,
                                          int variant) {
    if (!gemm_1bit_fp4_usable(pl)) return cudaErrorNotSupported;
    if (variant == 0) return launch_fp4_pair<128, 3>(pl, Y, s);
    if (variant == 1) return launch_fp4_pair<64, 4>(pl, Y, s);
    if (variant == 2) return launch_fp4_pair<96, 3>(pl, Y, s);
    return launch_fp4_pair<112, 3>(pl, Y, s);
}

cudaError_t launch_gemm_1bit_fp4(const tcbf_plan_s &pl, const uint32_t *Wb, const uint32_t *Xb,
                                 int32_t *Y, cudaStream_t s, int variant) {
    if (!gemm_1bit_fp4_usable(pl)) return cudaErrorNotSupported;
    cudaError_t e = launch_expand(pl, 0, Wb, s);
    if (e == cudaSuccess) e = launch_expand(pl, 1, Xb, s);
    if (e == cudaSuccess) e = launch_gemm_1bit_fp4_expanded(pl, Y, s, variant);
    return e;
}

}  // namespace tcbf
