// gemm_f16.cu — FP16 complex GEMM on the sm_103a tensor cores (tcgen05).
//
// Y[b] = W[b'] X[b] (Eq. 3) with the complex product of Sec. III-B built
// from four real MMAs per K step, accumulated in FP32 in tensor memory:
//     D_re += Wr Xr,  D_re += (-Wi) Xi,  D_im += Wr Xi,  D_im += Wi Xr.
// The paper negates Im in registers (its step 3); here the MMA instruction
// descriptor's negate-A bit does it, so no operand is modified.
//
// Split-FP8 (8-bit float formats are the paper's future work, Sec. VI): the
// same kernel with FMT = kFmtSplit8 reads packed rows of 64-element K blocks of
// 64 E4M3 "hi" bytes then 64 "lo" bytes (the same 128-byte swizzled rows and
// TMA boxes as FP16), issues Wh Xh + Wh Xl + Wl Xh as 12 kind::f8f6f4 MMAs
// per 32-element K step, and rescales each output by 2^-(eW[m] + eX[n]),
// the per-row power-of-two scales of the split.
//
// Block-scaled split-FP8 (FMT = kFmtSplit8Blk, plans with
// TCBF_FLAG_FP8_BLOCK_SCALES): the same hi/lo rows with a UE8M0 scale per
// 32 k of each row and sample; every stage also brings the two 512-byte
// scale tiles of its W rows and X samples, which the MMA thread copies into
// tensor memory (tcgen05.cp) before issuing kind::mxf8f6f4 block-scaled
// MMAs, so the tensor cores apply the scales and the epilogue stores the
// sums as they are.
//
// TF32 (for callers whose data arrives in FP32; the paper names more input
// formats as future work, Sec. VI): FMT = kFmtTf32 reads planes of FP32
// values already rounded to TF32, 32 per 128-byte row, and issues the same
// four real products as kind::tf32 MMAs of K = 8.
//
// Persistent, warp-specialised kernel (one CTA per SM, 192 threads):
//   warp 0      TMA producer: both planes of a W tile (128 x 64) and of an
//               X tile (BN x 64) per stage into a STAGES-deep shared-memory
//               ring (Sec. III-C: multi-stage buffers filled asynchronously)
//   warp 1      TMEM owner and single-thread MMA issuer
//   warps 2-5   epilogue: TMEM -> registers -> interleaved complex64 Y
// Tiles (batch, m-tile, n-tile) are strided over the CTAs; the two TMEM
// accumulator sets are double-buffered when they fit, so the epilogue of
// one tile overlaps the MMAs of the next.  All waits are bounded.
//
// Long K: the tensor core's FP32 accumulation truncates, so its relative
// error grows linearly with K (measured ~2.4e-9 K, biased toward zero).
// For K > kPromoteK the K loop is cut into chunks of kChunkBlocks stages;
// each chunk accumulates from zero into a TMEM partial P and the epilogue
// warps add P into a running sum S with FP32 round-to-nearest adds, so the
// error stays at the chunk's level.  The chunks alternate between the two
// accumulators: chunk c's P lands in one while the other holds S (the sum
// of chunks before c); the epilogue writes S + P over P, which then holds
// the sum, and frees S's accumulator for chunk c + 1.  The MMAs wait only
// for that add, and a tile's output drains while the next tile's first
// chunk runs.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>

#include "ptx.cuh"
#include "tiles.cuh"
#include "tcbf_internal.h"

namespace tcbf {
namespace {

using namespace dev;

constexpr int BM = 128;        // rows of W per tile (TMEM lanes)
constexpr int BK = 64;         // K elements per stage: one 128-byte swizzled row
constexpr int kThreads = 192;
constexpr int kPromoteK = 4096;     // K above this is accumulated in promoted chunks
constexpr int kChunkBlocks = 32;    // stages (x 64 K) per promoted chunk

// Operand formats of the kernel template: FP16 planes, E4M3 hi/lo rows, or
// TF32 planes (FP32 storage).  Every format fills 128-byte rows per stage.
constexpr int kFmtF16 = 0;
constexpr int kFmtSplit8 = 1;
constexpr int kFmtTf32 = 2;
constexpr int kFmtSplit8Blk = 3;
// Tensor-memory column of the block-scaled kernel's scale factors: per
// stage 8 columns (4 for the W tile, 4 for the X tile) above the
// accumulators of its 64-sample tiles.
constexpr int kSfCol = 256;

struct GemmArgs {
    float *Y;
    const int32_t *w_exps;     // split-FP8 scale exponents [w_batches][M] (else unused)
    const int32_t *x_exps;     // split-FP8 scale exponents [batch][N]
    const uint8_t *w_sf;       // block-scaled FP8: W scale tiles [w_batches][w_sf_tiles][num_kb][512]
    const uint8_t *x_sf;       // block-scaled FP8: X scale tiles [batch][x_sf_groups][num_kb][512]
    int w_sf_tiles, x_sf_groups;
    int tma_store;             // 1: Y written by TMA bulk tensor stores (needs N even)
    uint32_t *status;
    int M, N, K;
    int per_w;
    TileMap tiles;
    int num_kb;
    int kps;                   // K elements per stage: 64, or 128 for hi-only FP8 rows
    int kc_blocks;             // stages per accumulation chunk (num_kb when not promoting)
    int chunks;                // accumulation chunks per tile
    int total_tiles;
    int products;              // split-FP8: 1 (hi hi), 3 (+ hi lo, lo hi) or 4 (+ lo lo)
    int drop_fill;             // test hook: CTA 0 leaves out this operand load (-1: none)
};

constexpr int pow2_cols(int c) {
    return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512;
}

template <int BN, int STAGES, bool BLK = false>
struct Cfg {
    static constexpr int A_PLANE = BM * BK * 2;              // bytes of one W plane tile
    static constexpr int B_PLANE = BN * BK * 2;              // bytes of one X plane tile
    static constexpr int A_BYTES = 2 * A_PLANE;
    static constexpr int B_BYTES = 2 * B_PLANE;
    static constexpr int SF_BYTES = BLK ? 2 * kFp8BlkTile : 0;   // W and X scale tiles
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES + SF_BYTES;
    static constexpr int ACC_BUFS = (4 * BN <= 512) ? 2 : 1;
    static constexpr int TMEM_COLS = BLK ? 512 : pow2_cols(ACC_BUFS * 2 * BN);
    static_assert(!BLK || (ACC_BUFS * 2 * BN <= kSfCol && kSfCol + 8 * STAGES <= 512),
                  "block-scaled: accumulators below the scale columns");
    static constexpr int STAGING_BYTES = 4 * 2 * 4096;        // 4 epilogue warps x 2 x (32 rows x 128 B)
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + STAGING_BYTES + 256 + 1024;
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M=128");
    static_assert(SMEM_BYTES <= 232448, "shared memory");
};

// 2^-e as a float (|e| <= 100, so the result is a normal power of two).
__device__ __forceinline__ float pow2_neg(int e) { return __int_as_float((127 - e) << 23); }

__device__ __forceinline__ void decode_tile(int t, const GemmArgs &a, int &b, int &mt, int &nt) {
    tile_decode(a.tiles, t, b, mt, nt);
}

// Split-FP8 MMAs of one 32-K step j: (W part, X part) byte offsets (hi, hi),
// (hi, lo), (lo, hi), (lo, lo), the first NP of them; the lo bytes sit 64
// bytes into each 128-byte row.  Hi-only rows (NP = 1) hold 128 hi bytes per
// stage row, j = 0..3.  One-SM (PAIR false) or two-SM MMAs.
template <int NP, bool PAIR>
__device__ __forceinline__ void split_step(uint32_t d_re, uint32_t d_im, uint32_t a, uint32_t bx,
                                           int a_plane, int b_plane, int j, bool first,
                                           uint32_t idesc, uint32_t idesc_neg) {
#pragma unroll
    for (int pr = 0; pr < NP; ++pr) {
        const uint32_t wo = (pr >= 2 ? 64u : 0u) + 32u * j;
        const uint32_t xo = ((pr & 1) ? 64u : 0u) + 32u * j;
        const uint64_t ar = sdesc_kmajor_sw128(a + wo);
        const uint64_t ai = sdesc_kmajor_sw128(a + a_plane + wo);
        const uint64_t br = sdesc_kmajor_sw128(bx + xo);
        const uint64_t bi = sdesc_kmajor_sw128(bx + b_plane + xo);
        const uint32_t accum = (first && pr == 0) ? 0u : 1u;
        if (PAIR) {
            mma_f8f6f4_pair(d_re, ar, br, idesc, accum);
            mma_f8f6f4_pair(d_re, ai, bi, idesc_neg, 1u);
            mma_f8f6f4_pair(d_im, ar, bi, idesc, accum);
            mma_f8f6f4_pair(d_im, ai, br, idesc, 1u);
        } else {
            mma_f8f6f4(d_re, ar, br, idesc, accum);
            mma_f8f6f4(d_re, ai, bi, idesc_neg, 1u);
            mma_f8f6f4(d_im, ar, bi, idesc, accum);
            mma_f8f6f4(d_im, ai, br, idesc, 1u);
        }
    }
}

// Block-scaled split-FP8 MMAs of one 32-K step j, the first NP products as
// in split_step; the scale bytes of the stage's tiles in tensor memory are
// hi codes of its two 32-k blocks (ids 0, 1) then their lo codes (2, 3), or
// for hi-only rows the hi codes of its four blocks (ids 0-3).
template <int NP, int BN>
__device__ __forceinline__ void split_step_blk(uint32_t d_re, uint32_t d_im, uint32_t a,
                                               uint32_t bx, int a_plane, int b_plane, int j,
                                               bool first, uint32_t sfa, uint32_t sfb) {
#pragma unroll
    for (int pr = 0; pr < NP; ++pr) {
        const uint32_t wo = (pr >= 2 ? 64u : 0u) + 32u * j;
        const uint32_t xo = ((pr & 1) ? 64u : 0u) + 32u * j;
        const uint32_t sa = (pr >= 2 ? 2u : 0u) + static_cast<uint32_t>(j);
        const uint32_t sb = ((pr & 1) ? 2u : 0u) + static_cast<uint32_t>(j);
        const uint32_t idesc = idesc_mxf8(BM, BN, sa, sb, false);
        const uint32_t idesc_neg = idesc_mxf8(BM, BN, sa, sb, true);
        const uint64_t ar = sdesc_kmajor_sw128(a + wo);
        const uint64_t ai = sdesc_kmajor_sw128(a + a_plane + wo);
        const uint64_t br = sdesc_kmajor_sw128(bx + xo);
        const uint64_t bi = sdesc_kmajor_sw128(bx + b_plane + xo);
        const uint32_t accum = (first && pr == 0) ? 0u : 1u;
        mma_mxf8(d_re, ar, br, idesc, sfa, sfb, accum);
        mma_mxf8(d_re, ai, bi, idesc_neg, sfa, sfb, 1u);
        mma_mxf8(d_im, ar, bi, idesc, sfa, sfb, accum);
        mma_mxf8(d_im, ai, br, idesc, sfa, sfb, 1u);
    }
}

template <int BN, int STAGES, int FMT, int CL>
__global__ void __launch_bounds__(kThreads, 1)
    cgemm_tc_kernel(const __grid_constant__ CUtensorMap tmW,
                     const __grid_constant__ CUtensorMap tmX,
                     const __grid_constant__ CUtensorMap tmY, const GemmArgs args) {
    constexpr bool BLK = FMT == kFmtSplit8Blk;
    using C = Cfg<BN, STAGES, BLK>;
    constexpr bool SPLIT = FMT == kFmtSplit8 || BLK;
    constexpr bool TF32 = FMT == kFmtTf32;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
    const uint32_t s0 = smem_u32(smem);

    // output staging after the stage ring, then the barrier block
    const uint32_t staging0 = s0 + STAGES * C::STAGE_BYTES;
    const uint32_t bar0 = staging0 + C::STAGING_BYTES;
    const uint32_t full0 = bar0;                       // STAGES x 8 bytes
    const uint32_t empty0 = full0 + 8 * STAGES;        // STAGES x 8
    const uint32_t tfull0 = empty0 + 8 * STAGES;       // 2 x 8
    const uint32_t tempty0 = tfull0 + 16;              // 2 x 8
    const uint32_t done_bar = tempty0 + 16;            // 8
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + STAGES * C::STAGE_BYTES +
                                                       C::STAGING_BYTES + 16 * STAGES + 40);
    volatile uint32_t *abort_flag = tmem_slot + 1;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    // Clusters of CL CTAs along M share each X tile: every CTA loads a 1/CL
    // row slice and multicasts it to all, and every CTA's MMA completion is
    // committed to all CTAs' empty barriers (count CL).  The cluster walks
    // cluster tiles (batch, group of CL m-tiles, n-tile) in lockstep.
    const int rank = CL > 1 ? static_cast<int>(cluster_ctarank()) : 0;
    const int t_first = CL > 1 ? static_cast<int>(cluster_id_x()) : static_cast<int>(blockIdx.x);
    const int t_step = CL > 1 ? static_cast<int>(nclusters_x()) : static_cast<int>(gridDim.x);
    constexpr uint16_t kMask = static_cast<uint16_t>((1u << CL) - 1u);
    auto decode = [&](int t, int &b, int &mt, int &nt) {
        if (CL == 1) {
            decode_tile(t, args, b, mt, nt);
        } else {
            const int groups = (args.tiles.m_tiles + CL - 1) / CL;
            const int per_b = groups * args.tiles.n_tiles;
            b = t / per_b;
            const int local = t - b * per_b;
            nt = local % args.tiles.n_tiles;
            mt = (local / args.tiles.n_tiles) * CL + rank;
        }
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, CL);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, 128);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
        tma_prefetch_desc(&tmW);
        tma_prefetch_desc(&tmX);
        if (args.tma_store) tma_prefetch_desc(&tmY);
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    if (CL > 1) cluster_sync();            // peers' barriers exist before any multicast
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued = 0;
            bool ok = true;
            for (int t = t_first; t < args.total_tiles && ok; t += t_step) {
                int b, mt, nt;
                decode(t, b, mt, nt);
                const int bw = b / args.per_w;
                for (int kb = 0; kb < args.num_kb; ++kb) {
                    if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = full0 + 8 * stage;
                    const uint32_t dst = s0 + stage * C::STAGE_BYTES;
                    // x: 128 bytes per stage in both formats (64 FP16, or 64 hi + 64 lo bytes)
                    const int x = kb * (SPLIT ? 128 : args.kps);
                    if (CL == 1) {
                        // the failure-path test hook leaves one load (and its arrival) out
                        if (blockIdx.x != 0 || static_cast<int>(issued) != args.drop_fill) {
                            mbar_arrive_expect_tx(fb, C::STAGE_BYTES);
                            tma_load_3d(dst, &tmW, fb, x, mt * BM, 2 * bw);
                            tma_load_3d(dst + C::A_BYTES, &tmX, fb, x, nt * BN, 2 * b);
                            if (BLK) {   // the stage's W and X scale tiles
                                const uint32_t sdst = dst + C::A_BYTES + C::B_BYTES;
                                bulk_load(sdst,
                                          args.w_sf + ((static_cast<size_t>(bw) * args.w_sf_tiles + mt) *
                                                           args.num_kb + kb) * kFp8BlkTile,
                                          kFp8BlkTile, fb);
                                bulk_load(sdst + kFp8BlkTile,
                                          args.x_sf + ((static_cast<size_t>(b) * args.x_sf_groups + nt) *
                                                           args.num_kb + kb) * kFp8BlkTile,
                                          kFp8BlkTile, fb);
                            }
                        }
                    } else {
                        mbar_arrive_expect_tx(fb, C::STAGE_BYTES);
                        tma_load_3d(dst, &tmW, fb, x, mt * BM, 2 * bw);
                        constexpr int kRows = BN / CL;
#pragma unroll
                        for (int pl = 0; pl < 2; ++pl)
                            tma_load_3d_mc(dst + C::A_BYTES + pl * C::B_PLANE + rank * kRows * 128,
                                           &tmX, fb, x, nt * BN + rank * kRows, 2 * b + pl, kMask);
                    }
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
                // let every copy this thread started land before the CTA exits
                for (int s = 0; s < STAGES; ++s) {
                    if (issued > static_cast<uint32_t>(s)) {
                        const uint32_t count = (issued - s + STAGES - 1) / STAGES;
                        if (!mbar_wait(full0 + 8 * s, (count - 1) & 1u))
                            atomicOr(args.status, kErrTimeoutDrain);
                    }
                }
            } else if (CL > 1) {
                // every CTA's release of every slot this CTA filled has arrived,
                // so no peer still signals into this CTA's barriers
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
        // ------------------------------------------------------- MMA issuer
        if (lane == 0) {
            // A / B format: F16 and E4M3 are 0 in their kinds, TF32 is 2
            constexpr uint32_t kIdesc = idesc_f32acc(BM, BN, TF32 ? 2u : 0u, false);
            constexpr uint32_t kIdescNeg = idesc_f32acc(BM, BN, TF32 ? 2u : 0u, true);
            int stage = 0;
            uint32_t phase = 0;
            int ev = 0;                                  // accumulator hand-offs so far
            // promoted long K alternates the two accumulators (the launchers
            // take K > kPromoteK only when two fit)
            const int nbuf = C::ACC_BUFS;
            bool ok = true;
            for (int t = t_first; t < args.total_tiles && ok; t += t_step) {
                for (int ch = 0; ch < args.chunks; ++ch, ++ev) {
                    const int acc = ev % nbuf;
                    const uint32_t aphase = (ev / nbuf) & 1;
                    if (!mbar_wait(tempty0 + 8 * acc, aphase ^ 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_re = tmem_base + acc * 2 * BN;
                    const uint32_t d_im = d_re + BN;
                    const int kb0 = ch * args.kc_blocks;
                    const int kb1 = min(args.num_kb, kb0 + args.kc_blocks);
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!mbar_wait(full0 + 8 * stage, phase) || *abort_flag) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a = s0 + stage * C::STAGE_BYTES;
                        const uint32_t bx = a + C::A_BYTES;
                        if (!SPLIT) {
                            // 32 bytes per MMA step: 16 FP16 or 8 TF32 elements
                            constexpr int kStep = TF32 ? 8 : 16;
                            const int ksteps = min(4, (args.K - kb * args.kps + kStep - 1) / kStep);
                            for (int j = 0; j < ksteps; ++j) {
                                const uint64_t ar = sdesc_kmajor_sw128(a + 32 * j);
                                const uint64_t ai = sdesc_kmajor_sw128(a + C::A_PLANE + 32 * j);
                                const uint64_t br = sdesc_kmajor_sw128(bx + 32 * j);
                                const uint64_t bi = sdesc_kmajor_sw128(bx + C::B_PLANE + 32 * j);
                                const uint32_t accum = (kb > kb0 || j > 0) ? 1u : 0u;
                                if (TF32) {
                                    mma_tf32(d_re, ar, br, kIdesc, accum);
                                    mma_tf32(d_re, ai, bi, kIdescNeg, 1u);
                                    mma_tf32(d_im, ar, bi, kIdesc, accum);
                                    mma_tf32(d_im, ai, br, kIdesc, 1u);
                                } else {
                                    mma_f16(d_re, ar, br, kIdesc, accum);
                                    mma_f16(d_re, ai, bi, kIdescNeg, 1u);
                                    mma_f16(d_im, ar, bi, kIdesc, accum);
                                    mma_f16(d_im, ai, br, kIdesc, 1u);
                                }
                            }
                        } else if (BLK) {
                            // the stage's scale tiles into its tensor-memory columns,
                            // ordered before this thread's MMAs below
                            const uint32_t sft = tmem_base + kSfCol + 8 * stage;
                            const uint32_t ssrc = bx + C::B_BYTES;
                            tmem_cp_32x128b_x4(sft, ssrc);
                            tmem_cp_32x128b_x4(sft + 4, ssrc + kFp8BlkTile);
                            const int ksteps = min(args.kps / 32, (args.K - kb * args.kps + 31) / 32);
                            for (int j = 0; j < ksteps; ++j) {
                                const bool first = kb == kb0 && j == 0;
                                if (args.products == 3)
                                    split_step_blk<3, BN>(d_re, d_im, a, bx, C::A_PLANE, C::B_PLANE, j,
                                                          first, sft, sft + 4);
                                else if (args.products == 1)
                                    split_step_blk<1, BN>(d_re, d_im, a, bx, C::A_PLANE, C::B_PLANE, j,
                                                          first, sft, sft + 4);
                                else
                                    split_step_blk<4, BN>(d_re, d_im, a, bx, C::A_PLANE, C::B_PLANE, j,
                                                          first, sft, sft + 4);
                            }
                        } else {
                            // 32 E4M3 per step; (W part, X part) byte offsets:
                            // (hi, hi), (hi, lo), (lo, hi), (lo, lo), the first
                            // args.products of them (hi-only rows: 4 steps)
                            const int ksteps = min(args.kps / 32, (args.K - kb * args.kps + 31) / 32);
                            for (int j = 0; j < ksteps; ++j) {
                                const bool first = kb == kb0 && j == 0;
                                if (args.products == 3)
                                    split_step<3, false>(d_re, d_im, a, bx, C::A_PLANE, C::B_PLANE, j,
                                                         first, kIdesc, kIdescNeg);
                                else if (args.products == 1)
                                    split_step<1, false>(d_re, d_im, a, bx, C::A_PLANE, C::B_PLANE, j,
                                                         first, kIdesc, kIdescNeg);
                                else
                                    split_step<4, false>(d_re, d_im, a, bx, C::A_PLANE, C::B_PLANE, j,
                                                         first, kIdesc, kIdescNeg);
                            }
                        }
                        if (CL == 1)
                            mma_commit(empty0 + 8 * stage);
                        else
                            mma_commit_mc(empty0 + 8 * stage, kMask);
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    mma_commit(tfull0 + 8 * acc);
                }
            }
            if (!ok) {
                atomicOr(args.status, kErrTimeoutMma);
                *abort_flag = 1;
            }
            // every MMA issued must finish before tensor memory is released
            mma_commit(done_bar);
            if (!mbar_wait(done_bar, 0)) atomicOr(args.status, kErrTimeoutDrain);
        }
    } else {
        // --------------------------------------------------------- epilogue
        // Each warp owns 32 accumulator rows (its TMEM lane quarter).  Per
        // 16-column chunk it loads re and im, interleaves them into complex64
        // and either stages the 32 x 128-byte block in shared memory (128-byte
        // swizzle, conflict-free) for one TMA bulk tensor store, or (odd N)
        // stores its row directly.
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t stage_buf = staging0 + (warp - 2) * 8192;
        const bool vec_ok = (args.N & 1) == 0;
        int ev = 0;
        const int nbuf = C::ACC_BUFS;
        const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
        int chunk_count = 0;
        bool ok = true;
        for (int t = t_first; t < args.total_tiles && ok; t += t_step) {
            int b, mt, nt;
            decode(t, b, mt, nt);
            const int m = mt * BM + row;
            float *yrow = args.Y + (static_cast<size_t>(b) * args.M + m) * args.N * 2;
            float row_scale = 1.f;
            if (SPLIT && !BLK && m < args.M)
                row_scale = pow2_neg(__ldg(args.w_exps + static_cast<size_t>(b / args.per_w) * args.M + m));
            for (int ch = 0; ch < args.chunks; ++ch, ++ev) {
                const int acc = ev % nbuf;
                const uint32_t aphase = (ev / nbuf) & 1;
                if (!mbar_wait(tfull0 + 8 * acc, aphase) || *abort_flag) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tP = tmem_base + lane_off + acc * 2 * BN;
                if (ch > 0) {
                    // promote: the running sum S (the previous chunk's accumulator)
                    // plus this chunk's P, FP32 round-to-nearest, into this
                    // accumulator; then S's accumulator is free for the next chunk
                    const uint32_t tS = tmem_base + lane_off + (acc ^ 1) * 2 * BN;
#pragma unroll 1
                    for (int g = 0; g < BN / 16; ++g) {
                        float pr[16], pi[16], sr[16], si[16];
                        tmem_ld_2x16(tP + g * 16, tP + BN + g * 16, pr, pi);
                        tmem_ld_2x16(tS + g * 16, tS + BN + g * 16, sr, si);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            pr[i] = __fadd_rn(sr[i], pr[i]);
                            pi[i] = __fadd_rn(si[i], pi[i]);
                        }
                        tmem_st_2x16(tP + g * 16, tP + BN + g * 16, pr, pi);
                    }
                    tmem_st_wait();
                    tc_fence_before();
                    mbar_arrive(tempty0 + 8 * (acc ^ 1));
                }
                // a chunk before the last keeps its sum in its accumulator
                if (ch + 1 < args.chunks) continue;
#pragma unroll 1
                for (int c = 0; c < BN / 16; ++c) {
                    float re[16], im[16];
                    tmem_ld_2x16(tP + c * 16, tP + BN + c * 16, re, im);
                    const int n0 = nt * BN + c * 16;
                    if (SPLIT && !BLK) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int n = min(n0 + i, args.N - 1);
                            const float f = row_scale * pow2_neg(__ldg(args.x_exps + static_cast<size_t>(b) * args.N + n));
                            re[i] *= f;
                            im[i] *= f;
                        }
                    }
                    if (args.tma_store) {
                        if (n0 < args.N) {
                            const uint32_t buf = stage_buf + (chunk_count & 1) * 4096;
                            if (lane == 0) bulk_wait_read<1>();   // buffer's previous store has read it
                            __syncwarp();
                            const uint32_t rbase = buf + lane * 128;
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                st_shared_v4(rbase + ((j ^ (lane & 7)) << 4), re[2 * j], im[2 * j],
                                             re[2 * j + 1], im[2 * j + 1]);
                            fence_async_smem();
                            __syncwarp();
                            if (lane == 0) {
                                tma_store_3d(&tmY, buf, 2 * n0, mt * BM + quarter * 32, b);
                                bulk_commit();
                            }
                            ++chunk_count;
                        }
                    } else if (m < args.M && n0 < args.N) {
                        if (vec_ok && n0 + 16 <= args.N) {
                            float4 *dst = reinterpret_cast<float4 *>(yrow + 2 * n0);
#pragma unroll
                            for (int i = 0; i < 8; ++i)
                                dst[i] = make_float4(re[2 * i], im[2 * i], re[2 * i + 1], im[2 * i + 1]);
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if (n0 + i < args.N) {
                                    yrow[2 * (n0 + i)] = re[i];
                                    yrow[2 * (n0 + i) + 1] = im[i];
                                }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(tempty0 + 8 * acc);
            }
        }
        if (args.tma_store && lane == 0) bulk_wait<0>();   // all of this warp's stores done
        __syncwarp();
        if (!ok && lane == 0) {
            atomicOr(args.status, kErrTimeoutEpilogue);
            *abort_flag = 1;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (CL > 1) cluster_sync();            // no CTA leaves while peers may signal it
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, C::TMEM_COLS);
    }
}

// ===========================================================================
// Two-SM tiles (cta_group::2).  A cluster of two CTAs on two SMs computes a
// 256 x BN tile with M = 256 MMAs issued by the even CTA: each CTA holds 128
// rows of W (A) and BN/2 rows of X (half of B) at the same shared-memory
// offsets, and its tensor memory holds its 128 rows x BN columns of Re and
// Im.  Per SM the tensor core then reads A 128 x K and B BN/2 x K per MMA, a
// quarter less shared-memory traffic than a one-SM 128 x BN tile, with the
// same double-buffered accumulators.  Both CTAs' TMA loads complete on the
// even CTA's full barrier; its MMA completions are committed to both CTAs'
// empty and accumulator barriers; both CTAs' epilogues release an
// accumulator on the even CTA's barrier.
// ===========================================================================
template <int BN, int STAGES>
struct CfgPair {
    static constexpr int A_PLANE = BM * BK * 2;
    static constexpr int B_PLANE = (BN / 2) * BK * 2;
    static constexpr int A_BYTES = 2 * A_PLANE;
    static constexpr int STAGE_BYTES = A_BYTES + 2 * B_PLANE;     // per CTA
    static constexpr int ACC_BUFS = (4 * BN <= 512) ? 2 : 1;
    static constexpr int TMEM_COLS = pow2_cols(ACC_BUFS * 2 * BN);
    static constexpr int STAGING_BYTES = 4 * 2 * 4096;
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + STAGING_BYTES + 256 + 1024;
    static_assert(BN % 32 == 0 && BN <= 256, "pair N");
    static_assert(SMEM_BYTES <= 232448, "shared memory");
};

template <int BN, int STAGES, int FMT>
__global__ void __launch_bounds__(kThreads, 1)
    cgemm_pair_kernel(const __grid_constant__ CUtensorMap tmW,
                      const __grid_constant__ CUtensorMap tmX,
                      const __grid_constant__ CUtensorMap tmY, const GemmArgs args) {
    using C = CfgPair<BN, STAGES>;
    constexpr bool SPLIT = FMT == kFmtSplit8;
    constexpr bool TF32 = FMT == kFmtTf32;
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
    // (batch, 256-row pair tile, n-tile) of pair tile t, n fastest
    auto decode = [&](int t, int &b, int &mp, int &nt) {
        const int groups = (args.tiles.m_tiles + 1) / 2;
        const int per_b = groups * args.tiles.n_tiles;
        b = t / per_b;
        const int local = t - b * per_b;
        nt = local % args.tiles.n_tiles;
        mp = local / args.tiles.n_tiles;
    };

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
                    const int x = kb * (SPLIT ? 128 : args.kps);
                    tma_load_3d_pair(dst, &tmW, fb, x, mp * 256 + 128 * rank, 2 * bw);
                    tma_load_3d_pair(dst + C::A_BYTES, &tmX, fb, x, nt * BN + rank * (BN / 2), 2 * b);
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
            constexpr uint32_t kIdesc = idesc_f32acc(256, BN, TF32 ? 2u : 0u, false);
            constexpr uint32_t kIdescNeg = idesc_f32acc(256, BN, TF32 ? 2u : 0u, true);
            int stage = 0;
            uint32_t phase = 0;
            int ev = 0;
            // promoted long K alternates the two accumulators (the launchers
            // take K > kPromoteK only when two fit)
            const int nbuf = C::ACC_BUFS;
            bool ok = true;
            for (int t = t_first; t < args.total_tiles && ok; t += t_step) {
                for (int ch = 0; ch < args.chunks; ++ch, ++ev) {
                    const int acc = ev % nbuf;
                    const uint32_t aphase = (ev / nbuf) & 1;
                    if (!mbar_wait(tempty0 + 8 * acc, aphase ^ 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_re = tmem_base + acc * 2 * BN;
                    const uint32_t d_im = d_re + BN;
                    const int kb0 = ch * args.kc_blocks;
                    const int kb1 = min(args.num_kb, kb0 + args.kc_blocks);
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!mbar_wait(full0 + 8 * stage, phase) || *abort_flag) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a = s0 + stage * C::STAGE_BYTES;
                        const uint32_t bx = a + C::A_BYTES;
                        if (!SPLIT) {
                            constexpr int kStep = TF32 ? 8 : 16;
                            const int ksteps = min(4, (args.K - kb * args.kps + kStep - 1) / kStep);
                            for (int j = 0; j < ksteps; ++j) {
                                const uint64_t ar = sdesc_kmajor_sw128(a + 32 * j);
                                const uint64_t ai = sdesc_kmajor_sw128(a + C::A_PLANE + 32 * j);
                                const uint64_t br = sdesc_kmajor_sw128(bx + 32 * j);
                                const uint64_t bi = sdesc_kmajor_sw128(bx + C::B_PLANE + 32 * j);
                                const uint32_t accum = (kb > kb0 || j > 0) ? 1u : 0u;
                                if (TF32) {
                                    mma_tf32_pair(d_re, ar, br, kIdesc, accum);
                                    mma_tf32_pair(d_re, ai, bi, kIdescNeg, 1u);
                                    mma_tf32_pair(d_im, ar, bi, kIdesc, accum);
                                    mma_tf32_pair(d_im, ai, br, kIdesc, 1u);
                                } else {
                                    mma_f16_pair(d_re, ar, br, kIdesc, accum);
                                    mma_f16_pair(d_re, ai, bi, kIdescNeg, 1u);
                                    mma_f16_pair(d_im, ar, bi, kIdesc, accum);
                                    mma_f16_pair(d_im, ai, br, kIdesc, 1u);
                                }
                            }
                        } else {
                            const int ksteps = min(args.kps / 32, (args.K - kb * args.kps + 31) / 32);
                            for (int j = 0; j < ksteps; ++j) {
                                const bool first = kb == kb0 && j == 0;
                                if (args.products == 3)
                                    split_step<3, true>(d_re, d_im, a, bx, C::A_PLANE, C::B_PLANE, j,
                                                        first, kIdesc, kIdescNeg);
                                else if (args.products == 1)
                                    split_step<1, true>(d_re, d_im, a, bx, C::A_PLANE, C::B_PLANE, j,
                                                        first, kIdesc, kIdescNeg);
                                else
                                    split_step<4, true>(d_re, d_im, a, bx, C::A_PLANE, C::B_PLANE, j,
                                                        first, kIdesc, kIdescNeg);
                            }
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
        const bool vec_ok = (args.N & 1) == 0;
        int ev = 0;
        const int nbuf = C::ACC_BUFS;
        const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
        int chunk_count = 0;
        bool ok = true;
        for (int t = t_first; t < args.total_tiles && ok; t += t_step) {
            int b, mp, nt;
            decode(t, b, mp, nt);
            const int mrow0 = mp * 256 + 128 * rank;           // this CTA's first row
            const int m = mrow0 + row;
            float *yrow = args.Y + (static_cast<size_t>(b) * args.M + m) * args.N * 2;
            float row_scale = 1.f;
            if (SPLIT && m < args.M)
                row_scale = pow2_neg(__ldg(args.w_exps + static_cast<size_t>(b / args.per_w) * args.M + m));
            for (int ch = 0; ch < args.chunks; ++ch, ++ev) {
                const int acc = ev % nbuf;
                const uint32_t aphase = (ev / nbuf) & 1;
                if (!mbar_wait(tfull0 + 8 * acc, aphase) || *abort_flag) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tP = tmem_base + lane_off + acc * 2 * BN;
                if (ch > 0) {
                    // promote: the running sum S (the previous chunk's accumulator)
                    // plus this chunk's P, FP32 round-to-nearest, into this
                    // accumulator; then S's accumulator is free for the next chunk
                    const uint32_t tS = tmem_base + lane_off + (acc ^ 1) * 2 * BN;
#pragma unroll 1
                    for (int g = 0; g < BN / 16; ++g) {
                        float pr[16], pi[16], sr[16], si[16];
                        tmem_ld_2x16(tP + g * 16, tP + BN + g * 16, pr, pi);
                        tmem_ld_2x16(tS + g * 16, tS + BN + g * 16, sr, si);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            pr[i] = __fadd_rn(sr[i], pr[i]);
                            pi[i] = __fadd_rn(si[i], pi[i]);
                        }
                        tmem_st_2x16(tP + g * 16, tP + BN + g * 16, pr, pi);
                    }
                    tmem_st_wait();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive_remote(tempty0_lead + 8 * (acc ^ 1));
                }
                // a chunk before the last keeps its sum in its accumulator
                if (ch + 1 < args.chunks) continue;
                {
#pragma unroll 1
                    for (int c = 0; c < BN / 16; ++c) {
                        float re[16], im[16];
                        tmem_ld_2x16(tP + c * 16, tP + BN + c * 16, re, im);
                        const int n0 = nt * BN + c * 16;
                        if (SPLIT) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const int n = min(n0 + i, args.N - 1);
                                const float f = row_scale * pow2_neg(__ldg(args.x_exps + static_cast<size_t>(b) * args.N + n));
                                re[i] *= f;
                                im[i] *= f;
                            }
                        }
                        if (args.tma_store) {
                            if (n0 < args.N) {
                                const uint32_t buf = stage_buf + (chunk_count & 1) * 4096;
                                if (lane == 0) bulk_wait_read<1>();
                                __syncwarp();
                                const uint32_t rbase = buf + lane * 128;
#pragma unroll
                                for (int j = 0; j < 8; ++j)
                                    st_shared_v4(rbase + ((j ^ (lane & 7)) << 4), re[2 * j], im[2 * j],
                                                 re[2 * j + 1], im[2 * j + 1]);
                                fence_async_smem();
                                __syncwarp();
                                if (lane == 0) {
                                    tma_store_3d(&tmY, buf, 2 * n0, mrow0 + quarter * 32, b);
                                    bulk_commit();
                                }
                                ++chunk_count;
                            }
                        } else if (m < args.M && n0 < args.N) {
                            if (vec_ok && n0 + 16 <= args.N) {
                                float4 *dst = reinterpret_cast<float4 *>(yrow + 2 * n0);
#pragma unroll
                                for (int i = 0; i < 8; ++i)
                                    dst[i] = make_float4(re[2 * i], im[2 * i], re[2 * i + 1], im[2 * i + 1]);
                            } else {
#pragma unroll
                                for (int i = 0; i < 16; ++i)
                                    if (n0 + i < args.N) {
                                        yrow[2 * (n0 + i)] = re[i];
                                        yrow[2 * (n0 + i) + 1] = im[i];
                                    }
                            }
                        }
                    }
                }
                // this warp is done with the accumulator (its values are in registers):
                // release it on the even CTA at CTA scope
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(tempty0_lead + 8 * acc);
            }
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

template <int BN, int STAGES, int FMT, int CL>
cudaError_t launch_cfg(const tcbf_plan_s &pl, const void *Wp, const void *Xp, float *Y,
                       cudaStream_t s, int raster) {
    if (CL > 1 && pl.m_prefix)   // uneven batches walk per-batch m-tiles: no clusters
        return launch_cfg<BN, STAGES, FMT, 1>(pl, Wp, Xp, Y, s, raster);
    // row length in elements of the tensor map: FP16 elements or split-FP8 bytes
    constexpr bool BLK = FMT == kFmtSplit8Blk;
    constexpr bool SPLIT = FMT == kFmtSplit8 || BLK;
    constexpr bool TF32 = FMT == kFmtTf32;
    static_assert(!BLK || BN == kFp8BlkRowsX, "block-scaled tiles span one X scale group");
    const int64_t row = SPLIT ? pl.Kb2 : pl.Kp;
    const CUtensorMapDataType dt = SPLIT  ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                   : TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                          : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const int64_t esz = SPLIT ? 1 : TF32 ? 4 : 2;
    using C = Cfg<BN, STAGES, BLK>;
    const tcbf_problem &p = pl.p;
    CUtensorMap tmW, tmX;
    {
        const uint64_t dims[3] = {static_cast<uint64_t>(row), static_cast<uint64_t>(p.M),
                                  static_cast<uint64_t>(2 * p.w_batches)};
        const uint64_t strides[2] = {static_cast<uint64_t>(row * esz),
                                     static_cast<uint64_t>(w_plane_rows(pl) * row * esz)};
        const uint32_t box[3] = {static_cast<uint32_t>(128 / esz), BM, 2};
        if (encode_tiled(&tmW, dt, 3, const_cast<void *>(Wp), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const uint64_t dims[3] = {static_cast<uint64_t>(row), static_cast<uint64_t>(p.N),
                                  static_cast<uint64_t>(2 * p.batch)};
        const uint64_t strides[2] = {static_cast<uint64_t>(row * esz),
                                     static_cast<uint64_t>(p.N * row * esz)};
        // clusters: each CTA loads a BN/CL-row slice of one plane per multicast
        const uint32_t box[3] = {static_cast<uint32_t>(128 / esz),
                                 static_cast<uint32_t>(BN / CL), CL == 1 ? 2u : 1u};
        if (encode_tiled(&tmX, dt, 3, const_cast<void *>(Xp), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    CUtensorMap tmY;
    const int tma_store = (p.N % 2 == 0) ? 1 : 0;
    if (tma_store) {
        const uint64_t dims[3] = {static_cast<uint64_t>(2 * p.N), static_cast<uint64_t>(p.M),
                                  static_cast<uint64_t>(p.batch)};
        const uint64_t strides[2] = {static_cast<uint64_t>(p.N * 8),
                                     static_cast<uint64_t>(p.M * p.N * 8)};
        const uint32_t box[3] = {32, 32, 1};
        if (encode_tiled(&tmY, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, Y, dims, strides, box,
                         CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    } else {
        tmY = tmX;   // unused
    }
    GemmArgs a;
    a.Y = Y;
    a.w_exps = (!SPLIT || BLK) ? nullptr
               : pl.w_exps ? pl.w_exps
                           : reinterpret_cast<const int32_t *>(static_cast<const uint8_t *>(Wp) +
                                                               p.w_batches * 2 * p.M * row);
    a.x_exps = (SPLIT && !BLK) ? reinterpret_cast<const int32_t *>(static_cast<const uint8_t *>(Xp) +
                                                                   p.batch * 2 * p.N * row)
                               : nullptr;
    // block-scaled FP8: the scale tiles after the packed bytes (a sub-plan's
    // W tiles given by the caller through w_exps)
    a.w_sf = !BLK ? nullptr
             : pl.w_exps ? reinterpret_cast<const uint8_t *>(pl.w_exps)
                         : static_cast<const uint8_t *>(Wp) + p.w_batches * 2 * p.M * row;
    a.x_sf = BLK ? static_cast<const uint8_t *>(Xp) + p.batch * 2 * p.N * row : nullptr;
    a.w_sf_tiles = static_cast<int>(ceil_div(w_plane_rows(pl), kFp8BlkRowsW));
    a.x_sf_groups = static_cast<int>(ceil_div(p.N, kFp8BlkRowsX));
    a.tma_store = tma_store;
    a.products = split_products(pl);
    a.drop_fill = (CL == 1 && pl.debug_drop_fill >= 0) ? static_cast<int>(pl.debug_drop_fill) : -1;
    a.status = pl.status;
    a.M = static_cast<int>(p.M);
    a.N = static_cast<int>(p.N);
    a.K = static_cast<int>(p.K);
    a.per_w = static_cast<int>(pl.per_w);
    a.tiles.prefix = pl.m_prefix;
    a.tiles.batch = static_cast<int>(p.batch);
    a.tiles.m_tiles = static_cast<int>(ceil_div(p.M, BM));
    a.tiles.n_tiles = static_cast<int>(ceil_div(p.N, BN));
    a.tiles.raster = raster;
    // hi-only FP8 rows carry 128 K in each 128-byte stage row, the other
    // formats 64 (FP16, or 64 hi + 64 lo bytes); chunks stay 2048 K
    a.kps = (SPLIT && fp8_hi_only(p.flags)) ? 2 * BK : TF32 ? BK / 2 : BK;
    a.num_kb = static_cast<int>(ceil_div(p.K, a.kps));
    if (p.K > kPromoteK) {
        if (4 * BN > 512) return cudaErrorInvalidConfiguration;   // no TMEM room for the sum
        a.kc_blocks = kChunkBlocks * BK / a.kps;
    } else {
        a.kc_blocks = a.num_kb;
    }
    a.chunks = (a.num_kb + a.kc_blocks - 1) / a.kc_blocks;
    const int64_t m_units = CL == 1 ? (pl.m_prefix ? pl.m_tiles_sum : int64_t(a.tiles.m_tiles) * p.batch)
                                    : ceil_div(a.tiles.m_tiles, CL) * p.batch;
    const int64_t total = m_units * a.tiles.n_tiles;     // tiles, or cluster tiles
    if (total > 0x7fffffff) return cudaErrorInvalidValue;
    a.total_tiles = static_cast<int>(total);
    auto kern = cgemm_tc_kernel<BN, STAGES, FMT, CL>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (CL == 1) {
        const int grid = static_cast<int>(std::min<int64_t>(total, pl.num_sms));
        kern<<<grid, kThreads, C::SMEM_BYTES, s>>>(tmW, tmX, tmY, a);
        return cudaGetLastError();
    }
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = C::SMEM_BYTES;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // persistent grid: as many clusters as can be resident at once
    // resident clusters per device, measured once (benign if two threads both measure)
    static std::atomic<int> max_clusters[64];
    int mc = max_clusters[pl.device & 63].load(std::memory_order_relaxed);
    if (mc == 0) {
        cfg.gridDim = dim3(pl.num_sms / CL * CL);
        e = cudaOccupancyMaxActiveClusters(&mc, kern, &cfg);
        if (e != cudaSuccess) return e;
        if (mc < 1) return cudaErrorInvalidConfiguration;
        max_clusters[pl.device & 63].store(mc, std::memory_order_relaxed);
    }
    cfg.gridDim = dim3(static_cast<unsigned>(std::min<int64_t>(total, mc)) * CL);
    e = cudaLaunchKernelEx(&cfg, kern, tmW, tmX, tmY, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int BN, int STAGES, int FMT>
cudaError_t launch_pair(const tcbf_plan_s &pl, const void *Wp, const void *Xp, float *Y,
                        cudaStream_t s, int raster) {
    if (pl.m_prefix)   // uneven batches walk per-batch m-tiles: one-SM tiles
        return launch_cfg<BN, 3, FMT, 1>(pl, Wp, Xp, Y, s, raster);
    using C = CfgPair<BN, STAGES>;
    constexpr bool SPLIT = FMT == kFmtSplit8;
    constexpr bool TF32 = FMT == kFmtTf32;
    const int64_t row = SPLIT ? pl.Kb2 : pl.Kp;
    const CUtensorMapDataType dt = SPLIT  ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                   : TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                          : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const int64_t esz = SPLIT ? 1 : TF32 ? 4 : 2;
    const tcbf_problem &p = pl.p;
    CUtensorMap tmW, tmX, tmY;
    {
        const uint64_t dims[3] = {static_cast<uint64_t>(row), static_cast<uint64_t>(p.M),
                                  static_cast<uint64_t>(2 * p.w_batches)};
        const uint64_t strides[2] = {static_cast<uint64_t>(row * esz),
                                     static_cast<uint64_t>(w_plane_rows(pl) * row * esz)};
        const uint32_t box[3] = {static_cast<uint32_t>(128 / esz), BM, 2};
        if (encode_tiled(&tmW, dt, 3, const_cast<void *>(Wp), dims, strides, box,
                         CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const uint64_t dims[3] = {static_cast<uint64_t>(row), static_cast<uint64_t>(p.N),
                                  static_cast<uint64_t>(2 * p.batch)};
        const uint64_t strides[2] = {static_cast<uint64_t>(row * esz),
                                     static_cast<uint64_t>(p.N * row * esz)};
        const uint32_t box[3] = {static_cast<uint32_t>(128 / esz), BN / 2, 2};   // this CTA's half
        if (encode_tiled(&tmX, dt, 3, const_cast<void *>(Xp), dims, strides, box,
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
        if (encode_tiled(&tmY, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, Y, dims, strides, box,
                         CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    } else {
        tmY = tmX;   // unused
    }
    GemmArgs a;
    a.Y = Y;
    a.w_exps = !SPLIT ? nullptr
               : pl.w_exps ? pl.w_exps
                           : reinterpret_cast<const int32_t *>(static_cast<const uint8_t *>(Wp) +
                                                               p.w_batches * 2 * p.M * row);
    a.x_exps = SPLIT ? reinterpret_cast<const int32_t *>(static_cast<const uint8_t *>(Xp) +
                                                        p.batch * 2 * p.N * row)
                     : nullptr;
    a.w_sf = nullptr;
    a.x_sf = nullptr;
    a.w_sf_tiles = a.x_sf_groups = 0;
    a.tma_store = tma_store;
    a.products = split_products(pl);
    a.drop_fill = -1;
    a.status = pl.status;
    a.M = static_cast<int>(p.M);
    a.N = static_cast<int>(p.N);
    a.K = static_cast<int>(p.K);
    a.per_w = static_cast<int>(pl.per_w);
    a.tiles.prefix = nullptr;
    a.tiles.batch = static_cast<int>(p.batch);
    a.tiles.m_tiles = static_cast<int>(ceil_div(p.M, BM));
    a.tiles.n_tiles = static_cast<int>(ceil_div(p.N, BN));
    a.tiles.raster = 0;
    // hi-only FP8 rows carry 128 K in each 128-byte stage row, the other
    // formats 64 (FP16, or 64 hi + 64 lo bytes); chunks stay 2048 K
    a.kps = (SPLIT && fp8_hi_only(p.flags)) ? 2 * BK : TF32 ? BK / 2 : BK;
    a.num_kb = static_cast<int>(ceil_div(p.K, a.kps));
    if (p.K > kPromoteK) {
        if (4 * BN > 512) return cudaErrorInvalidConfiguration;
        a.kc_blocks = kChunkBlocks * BK / a.kps;
    } else {
        a.kc_blocks = a.num_kb;
    }
    a.chunks = (a.num_kb + a.kc_blocks - 1) / a.kc_blocks;
    const int64_t total = ceil_div(a.tiles.m_tiles, 2) * p.batch * a.tiles.n_tiles;
    if (total > 0x7fffffff) return cudaErrorInvalidValue;
    a.total_tiles = static_cast<int>(total);
    auto kern = cgemm_pair_kernel<BN, STAGES, FMT>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = C::SMEM_BYTES;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // resident clusters per device, measured once (benign if two threads both measure)
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

struct ConfigEntry {
    const char *name;
    int bn;
    int raster;
    cudaError_t (*fn)(const tcbf_plan_s &, const void *, const void *, float *, cudaStream_t, int);
};

const ConfigEntry kConfigs[] = {
    {"f16 BM128 BN128 BK64 stages3 tmem-double n-fastest", 128, 0, launch_cfg<128, 3, kFmtF16, 1>},
    {"f16 BM128 BN256 BK64 stages2 tmem-single n-fastest", 256, 0, launch_cfg<256, 2, kFmtF16, 1>},
    {"f16 BM128 BN64 BK64 stages4 tmem-double n-fastest", 64, 0, launch_cfg<64, 4, kFmtF16, 1>},
    {"f16 BM128 BN128 BK64 stages3 tmem-double m-fastest", 128, 1, launch_cfg<128, 3, kFmtF16, 1>},
    {"f16 BM128 BN256 BK64 stages2 tmem-single m-fastest", 256, 1, launch_cfg<256, 2, kFmtF16, 1>},
    {"f16 BM128 BN64 BK64 stages4 tmem-double m-fastest", 64, 1, launch_cfg<64, 4, kFmtF16, 1>},
    {"f16 BM128 BN128 BK64 stages3 tmem-double cluster2 X-multicast", 128, 0, launch_cfg<128, 3, kFmtF16, 2>},
    {"f16 BM128 BN128 BK64 stages3 tmem-double cluster4 X-multicast", 128, 0, launch_cfg<128, 3, kFmtF16, 4>},
    {"f16 2-SM pair BM256 BN128 BK64 stages4 tmem-double", 128, 0, launch_pair<128, 4, kFmtF16>},
};

// split-FP8: the same tile shapes, index for index
const ConfigEntry kConfigsSplit[] = {
    {"fp8split BM128 BN128 BK64 stages3 tmem-double n-fastest", 128, 0, launch_cfg<128, 3, kFmtSplit8, 1>},
    {"fp8split BM128 BN256 BK64 stages2 tmem-single n-fastest", 256, 0, launch_cfg<256, 2, kFmtSplit8, 1>},
    {"fp8split BM128 BN64 BK64 stages4 tmem-double n-fastest", 64, 0, launch_cfg<64, 4, kFmtSplit8, 1>},
    {"fp8split BM128 BN128 BK64 stages3 tmem-double m-fastest", 128, 1, launch_cfg<128, 3, kFmtSplit8, 1>},
    {"fp8split BM128 BN256 BK64 stages2 tmem-single m-fastest", 256, 1, launch_cfg<256, 2, kFmtSplit8, 1>},
    {"fp8split BM128 BN64 BK64 stages4 tmem-double m-fastest", 64, 1, launch_cfg<64, 4, kFmtSplit8, 1>},
    {"fp8split BM128 BN128 BK64 stages3 tmem-double cluster2 X-multicast", 128, 0, launch_cfg<128, 3, kFmtSplit8, 2>},
    {"fp8split BM128 BN128 BK64 stages3 tmem-double cluster4 X-multicast", 128, 0, launch_cfg<128, 3, kFmtSplit8, 4>},
    {"fp8split 2-SM pair BM256 BN128 BK64 stages4 tmem-double", 128, 0, launch_pair<128, 4, kFmtSplit8>},
};

// block-scaled split-FP8: 128 x 64 tiles (a tile spans one 64-sample X
// scale group; the scale columns sit above the accumulators in TMEM)
const ConfigEntry kConfigsSplitBlk[] = {
    {"fp8split block-scaled mxf8f6f4 BM128 BN64 BK64 stages3 tmem-double n-fastest", 64, 0,
     launch_cfg<64, 3, kFmtSplit8Blk, 1>},
    {"fp8split block-scaled mxf8f6f4 BM128 BN64 BK64 stages3 tmem-double m-fastest", 64, 1,
     launch_cfg<64, 3, kFmtSplit8Blk, 1>},
};

// TF32: the same tile shapes, index for index (32 K per 128-byte stage row)
const ConfigEntry kConfigsTf32[] = {
    {"tf32 BM128 BN128 BK32 stages3 tmem-double n-fastest", 128, 0, launch_cfg<128, 3, kFmtTf32, 1>},
    {"tf32 BM128 BN256 BK32 stages2 tmem-single n-fastest", 256, 0, launch_cfg<256, 2, kFmtTf32, 1>},
    {"tf32 BM128 BN64 BK32 stages4 tmem-double n-fastest", 64, 0, launch_cfg<64, 4, kFmtTf32, 1>},
    {"tf32 BM128 BN128 BK32 stages3 tmem-double m-fastest", 128, 1, launch_cfg<128, 3, kFmtTf32, 1>},
    {"tf32 BM128 BN256 BK32 stages2 tmem-single m-fastest", 256, 1, launch_cfg<256, 2, kFmtTf32, 1>},
    {"tf32 BM128 BN64 BK32 stages4 tmem-double m-fastest", 64, 1, launch_cfg<64, 4, kFmtTf32, 1>},
    {"tf32 BM128 BN128 BK32 stages3 tmem-double cluster2 X-multicast", 128, 0, launch_cfg<128, 3, kFmtTf32, 2>},
    {"tf32 BM128 BN128 BK32 stages3 tmem-double cluster4 X-multicast", 128, 0, launch_cfg<128, 3, kFmtTf32, 4>},
    {"tf32 2-SM pair BM256 BN128 BK32 stages4 tmem-double", 128, 0, launch_pair<128, 4, kFmtTf32>},
};

}  // namespace

int gemm_f16_num_configs() { return static_cast<int>(sizeof(kConfigs) / sizeof(kConfigs[0])); }

const char *gemm_f16_config_name(int config) {
    if (config < 0 || config >= gemm_f16_num_configs()) return "invalid";
    return kConfigs[config].name;
}

bool gemm_f16_config_valid(int config, int64_t K) {
    if (config < 0 || config >= gemm_f16_num_configs()) return false;
    return K <= kPromoteK || kConfigs[config].bn <= 128;
}

const char *gemm_split8_config_name(int config) {
    if (config < 0 || config >= gemm_f16_num_configs()) return "invalid";
    return kConfigsSplit[config].name;
}

const char *gemm_tf32_config_name(int config) {
    if (config < 0 || config >= gemm_f16_num_configs()) return "invalid";
    return kConfigsTf32[config].name;
}

cudaError_t launch_gemm_tf32(const tcbf_plan_s &pl, const void *Wp, const void *Xp, float *Y,
                             cudaStream_t s) {
    const int c = (pl.config >= 0 && pl.config < gemm_f16_num_configs()) ? pl.config : 0;
    return kConfigsTf32[c].fn(pl, Wp, Xp, Y, s, kConfigsTf32[c].raster);
}

int gemm_split8_blk_num_configs() {
    return static_cast<int>(sizeof(kConfigsSplitBlk) / sizeof(kConfigsSplitBlk[0]));
}

const char *gemm_split8_blk_config_name(int config) {
    if (config < 0 || config >= gemm_split8_blk_num_configs()) return "invalid";
    return kConfigsSplitBlk[config].name;
}

cudaError_t launch_gemm_split8(const tcbf_plan_s &pl, const void *Wp, const void *Xp, float *Y,
                               cudaStream_t s) {
    if (fp8_block_scaled(pl.p.flags)) {
        const int c = (pl.config >= 0 && pl.config < gemm_split8_blk_num_configs()) ? pl.config : 0;
        return kConfigsSplitBlk[c].fn(pl, Wp, Xp, Y, s, kConfigsSplitBlk[c].raster);
    }
    const int c = (pl.config >= 0 && pl.config < gemm_f16_num_configs()) ? pl.config : 0;
    return kConfigsSplit[c].fn(pl, Wp, Xp, Y, s, kConfigsSplit[c].raster);
}

cudaError_t launch_gemm_f16(const tcbf_plan_s &pl, const void *Wp, const void *Xp, float *Y,
                            cudaStream_t s) {
    if (pl.p.flags & TCBF_FLAG_STACKED_X) return launch_gemm_f16_stacked(pl, Wp, Xp, Y, s);
    if (interleaved_x(pl)) {
        if (ix_fused_ok(pl)) return launch_gemm_f16_ix(pl, Wp, Xp, Y, s);
        // shapes the fused kernel cannot take: transpose/pack into the plan's
        // planes, then the planar four-MMA kernel
        if (!pl.ix_planes) return cudaErrorInvalidValue;
        const cudaError_t e = launch_pack_f16_x(pl, TCBF_SRC_CF16, Xp, pl.ix_planes, s);
        if (e != cudaSuccess) return e;
        return kConfigs[0].fn(pl, Wp, pl.ix_planes, Y, s, kConfigs[0].raster);
    }
    const int c = (pl.config >= 0 && pl.config < gemm_f16_num_configs()) ? pl.config : 0;
    return kConfigs[c].fn(pl, Wp, Xp, Y, s, kConfigs[c].raster);
}

}  // namespace tcbf
