// gemm_f16_ix.cu — FP16 complex GEMM that reads the samples in their
// interleaved complex layout, with no transpose/pack pass over X.
//
// The paper's GEMM needs its inputs split into real and imaginary planes and
// tiled in device memory, which a separate transpose kernel does (Sec. III);
// skipping that pass is one of its future-work items (Sec. VI).  The
// caller's samples X[b] are K rows of N interleaved complex FP16 values: a
// real K x 2N matrix whose 2N columns are contiguous, which is exactly an
// MN-major B operand of the tensor core, loaded by TMA as it lies in memory.
// A real MMA with that operand gives, per beam, the products with Xr and Xi
// side by side in adjacent columns:
//     (Wr X)[m, 2n] = (Wr Xr)[m, n],   (Wr X)[m, 2n + 1] = (Wr Xi)[m, n],
//     (Wi X)[m, 2n] = (Wi Xr)[m, n],   (Wi X)[m, 2n + 1] = (Wi Xi)[m, n],
// and the complex product of Sec. III-B is
//     Re = (Wr X)[2n] - (Wi X)[2n + 1],   Im = (Wr X)[2n + 1] + (Wi X)[2n].
// The A operand (packed W planes) is loaded as 8-row groups alternating the
// planes: rows 16g .. 16g+7 hold Wr of beams 8g .. 8g+7 and rows 16g+8 ..
// 16g+15 hold Wi of the same beams.  One M = 128 MMA then forms Wr X and
// Wi X of 64 beams at once, and in tensor memory the two products of a beam
// sit in lanes r and r + 8 of a 16-lane group, which one .16x256b TMEM load
// hands to the same thread: Re and Im form in FP32 registers.  One N = 256 MMA per
// 16-K step covers 64 beams x 128 samples on one SM, or, on SM pairs
// (cta_group::2, M = 256), 128 beams x 128 samples with each CTA holding 64
// beams of W and 64 samples (128 real columns) of X.  A tile's accumulator
// takes 256 TMEM columns, so two of them let one tile drain while the next
// tile's MMAs run.  Long K is accumulated in promoted chunks as in the
// planar kernels: the chunks alternate between the two accumulators, the
// FP32 round-to-nearest running sum moving into each new chunk's one.
// Every wait is bounded.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>

#include "ptx.cuh"
#include "tcbf_internal.h"

namespace tcbf {
namespace {

using namespace dev;

constexpr int IBN = 128;              // samples per tile: 256 real columns
constexpr int kIxThreads = 320;       // producer, MMA issuer, 8 epilogue warps
constexpr int kIxPromoteK = 4096;     // K above this is accumulated in promoted chunks
constexpr int kIxChunkK = 2048;       // K per promoted chunk
constexpr int kIxGroupM = 8;          // beam tiles per group of the tile order

// BKS: K per stage (64 or 128).  A stage holds the CTA's 64 beams of W as
// BKS / 64 blocks of 128 rows x 128 bytes (64 K each), then its columns of
// X as chunks of 64 real columns x BKS K rows.
template <bool PAIR, int BKS, int STAGES>
struct CfgIx {
    static constexpr int A_BLOCK = 128 * 64 * 2;              // 16 KB: 64 beams x 2 planes x 64 K
    static constexpr int A_BYTES = A_BLOCK * (BKS / 64);
    static constexpr int A_GROUP = 16 * 128;                  // 2 KB: one 8-beam group, both planes
    static constexpr int B_COLS = PAIR ? IBN : 2 * IBN;       // real columns of X in this CTA
    static constexpr int B_CHUNK = BKS * 128;                 // 64 columns x BKS K rows
    static constexpr int B_BYTES = B_COLS / 64 * B_CHUNK;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int ACC_COLS = 2 * IBN;                  // 256 columns per accumulator
    static constexpr int TMEM_COLS = 2 * ACC_COLS;
    static constexpr int STAGE_BUF = 2 * 8 * 128;             // 8 beams x 32 samples of Y
    static constexpr int STAGING_BYTES = 8 * 2 * STAGE_BUF;   // two buffers per epilogue warp
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + STAGING_BYTES + 256 + 1024;
    static_assert(SMEM_BYTES <= 232448, "shared memory");
    static_assert(16 * STAGES + 48 <= 256, "barrier block");
};

struct IxArgs {
    uint32_t *status;
    int M, N, K;
    int per_w;
    int batch;
    int m_tiles;        // beam tiles per batch: 64 beams (one SM) or 128 (SM pair)
    int n_tiles;        // sample tiles per batch (128 samples)
    int num_kb;         // K blocks of BKS
    int w5d;            // W loaded by one 5-D box per 64 K (M % 8 == 0), else per 8-beam group
    int x4d;            // X loaded by one 4-D box per stage (N % 32 == 0), else per 64 columns
    int y4d;            // Y stored by one 4-D box per 32 samples (N % 16 == 0), else two 3-D
    int kc_blocks;      // blocks per accumulation chunk
    int chunks;
    int total_tiles;
};

// Promotion of a long-K chunk by an interleaved-X epilogue warp (its 16
// TMEM lanes): the running sum S (at tS, the previous chunk's accumulator)
// plus the chunk's P (at tP), FP32 round-to-nearest, written over P.
template <int ACC_COLS>
__device__ __forceinline__ void ix_promote(uint32_t tP, uint32_t tS) {
#pragma unroll 1
    for (int g = 0; g < ACC_COLS / 64; ++g) {
        float v[32], sv[32];
        tmem_ld_16x256b_x8(tP + 64 * g, v);
        tmem_ld_16x256b_x8(tS + 64 * g, sv);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = __fadd_rn(sv[i], v[i]);
        tmem_st_16x256b_x8(tP + 64 * g, v);
    }
    tmem_st_wait();
}

// The output of one tile by an interleaved-X epilogue warp (the warp's 16
// TMEM lanes from tP): Re and Im of its 8 beams x 128 samples, stored 32
// samples at a time: two 1 KB boxes of 8 beams x 16 samples, one 4-D store
// of both when N % 16 == 0 (y4d: Y seen as 16-sample chunks x beams x
// batches), else two 3-D stores.
template <int ACC_COLS, int STAGE_BUF, int NBUF = 2>
__device__ __forceinline__ void ix_drain(uint32_t tP, int lane, uint32_t stage_buf, int &nstore,
                                         int nt, int N, int beam0, int b, const CUtensorMap *tmY,
                                         int y4d) {
    const int rb = lane >> 2;                             // beam within the group
    const int sq = lane & 3;                              // sample within each 4
    // the next block's tensor-memory load is issued before this block is
    // staged and stored, so its latency overlaps the stores
    float v[32];
    tmem_ld_16x256b_x8_nowait(tP, v);
#pragma unroll 1
    for (int c = 0; c < ACC_COLS / 64; ++c) {
        tmem_wait_ld_32(v);
        // v[4i..4i+3] = Wr Xr, Wr Xi, Wi Xr, Wi Xi of sample 4i + sq
        float re[8], im[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            re[i] = __fsub_rn(v[4 * i], v[4 * i + 3]);
            im[i] = __fadd_rn(v[4 * i + 1], v[4 * i + 2]);
        }
        if (c + 1 < ACC_COLS / 64) tmem_ld_16x256b_x8_nowait(tP + 64 * (c + 1), v);
        const int n0 = nt * IBN + 32 * c;     // first sample of the block
        if (n0 < N) {
            const uint32_t buf = stage_buf + (NBUF == 2 ? (nstore & 1) * STAGE_BUF : 0);
            if (lane == 0) {                       // the buffer's last stores have read it
                if (NBUF == 2)
                    bulk_wait_read<1>();
                else
                    bulk_wait_read<0>();
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int s16 = 4 * (i & 3) + sq;          // sample within its box
                const uint32_t addr = buf + (i >> 2) * 1024 + rb * 128 +
                                      ((((s16 >> 1) ^ rb) & 7) << 4) + ((s16 & 1) << 3);
                st_shared_v2(addr, re[i], im[i]);
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                if (y4d) {
                    tma_store_4d(tmY, buf, 0, beam0, n0 / 16, b);
                } else {
                    tma_store_3d(tmY, buf, 2 * n0, beam0, b);
                    if (n0 + 16 < N) tma_store_3d(tmY, buf + 1024, 2 * (n0 + 16), beam0, b);
                }
                bulk_commit();
            }
            ++nstore;
        }
    }
}

template <bool PAIR, int BKS, int STAGES>
__global__ void __launch_bounds__(kIxThreads, 1)
    cgemm_ix_kernel(const __grid_constant__ CUtensorMap tmW,
                    const __grid_constant__ CUtensorMap tmX,
                    const __grid_constant__ CUtensorMap tmY, const IxArgs args) {
    using C = CfgIx<PAIR, BKS, STAGES>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
    const uint32_t s0 = smem_u32(smem);
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
    const int rank = PAIR ? static_cast<int>(cluster_ctarank()) : 0;
    const bool leader = rank == 0;
    const int t_first = PAIR ? static_cast<int>(cluster_id_x()) : static_cast<int>(blockIdx.x);
    const int t_step = PAIR ? static_cast<int>(nclusters_x()) : static_cast<int>(gridDim.x);
    constexpr uint16_t kBoth = 3;
    // (batch, beam tile, sample tile) of tile t: groups of kIxGroupM beam
    // tiles, beam tiles fastest inside a group, then sample tiles
    auto decode = [&](int t, int &b, int &mt, int &nt) {
        const int per_b = args.m_tiles * args.n_tiles;
        b = t / per_b;
        const int local = t - b * per_b;
        const int group = local / (kIxGroupM * args.n_tiles);
        const int first = group * kIxGroupM;
        const int gm = min(kIxGroupM, args.m_tiles - first);
        const int in = local - group * kIxGroupM * args.n_tiles;
        mt = first + in % gm;
        nt = in / gm;
    };
    // first beam of this CTA's 64
    auto beam_base = [&](int mt) { return PAIR ? mt * 128 + 64 * rank : mt * 64; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);          // used in the even CTA of a pair
            mbar_init(empty0 + 8 * s, 1);         // the MMA issuer's commit
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, PAIR ? 16 : 8);  // 8 epilogue warps per CTA
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
        tma_prefetch_desc(&tmW);
        tma_prefetch_desc(&tmX);
        tma_prefetch_desc(&tmY);
    }
    if (warp == 1) {
        if (PAIR) {
            tmem_alloc_pair(smem_u32(tmem_slot), C::TMEM_COLS);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint32_t full0_lead = PAIR ? mapa_shared(full0, 0) : full0;
    const uint32_t tempty0_lead = PAIR ? mapa_shared(tempty0, 0) : tempty0;

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
                const int beam0 = beam_base(mt);
                const int col0 = 2 * nt * IBN + rank * C::B_COLS;   // first real column of X
                for (int kb = 0; kb < args.num_kb; ++kb) {
                    if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    const uint32_t dst = s0 + stage * C::STAGE_BYTES;
                    const int k0 = kb * BKS;
                    uint32_t fb;
                    if (PAIR) {
                        if (leader) mbar_arrive_expect_tx(full0 + 8 * stage, 2 * C::STAGE_BYTES);
                        fb = full0_lead + 8 * stage;
                    } else {
                        fb = full0 + 8 * stage;
                        mbar_arrive_expect_tx(fb, C::STAGE_BYTES);
                    }
                    // W: per 64 K, 8 groups of 8 beams, each group Wr rows then Wi rows
#pragma unroll
                    for (int kk = 0; kk < BKS / 64; ++kk) {
                        const uint32_t wdst = dst + kk * C::A_BLOCK;
                        if (args.w5d) {
                            if (PAIR)
                                tma_load_5d_pair(wdst, &tmW, fb, k0 + 64 * kk, 0, 0, beam0 / 8, bw);
                            else
                                tma_load_5d(wdst, &tmW, fb, k0 + 64 * kk, 0, 0, beam0 / 8, bw);
                        } else {
                            for (int g = 0; g < 8; ++g) {
                                if (PAIR)
                                    tma_load_3d_pair(wdst + g * C::A_GROUP, &tmW, fb, k0 + 64 * kk,
                                                     beam0 + 8 * g, 2 * bw);
                                else
                                    tma_load_3d(wdst + g * C::A_GROUP, &tmW, fb, k0 + 64 * kk,
                                                beam0 + 8 * g, 2 * bw);
                            }
                        }
                    }
                    // X: the CTA's columns, 64 per chunk
                    const uint32_t xdst = dst + C::A_BYTES;
                    if (args.x4d) {
                        if (PAIR)
                            tma_load_4d_pair(xdst, &tmX, fb, 0, k0, col0 / 64, b);
                        else
                            tma_load_4d(xdst, &tmX, fb, 0, k0, col0 / 64, b);
                    } else {
                        for (int c = 0; c < C::B_COLS / 64; ++c) {
                            if (PAIR)
                                tma_load_3d_pair(xdst + c * C::B_CHUNK, &tmX, fb, col0 + 64 * c, k0, b);
                            else
                                tma_load_3d(xdst + c * C::B_CHUNK, &tmX, fb, col0 + 64 * c, k0, b);
                        }
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
                // let every copy this CTA started land before it exits (in a
                // pair both CTAs' copies complete on the even CTA's barriers)
                if (leader) {
                    for (int s = 0; s < STAGES; ++s) {
                        if (issued > static_cast<uint32_t>(s)) {
                            const uint32_t count = (issued - s + STAGES - 1) / STAGES;
                            if (!mbar_wait(full0 + 8 * s, (count - 1) & 1u))
                                atomicOr(args.status, kErrTimeoutDrain);
                        }
                    }
                }
            } else if (PAIR) {
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
        // ---------------------------------------- MMA issuer (even CTA of a pair)
        if (lane == 0 && leader) {
            constexpr uint32_t kIdesc = idesc_f32acc_bmn(PAIR ? 256 : 128, 2 * IBN, 0);
            int stage = 0;
            uint32_t phase = 0;
            int ev = 0;
            const int nbuf = 2;   // promoted long K alternates them too
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
                    const uint32_t d = tmem_base + acc * C::ACC_COLS;
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
                        const int ksteps = min(BKS / 16, (args.K - kb * BKS + 15) / 16);
                        for (int j = 0; j < ksteps; ++j) {
                            const uint32_t accum = (kb > kb0 || j > 0) ? 1u : 0u;
                            // A: 32 bytes of K per step inside the 128-byte rows of
                            // its 64-K block; B: 16 K rows (two 1024-byte atoms) per
                            // step, 64-column chunks B_CHUNK apart
                            const uint64_t ad = sdesc_kmajor_sw128(a + (j >> 2) * C::A_BLOCK + 32 * (j & 3));
                            const uint64_t bd = sdesc_mnmajor_sw128(bx + 2048 * j, C::B_CHUNK, 1024);
                            if (PAIR)
                                mma_f16_pair(d, ad, bd, kIdesc, accum);
                            else
                                mma_f16(d, ad, bd, kIdesc, accum);
                        }
                        if (PAIR)
                            mma_commit_pair(empty0 + 8 * stage, kBoth);
                        else
                            mma_commit(empty0 + 8 * stage);
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    if (PAIR)
                        mma_commit_pair(tfull0 + 8 * acc, kBoth);
                    else
                        mma_commit(tfull0 + 8 * acc);
                }
            }
            if (!ok) {
                atomicOr(args.status, kErrTimeoutMma);
                *abort_flag = 1;
            }
            // every MMA issued must finish before tensor memory is released
            if (PAIR)
                mma_commit_pair(done_bar, 1);
            else
                mma_commit(done_bar);
            if (!mbar_wait(done_bar, 0)) atomicOr(args.status, kErrTimeoutDrain);
        }
    } else {
        // ---------------------------------------------------------- epilogue
        // Warps 2-9: warp w owns the 16 TMEM lanes 32 (w % 4) + 16 h .. +15,
        // h = (w - 2) / 4, i.e. one 8-beam group: Wr X of the 8 beams in its
        // first 8 lanes and Wi X of the same beams in the last 8.  A .16x256b
        // load hands each thread both products of one beam at the same two
        // columns (the Xr and Xi terms of one sample), so Re and Im form in
        // registers.  Per 64 columns (32 samples) the warp stages 8 beams x
        // 32 samples as two 8 x 128-byte boxes (128-byte swizzle) and stores
        // them with TMA.
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const uint32_t lane_off = static_cast<uint32_t>(quarter * 32 + half * 16) << 16;
        const uint32_t stage_buf = staging0 + (warp - 2) * 2 * C::STAGE_BUF;
        const int nbuf = 2;
        int ev = 0;
        int nstore = 0;
        bool ok = true;
        for (int t = t_first; t < args.total_tiles && ok; t += t_step) {
            int b, mt, nt;
            decode(t, b, mt, nt);
            const int beam0 = beam_base(mt) + 16 * quarter + 8 * half;
            for (int ch = 0; ch < args.chunks; ++ch, ++ev) {
                const int acc = ev % nbuf;
                const uint32_t aphase = (ev / nbuf) & 1;
                if (!mbar_wait(tfull0 + 8 * acc, aphase) || *abort_flag) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tP = tmem_base + lane_off + acc * C::ACC_COLS;
                if (ch > 0) {
                    // the sum moves into this chunk's accumulator; the previous
                    // one is then free for the next chunk's MMAs
                    ix_promote<C::ACC_COLS>(tP, tmem_base + lane_off + (acc ^ 1) * C::ACC_COLS);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if (PAIR)
                            mbar_arrive_remote(tempty0_lead + 8 * (acc ^ 1));
                        else
                            mbar_arrive(tempty0 + 8 * (acc ^ 1));
                    }
                }
                // a chunk before the last keeps its sum in its accumulator
                if (ch + 1 < args.chunks) continue;
                ix_drain<C::ACC_COLS, C::STAGE_BUF>(tP, lane, stage_buf, nstore, nt, args.N, beam0,
                                                   b, &tmY, args.y4d);
                // this warp is done with the accumulator: release it (in a pair,
                // on the even CTA's barrier; its values are in registers or
                // staged, so no cluster-scope fence is needed)
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (PAIR)
                        mbar_arrive_remote(tempty0_lead + 8 * acc);
                    else
                        mbar_arrive(tempty0 + 8 * acc);
                }
            }
        }
        if (lane == 0) bulk_wait<0>();   // all of this warp's stores done
        __syncwarp();
        if (!ok && lane == 0) {
            atomicOr(args.status, kErrTimeoutEpilogue);
            *abort_flag = 1;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync();             // no CTA leaves while its peer may signal it
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        if (PAIR)
            tmem_dealloc_pair(tmem_base, C::TMEM_COLS);
        else
            tmem_dealloc(tmem_base, C::TMEM_COLS);
    }
}

// Y [batch][M][2N] FP32 for the interleaved-X epilogue: 16-sample chunks x
// beams x batches (y4d, N % 16 == 0: a box is two chunks of 8 beams, 2 KB)
// or columns x beams x batches (boxes of one chunk of 8 beams, 1 KB).
CUresult encode_ix_y(CUtensorMap *tmY, float *Y, const tcbf_problem &p, int y4d) {
    if (y4d) {
        const uint64_t dims[4] = {32, static_cast<uint64_t>(p.M), static_cast<uint64_t>(p.N / 16),
                                  static_cast<uint64_t>(p.batch)};
        const uint64_t strides[3] = {static_cast<uint64_t>(p.N * 8), 128,
                                     static_cast<uint64_t>(p.M * p.N * 8)};
        const uint32_t box[4] = {32, 8, 2, 1};
        return encode_tiled(tmY, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Y, dims, strides, box,
                            CU_TENSOR_MAP_SWIZZLE_128B);
    }
    const uint64_t dims[3] = {static_cast<uint64_t>(2 * p.N), static_cast<uint64_t>(p.M),
                              static_cast<uint64_t>(p.batch)};
    const uint64_t strides[2] = {static_cast<uint64_t>(p.N * 8), static_cast<uint64_t>(p.M * p.N * 8)};
    const uint32_t box[3] = {32, 8, 1};
    return encode_tiled(tmY, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, Y, dims, strides, box,
                        CU_TENSOR_MAP_SWIZZLE_128B);
}

template <bool PAIR, int BKS, int STAGES>
cudaError_t launch_ix(const tcbf_plan_s &pl, const void *Wp, const void *X, float *Y,
                      cudaStream_t s) {
    using C = CfgIx<PAIR, BKS, STAGES>;
    const tcbf_problem &p = pl.p;
    // the samples' rows (4N bytes) must be 16-byte multiples for TMA
    if (p.N % 4 != 0 || pl.m_prefix) return cudaErrorInvalidValue;
    CUtensorMap tmW, tmX, tmY;
    const int w5d = p.M % 8 == 0 ? 1 : 0;
    const int x4d = p.N % 32 == 0 ? 1 : 0;
    const uint64_t wrow = static_cast<uint64_t>(pl.Kp * 2);
    const uint64_t wplane = static_cast<uint64_t>(w_plane_rows(pl)) * wrow;
    if (w5d) {
        // packed W [w_batches][2][rows][Kp] as (k, row in group, plane, group,
        // weight batch): one box = 64 K of 8 groups x both planes x 8 rows
        const uint64_t dims[5] = {static_cast<uint64_t>(pl.Kp), 8, 2, static_cast<uint64_t>(p.M / 8),
                                  static_cast<uint64_t>(p.w_batches)};
        const uint64_t strides[4] = {wrow, wplane, 8 * wrow, 2 * wplane};
        const uint32_t box[5] = {64, 8, 2, 8, 1};
        if (encode_tiled(&tmW, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 5, const_cast<void *>(Wp), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    } else {
        // (k, row, plane + 2 x weight batch): boxes of 64 K x 8 beams x both planes
        const uint64_t dims[3] = {static_cast<uint64_t>(pl.Kp), static_cast<uint64_t>(p.M),
                                  static_cast<uint64_t>(2 * p.w_batches)};
        const uint64_t strides[2] = {wrow, wplane};
        const uint32_t box[3] = {64, 8, 2};
        if (encode_tiled(&tmW, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void *>(Wp), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const uint64_t xrow = static_cast<uint64_t>(p.N * 4);
    if (x4d) {
        // X [batch][K][2N] FP16 as (column in chunk, k, 64-column chunk, batch):
        // one box = the CTA's chunks x BKS rows
        const uint64_t dims[4] = {64, static_cast<uint64_t>(p.K), static_cast<uint64_t>(2 * p.N / 64),
                                  static_cast<uint64_t>(p.batch)};
        const uint64_t strides[3] = {xrow, 128, static_cast<uint64_t>(p.K) * xrow};
        const uint32_t box[4] = {64, BKS, C::B_COLS / 64, 1};
        if (encode_tiled(&tmX, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, const_cast<void *>(X), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    } else {
        // X [batch][K][2N] FP16 as it lies: boxes of 64 real columns x BKS rows
        const uint64_t dims[3] = {static_cast<uint64_t>(2 * p.N), static_cast<uint64_t>(p.K),
                                  static_cast<uint64_t>(p.batch)};
        const uint64_t strides[2] = {xrow, static_cast<uint64_t>(p.K) * xrow};
        const uint32_t box[3] = {64, BKS, 1};
        if (encode_tiled(&tmX, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void *>(X), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const int y4d = p.N % 16 == 0 ? 1 : 0;
    if (encode_ix_y(&tmY, Y, p, y4d) != CUDA_SUCCESS) return cudaErrorInvalidValue;
    IxArgs a;
    a.status = pl.status;
    a.M = static_cast<int>(p.M);
    a.N = static_cast<int>(p.N);
    a.K = static_cast<int>(p.K);
    a.per_w = static_cast<int>(pl.per_w);
    a.batch = static_cast<int>(p.batch);
    a.m_tiles = static_cast<int>(ceil_div(p.M, PAIR ? 128 : 64));
    a.n_tiles = static_cast<int>(ceil_div(p.N, IBN));
    a.num_kb = static_cast<int>(ceil_div(p.K, BKS));
    a.kc_blocks = p.K > kIxPromoteK ? kIxChunkK / BKS : a.num_kb;
    a.w5d = w5d;
    a.x4d = x4d;
    a.y4d = y4d;
    a.chunks = (a.num_kb + a.kc_blocks - 1) / a.kc_blocks;
    const int64_t total = int64_t(a.m_tiles) * a.n_tiles * p.batch;
    if (total > 0x7fffffff) return cudaErrorInvalidValue;
    a.total_tiles = static_cast<int>(total);
    auto kern = cgemm_ix_kernel<PAIR, BKS, STAGES>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (!PAIR) {
        const int grid = static_cast<int>(std::min<int64_t>(total, pl.num_sms));
        kern<<<grid, kIxThreads, C::SMEM_BYTES, s>>>(tmW, tmX, tmY, a);
        return cudaGetLastError();
    }
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kIxThreads);
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

// ===========================================================================
// Resident weights, for short K (K <= 384, the radio block's 288): each CTA of
// a pair keeps its 64 beams of W for all of K in shared memory (up to six
// 16 KB blocks of 64 K, 8-beam groups alternating Wr and Wi as above) and
// runs every sample tile of its (batch, 128-beam) unit against them, so only
// X streams through the ring: per output, half the operand bytes from L2 of
// the streaming kernel.  A unit's W is loaded once its predecessor's MMAs
// are done (the MMA thread commits a W-empty barrier after a unit's last
// tile), while the producer already streams the new unit's X.  A pair runs
// the per_w products that share a weight batch back to back on the same
// resident W (one W load per super-unit of weight batch x 128 beams) unless
// those coarser super-units would leave the last wave of pairs emptier (small
// batches), and super-units run beam rows fastest, so the pairs working at
// one time share the same products' X in L2.  One accumulation chunk (no promotion at this K).
// The X ring's depth is what bounds the kernel (its loads wait on L2
// latency, not bandwidth: half the X bytes per stage ran in the same time),
// so the four-stage form (K <= 320: up to five W blocks) gives up the
// second staging buffer of each epilogue warp to fit a fourth 32 KB stage
// (radio block 4.52 -> 3.97 ms); the three-stage form keeps two staging
// buffers and covers K <= 384.
// ===========================================================================
// STAGES X stages of BKS K rows each, NBUF staging buffers per epilogue
// warp, W resident for K <= MAXK (MAXK / 64 blocks)
template <int STAGES, int BKS, int NBUF_, int MAXK>
struct CfgIxW {
    static constexpr int MAX_K = MAXK;
    static constexpr int NBUF = NBUF_;
    static constexpr int W_BLOCK = 128 * 64 * 2;              // 64 beams x 2 planes x 64 K
    static constexpr int B_CHUNK = BKS * 128;                 // 64 real columns x BKS K rows
    static constexpr int X_STAGE = 2 * B_CHUNK;               // this CTA's 128 real columns
    static constexpr int ACC_COLS = 2 * IBN;
    static constexpr int TMEM_COLS = 2 * ACC_COLS;
    static constexpr int STAGE_BUF = 2 * 8 * 128;
    static constexpr int STAGING_BYTES = 8 * NBUF * STAGE_BUF;
    static constexpr int BAR_BYTES = 16 * STAGES + 64;
    static_assert(BAR_BYTES <= 256, "barrier block");
    static __host__ __device__ constexpr int smem_bytes(int kb64) {
        return kb64 * W_BLOCK + STAGES * X_STAGE + STAGING_BYTES + 256 + 1024;
    }
    static_assert(BKS % 16 == 0 && B_CHUNK % 1024 == 0, "whole 8-row swizzle atoms per stage");
    static_assert((MAX_K / 64) * W_BLOCK + STAGES * X_STAGE + STAGING_BYTES + 256 + 1024 <= 232448,
                  "shared memory");
};

struct IxWArgs {
    uint32_t *status;
    int M, N, K;
    int per_w;
    int kb64;           // 64-K blocks of resident W
    int m_tiles;        // 128-beam pair rows per batch
    int n_tiles;        // 128-sample tiles per batch
    int num_kb;         // X stages per tile
    int group;          // products per super-unit: 1, or per_w (they share W)
    int total_su;       // batch / group x m_tiles super-units
    int w5d, x4d, y4d;
};

template <int STAGES, int BKS, int NBUF, int MAXK>
__global__ void __launch_bounds__(kIxThreads, 1)
    cgemm_ix_wres_kernel(const __grid_constant__ CUtensorMap tmW,
                         const __grid_constant__ CUtensorMap tmX,
                         const __grid_constant__ CUtensorMap tmY, const IxWArgs args) {
    using C = CfgIxW<STAGES, BKS, NBUF, MAXK>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t *smem = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
    const uint32_t s0 = smem_u32(smem);
    const uint32_t w0 = s0;                                        // resident W
    const uint32_t x0 = s0 + args.kb64 * C::W_BLOCK;               // X ring
    const uint32_t staging0 = x0 + STAGES * C::X_STAGE;
    const uint32_t bar0 = staging0 + C::STAGING_BYTES;
    const uint32_t full0 = bar0;                       // STAGES x 8 bytes
    const uint32_t empty0 = full0 + 8 * STAGES;        // STAGES x 8
    const uint32_t tfull0 = empty0 + 8 * STAGES;       // 2 x 8
    const uint32_t tempty0 = tfull0 + 16;              // 2 x 8
    const uint32_t done_bar = tempty0 + 16;            // 8
    const uint32_t wfull = done_bar + 8;               // 8: this unit's W has landed
    const uint32_t wempty = wfull + 8;                 // 8: the last unit's MMAs are done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + (bar0 - s0) + 16 * STAGES + 56);
    volatile uint32_t *abort_flag = tmem_slot + 1;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int rank = static_cast<int>(cluster_ctarank());
    const bool leader = rank == 0;
    const int u_first = static_cast<int>(cluster_id_x());
    const int u_step = static_cast<int>(nclusters_x());
    constexpr uint16_t kBoth = 3;
    // The pair's i-th unit: super-units (group of products, 128-beam row)
    // strided over the pairs, each run as its `group` products one after the
    // other; when the group is the products that share a weight batch, the
    // resident W is loaded once per super-unit.
    auto unit = [&](int i, int &b, int &mt, int &sub) -> bool {
        const int su = u_first + (i / args.group) * u_step;
        if (su >= args.total_su) return false;
        sub = i - (i / args.group) * args.group;
        const int bg = su / args.m_tiles;
        mt = su - bg * args.m_tiles;
        b = bg * args.group + sub;
        return true;
    };

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(full0 + 8 * st, 1);
            mbar_init(empty0 + 8 * st, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, 16);     // 8 epilogue warps x 2 CTAs
        }
        mbar_init(done_bar, 1);
        mbar_init(wfull, 1);
        mbar_init(wempty, 1);
        *abort_flag = 0;
        fence_mbar_init();
        tma_prefetch_desc(&tmW);
        tma_prefetch_desc(&tmX);
        tma_prefetch_desc(&tmY);
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
    const uint32_t wfull_lead = mapa_shared(wfull, 0);

    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued = 0, wuse = 0;
            bool ok = true;
            int b, mt, sub;
            for (int i = 0; ok && unit(i, b, mt, sub); ++i) {
                const int bw = b / args.per_w;
                const int beam0 = mt * 128 + 64 * rank;
                if (sub == 0) {
                    // the super-unit's W, once the previous one's MMAs no longer read it
                    if (!mbar_wait(wempty, (wuse & 1u) ^ 1u) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    if (leader) mbar_arrive_expect_tx(wfull, 2 * args.kb64 * C::W_BLOCK);
                    for (int kk = 0; kk < args.kb64; ++kk) {
                        const uint32_t wdst = w0 + kk * C::W_BLOCK;
                        if (args.w5d) {
                            tma_load_5d_pair(wdst, &tmW, wfull_lead, 64 * kk, 0, 0, beam0 / 8, bw);
                        } else {
                            for (int g = 0; g < 8; ++g)
                                tma_load_3d_pair(wdst + g * 2048, &tmW, wfull_lead, 64 * kk,
                                                 beam0 + 8 * g, 2 * bw);
                        }
                    }
                    ++wuse;
                }
                for (int nt = 0; nt < args.n_tiles && ok; ++nt) {
                    const int col0 = 2 * nt * IBN + rank * 128;
                    for (int kb = 0; kb < args.num_kb; ++kb) {
                        if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u) || *abort_flag) {
                            ok = false;
                            break;
                        }
                        if (leader) mbar_arrive_expect_tx(full0 + 8 * stage, 2 * C::X_STAGE);
                        const uint32_t fb = full0_lead + 8 * stage;
                        const uint32_t xdst = x0 + stage * C::X_STAGE;
                        if (args.x4d) {
                            tma_load_4d_pair(xdst, &tmX, fb, 0, kb * BKS, col0 / 64, b);
                        } else {
                            for (int c = 0; c < 2; ++c)
                                tma_load_3d_pair(xdst + c * C::B_CHUNK, &tmX, fb, col0 + 64 * c,
                                                 kb * BKS, b);
                        }
                        ++issued;
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
            if (!ok) {
                atomicOr(args.status, kErrTimeoutProducer);
                *abort_flag = 1;
                if (leader) {
                    // every copy started must land before the CTAs exit
                    for (int st = 0; st < STAGES; ++st) {
                        if (issued > static_cast<uint32_t>(st)) {
                            const uint32_t count = (issued - st + STAGES - 1) / STAGES;
                            if (!mbar_wait(full0 + 8 * st, (count - 1) & 1u))
                                atomicOr(args.status, kErrTimeoutDrain);
                        }
                    }
                    if (wuse > 0 && !mbar_wait(wfull, (wuse - 1) & 1u))
                        atomicOr(args.status, kErrTimeoutDrain);
                }
            } else {
                // the even CTA's releases of every slot and W this CTA filled have arrived
                for (int st = 0; st < STAGES; ++st) {
                    if (issued > static_cast<uint32_t>(st)) {
                        const uint32_t count = (issued - st + STAGES - 1) / STAGES;
                        if (!mbar_wait(empty0 + 8 * st, (count - 1) & 1u))
                            atomicOr(args.status, kErrTimeoutDrain);
                    }
                }
                if (wuse > 0 && !mbar_wait(wempty, (wuse - 1) & 1u))
                    atomicOr(args.status, kErrTimeoutDrain);
            }
        }
    } else if (warp == 1) {
        // ----------------------------------------- MMA issuer, even CTA only
        if (lane == 0 && leader) {
            constexpr uint32_t kIdesc = idesc_f32acc_bmn(256, 2 * IBN, 0);
            int stage = 0;
            uint32_t phase = 0, wuse = 0;
            int ev = 0;
            bool ok = true;
            int b, mt, sub;
            for (int i = 0; ok && unit(i, b, mt, sub); ++i) {
                if (sub == 0) {
                    if (!mbar_wait(wfull, wuse & 1u) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                }
                for (int nt = 0; nt < args.n_tiles && ok; ++nt, ++ev) {
                    const int acc = ev & 1;
                    if (!mbar_wait(tempty0 + 8 * acc, ((ev >> 1) & 1u) ^ 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem_base + acc * C::ACC_COLS;
                    for (int kb = 0; kb < args.num_kb; ++kb) {
                        if (!mbar_wait(full0 + 8 * stage, phase) || *abort_flag) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t bx = x0 + stage * C::X_STAGE;
                        const int ksteps = min(BKS / 16, (args.K - kb * BKS + 15) / 16);
                        for (int j = 0; j < ksteps; ++j) {
                            const int kg = kb * BKS + 16 * j;       // K of this step
                            const uint64_t ad =
                                sdesc_kmajor_sw128(w0 + (kg >> 6) * C::W_BLOCK + 32 * ((kg >> 4) & 3));
                            const uint64_t bd = sdesc_mnmajor_sw128(bx + 2048 * j, C::B_CHUNK, 1024);
                            mma_f16_pair(d, ad, bd, kIdesc, (kb > 0 || j > 0) ? 1u : 0u);
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
                if (!ok) break;
                if (sub == args.group - 1) {
                    mma_commit_pair(wempty, kBoth);    // the super-unit's W may be replaced
                    ++wuse;
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
        // ---------------------------------------------------------- epilogue
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const uint32_t lane_off = static_cast<uint32_t>(quarter * 32 + half * 16) << 16;
        const uint32_t stage_buf = staging0 + (warp - 2) * C::NBUF * C::STAGE_BUF;
        int ev = 0;
        int nstore = 0;
        bool ok = true;
        int b, mt, sub;
        for (int i = 0; ok && unit(i, b, mt, sub); ++i) {
            const int beam0 = mt * 128 + 64 * rank + 16 * quarter + 8 * half;
            for (int nt = 0; nt < args.n_tiles; ++nt, ++ev) {
                const int acc = ev & 1;
                if (!mbar_wait(tfull0 + 8 * acc, (ev >> 1) & 1u) || *abort_flag) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tP = tmem_base + lane_off + acc * C::ACC_COLS;
                ix_drain<C::ACC_COLS, C::STAGE_BUF, C::NBUF>(tP, lane, stage_buf, nstore, nt,
                                                            args.N,
                                                   beam0, b, &tmY, args.y4d);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(tempty0_lead + 8 * acc);
            }
        }
        if (lane == 0) bulk_wait<0>();
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

template <int STAGES, int BKS, int NBUF, int MAXK>
cudaError_t launch_ix_wres(const tcbf_plan_s &pl, const void *Wp, const void *X, float *Y,
                           cudaStream_t s) {
    using C = CfgIxW<STAGES, BKS, NBUF, MAXK>;
    const tcbf_problem &p = pl.p;
    if (p.N % 4 != 0 || pl.m_prefix || p.K > C::MAX_K) return cudaErrorInvalidValue;
    CUtensorMap tmW, tmX, tmY;
    const int w5d = p.M % 8 == 0 ? 1 : 0;
    const int x4d = p.N % 32 == 0 ? 1 : 0;
    const uint64_t wrow = static_cast<uint64_t>(pl.Kp * 2);
    const uint64_t wplane = static_cast<uint64_t>(w_plane_rows(pl)) * wrow;
    if (w5d) {
        const uint64_t dims[5] = {static_cast<uint64_t>(pl.Kp), 8, 2, static_cast<uint64_t>(p.M / 8),
                                  static_cast<uint64_t>(p.w_batches)};
        const uint64_t strides[4] = {wrow, wplane, 8 * wrow, 2 * wplane};
        const uint32_t box[5] = {64, 8, 2, 8, 1};
        if (encode_tiled(&tmW, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 5, const_cast<void *>(Wp), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    } else {
        const uint64_t dims[3] = {static_cast<uint64_t>(pl.Kp), static_cast<uint64_t>(p.M),
                                  static_cast<uint64_t>(2 * p.w_batches)};
        const uint64_t strides[2] = {wrow, wplane};
        const uint32_t box[3] = {64, 8, 2};
        if (encode_tiled(&tmW, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void *>(Wp), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const uint64_t xrow = static_cast<uint64_t>(p.N * 4);
    if (x4d) {
        const uint64_t dims[4] = {64, static_cast<uint64_t>(p.K), static_cast<uint64_t>(2 * p.N / 64),
                                  static_cast<uint64_t>(p.batch)};
        const uint64_t strides[3] = {xrow, 128, static_cast<uint64_t>(p.K) * xrow};
        const uint32_t box[4] = {64, BKS, 2, 1};
        if (encode_tiled(&tmX, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, const_cast<void *>(X), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    } else {
        const uint64_t dims[3] = {static_cast<uint64_t>(2 * p.N), static_cast<uint64_t>(p.K),
                                  static_cast<uint64_t>(p.batch)};
        const uint64_t strides[2] = {xrow, static_cast<uint64_t>(p.K) * xrow};
        const uint32_t box[3] = {64, BKS, 1};
        if (encode_tiled(&tmX, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void *>(X), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const int y4d = p.N % 16 == 0 ? 1 : 0;
    if (encode_ix_y(&tmY, Y, p, y4d) != CUDA_SUCCESS) return cudaErrorInvalidValue;
    IxWArgs a;
    a.status = pl.status;
    a.M = static_cast<int>(p.M);
    a.N = static_cast<int>(p.N);
    a.K = static_cast<int>(p.K);
    a.per_w = static_cast<int>(pl.per_w);
    a.kb64 = static_cast<int>(ceil_div(p.K, 64));
    a.m_tiles = static_cast<int>(ceil_div(p.M, 128));
    a.n_tiles = static_cast<int>(ceil_div(p.N, IBN));
    a.num_kb = static_cast<int>(ceil_div(p.K, BKS));
    a.w5d = w5d;
    a.x4d = x4d;
    a.y4d = y4d;
    // products sharing a weight batch run back to back on one resident W
    // unless the coarser super-units would fill the last wave of pairs
    // worse (small batches)
    const int64_t pairs = std::max(1, pl.num_sms / 2);
    auto fill = [&](int64_t n) {
        return static_cast<double>(n) / static_cast<double>(ceil_div(n, pairs) * pairs);
    };
    const int64_t per_unit = int64_t(a.m_tiles) * p.batch;
    if (per_unit > 0x7fffffff) return cudaErrorInvalidValue;
    a.group = (pl.per_w > 1 && fill(per_unit / pl.per_w) >= fill(per_unit) - 0.01)
                  ? static_cast<int>(pl.per_w)
                  : 1;
    const int64_t units = per_unit / a.group;
    a.total_su = static_cast<int>(units);
    const int smem = C::smem_bytes(a.kb64);
    auto kern = cgemm_ix_wres_kernel<STAGES, BKS, NBUF, MAXK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::smem_bytes(C::MAX_K / 64));
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kIxThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // resident pairs per device at the largest shared-memory size, measured once
    static std::atomic<int> max_clusters[64];
    int mc = max_clusters[pl.device & 63].load(std::memory_order_relaxed);
    if (mc == 0) {
        cudaLaunchConfig_t q = cfg;
        q.dynamicSmemBytes = C::smem_bytes(C::MAX_K / 64);
        q.gridDim = dim3(pl.num_sms / 2 * 2);
        e = cudaOccupancyMaxActiveClusters(&mc, kern, &q);
        if (e != cudaSuccess) return e;
        if (mc < 1) return cudaErrorInvalidConfiguration;
        max_clusters[pl.device & 63].store(mc, std::memory_order_relaxed);
    }
    cfg.gridDim = dim3(static_cast<unsigned>(std::min<int64_t>(units, mc)) * 2);
    e = cudaLaunchKernelEx(&cfg, kern, tmW, tmX, tmY, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

struct IxConfig {
    const char *name;
    cudaError_t (*fn)(const tcbf_plan_s &, const void *, const void *, float *, cudaStream_t);
    int max_k;   // largest K the configuration takes (0: any)
};

const IxConfig kIxConfigs[] = {
    {"f16 interleaved-X MN-major B N256 2-SM pair BM128 BN128 resident-W (K<=320) BK128 stages4 "
     "tmem-double",
     launch_ix_wres<4, 128, 1, 320>, 320},
    {"f16 interleaved-X MN-major B N256 2-SM pair BM128 BN128 BK128 stages3 tmem-double",
     launch_ix<true, 128, 3>, 0},
    {"f16 interleaved-X MN-major B N256 2-SM pair BM128 BN128 BK64 stages6 tmem-double",
     launch_ix<true, 64, 6>, 0},
    {"f16 interleaved-X MN-major B N256 BM64 BN128 BK64 stages4 tmem-double",
     launch_ix<false, 64, 4>, 0},
    {"f16 interleaved-X MN-major B N256 2-SM pair BM128 BN128 resident-W (K<=384) BK128 stages3 "
     "tmem-double",
     launch_ix_wres<3, 128, 2, 384>, 384},
    {"f16 interleaved-X MN-major B N256 2-SM pair BM128 BN128 resident-W (K<=320) BK96 stages5 "
     "tmem-double",
     launch_ix_wres<5, 96, 1, 320>, 320},
    {"f16 interleaved-X MN-major B N256 2-SM pair BM128 BN128 resident-W (K<=320) BK64 stages8 "
     "tmem-double",
     launch_ix_wres<8, 64, 1, 320>, 320},
};

}  // namespace

int gemm_f16_ix_num_configs() { return static_cast<int>(sizeof(kIxConfigs) / sizeof(kIxConfigs[0])); }

bool gemm_f16_ix_config_valid(int config, int64_t K) {
    if (config < 0 || config >= gemm_f16_ix_num_configs()) return false;
    return kIxConfigs[config].max_k == 0 || K <= kIxConfigs[config].max_k;
}

// Resident W when it fits, then streamed W.  Up to K = 320 the ring of the
// two resident forms that keeps more K rows of X in flight (stages x the
// mean K of a stage over one tile): 96-K stages for K = 288 (three full
// stages per tile) or below 97, 128-K ones for K = 256 or 320.
int gemm_f16_ix_default_config(int64_t K) {
    if (K <= 320) {
        const double rows128 = 4.0 * static_cast<double>(K) / static_cast<double>(ceil_div(K, 128));
        const double rows96 = 5.0 * static_cast<double>(K) / static_cast<double>(ceil_div(K, 96));
        return rows96 > rows128 ? 5 : 0;
    }
    return K <= 384 ? 4 : 1;
}

const char *gemm_f16_ix_config_name(int config) {
    if (config < 0 || config >= gemm_f16_ix_num_configs()) return "invalid";
    return kIxConfigs[config].name;
}

cudaError_t launch_gemm_f16_ix(const tcbf_plan_s &pl, const void *Wp, const void *X, float *Y,
                               cudaStream_t s) {
    const int c = (pl.config >= 0 && pl.config < gemm_f16_ix_num_configs()) ? pl.config : 0;
    return kIxConfigs[c].fn(pl, Wp, X, Y, s);
}

}  // namespace tcbf
