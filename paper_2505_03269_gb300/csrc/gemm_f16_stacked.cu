// gemm_f16_stacked.cu — FP16 complex GEMM with stacked sample planes.
//
// The complex product of Sec. III-B needs four real products per K step.
// The one-SM kernel in gemm_f16.cu issues them as four N = 128 MMAs into
// separate Re and Im accumulators; at N = 128 a new A and B tile enter the
// tensor core for every 64-clock MMA, which holds it near 64% of its peak.
// Here the packed samples carry a third, negated plane, [-Xi, Xr, Xi], and
// the B operand of each MMA is two of those planes stacked along N (256
// rows: 128 samples twice):
//     Wr [Xr ; Xi]  +  Wi [-Xi ; Xr]  =  [ Wr Xr - Wi Xi | Wr Xi + Wi Xr ]
//                                      =  [ Re | Im ]
// so one K step is two N = 256 MMAs into one 256-column accumulator
// (Re in columns 0-127, Im in 128-255), each output element still summed
// in the same order (Wr Xr then -Wi Xi; Wr Xi then Wi Xr).  This suits
// compute-bound shapes (the ultrasound block: 65536 voxels x 16384 receiver
// frequency bins x 256 frames); it costs a third X plane in memory and in
// every stage.  K is staged in 32-element blocks with 64-byte swizzle (one
// stage: both W planes 16 KB + three X planes 24 KB) so that five stages
// fit beside the output staging.  Long K is accumulated in promoted chunks
// as in the planar kernels (Sec. III-B's FP32 accumulation): the chunks
// alternate between the accumulators in TMEM columns 0-255 and 256-511, the
// running sum moving into each new chunk's accumulator.
// The default configuration runs the same product on SM pairs (M = 256,
// cta_group::2), see cgemm_stacked_pair_kernel.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>

#include "ptx.cuh"
#include "tiles.cuh"
#include "tcbf_internal.h"

namespace tcbf {
namespace {

using namespace dev;

constexpr int SBM = 128;                // beams per tile (TMEM lanes)
constexpr int SBN = 128;                // samples per tile
constexpr int SBK = 32;                 // K per stage: one 64-byte row
constexpr int kStkThreads = 192;
constexpr int kStkPromoteK = 4096;      // K above this is accumulated in promoted chunks
constexpr int kStkChunkBlocks = 64;     // stages (x 32 K) per promoted chunk

template <int STAGES>
struct CfgStk {
    static constexpr int W_PLANE = SBM * SBK * 2;            // 8 KB
    static constexpr int X_PLANE = SBN * SBK * 2;            // 8 KB
    static constexpr int W_BYTES = 2 * W_PLANE;
    static constexpr int X_BYTES = 3 * X_PLANE;
    static constexpr int STAGE_BYTES = W_BYTES + X_BYTES;    // 40 KB
    static constexpr int TMEM_COLS = 512;                    // 2 x [Re 128 | Im 128]
    static constexpr int STAGING_BYTES = 4 * 4096;           // one 32 x 128 B buffer per epilogue warp
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + STAGING_BYTES + 256 + 1024;
    static_assert(SMEM_BYTES <= 232448, "shared memory");
};

struct StkArgs {
    float *Y;
    uint32_t *status;
    int tma_store;
    int M, N, K;
    int per_w;
    TileMap tiles;
    int num_kb;            // 32-element K blocks
    int kc_blocks;         // blocks per accumulation chunk
    int chunks;
    int total_tiles;
    // SM-pair tiles from split_first on (the last, partial wave) run as
    // split_parts units of whole accumulation chunks each (split_first =
    // total_tiles: no split); total_units counts whole tiles and parts
    int split_first;
    int split_parts;
    int total_units;
};

template <int STAGES, int CL>
__global__ void __launch_bounds__(kStkThreads, 1)
    cgemm_stacked_kernel(const __grid_constant__ CUtensorMap tmW,
                         const __grid_constant__ CUtensorMap tmX,
                         const __grid_constant__ CUtensorMap tmY, const StkArgs args) {
    using C = CfgStk<STAGES>;
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

    // Clusters of CL CTAs along M share each X block: every CTA loads a 1/CL
    // slice of the samples (all three planes) and multicasts it to all, and
    // every CTA's MMA completion is committed to all CTAs' empty barriers
    // (count CL).  The cluster walks (batch, CL m-tiles, n-tile) in lockstep.
    const int rank = CL > 1 ? static_cast<int>(cluster_ctarank()) : 0;
    const int t_first = CL > 1 ? static_cast<int>(cluster_id_x()) : static_cast<int>(blockIdx.x);
    const int t_step = CL > 1 ? static_cast<int>(nclusters_x()) : static_cast<int>(gridDim.x);
    constexpr uint16_t kMask = static_cast<uint16_t>((1u << CL) - 1u);
    auto decode = [&](int t, int &b, int &mt, int &nt) {
        if (CL == 1) {
            tile_decode(args.tiles, t, b, mt, nt);
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
                    mbar_arrive_expect_tx(fb, C::STAGE_BYTES);
                    tma_load_3d(dst, &tmW, fb, kb * SBK, mt * SBM, 2 * bw);
                    if (CL == 1) {
                        tma_load_3d(dst + C::W_BYTES, &tmX, fb, kb * SBK, nt * SBN, 3 * b);
                    } else {
                        constexpr int kRows = SBN / CL;
#pragma unroll
                        for (int pl = 0; pl < 3; ++pl)
                            tma_load_3d_mc(dst + C::W_BYTES + pl * C::X_PLANE + rank * kRows * 64,
                                           &tmX, fb, kb * SBK, nt * SBN + rank * kRows, 3 * b + pl,
                                           kMask);
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
            constexpr uint32_t kIdesc = idesc_f32acc(SBM, 2 * SBN, 0, false);
            int stage = 0;
            uint32_t phase = 0;
            int ev = 0;                                  // accumulator hand-offs so far
            bool ok = true;
            for (int t = t_first; t < args.total_tiles && ok; t += t_step) {
                for (int ch = 0; ch < args.chunks; ++ch, ++ev) {
                    const int acc = ev & 1;
                    const uint32_t aphase = (ev >> 1) & 1;
                    if (!mbar_wait(tempty0 + 8 * acc, aphase ^ 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem_base + acc * 2 * SBN;
                    const int kb0 = ch * args.kc_blocks;
                    const int kb1 = min(args.num_kb, kb0 + args.kc_blocks);
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!mbar_wait(full0 + 8 * stage, phase) || *abort_flag) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a = s0 + stage * C::STAGE_BYTES;   // Wr, Wi
                        const uint32_t x = a + C::W_BYTES;                 // -Xi, Xr, Xi
                        const int ksteps = min(SBK / 16, (args.K - kb * SBK + 15) / 16);
                        for (int j = 0; j < ksteps; ++j) {
                            const uint32_t accum = (kb > kb0 || j > 0) ? 1u : 0u;
                            // Wr [Xr; Xi] -> [Wr Xr | Wr Xi]
                            mma_f16(d, sdesc_kmajor_sw64(a + 32 * j),
                                    sdesc_kmajor_sw64(x + C::X_PLANE + 32 * j), kIdesc, accum);
                            // Wi [-Xi; Xr] -> [-Wi Xi | Wi Xr]
                            mma_f16(d, sdesc_kmajor_sw64(a + C::W_PLANE + 32 * j),
                                    sdesc_kmajor_sw64(x + 32 * j), kIdesc, 1u);
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
        // As in the one-SM kernel: each warp owns 32 accumulator rows; per
        // 16-column chunk it loads Re and Im, interleaves them into complex64
        // and stages the 32 x 128-byte block (128-byte swizzle) for one TMA
        // store, or (odd N) stores its row directly.
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t stage_buf = staging0 + (warp - 2) * 4096;
        const bool vec_ok = (args.N & 1) == 0;
        int ev = 0;
        const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
        bool ok = true;
        for (int t = t_first; t < args.total_tiles && ok; t += t_step) {
            int b, mt, nt;
            decode(t, b, mt, nt);
            const int m = mt * SBM + row;
            float *yrow = args.Y + (static_cast<size_t>(b) * args.M + m) * args.N * 2;
            for (int ch = 0; ch < args.chunks; ++ch, ++ev) {
                const int acc = ev & 1;
                const uint32_t aphase = (ev >> 1) & 1;
                if (!mbar_wait(tfull0 + 8 * acc, aphase) || *abort_flag) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tP = tmem_base + lane_off + acc * 2 * SBN;
                if (ch > 0) {
                    // promote: the running sum S (the previous chunk's accumulator)
                    // plus this chunk's P, FP32 round-to-nearest, into this
                    // accumulator; then S's accumulator is free for the next chunk
                    const uint32_t tS = tmem_base + lane_off + (acc ^ 1) * 2 * SBN;
#pragma unroll 1
                    for (int g = 0; g < SBN / 16; ++g) {
                        float pr[16], pi[16], sr[16], si[16];
                        tmem_ld_2x16(tP + g * 16, tP + SBN + g * 16, pr, pi);
                        tmem_ld_2x16(tS + g * 16, tS + SBN + g * 16, sr, si);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            pr[i] = __fadd_rn(sr[i], pr[i]);
                            pi[i] = __fadd_rn(si[i], pi[i]);
                        }
                        tmem_st_2x16(tP + g * 16, tP + SBN + g * 16, pr, pi);
                    }
                    tmem_st_wait();
                    tc_fence_before();
                    mbar_arrive(tempty0 + 8 * (acc ^ 1));
                }
                // a chunk before the last keeps its sum in its accumulator
                if (ch + 1 < args.chunks) continue;
#pragma unroll 1
                for (int c = 0; c < SBN / 16; ++c) {
                    float re[16], im[16];
                    tmem_ld_2x16(tP + c * 16, tP + SBN + c * 16, re, im);
                    const int n0 = nt * SBN + c * 16;
                    if (args.tma_store) {
                        if (n0 < args.N) {
                            if (lane == 0) bulk_wait_read<0>();   // the buffer's last store has read it
                            __syncwarp();
                            const uint32_t rbase = stage_buf + lane * 128;
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                st_shared_v4(rbase + ((j ^ (lane & 7)) << 4), re[2 * j], im[2 * j],
                                             re[2 * j + 1], im[2 * j + 1]);
                            fence_async_smem();
                            __syncwarp();
                            if (lane == 0) {
                                tma_store_3d(&tmY, stage_buf, 2 * n0, mt * SBM + quarter * 32, b);
                                bulk_commit();
                            }
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

template <int STAGES, int CL>
cudaError_t launch_stacked(const tcbf_plan_s &pl, const void *Wp, const void *Xp, float *Y,
                           cudaStream_t s, int raster) {
    if (CL > 1 && pl.m_prefix)   // uneven batches walk per-batch m-tiles: no clusters
        return launch_stacked<STAGES, 1>(pl, Wp, Xp, Y, s, raster);
    using C = CfgStk<STAGES>;
    const tcbf_problem &p = pl.p;
    const int64_t row = pl.Kp;
    CUtensorMap tmW, tmX, tmY;
    {
        const uint64_t dims[3] = {static_cast<uint64_t>(row), static_cast<uint64_t>(p.M),
                                  static_cast<uint64_t>(2 * p.w_batches)};
        const uint64_t strides[2] = {static_cast<uint64_t>(row * 2),
                                     static_cast<uint64_t>(w_plane_rows(pl) * row * 2)};
        const uint32_t box[3] = {SBK, SBM, 2};
        if (encode_tiled(&tmW, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void *>(Wp), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_64B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const uint64_t dims[3] = {static_cast<uint64_t>(row), static_cast<uint64_t>(p.N),
                                  static_cast<uint64_t>(3 * p.batch)};
        const uint64_t strides[2] = {static_cast<uint64_t>(row * 2),
                                     static_cast<uint64_t>(p.N * row * 2)};
        // clusters: each CTA loads a SBN/CL-row slice of one plane per multicast
        const uint32_t box[3] = {SBK, static_cast<uint32_t>(SBN / CL), CL == 1 ? 3u : 1u};
        if (encode_tiled(&tmX, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void *>(Xp), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_64B) != CUDA_SUCCESS)
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
    StkArgs a;
    a.Y = Y;
    a.status = pl.status;
    a.tma_store = tma_store;
    a.M = static_cast<int>(p.M);
    a.N = static_cast<int>(p.N);
    a.K = static_cast<int>(p.K);
    a.per_w = static_cast<int>(pl.per_w);
    a.tiles.prefix = pl.m_prefix;
    a.tiles.batch = static_cast<int>(p.batch);
    a.tiles.m_tiles = static_cast<int>(ceil_div(p.M, SBM));
    a.tiles.n_tiles = static_cast<int>(ceil_div(p.N, SBN));
    a.tiles.raster = raster;
    a.num_kb = static_cast<int>(ceil_div(p.K, SBK));
    a.kc_blocks = p.K > kStkPromoteK ? kStkChunkBlocks : a.num_kb;
    a.chunks = (a.num_kb + a.kc_blocks - 1) / a.kc_blocks;
    const int64_t m_units = CL == 1 ? (pl.m_prefix ? pl.m_tiles_sum : int64_t(a.tiles.m_tiles) * p.batch)
                                    : ceil_div(a.tiles.m_tiles, CL) * p.batch;
    const int64_t total = m_units * a.tiles.n_tiles;     // tiles, or cluster tiles
    if (total > 0x7fffffff) return cudaErrorInvalidValue;
    a.total_tiles = static_cast<int>(total);
    a.split_first = a.total_tiles;                       // one-SM tiles run whole
    a.split_parts = 1;
    a.total_units = a.total_tiles;
    auto kern = cgemm_stacked_kernel<STAGES, CL>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (CL == 1) {
        const int grid = static_cast<int>(std::min<int64_t>(total, pl.num_sms));
        kern<<<grid, kStkThreads, C::SMEM_BYTES, s>>>(tmW, tmX, tmY, a);
        return cudaGetLastError();
    }
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kStkThreads);
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

// ===========================================================================
// Two-SM stacked tiles (cta_group::2): a cluster of two CTAs computes a
// 256-row x 128-sample tile with M = 256, N = 256 MMAs issued by the even
// CTA.  Each B operand is split across the pair by rows (samples): of
// B1 = [Xr; Xi] the even CTA holds Xr and the odd one Xi, of B2 = [-Xi; Xr]
// the even CTA holds -Xi and the odd one Xr, each at the same shared-memory
// offset, so every CTA loads two of the three packed planes and each SM's
// tensor core takes 128 rows of W and 128 of X per MMA, a third less than a
// one-SM N = 256 tile.  Stages hold 64 K in 128-byte swizzled rows.  Both
// CTAs' loads complete on the even CTA's full barrier, its MMA completions
// are committed to both CTAs, and both CTAs' epilogues release an
// accumulator on the even CTA's barrier.  Promotion as in the one-SM kernel.
// With promoted long K, the tiles of a partial last wave can run as parts of
// whole chunks on the pairs that wave leaves idle (pair_split); a part stores
// its chunks to Y or to the plan's workspace, and stacked_tail_fixup_kernel
// adds them in chunk order after the launch.
// ===========================================================================
constexpr int PBK = 64;                  // K per stage: one 128-byte row
constexpr int kStkPairChunkBlocks = 32;  // stages (x 64 K) per promoted chunk
constexpr int kStkPairStages = 3;
// Pair tiles run in groups of kPairGroupM pair rows, samples fastest within
// a group: the clusters running at one time then share their W rows and
// their X columns in L2.  With samples fastest over all rows, a product
// whose X does not fit in L2 streams all of X once per pair row.
constexpr int kPairGroupM = 8;

template <int STAGES>
struct CfgStkPair {
    static constexpr int PLANE = 128 * PBK * 2;               // 16 KB: 128 rows x 128 B
    static constexpr int W_BYTES = 2 * PLANE;                 // Wr, Wi (this CTA's 128 rows)
    static constexpr int STAGE_BYTES = W_BYTES + 2 * PLANE;   // + the CTA's halves of B1, B2
    static constexpr int TMEM_COLS = 512;                     // 2 x [Re 128 | Im 128]
    static constexpr int STAGING_BYTES = 4 * 4096;
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + STAGING_BYTES + 256 + 1024;
    static_assert(SMEM_BYTES <= 232448, "shared memory");
};

// (batch, 256-row pair tile, sample tile) of pair tile t: groups of
// kPairGroupM pair rows (the last one possibly shorter), pair rows fastest
// inside a group, then sample tiles
__host__ __device__ __forceinline__ void pair_decode(const StkArgs &a, int t, int &b, int &mp,
                                                     int &nt) {
    const int m_pairs = (a.tiles.m_tiles + 1) / 2;
    const int per_b = m_pairs * a.tiles.n_tiles;
    b = t / per_b;
    const int local = t - b * per_b;
    const int group = local / (kPairGroupM * a.tiles.n_tiles);
    const int first = group * kPairGroupM;
    const int gm = min(kPairGroupM, m_pairs - first);
    const int in = local - group * kPairGroupM * a.tiles.n_tiles;
    mp = first + in % gm;
    nt = in / gm;
}

// Unit u of the SM-pair kernel: whole tile u, or, from split_first on, part
// j of a tail tile, its chunks [c0, c1).  Returns whether it is a part.
__device__ __forceinline__ bool pair_unit(const StkArgs &a, int u, int &t, int &c0, int &c1) {
    if (u < a.split_first) {
        t = u;
        c0 = 0;
        c1 = a.chunks;
        return false;
    }
    const int v = u - a.split_first;
    const int j = v % a.split_parts;
    t = a.split_first + v / a.split_parts;
    c0 = j * a.chunks / a.split_parts;
    c1 = (j + 1) * a.chunks / a.split_parts;
    return true;
}

template <int STAGES>
__global__ void __launch_bounds__(kStkThreads, 1)
    cgemm_stacked_pair_kernel(const __grid_constant__ CUtensorMap tmW,
                              const __grid_constant__ CUtensorMap tmX,
                              const __grid_constant__ CUtensorMap tmY,
                              const __grid_constant__ CUtensorMap tmS, const StkArgs args) {
    using C = CfgStkPair<STAGES>;
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
        if (args.split_first < args.total_tiles) tma_prefetch_desc(&tmS);
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
            for (int u = t_first; u < args.total_units && ok; u += t_step) {
                int t, c0, c1, b, mp, nt;
                pair_unit(args, u, t, c0, c1);
                pair_decode(args, t, b, mp, nt);
                const int bw = b / args.per_w;
                const int kb_end = min(args.num_kb, c1 * args.kc_blocks);
                for (int kb = c0 * args.kc_blocks; kb < kb_end; ++kb) {
                    if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = full0_lead + 8 * stage;
                    if (leader) mbar_arrive_expect_tx(full0 + 8 * stage, 2 * C::STAGE_BYTES);
                    const uint32_t dst = s0 + stage * C::STAGE_BYTES;
                    const int x = kb * PBK;
                    tma_load_3d_pair(dst, &tmW, fb, x, mp * 256 + 128 * rank, 2 * bw);
                    tma_load_3d_pair(dst + C::W_BYTES, &tmX, fb, x, nt * SBN, 3 * b + plane_b1);
                    tma_load_3d_pair(dst + C::W_BYTES + C::PLANE, &tmX, fb, x, nt * SBN,
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
            constexpr uint32_t kIdesc = idesc_f32acc(256, 2 * SBN, 0, false);
            int stage = 0;
            uint32_t phase = 0;
            int ev = 0;
            bool ok = true;
            for (int u = t_first; u < args.total_units && ok; u += t_step) {
                int t, c0, c1;
                pair_unit(args, u, t, c0, c1);
                for (int ch = c0; ch < c1; ++ch, ++ev) {
                    const int acc = ev & 1;
                    const uint32_t aphase = (ev >> 1) & 1;
                    if (!mbar_wait(tempty0 + 8 * acc, aphase ^ 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem_base + acc * 2 * SBN;
                    const int kb0 = ch * args.kc_blocks;
                    const int kb1 = min(args.num_kb, kb0 + args.kc_blocks);
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!mbar_wait(full0 + 8 * stage, phase) || *abort_flag) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a = s0 + stage * C::STAGE_BYTES;   // Wr, Wi
                        const uint32_t x = a + C::W_BYTES;                 // B1 half, B2 half
                        const int ksteps = min(PBK / 16, (args.K - kb * PBK + 15) / 16);
                        for (int j = 0; j < ksteps; ++j) {
                            const uint32_t accum = (kb > kb0 || j > 0) ? 1u : 0u;
                            // Wr [Xr; Xi] -> [Wr Xr | Wr Xi]
                            mma_f16_pair(d, sdesc_kmajor_sw128(a + 32 * j),
                                         sdesc_kmajor_sw128(x + 32 * j), kIdesc, accum);
                            // Wi [-Xi; Xr] -> [-Wi Xi | Wi Xr]
                            mma_f16_pair(d, sdesc_kmajor_sw128(a + C::PLANE + 32 * j),
                                         sdesc_kmajor_sw128(x + C::PLANE + 32 * j), kIdesc, 1u);
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
        const uint32_t stage_buf = staging0 + (warp - 2) * 4096;
        const bool vec_ok = (args.N & 1) == 0;
        int ev = 0;
        const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
        bool ok = true;
        for (int u = t_first; u < args.total_units && ok; u += t_step) {
            int t, c0, c1, b, mp, nt;
            const bool part = pair_unit(args, u, t, c0, c1);
            pair_decode(args, t, b, mp, nt);
            const int mrow0 = mp * 256 + 128 * rank;           // this CTA's first row
            const int m = mrow0 + row;
            float *yrow = args.Y + (static_cast<size_t>(b) * args.M + m) * args.N * 2;
            for (int ch = c0; ch < c1; ++ch, ++ev) {
                const int acc = ev & 1;
                const uint32_t aphase = (ev >> 1) & 1;
                if (!mbar_wait(tfull0 + 8 * acc, aphase) || *abort_flag) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tP = tmem_base + lane_off + acc * 2 * SBN;
                if (!part && ch > 0) {
                    // promote: the running sum S (the previous chunk's accumulator)
                    // plus this chunk's P, FP32 round-to-nearest, into this
                    // accumulator; then S's accumulator is free for the next chunk
                    const uint32_t tS = tmem_base + lane_off + (acc ^ 1) * 2 * SBN;
#pragma unroll 1
                    for (int g = 0; g < SBN / 16; ++g) {
                        float pr[16], pi[16], sr[16], si[16];
                        tmem_ld_2x16(tP + g * 16, tP + SBN + g * 16, pr, pi);
                        tmem_ld_2x16(tS + g * 16, tS + SBN + g * 16, sr, si);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            pr[i] = __fadd_rn(sr[i], pr[i]);
                            pi[i] = __fadd_rn(si[i], pi[i]);
                        }
                        tmem_st_2x16(tP + g * 16, tP + SBN + g * 16, pr, pi);
                    }
                    tmem_st_wait();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive_remote(tempty0_lead + 8 * (acc ^ 1));
                }
                // a chunk before the last keeps its sum in its accumulator
                if (!part && ch + 1 < c1) continue;
                // a part stores each of its chunks: a tail tile's first chunk to
                // Y, the later ones to its workspace slots (a second kernel adds them)
                const bool to_ws = part && ch > 0;
                const int slot = (t - args.split_first) * (args.chunks - 1) + ch - 1;
#pragma unroll 1
                for (int c = 0; c < SBN / 16; ++c) {
                    float re[16], im[16];
                    tmem_ld_2x16(tP + c * 16, tP + SBN + c * 16, re, im);
                    const int n0 = nt * SBN + c * 16;
                    if (args.tma_store) {
                        if (n0 < args.N) {
                            if (lane == 0) bulk_wait_read<0>();
                            __syncwarp();
                            const uint32_t rbase = stage_buf + lane * 128;
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                st_shared_v4(rbase + ((j ^ (lane & 7)) << 4), re[2 * j], im[2 * j],
                                             re[2 * j + 1], im[2 * j + 1]);
                            fence_async_smem();
                            __syncwarp();
                            if (lane == 0) {
                                if (to_ws)
                                    tma_store_3d(&tmS, stage_buf, 32 * c, 128 * rank + quarter * 32, slot);
                                else
                                    tma_store_3d(&tmY, stage_buf, 2 * n0, mrow0 + quarter * 32, b);
                                bulk_commit();
                            }
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

// After a launch whose last wave was split: Y holds the first chunk of each
// tail tile; its later chunks come from the workspace and are added in chunk
// order with FP32 round-to-nearest, as the unsplit kernel promotes them, so
// the result is the same bit for bit.
__global__ void stacked_tail_fixup_kernel(const StkArgs args, const float2 *__restrict__ ws) {
    constexpr int kPerTile = 256 * SBN;     // (row, sample) pairs of a pair tile
    const int64_t total = int64_t(args.total_tiles - args.split_first) * kPerTile;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int tt = static_cast<int>(i / kPerTile);
        const int e = static_cast<int>(i - int64_t(tt) * kPerTile);
        const int r = e / SBN;
        int b, mp, nt;
        pair_decode(args, args.split_first + tt, b, mp, nt);
        const int m = mp * 256 + r;
        const int n = nt * SBN + (e - r * SBN);
        if (m >= args.M || n >= args.N) continue;
        float2 *y = reinterpret_cast<float2 *>(args.Y) + (static_cast<size_t>(b) * args.M + m) * args.N + n;
        float2 v = *y;
        const float2 *q = ws + static_cast<size_t>(tt) * (args.chunks - 1) * kPerTile + e;
        for (int c = 1; c < args.chunks; ++c, q += kPerTile) {
            const float2 w = __ldg(q);
            v.x = __fadd_rn(v.x, w.x);
            v.y = __fadd_rn(v.y, w.y);
        }
        *y = v;
    }
}

// Pair tiles and accumulation chunks of a plan on the SM-pair kernel.
void pair_shape(const tcbf_plan_s &pl, StkArgs &a) {
    const tcbf_problem &p = pl.p;
    a.tiles.m_tiles = static_cast<int>(ceil_div(p.M, 128));
    a.tiles.n_tiles = static_cast<int>(ceil_div(p.N, SBN));
    a.num_kb = static_cast<int>(ceil_div(p.K, PBK));
    a.kc_blocks = p.K > kStkPromoteK ? kStkPairChunkBlocks : a.num_kb;
    a.chunks = (a.num_kb + a.kc_blocks - 1) / a.kc_blocks;
}

// Resident SM pairs of the pair kernel on the plan's device, measured once
// (benign if two threads both measure).
template <int STAGES>
cudaError_t pair_max_clusters(const tcbf_plan_s &pl, int &mc) {
    static std::atomic<int> cache[64];
    mc = cache[pl.device & 63].load(std::memory_order_relaxed);
    if (mc > 0) return cudaSuccess;
    using C = CfgStkPair<STAGES>;
    auto kern = cgemm_stacked_pair_kernel<STAGES>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl.num_sms / 2 * 2);
    cfg.blockDim = dim3(kStkThreads);
    cfg.dynamicSmemBytes = C::SMEM_BYTES;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaOccupancyMaxActiveClusters(&mc, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (mc < 1) return cudaErrorInvalidConfiguration;
    cache[pl.device & 63].store(mc, std::memory_order_relaxed);
    return cudaSuccess;
}

// The split of the last, partial wave: its r pair tiles run as s units each
// of whole accumulation chunks on the SM pairs the wave leaves idle, s =
// min(chunks, pairs / r) >= 2.  Only for promoted long K (two or more
// chunks) with Y stored by the TMA, and while the workspace for the tail
// tiles' later chunks (r x (chunks - 1) pair tiles of 256 KB) stays within
// kTailWsMaxBytes.
constexpr size_t kTailWsMaxBytes = size_t(64) << 20;
constexpr size_t kTailSlotBytes = size_t(256) * SBN * 8;
void pair_split(StkArgs &a, int pairs) {
    a.split_first = a.total_tiles;
    a.split_parts = 1;
    a.total_units = a.total_tiles;
    if (!a.tma_store || a.chunks < 2 || pairs < 2) return;
    const int r = a.total_tiles % pairs;
    if (r == 0) return;
    const int parts = std::min(a.chunks, pairs / r);
    if (parts < 2 || size_t(r) * (a.chunks - 1) * kTailSlotBytes > kTailWsMaxBytes) return;
    a.split_first = a.total_tiles - r;
    a.split_parts = parts;
    a.total_units = a.split_first + r * parts;
}

size_t pair_split_ws_bytes(const StkArgs &a) {
    return size_t(a.total_tiles - a.split_first) * (a.chunks - 1) * kTailSlotBytes;
}

template <int STAGES>
cudaError_t launch_stacked_pair(const tcbf_plan_s &pl, const void *Wp, const void *Xp, float *Y,
                                cudaStream_t s, int raster) {
    if (pl.m_prefix)   // uneven batches walk per-batch m-tiles: one-SM tiles
        return launch_stacked<5, 1>(pl, Wp, Xp, Y, s, raster);
    using C = CfgStkPair<STAGES>;
    const tcbf_problem &p = pl.p;
    const int64_t row = pl.Kp;
    CUtensorMap tmW, tmX, tmY;
    {
        const uint64_t dims[3] = {static_cast<uint64_t>(row), static_cast<uint64_t>(p.M),
                                  static_cast<uint64_t>(2 * p.w_batches)};
        const uint64_t strides[2] = {static_cast<uint64_t>(row * 2),
                                     static_cast<uint64_t>(w_plane_rows(pl) * row * 2)};
        const uint32_t box[3] = {PBK, 128, 2};
        if (encode_tiled(&tmW, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void *>(Wp), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const uint64_t dims[3] = {static_cast<uint64_t>(row), static_cast<uint64_t>(p.N),
                                  static_cast<uint64_t>(3 * p.batch)};
        const uint64_t strides[2] = {static_cast<uint64_t>(row * 2),
                                     static_cast<uint64_t>(p.N * row * 2)};
        const uint32_t box[3] = {PBK, SBN, 1};              // one plane of 128 samples
        if (encode_tiled(&tmX, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void *>(Xp), dims,
                         strides, box, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
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
    StkArgs a;
    a.Y = Y;
    a.status = pl.status;
    a.tma_store = tma_store;
    a.M = static_cast<int>(p.M);
    a.N = static_cast<int>(p.N);
    a.K = static_cast<int>(p.K);
    a.per_w = static_cast<int>(pl.per_w);
    a.tiles.prefix = nullptr;
    a.tiles.batch = static_cast<int>(p.batch);
    a.tiles.raster = 0;
    pair_shape(pl, a);
    const int64_t total = ceil_div(a.tiles.m_tiles, 2) * p.batch * a.tiles.n_tiles;   // pair tiles
    if (total > 0x7fffffff / 8) return cudaErrorInvalidValue;
    a.total_tiles = static_cast<int>(total);
    int mc = 0;
    cudaError_t e = pair_max_clusters<STAGES>(pl, mc);
    if (e != cudaSuccess) return e;
    pair_split(a, mc);
    // the split needs the plan's workspace (made with the plan); without it,
    // or with a smaller one, the tiles run whole (the same results)
    CUtensorMap tmS = tmX;
    const bool split = a.split_first < a.total_tiles;
    if (split && (!pl.tail_ws || pl.tail_ws_bytes < pair_split_ws_bytes(a))) pair_split(a, 0);
    if (a.split_first < a.total_tiles) {
        const uint64_t dims[3] = {uint64_t(2 * SBN), 256,
                                  uint64_t(pair_split_ws_bytes(a) / kTailSlotBytes)};
        const uint64_t strides[2] = {uint64_t(2 * SBN * 4), uint64_t(kTailSlotBytes)};
        const uint32_t box[3] = {32, 32, 1};
        if (encode_tiled(&tmS, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, pl.tail_ws, dims, strides, box,
                         CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    auto kern = cgemm_stacked_pair_kernel<STAGES>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kStkThreads);
    cfg.dynamicSmemBytes = C::SMEM_BYTES;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(std::min(a.total_units, mc)) * 2);
    e = cudaLaunchKernelEx(&cfg, kern, tmW, tmX, tmY, tmS, a);
    if (e != cudaSuccess) return e;
    if (a.split_first < a.total_tiles) {
        const int64_t n = int64_t(a.total_tiles - a.split_first) * 256 * SBN;
        const int grid = static_cast<int>(std::min<int64_t>(ceil_div(n, 256), int64_t(pl.num_sms) * 8));
        stacked_tail_fixup_kernel<<<grid, 256, 0, s>>>(a, static_cast<const float2 *>(pl.tail_ws));
    }
    return cudaGetLastError();
}

struct StkConfig {
    const char *name;
    int raster;
    cudaError_t (*fn)(const tcbf_plan_s &, const void *, const void *, float *, cudaStream_t, int);
};

const StkConfig kStkConfigs[] = {
    {"f16 stacked-X N256 2-SM pair BM256 BN128 BK64 stages3 tmem-double", 0,
     launch_stacked_pair<kStkPairStages>},
    {"f16 stacked-X N256 BM128 BN128 BK32-sw64 stages5 tmem-double cluster2 X-multicast", 0,
     launch_stacked<5, 2>},
    {"f16 stacked-X N256 BM128 BN128 BK32-sw64 stages5 tmem-double n-fastest", 0, launch_stacked<5, 1>},
    {"f16 stacked-X N256 BM128 BN128 BK32-sw64 stages5 tmem-double cluster4 X-multicast", 0,
     launch_stacked<5, 4>},
    {"f16 stacked-X N256 BM128 BN128 BK32-sw64 stages5 tmem-double m-fastest", 1, launch_stacked<5, 1>},
};

}  // namespace

int gemm_f16_stacked_num_configs() {
    return static_cast<int>(sizeof(kStkConfigs) / sizeof(kStkConfigs[0]));
}

const char *gemm_f16_stacked_config_name(int config) {
    if (config < 0 || config >= gemm_f16_stacked_num_configs()) return "invalid";
    return kStkConfigs[config].name;
}

size_t stacked_tail_ws_bytes(const tcbf_plan_s &pl) {
    if (pl.m_prefix) return 0;
    StkArgs a = {};
    a.tma_store = (pl.p.N % 2 == 0) ? 1 : 0;
    pair_shape(pl, a);
    const int64_t total = ceil_div(a.tiles.m_tiles, 2) * pl.p.batch * a.tiles.n_tiles;
    if (total > 0x7fffffff / 8) return 0;
    a.total_tiles = static_cast<int>(total);
    int mc = 0;
    if (pair_max_clusters<kStkPairStages>(pl, mc) != cudaSuccess) return 0;
    pair_split(a, mc);
    return a.split_first < a.total_tiles ? pair_split_ws_bytes(a) : 0;
}

cudaError_t launch_gemm_f16_stacked(const tcbf_plan_s &pl, const void *Wp, const void *Xp, float *Y,
                                    cudaStream_t s) {
    const int c = (pl.config >= 0 && pl.config < gemm_f16_stacked_num_configs()) ? pl.config : 0;
    return kStkConfigs[c].fn(pl, Wp, Xp, Y, s, kStkConfigs[c].raster);
}

}  // namespace tcbf
