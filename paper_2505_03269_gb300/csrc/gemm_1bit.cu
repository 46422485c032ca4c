// gemm_1bit.cu — exact 1-bit complex GEMM on the sm_103a tensor cores.
//
// Values are +-1 +-i, one bit per component (Fig. 1: bit 1 = +1, bit 0 = -1).
// The paper computes the real dot products K - 2 popc(A xor B) (Eq. 4) with
// b1 tensor-core MMAs, or the AND form (Eq. 6) on Hopper.  On this GPU the
// legacy b1 AND-popc MMA measures 146 TeraOps/s against 4788 for FP8
// tcgen05 MMAs (peak microbenchmarks), and tcgen05 has no integer kind, so
// the bits are expanded on chip to E4M3 +-1.0 (0 for k >= K, so no padding
// correction as in Eq. 5 is needed) and multiplied with kind::f8f6f4 into
// FP32 accumulators.  Every partial sum is an integer of magnitude <= 2K,
// exact in FP32 for K < 2^23, so the result equals K - 2 Hamming exactly.
//
// Warp roles (544 or 672 threads, one CTA per SM, persistent over tiles):
//   warp 0      TMEM owner and single-thread MMA issuer (4 real MMAs per
//               K step, negate-A for -Im(W) Im(X), as in the FP16 kernel)
//   warps 1-12  converters: each thread takes every 384th row-plane of the
//               stage (the W planes' rows, then the X planes' rows), a 16-byte
//               load of its packed words (L2-resident) and its expansion to
//               E4M3 in the 128-byte-swizzled K-major layout the MMA reads,
//               one stage of 128 K per ring slot.  The expansion is latency-
//               bound per thread, so the row-planes are spread evenly (two per
//               thread for 128 x 256 tiles) rather than split by operand.
//   warps 13-   epilogue: TMEM -> int32 pairs -> staged TMA stores; eight
//               warps (two per TMEM lane quarter, one 4 KB staging buffer
//               each) when the accumulator is single-buffered, so that its
//               drain holds up the next tile's MMAs for less time, else four
#include <algorithm>
#include <cstring>

#include "ptx.cuh"
#include "tiles.cuh"
#include "tcbf_internal.h"

namespace tcbf {
namespace {

using namespace dev;

constexpr int BM = 128;
constexpr int BKE = 128;             // K elements per stage (one 128-byte E4M3 row)
constexpr int kConv = 384;           // converter threads

struct Args1 {
    int32_t *Y;
    const uint32_t *Wb;
    const uint32_t *Xb;
    uint32_t *status;
    int tma_store;
    int M, N, K, Kw;
    int w_rows;            // rows between packed W planes (M, or more for a row range)
    int per_w;
    TileMap tiles;
    int num_kb, total_tiles;
};

// STK: stacked sample planes [-Xi, Xr, Xi] (the converters write the first
// with flipped signs) so that Wr [Xr; Xi] + Wi [-Xi; Xr] = [Re | Im] is two
// N = 2 BN MMAs per 32-K step into one 2 BN-column accumulator.
template <int BN, int STAGES, bool STK = false>
struct Cfg1 {
    static constexpr int XPL = STK ? 3 : 2;                   // X planes per stage
    static constexpr int A_PLANE = BM * BKE;
    static constexpr int B_PLANE = BN * BKE;
    static constexpr int A_BYTES = 2 * A_PLANE;
    static constexpr int STAGE_BYTES = A_BYTES + XPL * B_PLANE;
    static constexpr int ACC_BUFS = (4 * BN <= 512) ? 2 : 1;
    static constexpr int TMEM_COLS = ACC_BUFS * 2 * BN <= 256 ? 256 : 512;
    static constexpr int EPI_WARPS = ACC_BUFS == 1 ? 8 : 4;
    static constexpr int THREADS = 32 + kConv + 32 * EPI_WARPS;
    static constexpr int STAGING_BYTES = 4 * 2 * 4096;
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + STAGING_BYTES + 256 + 1024;
    static_assert(SMEM_BYTES <= 232448, "shared memory");
};

__device__ __forceinline__ void decode_tile(int t, const Args1 &a, int &b, int &mt, int &nt) {
    tile_decode(a.tiles, t, b, mt, nt);
}

// 4 sign bits -> 4 E4M3 bytes: bit 1 -> 0x38 (+1.0), bit 0 -> 0xB8 (-1.0);
// NEG gives the negated values.  The multiply places bit j at bit 8j + 7
// (copies at offsets 7, 14, 21, 28 do not overlap for a 4-bit value).
template <bool NEG = false>
__device__ __forceinline__ uint32_t expand4(uint32_t nib) {
    return (NEG ? 0x38383838u : 0xB8B8B8B8u) ^ ((nib * 0x10204080u) & 0x80808080u);
}

// 16 sign bits -> 16 E4M3 bytes; bytes whose element index is >= valid are 0.
template <bool NEG = false>
__device__ __forceinline__ uint4 expand16(uint32_t bits, int valid) {
    uint4 v;
    v.x = expand4<NEG>(bits & 15u);
    v.y = expand4<NEG>((bits >> 4) & 15u);
    v.z = expand4<NEG>((bits >> 8) & 15u);
    v.w = expand4<NEG>((bits >> 12) & 15u);
    if (valid < 16) {
        uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int keep = min(max(valid - 4 * q, 0), 4);   // bytes of this word below K
            const uint32_t mask = keep >= 4 ? 0xFFFFFFFFu : ((1u << (8 * keep)) - 1u);
            w[q] &= mask;
        }
        v = make_uint4(w[0], w[1], w[2], w[3]);
    }
    return v;
}

__device__ __forceinline__ void st_shared_u4(uint32_t addr, uint4 v) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

// Expand one row's 128 K (4 words) of one plane (negated if NEG) into the
// swizzled slot.  Full stages (valid >= 128) take the unmasked path.
template <bool NEG = false>
__device__ __forceinline__ void expand_row(uint32_t row_base, int r, uint4 words, int valid) {
    const uint32_t w[4] = {words.x, words.y, words.z, words.w};
    const uint32_t sw = static_cast<uint32_t>(r & 7);
    if (valid >= BKE) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint32_t bits = w[c >> 1] >> (16 * (c & 1));
            uint4 v;
            v.x = expand4<NEG>(bits & 15u);
            v.y = expand4<NEG>((bits >> 4) & 15u);
            v.z = expand4<NEG>((bits >> 8) & 15u);
            v.w = expand4<NEG>((bits >> 12) & 15u);
            st_shared_u4(row_base + ((c ^ sw) << 4), v);
        }
    } else {
#pragma unroll 1
        for (int c = 0; c < 8; ++c) {
            const uint32_t bits = (w[c >> 1] >> (16 * (c & 1))) & 0xFFFFu;
            st_shared_u4(row_base + ((c ^ sw) << 4), expand16<NEG>(bits, valid - 16 * c));
        }
    }
}

// Row-planes of one stage: 2 x BM of W (Wr rows, then Wi rows) and 2 x BN
// of X; converter thread ct takes ct, ct + kConv, ...  Each holds its packed
// words and the number of valid K elements (0 for rows beyond M or N, which
// are written as zeros).
template <int BN, bool STK = false>
struct StageWords {
    static constexpr int XPL = STK ? 3 : 2;
    static constexpr int RP = (2 * BM + XPL * BN + kConv - 1) / kConv;   // row-planes per thread
    uint4 w[RP];
    int valid[RP];
};

// Walks this CTA's flattened (tile, stage) sequence for one converter
// thread, two stages ahead of the expansion.  The tile decode and the row
// addresses of the thread's row-planes are computed once per tile; a stage
// then only advances K by 128 (4 words).
template <int BN, bool STK = false>
struct StageCursor {
    static constexpr int RP = StageWords<BN, STK>::RP;
    static constexpr int XPL = StageWords<BN, STK>::XPL;
    const uint32_t *row[RP];     // packed words of the current tile's row-planes (nullptr: zero row)
    int t, kb, num_kb, total, step;

    __device__ void start_tile(const Args1 &args, int ct) {
        if (t >= total) return;
        int b, mt, nt;
        decode_tile(t, args, b, mt, nt);
#pragma unroll
        for (int j = 0; j < RP; ++j) {
            const int rp = ct + j * kConv;
            row[j] = nullptr;
            if (rp < 2 * BM) {
                const int plane = rp / BM, mrow = mt * BM + rp % BM;
                if (mrow < args.M)
                    row[j] = args.Wb +
                             (static_cast<size_t>((b / args.per_w) * 2 + plane) * args.w_rows + mrow) * args.Kw;
            } else if (rp < 2 * BM + XPL * BN) {
                const int x = rp - 2 * BM;
                // stacked slots -Xi, Xr, Xi read the imaginary, real, imaginary bits
                const int slot = x / BN, nrow = nt * BN + x % BN;
                const int plane = STK ? (slot == 1 ? 0 : 1) : slot;
                if (nrow < args.N)
                    row[j] = args.Xb + (static_cast<size_t>(b * 2 + plane) * args.N + nrow) * args.Kw;
            }
        }
    }

    __device__ void init(const Args1 &args, int ct) {
        t = blockIdx.x;
        kb = 0;
        num_kb = args.num_kb;
        total = args.total_tiles;
        step = gridDim.x;
        start_tile(args, ct);
    }

    // the words of the cursor's stage, then advance to the next stage
    __device__ void load(const Args1 &args, int ct, StageWords<BN, STK> &w) {
#pragma unroll
        for (int j = 0; j < RP; ++j) {
            w.w[j] = make_uint4(0, 0, 0, 0);
            w.valid[j] = 0;
        }
        if (t >= total) return;
        const int valid = args.K - kb * BKE;
#pragma unroll
        for (int j = 0; j < RP; ++j)
            if (row[j]) {
                w.w[j] = __ldg(reinterpret_cast<const uint4 *>(row[j] + kb * 4));
                w.valid[j] = valid;
            }
        if (++kb == num_kb) {
            kb = 0;
            t += step;
            start_tile(args, ct);
        }
    }
};

template <int BN, int STAGES, bool STK>
__global__ void __launch_bounds__(Cfg1<BN, STAGES, STK>::THREADS, 1)
    cgemm_1bit_kernel(const __grid_constant__ CUtensorMap tmY, const Args1 args) {
    using C = Cfg1<BN, STAGES, STK>;
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

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, kConv / 32);       // one arrival per converter warp
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, 32 * C::EPI_WARPS);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
        if (args.tma_store) tma_prefetch_desc(&tmY);
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t kIdesc = idesc_f32acc(BM, BN, 0, false);     // E4M3 x E4M3
            constexpr uint32_t kIdescNeg = idesc_f32acc(BM, BN, 0, true);
            int stage = 0;
            uint32_t phase = 0;
            int local = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < args.total_tiles && ok; t += gridDim.x, ++local) {
                const int acc = local % C::ACC_BUFS;
                const uint32_t aphase = (local / C::ACC_BUFS) & 1;
                if (!mbar_wait(tempty0 + 8 * acc, aphase ^ 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_re = tmem_base + acc * 2 * BN;
                const uint32_t d_im = d_re + BN;
                for (int kb = 0; kb < args.num_kb; ++kb) {
                    if (!mbar_wait(full0 + 8 * stage, phase) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = s0 + stage * C::STAGE_BYTES;
                    const uint32_t bx = a + C::A_BYTES;
                    const int ksteps = min(BKE / 32, (args.K - kb * BKE + 31) / 32);
                    if (STK) {
                        // Wr [Xr; Xi] + Wi [-Xi; Xr] -> [Re | Im] (slots -Xi, Xr, Xi)
                        constexpr uint32_t kIdesc2 = idesc_f32acc(BM, 2 * BN, 0, false);
                        for (int j = 0; j < ksteps; ++j) {
                            const uint32_t accum = (kb > 0 || j > 0) ? 1u : 0u;
                            mma_f8f6f4(d_re, sdesc_kmajor_sw128(a + 32 * j),
                                       sdesc_kmajor_sw128(bx + C::B_PLANE + 32 * j), kIdesc2, accum);
                            mma_f8f6f4(d_re, sdesc_kmajor_sw128(a + C::A_PLANE + 32 * j),
                                       sdesc_kmajor_sw128(bx + 32 * j), kIdesc2, 1u);
                        }
                    } else
                    for (int j = 0; j < ksteps; ++j) {
                        const uint64_t ar = sdesc_kmajor_sw128(a + 32 * j);
                        const uint64_t ai = sdesc_kmajor_sw128(a + C::A_PLANE + 32 * j);
                        const uint64_t br = sdesc_kmajor_sw128(bx + 32 * j);
                        const uint64_t bi = sdesc_kmajor_sw128(bx + C::B_PLANE + 32 * j);
                        const uint32_t accum = (kb > 0 || j > 0) ? 1u : 0u;
                        mma_f8f6f4(d_re, ar, br, kIdesc, accum);
                        mma_f8f6f4(d_re, ai, bi, kIdescNeg, 1u);
                        mma_f8f6f4(d_im, ar, bi, kIdesc, accum);
                        mma_f8f6f4(d_im, ai, br, kIdesc, 1u);
                    }
                    mma_commit(empty0 + 8 * stage);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(tfull0 + 8 * acc);
            }
            if (!ok) {
                atomicOr(args.status, kErrTimeoutMma);
                *abort_flag = 1;
            }
            mma_commit(done_bar);
            if (!mbar_wait(done_bar, 0)) atomicOr(args.status, kErrTimeoutDrain);
        }
    } else if (warp <= kConv / 32) {
        // ------------------------------------------------------- converters
        // The (tile, stage) sequence of this CTA is flattened and the packed
        // words of stage i + 2 are loaded while stage i is expanded, so the
        // L2 latency of the 16-byte loads is covered.
        const int ct = threadIdx.x - 32;               // 0..kConv-1
        const int my_tiles = (args.total_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
        const int iters = my_tiles * args.num_kb;
        StageCursor<BN, STK> cursor;
        cursor.init(args, ct);
        StageWords<BN, STK> cur, nxt;
        cursor.load(args, ct, cur);
        cursor.load(args, ct, nxt);
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int i = 0; i < iters; ++i) {
            StageWords<BN, STK> ahead;
            cursor.load(args, ct, ahead);
            if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u) || *abort_flag) {
                ok = false;
                break;
            }
            const uint32_t a = s0 + stage * C::STAGE_BYTES;
#pragma unroll
            for (int j = 0; j < StageWords<BN, STK>::RP; ++j) {
                const int rp = ct + j * kConv;
                if (rp < 2 * BM) {
                    const int r = rp % BM;
                    expand_row(a + (rp / BM) * C::A_PLANE + r * 128, r, cur.w[j], cur.valid[j]);
                } else if (rp < 2 * BM + C::XPL * BN) {
                    const int x = rp - 2 * BM, r = x % BN;
                    const uint32_t dst = a + C::A_BYTES + (x / BN) * C::B_PLANE + r * 128;
                    if (STK && x < BN)                     // slot 0 holds -Xi
                        expand_row<true>(dst, r, cur.w[j], cur.valid[j]);
                    else
                        expand_row(dst, r, cur.w[j], cur.valid[j]);
                }
            }
            fence_async_smem();                        // generic writes -> tensor core reads
            __syncwarp();
            if (lane == 0) mbar_arrive(full0 + 8 * stage);
            if (++stage == STAGES) {
                stage = 0;
                phase ^= 1u;
            }
            cur = nxt;
            nxt = ahead;
        }
        if (!ok && ct == 0) {
            atomicOr(args.status, kErrTimeoutProducer);
            *abort_flag = 1;
        }
    } else {
        // --------------------------------------------------------- epilogue
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const int ew = warp - 1 - kConv / 32;          // epilogue warp 0 .. EPI_WARPS - 1
        constexpr int kChunks = BN / 16 / (C::EPI_WARPS / 4);
        const int c0 = (ew >> 2) * kChunks;            // this warp's 16-column chunks
        // eight warps: one 4 KB buffer each; four: two each
        const uint32_t stage_buf = staging0 + ew * (C::EPI_WARPS == 8 ? 4096 : 8192);
        const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
        int local = 0;
        int chunk_count = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < args.total_tiles && ok; t += gridDim.x, ++local) {
            const int acc = local % C::ACC_BUFS;
            const uint32_t aphase = (local / C::ACC_BUFS) & 1;
            if (!mbar_wait(tfull0 + 8 * acc, aphase) || *abort_flag) {
                ok = false;
                break;
            }
            tc_fence_after();
            int b, mt, nt;
            decode_tile(t, args, b, mt, nt);
            const int m = mt * BM + row;
            const uint32_t tP = tmem_base + lane_off + acc * 2 * BN;
            int32_t *yrow = args.Y + (static_cast<size_t>(b) * args.M + m) * args.N * 2;
#pragma unroll 1
            for (int c = c0; c < c0 + kChunks; ++c) {
                float re[16], im[16];
                tmem_ld_2x16(tP + c * 16, tP + BN + c * 16, re, im);
                const int n0 = nt * BN + c * 16;
                if (args.tma_store) {
                    if (n0 < args.N) {
                        const uint32_t buf =
                            stage_buf + (C::EPI_WARPS == 8 ? 0 : (chunk_count & 1) * 4096);
                        if (lane == 0) {
                            if (C::EPI_WARPS == 8)
                                bulk_wait_read<0>();   // the buffer's last store has read it
                            else
                                bulk_wait_read<1>();
                        }
                        __syncwarp();
                        const uint32_t rbase = buf + lane * 128;
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            st_shared_u4(rbase + ((j ^ (lane & 7)) << 4),
                                         make_uint4(__float2int_rn(re[2 * j]), __float2int_rn(im[2 * j]),
                                                    __float2int_rn(re[2 * j + 1]),
                                                    __float2int_rn(im[2 * j + 1])));
                        fence_async_smem();
                        __syncwarp();
                        if (lane == 0) {
                            tma_store_3d(&tmY, buf, 2 * n0, mt * BM + quarter * 32, b);
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
            tc_fence_before();
            mbar_arrive(tempty0 + 8 * acc);
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
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, C::TMEM_COLS);
    }
}

template <int BN, int STAGES, bool STK = false>
cudaError_t launch1(const tcbf_plan_s &pl, const uint32_t *Wb, const uint32_t *Xb, int32_t *Y,
                    cudaStream_t s, int raster) {
    using C = Cfg1<BN, STAGES, STK>;
    const tcbf_problem &p = pl.p;
    CUtensorMap tmY;
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
    Args1 a;
    a.Y = Y;
    a.Wb = Wb;
    a.Xb = Xb;
    a.status = pl.status;
    a.tma_store = tma_store;
    a.M = static_cast<int>(p.M);
    a.w_rows = static_cast<int>(w_plane_rows(pl));
    a.N = static_cast<int>(p.N);
    a.K = static_cast<int>(p.K);
    a.Kw = static_cast<int>(pl.Kw);
    a.per_w = static_cast<int>(pl.per_w);
    a.tiles.prefix = pl.m_prefix;
    a.tiles.batch = static_cast<int>(p.batch);
    a.tiles.m_tiles = static_cast<int>(ceil_div(p.M, BM));
    a.tiles.n_tiles = static_cast<int>(ceil_div(p.N, BN));
    a.tiles.raster = raster;
    a.num_kb = static_cast<int>(ceil_div(p.K, BKE));
    const int64_t total = (pl.m_prefix ? pl.m_tiles_sum : int64_t(a.tiles.m_tiles) * p.batch) *
                          a.tiles.n_tiles;
    if (total > 0x7fffffff) return cudaErrorInvalidValue;
    a.total_tiles = static_cast<int>(total);
    auto kern = cgemm_1bit_kernel<BN, STAGES, STK>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int grid = static_cast<int>(std::min<int64_t>(total, pl.num_sms));
    kern<<<grid, C::THREADS, C::SMEM_BYTES, s>>>(tmY, a);
    return cudaGetLastError();
}

struct Config1 {
    const char *name;
    int raster;
    cudaError_t (*fn)(const tcbf_plan_s &, const uint32_t *, const uint32_t *, int32_t *,
                      cudaStream_t, int);
};

// The 4-bit tensor path (gemm_1bit_fp4.cu); plans it cannot take (no scratch,
// K > 2^23, uneven batches) run configuration 0 instead.
template <int V>
cudaError_t launch_fp4_or_e4m3(const tcbf_plan_s &pl, const uint32_t *Wb, const uint32_t *Xb,
                               int32_t *Y, cudaStream_t s, int) {
    const cudaError_t e = launch_gemm_1bit_fp4(pl, Wb, Xb, Y, s, V);
    if (e == cudaErrorNotSupported) return launch1<256, 2>(pl, Wb, Xb, Y, s, 0);
    return e;
}

const Config1 kConfigs1[] = {
    {"1bit->e4m3 BM128 BN256 BK128 stages2 tmem-single n-fastest", 0, launch1<256, 2>},
    {"1bit->e4m3 BM128 BN128 BK128 stages3 tmem-double n-fastest", 0, launch1<128, 3>},
    {"1bit->e4m3 BM128 BN256 BK128 stages2 tmem-single m-fastest", 1, launch1<256, 2>},
    {"1bit->e4m3 BM128 BN128 BK128 stages3 tmem-double m-fastest", 1, launch1<128, 3>},
    {"1bit->e4m3 stacked [-Xi,Xr,Xi] N256 BM128 BN128 BK128 stages2 tmem-double n-fastest", 0,
     launch1<128, 2, true>},
    {"1bit->e2m1 mxf4 stacked [-Xi,Xr,Xi] N256 2-SM pair BM256 BN128 BK256 stages3 tmem-single", 0,
     launch_fp4_or_e4m3<0>},
    {"1bit->e2m1 mxf4 stacked [-Xi,Xr,Xi] N128 2-SM pair BM256 BN64 BK256 stages4 tmem-double", 0,
     launch_fp4_or_e4m3<1>},
    {"1bit->e2m1 mxf4 stacked [-Xi,Xr,Xi] N192 2-SM pair BM256 BN96 BK256 stages3 tmem-double", 0,
     launch_fp4_or_e4m3<2>},
    {"1bit->e2m1 mxf4 stacked [-Xi,Xr,Xi] N224 2-SM pair BM256 BN112 BK256 stages3 tmem-double", 0,
     launch_fp4_or_e4m3<3>},
};
constexpr int kFirstFp4Config = 5;

}  // namespace

int gemm_1bit_num_configs() { return static_cast<int>(sizeof(kConfigs1) / sizeof(kConfigs1[0])); }

bool gemm_1bit_config_fp4(int config) {
    return config >= kFirstFp4Config && config < gemm_1bit_num_configs();
}

int gemm_1bit_fp4_variant(int config) {
    return gemm_1bit_config_fp4(config) ? config - kFirstFp4Config : -1;
}

// K up to 6144: 256 x 112 tiles with two accumulators (columns 0 and 256),
// so each tile's drain overlaps the next tile's MMAs; longer K: the
// full-width N = 256 tiles with one accumulator.  Measured (GEMM on
// expanded planes): the radio 1-bit block (K = 1024, 64 batches) 1.82 ms
// against 1.94 for 256 x 96 tiles and 2.51 for N = 256; single products
// M = N = K = 2000 to 6144 3-10% faster with the 256 x 112 tiles, 8192 the
// same, and K = 65536 16.5 ms against 18.3 (256 x 112).
int gemm_1bit_fp4_default_config(int64_t K) { return K <= 6144 ? kFirstFp4Config + 3 : kFirstFp4Config; }

const char *gemm_1bit_config_name(int config) {
    if (config < 0 || config >= gemm_1bit_num_configs()) return "invalid";
    return kConfigs1[config].name;
}

cudaError_t launch_gemm_1bit(const tcbf_plan_s &pl, const uint32_t *Wb, const uint32_t *Xb,
                             int32_t *Y, cudaStream_t s) {
    const int c = (pl.config >= 0 && pl.config < gemm_1bit_num_configs()) ? pl.config : 0;
    return kConfigs1[c].fn(pl, Wb, Xb, Y, s, kConfigs1[c].raster);
}

}  // namespace tcbf
