// host_pipe.cu — tcbf_beamform_host: the step for host-resident data, with
// the host<->device copies of each chunk of batches overlapped with the
// pack + beamform of its neighbours.  Host code only; every step of the
// computation runs in the library's kernels.
//
// Per chunk c (slot s = c mod kSlots, batches [b0, b0 + nb)):
//   h2d stream:     [wait comp[s] of chunk c - kSlots]  X_host -> Xsrc[s]   -> h2d[s]
//   compute stream: wait h2d[s], [wait d2h[s] of chunk c - kSlots]
//                   pack Xsrc[s] -> Xp[s]; beamform Wp, Xp[s] -> Yd[s]       -> comp[s]
//   d2h streams:    wait comp[s]; Yd[s] -> Y_host, split over kD2h streams   -> d2h[s]
// The chunk's work goes to a sub-plan (batch = nb, w_batches = nb / per_w)
// whose W is the matching sub-range of the packed weights.
//
// A single-batch problem has nothing to overlap across batches, so it is cut
// into ranges of W rows instead: X is copied in and packed once, then each
// range's GEMM (a sub-plan over rows [m0, m0 + rows) of the same packed W)
// writes slot s and its rows of Y are copied out while the next range
// computes.  Ranges are whole waves of 128-row tiles over all SMs, so the
// persistent grid stays full.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <new>

#include "tcbf_internal.h"

namespace tcbf {
namespace {

constexpr int kSlots = 3;   // chunks in flight: one copying in, one computing, one copying out
constexpr int kD2h = 2;     // device-to-host streams per chunk (Y is the large direction)
constexpr int kRowRanges = 4;   // row ranges of a single-batch problem (about)

}  // namespace
}  // namespace tcbf

struct tcbf_host_pipe {
    int64_t chunk = 0;                 // batches the staging holds per slot
    void *xsrc[tcbf::kSlots] = {};
    void *xp[tcbf::kSlots] = {};
    void *yd[tcbf::kSlots] = {};
    cudaStream_t h2d = nullptr, comp = nullptr;
    cudaStream_t d2h[tcbf::kD2h] = {};
    cudaEvent_t ev_h2d[tcbf::kSlots] = {}, ev_comp[tcbf::kSlots] = {};
    cudaEvent_t ev_d2h[tcbf::kSlots][tcbf::kD2h] = {};
    cudaEvent_t ev_entry = nullptr, ev_exit[tcbf::kD2h] = {};
    bool used[tcbf::kSlots] = {};      // slot has work enqueued (its events are recorded)
};

namespace tcbf {
namespace {

void free_staging(tcbf_host_pipe &hp) {
    for (int s = 0; s < kSlots; ++s) {
        if (hp.xsrc[s]) cudaFree(hp.xsrc[s]);
        if (hp.xp[s]) cudaFree(hp.xp[s]);
        if (hp.yd[s]) cudaFree(hp.yd[s]);
        hp.xsrc[s] = hp.xp[s] = hp.yd[s] = nullptr;
        hp.used[s] = false;
    }
    hp.chunk = 0;
}

void destroy_pipe(tcbf_host_pipe *hp) {
    if (!hp) return;
    free_staging(*hp);
    if (hp->h2d) cudaStreamDestroy(hp->h2d);
    if (hp->comp) cudaStreamDestroy(hp->comp);
    for (int i = 0; i < kD2h; ++i) {
        if (hp->d2h[i]) cudaStreamDestroy(hp->d2h[i]);
        if (hp->ev_exit[i]) cudaEventDestroy(hp->ev_exit[i]);
    }
    for (int s = 0; s < kSlots; ++s) {
        if (hp->ev_h2d[s]) cudaEventDestroy(hp->ev_h2d[s]);
        if (hp->ev_comp[s]) cudaEventDestroy(hp->ev_comp[s]);
        for (int i = 0; i < kD2h; ++i)
            if (hp->ev_d2h[s][i]) cudaEventDestroy(hp->ev_d2h[s][i]);
    }
    if (hp->ev_entry) cudaEventDestroy(hp->ev_entry);
    delete hp;
}

tcbf_host_pipe *make_pipe() {
    auto *hp = new (std::nothrow) tcbf_host_pipe;
    if (!hp) return nullptr;
    bool ok = cudaStreamCreateWithFlags(&hp->h2d, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&hp->comp, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&hp->ev_entry, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < kD2h && ok; ++i)
        ok = cudaStreamCreateWithFlags(&hp->d2h[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&hp->ev_exit[i], cudaEventDisableTiming) == cudaSuccess;
    for (int s = 0; s < kSlots && ok; ++s) {
        ok = cudaEventCreateWithFlags(&hp->ev_h2d[s], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&hp->ev_comp[s], cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; i < kD2h && ok; ++i)
            ok = cudaEventCreateWithFlags(&hp->ev_d2h[s][i], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        destroy_pipe(hp);
        return nullptr;
    }
    return hp;
}

int64_t src_bytes(int src_type) { return src_type == TCBF_SRC_CF16 ? 4 : 8; }

// Packed bytes of `nb` batches of X (which = 1) for the plan's mode.
int64_t packed_x_bytes(const tcbf_plan_s &pl, int64_t nb) {
    const int64_t N = pl.p.N;
    switch (pl.p.mode) {
        case TCBF_MODE_FP16:
            if (interleaved_x(pl)) return nb * pl.p.K * N * 4;   // the caller's layout, FP16
            return nb * x_planes(pl) * N * pl.Kp * 2;
        case TCBF_MODE_1BIT: return nb * 2 * N * pl.Kw * 4;
        case TCBF_MODE_TF32: return nb * 2 * N * pl.Kp * 4;
        default:
            if (fp8_block_scaled(pl.p.flags))
                return nb * 2 * N * pl.Kb2 + fp8blk_sf_bytes(nb, N, pl.p.K, pl.p.flags, 1);
            return nb * 2 * N * pl.Kb2 + nb * N * 4;
    }
}

// Bytes of one packed W row in one plane.
int64_t packed_w_row_bytes(const tcbf_plan_s &pl) {
    switch (pl.p.mode) {
        case TCBF_MODE_FP16: return pl.Kp * 2;
        case TCBF_MODE_1BIT: return pl.Kw * 4;
        case TCBF_MODE_TF32: return pl.Kp * 4;
        default: return pl.Kb2;
    }
}

// Bytes of one packed W batch's planes (the exponents of split-FP8 follow
// all w_batches' planes).
int64_t packed_w_batch_bytes(const tcbf_plan_s &pl) {
    const int64_t M = pl.p.M;
    switch (pl.p.mode) {
        case TCBF_MODE_FP16: return 2 * M * pl.Kp * 2;
        case TCBF_MODE_1BIT: return 2 * M * pl.Kw * 4;
        case TCBF_MODE_TF32: return 2 * M * pl.Kp * 4;
        default: return 2 * M * pl.Kb2;
    }
}

// Interleaved-X FP16 plans read an FP16 source as it was copied in: no pack.
bool reads_source(const tcbf_plan_s &pl, int src_type) {
    return pl.p.mode == TCBF_MODE_FP16 && interleaved_x(pl) && src_type == TCBF_SRC_CF16;
}

cudaError_t pack_x(const tcbf_plan_s &pl, int src_type, const void *src, void *dst, cudaStream_t s) {
    if (pl.p.mode == TCBF_MODE_FP16)
        return interleaved_x(pl) ? launch_copy_x_cf16(pl, src_type, src, dst, s)
                                 : launch_pack_f16_x(pl, src_type, src, dst, s);
    if (pl.p.mode == TCBF_MODE_1BIT) return launch_pack_bits_x(pl, src_type, src, dst, s);
    if (pl.p.mode == TCBF_MODE_TF32) return launch_pack_tf32_x(pl, src_type, src, dst, s);
    return launch_pack_split8_x(pl, src_type, src, dst, s);
}

cudaError_t beamform(const tcbf_plan_s &pl, const void *Wp, const void *Xp, void *Y, cudaStream_t s) {
    if (pl.p.mode == TCBF_MODE_FP16) return launch_gemm_f16(pl, Wp, Xp, static_cast<float *>(Y), s);
    if (pl.p.mode == TCBF_MODE_1BIT)
        return launch_gemm_1bit(pl, static_cast<const uint32_t *>(Wp),
                                static_cast<const uint32_t *>(Xp), static_cast<int32_t *>(Y), s);
    if (pl.p.mode == TCBF_MODE_TF32) return launch_gemm_tf32(pl, Wp, Xp, static_cast<float *>(Y), s);
    return launch_gemm_split8(pl, Wp, Xp, static_cast<float *>(Y), s);
}

// (Re)allocates the staging for `chunk` batches per slot.  Waits for work
// still using the old staging first.
cudaError_t ensure_staging(const tcbf_plan_s &pl, tcbf_host_pipe &hp, int64_t chunk) {
    if (hp.chunk >= chunk) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < kSlots && e == cudaSuccess; ++s)
        if (hp.used[s])
            for (int i = 0; i < kD2h && e == cudaSuccess; ++i) e = cudaEventSynchronize(hp.ev_d2h[s][i]);
    if (e != cudaSuccess) return e;
    free_staging(hp);
    const int64_t xs = chunk * pl.p.K * pl.p.N * 8;   // room for either source type
    const int64_t xp = packed_x_bytes(pl, chunk);
    const int64_t yb = chunk * pl.p.M * pl.p.N * 8;
    for (int s = 0; s < kSlots && e == cudaSuccess; ++s) {
        e = cudaMalloc(&hp.xsrc[s], static_cast<size_t>(xs));
        if (e == cudaSuccess) e = cudaMalloc(&hp.xp[s], static_cast<size_t>(xp));
        if (e == cudaSuccess) e = cudaMalloc(&hp.yd[s], static_cast<size_t>(yb));
    }
    if (e != cudaSuccess) {
        free_staging(hp);
        return e;
    }
    hp.chunk = chunk;
    return cudaSuccess;
}

tcbf_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return TCBF_OK;
    if (e == cudaErrorMemoryAllocation) return TCBF_ERR_OOM;
    return TCBF_ERR_CUDA;
}

}  // namespace

void host_pipe_destroy(tcbf_plan_s &pl) {
    if (!pl.pipe) return;
    // staging may still be read by copies in flight
    for (int s = 0; s < kSlots; ++s)
        if (pl.pipe->used[s])
            for (int i = 0; i < kD2h; ++i) cudaEventSynchronize(pl.pipe->ev_d2h[s][i]);
    destroy_pipe(pl.pipe);
    pl.pipe = nullptr;
}

}  // namespace tcbf

using namespace tcbf;

TCBF_EXPORT tcbf_status tcbf_beamform_host(tcbf_plan_t plan, const void *X_host, int src_type,
                                           const void *Wp, void *Y_host, int64_t chunk,
                                           tcbf_stream_t stream) {
    if (!plan || !X_host || !Wp || !Y_host || chunk < 0) return TCBF_ERR_INVALID_ARG;
    if (src_type != TCBF_SRC_CF16 && src_type != TCBF_SRC_CF32) return TCBF_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(Wp) & 15u) return TCBF_ERR_INVALID_ARG;
    if (plan->m_prefix) return TCBF_ERR_UNSUPPORTED;
    const tcbf_problem &p = plan->p;
    const int64_t per_w = plan->per_w;
    if (chunk == 0) chunk = per_w * ((p.batch / per_w + 15) / 16);
    if (chunk % per_w != 0) return TCBF_ERR_INVALID_ARG;
    if (chunk > p.batch) chunk = p.batch;

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != plan->device && cudaSetDevice(plan->device) != cudaSuccess) return TCBF_ERR_CUDA;
    struct Restore {
        int dev;
        ~Restore() {
            if (dev >= 0) cudaSetDevice(dev);
        }
    } restore{prev};

    if (!plan->pipe && !(plan->pipe = make_pipe())) return TCBF_ERR_CUDA;
    tcbf_host_pipe &hp = *plan->pipe;
    cudaError_t e = ensure_staging(*plan, hp, chunk);
    if (e != cudaSuccess) return status_of(e);

    cudaStream_t user = static_cast<cudaStream_t>(stream);
    e = cudaEventRecord(hp.ev_entry, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.h2d, hp.ev_entry, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.comp, hp.ev_entry, 0);
    for (int i = 0; i < kD2h && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(hp.d2h[i], hp.ev_entry, 0);

    const int64_t xsrc_per_b = p.K * p.N * src_bytes(src_type);
    const int64_t y_per_b = p.M * p.N * 8;
    const int64_t wb = packed_w_batch_bytes(*plan);
    const int32_t *w_exps_all =
        p.mode == TCBF_MODE_FP8SPLIT
            ? reinterpret_cast<const int32_t *>(static_cast<const uint8_t *>(Wp) + p.w_batches * wb)
            : nullptr;
    // block-scaled FP8: W's scale tiles (128 rows per tile, `st` stages each)
    // instead of one exponent per row
    const bool blk = p.mode == TCBF_MODE_FP8SPLIT && fp8_block_scaled(p.flags);
    const int64_t st_bytes = fp8blk_stages(p.K, p.flags) * kFp8BlkTile;
    const int64_t w_tiles = ceil_div(p.M, kFp8BlkRowsW);
    auto w_scales = [&](int64_t wb_first, int64_t m_first) -> const int32_t * {
        if (!w_exps_all) return nullptr;
        if (!blk) return w_exps_all + wb_first * p.M + m_first;
        const uint8_t *t = reinterpret_cast<const uint8_t *>(w_exps_all);
        return reinterpret_cast<const int32_t *>(t + (wb_first * w_tiles + m_first / kFp8BlkRowsW) *
                                                         st_bytes);
    };
    const auto *xh = static_cast<const uint8_t *>(X_host);
    auto *yh = static_cast<uint8_t *>(Y_host);

    if (p.batch == 1) {
        // ---- one batch: X in and packed once, then ranges of W rows
        const int64_t n_tiles = ceil_div(p.N, 128);
        const int64_t rows_wave = 128 * std::max<int64_t>(1, plan->num_sms / n_tiles);
        const int64_t rows = round_up(ceil_div(p.M, kRowRanges), rows_wave);
        const int64_t wrow = packed_w_row_bytes(*plan);
        for (int s = 0; s < kSlots && e == cudaSuccess; ++s)
            if (hp.used[s]) e = cudaStreamWaitEvent(hp.h2d, hp.ev_comp[s], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hp.xsrc[0], xh, static_cast<size_t>(xsrc_per_b), cudaMemcpyHostToDevice,
                                hp.h2d);
        if (e == cudaSuccess) e = cudaEventRecord(hp.ev_h2d[0], hp.h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.comp, hp.ev_h2d[0], 0);
        const void *xg = reads_source(*plan, src_type) ? hp.xsrc[0] : hp.xp[0];
        if (e == cudaSuccess && xg == hp.xp[0])
            e = pack_x(*plan, src_type, hp.xsrc[0], hp.xp[0], hp.comp);
        int64_t c = 0;
        for (int64_t m0 = 0; m0 < p.M && e == cudaSuccess; m0 += rows, ++c) {
            const int s = static_cast<int>(c % kSlots);
            const int64_t nr = std::min(rows, p.M - m0);
            tcbf_plan_s sub = *plan;
            sub.p.M = nr;
            sub.w_rows = p.M;
            sub.graph_exec = nullptr;
            sub.pipe = nullptr;
            sub.debug_drop_fill = -1;
            sub.w_exps = w_scales(0, m0);       // m0 is a multiple of 128
            const void *w_sub = static_cast<const uint8_t *>(Wp) + m0 * wrow;
            // the slot's Y is free once its last copy-out ran
            for (int i = 0; i < kD2h && e == cudaSuccess && hp.used[s]; ++i)
                e = cudaStreamWaitEvent(hp.comp, hp.ev_d2h[s][i], 0);
            if (e == cudaSuccess) e = beamform(sub, w_sub, xg, hp.yd[s], hp.comp);
            if (e == cudaSuccess) e = cudaEventRecord(hp.ev_comp[s], hp.comp);
            const int64_t ybytes = nr * p.N * 8;
            int64_t off = 0;
            for (int i = 0; i < kD2h && e == cudaSuccess; ++i) {
                int64_t part = (ybytes / kD2h + 15) / 16 * 16;
                if (i == kD2h - 1 || off + part > ybytes) part = ybytes - off;
                e = cudaStreamWaitEvent(hp.d2h[i], hp.ev_comp[s], 0);
                if (e == cudaSuccess && part > 0)
                    e = cudaMemcpyAsync(yh + m0 * p.N * 8 + off, static_cast<uint8_t *>(hp.yd[s]) + off,
                                        static_cast<size_t>(part), cudaMemcpyDeviceToHost, hp.d2h[i]);
                if (e == cudaSuccess) e = cudaEventRecord(hp.ev_d2h[s][i], hp.d2h[i]);
                off += part;
            }
            if (e == cudaSuccess) hp.used[s] = true;
        }
    } else {
        int64_t c = 0;
        for (int64_t b0 = 0; b0 < p.batch && e == cudaSuccess; b0 += chunk, ++c) {
            const int s = static_cast<int>(c % kSlots);
            const int64_t nb = b0 + chunk <= p.batch ? chunk : p.batch - b0;
            const int64_t wb0 = b0 / per_w;
            // the chunk's sub-plan: its batches, their weights
            tcbf_plan_s sub = *plan;
            sub.p.batch = nb;
            sub.p.w_batches = nb / per_w;
            sub.graph_exec = nullptr;
            sub.pipe = nullptr;
            sub.debug_drop_fill = -1;
            sub.w_exps = w_scales(wb0, 0);
            const void *w_sub = static_cast<const uint8_t *>(Wp) + wb0 * wb;

            // copy in (the slot's source buffer is free once its last pack ran)
            if (hp.used[s]) e = cudaStreamWaitEvent(hp.h2d, hp.ev_comp[s], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hp.xsrc[s], xh + b0 * xsrc_per_b, static_cast<size_t>(nb * xsrc_per_b),
                                    cudaMemcpyHostToDevice, hp.h2d);
            if (e == cudaSuccess) e = cudaEventRecord(hp.ev_h2d[s], hp.h2d);
            // compute (the slot's Y is free once its last copy-out ran)
            if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.comp, hp.ev_h2d[s], 0);
            for (int i = 0; i < kD2h && e == cudaSuccess && hp.used[s]; ++i)
                e = cudaStreamWaitEvent(hp.comp, hp.ev_d2h[s][i], 0);
            const void *xg = reads_source(sub, src_type) ? hp.xsrc[s] : hp.xp[s];
            if (e == cudaSuccess && xg == hp.xp[s])
                e = pack_x(sub, src_type, hp.xsrc[s], hp.xp[s], hp.comp);
            if (e == cudaSuccess) e = beamform(sub, w_sub, xg, hp.yd[s], hp.comp);
            if (e == cudaSuccess) e = cudaEventRecord(hp.ev_comp[s], hp.comp);
            // copy out, split by batches (or by bytes for one batch) over the d2h streams
            const int64_t ybytes = nb * y_per_b;
            int64_t off = 0;
            for (int i = 0; i < kD2h && e == cudaSuccess; ++i) {
                int64_t part = (ybytes / kD2h + 15) / 16 * 16;
                if (i == kD2h - 1 || off + part > ybytes) part = ybytes - off;
                e = cudaStreamWaitEvent(hp.d2h[i], hp.ev_comp[s], 0);
                if (e == cudaSuccess && part > 0)
                    e = cudaMemcpyAsync(yh + b0 * y_per_b + off, static_cast<uint8_t *>(hp.yd[s]) + off,
                                        static_cast<size_t>(part), cudaMemcpyDeviceToHost, hp.d2h[i]);
                if (e == cudaSuccess) e = cudaEventRecord(hp.ev_d2h[s][i], hp.d2h[i]);
                off += part;
            }
            if (e == cudaSuccess) hp.used[s] = true;
        }
    }
    // the caller's stream waits for every copy-out
    for (int i = 0; i < kD2h && e == cudaSuccess; ++i) {
        e = cudaEventRecord(hp.ev_exit[i], hp.d2h[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(user, hp.ev_exit[i], 0);
    }
    return status_of(e);
}
