// server.cu — continuous-batching beamforming server (host runtime).
//
// Requests (one block of samples for one resident weight set, in one of
// the three modes) arrive over time.  A scheduler thread admits every
// arrived request whose device buffers fit into a fixed arena (the HBM
// budget), issues its whole path on one of several CUDA streams
//   host X -> device, transpose/pack, beamform, device Y -> host
// and, as completion events fire, frees the buffers and admits the next
// arrivals.  Requests that arrive while others run are admitted as memory
// frees up and overlap with them on the device: a persistent GEMM launch
// covers min(tiles, SMs) SMs, so small requests share the GPU.  Every
// request runs the same kernels with the same tile configuration as it
// would alone, so its result does not depend on the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/tcbf_server.h"
#include "tcbf_internal.h"

namespace tcbf {
namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over one device allocation (offsets, 256-byte units).
class Arena {
  public:
    bool init(size_t bytes) {
        if (cudaMalloc(&base_, bytes) != cudaSuccess) {
            base_ = nullptr;
            return false;
        }
        size_ = bytes;
        free_[0] = bytes;
        return true;
    }
    ~Arena() {
        if (base_) cudaFree(base_);
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    // returns offset or SIZE_MAX
    size_t alloc(size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                live_[off] = bytes;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off) {
        auto it = live_.find(off);
        if (it == live_.end()) return;
        size_t len = it->second;
        live_.erase(it);
        used_ -= len;
        size_t start = off;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + len == nx->first) {
            len += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == start) {
                start = pv->first;
                len += pv->second;
                free_.erase(pv);
            }
        }
        free_[start] = len;
    }
    uint8_t *ptr(size_t off) const { return static_cast<uint8_t *>(base_) + off; }

  private:
    void *base_ = nullptr;
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;   // offset -> length
    std::map<size_t, size_t> live_;
};

struct WeightSet {
    int64_t M = 0, K = 0;
    const void *Wp = nullptr;
};

struct Req {
    tcbf_request r;
    uint64_t ticket = 0;
    int64_t M = 0, K = 0;
    const void *Wp = nullptr;
    size_t bytes_x = 0, bytes_xp = 0, bytes_y = 0;
    size_t off = SIZE_MAX;            // arena block
    int stream = -1;
    cudaEvent_t done = nullptr;
    double t_admit = 0, t_done = 0;
    int status = TCBF_OK;
};

}  // namespace
}  // namespace tcbf

struct tcbf_server_s {
    int device = 0;
    int num_sms = 0;
    int num_streams = 1;
    int max_inflight = 0;
    tcbf::Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<int> stream_load;
    uint32_t *status = nullptr;        // one 256-byte status block per stream
    std::map<std::pair<int, int>, tcbf::WeightSet> weights;   // (set, mode)
    std::mutex mu;
    std::condition_variable cv;
    std::deque<tcbf::Req *> pending;   // submitted, not admitted (arrival order)
    std::vector<tcbf::Req *> inflight;
    std::vector<tcbf::Req *> all;      // by ticket - 1
    std::thread worker;
    std::atomic<bool> stop{false};
    bool started = false;
    tcbf::Clock::time_point t0;
    size_t peak_used = 0;
    int peak_inflight = 0;
};

namespace tcbf {
namespace {

double now_s(const tcbf_server_s *s) {
    return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

size_t packed_bytes_for(int mode, int64_t rows, int64_t K) {
    switch (mode) {
        case TCBF_MODE_FP16: return size_t(2 * rows * packed_row_k(K) * 2);
        case TCBF_MODE_1BIT: return size_t(2 * rows * (round_up(K, 128) / 32) * 4);
        default: return size_t(2 * rows * 2 * round_up(K, 64) + rows * 4);
    }
}

tcbf_plan_s request_plan(const tcbf_server_s *s, const Req &q) {
    tcbf_plan_s pl;
    pl.p.batch = 1;
    pl.p.M = q.M;
    pl.p.N = q.r.N;
    pl.p.K = q.K;
    pl.p.w_batches = 1;
    pl.p.mode = q.r.mode;
    pl.p.flags = 0;
    pl.device = s->device;
    pl.num_sms = s->num_sms;
    pl.per_w = 1;
    pl.Kp = packed_row_k(q.K);
    pl.Kw = round_up(q.K, 128) / 32;
    pl.Kb2 = fp8_row_bytes(q.K, pl.p.flags);
    pl.config = 0;
    pl.status = s->status + 64 * q.stream;
    return pl;
}

// Issue the whole path of one admitted request on its stream.
cudaError_t issue(tcbf_server_s *s, Req &q) {
    cudaStream_t st = s->streams[q.stream];
    uint8_t *x = s->arena.ptr(q.off);
    uint8_t *xp = x + ((q.bytes_x + 255) & ~size_t(255));
    uint8_t *y = xp + ((q.bytes_xp + 255) & ~size_t(255));
    const tcbf_plan_s pl = request_plan(s, q);
    cudaError_t e = cudaMemcpyAsync(x, q.r.host_x, q.bytes_x, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    switch (q.r.mode) {
        case TCBF_MODE_FP16:
            e = launch_pack_f16_x(pl, q.r.src_type, x, xp, st);
            if (e == cudaSuccess) e = launch_gemm_f16(pl, q.Wp, xp, reinterpret_cast<float *>(y), st);
            break;
        case TCBF_MODE_1BIT:
            e = launch_pack_bits_x(pl, q.r.src_type, x, xp, st);
            if (e == cudaSuccess)
                e = launch_gemm_1bit(pl, static_cast<const uint32_t *>(q.Wp),
                                     reinterpret_cast<const uint32_t *>(xp),
                                     reinterpret_cast<int32_t *>(y), st);
            break;
        default:
            e = launch_pack_split8_x(pl, q.r.src_type, x, xp, st);
            if (e == cudaSuccess) e = launch_gemm_split8(pl, q.Wp, xp, reinterpret_cast<float *>(y), st);
            break;
    }
    if (e != cudaSuccess) return e;
    if (q.r.host_y) e = cudaMemcpyAsync(q.r.host_y, y, q.bytes_y, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaEventRecord(q.done, st);
}

void worker_loop(tcbf_server_s *s) {
    cudaSetDevice(s->device);
    constexpr int kLookahead = 8;     // arrived requests that may pass a blocked head
    while (true) {
        bool idle = true;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // completions
            for (size_t i = 0; i < s->inflight.size();) {
                Req *q = s->inflight[i];
                const cudaError_t e = cudaEventQuery(q->done);
                if (e == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                q->t_done = now_s(s);
                if (e != cudaSuccess) q->status = TCBF_ERR_CUDA;
                s->arena.release(q->off);
                s->stream_load[q->stream]--;
                s->inflight[i] = s->inflight.back();
                s->inflight.pop_back();
                idle = false;
            }
            // admission: arrived requests in arrival order; a request that does
            // not fit yet may be passed by up to kLookahead later arrivals
            const double t = now_s(s);
            int looked = 0;
            for (auto it = s->pending.begin(); it != s->pending.end() && looked < kLookahead;) {
                Req *q = *it;
                if (q->r.arrival_s > t) break;
                if (s->max_inflight > 0 && int(s->inflight.size()) >= s->max_inflight) break;
                const size_t need = ((q->bytes_x + 255) & ~size_t(255)) +
                                    ((q->bytes_xp + 255) & ~size_t(255)) + q->bytes_y;
                const size_t off = s->arena.alloc(need);
                if (off == SIZE_MAX) {
                    ++looked;
                    ++it;
                    continue;
                }
                q->off = off;
                int best = 0;
                for (int k = 1; k < s->num_streams; ++k)
                    if (s->stream_load[k] < s->stream_load[best]) best = k;
                q->stream = best;
                s->stream_load[best]++;
                q->t_admit = t;
                if (issue(s, *q) != cudaSuccess) q->status = TCBF_ERR_CUDA;
                s->inflight.push_back(q);
                s->peak_used = std::max(s->peak_used, s->arena.used());
                s->peak_inflight = std::max(s->peak_inflight, int(s->inflight.size()));
                it = s->pending.erase(it);
                idle = false;
            }
            if (s->stop && !s->pending.empty()) {
                for (Req *q : s->pending) q->status = TCBF_ERR_INVALID_ARG;   // dropped
                s->pending.clear();
            }
            if (s->pending.empty() && s->inflight.empty()) s->cv.notify_all();
            if (s->stop && s->inflight.empty()) break;
        }
        if (idle) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace
}  // namespace tcbf

using namespace tcbf;

TCBF_EXPORT tcbf_status tcbf_server_create(tcbf_server_t *out, int device, size_t arena_bytes,
                                           int num_streams, int max_inflight) {
    if (!out) return TCBF_ERR_INVALID_ARG;
    *out = nullptr;
    if (arena_bytes < 4096 || num_streams < 1 || num_streams > 64 || max_inflight < 0)
        return TCBF_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return TCBF_ERR_UNSUPPORTED;
    if (device < 0 || device >= ndev) return TCBF_ERR_INVALID_ARG;
    int major = 0, minor = 0, sms = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (major != 10 || minor != 3) return TCBF_ERR_UNSUPPORTED;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    auto *s = new (std::nothrow) tcbf_server_s;
    tcbf_status st = s ? TCBF_OK : TCBF_ERR_OOM;
    if (st == TCBF_OK) {
        s->device = device;
        s->num_sms = sms;
        s->num_streams = num_streams;
        s->max_inflight = max_inflight;
        if (!s->arena.init(arena_bytes)) st = TCBF_ERR_OOM;
    }
    if (st == TCBF_OK && (cudaMalloc(&s->status, 256 * size_t(num_streams)) != cudaSuccess ||
                          cudaMemset(s->status, 0, 256 * size_t(num_streams)) != cudaSuccess))
        st = TCBF_ERR_OOM;
    for (int i = 0; st == TCBF_OK && i < num_streams; ++i) {
        cudaStream_t q;
        if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) st = TCBF_ERR_CUDA;
        else s->streams.push_back(q);
        s->stream_load.push_back(0);
    }
    if (st != TCBF_OK && s) {
        for (auto q : s->streams) cudaStreamDestroy(q);
        if (s->status) cudaFree(s->status);
        delete s;
        s = nullptr;
    }
    cudaSetDevice(prev);
    *out = s;
    return st;
}

TCBF_EXPORT tcbf_status tcbf_server_register_weights(tcbf_server_t s, int set_id, int mode,
                                                     int64_t M, int64_t K, const void *Wp) {
    if (!s || !Wp || M < 1 || K < 1 || M > (int64_t(1) << 30) || K > (int64_t(1) << 30))
        return TCBF_ERR_INVALID_ARG;
    if (mode != TCBF_MODE_FP16 && mode != TCBF_MODE_FP8SPLIT && mode != TCBF_MODE_1BIT)
        return TCBF_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(Wp) & 15u) return TCBF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    WeightSet w;
    w.M = M;
    w.K = K;
    w.Wp = Wp;
    s->weights[{set_id, mode}] = w;
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_server_submit(tcbf_server_t s, const tcbf_request *r,
                                           uint64_t *ticket) {
    if (!s || !r || !r->host_x) return TCBF_ERR_INVALID_ARG;
    if (r->N < 1 || r->N > (int64_t(1) << 30)) return TCBF_ERR_INVALID_ARG;
    if (r->src_type != TCBF_SRC_CF16 && r->src_type != TCBF_SRC_CF32) return TCBF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->weights.find({r->set_id, r->mode});
    if (it == s->weights.end()) return TCBF_ERR_INVALID_ARG;
    auto *q = new (std::nothrow) Req;
    if (!q) return TCBF_ERR_OOM;
    q->r = *r;
    q->M = it->second.M;
    q->K = it->second.K;
    q->Wp = it->second.Wp;
    q->bytes_x = size_t(q->K * r->N) * (r->src_type == TCBF_SRC_CF16 ? 4 : 8);
    q->bytes_xp = packed_bytes_for(r->mode, r->N, q->K);
    q->bytes_y = size_t(q->M * r->N) * 8;
    const size_t need = ((q->bytes_x + 255) & ~size_t(255)) + ((q->bytes_xp + 255) & ~size_t(255)) +
                        q->bytes_y;
    if (need > s->arena.size()) {
        delete q;
        return TCBF_ERR_BUDGET;
    }
    if (cudaSetDevice(s->device) != cudaSuccess ||
        cudaEventCreateWithFlags(&q->done, cudaEventDisableTiming) != cudaSuccess) {
        delete q;
        return TCBF_ERR_CUDA;
    }
    s->all.push_back(q);
    q->ticket = s->all.size();
    // keep the pending queue in arrival order
    auto pos = s->pending.end();
    while (pos != s->pending.begin() && (*std::prev(pos))->r.arrival_s > r->arrival_s) --pos;
    s->pending.insert(pos, q);
    if (ticket) *ticket = q->ticket;
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_server_start(tcbf_server_t s) {
    if (!s) return TCBF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->started) return TCBF_ERR_INVALID_ARG;
    s->t0 = Clock::now();
    s->started = true;
    s->worker = std::thread(worker_loop, s);
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_server_wait_all(tcbf_server_t s, double timeout_s) {
    if (!s || !s->started) return TCBF_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [s] {
        return s->pending.empty() && s->inflight.empty();
    });
    return ok ? TCBF_OK : TCBF_ERR_TIMEOUT;
}

TCBF_EXPORT tcbf_status tcbf_server_result(tcbf_server_t s, uint64_t ticket,
                                           tcbf_request_result *out) {
    if (!s || !out) return TCBF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticket < 1 || ticket > s->all.size()) return TCBF_ERR_INVALID_ARG;
    const Req *q = s->all[ticket - 1];
    out->arrival_s = q->r.arrival_s;
    out->admit_s = q->t_admit;
    out->done_s = q->t_done;
    out->stream = q->stream;
    out->status = (q->t_done > 0) ? q->status : -1;
    out->ops = 8.0 * double(q->M) * double(q->r.N) * double(q->K);
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_server_stats(tcbf_server_t s, tcbf_server_counters *out) {
    if (!s || !out) return TCBF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->all.size();
    out->pending = s->pending.size();
    out->inflight = s->inflight.size();
    out->peak_inflight = s->peak_inflight;
    out->arena_bytes = s->arena.size();
    out->peak_arena_bytes = s->peak_used;
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_server_destroy(tcbf_server_t s) {
    if (!s) return TCBF_OK;
    if (s->started) {
        s->stop = true;
        s->worker.join();
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (auto q : s->all) {
        if (q->done) cudaEventDestroy(q->done);
        delete q;
    }
    for (auto q : s->streams) cudaStreamDestroy(q);
    if (s->status) cudaFree(s->status);
    delete s;
    cudaSetDevice(prev);
    return TCBF_OK;
}
