// noalloc.cu — an FP16 beamform entry point that allocates no device memory.
//
// The ordinary path needs a plan (which allocates a small device status
// word) and a caller-allocated buffer for the packed samples.  Some callers
// cannot allocate device memory at call time: code running while a stream
// is being captured into a CUDA graph, real-time acquisition loops where the
// implicit device synchronisation of cudaMalloc/cudaFree would break the
// timing, and plug-ins whose host framework owns the device memory budget.
// tcbf_beamform_fp16_noalloc serves them: the packed samples and the status
// word live in one file-scope __device__ array of fixed size, so the call
// only launches the existing pack and GEMM kernels on memory that exists
// from module load until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "tcbf_internal.h"

namespace tcbf {
namespace {

// Packed-sample capacity of the static scratch (bytes); the first 256 bytes
// of the array hold the device status word.
constexpr size_t kNoallocStatusBytes = 256;
constexpr size_t kNoallocScratchBytes = size_t(64) << 20;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocStatusBytes +
                                                                  kNoallocScratchBytes];

constexpr int kMaxDevices = 128;

struct DeviceSetup {
    bool ready = false;
    unsigned long long ctx_id = 0;      // context the address below belongs to (0: unknown)
    unsigned char *scratch = nullptr;   // device address of g_noalloc_scratch
    int num_sms = 0;
    bool sm103 = false;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

// Unique id of the current context (driver entry points fetched once), or 0
// when it cannot be read.  A cudaDeviceReset by the caller gives the device
// a new context in which the static array has a new address.
unsigned long long current_ctx_id() {
    typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
    typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
        get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Once per device and context, with that device current: the device address
// of the static array (its host-side name is only a stand-in) and device
// facts.  Repeated when the device's context has changed since (or its id
// cannot be read).
tcbf_status setup_device(int device, DeviceSetup &out) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup &d = g_setup[device];
    const unsigned long long ctx = current_ctx_id();
    if (!d.ready || ctx == 0 || ctx != d.ctx_id) {
        int major = 0, minor = 0, sms = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
            return TCBF_ERR_CUDA;
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
            return TCBF_ERR_CUDA;
        d.scratch = static_cast<unsigned char *>(p);
        d.num_sms = sms;
        d.sm103 = (major == 10 && minor == 3);
        d.ctx_id = ctx;
        d.ready = true;
    }
    out = d;
    return TCBF_OK;
}

}  // namespace
}  // namespace tcbf

using namespace tcbf;

TCBF_EXPORT tcbf_status tcbf_beamform_fp16_noalloc(const tcbf_problem *p, int device,
                                                   const void *Wp, const void *X, int src_type,
                                                   float *Y, int check, tcbf_stream_t stream) {
    if (!p || !Wp || !X || !Y) return TCBF_ERR_INVALID_ARG;
    tcbf_problem q = *p;
    if (q.w_batches == 0) q.w_batches = q.batch;
    if (q.batch < 1 || q.M < 1 || q.N < 1 || q.K < 1 || q.w_batches < 1 ||
        q.batch % q.w_batches != 0 || q.mode != TCBF_MODE_FP16 || q.flags != 0)
        return TCBF_ERR_INVALID_ARG;
    if (src_type != TCBF_SRC_CF16 && src_type != TCBF_SRC_CF32) return TCBF_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(Wp) | reinterpret_cast<uintptr_t>(X) |
         reinterpret_cast<uintptr_t>(Y)) & 15u)
        return TCBF_ERR_INVALID_ARG;
    if (q.M > (int64_t(1) << 30) || q.N > (int64_t(1) << 30) || q.K > (int64_t(1) << 30) ||
        q.batch > 65535)
        return TCBF_ERR_UNSUPPORTED;
    // the packed samples must fit the static scratch
    const int64_t Kp = packed_row_k(q.K);
    const double need = double(q.batch) * 2.0 * double(q.N) * double(Kp) * 2.0;
    if (need > double(kNoallocScratchBytes)) return TCBF_ERR_BUDGET;

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return TCBF_ERR_UNSUPPORTED;
    if (device < 0 || device >= ndev || device >= kMaxDevices) return TCBF_ERR_INVALID_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return TCBF_ERR_CUDA;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return TCBF_ERR_CUDA;
    tcbf_status st = TCBF_OK;
    DeviceSetup d;
    st = setup_device(device, d);
    if (st == TCBF_OK && !d.sm103) st = TCBF_ERR_UNSUPPORTED;
    if (st == TCBF_OK) {
        // a plan on the stack: same kernels, status word in the static array
        tcbf_plan_s pl;
        pl.p = q;
        pl.device = device;
        pl.num_sms = d.num_sms;
        pl.per_w = q.batch / q.w_batches;
        pl.Kp = Kp;
        pl.Kw = round_up(q.K, 128) / 32;
        pl.config = 0;
        pl.status = reinterpret_cast<uint32_t *>(d.scratch);
        void *packed_x = d.scratch + kNoallocStatusBytes;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        cudaError_t e = cudaMemsetAsync(pl.status, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess) e = launch_pack_f16_x(pl, src_type, X, packed_x, s);
        if (e == cudaSuccess) e = launch_gemm_f16(pl, Wp, packed_x, Y, s);
        if (e != cudaSuccess) {
            st = TCBF_ERR_CUDA;
        } else if (check) {
            // read the status word in order on the call's own stream (not the
            // legacy default stream, which would also wait for unrelated work)
            uint32_t word = 0;
            if (cudaMemcpyAsync(&word, pl.status, sizeof(word), cudaMemcpyDeviceToHost, s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                st = TCBF_ERR_CUDA;
            else if (word != 0)
                st = (word & 0xffu) ? TCBF_ERR_TIMEOUT : TCBF_ERR_DEVICE;
        }
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return st;
}
