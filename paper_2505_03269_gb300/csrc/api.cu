// api.cu — the C ABI (include/tcbf.h): plan validation and bookkeeping,
// argument checks, tensor-map encoding and kernel dispatch.  Host code only.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <new>
#include <vector>

#include "tcbf_internal.h"

namespace tcbf {
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Makes the plan's device current for the duration of a call.
class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
        ok_ = (prev_ == dev) || cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev_ >= 0) cudaSetDevice(prev_);
    }
    bool ok() const { return ok_; }

  private:
    int prev_ = -1;
    bool ok_ = false;
};

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

constexpr int64_t kMaxDim = int64_t(1) << 30;   // per-dimension limit (int32 tile indexing)

tcbf_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return TCBF_OK;
    if (e == cudaErrorMemoryAllocation) return TCBF_ERR_OOM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ||
        e == cudaErrorNoKernelImageForDevice || e == cudaErrorNotSupported)
        return TCBF_ERR_UNSUPPORTED;
    return TCBF_ERR_CUDA;
}

size_t packed_bytes(const tcbf_plan_s &pl, int which) {
    const tcbf_problem &p = pl.p;
    const int64_t nb = which == 0 ? p.w_batches : p.batch;
    const int64_t rows = which == 0 ? p.M : p.N;
    switch (p.mode) {
        case TCBF_MODE_FP16:
            if (which == 1 && interleaved_x(pl))   // the caller's layout: [batch][K][N] complex
                return static_cast<size_t>(nb * p.K * p.N * 4);
            return static_cast<size_t>(nb * (which == 0 ? 2 : x_planes(pl)) * rows * pl.Kp * 2);
        case TCBF_MODE_1BIT:
            return static_cast<size_t>(nb * 2 * rows * pl.Kw * 4);
        case TCBF_MODE_FP8SPLIT:   // hi/lo bytes, then one int32 scale exponent per row
            if (fp8_block_scaled(p.flags))   // ... or the scale tiles
                return static_cast<size_t>(nb * 2 * rows * pl.Kb2 +
                                           fp8blk_sf_bytes(nb, rows, p.K, p.flags, which));
            return static_cast<size_t>(nb * 2 * rows * pl.Kb2 + nb * rows * 4);
        case TCBF_MODE_TF32:       // FP32 planes holding TF32 values
            return static_cast<size_t>(nb * 2 * rows * pl.Kp * 4);
        default:
            return 0;
    }
}

// Packed X planes of an interleaved-X plan that the fused kernel cannot take.
cudaError_t alloc_ix_planes(tcbf_plan_s &pl) {
    const size_t bytes = static_cast<size_t>(pl.p.batch * 2 * pl.p.N * pl.Kp * 2);
    return cudaMalloc(&pl.ix_planes, bytes);
}

}  // namespace

CUresult encode_tiled(CUtensorMap *map, CUtensorMapDataType type, uint32_t rank, void *gaddr,
                      const uint64_t *dims, const uint64_t *strides_bytes, const uint32_t *box,
                      CUtensorMapSwizzle swizzle) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return CUDA_ERROR_NOT_SUPPORTED;
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return fn(map, type, rank, gaddr, reinterpret_cast<const cuuint64_t *>(dims),
              reinterpret_cast<const cuuint64_t *>(strides_bytes),
              reinterpret_cast<const cuuint32_t *>(box), estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

}  // namespace tcbf

using namespace tcbf;

TCBF_EXPORT const char *tcbf_status_string(tcbf_status s) {
    switch (s) {
        case TCBF_OK: return "ok";
        case TCBF_ERR_INVALID_ARG: return "invalid argument";
        case TCBF_ERR_UNSUPPORTED: return "unsupported (device or shape)";
        case TCBF_ERR_OOM: return "out of device memory";
        case TCBF_ERR_BUDGET: return "over memory budget";
        case TCBF_ERR_CUDA: return "CUDA error";
        case TCBF_ERR_TIMEOUT: return "device-side wait timed out";
        case TCBF_ERR_DEVICE: return "device-side check failed";
    }
    return "unknown status";
}

namespace {

// The layout TCBF_FLAG_AUTO_LAYOUT resolves to: stacked X when the shape's
// operations per byte of the stacked layout (packed W, packed X with its
// third plane, Y) reach the threshold, planar otherwise.
uint32_t auto_layout(const tcbf_problem &q) {
    const double Kp = static_cast<double>(packed_row_k(q.K));
    const double ops = 8.0 * q.batch * q.M * q.N * q.K;
    const double bytes = 4.0 * q.w_batches * q.M * Kp + 6.0 * q.batch * q.N * Kp +
                         8.0 * q.batch * q.M * q.N;
    return ops >= TCBF_AUTO_STACKED_MIN_INTENSITY * bytes ? TCBF_FLAG_STACKED_X : 0u;
}

// The FP16 transpose/pack of X into the plan's current layout.
cudaError_t pack_x_into(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                        cudaStream_t s) {
    return interleaved_x(pl) ? launch_copy_x_cf16(pl, src_type, src, dst, s)
                             : launch_pack_f16_x(pl, src_type, src, dst, s);
}

}  // namespace

TCBF_EXPORT tcbf_status tcbf_plan_create(tcbf_plan_t *out, const tcbf_problem *p, int device) {
    if (!out) return TCBF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!p) return TCBF_ERR_INVALID_ARG;
    tcbf_problem q = *p;
    if (q.w_batches == 0) q.w_batches = q.batch;
    if (q.batch < 1 || q.M < 1 || q.N < 1 || q.K < 1 || q.w_batches < 1) return TCBF_ERR_INVALID_ARG;
    if (q.batch % q.w_batches != 0) return TCBF_ERR_INVALID_ARG;
    if (q.mode != TCBF_MODE_FP16 && q.mode != TCBF_MODE_FP8SPLIT && q.mode != TCBF_MODE_1BIT &&
        q.mode != TCBF_MODE_TF32)
        return TCBF_ERR_INVALID_ARG;
    const uint32_t fp8_flags = TCBF_FLAG_FP8_HI_ONLY | TCBF_FLAG_FP8_FOUR_PRODUCTS;
    const uint32_t f16_flags = TCBF_FLAG_STACKED_X | TCBF_FLAG_INTERLEAVED_X;
    const uint32_t blk = TCBF_FLAG_FP8_BLOCK_SCALES;
    const uint32_t autol = TCBF_FLAG_AUTO_LAYOUT;
    if ((q.flags & ~(f16_flags | fp8_flags | blk | autol)) != 0) return TCBF_ERR_INVALID_ARG;
    if ((q.flags & autol) && (q.mode != TCBF_MODE_FP16 || (q.flags & f16_flags)))
        return TCBF_ERR_INVALID_ARG;
    if ((q.flags & f16_flags) && q.mode != TCBF_MODE_FP16) return TCBF_ERR_INVALID_ARG;
    if ((q.flags & f16_flags) == f16_flags) return TCBF_ERR_INVALID_ARG;   // one or the other
    if ((q.flags & (fp8_flags | blk)) && q.mode != TCBF_MODE_FP8SPLIT) return TCBF_ERR_INVALID_ARG;
    if ((q.flags & fp8_flags) == fp8_flags) return TCBF_ERR_INVALID_ARG;   // one or the other
    if (q.M > kMaxDim || q.N > kMaxDim || q.K > kMaxDim || q.batch > 65535)
        return TCBF_ERR_UNSUPPORTED;
    // 1-bit sums are exact integers in the FP32 accumulators while 2K < 2^24
    if (q.mode == TCBF_MODE_1BIT && q.K > (int64_t(1) << 22)) return TCBF_ERR_UNSUPPORTED;
    const bool autolayout = (q.flags & autol) != 0;
    if (autolayout) q.flags = (q.flags & ~autol) | auto_layout(q);

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return TCBF_ERR_UNSUPPORTED;
    if (device < 0 || device >= ndev) return TCBF_ERR_INVALID_ARG;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return TCBF_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3) return TCBF_ERR_UNSUPPORTED;   // sm_103 only

    auto *pl = new (std::nothrow) tcbf_plan_s;
    if (!pl) return TCBF_ERR_OOM;
    pl->p = q;
    pl->auto_layout = autolayout;
    pl->device = device;
    pl->num_sms = prop.multiProcessorCount;
    pl->per_w = q.batch / q.w_batches;
    pl->Kp = packed_row_k(q.K);
    pl->Kw = round_up(q.K, 128) / 32;
    pl->Kb2 = fp8_row_bytes(q.K, q.flags);
    pl->config = 0;
    {
        DeviceGuard g(device);
        if (!g.ok()) {
            delete pl;
            return TCBF_ERR_CUDA;
        }
        if (cudaMalloc(&pl->status, 256) != cudaSuccess) {
            delete pl;
            return TCBF_ERR_OOM;
        }
        if (cudaMemset(pl->status, 0, 256) != cudaSuccess) {
            cudaFree(pl->status);
            delete pl;
            return TCBF_ERR_CUDA;
        }
        // interleaved X that the fused kernel cannot read (rows of 4N bytes
        // not 16-byte multiples): the beamform call packs into these planes
        if (interleaved_x(*pl) && !ix_fused_ok(*pl)) {
            const cudaError_t e = alloc_ix_planes(*pl);
            if (e != cudaSuccess) {
                cudaFree(pl->status);
                delete pl;
                return e == cudaErrorMemoryAllocation ? TCBF_ERR_OOM : TCBF_ERR_CUDA;
            }
        }
        if (interleaved_x(*pl)) pl->config = gemm_f16_ix_default_config(q.K);
        // stacked X (or a layout the tuner may set to it) with promoted long
        // K: the workspace that lets the pair kernel split its last wave; a
        // plan without it runs those tiles whole
        if (q.mode == TCBF_MODE_FP16 && (q.flags & (TCBF_FLAG_STACKED_X | TCBF_FLAG_AUTO_LAYOUT))) {
            const size_t ws = stacked_tail_ws_bytes(*pl);
            if (ws > 0 && cudaMalloc(&pl->tail_ws, ws) == cudaSuccess) pl->tail_ws_bytes = ws;
            else pl->tail_ws = nullptr;
        }
        // 1-bit: the 4-bit tensor path by default when its planes fit
        if (q.mode == TCBF_MODE_1BIT && gemm_1bit_fp4_reserve(*pl) == cudaSuccess &&
            gemm_1bit_fp4_usable(*pl))
            pl->config = gemm_1bit_fp4_default_config(q.K);
    }
    *out = pl;
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_plan_destroy(tcbf_plan_t plan) {
    if (!plan) return TCBF_OK;
    {
        DeviceGuard g(plan->device);
        host_pipe_destroy(*plan);
        if (plan->graph_exec) cudaGraphExecDestroy(plan->graph_exec);
        if (plan->m_prefix) cudaFree(plan->m_prefix);
        if (plan->status) cudaFree(plan->status);
        if (plan->ix_planes) cudaFree(plan->ix_planes);
        if (plan->tail_ws) cudaFree(plan->tail_ws);
        gemm_1bit_fp4_release(*plan);
    }
    delete plan;
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_packed_size(tcbf_plan_t plan, int which, size_t *bytes) {
    if (!plan || !bytes || (which != 0 && which != 1)) return TCBF_ERR_INVALID_ARG;
    *bytes = packed_bytes(*plan, which);
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_workspace_size(tcbf_plan_t plan, size_t *bytes) {
    if (!plan || !bytes) return TCBF_ERR_INVALID_ARG;
    *bytes = 0;
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_transpose_pack(tcbf_plan_t plan, int which, int src_type,
                                            const void *src, void *dst, tcbf_stream_t stream) {
    if (!plan || !src || !dst || (which != 0 && which != 1)) return TCBF_ERR_INVALID_ARG;
    if (src_type != TCBF_SRC_CF16 && src_type != TCBF_SRC_CF32) return TCBF_ERR_INVALID_ARG;
    if (!aligned16(src) || !aligned16(dst)) return TCBF_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (plan->p.mode) {
        case TCBF_MODE_FP16:
            e = which == 0            ? launch_pack_f16_w(*plan, src_type, src, dst, s)
                : interleaved_x(*plan) ? launch_copy_x_cf16(*plan, src_type, src, dst, s)
                                       : launch_pack_f16_x(*plan, src_type, src, dst, s);
            break;
        case TCBF_MODE_1BIT:
            e = which == 0 ? launch_pack_bits_w(*plan, src_type, src, dst, s)
                           : launch_pack_bits_x(*plan, src_type, src, dst, s);
            break;
        case TCBF_MODE_FP8SPLIT:
            e = which == 0 ? launch_pack_split8_w(*plan, src_type, src, dst, s)
                           : launch_pack_split8_x(*plan, src_type, src, dst, s);
            break;
        case TCBF_MODE_TF32:
            e = which == 0 ? launch_pack_tf32_w(*plan, src_type, src, dst, s)
                           : launch_pack_tf32_x(*plan, src_type, src, dst, s);
            break;
        default:
            return TCBF_ERR_UNSUPPORTED;
    }
    return from_cuda(e);
}

TCBF_EXPORT tcbf_status tcbf_unpack_bits(tcbf_plan_t plan, int which, const uint32_t *src,
                                         void *dst, int dst_type, tcbf_stream_t stream) {
    if (!plan || !src || !dst || (which != 0 && which != 1)) return TCBF_ERR_INVALID_ARG;
    if (dst_type != TCBF_SRC_CF16 && dst_type != TCBF_SRC_CF32) return TCBF_ERR_INVALID_ARG;
    if (plan->p.mode != TCBF_MODE_1BIT) return TCBF_ERR_INVALID_ARG;
    if (!aligned16(src) || !aligned16(dst)) return TCBF_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    return from_cuda(launch_unpack_bits(*plan, which, src, dst_type, dst,
                                        static_cast<cudaStream_t>(stream)));
}

TCBF_EXPORT tcbf_status tcbf_beamform_fp16(tcbf_plan_t plan, const void *Wp, const void *Xp,
                                           float *Y, tcbf_stream_t stream) {
    if (!plan || !Wp || !Xp || !Y) return TCBF_ERR_INVALID_ARG;
    if (plan->p.mode != TCBF_MODE_FP16) return TCBF_ERR_INVALID_ARG;
    if (!aligned16(Wp) || !aligned16(Xp) || !aligned16(Y)) return TCBF_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    const cudaError_t e = launch_gemm_f16(*plan, Wp, Xp, Y, static_cast<cudaStream_t>(stream));
    plan->debug_drop_fill = -1;          // the test hook applies to one call
    return from_cuda(e);
}

TCBF_EXPORT tcbf_status tcbf_beamform_fp8split(tcbf_plan_t plan, const void *Wp, const void *Xp,
                                               float *Y, tcbf_stream_t stream) {
    if (!plan || !Wp || !Xp || !Y) return TCBF_ERR_INVALID_ARG;
    if (plan->p.mode != TCBF_MODE_FP8SPLIT) return TCBF_ERR_INVALID_ARG;
    if (!aligned16(Wp) || !aligned16(Xp) || !aligned16(Y)) return TCBF_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    const cudaError_t e = launch_gemm_split8(*plan, Wp, Xp, Y, static_cast<cudaStream_t>(stream));
    plan->debug_drop_fill = -1;          // the test hook applies to one call
    return from_cuda(e);
}

TCBF_EXPORT tcbf_status tcbf_beamform_tf32(tcbf_plan_t plan, const void *Wp, const void *Xp,
                                           float *Y, tcbf_stream_t stream) {
    if (!plan || !Wp || !Xp || !Y) return TCBF_ERR_INVALID_ARG;
    if (plan->p.mode != TCBF_MODE_TF32) return TCBF_ERR_INVALID_ARG;
    if (!aligned16(Wp) || !aligned16(Xp) || !aligned16(Y)) return TCBF_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    const cudaError_t e = launch_gemm_tf32(*plan, Wp, Xp, Y, static_cast<cudaStream_t>(stream));
    plan->debug_drop_fill = -1;          // the test hook applies to one call
    return from_cuda(e);
}

TCBF_EXPORT tcbf_status tcbf_debug_drop_fill(tcbf_plan_t plan, int64_t fill) {
    if (!plan) return TCBF_ERR_INVALID_ARG;
    if (fill < 0) {
        plan->debug_drop_fill = -1;
        return TCBF_OK;
    }
    if (plan->p.mode != TCBF_MODE_FP16 && plan->p.mode != TCBF_MODE_FP8SPLIT &&
        plan->p.mode != TCBF_MODE_TF32)
        return TCBF_ERR_UNSUPPORTED;
    // one-SM, non-cluster tile configurations only (the cluster and pair
    // kernels share barriers across CTAs)
    if ((plan->p.flags & (TCBF_FLAG_STACKED_X | TCBF_FLAG_INTERLEAVED_X)) || plan->config < 0 ||
        plan->config > 5)
        return TCBF_ERR_UNSUPPORTED;
    if (fill > 0x7fffffff) return TCBF_ERR_INVALID_ARG;
    plan->debug_drop_fill = fill;
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_beamform_1bit(tcbf_plan_t plan, const uint32_t *Wbits,
                                           const uint32_t *Xbits, int32_t *Y,
                                           tcbf_stream_t stream) {
    if (!plan || !Wbits || !Xbits || !Y) return TCBF_ERR_INVALID_ARG;
    if (plan->p.mode != TCBF_MODE_1BIT) return TCBF_ERR_INVALID_ARG;
    if (!aligned16(Wbits) || !aligned16(Xbits) || !aligned16(Y)) return TCBF_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    return from_cuda(launch_gemm_1bit(*plan, Wbits, Xbits, Y, static_cast<cudaStream_t>(stream)));
}

TCBF_EXPORT tcbf_status tcbf_expand_1bit(tcbf_plan_t plan, int which, const uint32_t *bits,
                                         tcbf_stream_t stream) {
    if (!plan || !bits || (which != 0 && which != 1)) return TCBF_ERR_INVALID_ARG;
    if (plan->p.mode != TCBF_MODE_1BIT || !aligned16(bits)) return TCBF_ERR_INVALID_ARG;
    if (!gemm_1bit_config_fp4(plan->config) || !gemm_1bit_fp4_usable(*plan))
        return TCBF_ERR_UNSUPPORTED;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    return from_cuda(launch_expand_1bit_fp4(*plan, which, bits, static_cast<cudaStream_t>(stream)));
}

TCBF_EXPORT tcbf_status tcbf_transpose_pack_expanded(tcbf_plan_t plan, int which, int src_type,
                                                     const void *src, tcbf_stream_t stream) {
    if (!plan || !src || (which != 0 && which != 1)) return TCBF_ERR_INVALID_ARG;
    if (src_type != TCBF_SRC_CF16 && src_type != TCBF_SRC_CF32) return TCBF_ERR_INVALID_ARG;
    if (plan->p.mode != TCBF_MODE_1BIT || !aligned16(src)) return TCBF_ERR_INVALID_ARG;
    if (!gemm_1bit_config_fp4(plan->config) || !gemm_1bit_fp4_usable(*plan))
        return TCBF_ERR_UNSUPPORTED;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    return from_cuda(
        launch_pack_1bit_fp4(*plan, which, src_type, src, static_cast<cudaStream_t>(stream)));
}

TCBF_EXPORT tcbf_status tcbf_beamform_1bit_expanded(tcbf_plan_t plan, int32_t *Y,
                                                    tcbf_stream_t stream) {
    if (!plan || !Y) return TCBF_ERR_INVALID_ARG;
    if (plan->p.mode != TCBF_MODE_1BIT || !aligned16(Y)) return TCBF_ERR_INVALID_ARG;
    if (!gemm_1bit_config_fp4(plan->config) || !gemm_1bit_fp4_usable(*plan))
        return TCBF_ERR_UNSUPPORTED;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    return from_cuda(launch_gemm_1bit_fp4_expanded(*plan, Y, static_cast<cudaStream_t>(stream),
                                                   gemm_1bit_fp4_variant(plan->config)));
}

TCBF_EXPORT tcbf_status tcbf_weights_from_geometry(tcbf_plan_t plan, const double *rx_pos,
                                                   const double *targets, int near_field,
                                                   const double *freqs, double c, void *Wp_out,
                                                   tcbf_stream_t stream) {
    if (!plan || !rx_pos || !targets || !freqs || !Wp_out) return TCBF_ERR_INVALID_ARG;
    if (near_field != 0 && near_field != 1) return TCBF_ERR_INVALID_ARG;
    if (!(c > 0.0)) return TCBF_ERR_INVALID_ARG;
    if (!aligned16(Wp_out) || (reinterpret_cast<uintptr_t>(rx_pos) & 7u) ||
        (reinterpret_cast<uintptr_t>(targets) & 7u) || (reinterpret_cast<uintptr_t>(freqs) & 7u))
        return TCBF_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    return from_cuda(launch_weights(*plan, rx_pos, targets, near_field, freqs, c, Wp_out,
                                    static_cast<cudaStream_t>(stream)));
}

TCBF_EXPORT tcbf_status tcbf_last_device_error(tcbf_plan_t plan) {
    if (!plan) return TCBF_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return TCBF_ERR_CUDA;
    uint32_t word = 0;
    if (cudaMemcpy(&word, plan->status, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TCBF_ERR_CUDA;
    if (word == 0) return TCBF_OK;
    cudaMemset(plan->status, 0, sizeof(word));
    return (word & 0xffu) ? TCBF_ERR_TIMEOUT : TCBF_ERR_DEVICE;
}

TCBF_EXPORT tcbf_status tcbf_plan_num_configs(tcbf_plan_t plan, int *count) {
    if (!plan || !count) return TCBF_ERR_INVALID_ARG;
    *count = plan->p.mode == TCBF_MODE_1BIT                  ? gemm_1bit_num_configs()
             : fp8_block_scaled(plan->p.flags)           ? gemm_split8_blk_num_configs()
             : (plan->p.flags & TCBF_FLAG_STACKED_X)     ? gemm_f16_stacked_num_configs()
             : (plan->p.flags & TCBF_FLAG_INTERLEAVED_X) ? gemm_f16_ix_num_configs()
                                                         : gemm_f16_num_configs();
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_plan_flags(tcbf_plan_t plan, uint32_t *flags) {
    if (!plan || !flags) return TCBF_ERR_INVALID_ARG;
    *flags = plan->p.flags;
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_plan_get_config(tcbf_plan_t plan, int *config) {
    if (!plan || !config) return TCBF_ERR_INVALID_ARG;
    *config = plan->config;
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_plan_set_config(tcbf_plan_t plan, int config) {
    if (!plan) return TCBF_ERR_INVALID_ARG;
    int n = 0;
    tcbf_plan_num_configs(plan, &n);
    if (config < 0 || config >= n) return TCBF_ERR_INVALID_ARG;
    if (plan->p.mode != TCBF_MODE_1BIT &&
        !(plan->p.flags & (TCBF_FLAG_STACKED_X | TCBF_FLAG_INTERLEAVED_X |
                           TCBF_FLAG_FP8_BLOCK_SCALES)) &&
        !gemm_f16_config_valid(config, plan->p.K))
        return TCBF_ERR_INVALID_ARG;
    if ((plan->p.flags & TCBF_FLAG_INTERLEAVED_X) && !gemm_f16_ix_config_valid(config, plan->p.K))
        return TCBF_ERR_INVALID_ARG;
    if (plan->p.mode == TCBF_MODE_1BIT && gemm_1bit_config_fp4(config)) {
        // the E2M1 planes live in the plan; plans the path cannot take
        // (uneven batches, K > 2^23) run configuration 0 instead
        DeviceGuard g(plan->device);
        if (!g.ok()) return TCBF_ERR_CUDA;
        if (gemm_1bit_fp4_reserve(*plan) != cudaSuccess) return TCBF_ERR_OOM;
    }
    plan->config = config;   // a captured graph keeps the configuration it was captured with
    return TCBF_OK;
}

TCBF_EXPORT const char *tcbf_config_name(tcbf_plan_t plan, int config) {
    if (!plan) return "invalid";
    if (plan->p.flags & TCBF_FLAG_STACKED_X) return gemm_f16_stacked_config_name(config);
    if (plan->p.flags & TCBF_FLAG_INTERLEAVED_X) return gemm_f16_ix_config_name(config);
    if (plan->p.mode == TCBF_MODE_FP16) return gemm_f16_config_name(config);
    if (plan->p.mode == TCBF_MODE_1BIT) return gemm_1bit_config_name(config);
    if (plan->p.mode == TCBF_MODE_TF32) return gemm_tf32_config_name(config);
    if (fp8_block_scaled(plan->p.flags)) return gemm_split8_blk_config_name(config);
    return gemm_split8_config_name(config);
}

// ---------------------------------------------------------------------------
// Uneven batches, autotuning and graph capture.
// ---------------------------------------------------------------------------
namespace {

cudaError_t launch_beamform(const tcbf_plan_s &pl, const void *Wp, const void *Xp, void *Y,
                            cudaStream_t s) {
    if (pl.p.mode == TCBF_MODE_FP16)
        return launch_gemm_f16(pl, Wp, Xp, static_cast<float *>(Y), s);
    if (pl.p.mode == TCBF_MODE_1BIT)
        return launch_gemm_1bit(pl, static_cast<const uint32_t *>(Wp),
                                static_cast<const uint32_t *>(Xp), static_cast<int32_t *>(Y), s);
    if (pl.p.mode == TCBF_MODE_TF32) return launch_gemm_tf32(pl, Wp, Xp, static_cast<float *>(Y), s);
    return launch_gemm_split8(pl, Wp, Xp, static_cast<float *>(Y), s);
}

cudaError_t launch_pack_x(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                          cudaStream_t s) {
    if (pl.p.mode == TCBF_MODE_FP16)
        return interleaved_x(pl) ? launch_copy_x_cf16(pl, src_type, src, dst, s)
                                 : launch_pack_f16_x(pl, src_type, src, dst, s);
    if (pl.p.mode == TCBF_MODE_1BIT) return launch_pack_bits_x(pl, src_type, src, dst, s);
    if (pl.p.mode == TCBF_MODE_TF32) return launch_pack_tf32_x(pl, src_type, src, dst, s);
    return launch_pack_split8_x(pl, src_type, src, dst, s);
}

bool config_ok(const tcbf_plan_s &pl, int c) {
    if (pl.p.mode == TCBF_MODE_1BIT)
        return c >= 0 && c < gemm_1bit_num_configs() &&
               (!gemm_1bit_config_fp4(c) || gemm_1bit_fp4_usable(pl));
    if (pl.p.flags & TCBF_FLAG_STACKED_X) return c >= 0 && c < gemm_f16_stacked_num_configs();
    if (pl.p.flags & TCBF_FLAG_INTERLEAVED_X) return gemm_f16_ix_config_valid(c, pl.p.K);
    if (fp8_block_scaled(pl.p.flags)) return c >= 0 && c < gemm_split8_blk_num_configs();
    return gemm_f16_config_valid(c, pl.p.K);
}

}  // namespace

TCBF_EXPORT tcbf_status tcbf_plan_set_batch_rows(tcbf_plan_t plan, const int64_t *rows) {
    if (!plan) return TCBF_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    if (!rows) {
        if (plan->m_prefix) cudaFree(plan->m_prefix);
        plan->m_prefix = nullptr;
        plan->m_tiles_sum = 0;
        return TCBF_OK;
    }
    const int64_t B = plan->p.batch;
    int *host = new (std::nothrow) int[B + 1];
    if (!host) return TCBF_ERR_OOM;
    int64_t acc = 0;
    host[0] = 0;
    for (int64_t b = 0; b < B; ++b) {
        if (rows[b] < 1 || rows[b] > plan->p.M) {
            delete[] host;
            return TCBF_ERR_INVALID_ARG;
        }
        acc += ceil_div(rows[b], 128);
        if (acc > 0x3fffffff) {
            delete[] host;
            return TCBF_ERR_UNSUPPORTED;
        }
        host[b + 1] = static_cast<int>(acc);
    }
    if (!plan->m_prefix && cudaMalloc(&plan->m_prefix, sizeof(int) * (B + 1)) != cudaSuccess) {
        plan->m_prefix = nullptr;
        delete[] host;
        return TCBF_ERR_OOM;
    }
    const cudaError_t e =
        cudaMemcpy(plan->m_prefix, host, sizeof(int) * (B + 1), cudaMemcpyHostToDevice);
    delete[] host;
    if (e != cudaSuccess) return TCBF_ERR_CUDA;
    // interleaved X with uneven rows runs pack + planar kernel through plan-owned planes
    if (interleaved_x(*plan) && !plan->ix_planes && alloc_ix_planes(*plan) != cudaSuccess)
        return TCBF_ERR_OOM;
    plan->m_tiles_sum = acc;
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_autotune(tcbf_plan_t plan, const void *Wp, const void *Xp, void *Y,
                                      int reps, tcbf_stream_t stream, int *best,
                                      float *ms_per_config) {
    if (!plan || !Wp || !Xp || !Y || reps < 1) return TCBF_ERR_INVALID_ARG;
    if (!aligned16(Wp) || !aligned16(Xp) || !aligned16(Y)) return TCBF_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    plan->debug_drop_fill = -1;
    int n = 0;
    tcbf_plan_num_configs(plan, &n);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return TCBF_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return TCBF_ERR_CUDA;
    }
    const int saved = plan->config;
    tcbf_status st = TCBF_OK;
    // 1-bit: the 4-bit configurations need the plan's E2M1 scratch; without
    // device memory for it they are left out
    if (plan->p.mode == TCBF_MODE_1BIT && !plan->m_prefix)
        for (int c = 0; c < n; ++c)
            if (gemm_1bit_config_fp4(c)) {
                gemm_1bit_fp4_reserve(*plan);
                break;
            }
    // Every valid configuration is warmed up and sized into groups of launches
    // of at least 0.2 ms; then the configurations are timed round-robin, `reps`
    // rounds, keeping each one's fastest group.  Interleaving the rounds keeps
    // a slow drift of the clocks (power, temperature) from favouring whichever
    // configuration happened to run first.
    std::vector<int> group(static_cast<size_t>(n), 0);
    std::vector<float> best_ms(static_cast<size_t>(n), -1.f);
    auto timed = [&](int c, int launches, float &ms) -> cudaError_t {
        plan->config = c;
        cudaError_t e = cudaEventRecord(e0, s);
        for (int r = 0; r < launches && e == cudaSuccess; ++r) e = launch_beamform(*plan, Wp, Xp, Y, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        return e;
    };
    for (int c = 0; c < n && st == TCBF_OK; ++c) {
        if (!config_ok(*plan, c)) continue;
        float ms = 0.f;
        cudaError_t e = timed(c, 1, ms);                               // warm-up
        if (e == cudaSuccess) e = timed(c, 1, ms);
        if (e != cudaSuccess) {
            st = from_cuda(e);
            break;
        }
        group[c] = std::max(1, std::min(1000, static_cast<int>(0.2f / std::max(ms, 1e-4f)) + 1));
    }
    for (int r = 0; r < reps && st == TCBF_OK; ++r)
        for (int c = 0; c < n && st == TCBF_OK; ++c) {
            if (group[c] == 0) continue;
            float ms = 0.f;
            const cudaError_t e = timed(c, group[c], ms);
            if (e != cudaSuccess) {
                st = from_cuda(e);
                break;
            }
            ms /= group[c];
            if (best_ms[c] < 0.f || ms < best_ms[c]) best_ms[c] = ms;
        }
    int best_c = -1;
    for (int c = 0; c < n; ++c) {
        if (ms_per_config) ms_per_config[c] = best_ms[c];
        if (best_ms[c] >= 0.f && (best_c < 0 || best_ms[c] < best_ms[best_c])) best_c = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    plan->config = (st == TCBF_OK && best_c >= 0) ? best_c : saved;
    if (best) *best = plan->config;
    return st;
}

TCBF_EXPORT tcbf_status tcbf_autotune_layout(tcbf_plan_t plan, const void *Wp, const void *X_src,
                                             int src_type, void *Y, int reps, tcbf_stream_t stream,
                                             uint32_t *flags, float *ms_per_layout) {
    if (!plan || !Wp || !X_src || !Y || reps < 1) return TCBF_ERR_INVALID_ARG;
    if (!plan->auto_layout) return TCBF_ERR_INVALID_ARG;
    if (src_type != TCBF_SRC_CF16 && src_type != TCBF_SRC_CF32) return TCBF_ERR_INVALID_ARG;
    if (!aligned16(Wp) || !aligned16(X_src) || !aligned16(Y)) return TCBF_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t base = plan->p.flags & ~(TCBF_FLAG_STACKED_X | TCBF_FLAG_INTERLEAVED_X);
    const uint32_t old_flags = plan->p.flags;
    const int old_config = plan->config;
    const uint32_t layouts[3] = {0u, TCBF_FLAG_STACKED_X, TCBF_FLAG_INTERLEAVED_X};
    // the interleaved layout only where the fused kernel takes it
    plan->p.flags = base | TCBF_FLAG_INTERLEAVED_X;
    const int n_layouts = ix_fused_ok(*plan) ? 3 : 2;
    // one scratch for the packed X of any layout (the stacked one is the largest)
    plan->p.flags = base | TCBF_FLAG_STACKED_X;
    size_t xbytes = 0;
    tcbf_packed_size(plan, 1, &xbytes);
    void *xp = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaMalloc(&xp, xbytes);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    tcbf_status st = from_cuda(ce);
    float ms[3] = {-1.f, -1.f, -1.f};
    int cfg[3] = {0, 0, 0};
    // each layout: its configurations autotuned on the packed X, then the
    // step (pack + beamform with the best configuration; for the interleaved
    // layout the pack is tcbf_transpose_pack's copy) timed, best of reps
    for (int l = 0; l < n_layouts && st == TCBF_OK; ++l) {
        plan->p.flags = base | layouts[l];
        plan->config = 0;
        ce = pack_x_into(*plan, src_type, X_src, xp, s);
        st = from_cuda(ce);
        if (st == TCBF_OK) st = tcbf_autotune(plan, Wp, xp, Y, reps, stream, &cfg[l], nullptr);
    }
    // then the steps of the layouts timed round-robin, each in groups of at
    // least about 1 ms after a warm-up step, keeping each one's fastest
    // group: a drift of the clocks (power, temperature) affects them alike
    int group[3] = {1, 1, 1};
    auto timed = [&](int l, int steps, float &t) -> cudaError_t {
        plan->p.flags = base | layouts[l];
        plan->config = cfg[l];
        cudaError_t e = cudaEventRecord(e0, s);
        for (int i = 0; i < steps && e == cudaSuccess; ++i) {
            e = pack_x_into(*plan, src_type, X_src, xp, s);
            if (e == cudaSuccess) e = launch_beamform(*plan, Wp, xp, Y, s);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        return e;
    };
    for (int l = 0; l < n_layouts && st == TCBF_OK; ++l) {
        float t = 0.f;
        st = from_cuda(timed(l, 1, t));
        if (st == TCBF_OK) st = from_cuda(timed(l, 1, t));
        group[l] = std::max(1, std::min(1000, static_cast<int>(1.0f / std::max(t, 1e-4f)) + 1));
    }
    for (int r = 0; r < reps && st == TCBF_OK; ++r)
        for (int l = 0; l < n_layouts && st == TCBF_OK; ++l) {
            float t = 0.f;
            st = from_cuda(timed(l, group[l], t));
            t /= group[l];
            if (st == TCBF_OK && (ms[l] < 0.f || t < ms[l])) ms[l] = t;
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (xp) cudaFree(xp);
    if (st != TCBF_OK) {
        plan->p.flags = old_flags;
        plan->config = old_config;
        return st;
    }
    int best = 0;
    for (int l = 1; l < n_layouts; ++l)
        if (ms[l] >= 0.f && ms[l] < ms[best]) best = l;
    plan->p.flags = base | layouts[best];
    plan->config = cfg[best];
    if (plan->p.flags != old_flags) {
        // staging and a captured step sized for the old layout
        host_pipe_destroy(*plan);
        if (plan->graph_exec) {
            cudaGraphExecDestroy(plan->graph_exec);
            plan->graph_exec = nullptr;
        }
    }
    if (flags) *flags = plan->p.flags;
    if (ms_per_layout)
        for (int l = 0; l < 3; ++l) ms_per_layout[l] = ms[l];
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_graph_capture(tcbf_plan_t plan, const void *X_src, int src_type,
                                           void *Xp, const void *Wp, void *Y) {
    if (!plan || !Xp || !Wp || !Y) return TCBF_ERR_INVALID_ARG;
    if (X_src && src_type != TCBF_SRC_CF16 && src_type != TCBF_SRC_CF32) return TCBF_ERR_INVALID_ARG;
    if ((X_src && !aligned16(X_src)) || !aligned16(Xp) || !aligned16(Wp) || !aligned16(Y))
        return TCBF_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    plan->debug_drop_fill = -1;
    if (plan->graph_exec) {
        cudaGraphExecDestroy(plan->graph_exec);
        plan->graph_exec = nullptr;
    }
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return TCBF_ERR_CUDA;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    cudaError_t le = cudaSuccess;
    if (e == cudaSuccess) {
        if (X_src) le = launch_pack_x(*plan, src_type, X_src, Xp, cs);
        if (le == cudaSuccess) le = launch_beamform(*plan, Wp, Xp, Y, cs);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess && le == cudaSuccess)
            e = cudaGraphInstantiate(&plan->graph_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
    }
    cudaStreamDestroy(cs);
    if (le != cudaSuccess) e = le;
    if (e != cudaSuccess) {
        plan->graph_exec = nullptr;
        return from_cuda(e);
    }
    return TCBF_OK;
}

TCBF_EXPORT tcbf_status tcbf_graph_launch(tcbf_plan_t plan, tcbf_stream_t stream) {
    if (!plan || !plan->graph_exec) return TCBF_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    if (!g.ok()) return TCBF_ERR_CUDA;
    return from_cuda(cudaGraphLaunch(plan->graph_exec, static_cast<cudaStream_t>(stream)));
}
