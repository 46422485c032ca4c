// tcbf_internal.h — host-side plan state and kernel launchers shared by
// the library's translation units (not part of the public ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/tcbf.h"

#define TCBF_EXPORT extern "C" __attribute__((visibility("default")))

struct tcbf_plan_s {
    tcbf_problem p;          // validated copy; w_batches filled in
    int device = 0;
    int num_sms = 0;
    int64_t per_w = 1;       // batch / w_batches
    int64_t Kp = 0;          // packed_row_k(K): FP16 / TF32 row length, elements
    int64_t Kw = 0;          // 1-bit row length in 32-bit words (multiple of 4)
    int64_t Kb2 = 0;         // FP8 row length in bytes (fp8_row_bytes)
    int config = 0;          // kernel configuration (tile shape) in use
    uint32_t *status = nullptr;   // device status word (256 bytes)
    // uneven batches: per-batch row counts and the device m-tile prefix
    int *m_prefix = nullptr;      // device [batch + 1], nullptr when all batches have M rows
    int64_t m_tiles_sum = 0;
    // captured step (tcbf_graph_capture)
    cudaGraphExec_t graph_exec = nullptr;
    // split-FP8 W scale exponents when Wp is a sub-range of a larger packed W
    // (chunks of tcbf_beamform_host); nullptr: they follow Wp's planes
    const int32_t *w_exps = nullptr;
    // staging, streams and events of tcbf_beamform_host, made at its first call
    struct tcbf_host_pipe *pipe = nullptr;
    // tcbf_debug_drop_fill: operand load left out by the next GEMM launch (-1: none)
    int64_t debug_drop_fill = -1;
    // rows between the planes of packed W (0: M).  Row-range sub-plans of
    // tcbf_beamform_host point into a larger packed W.
    int64_t w_rows = 0;
    // 1-bit plans on the 4-bit tensor path: E2M1 planes of W and X, made
    // when such a configuration is first set (nullptr until then)
    void *fp4_buf = nullptr;
    size_t fp4_bytes = 0;
    // plans with TCBF_FLAG_INTERLEAVED_X that the fused kernel cannot take
    // (N % 4 != 0, uneven batch rows): packed X planes the beamform call
    // packs into before running the planar kernel (nullptr otherwise)
    void *ix_planes = nullptr;
    // created with TCBF_FLAG_AUTO_LAYOUT: tcbf_autotune_layout may change
    // the packed-X layout
    bool auto_layout = false;
    // FP16 plans that may run the stacked SM-pair kernel with promoted long
    // K: partial chunk sums of the tiles of a split last wave (nullptr: no
    // split, the tiles run whole)
    void *tail_ws = nullptr;
    size_t tail_ws_bytes = 0;
};

namespace tcbf {

constexpr int kNumSmsGb300 = 152;

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Row length (elements) of the FP16 and TF32 packed planes: K rounded up to
// 64, so every row starts on a 128-byte line and each 128-byte box row that
// the GEMMs' tensor loads fetch (64 FP16 or 32 TF32 elements) is one whole
// line.  With rows of K rounded up to 8 only, a box row straddled two lines
// whenever K % 64 != 0 and the compute-bound kernels ran 20-27% slower.
inline int64_t packed_row_k(int64_t K) { return round_up(K, 64); }

// cuTensorMapEncodeTiled fetched from the driver at first use.
CUresult encode_tiled(CUtensorMap *map, CUtensorMapDataType type, uint32_t rank, void *gaddr,
                      const uint64_t *dims, const uint64_t *strides_bytes, const uint32_t *box,
                      CUtensorMapSwizzle swizzle);

// Launchers (return a cudaError_t from the launch).
cudaError_t launch_pack_f16_w(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                              cudaStream_t s);
cudaError_t launch_pack_f16_x(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                              cudaStream_t s);
cudaError_t launch_pack_bits_w(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                               cudaStream_t s);
cudaError_t launch_pack_bits_x(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                               cudaStream_t s);

// TF32 planes (FP32 storage, values rounded to TF32).
cudaError_t launch_pack_tf32_w(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                               cudaStream_t s);
cudaError_t launch_pack_tf32_x(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                               cudaStream_t s);
cudaError_t launch_gemm_tf32(const tcbf_plan_s &pl, const void *Wp, const void *Xp, float *Y,
                             cudaStream_t s);
const char *gemm_tf32_config_name(int config);    // TF32 uses the FP16 tile table

// 1-bit planes back to interleaved complex +-1 values (FP16 or FP32).
cudaError_t launch_unpack_bits(const tcbf_plan_s &pl, int which, const uint32_t *src, int dst_type,
                               void *dst, cudaStream_t s);

cudaError_t launch_pack_split8_w(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                                 cudaStream_t s);
cudaError_t launch_pack_split8_x(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                                 cudaStream_t s);
cudaError_t launch_gemm_split8(const tcbf_plan_s &pl, const void *Wp, const void *Xp, float *Y,
                               cudaStream_t s);

int gemm_f16_num_configs();
const char *gemm_f16_config_name(int config);
bool gemm_f16_config_valid(int config, int64_t K);
const char *gemm_split8_config_name(int config);   // split-FP8 uses the FP16 tile table
// Block-scaled split-FP8 (TCBF_FLAG_FP8_BLOCK_SCALES) has its own table.
int gemm_split8_blk_num_configs();
const char *gemm_split8_blk_config_name(int config);
cudaError_t launch_gemm_f16(const tcbf_plan_s &pl, const void *Wp, const void *Xp, float *Y,
                            cudaStream_t s);

// Stacked-plane FP16 GEMM (plans with TCBF_FLAG_STACKED_X).
int gemm_f16_stacked_num_configs();
const char *gemm_f16_stacked_config_name(int config);
// Workspace the stacked SM-pair kernel needs to split the plan's last wave
// of tiles (0: it runs them whole).
size_t stacked_tail_ws_bytes(const tcbf_plan_s &pl);
cudaError_t launch_gemm_f16_stacked(const tcbf_plan_s &pl, const void *Wp, const void *Xp, float *Y,
                                    cudaStream_t s);

// FP16 GEMM on interleaved complex X (plans with TCBF_FLAG_INTERLEAVED_X).
int gemm_f16_ix_num_configs();
const char *gemm_f16_ix_config_name(int config);
// Configuration 0 (resident weights) needs K <= 384; the default is it there,
// else the streaming SM-pair configuration.
bool gemm_f16_ix_config_valid(int config, int64_t K);
int gemm_f16_ix_default_config(int64_t K);
cudaError_t launch_gemm_f16_ix(const tcbf_plan_s &pl, const void *Wp, const void *X, float *Y,
                               cudaStream_t s);
inline bool interleaved_x(const tcbf_plan_s &pl) {
    return (pl.p.flags & TCBF_FLAG_INTERLEAVED_X) != 0;
}
// Whether the fused interleaved-X kernel can take the plan (else it runs
// pack + planar kernel through ix_planes).
inline bool ix_fused_ok(const tcbf_plan_s &pl) { return pl.p.N % 4 == 0 && !pl.m_prefix; }
// X of an interleaved plan from a source of either type: an FP16 source is
// copied (nothing when src == dst), an FP32 source rounded to FP16.
cudaError_t launch_copy_x_cf16(const tcbf_plan_s &pl, int src_type, const void *src, void *dst,
                               cudaStream_t s);

// Split-FP8 products per 32-K step: 1 (plain FP8), 3 (hi+lo split) or 4.
inline int split_products(const tcbf_plan_s &pl) {
    if (pl.p.flags & TCBF_FLAG_FP8_HI_ONLY) return 1;
    if (pl.p.flags & TCBF_FLAG_FP8_FOUR_PRODUCTS) return 4;
    return 3;
}

// FP8 packed rows hold K in 64-element blocks: 64 E4M3 hi bytes, then 64
// lo bytes unless the plan keeps the hi product only (TCBF_FLAG_FP8_HI_ONLY:
// one byte per element, hi byte k at offset k).
inline bool fp8_hi_only(uint32_t flags) { return (flags & TCBF_FLAG_FP8_HI_ONLY) != 0; }
inline int64_t fp8_block_bytes(uint32_t flags) { return fp8_hi_only(flags) ? 64 : 128; }
inline int64_t fp8_row_bytes(int64_t K, uint32_t flags) {
    return round_up(K, 64) / 64 * fp8_block_bytes(flags);
}

// Block-scaled FP8 (TCBF_FLAG_FP8_BLOCK_SCALES): UE8M0 codes per 32 k in
// 512-byte tiles of 128 W rows or 64 X samples per stage of
// fp8blk_stage_k(flags) k, after the packed bytes.
inline bool fp8_block_scaled(uint32_t flags) { return (flags & TCBF_FLAG_FP8_BLOCK_SCALES) != 0; }
constexpr int kFp8BlkTile = 512;
constexpr int kFp8BlkRowsW = 128;
constexpr int kFp8BlkRowsX = 64;
inline int64_t fp8blk_stage_k(uint32_t flags) { return fp8_hi_only(flags) ? 128 : 64; }
inline int64_t fp8blk_stages(int64_t K, uint32_t flags) {
    return (K + fp8blk_stage_k(flags) - 1) / fp8blk_stage_k(flags);
}
// Bytes of the scale tiles of operand `which` (0: W, 1: X) of nb batches.
inline int64_t fp8blk_sf_bytes(int64_t nb, int64_t rows, int64_t K, uint32_t flags, int which) {
    const int64_t per = which == 0 ? kFp8BlkRowsW : kFp8BlkRowsX;
    return nb * ((rows + per - 1) / per) * fp8blk_stages(K, flags) * kFp8BlkTile;
}

// Rows between the planes of the packed W a GEMM launch reads.
inline int64_t w_plane_rows(const tcbf_plan_s &pl) { return pl.w_rows ? pl.w_rows : pl.p.M; }

// Planes of packed FP16 X: 3 with TCBF_FLAG_STACKED_X, else 2.
inline int64_t x_planes(const tcbf_plan_s &pl) {
    return (pl.p.flags & TCBF_FLAG_STACKED_X) ? 3 : 2;
}

int gemm_1bit_num_configs();
const char *gemm_1bit_config_name(int config);
cudaError_t launch_gemm_1bit(const tcbf_plan_s &pl, const uint32_t *Wb, const uint32_t *Xb,
                             int32_t *Y, cudaStream_t s);
// Configurations of the 1-bit table that run on the 4-bit tensor path.
bool gemm_1bit_config_fp4(int config);

// 1-bit GEMM on the 4-bit tensor path (gemm_1bit_fp4.cu): device scratch for
// the E2M1 planes (reserve: allocate once per plan; release: free), whether
// a plan can take the path (scratch present, K <= 2^23, no uneven batches),
// and the launch (variant 0: 256 x 128 pair tiles, one accumulator;
// 1: 256 x 64, two; 2: 256 x 96, two; 3: 256 x 112, two).  cudaErrorNotSupported when the
// plan cannot take it.
size_t gemm_1bit_fp4_scratch_bytes(const tcbf_plan_s &pl);
cudaError_t gemm_1bit_fp4_reserve(tcbf_plan_s &pl);
void gemm_1bit_fp4_release(tcbf_plan_s &pl);
bool gemm_1bit_fp4_usable(const tcbf_plan_s &pl);
cudaError_t launch_gemm_1bit_fp4(const tcbf_plan_s &pl, const uint32_t *Wb, const uint32_t *Xb,
                                 int32_t *Y, cudaStream_t s, int variant);
// Its two halves: expansion of one operand (which 0: W, 1: X) into the
// scratch, and the GEMM on the planes there.
cudaError_t launch_expand_1bit_fp4(const tcbf_plan_s &pl, int which, const uint32_t *bits,
                                   cudaStream_t s);
cudaError_t launch_gemm_1bit_fp4_expanded(const tcbf_plan_s &pl, int32_t *Y, cudaStream_t s,
                                          int variant);
// Sign quantisation of interleaved complex W (which 0) or X (which 1)
// straight into the E2M1 planes, without the packed bits.
cudaError_t launch_pack_1bit_fp4(const tcbf_plan_s &pl, int which, int src_type, const void *src,
                                 cudaStream_t s);
// Variant (0-2) of a 4-bit configuration of the 1-bit table, -1 otherwise.
int gemm_1bit_fp4_variant(int config);
// The configuration a 1-bit plan starts with when it can take the 4-bit path.
int gemm_1bit_fp4_default_config(int64_t K);

// Releases the staging of tcbf_beamform_host (plan destruction).
void host_pipe_destroy(tcbf_plan_s &pl);

cudaError_t launch_weights(const tcbf_plan_s &pl, const double *rx, const double *tg,
                           int near_field, const double *freqs, double c, void *Wp,
                           cudaStream_t s);

}  // namespace tcbf
