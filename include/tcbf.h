/*
 * tcbf.h — C ABI of the GB300 tensor-core beamformer.
 *
 * Beamforming of many samples at once is the complex matrix product
 * Y = W X (Sec. II, Eq. 3): W holds the steering weights (M beams x K
 * receivers), X the sensor samples (K receivers x N samples), Y the beams
 * (M x N).  A problem is a batch of such products (Sec. III: "batch size
 * option"; Sec. V-B: batch = polarisations x channels).  As in Sec. III the
 * caller supplies inputs, outputs and their shapes; the library chooses
 * kernels and tile shapes.
 *
 * Conventions that hold for every call:
 *  - All buffers are owned by the caller.  Unless stated otherwise a pointer
 *    argument is DEVICE memory of the plan's device, 256-byte aligned (any
 *    torch/cudaMalloc allocation is).  The plan owns host state, a small
 *    device status word and the device scratch some configurations need,
 *    which it allocates itself: the E2M1 planes of 1-bit plans on the 4-bit
 *    path, the planes an interleaved-X plan packs into when the fused kernel
 *    cannot read X, and the chunk sums of a stacked-X FP16 plan whose last
 *    partial wave of tiles is split (K > 4096; at most 64 MiB).  Calls on
 *    one plan share these and must not overlap on the GPU.
 *  - Calls that take a stream are asynchronous and stream-ordered; argument
 *    errors are returned synchronously and nothing is launched.  Errors that
 *    only the device can see (a bounded wait that ran out) are recorded in
 *    the plan's status word and read by tcbf_last_device_error().
 *  - No call aborts, exits or traps.
 *  - Complex values are interleaved (re, im) unless stated otherwise; all
 *    matrices are row-major and batches are contiguous.
 *  - Shapes are any value >= 1; padding is internal.
 *  - Throughput is counted as 8*batch*M*N*K useful operations (Sec. IV-A).
 */
#ifndef TCBF_H
#define TCBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tcbf_plan_s *tcbf_plan_t;
/* A cudaStream_t passed as an opaque handle; NULL is the legacy default stream. */
typedef void *tcbf_stream_t;

typedef enum {
    TCBF_OK = 0,
    TCBF_ERR_INVALID_ARG = 1,  /* null/misaligned pointer, bad shape, wrong mode for this call */
    TCBF_ERR_UNSUPPORTED = 2,  /* no GPU, not sm_103, or a shape beyond the library limits */
    TCBF_ERR_OOM = 3,          /* the plan's small device allocation failed */
    TCBF_ERR_BUDGET = 4,       /* serving admission: request exceeds the memory budget */
    TCBF_ERR_CUDA = 5,         /* a CUDA runtime/driver call failed */
    TCBF_ERR_TIMEOUT = 6,      /* a device-side bounded wait ran out (see tcbf_last_device_error) */
    TCBF_ERR_DEVICE = 7        /* another device-side check failed */
} tcbf_status;

typedef enum {
    TCBF_MODE_FP16 = 0,        /* FP16 planar re/im inputs, FP32 accumulate (Sec. III) */
    TCBF_MODE_FP8SPLIT = 1,    /* e4m3 hi+lo split of each operand, FP32 accumulate (FP8: Sec. VI) */
    TCBF_MODE_1BIT = 2,        /* +-1+-i values, one bit per component, exact int32 (Sec. III-D) */
    TCBF_MODE_TF32 = 3         /* FP32 planar inputs rounded to TF32, FP32 accumulate (formats
                                  beyond 16 bits: Sec. VI) */
} tcbf_mode;

/* Source element types accepted by tcbf_transpose_pack. */
typedef enum {
    TCBF_SRC_CF16 = 0,         /* interleaved complex FP16: 4 bytes per value */
    TCBF_SRC_CF32 = 1          /* interleaved complex FP32: 8 bytes per value, rounded RN to FP16 */
} tcbf_src_type;

typedef struct {
    int64_t batch;      /* number of independent products in the problem (>= 1) */
    int64_t M;          /* beams (rows of W and Y) */
    int64_t N;          /* samples (columns of X and Y) */
    int64_t K;          /* receivers (summed over) */
    int64_t w_batches;  /* distinct weight matrices; batch b uses W[b / (batch / w_batches)].
                           0 means batch. Must divide batch. */
    int32_t mode;       /* tcbf_mode */
    uint32_t flags;     /* tcbf_flag bits; others reserved, must be 0 */
} tcbf_problem;

/* Problem flags. */
typedef enum {
    /* FP16 only: packed X carries a third, negated plane ([-Xi, Xr, Xi],
     * see the layouts below) so that the GEMM issues the complex product of
     * Sec. III-B as two N = 256 MMAs per K step (Wr [Xr; Xi] + Wi [-Xi; Xr]
     * = [Re | Im]) instead of four N = 128 ones.  For compute-bound shapes
     * (large K and M, small N); it costs 1.5 x the packed X bytes.  Selects
     * the stacked kernel configurations. */
    TCBF_FLAG_STACKED_X = 1u,
    /* FP8-split only: the number of E4M3 products per complex K step.  By
     * default three (Wh Xh + Wh Xl + Wl Xh, the hi+lo split that wins back
     * accuracy); TCBF_FLAG_FP8_HI_ONLY keeps only Wh Xh, the plain E4M3
     * product with the same per-row power-of-two scales (a third of the MMA
     * work, E4M3 accuracy: a few percent on Gaussian data) and packs one
     * byte per element (the hi bytes alone, see the layouts below);
     * TCBF_FLAG_FP8_FOUR_PRODUCTS adds Wl Xl on the hi+lo layout.  The paper
     * names 8-bit floats only as future work (Sec. VI). */
    TCBF_FLAG_FP8_HI_ONLY = 2u,
    TCBF_FLAG_FP8_FOUR_PRODUCTS = 4u,
    /* FP16 only: the beamform call reads X in the caller's interleaved
     * complex layout, [batch][K][N] binary16 (the source layout of
     * tcbf_transpose_pack), with no transpose/pack pass (the paper's
     * future-work item of skipping the transpose, Sec. VI).  The GEMM loads
     * X as an MN-major tensor-core operand, issues one real MMA per K step
     * that forms Wr X and Wi X side by side, and combines them into Re and
     * Im in FP32 before the store.  Packed W is the FP16 layout below.  For
     * such a plan tcbf_packed_size(1) is batch*K*N*4 bytes and
     * tcbf_transpose_pack(which = 1) only copies (FP16 source) or rounds
     * (FP32 source) into that layout.  Needs N % 4 == 0 for the fused
     * kernel; other N, and uneven batch rows, run the transpose/pack into
     * plan-owned planes and the planar kernel inside the beamform call.
     * Not combined with TCBF_FLAG_STACKED_X.  Selects the interleaved-X
     * kernel configurations. */
    TCBF_FLAG_INTERLEAVED_X = 8u,
    /* FP8-split only (with or without TCBF_FLAG_FP8_HI_ONLY /
     * _FOUR_PRODUCTS): the scale is per 32 consecutive k of each W row and
     * each X sample instead of per row: e is the largest integer with
     * amax * 2^e <= 448 over the block's 32 k of both planes, hi =
     * RN_e4m3(v 2^e) and lo = RN_e4m3(16 (v 2^e - hi)) (lo kept 16 times
     * larger, its scale 2^-(e + 4), so it keeps E4M3's precision).  The
     * tensor cores apply the scales themselves (block-scaled E4M3 MMAs,
     * kind::mxf8f6f4 with UE8M0 scales).  The scales follow the packed
     * bytes as 512-byte tiles, see the layouts below.  The paper's future
     * work on 8-bit floats (Sec. VI); the benchmark spec's per-tile scales. */
    TCBF_FLAG_FP8_BLOCK_SCALES = 16u,
    /* FP16 only, not combined with TCBF_FLAG_STACKED_X or
     * TCBF_FLAG_INTERLEAVED_X: the plan chooses the packed-X layout.  At
     * creation it takes TCBF_FLAG_STACKED_X
     * when the problem is compute-bound: its arithmetic intensity, 8 B M N K
     * operations over the bytes of the stacked layout's packed W and X and
     * of Y, is at least TCBF_AUTO_STACKED_MIN_INTENSITY operations per byte
     * (above the GB300's tensor/HBM ridge of about 280, where the stacked
     * kernel's two N = 256 MMAs per K step tend to beat the four N = 128
     * ones), and the planar layout otherwise; tcbf_autotune_layout then
     * replaces that guess by measurement over the planar, stacked and
     * interleaved layouts.  The chosen bit replaces this one
     * in the plan's flags (tcbf_plan_flags): callers that write packed X
     * themselves read it there; tcbf_transpose_pack and tcbf_packed_size
     * follow it. */
    TCBF_FLAG_AUTO_LAYOUT = 32u
} tcbf_flag;

/* The intensity (operations per byte) from which TCBF_FLAG_AUTO_LAYOUT
 * starts a plan on the stacked layout. */
#define TCBF_AUTO_STACKED_MIN_INTENSITY 400

/*
 * Packed operand layouts (produced by tcbf_transpose_pack or
 * tcbf_weights_from_geometry, consumed by tcbf_beamform_*).  The GEMM
 * needs its inputs split into real and imaginary planes (Sec. VI) and tiled
 * in device memory (Sec. III); here both operands are stored K-contiguous:
 *   FP16 W : [w_batches][2][M][Kp] binary16, Kp = K rounded up to 64 (rows of
 *            whole 128-byte lines), zero pad
 *   FP16 X : [batch][2][N][Kp]     binary16 (X transposed: samples are rows);
 *            with TCBF_FLAG_STACKED_X [batch][3][N][Kp], planes -Xi, Xr, Xi
 *            (-Xi: the Xi plane with every sign bit flipped, its pad -0.0);
 *            with TCBF_FLAG_INTERLEAVED_X [batch][K][N] interleaved complex
 *            binary16 (not transposed, no padding)
 *   1-bit W: [w_batches][2][M][Kw] uint32,   Kw = 4 * ceil(K / 128)
 *   1-bit X: [batch][2][N][Kw]     uint32
 * Plane 0 is the real part, plane 1 the imaginary part.  1-bit element k
 * of a row is bit (k % 32) of word (k / 32); bit 1 is +1, bit 0 is -1
 * (Fig. 1).  Bits at k >= K are ignored by the GEMM.
 *   FP8-split W: [w_batches][2][M][Kb2] bytes, X: [batch][2][N][Kb2] bytes,
 *   Kb2 = 2 * (K rounded up to 64): each row holds K in blocks of 64
 *   elements, 64 E4M3 "hi" bytes followed by 64 E4M3 "lo" bytes.  After the
 *   bytes come int32 scale exponents, one per row ([w_batches][M] or
 *   [batch][N], shared by both planes): e is the largest integer with
 *   amax * 2^e <= 448 (amax over the row's K elements of both planes, after
 *   rounding to FP16), hi = RN_e4m3(v 2^e), lo = RN_e4m3(v 2^e - hi), both
 *   saturating, so v ~ (hi + lo) 2^-e.  tcbf_packed_size includes the
 *   exponents.  With TCBF_FLAG_FP8_HI_ONLY the rows hold the hi bytes alone,
 *   Kb2 = K rounded up to 64 (hi byte of element k at offset k), followed by
 *   the same exponents.
 *   With TCBF_FLAG_FP8_BLOCK_SCALES the bytes are as above and the scales
 *   follow them as UE8M0 codes (127 - e for hi, 123 - e for lo) in tiles of
 *   512 bytes, one per (operand batch, row tile, stage of S k), S = 64
 *   (hi+lo rows) or 128 (hi only), T = ceil(K / S) stages:
 *     W: [w_batches][ceil(M / 128)][T][32][4][4] bytes, byte [l][g][j] the
 *        code of row 128 t + 32 g + l;
 *     X: [batch][ceil(N / 64)][T][32][4][4] bytes, byte [l][g][j] the code
 *        of sample 64 t + 32 g + l (g < 2; g = 2, 3 hold 127);
 *   j: hi codes of the stage's two 32-k blocks, then their lo codes
 *   (hi+lo rows), or the hi codes of its four blocks (hi only).  Rows beyond
 *   M or N hold 127.
 *   TF32 W : [w_batches][2][M][Kp] FP32, X : [batch][2][N][Kp] FP32, each
 *            value rounded to TF32 (nearest, ties to even, to 10 mantissa
 *            bits; the low 13 bits zero), zero pad.  FP16 sources convert
 *            exactly; FP32 sources are rounded.
 */

/* Create a plan for problem *p on CUDA device `device`.  Validates the
 * shape, checks for an sm_103 device and allocates the plan's 256-byte
 * device status word and the scratch its default configuration and layout
 * need.  *out is set to NULL on error. */
tcbf_status tcbf_plan_create(tcbf_plan_t *out, const tcbf_problem *p, int device);

/* Destroy a plan (NULL is accepted).  The caller must not have work that
 * uses the plan in flight. */
tcbf_status tcbf_plan_destroy(tcbf_plan_t plan);

/* The plan's flags as it uses them: the caller's, with
 * TCBF_FLAG_AUTO_LAYOUT replaced by the layout it chose. */
tcbf_status tcbf_plan_flags(tcbf_plan_t plan, uint32_t *flags);

/* Bytes of the packed operand `which` (0 = W, 1 = X) for this plan. */
tcbf_status tcbf_packed_size(tcbf_plan_t plan, int which, size_t *bytes);

/* Bytes of caller-provided workspace the beamform calls need (currently 0). */
tcbf_status tcbf_workspace_size(tcbf_plan_t plan, size_t *bytes);

/*
 * Transpose/pack kernel (Sec. III: "the matrix-matrix multiplication kernel
 * requires that the input matrices are tiled in device memory ... handled
 * through a transpose kernel"; for 1-bit "32 consecutive 1-bit samples must
 * be stored in a single 32-bit integer").
 *   which = 0: src is W, [w_batches][M][K] complex of type src_type;
 *   which = 1: src is X, [batch][K][N] complex of type src_type.
 *   dst: packed layout of the plan's mode (see above), tcbf_packed_size bytes.
 * FP16/FP8 modes de-interleave (and for X transpose) into planes; 1-bit mode
 * keeps only the sign of each component (v >= 0 -> bit 1, so -0 -> +1;
 * NaN -> bit 0) and packs 32 per word along K.  src and dst must not overlap.
 */
tcbf_status tcbf_transpose_pack(tcbf_plan_t plan, int which, int src_type, const void *src,
                                void *dst, tcbf_stream_t stream);

/*
 * 1-bit unpacking (Sec. III: the library provides packing and unpacking for
 * 1-bit data), the inverse of tcbf_transpose_pack on a 1-bit plan: packed
 * bit planes back to interleaved complex values, bit 1 -> +1 and bit 0 -> -1
 * (Fig. 1), exactly.
 *   which = 0: src = packed W [w_batches][2][M][Kw] uint32,
 *              dst = [w_batches][M][K] interleaved complex
 *   which = 1: src = packed X [batch][2][N][Kw] uint32,
 *              dst = [batch][K][N] interleaved complex (un-transposed)
 *   dst_type:  TCBF_SRC_CF16 (4 bytes per value) or TCBF_SRC_CF32 (8 bytes)
 * Bits at k >= K are ignored.  Both pointers DEVICE, 16-byte aligned.
 * TCBF_ERR_INVALID_ARG for another mode or a bad which / dst_type.
 */
tcbf_status tcbf_unpack_bits(tcbf_plan_t plan, int which, const uint32_t *src, void *dst,
                             int dst_type, tcbf_stream_t stream);

/*
 * FP16 complex GEMM, Y[b] = W[b'] X[b] (Eq. 3), four real tensor-core MMAs
 * per complex tile (Sec. III-B) accumulated in FP32.
 *   Wp, Xp: FP16 packed operands of this plan (mode TCBF_MODE_FP16).
 *   Y: [batch][M][N] interleaved complex FP32 (8 bytes per value), written
 *      in full.  Y must not overlap Wp or Xp.
 * Above K = 4096 the sums are promoted to FP32 round-to-nearest every 2048 K.
 * A stacked-X plan on SM pairs may run the tiles of its last partial wave as
 * parts of whole 2048-K chunks on the pairs that wave leaves idle, and then
 * launches a second kernel that adds their later chunks in chunk order (the
 * same bits as whole tiles).
 */
tcbf_status tcbf_beamform_fp16(tcbf_plan_t plan, const void *Wp, const void *Xp, float *Y,
                               tcbf_stream_t stream);

/*
 * Split-FP8 complex GEMM: Y ~= Wh Xh + Wh Xl + Wl Xh summed in FP32 and
 * scaled back (FP8 formats: Sec. VI future work).  Wp, Xp: FP8-split packed
 * operands of this plan (mode TCBF_MODE_FP8SPLIT).  Y as for FP16.
 */
tcbf_status tcbf_beamform_fp8split(tcbf_plan_t plan, const void *Wp, const void *Xp, float *Y,
                                   tcbf_stream_t stream);

/*
 * TF32 complex GEMM for data that arrives in FP32: the FP16 product of
 * Sec. III-B with kind::tf32 MMAs (10 mantissa bits like FP16, FP32's
 * exponent range, half the FP16 tensor rate).  Wp, Xp: TF32 packed operands
 * of this plan (mode TCBF_MODE_TF32).  Y as for FP16.
 */
tcbf_status tcbf_beamform_tf32(tcbf_plan_t plan, const void *Wp, const void *Xp, float *Y,
                               tcbf_stream_t stream);

/*
 * 1-bit complex GEMM (Sec. III-D, Eq. 4-6), exact.  Wbits, Xbits: 1-bit
 * packed operands (mode TCBF_MODE_1BIT).  Y: [batch][M][N] interleaved
 * int32 pairs (re, im), each |value| <= 2K.
 *
 * Two arithmetic paths, chosen by the plan's configuration: bits expanded
 * on chip to E4M3 +-1 (FP8 MMAs; configurations "1bit->e4m3 ..."), or the
 * 4-bit tensor path (configurations "1bit->e2m1 ..."): each call expands
 * W and X into E2M1 +-1 planes held by the plan (tcbf_expand_1bit below),
 * then runs block-scaled 4-bit MMAs with unit scales.  Both are exact for
 * K <= 2^23 (every partial sum an integer of magnitude <= 2K in FP32).
 * tcbf_plan_create gives a 1-bit plan the 4-bit path by default when
 * K <= 2^23 and its planes fit in device memory (256 x 112 tiles with two
 * accumulators for K <= 6144, else 256 x 128 tiles with one): (w_batches x 2 x M +
 * batch x 3 x N) rows of 16 x Kw bytes, owned by the plan and freed by
 * tcbf_plan_destroy; otherwise configuration 0 (E4M3).  Selecting a 4-bit
 * configuration with tcbf_plan_set_config allocates the planes if needed
 * (TCBF_ERR_OOM when they do not fit).  Plans the 4-bit path cannot take
 * (uneven batch rows, K > 2^23) run configuration 0 instead.
 */
tcbf_status tcbf_beamform_1bit(tcbf_plan_t plan, const uint32_t *Wbits, const uint32_t *Xbits,
                               int32_t *Y, tcbf_stream_t stream);

/*
 * The two halves of tcbf_beamform_1bit on the 4-bit tensor path, for
 * callers that keep W fixed over many blocks of samples (the beamformer's
 * usual case: expand W once, then X and the GEMM per block).
 *
 * tcbf_expand_1bit: expand packed bits into the plan's E2M1 planes.
 *   which = 0: bits = packed W [w_batches][2][M][Kw] uint32; which = 1:
 *   packed X [batch][2][N][Kw] (the layouts of tcbf_beamform_1bit; bits at
 *   k >= K are ignored).  W becomes the planes Wr, Wi and X the planes
 *   -Xi, Xr, Xi, each element 0x2 (+1), 0xA (-1) or 0 (k >= K), two per
 *   byte.  Asynchronous on `stream`; the planes stay until the next
 *   expansion of the same operand or tcbf_plan_destroy.
 * tcbf_beamform_1bit_expanded: Y = W X (Eq. 3) from the planes last
 *   expanded; Y as for tcbf_beamform_1bit.  The configuration in use when
 *   it is called chooses the tile shape.
 * Errors: TCBF_ERR_INVALID_ARG (null plan or pointer, pointer not 16-byte
 * aligned, which not 0 or 1, plan not TCBF_MODE_1BIT), TCBF_ERR_UNSUPPORTED
 * (configuration not on the 4-bit path, or the plan cannot take it: uneven
 * batch rows, K > 2^23), TCBF_ERR_CUDA (launch failure).
 */
tcbf_status tcbf_expand_1bit(tcbf_plan_t plan, int which, const uint32_t *bits,
                             tcbf_stream_t stream);
/*
 * tcbf_transpose_pack_expanded: the transpose/pack of Sec. III for a 1-bit
 * plan on the 4-bit tensor path, writing the plan's E2M1 planes straight
 * from interleaved complex values (one pass, no packed bits):
 *   which = 0: src is W, [w_batches][M][K] complex of type src_type;
 *   which = 1: src is X, [batch][K][N] complex of type src_type.
 * Each component is sign-quantised as by tcbf_transpose_pack (v >= 0 -> +1,
 * so -0 -> +1; negative and NaN -> -1) and lands in the planes that
 * tcbf_expand_1bit would write from the packed bits of the same values; the
 * planes stay until the next pack or expansion of the same operand.  src
 * DEVICE, 16-byte aligned.  Errors as for tcbf_expand_1bit, and
 * TCBF_ERR_INVALID_ARG for a bad src_type.
 */
tcbf_status tcbf_transpose_pack_expanded(tcbf_plan_t plan, int which, int src_type,
                                         const void *src, tcbf_stream_t stream);
tcbf_status tcbf_beamform_1bit_expanded(tcbf_plan_t plan, int32_t *Y, tcbf_stream_t stream);

/*
 * Steering weights from geometry (Eq. 1-2): for weight batch b, beam m and
 * receiver k,
 *   far field  (near_field = 0): tau = (p_k . s_m) / c, A = 1, s_m a unit direction;
 *   near field (near_field = 1): d = |t_m - p_k|, tau = d / c, A = 1 / d;
 *   w = A exp(-2 pi i f[b,k] tau).
 * The phase f*tau is formed and reduced modulo one cycle in FP64; sine and
 * cosine of the reduced phase are taken in FP32.  Inputs are device FP64
 * arrays: rx_pos [K][3] (m), targets [M][3], freqs [w_batches][K] (Hz);
 * c in m/s.  Wp_out receives W packed for the plan's mode (FP16 planes,
 * sign bits, or FP8 split), tcbf_packed_size(plan, 0) bytes.
 */
tcbf_status tcbf_weights_from_geometry(tcbf_plan_t plan, const double *rx_pos,
                                       const double *targets, int near_field,
                                       const double *freqs, double c, void *Wp_out,
                                       tcbf_stream_t stream);

/* Synchronise the plan's device, read and clear its device status word.
 * Returns TCBF_OK, TCBF_ERR_TIMEOUT or TCBF_ERR_DEVICE. */
tcbf_status tcbf_last_device_error(tcbf_plan_t plan);

/* NOT PART OF THE BEAMFORMING API: test infrastructure shipped in the
 * library so that the failure path can be exercised on a real GPU.
 * Test hook for the device-side failure path (every wait in the GEMM
 * kernels gives up after 2 s and records it in the status word).  The next
 * tcbf_beamform_fp16 / tcbf_beamform_fp8split call on this plan launches
 * with the operand load number `fill` (0-based, in the first CTA's order of
 * stages) left out: its shared-memory slot is never marked full, so the
 * MMA issuer's wait runs out, the CTA records the timeout, lets its other
 * copies land, releases tensor memory and returns (after about 4 s); other
 * CTAs finish normally and that CTA's tiles of Y are left unwritten.
 * tcbf_last_device_error then returns TCBF_ERR_TIMEOUT and the device
 * context stays usable.  Applies to one call, then clears; fill < 0 clears
 * it at once.  Supported on plans running a one-SM, non-cluster tile
 * configuration of the FP16 or FP8 GEMM (configurations 0-5, no stacked
 * planes, even batches), else TCBF_ERR_UNSUPPORTED.  Nothing faults, traps
 * or spins without a limit. */
tcbf_status tcbf_debug_drop_fill(tcbf_plan_t plan, int64_t fill);

/* Static text for a status code. */
const char *tcbf_status_string(tcbf_status s);

/*
 * FP16 beamform that allocates no device memory.  The paper has no
 * counterpart; this call exists for callers that cannot allocate device
 * memory when they beamform: code running while a stream is being captured
 * into a CUDA graph, real-time acquisition loops where the implicit device
 * synchronisation of cudaMalloc/cudaFree would break their timing, and
 * plug-ins whose host framework owns the device memory budget.  It needs no
 * plan and no packed-sample buffer: the packed samples and the device status
 * word go into one file-scope static device array, 64 MiB of packed samples
 * plus 256 bytes, which every GPU that loads the library holds until the
 * process exits.
 *   p:       problem (mode TCBF_MODE_FP16), validated as by tcbf_plan_create.
 *   Wp:      packed FP16 weights (tcbf_transpose_pack / tcbf_weights_from_geometry
 *            of a plan with the same problem).
 *   X:       [batch][K][N] interleaved complex samples of type src_type (tcbf_src_type).
 *   Y:       [batch][M][N] interleaved complex FP32 output.
 *   check:   0 = return after launching; nonzero = wait for the stream and
 *            report a device-side timeout as TCBF_ERR_TIMEOUT.
 * Returns TCBF_ERR_BUDGET (nothing launched) when batch*2*N*round_up(K,64)*2
 * bytes of packed samples exceed 64 MiB.  The first call on a device looks
 * up the array's device address and the device's properties; make that
 * first call before any stream capture.  The lookup is repeated when the
 * device's context has changed since (after a cudaDeviceReset by the
 * caller), as the array then has a new address.  Every call uses the same array and
 * clears the status word it needs; the packed-sample region keeps the last
 * call's contents.  Calls whose work overlaps on the GPU (other streams, or
 * other host threads) race on the array and must be serialised by the caller.
 */
tcbf_status tcbf_beamform_fp16_noalloc(const tcbf_problem *p, int device, const void *Wp,
                                       const void *X, int src_type, float *Y, int check,
                                       tcbf_stream_t stream);

/* Number of kernel configurations (tile shapes) the plan's mode offers,
 * the one in use, and a way to pick one (the autotuner's hook). */
tcbf_status tcbf_plan_num_configs(tcbf_plan_t plan, int *count);
tcbf_status tcbf_plan_get_config(tcbf_plan_t plan, int *config);
tcbf_status tcbf_plan_set_config(tcbf_plan_t plan, int config);
/* Human-readable description of configuration `config` (static string). */
const char *tcbf_config_name(tcbf_plan_t plan, int config);

/*
 * Uneven batches (Sec. V-B: every channel/polarisation is one product; here
 * each may have its own beam count).  rows: HOST array of `batch` entries,
 * 1 <= rows[b] <= M; NULL returns to uniform batches.  Layouts keep M rows
 * per batch; the kernels compute only the tiles covering rows[b] rows, all
 * batches still in one persistent launch.  Rows m >= rows[b] of Y[b] up to
 * the next multiple of 128 are overwritten with unspecified values; rows
 * beyond that are left untouched.  Allocates a (batch+1)-int device table
 * owned by the plan (synchronous).
 */
tcbf_status tcbf_plan_set_batch_rows(tcbf_plan_t plan, const int64_t *rows);

/*
 * Autotuner (Sec. IV-A: the work per block and the number of buffers are
 * tuned per GPU and shape).  Times every valid configuration of the plan's
 * mode with CUDA events on `stream` on the caller's packed operands and
 * output: each is warmed up and sized into a group of launches lasting at
 * least 0.2 ms, then the configurations are timed round-robin for `reps`
 * rounds (so a slow drift of the clocks affects them alike) and each keeps
 * its fastest group.  Selects the fastest and leaves it set on the plan.
 * Synchronises the stream.  *best receives the chosen configuration;
 * ms_per_config (nullable, tcbf_plan_num_configs entries) the milliseconds
 * per launch of each one's fastest group, -1 for configurations not valid
 * for this shape.  Y is overwritten.  All modes.
 */
tcbf_status tcbf_autotune(tcbf_plan_t plan, const void *Wp, const void *Xp, void *Y, int reps,
                          tcbf_stream_t stream, int *best, float *ms_per_config);

/*
 * Layout autotuner for plans created with TCBF_FLAG_AUTO_LAYOUT (else
 * TCBF_ERR_INVALID_ARG).  For the planar, the stacked and (when N % 4 == 0
 * and the batch rows are uniform, so that the fused kernel takes it) the
 * interleaved X layout in turn it packs X_src ([batch][K][N] complex of
 * src_type, the tcbf_transpose_pack source) into a scratch buffer it
 * allocates (for the interleaved layout: copies it, as tcbf_transpose_pack
 * does) and runs tcbf_autotune over that layout's configurations (`reps`
 * rounds); then it times the layouts' steps, pack + beamform with each one's
 * best configuration, round-robin for `reps` rounds in groups of at least
 * about 1 ms, keeping each one's fastest group.  The plan keeps the fastest
 * layout and
 * its configuration; *flags (nullable) receives the plan's new flags and
 * ms_per_layout (nullable, 3 entries) the step milliseconds of the planar,
 * stacked and interleaved layouts (-1 for one not timed).  A plan that ends
 * on the interleaved layout can also be given X itself instead of its copy
 * (TCBF_FLAG_INTERLEAVED_X), which saves the copy.  Wp is the packed W (the same bytes for both
 * layouts); Y is overwritten.  Synchronises the stream and frees the
 * scratch before it returns.  When the layout changes, packed X made
 * before the call no longer fits the plan (repack it; tcbf_packed_size(1)
 * may have changed), and the plan's tcbf_beamform_host staging and
 * captured graph are released.
 */
tcbf_status tcbf_autotune_layout(tcbf_plan_t plan, const void *Wp, const void *X_src, int src_type,
                                 void *Y, int reps, tcbf_stream_t stream, uint32_t *flags,
                                 float *ms_per_layout);

/*
 * Capture one step into a CUDA graph owned by the plan: the transpose/pack
 * of X_src into Xp (skipped when X_src is NULL) followed by the beamform of
 * Wp and Xp into Y, with the plan's current configuration.  Pointers are
 * baked into the graph; replace the graph by capturing again.  All modes.
 * tcbf_graph_launch replays it on `stream` (one launch of the whole step;
 * TCBF_ERR_INVALID_ARG if nothing was captured).
 */
tcbf_status tcbf_graph_capture(tcbf_plan_t plan, const void *X_src, int src_type, void *Xp,
                               const void *Wp, void *Y);
tcbf_status tcbf_graph_launch(tcbf_plan_t plan, tcbf_stream_t stream);

/*
 * The whole step for HOST-resident data: Y_host[b] = W[b / per_w] X_host[b]
 * (Eq. 3) for every batch b, in every mode.  The paper's library sits inside
 * an instrument's processing pipeline (Sec. V); this is the call such a
 * pipeline makes when its samples arrive in host memory.  The data movement
 * around the kernels is this library's own: the batches go through in
 * chunks, each chunk's X copied host-to-device on one stream, packed and
 * beamformed on a second, and its Y copied device-to-host on two more, so
 * the copies of one chunk overlap the compute of its neighbours.
 *   X_host: HOST [batch][K][N] interleaved complex of type src_type
 *           (tcbf_src_type), as for tcbf_transpose_pack(which = 1).
 *   Wp:     DEVICE packed weights of the plan's mode (tcbf_transpose_pack
 *           which = 0 or tcbf_weights_from_geometry), all w_batches.
 *   Y_host: HOST [batch][M][N] interleaved complex, 8 bytes per value:
 *           FP32 (FP16 and split-FP8 plans) or int32 (1-bit plans).
 *   chunk:  batches per chunk, a positive multiple of batch / w_batches (the
 *           last chunk may be shorter); 0 picks about batch / 16.
 * A single-batch problem (batch = 1) is cut into ranges of W rows instead:
 * X is copied in and packed once, then each range of about M / 4 rows
 * (whole waves of 128-row tiles over the SMs) is beamformed and its rows of
 * Y copied out while the next range computes; chunk must be 0 or 1.
 * Device staging for three chunks (source X, packed X, Y) is allocated at
 * the first call, or when `chunk` grows, and kept by the plan until
 * tcbf_plan_destroy; TCBF_ERR_OOM if it cannot be had.  The work starts
 * after everything already enqueued on `stream`, and `stream` waits for the
 * last copy, so work enqueued on it later sees Y_host complete; the call
 * itself does not block the host.  Host buffers must stay valid and X_host
 * unmodified until then; page-locked host memory is needed for the copies to
 * overlap (pageable memory gives the same result, serialised).  Calls on one
 * plan share its staging, so they must be ordered (enqueue them on one
 * stream).  Uneven batches (tcbf_plan_set_batch_rows) are not supported:
 * TCBF_ERR_UNSUPPORTED.  Device errors surface through
 * tcbf_last_device_error as for the other calls.
 */
tcbf_status tcbf_beamform_host(tcbf_plan_t plan, const void *X_host, int src_type, const void *Wp,
                               void *Y_host, int64_t chunk, tcbf_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TCBF_H */
