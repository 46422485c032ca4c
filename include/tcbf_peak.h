/*
 * tcbf_peak.h — on-chip peak microbenchmarks of the GB300 build.
 *
 * NOT PART OF THE BEAMFORMING API: measurement infrastructure shipped in the
 * library (the benchmark's roofline denominators and the 1-bit path choice).
 *
 * Like the paper's tensor-core micro-benchmarks (Sec. III-A, Table I) they
 * keep operands on chip so memory bandwidth does not limit them; they supply
 * the per-precision peak denominators and the measurements behind the 1-bit
 * kernel choice (Sec. III-D/E).
 */
#ifndef TCBF_PEAK_H
#define TCBF_PEAK_H

#include "tcbf.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Run microbenchmark `kind` once for warm-up and once timed (CUDA events) on
 * device `device`, one CTA per SM for the tcgen05 kinds, 4 x 256-thread
 * blocks per SM for the warp-level kinds:
 *   0 tcgen05 kind::f16 M128 N256 K16, 1 tcgen05 kind::f8f6f4 (E4M3) M128 N256 K32,
 *   2 tcgen05 kind::i8 (not available on sm_103a: always TCBF_ERR_UNSUPPORTED),
 *   3 mma.sync m16n8k16 f16->f32,
 *   4 mma.sync m16n8k256 b1 AND-popc, 5 CUDA-core popc(xor) on 32-bit words,
 *   6 tcgen05 kind::f16 M128 N128 K16 (the beamformer's one-SM tile MMA),
 *   7 tcgen05 kind::mxf4 M128 N256 K64 (packed E2M1 with unit UE8M0 block
 *     scales: the 1-bit GEMM's 4-bit path),
 *   8 tcgen05 kind::mxf4nvf4 M128 N256 K64 with unit UE4M3 scales per 16 K,
 *   9 tcgen05 kind::mxf4nvf4 M128 N256 K64 with unit UE8M0 scales per 32 K.
 * iters: MMAs (or loop trips) per issuing thread.  On success *seconds is the
 * timed launch's duration and *ops the operations it performed (2 per
 * multiply-accumulate).  Allocates and frees a 256-byte status word.
 * Returns TCBF_ERR_UNSUPPORTED on a device other than sm_103.
 */
tcbf_status tcbf_peak_run(int kind, int device, int iters, double *seconds, double *ops);

/*
 * HBM stream with a chosen read/write mix, the ceiling of a memory-bound
 * kernel's byte mix (the beamformer's output-heavy steps): read_bytes are
 * read with 16-byte loads, then write_bytes written with 16-byte stores, by
 * blocks_per_sm x SMs blocks of 256 threads (each thread reads its share,
 * then writes its share; the threads' reads and writes overlap).  Both sizes
 * multiples of 16 bytes; blocks_per_sm in [1, 64].  Allocates and frees the
 * two device buffers.  *seconds: the fastest of three timed launches after a
 * warm-up (CUDA events).  TCBF_ERR_OOM when the buffers do not fit.
 */
tcbf_status tcbf_peak_stream(int device, int64_t read_bytes, int64_t write_bytes, int blocks_per_sm,
                             double *seconds);

#ifdef __cplusplus
}
#endif
#endif /* TCBF_PEAK_H */
