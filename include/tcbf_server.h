/*
 * tcbf_server.h — continuous-batching beamforming server of the GB300 build.
 *
 * The paper's library executes one (batched) product per call; its
 * applications feed it blocks of samples as they are recorded (Sec. V: the
 * ultrasound and LOFAR pipelines).  This server turns the library into a
 * request loop: blocks of samples for resident weight sets arrive over time
 * in any of the three modes, are admitted while their device buffers fit an
 * HBM budget, and run concurrently on several streams; when a request
 * completes, its memory is freed and waiting arrivals are admitted.  Each
 * request runs exactly the kernels and tile configuration it would run
 * alone, so its result is the same alone and in the mix.
 *
 * All functions are thread-safe.  Pointers marked HOST are host memory
 * (page-locked memory is required for the copies to overlap); others are
 * device memory of the server's device.
 */
#ifndef TCBF_SERVER_H
#define TCBF_SERVER_H

#include "tcbf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tcbf_server_s *tcbf_server_t;

typedef struct {
    int32_t set_id;        /* resident weight set (registered for this mode) */
    int32_t mode;          /* tcbf_mode */
    int64_t N;             /* samples in the block */
    int32_t src_type;      /* tcbf_src_type of host_x */
    uint32_t flags;        /* reserved, 0 */
    const void *host_x;    /* HOST [K][N] interleaved complex samples (K of the weight set) */
    void *host_y;          /* HOST [M][N] output, 8 bytes per value (complex FP32, or int32
                              pairs in 1-bit mode); NULL: results stay on the device and
                              are discarded when the request completes */
    double arrival_s;      /* arrival time, seconds after tcbf_server_start */
} tcbf_request;

typedef struct {
    double arrival_s;      /* as submitted */
    double admit_s;        /* when the scheduler issued it (seconds after start) */
    double done_s;         /* when its completion event was observed */
    int32_t stream;        /* stream it ran on */
    int32_t status;        /* TCBF_OK, a tcbf_status, or -1 while not finished */
    double ops;            /* 8 * M * N * K useful operations */
} tcbf_request_result;

typedef struct {
    uint64_t submitted, pending, inflight;
    int64_t peak_inflight;
    uint64_t arena_bytes, peak_arena_bytes;
} tcbf_server_counters;

/* Create a server on `device` with a device arena of arena_bytes (the HBM
 * budget for request buffers: raw samples, packed samples and output of
 * every admitted request), num_streams streams (1..64) and at most
 * max_inflight admitted requests (0 = no limit).  Allocates the arena. */
tcbf_status tcbf_server_create(tcbf_server_t *out, int device, size_t arena_bytes,
                               int num_streams, int max_inflight);

/* Register a resident weight set: Wp is packed W of shape M x K for `mode`
 * (tcbf_transpose_pack / tcbf_weights_from_geometry of a plan with batch 1).
 * The caller keeps Wp alive while the server may use it. */
tcbf_status tcbf_server_register_weights(tcbf_server_t s, int set_id, int mode, int64_t M,
                                         int64_t K, const void *Wp);

/* Queue a request; *ticket (1, 2, ...) identifies it.  TCBF_ERR_BUDGET if its
 * buffers could never fit the arena; TCBF_ERR_INVALID_ARG for an unknown
 * (set, mode).  May be called before or after tcbf_server_start. */
tcbf_status tcbf_server_submit(tcbf_server_t s, const tcbf_request *r, uint64_t *ticket);

/* Start the scheduler thread; arrival times count from this call. */
tcbf_status tcbf_server_start(tcbf_server_t s);

/* Block until every submitted request has completed, or timeout_s passes
 * (TCBF_ERR_TIMEOUT). */
tcbf_status tcbf_server_wait_all(tcbf_server_t s, double timeout_s);

/* Timing and status of one request. */
tcbf_status tcbf_server_result(tcbf_server_t s, uint64_t ticket, tcbf_request_result *out);

/* Counters: submitted, pending, in flight, peak in flight, arena use. */
tcbf_status tcbf_server_stats(tcbf_server_t s, tcbf_server_counters *out);

/* Stop the scheduler after the admitted requests finish (requests not yet
 * admitted are dropped) and free everything. */
tcbf_status tcbf_server_destroy(tcbf_server_t s);

#ifdef __cplusplus
}
#endif
#endif /* TCBF_SERVER_H */
