/*
 * rmdec_serve — continuous-batching request server over rmdec decoder handles.
 *
 * Not part of the paper's method (which decodes one received word at a time); this is the
 * serving layer for many concurrent decode requests of mixed codes: requests arrive on any
 * host thread, are admitted as device memory frees up, are packed per code into batches as
 * CUDA streams free up, and complete independently. Decoding itself is rmdec_decode
 * (include/rmdec.h), or rmdec_group_decode for batches that mix codes; every frame is decoded
 * independently and identically either way, so a request's result does not depend on what it
 * was batched with.
 *
 * Threading: all CUDA work runs on one worker thread owned by the server; submit/poll/stats
 * may be called from any thread. Decoder handles registered with a server must not be used
 * elsewhere while the server runs (the server does not own them; destroy them after the
 * server).
 */
#ifndef RMDEC_SERVE_H
#define RMDEC_SERVE_H

#include <stdint.h>

#include "rmdec.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rmdec_server *rmdec_server_t;

typedef struct {
    int n_streams;            /* CUDA streams (batches in flight), 1..16 */
    int64_t arena_bytes;      /* device memory for resident request LLRs and outputs */
    int64_t max_batch_frames; /* frames per batch cap (one kernel launch); a batch is also kept
                               * within arena_bytes, so requests that fit the arena only one at
                               * a time are admitted one at a time */
    int64_t min_batch_frames; /* a batch waits up to max_wait_us for this many frames */
    int64_t max_wait_us;      /* longest time a request waits for batch companions */
    int fuse_codes;           /* 1: batch small requests (below one full wave of their code's own
                               * launch) of different codes that can share a grouped launch
                               * (include/rmdec_group.h: p-FHT-FSCL decoders of one list size L in
                               * {1, 2, 4, 8}, up to 16 codes per family) and decode them with one
                               * rmdec_group_decode call; 0: one code per batch */
} rmdec_server_config;

typedef struct {
    int64_t submitted, completed, frames_completed, batches;
    int64_t queued, in_flight;       /* requests waiting for admission / admitted, not done */
    double latency_p50_us, latency_p99_us;  /* over the most recent 65,536 completed requests */
    double latency_max_us;                   /* over all completed requests */
    double busy_seconds;             /* wall time from first submit to last completion */
    int64_t cancelled;               /* requests cancelled before admission */
} rmdec_server_stats;

/* Creates a server on the current CUDA device; allocates the arena and the streams and starts
 * the worker thread. */
rmdec_status rmdec_server_create(rmdec_server_t *out, const rmdec_server_config *cfg);

/* Registers a decoder handle; *code_id identifies it in submissions. */
rmdec_status rmdec_server_add_decoder(rmdec_server_t s, rmdec_t h, int *code_id);

/* Queues a request of n_frames frames: llr_host [n_frames][N] of the handle's dtype (pinned host
 * memory gives the best copy rate), bits_out_host [n_frames][ceil(K/32)] uint32. Both buffers
 * must stay valid until rmdec_server_poll reports completion. Requests larger than the arena
 * or than max_batch_frames fail with RMDEC_EINVAL. *request receives an id (> 0). */
rmdec_status rmdec_server_submit(rmdec_server_t s, int code_id, const void *llr_host, int64_t n_frames,
                                 uint32_t *bits_out_host, uint64_t *request);

/* Waits up to timeout_us (0 = check) for a request: RMDEC_OK when its bits are in the host
 * buffer (the request is retired; *latency_us, if not NULL, receives submit-to-completion
 * time), RMDEC_EBUSY / RMDEC_ETIMEDOUT otherwise, RMDEC_EINVAL for an unknown id,
 * RMDEC_ECUDA if its batch failed, RMDEC_ECANCELED (retired) if it was cancelled. */
rmdec_status rmdec_server_poll(rmdec_server_t s, uint64_t request, int64_t timeout_us, double *latency_us);

/* Cancels a request that has not been admitted yet: it will never touch its buffers, and
 * rmdec_server_poll retires it with RMDEC_ECANCELED. RMDEC_EBUSY if it was already admitted
 * (its batch completes normally), RMDEC_EINVAL for an unknown id. */
rmdec_status rmdec_server_cancel(rmdec_server_t s, uint64_t request);

/* Counters over the requests so far, and latency percentiles over the most recent 65,536
 * completed requests (the server keeps a bounded record; the maximum covers all of them). */
rmdec_status rmdec_server_stats_get(rmdec_server_t s, rmdec_server_stats *out);

/* Stops the worker after draining in-flight batches, frees device memory. Queued requests
 * that were never admitted are dropped. */
void rmdec_server_destroy(rmdec_server_t s);

const char *rmdec_server_last_error(rmdec_server_t s);

#ifdef __cplusplus
}
#endif

#endif /* RMDEC_SERVE_H */
