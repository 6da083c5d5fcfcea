/*
 * rmdec_group — one kernel launch over frames of several decoders (different codes RM(r, m),
 * numbers of parallel decoders P and LLR types), for batches that mix codes.
 *
 * Each frame is decoded exactly as rmdec_decode decodes it with the same handle (Algorithm 5
 * over the handle's P decoders, each following Algorithm 2 with FHTL nodes, Algorithms 3-4
 * and Eq. (8), and SPCL nodes, Eqs. (2)-(6), of arXiv 2108.12550): results are bit-identical.
 * Grouping is not part of the paper's method; it packs uneven work into one persistent
 * launch, so that many small per-code batches need neither a launch each nor a stream each
 * and together fill the GPU. A grouped launch runs every member with the largest member's
 * shared-memory and register footprint, so segments large enough to fill the GPU on their
 * own are better off in their decoder's own launch, and by default go there.
 *
 * Members: p-FHT-FSCL and FHT-FSCL handles (rmdec_create, rmdec_create_fhtfscl) that share
 * one list size L in {1, 2, 4, 8}; any (m, r) with m <= 9 and r in {2, 3} that those
 * constructors accept, any P, any dtype. Aut-SSC handles, codes of length 1024, RM(4, m),
 * RM(1, m) / RM(m-1, m) decoders and the tensor-core Hadamard variant are not supported
 * (decode them with rmdec_decode).
 */
#ifndef RMDEC_GROUP_H
#define RMDEC_GROUP_H

#include <stdint.h>

#include "rmdec.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rmdec_group *rmdec_group_t;

/* One run of frames of one member. */
typedef struct {
    int decoder;           /* index into the create call's decoder array */
    const void *llr_dev;   /* device [n_frames][N] of that handle's dtype, 16-byte aligned */
    int64_t n_frames;      /* >= 0; empty segments are skipped */
    uint32_t *bits_out_dev; /* device [n_frames][ceil(K/32)] information bits u_I, I ascending */
} rmdec_segment;

/* Creates a group over n_decoders (1..16) handles. The group keeps the handle pointers, not
 * copies: the handles must outlive it, and tables changed with rmdec_set_perms or a new dtype
 * are picked up by the next decode. Host-side only: RMDEC_EINVAL for a null or unsupported
 * handle or for mixed list sizes (rmdec_last_error(NULL) says which). */
rmdec_status rmdec_group_create(rmdec_group_t *out, const rmdec_t *decoders, int n_decoders);

/* Decodes n_segs segments, asynchronously on `stream` (a cudaStream_t, NULL = default
 * stream). Segments too small to fill the GPU alone (see rmdec_group_set_split) are ordered
 * by decreasing work per frame and share one grouped launch (more than 224 such segments
 * take several launches); each larger segment then runs in its own decoder's launch, which
 * keeps that decoder's own occupancy. All launches go to `stream` in that order. Uploads
 * member tables on first use (synchronous), so call once before any stream capture.
 * RMDEC_EINVAL for a bad segment (unknown decoder, negative count, null or misaligned
 * pointer); nothing is launched then. */
rmdec_status rmdec_group_decode(rmdec_group_t g, const rmdec_segment *segs, int n_segs, void *stream);

/* Which segments leave the grouped launch: those of at least min_frames_alone frames
 * (0, the default: half a wave of the decoder's own launch, a wave being SMs x its resident
 * CTAs; < 0: none, every segment is grouped). Never changes results. */
rmdec_status rmdec_group_set_split(rmdec_group_t g, int64_t min_frames_alone);

/* Launch shape of the group's launches: warps per CTA (1..20) and a cap on CTAs per SM
 * (0 = the occupancy limit). 0 warps = the default: the CTA of 1..4 warps with the most
 * resident warps per SM, except that a launch of at most one wave of that shape takes the
 * CTA of 1..20 warps whose busiest CTA runs the fewest decoder rounds (weighted by each code's
 * work per decoder). Never changes results. */
rmdec_status rmdec_group_set_tuning(rmdec_group_t g, int warps_per_cta, int ctas_per_sm);

void rmdec_group_destroy(rmdec_group_t g);

/* Last failure on this group (or of the last failed create when g is NULL); never NULL. */
const char *rmdec_group_last_error(rmdec_group_t g);

#ifdef __cplusplus
}
#endif

#endif /* RMDEC_GROUP_H */
