/*
 * rmdec — batched GPU decoding of Reed-Muller codes RM(r, m) with permuted fast
 * successive-cancellation list decoding and the fast Hadamard transform (p-FHT-FSCL-L-M),
 * after Doan, Hashemi and Gross, "Successive-Cancellation Decoding of Reed-Muller Codes
 * with Fast Hadamard Transform" (arXiv 2108.12550), Algorithms 2-5.
 *
 * Plain C ABI. Pointers are host or device memory as stated per argument; no handle keeps
 * a caller pointer after the call's stream work completes. No C++ exception crosses this
 * boundary. Every entry point returns an rmdec_status; on failure nothing was launched
 * (unless stated otherwise) and rmdec_last_error(h) describes the failure.
 *
 * Notation: N = 2^m code length, K = sum_{i<=r} C(m, i) information bits,
 * P = number of parallel decoders (the paper's M, Algorithm 5), L = list size.
 * Bit layouts: bit j of a packed bit vector is bit (j % 32) of 32-bit word j / 32.
 */
#ifndef RMDEC_H
#define RMDEC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rmdec_ctx *rmdec_t;

typedef enum {
    RMDEC_OK = 0,
    RMDEC_EINVAL = -1,      /* bad argument or unsupported (m, r, P, L) combination */
    RMDEC_ENOMEM = -2,      /* device or host allocation failed */
    RMDEC_ECUDA = -3,       /* a CUDA runtime call failed (message in rmdec_last_error) */
    RMDEC_EBUSY = -4,       /* rmdec_poll: the ticket's work has not finished yet */
    RMDEC_ETIMEDOUT = -5,   /* rmdec_poll: still running when the timeout expired */
    RMDEC_EDEVICE = -6,     /* no usable CUDA device */
    RMDEC_ECANCELED = -7,   /* rmdec_server_poll: the request was cancelled before admission */
} rmdec_status;

/* LLR element type of the input frames.
 * F32: IEEE single. F16: IEEE half, widened to single on load.
 * I8 / I16: quantised LLR codes q (LLR = q * step for the caller's step). Integer inputs are
 * decoded in exact integer arithmetic on the codes (every intermediate value is an integer
 * below 2^24 and is represented exactly), so results, path metrics and tie-breaks are
 * bit-identical to an exact integer decoder. Path metrics are reported in code units.
 * I16 codes are clamped to |q| <= 2^(24-m) - 1 on load so that exactness holds. */
typedef enum {
    RMDEC_LLR_F32 = 0,
    RMDEC_LLR_I8 = 1,
    RMDEC_LLR_F16 = 2,
    RMDEC_LLR_I16 = 3,
} rmdec_dtype;

/* Creates a p-FHT-FSCL-L-P decoder for RM(r, m) (Algorithm 5 with Algorithm 2 per decoder).
 * Supported, with 1 <= P <= 128:
 *   - 4 <= m <= 10, r in {2, 3} with r <= m - 2, and 6 <= m <= 9, r = 4 (the root is a
 *     permuted node, 1 < r < m - 1; r - 1 permuted levels), L in {1, 2, 4, 8, 16}, and
 *     L = 32 for m <= 9 (P = M_1 = 100, L = 1 is the paper's p-FHT-FSCL-1-100);
 *   - 2 <= m <= 10, r = 1 or r = m - 1, L in {1, 2, 4, 8, 16, 32}: the root is itself an FHTL
 *     (RM(1, m), Algorithms 3-4) or SPCL (RM(m-1, m), Eqs. (2)-(6)) node. Algorithm 2 decodes
 *     such a root before any permuted node and never undoes the initial permutations outside
 *     the permuted branch; the permutations, automorphisms of the code, would only copy the
 *     same candidate words into every path. Every decoder therefore decodes y with one live
 *     path, which returns the maximum-likelihood word (largest |c_k|, ties to the smaller k;
 *     or the hard decision with the least reliable bit fixing the parity), decoder 0 winning.
 *     L and P do not change the result; the permutation table is kept but unused.
 * The affine permutations x -> Ax + b of GA(m) that Algorithm 2 draws (L initial ones and
 * 2L candidates at each of the r - 1 permuted nodes, per decoder) are sampled on the host
 * from perm_seed with Philox4x32-10 (counter (p, q, attempt, 'PERM'), key = perm_seed) and
 * rejection of singular A; rmdec_get_perms returns them and rmdec_set_perms replaces them.
 * No GPU work happens here: device state is built on the first decode.
 * *out receives the handle (NULL on failure). */
rmdec_status rmdec_create(rmdec_t *out, int m, int r, int P, int L, uint64_t perm_seed);

/* Creates an FHT-FSCL-L decoder: the same tree without permutations, started from a single
 * live path (the decoder the paper's permuted decoder improves on; its Fig. 4 dashed curves).
 * Equivalent to p-FHT-FSCL-L-1 with identity permutations whose paths 1..L-1 start inactive.
 * Same support limits as rmdec_create with P = 1; the permutation table is fixed (identity). */
rmdec_status rmdec_create_fhtfscl(rmdec_t *out, int m, int r, int L);

/* Creates an Aut-SSC-P baseline decoder (the permuted simplified SC decoder the paper
 * compares against, Section III-B, Table 5): SSC decoding (repetition, SPC and f/g nodes,
 * L = 1) of each of P_ssc GA(m)-permuted copies of the frame, keeping the candidate with the
 * smallest correlation discrepancy (earliest permutation on ties).
 * Supported: 4 <= m <= 9, 1 <= r <= min(3, m - 2), 1 <= P_ssc <= 1024. Permutation q is drawn with
 * counter (0x53534300, q, attempt, 'PERM'). */
rmdec_status rmdec_create_aut_ssc(rmdec_t *out, int m, int r, int P_ssc, uint64_t perm_seed);

/* Releases the handle and its device memory. Waits for the handle's outstanding work. */
void rmdec_destroy(rmdec_t h);

/* Sets the LLR element type read by the decode calls (default RMDEC_LLR_F32). The decoder's
 * input is the vector of channel LLRs y = 2r/sigma^2 of a BPSK word over AWGN (Section II-A);
 * the paper computes in floating point throughout. The narrower types are this library's
 * storage formats for that vector, not part of the paper's method: F16 is widened to F32 on
 * load; I8/I16 codes are decoded exactly in integer arithmetic (see rmdec_dtype). Takes
 * effect on the next decode; an unknown type returns RMDEC_EINVAL. */
rmdec_status rmdec_set_dtype(rmdec_t h, rmdec_dtype t);

/* How FHTL nodes (Algorithms 3-4) compute the Walsh-Hadamard spectrum c = H y of their LLRs
 * (the fast Hadamard transform of Algorithm 4).
 * SHUFFLE (default): FP32 butterflies in registers and across lanes (warp shuffles).
 * TENSOR: nodes of 16 to 256 points multiply by H_16 on the tensor cores, with
 *   H_{2^s} = H_{2^(s-4)} (x) H_16 applied as H_16 X H_16 to the LLRs laid out as a
 *   2^(s-4) x 16 matrix X (two m16n8k16 MMAs per product): LLRs and the intermediate product
 *   enter as FP16 (rounded), sums accumulate in FP32, path metrics stay FP32. Smaller nodes
 *   keep the butterflies. An approximation of the FP32 transform (decisions may differ
 *   where FP16 rounding moves a candidate); integer inputs are no longer exact. Available
 *   for RM(2, 9) and RM(3, 9) with L in {4, 8} (RMDEC_EINVAL otherwise). Not groupable. */
typedef enum {
    RMDEC_HADAMARD_SHUFFLE = 0,
    RMDEC_HADAMARD_TENSOR = 1,
} rmdec_hadamard;
rmdec_status rmdec_set_hadamard(rmdec_t h, rmdec_hadamard mode);

/* Which kernel runs a p-FHT-FSCL decode (Algorithms 2-5; the same method either way).
 * AUTO (default): WARP, and PATH for launches of at least 512 (RM(2, m <= 5)), 2,048 (RM(2, 6),
 *   RM(2, 7), RM(3, m)) or 8,192 (RM(2, 8)) frames where it exists and was measured faster for
 *   the decoder's P and L (the warp kernel answers small launches sooner, the path kernel has
 *   the higher throughput unless the decoders' tables leave it few CTAs per SM or its L = 8
 *   candidate lists cost more). PATH by default for P in: RM(2, m <= 6) 1..128 (L = 8: 1..32);
 *   RM(3, 5) and RM(3, 6) 1..128 (L = 4: 1..64; L = 8: 1..20 and 1..16); RM(2, 7) 4..128
 *   (L = 4: 4..64; L = 8: 4..8); RM(3, 7) 4..128 (L = 4: 1..32; L = 8: 4); RM(2, 8) 4..128
 *   (L = 4: 4..20; L = 8: never). rmdec_kernel_for reports the choice for a launch size.
 * WARP: one warp per decoder, the L paths spread over its lanes and the tree's LLR buffers in
 *   shared memory; every supported code.
 * PATH: one thread per list path (two for m = 8), the tree's LLRs in registers, the decoders
 *   of a frame in one lane group; RM(2, m) with 4 <= m <= 8 and RM(3, m) with 5 <= m <= 7, L in
 *   {1, 2, 4, 8}, FP32 butterflies
 *   (RMDEC_EINVAL otherwise). Integer inputs decode identically under both; FP32 inputs may
 *   differ where two FHTL candidates of one path round to the same FP32 metric (WARP then
 *   prefers the smaller index, PATH the larger |c_k|). Segments of a grouped launch that
 *   their decoder's own launch would give to PATH are decoded in that launch (rmdec_group.h). */
typedef enum {
    RMDEC_KERNEL_AUTO = 0,
    RMDEC_KERNEL_WARP = 1,
    RMDEC_KERNEL_PATH = 2,
} rmdec_kernel;
rmdec_status rmdec_set_kernel(rmdec_t h, rmdec_kernel kernel);
/* The kernel that decodes a launch of n_frames frames with the handle's current settings:
 * RMDEC_KERNEL_PATH or RMDEC_KERNEL_WARP (also reported for Aut-SSC handles and for RM(1, m) and
 * RM(m-1, m) roots, whose kernels have no path-per-thread form). Uploads the handle's tables to
 * the current device if needed (as a decode would). Not part of the paper's method. */
rmdec_status rmdec_kernel_for(rmdec_t h, int64_t n_frames, rmdec_kernel *kernel);

/* Number of uint16 permutation records the handle holds (11 uint16 per record:
 * [c_0 .. c_9, b] with c_t = A e_t; the record maps index i to b XOR sum_{t: i_t = 1} c_t).
 * p-FHT-FSCL layout: decoder-major, per decoder L initial records then (r-1) * 2L candidate
 * records (level j = 0 .. r-2 is the node RM(r-j, m-j), records of GA(m-j)).
 * Aut-SSC layout: P_ssc records of GA(m). */
rmdec_status rmdec_perm_count(rmdec_t h, int64_t *n_records);
/* Host copies in / out of the permutation table (n_records must equal rmdec_perm_count).
 * set_perms rejects records that are not invertible affine maps of the right size. New
 * records reach the device at the next decode of the handle, which first waits for all work
 * on the device (so that no queued decode reads a half-written table) and then overwrites the
 * handle's device tables in place: graphs (rmdec_graph_create) and grouped launches that use
 * the handle decode with the new permutations from then on. */
rmdec_status rmdec_get_perms(rmdec_t h, uint16_t *perms_host, int64_t n_records);
rmdec_status rmdec_set_perms(rmdec_t h, const uint16_t *perms_host, int64_t n_records);

/* Code parameters of RM(r, m) (Section II-A): *n = N = 2^m, *k = K = sum_{i<=r} C(m, i),
 * *info_idx = the K information positions I = {i : popcount(i) >= m - r} in ascending order,
 * i.e. the rows of G^{(x)m} of weight at least 2^(m-r) (owned by the handle, valid until
 * rmdec_destroy). The decoded bits of every decode call are u_I in this order. Any output
 * pointer may be NULL. */
rmdec_status rmdec_info(rmdec_t h, int *n, int *k, const int **info_idx);

/* Decodes n_frames frames, asynchronously on `stream` (a cudaStream_t; NULL = legacy default
 * stream). llr_dev: device, [n_frames][N] elements of the handle's dtype, row-major, 16-byte
 * aligned. bits_out_dev: device, [n_frames][ceil(K/32)] uint32, the decoded information bits
 * u_I in ascending order of I (u = x G^{(x)m} of the selected codeword x, Section II-A).
 * n_frames == 0 is a no-op. The first call on a handle uploads its tables (synchronous).
 * LLRs are expected to be finite: a frame holding NaN or infinite values still yields a
 * codeword of one of the decoders (which one is unspecified) and leaves the other frames of
 * the batch unaffected. */
rmdec_status rmdec_decode(rmdec_t h, const void *llr_dev, int64_t n_frames, uint32_t *bits_out_dev,
                          void *stream);

/* As rmdec_decode, plus optional per-frame diagnostics (any may be NULL), all device:
 * cw_out_dev [n_frames][ceil(N/32)] uint32 the selected codeword x; pm_out_dev [n_frames]
 * float its path metric (equal to its correlation discrepancy with the channel LLRs);
 * best_out_dev [n_frames] int32 the decoder (p-FHT-FSCL) or permutation (Aut-SSC) that won. */
rmdec_status rmdec_decode_debug(rmdec_t h, const void *llr_dev, int64_t n_frames, uint32_t *bits_out_dev,
                                uint32_t *cw_out_dev, float *pm_out_dev, int32_t *best_out_dev, void *stream);

/* End-to-end decode from and to HOST memory: copies the LLRs in, decodes, copies the bits
 * out, and returns after the work has completed. Decoding and the copy back run on `stream`;
 * batches of 16 or more waves of the launch shape are uploaded in 2-8 chunks on a
 * handle-owned copy stream that runs ahead of the decodes (each chunk's decode waits for its
 * upload), so uploads overlap decoding. Pinned host buffers give full copy bandwidth and the
 * overlap; pageable ones work but are staged by the driver. Uses a handle-owned device
 * staging area grown on demand. */
rmdec_status rmdec_decode_host(rmdec_t h, const void *llr_host, int64_t n_frames, uint32_t *bits_out_host,
                               void *stream);

/* Asynchronous submission: enqueues rmdec_decode on `stream`, records a completion event and
 * returns a ticket (> 0). The caller keeps the buffers alive until rmdec_poll reports
 * completion. At most 1024 tickets may be outstanding per handle (RMDEC_EBUSY beyond).
 * Not part of the paper's method (which decodes one received word at a time): an interface
 * for callers that overlap decoding with other work; the decode itself is rmdec_decode's. */
rmdec_status rmdec_submit(rmdec_t h, const void *llr_dev, int64_t n_frames, uint32_t *bits_out_dev,
                          void *stream, uint64_t *ticket);

/* Waits up to timeout_us microseconds (0 = just check) for a ticket. Returns RMDEC_OK once
 * complete (the ticket is then retired), RMDEC_EBUSY if timeout_us == 0 and not complete,
 * RMDEC_ETIMEDOUT if the wait expired, RMDEC_EINVAL for an unknown ticket. Host-side only
 * (an event query, then sleeps of 20 us); no device code waits. Not part of the paper's
 * method: the completion half of rmdec_submit. */
rmdec_status rmdec_poll(rmdec_t h, uint64_t ticket, int64_t timeout_us);

/* Launch shape: warps per CTA (1..20, at most P; Aut-SSC handles use at most 4; the decoders
 * of a frame are split across a CTA's warps; path-per-thread kernels (rmdec_set_kernel) take
 * 1..4 warps, which split the decoder batches of the CTA's frames) and a cap on resident CTAs per SM (0 = the
 * occupancy limit); 0 warps = the default: for path-per-thread kernels one warp per decoder
 * batch of a frame (up to four); for p-FHT-FSCL kernels whose CTA decodes one frame,
 * 4 (else 3, else 2) warps when that splits the P decoders evenly and keeps at least two thirds
 * of the most resident warps per SM; otherwise the most resident warps per SM, then warps that
 * split the P decoders evenly, then two or more decoders per warp and two or more CTAs per
 * SM, then the narrowest CTA; a launch of at most four waves of that shape takes the shape
 * with the fewest waves x rounds of decoders per warp instead (wider CTAs run more of each
 * frame's decoders at once; see also rmdec_autotune). A shape
 * whose shared memory does not fit fails the next decode with RMDEC_EINVAL. Takes effect on
 * the next decode. Not part of the paper's method: it only changes scheduling, never
 * results. */
rmdec_status rmdec_set_tuning(rmdec_t h, int warps_per_cta, int ctas_per_sm);
rmdec_status rmdec_get_tuning(rmdec_t h, int *warps_per_cta, int *ctas_per_sm);

/* Times every candidate launch shape on n_frames synthetic frames (allocated and freed inside
 * this call; synchronous on `stream`) and keeps the fastest. With a non-NULL cache_path, a
 * choice stored there for the same device, code, P, L and dtype is reused without timing, and a
 * new choice is appended (one text line per entry). Call before any stream capture. */
rmdec_status rmdec_autotune(rmdec_t h, int64_t n_frames, const char *cache_path, void *stream);

/* A captured host-to-host decode pipeline for fixed buffers: copy n_frames LLRs from
 * llr_host, decode, copy the information bits to bits_out_host (layouts as in
 * rmdec_decode_host), recorded once as a CUDA graph and replayed with one launch. The graph
 * owns its device buffers; the host buffers must outlive it (pinned memory recommended). The
 * graph reads the handle's device tables at every replay: the handle must outlive the graph,
 * and a replay after rmdec_set_perms (and a decode that uploads the new tables) decodes with
 * the new permutations. The launch shape and LLR type are fixed at capture. */
typedef struct rmdec_graph *rmdec_graph_t;
rmdec_status rmdec_graph_create(rmdec_t h, const void *llr_host, int64_t n_frames, uint32_t *bits_out_host,
                                rmdec_graph_t *out);
/* Enqueues one replay on `stream` (asynchronous; synchronise the stream to read the bits). */
rmdec_status rmdec_graph_launch(rmdec_graph_t g, void *stream);
void rmdec_graph_destroy(rmdec_graph_t g);

/* Test hook for failure handling: the next n device allocations made by this library
 * (decoder tables, staging, graph and autotuning buffers, server arenas) fail as if the
 * device were out of memory, so that callers can exercise their RMDEC_ENOMEM paths without
 * exhausting a shared GPU; n = 0 disarms it. Process-wide. Not part of the paper's method. */
rmdec_status rmdec_debug_fail_device_allocs(int64_t n);

/* Decoding for callers that cannot allocate device memory. The paper has no counterpart:
 * this entry point exists for deployments, not for the method. Some callers may not call
 * cudaMalloc at decode time: code inside a framework whose caching allocator owns all device
 * memory, real-time loops that fix their memory budget at start-up, or plug-ins loaded into a
 * host process that forbids device allocations after initialisation. rmdec_decode allocates
 * the handle's permutation and position tables on the device at its first call; this call
 * instead uploads them, on `stream`, into one fixed device array that the library holds
 * (128 KiB, present on every GPU that loads the library until the process exits) and runs
 * the same decoder kernel. It calls no cudaMalloc, cudaFree or other allocating routine.
 * Arguments, layouts and results are those of rmdec_decode (llr_dev and bits_out_dev are
 * device buffers owned by the caller; llr_dev 16-byte aligned).
 * Limits and rules:
 *   - the decoder's tables must fit the array: per decoder 2 * (r-1) * 2L maps of 22 bytes for
 *     p-FHT-FSCL (one map of 22 bytes per permutation for Aut-SSC), plus 2K bytes of
 *     positions; larger configurations (e.g. RM(3,9) with P = 128, L = 8) return RMDEC_EINVAL
 *     and launch nothing;
 *   - the first call on each device looks up the array's device address (with that device
 *     current); make that first call before any stream capture;
 *   - every call shares the one array, which keeps the last call's tables: calls whose work
 *     overlaps on the GPU (other streams, other threads, other handles) race and may decode
 *     with another handle's tables. Issue them on one stream, or wait for the previous call.
 *   - the handle's launch-shape request (rmdec_set_tuning) is honoured; diagnostics outputs
 *     are not offered. */
rmdec_status rmdec_decode_noalloc(rmdec_t h, const void *llr_dev, int64_t n_frames, uint32_t *bits_out_dev,
                                  void *stream);

/* Per-thread description of the last failure on this handle (or of the last failed create
 * when h is NULL). Never NULL; valid until the next call on the same handle. */
const char *rmdec_last_error(rmdec_t h);

#ifdef __cplusplus
}
#endif

#endif /* RMDEC_H */
