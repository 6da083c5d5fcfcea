// C-ABI of the rmdec library: handle management, permutation tables, kernel dispatch and
// the asynchronous ticket interface. See include/rmdec.h for the contract of each call.
#include <atomic>
#include <cerrno>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <thread>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/rmdec.h"
#include "pfht_kernel.cuh"
#include "rmdec_internal.h"

namespace {

constexpr int kMaxM = 10;
constexpr int kRec = 11;
constexpr uint32_t kPermTag = 0x5045524Du;     // 'PERM'
constexpr uint32_t kSscStream = 0x53534300u;   // 'SSC\0'
constexpr int kMaxTickets = 1024;
constexpr int kHostChunks = 8;  // rmdec_decode_host: chunks of a large batch (upload/decode overlap)

// ------------------------------------------------------------ Philox4x32-10 ---
// Counter-based generator of Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of two
// 32x32->64 multiplies with the round keys bumped by the Weyl constants between rounds.
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    memcpy(out, c, sizeof c);
}

int gf2_rank(const uint16_t* cols, int s) {
    uint16_t v[kMaxM];
    memcpy(v, cols, sizeof(uint16_t) * s);
    int rank = 0;
    for (int bit = 0; bit < s && rank < s; bit++) {
        int piv = -1;
        for (int i = rank; i < s; i++)
            if ((v[i] >> bit) & 1) { piv = i; break; }
        if (piv < 0) continue;
        std::swap(v[rank], v[piv]);
        for (int i = 0; i < s; i++)
            if (i != rank && ((v[i] >> bit) & 1)) v[i] ^= v[rank];
        rank++;
    }
    return rank;
}

// Element of GA(s): draw a = 0, 1, ... with counter (stream, q, a, 'PERM') until the s x s
// matrix of bits [t*s, (t+1)*s) (column t) is invertible; b is bits [s*s, s*s + s).
void sample_ga(int s, uint64_t seed, uint32_t stream, uint32_t q, uint16_t* rec) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t a = 0;; a++) {
        const uint32_t ctr[4] = {stream, q, a, kPermTag};
        uint32_t w[4];
        philox4x32_10(ctr, key, w);
        auto bit = [&](int i) { return (w[i >> 5] >> (i & 31)) & 1u; };
        uint16_t r[kRec] = {0};
        for (int t = 0; t < s; t++)
            for (int i = 0; i < s; i++) r[t] |= (uint16_t)(bit(t * s + i) << i);
        for (int i = 0; i < s; i++) r[kMaxM] |= (uint16_t)(bit(s * s + i) << i);
        if (gf2_rank(r, s) == s) {
            memcpy(rec, r, sizeof r);
            return;
        }
    }
}

bool record_valid(const uint16_t* r, int s) {
    for (int t = s; t < kMaxM; t++)
        if (r[t]) return false;
    for (int t = 0; t < s; t++)
        if (r[t] >> s) return false;
    if (r[kMaxM] >> s) return false;
    return gf2_rank(r, s) == s;
}

// sigma = outer o inner as a record: sigma(i) = outer(inner(i)).
void compose(const uint16_t* outer, const uint16_t* inner, int s, uint16_t* out) {
    auto lin = [&](int v) {
        int o = 0;
        for (int t = 0; t < s; t++)
            if ((v >> t) & 1) o ^= outer[t];
        return o;
    };
    memset(out, 0, sizeof(uint16_t) * kRec);
    for (int t = 0; t < s; t++) out[t] = (uint16_t)lin(inner[t]);
    out[kMaxM] = (uint16_t)(lin(inner[kMaxM]) ^ outer[kMaxM]);
}

// Inverse of the invertible affine map x -> A x ^ b of GF(2)^s as a record:
// x -> A^-1 x ^ A^-1 b (Gauss-Jordan elimination on the rows of [A | I]).
void invert(const uint16_t* r, int s, uint16_t* out) {
    uint32_t row[kMaxM];
    for (int i = 0; i < s; i++) {
        uint32_t a = 0;
        for (int t = 0; t < s; t++) a |= (uint32_t)((r[t] >> i) & 1u) << t;  // A[i][t] = bit i of column t
        row[i] = a | (1u << (s + i));
    }
    for (int col = 0; col < s; col++) {
        int piv = col;
        while (!((row[piv] >> col) & 1u)) piv++;  // exists: A is invertible
        std::swap(row[col], row[piv]);
        for (int i = 0; i < s; i++)
            if (i != col && ((row[i] >> col) & 1u)) row[i] ^= row[col];
    }
    memset(out, 0, sizeof(uint16_t) * kRec);
    for (int t = 0; t < s; t++)
        for (int i = 0; i < s; i++) out[t] |= (uint16_t)(((row[i] >> (s + t)) & 1u) << i);
    uint16_t v = 0;
    for (int t = 0; t < s; t++)
        if ((r[kMaxM] >> t) & 1u) v ^= out[t];
    out[kMaxM] = v;
}

int n_perm_levels(int m, int r) { return (1 < r && r < m - 1) ? r - 1 : 0; }

thread_local std::string g_create_error;
std::atomic<int64_t> g_failing_allocs{0};  // device allocations still to fail (test hook)

}  // namespace

struct rmdec_ctx {
    int algo = 0;  // 0: p-FHT-FSCL-L-P, 1: Aut-SSC-P, 2: p-FHT-FSCL of RM(1, m) or RM(m-1, m)
    bool single_start = false;  // FHT-FSCL: identity permutations, one live initial path
    int m = 0, r = 0, P = 0, L = 1, n = 0, k = 0;
    rmdec_dtype dtype = RMDEC_LLR_F32;
    rmdec_hadamard hadamard = RMDEC_HADAMARD_SHUFFLE;
    rmdec_kernel kernel = RMDEC_KERNEL_AUTO;
    std::vector<uint16_t> perms;  // host table in the documented layout
    std::vector<int> info;
    bool dirty = true;
    int device = -1;
    uint16_t* d_recs = nullptr;
    uint16_t* d_info = nullptr;
    rmdec_host::KernelEntry kern;
    // RMDEC_KERNEL_AUTO: the path-per-thread kernel, used for launches of at least
    // kern_path.min_frames frames (fn null: none), and its launch shape
    rmdec_host::KernelEntry kern_path;
    int path_warps = 1, path_blocks_per_sm = 0;
    size_t path_smem = 0;
    int warps = 4;
    int req_warps = 0, req_ctas = 0;  // requested launch shape (0 = default)
    bool shape_dirty = true;
    int sm_count = 0;
    int blocks_per_sm = 0;
    size_t smem = 0;
    bool auto_shape = true;          // shape chosen by configure_shape's default rule
    std::vector<int> occ_w;          // resident CTAs per SM for W = 1.. warps per CTA (0: not resident)
    std::vector<size_t> smem_w;      // dynamic shared memory for W warps per CTA
    void* d_stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t copy_stream = nullptr;       // rmdec_decode_host's uploads of large batches
    cudaEvent_t chunk_ev[kHostChunks + 1] = {};  // per-chunk upload done; [kHostChunks]: start
    std::map<uint64_t, cudaEvent_t> tickets;
    uint64_t next_ticket = 1;
    std::string err;

    rmdec_status fail(rmdec_status st, const char* fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        err = buf;
        return st;
    }
    rmdec_status cuda_fail(cudaError_t e, const char* what) {
        return fail(RMDEC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    }
    int records_per_decoder() const { return algo != 1 ? L + n_perm_levels(m, r) * 2 * L : 1; }
    int64_t n_records() const { return algo != 1 ? (int64_t)P * records_per_decoder() : P; }
    int record_size(int q) const {  // GA(s) of record q within a decoder
        if (algo == 1 || q < L) return m;
        return m - (q - L) / (2 * L);
    }
};

namespace {

size_t llr_elem_bytes(rmdec_dtype t) {
    switch (t) {
        case RMDEC_LLR_F32: return 4;
        case RMDEC_LLR_I8: return 1;
        case RMDEC_LLR_F16: return 2;
        case RMDEC_LLR_I16: return 2;
    }
    return 4;
}

bool lookup_kernel(rmdec_ctx* h, rmdec_host::KernelEntry* e) {
    using namespace rmdec_host;
    *e = KernelEntry();  // the per-kernel lookups fill only the fields their kind uses
    if (h->algo == 1) return lookup_autssc(h->m, h->r, e);
    if (h->algo == 2) return lookup_mlroot(h->m, h->r, e);
    if (h->hadamard == RMDEC_HADAMARD_TENSOR) return lookup_pfht_tc(h->m, h->r, h->L, e);
    if (h->kernel == RMDEC_KERNEL_PATH) return lookup_pfht_ppt(h->m, h->r, h->L, h->P, e);
    if (h->L == 32) {
        if (h->m == 9) return lookup_pfht_l32_m9(h->r, e);
        if (h->m == 8) return lookup_pfht_l32_m8(h->r, e);
        return lookup_pfht_l32_small(h->m, h->r, e);
    }
    if (h->r == 4) return h->m == 9 ? lookup_pfht_r4_m9(h->L, e) : lookup_pfht_r4_small(h->m, h->L, e);
    switch (h->m) {
        case 4: return lookup_pfht_m4(h->r, h->L, e);
        case 5: return lookup_pfht_m5(h->r, h->L, e);
        case 6: return lookup_pfht_m6(h->r, h->L, e);
        case 7: return lookup_pfht_m7(h->r, h->L, e);
        case 8: return lookup_pfht_m8(h->r, h->L, e);
        case 9: return lookup_pfht_m9(h->r, h->L, e);
        case 10: return lookup_pfht_m10(h->r, h->L, e);
    }
    return false;
}

// RMDEC_KERNEL_AUTO: the path-per-thread kernel that takes the larger launches, if any.
bool lookup_path_alternative(rmdec_ctx* h, rmdec_host::KernelEntry* e) {
    *e = rmdec_host::KernelEntry();
    if (h->algo != 0 || h->kernel != RMDEC_KERNEL_AUTO || h->hadamard != RMDEC_HADAMARD_SHUFFLE) return false;
    if (!rmdec_host::lookup_pfht_ppt(h->m, h->r, h->L, h->P, e)) return false;
    if (!e->auto_ok) *e = rmdec_host::KernelEntry();  // slower for this P and L: not by default
    return e->fn != nullptr;
}

// Device records: p-FHT-FSCL: per decoder, level 0 holds the 2L root candidates composed with
// the initial permutation of their source path (pi^init_{c mod L} o pi_c, one GA(m) element, since
// every root path starts from the same channel LLRs), levels 1.. hold the 2L candidates as given;
// then the inverse of each of these maps in the same order (the kernel un-permutes decided
// words by gathering through them).
std::vector<uint16_t> device_records(const rmdec_ctx* h) {
    std::vector<uint16_t> out;
    if (h->algo == 1) return h->perms;
    const int rpd = h->records_per_decoder(), nlev = n_perm_levels(h->m, h->r), L = h->L;
    const size_t nrec = (size_t)nlev * 2 * L;  // maps per decoder
    out.resize((size_t)h->P * 2 * nrec * kRec);
    for (int p = 0; p < h->P; p++) {
        const uint16_t* base = h->perms.data() + (size_t)p * rpd * kRec;
        uint16_t* dst = out.data() + (size_t)p * 2 * nrec * kRec;
        for (int lev = 0; lev < nlev; lev++)
            for (int c = 0; c < 2 * L; c++) {
                const uint16_t* cand = base + (size_t)(L + lev * 2 * L + c) * kRec;
                const size_t q = (size_t)lev * 2 * L + c;
                uint16_t* o = dst + q * kRec;
                if (lev == 0) compose(base + (size_t)(c % L) * kRec, cand, h->m, o);
                else memcpy(o, cand, sizeof(uint16_t) * kRec);
                invert(o, h->m - lev, dst + (nrec + q) * kRec);
            }
    }
    return out;
}

rmdec_status ensure_device(rmdec_ctx* h) {
    if (!h->dirty) return RMDEC_OK;
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return h->fail(RMDEC_EDEVICE, "no CUDA device: %s", cudaGetErrorString(e));
    if (!lookup_kernel(h, &h->kern)) return h->fail(RMDEC_EINVAL, "no kernel for m=%d r=%d L=%d", h->m, h->r, h->L);
    lookup_path_alternative(h, &h->kern_path);
    if ((e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return h->cuda_fail(e, "cudaDeviceGetAttribute");
    std::vector<uint16_t> recs = device_records(h);
    if (h->d_recs && h->d_info && h->device == dev) {
        // The table sizes are fixed per handle, so new permutations (rmdec_set_perms) go into
        // the existing buffers: pointers that captured graphs and grouped launches hold stay
        // valid and read the new tables. Wait until every queued use of the old ones is done.
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return h->cuda_fail(e, "synchronize before table update");
    } else {
        if (h->d_recs) cudaFree(h->d_recs);
        if (h->d_info) cudaFree(h->d_info);
        h->d_recs = nullptr;
        h->d_info = nullptr;
        if ((e = rmdec_host::device_alloc(reinterpret_cast<void**>(&h->d_recs), std::max<size_t>(recs.size(), 1) * 2)) != cudaSuccess) return h->fail(RMDEC_ENOMEM, "cudaMalloc records: %s", cudaGetErrorString(e));
        if ((e = rmdec_host::device_alloc(reinterpret_cast<void**>(&h->d_info), std::max<size_t>(h->info.size(), 1) * 2)) != cudaSuccess) return h->fail(RMDEC_ENOMEM, "cudaMalloc info: %s", cudaGetErrorString(e));
    }
    std::vector<uint16_t> info16(h->info.begin(), h->info.end());
    if ((e = cudaMemcpy(h->d_recs, recs.data(), recs.size() * 2, cudaMemcpyHostToDevice)) != cudaSuccess) return h->cuda_fail(e, "upload records");
    if ((e = cudaMemcpy(h->d_info, info16.data(), info16.size() * 2, cudaMemcpyHostToDevice)) != cudaSuccess) return h->cuda_fail(e, "upload info");
    h->shape_dirty = true;
    h->device = dev;
    h->dirty = false;
    return RMDEC_OK;
}

// p-FHT-FSCL kernels whose CTA decodes one frame at a time with all its warps (the P
// decoders split across them); the other kernels give each warp frames of its own.
bool block_per_frame(const rmdec_ctx* h, const rmdec_host::KernelEntry& k) { return h->algo == 0 && !k.frames_per_warp; }

// Widest CTA a handle's kernel accepts: pfht_kernel is built for up to kMaxWarps warps, and
// more warps than decoders would idle.
int max_warps_per_cta(const rmdec_ctx* h, const rmdec_host::KernelEntry& k) {
    if (h->algo == 2) return 8;           // one frame per warp
    if (k.frames_per_warp) return 4;      // path-per-thread kernels: up to 128 threads
    return h->algo == 0 ? std::min(h->P, rmdec_dev::kMaxWarps) : 4;
}

// Default warps per CTA, given the resident CTAs occ_for(W) of each width W <= wmax.
// Path-per-thread kernels: one.
// Warp-per-decoder kernels, whose CTA decodes one frame with all its warps: four warps (else three, else two)
// when that width splits the P decoders evenly and keeps at least two thirds of the most
// resident warps. Its warps run their decoders in lockstep (a block barrier at every leaf),
// which keeps them on the same code; the trees of the longer codes exceed the instruction
// caches, so this pays more than the last resident warps. Measured (M frames/s, FP32, L = 4;
// the narrowest-CTA default that preceded it in parentheses): RM(2,9) P=20 6.46 at 4 x 5 (the
// same shape), RM(3,9) P=20 2.90 (2.73 at 2 x 10), RM(3,9) P=8 7.11 (6.65), RM(3,8) P=8 12.86
// (12.15 at 1 x 20), RM(2,10) P=8 5.93 (5.35 at 2 x 5), RM(3,10) P=8 2.79 (2.28 at 6 x 2); no
// other width was more than 6% faster on any of 15 codes and list sizes.
// Otherwise, and for the kernels that decode one frame per warp: the most resident
// warps per SM; among equals, widths that split the P decoders evenly, then at least two
// decoders per warp and two or more CTAs per SM (a lone decoder per warp, or a lone CTA,
// leaves the SM idle at every frame boundary), then the narrowest CTA.
template <typename Occ>
int default_warps(const rmdec_ctx* h, const rmdec_host::KernelEntry& k, int wmax, Occ occ_for) {
    // path-per-thread kernels: one warp per CTA (measured: splitting a frame's decoder batches
    // over the warps of a CTA shortens a lone frame's wait but lowers the throughput of large
    // launches, which are the ones these kernels take; RM(2,8) P=20 L=4, 65,536 frames: 5.30 ms
    // at one warp, 8.52 ms at four)
    if (k.frames_per_warp) return 1;
    const bool bpf = block_per_frame(h, k);
    int most = 0;
    for (int c = 1; c <= wmax; c++) most = std::max(most, occ_for(c) * c);
    if (bpf)
        for (int c : {4, 3, 2})
            if (c <= wmax && h->P % c == 0 && 3 * occ_for(c) * c >= 2 * most) return c;
    auto score = [&](int c) {
        const int occ = occ_for(c);
        const bool even = !bpf || h->P % c == 0;
        const bool two_each = !bpf || h->P >= 2 * c;
        return std::make_tuple(occ * c, even, two_each, occ >= 2, -c);
    };
    auto best = score(1);
    int W = 1;
    for (int c = 2; c <= wmax; c++)
        if (score(c) > best) {
            best = score(c);
            W = c;
        }
    return W;
}

// Launch shape: warps per CTA (decoders of a frame split across warps) and resident CTAs.
rmdec_status configure_shape(rmdec_ctx* h) {
    if (!h->shape_dirty) return RMDEC_OK;
    cudaError_t e;
    int max_optin = 0;
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    // permit the device maximum so that handles of different sizes sharing this kernel can
    // launch in any order
    if ((e = cudaFuncSetAttribute(h->kern.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin)) != cudaSuccess)
        return h->cuda_fail(e, "cudaFuncSetAttribute");
    const int wmax = max_warps_per_cta(h, h->kern);
    auto smem_for = [&](int W) { return (size_t)h->kern.fixed_bytes(h->P, h->k, W) + 16 + (size_t)W * h->kern.warp_bytes; };
    auto occ_for = [&](int W) {
        int o = 0;
        if (smem_for(W) > (size_t)max_optin) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, h->kern.fn, 32 * W, smem_for(W)) != cudaSuccess) return 0;
        return o;
    };
    h->occ_w.assign(wmax + 1, 0);
    h->smem_w.assign(wmax + 1, 0);
    for (int c = 1; c <= wmax; c++) {
        h->occ_w[c] = occ_for(c);
        h->smem_w[c] = smem_for(c);
    }
    int W = h->req_warps;
    if (!W)
        if (const char* s = getenv("RMDEC_WARPS")) W = atoi(s);
    h->auto_shape = W == 0;
    if (!W) W = default_warps(h, h->kern, wmax, occ_for);
    W = std::max(1, std::min(wmax, W));
    h->warps = W;
    h->smem = smem_for(W);
    if ((int)h->smem > max_optin) return h->fail(RMDEC_EINVAL, "configuration needs %zu B shared memory (max %d)", h->smem, max_optin);
    const int occ = occ_for(W);
    if (occ < 1) return h->fail(RMDEC_EINVAL, "kernel cannot be resident (smem %zu)", h->smem);
    h->blocks_per_sm = h->req_ctas ? std::min(h->req_ctas, occ) : occ;
    if (h->kern_path.fn) {
        // the path-per-thread alternative: the requested width (at most its four warps) or one
        const rmdec_host::KernelEntry& k = h->kern_path;
        if ((e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin)) != cudaSuccess)
            return h->cuda_fail(e, "cudaFuncSetAttribute");
        const int pw = h->req_warps ? std::max(1, std::min(max_warps_per_cta(h, k), h->req_warps)) : 1;
        const size_t ps = (size_t)k.fixed_bytes(h->P, h->k, pw) + 16 + (size_t)pw * k.warp_bytes;
        int po = 0;
        if (ps > (size_t)max_optin || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&po, k.fn, 32 * pw, ps) != cudaSuccess) po = 0;
        if (po < 1) {
            h->kern_path = rmdec_host::KernelEntry();  // not resident: the warp kernel takes every launch
        } else {
            h->path_warps = pw;
            h->path_smem = ps;
            h->path_blocks_per_sm = h->req_ctas ? std::min(h->req_ctas, po) : po;
        }
    }
    h->shape_dirty = false;
    return RMDEC_OK;
}

rmdec_status launch(rmdec_ctx* h, const void* llr, int64_t n_frames, uint32_t* bits, uint32_t* cw, float* pm,
                    int32_t* best, cudaStream_t stream) {
    if (n_frames < 0) return h->fail(RMDEC_EINVAL, "n_frames < 0");
    if (n_frames == 0) return RMDEC_OK;
    if (!llr || !bits) return h->fail(RMDEC_EINVAL, "null llr or output pointer");
    if (reinterpret_cast<uintptr_t>(llr) % 16) return h->fail(RMDEC_EINVAL, "llr buffer must be 16-byte aligned");
    rmdec_status st = ensure_device(h);
    if (st == RMDEC_OK) st = configure_shape(h);
    if (st != RMDEC_OK) return st;
    if (h->kern_path.fn && n_frames >= h->kern_path.min_frames) {
        // large launches of short codes: the path-per-thread kernel (see lookup_pfht_ppt)
        rmdec_dev::LaunchArgs a;
        a.llr = llr;
        a.dtype = (int)h->dtype;
        a.qclamp = (float)((1 << (24 - h->m)) - 1);
        a.n_frames = n_frames;
        a.P = h->P;
        a.recs = h->d_recs;
        a.info = h->d_info;
        a.K = h->k;
        a.info_out = bits;
        a.cw_out = cw;
        a.pm_out = pm;
        a.best_out = best;
        a.single_start = h->single_start ? 1 : 0;
        const int64_t want = (n_frames + h->kern_path.frames_per_warp - 1) / h->kern_path.frames_per_warp;
        const unsigned grid = (unsigned)std::min<int64_t>(want, (int64_t)h->sm_count * h->path_blocks_per_sm);
        void* args[] = {&a};
        nvtxRangePushA("rmdec_decode pfht path-per-thread");
        cudaError_t e = cudaLaunchKernel(h->kern_path.fn, dim3(grid), dim3(32 * h->path_warps), args, h->path_smem, stream);
        nvtxRangePop();
        if (e != cudaSuccess) return h->cuda_fail(e, "kernel launch");
        return RMDEC_OK;
    }
    // Launches of a few waves: the last, partial wave costs a whole frame's worth of decoder
    // rounds (P / W decoders one after another per warp), so such launches take the shape
    // that minimises waves x rounds (ties: the default shape). Larger launches keep the
    // default, whose per-warp throughput is measured best.
    int W = h->warps, per_sm = h->blocks_per_sm;
    size_t smem = h->smem;
    const int64_t cap0 = (int64_t)h->sm_count * h->blocks_per_sm;
    if (h->auto_shape && !h->req_ctas && block_per_frame(h, h->kern) && n_frames <= 4 * cap0) {
        auto cost = [&](int c) {
            const int64_t cap = (int64_t)h->sm_count * h->occ_w[c];
            return ((n_frames + cap - 1) / cap) * (int64_t)((h->P + c - 1) / c);
        };
        int64_t best = cost(W);
        for (int c = 1; c < (int)h->occ_w.size(); c++) {
            if (h->occ_w[c] <= 0 || c == h->warps) continue;
            const int64_t v = cost(c);
            if (v < best) {
                best = v;
                W = c;
                per_sm = h->occ_w[c];
                smem = h->smem_w[c];
            }
        }
    }
    rmdec_dev::LaunchArgs a;
    a.llr = llr;
    a.dtype = (int)h->dtype;
    a.qclamp = (float)((1 << (24 - h->m)) - 1);
    a.n_frames = n_frames;
    a.P = h->P;
    a.recs = h->d_recs;
    a.info = h->d_info;
    a.K = h->k;
    a.info_out = bits;
    a.cw_out = cw;
    a.pm_out = pm;
    a.best_out = best;
    a.single_start = h->single_start ? 1 : 0;
    const int64_t cap = (int64_t)h->sm_count * per_sm;
    // p-FHT-FSCL and Aut-SSC CTAs take one frame at a time; the first-order/parity-check root
    // kernel decodes one frame per warp, the path-per-thread kernel frames_per_warp per CTA
    int64_t want = n_frames;
    if (h->algo == 2) want = (n_frames + W - 1) / W;
    else if (h->kern.frames_per_warp) want = (n_frames + h->kern.frames_per_warp - 1) / h->kern.frames_per_warp;
    const unsigned grid = (unsigned)std::min<int64_t>(want, cap);
    void* args[] = {&a};
    nvtxRangePushA(h->algo == 1 ? "rmdec_decode aut-ssc" : "rmdec_decode pfht");
    cudaError_t e = cudaLaunchKernel(h->kern.fn, dim3(grid), dim3(32 * W), args, smem, stream);
    nvtxRangePop();
    if (e != cudaSuccess) return h->cuda_fail(e, "kernel launch");
    return RMDEC_OK;
}

rmdec_status make_handle(rmdec_t* out, int algo, int m, int r, int P, int L, uint64_t seed) {
    if (!out) {
        g_create_error = "null output handle pointer";
        return RMDEC_EINVAL;
    }
    *out = nullptr;
    bool ml_root = false;  // RM(1, m) or RM(m-1, m): the root is an FHTL or SPCL node
    if (algo == 0) {
        ml_root = m >= 2 && m <= 10 && (r == 1 || r == m - 1);
        const bool pl_ok = P >= 1 && P <= 128 && L >= 1 && L <= (ml_root || m <= 9 ? 32 : 16) && (L & (L - 1)) == 0;
        const bool code_ok = ml_root || (m >= 4 && m <= 10 && r >= 2 && r <= 3 && r <= m - 2) ||
                             (r == 4 && m >= 6 && m <= 9);
        if (!code_ok || !pl_ok) {
            g_create_error = "unsupported p-FHT-FSCL configuration (need 1<=P<=128 and either 4<=m<=10, r in {2,3}, "
                             "r<=m-2, or 6<=m<=9, r=4, with L in {1,2,4,8,16} (32 for m<=9); or 2<=m<=10, "
                             "r in {1,m-1}, L in {1,2,4,8,16,32})";
            return RMDEC_EINVAL;
        }
    } else {
        if (m < 4 || m > 9 || r < 1 || r > 3 || r > m - 2 || P < 1 || P > 1024) {
            g_create_error = "unsupported Aut-SSC configuration (need 4<=m<=9, 1<=r<=min(3,m-2), 1<=P_ssc<=1024)";
            return RMDEC_EINVAL;
        }
    }
    rmdec_ctx* h = new (std::nothrow) rmdec_ctx;
    if (!h) {
        g_create_error = "host allocation failed";
        return RMDEC_ENOMEM;
    }
    h->algo = ml_root ? 2 : algo;
    h->m = m;
    h->r = r;
    h->P = P;
    h->L = algo == 0 ? L : 1;
    h->n = 1 << m;
    for (int i = 0; i < h->n; i++)
        if (__builtin_popcount((unsigned)i) >= m - r) h->info.push_back(i);
    h->k = (int)h->info.size();
    h->perms.assign((size_t)h->n_records() * kRec, 0);
    if (h->algo != 1) {
        const int rpd = h->records_per_decoder();
        for (int p = 0; p < P; p++)
            for (int q = 0; q < rpd; q++)
                sample_ga(h->record_size(q), seed, (uint32_t)p, (uint32_t)q, &h->perms[((size_t)p * rpd + q) * kRec]);
    } else {
        for (int q = 0; q < P; q++) sample_ga(m, seed, kSscStream, (uint32_t)q, &h->perms[(size_t)q * kRec]);
    }
    *out = h;
    return RMDEC_OK;
}

}  // namespace

namespace rmdec_host {
size_t llr_elem_bytes_of(rmdec_ctx* h) { return llr_elem_bytes(h->dtype); }

cudaError_t device_alloc(void** p, size_t bytes) {
    int64_t n = g_failing_allocs.load();
    while (n > 0)
        if (g_failing_allocs.compare_exchange_weak(n, n - 1)) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

rmdec_status member_info(rmdec_ctx* h, bool prepare, MemberInfo* out) {
    if (!h || !out) return RMDEC_EINVAL;
    if (prepare) {
        rmdec_status st = ensure_device(h);
        if (st == RMDEC_OK) st = configure_shape(h);
        if (st != RMDEC_OK) return st;
    }
    out->algo = h->algo;
    out->m = h->m;
    out->r = h->r;
    out->L = h->L;
    out->P = h->P;
    out->n = h->n;
    out->k = h->k;
    out->single = h->single_start ? 1 : 0;
    out->dtype = (int)h->dtype;
    out->hadamard = (int)h->hadamard;
    out->d_recs = h->dirty ? nullptr : h->d_recs;
    out->d_info = h->dirty ? nullptr : h->d_info;
    out->warp_bytes = h->dirty ? 0 : h->kern.warp_bytes;
    out->nrec = h->dirty ? 0 : h->kern.nrec;
    out->device = h->dirty ? -1 : h->device;
    out->wave = (h->dirty || h->shape_dirty) ? 0 : (int64_t)h->sm_count * h->blocks_per_sm;
    out->path_min_frames = h->dirty ? -1 : (h->kern.frames_per_warp ? 0 : (h->kern_path.fn ? h->kern_path.min_frames : -1));
    return RMDEC_OK;
}
}  // namespace rmdec_host

extern "C" {

rmdec_status rmdec_create(rmdec_t* out, int m, int r, int P, int L, uint64_t perm_seed) {
    return make_handle(out, 0, m, r, P, L, perm_seed);
}

rmdec_status rmdec_create_fhtfscl(rmdec_t* out, int m, int r, int L) {
    rmdec_status st = make_handle(out, 0, m, r, 1, L, 0);
    if (st != RMDEC_OK) return st;
    rmdec_ctx* h = *out;
    h->single_start = true;
    const int rpd = h->records_per_decoder();
    for (int q = 0; q < rpd; q++) {  // identity permutations: A = I, b = 0
        uint16_t* rec = &h->perms[(size_t)q * kRec];
        memset(rec, 0, sizeof(uint16_t) * kRec);
        for (int t = 0; t < h->record_size(q); t++) rec[t] = (uint16_t)(1u << t);
    }
    return RMDEC_OK;
}

rmdec_status rmdec_create_aut_ssc(rmdec_t* out, int m, int r, int P_ssc, uint64_t perm_seed) {
    return make_handle(out, 1, m, r, P_ssc, 1, perm_seed);
}

void rmdec_destroy(rmdec_t h) {
    if (!h) return;
    for (auto& kv : h->tickets) {
        cudaEventSynchronize(kv.second);
        cudaEventDestroy(kv.second);
    }
    if (h->d_recs) cudaFree(h->d_recs);
    if (h->d_info) cudaFree(h->d_info);
    if (h->d_stage) cudaFree(h->d_stage);
    if (h->copy_stream) {
        cudaStreamSynchronize(h->copy_stream);
        cudaStreamDestroy(h->copy_stream);
    }
    for (auto& ev : h->chunk_ev)
        if (ev) cudaEventDestroy(ev);
    delete h;
}

rmdec_status rmdec_set_dtype(rmdec_t h, rmdec_dtype t) {
    if (!h) return RMDEC_EINVAL;
    if (t != RMDEC_LLR_F32 && t != RMDEC_LLR_I8 && t != RMDEC_LLR_F16 && t != RMDEC_LLR_I16)
        return h->fail(RMDEC_EINVAL, "unknown dtype %d", (int)t);
    h->dtype = t;
    return RMDEC_OK;
}

rmdec_status rmdec_set_hadamard(rmdec_t h, rmdec_hadamard mode) {
    if (!h) return RMDEC_EINVAL;
    if (mode != RMDEC_HADAMARD_SHUFFLE && mode != RMDEC_HADAMARD_TENSOR)
        return h->fail(RMDEC_EINVAL, "unknown Hadamard mode %d", (int)mode);
    rmdec_host::KernelEntry e;
    if (mode == RMDEC_HADAMARD_TENSOR && (h->algo != 0 || !rmdec_host::lookup_pfht_tc(h->m, h->r, h->L, &e)))
        return h->fail(RMDEC_EINVAL, "no tensor-core Hadamard kernel for this decoder (RM(2|3, 9), L in {4, 8})");
    if (mode != h->hadamard) {
        h->hadamard = mode;
        h->dirty = true;  // the next decode looks up the kernel again
        h->shape_dirty = true;
    }
    return RMDEC_OK;
}

rmdec_status rmdec_set_kernel(rmdec_t h, rmdec_kernel kernel) {
    if (!h) return RMDEC_EINVAL;
    if (kernel != RMDEC_KERNEL_AUTO && kernel != RMDEC_KERNEL_WARP && kernel != RMDEC_KERNEL_PATH)
        return h->fail(RMDEC_EINVAL, "unknown kernel choice %d", (int)kernel);
    rmdec_host::KernelEntry e;
    if (kernel == RMDEC_KERNEL_PATH &&
        (h->algo != 0 || h->hadamard != RMDEC_HADAMARD_SHUFFLE || !rmdec_host::lookup_pfht_ppt(h->m, h->r, h->L, h->P, &e)))
        return h->fail(RMDEC_EINVAL, "no path-per-thread kernel for this decoder (RM(2, m), 4 <= m <= 8, or RM(3, m), 5 <= m <= 7; L <= 8)");
    if (kernel != h->kernel) {
        h->kernel = kernel;
        h->dirty = true;  // the next decode looks up the kernel again
        h->shape_dirty = true;
    }
    return RMDEC_OK;
}

rmdec_status rmdec_kernel_for(rmdec_t h, int64_t n_frames, rmdec_kernel* kernel) {
    if (!h || !kernel) return RMDEC_EINVAL;
    if (n_frames < 0) return h->fail(RMDEC_EINVAL, "n_frames < 0");
    rmdec_status st = ensure_device(h);
    if (st == RMDEC_OK) st = configure_shape(h);
    if (st != RMDEC_OK) return st;
    const bool path = h->kern.frames_per_warp != 0 || (h->kern_path.fn && n_frames >= h->kern_path.min_frames);
    *kernel = path ? RMDEC_KERNEL_PATH : RMDEC_KERNEL_WARP;
    return RMDEC_OK;
}

rmdec_status rmdec_perm_count(rmdec_t h, int64_t* n_records) {
    if (!h || !n_records) return RMDEC_EINVAL;
    *n_records = h->n_records();
    return RMDEC_OK;
}

rmdec_status rmdec_get_perms(rmdec_t h, uint16_t* perms_host, int64_t n_records) {
    if (!h) return RMDEC_EINVAL;
    if (!perms_host || n_records != h->n_records())
        return h->fail(RMDEC_EINVAL, "expected %lld records", (long long)h->n_records());
    memcpy(perms_host, h->perms.data(), h->perms.size() * sizeof(uint16_t));
    return RMDEC_OK;
}

rmdec_status rmdec_set_perms(rmdec_t h, const uint16_t* perms_host, int64_t n_records) {
    if (!h) return RMDEC_EINVAL;
    if (!perms_host || n_records != h->n_records())
        return h->fail(RMDEC_EINVAL, "expected %lld records", (long long)h->n_records());
    const int rpd = h->records_per_decoder();
    for (int64_t q = 0; q < n_records; q++)
        if (!record_valid(perms_host + q * kRec, h->record_size((int)(q % rpd))))
            return h->fail(RMDEC_EINVAL, "record %lld is not an invertible affine map of the right size", (long long)q);
    memcpy(h->perms.data(), perms_host, h->perms.size() * sizeof(uint16_t));
    h->dirty = true;
    return RMDEC_OK;
}

rmdec_status rmdec_info(rmdec_t h, int* n, int* k, const int** info_idx) {
    if (!h) return RMDEC_EINVAL;
    if (n) *n = h->n;
    if (k) *k = h->k;
    if (info_idx) *info_idx = h->info.data();
    return RMDEC_OK;
}

rmdec_status rmdec_decode(rmdec_t h, const void* llr_dev, int64_t n_frames, uint32_t* bits_out_dev, void* stream) {
    if (!h) return RMDEC_EINVAL;
    return launch(h, llr_dev, n_frames, bits_out_dev, nullptr, nullptr, nullptr, (cudaStream_t)stream);
}

rmdec_status rmdec_decode_debug(rmdec_t h, const void* llr_dev, int64_t n_frames, uint32_t* bits_out_dev,
                                uint32_t* cw_out_dev, float* pm_out_dev, int32_t* best_out_dev, void* stream) {
    if (!h) return RMDEC_EINVAL;
    return launch(h, llr_dev, n_frames, bits_out_dev, cw_out_dev, pm_out_dev, best_out_dev, (cudaStream_t)stream);
}

rmdec_status rmdec_decode_host(rmdec_t h, const void* llr_host, int64_t n_frames, uint32_t* bits_out_host, void* stream) {
    if (!h) return RMDEC_EINVAL;
    if (n_frames < 0 || (n_frames > 0 && (!llr_host || !bits_out_host))) return h->fail(RMDEC_EINVAL, "bad arguments");
    if (n_frames == 0) return RMDEC_OK;
    const size_t in_bytes = (size_t)n_frames * h->n * llr_elem_bytes(h->dtype);
    const size_t in_pad = (in_bytes + 255) / 256 * 256;
    const size_t out_bytes = (size_t)n_frames * ((h->k + 31) / 32) * 4;
    cudaError_t e;
    if (in_pad + out_bytes > h->stage_bytes) {
        if (h->d_stage) {
            cudaFree(h->d_stage);
            h->d_stage = nullptr;
            h->stage_bytes = 0;
        }
        if ((e = rmdec_host::device_alloc(&h->d_stage, in_pad + out_bytes)) != cudaSuccess)
            return h->fail(RMDEC_ENOMEM, "staging allocation of %zu bytes: %s", in_pad + out_bytes, cudaGetErrorString(e));
        h->stage_bytes = in_pad + out_bytes;
    }
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t* d_in = static_cast<uint8_t*>(h->d_stage);
    uint32_t* d_out = reinterpret_cast<uint32_t*>(d_in + in_pad);
    rmdec_status st = ensure_device(h);
    if (st == RMDEC_OK) st = configure_shape(h);
    if (st != RMDEC_OK) return st;
    // Large batches go in chunks of at least 8 waves: chunk c + 1 is uploaded on the handle's
    // copy stream while chunk c decodes on `stream`, each decode waiting for its chunk's upload.
    const int64_t wave = (int64_t)h->sm_count * h->blocks_per_sm;
    const int chunks = n_frames >= 64 * wave ? kHostChunks : n_frames >= 32 * wave ? 4 : n_frames >= 16 * wave ? 2 : 1;
    if (chunks == 1) {
        if ((e = cudaMemcpyAsync(d_in, llr_host, in_bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) return h->cuda_fail(e, "H2D");
        st = launch(h, d_in, n_frames, d_out, nullptr, nullptr, nullptr, s);
        if (st != RMDEC_OK) return st;
    } else {
        if (!h->copy_stream) {
            if ((e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking)) != cudaSuccess) return h->cuda_fail(e, "copy stream");
            for (auto& ev : h->chunk_ev)
                if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return h->cuda_fail(e, "chunk events");
        }
        // uploads start after the work already queued on `stream` (which may read the buffer)
        if ((e = cudaEventRecord(h->chunk_ev[kHostChunks], s)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(h->copy_stream, h->chunk_ev[kHostChunks], 0)) != cudaSuccess)
            return h->cuda_fail(e, "copy stream order");
        const size_t fb = (size_t)h->n * llr_elem_bytes(h->dtype), ow = (size_t)((h->k + 31) / 32);
        for (int c = 0; c < chunks; c++) {
            const int64_t f0 = n_frames * c / chunks, f1 = n_frames * (c + 1) / chunks;
            if ((e = cudaMemcpyAsync(d_in + (size_t)f0 * fb, static_cast<const uint8_t*>(llr_host) + (size_t)f0 * fb,
                                     (size_t)(f1 - f0) * fb, cudaMemcpyHostToDevice, h->copy_stream)) != cudaSuccess ||
                (e = cudaEventRecord(h->chunk_ev[c], h->copy_stream)) != cudaSuccess)
                return h->cuda_fail(e, "H2D");
        }
        for (int c = 0; c < chunks; c++) {
            const int64_t f0 = n_frames * c / chunks, f1 = n_frames * (c + 1) / chunks;
            if ((e = cudaStreamWaitEvent(s, h->chunk_ev[c], 0)) != cudaSuccess) return h->cuda_fail(e, "chunk order");
            st = launch(h, d_in + (size_t)f0 * fb, f1 - f0, d_out + (size_t)f0 * ow, nullptr, nullptr, nullptr, s);
            if (st != RMDEC_OK) return st;
        }
    }
    if ((e = cudaMemcpyAsync(bits_out_host, d_out, out_bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return h->cuda_fail(e, "D2H");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return h->cuda_fail(e, "synchronize");
    return RMDEC_OK;
}

rmdec_status rmdec_submit(rmdec_t h, const void* llr_dev, int64_t n_frames, uint32_t* bits_out_dev, void* stream,
                          uint64_t* ticket) {
    if (!h) return RMDEC_EINVAL;
    if (!ticket) return h->fail(RMDEC_EINVAL, "null ticket pointer");
    if ((int)h->tickets.size() >= kMaxTickets) return h->fail(RMDEC_EBUSY, "too many outstanding tickets");
    rmdec_status st = launch(h, llr_dev, n_frames, bits_out_dev, nullptr, nullptr, nullptr, (cudaStream_t)stream);
    if (st != RMDEC_OK) return st;
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return h->cuda_fail(e, "cudaEventCreate");
    if ((e = cudaEventRecord(ev, (cudaStream_t)stream)) != cudaSuccess) {
        cudaEventDestroy(ev);
        return h->cuda_fail(e, "cudaEventRecord");
    }
    const uint64_t t = h->next_ticket++;
    h->tickets[t] = ev;
    *ticket = t;
    return RMDEC_OK;
}

rmdec_status rmdec_poll(rmdec_t h, uint64_t ticket, int64_t timeout_us) {
    if (!h) return RMDEC_EINVAL;
    auto it = h->tickets.find(ticket);
    if (it == h->tickets.end()) return h->fail(RMDEC_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(it->second);
        if (e == cudaSuccess) {
            cudaEventDestroy(it->second);
            h->tickets.erase(it);
            return RMDEC_OK;
        }
        if (e != cudaErrorNotReady) return h->cuda_fail(e, "cudaEventQuery");
        if (timeout_us <= 0) return h->fail(RMDEC_EBUSY, "ticket %llu still running", (unsigned long long)ticket);
        const auto us = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
        if (us >= timeout_us) return h->fail(RMDEC_ETIMEDOUT, "ticket %llu not finished after %lld us", (unsigned long long)ticket, (long long)timeout_us);
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

rmdec_status rmdec_set_tuning(rmdec_t h, int warps_per_cta, int ctas_per_sm) {
    if (!h) return RMDEC_EINVAL;
    if (warps_per_cta < 0 || warps_per_cta > rmdec_dev::kMaxWarps || ctas_per_sm < 0 || ctas_per_sm > 32)
        return h->fail(RMDEC_EINVAL, "warps_per_cta must be 0..%d and ctas_per_sm 0..32", rmdec_dev::kMaxWarps);
    h->req_warps = warps_per_cta;
    h->req_ctas = ctas_per_sm;
    h->shape_dirty = true;
    return RMDEC_OK;
}

rmdec_status rmdec_get_tuning(rmdec_t h, int* warps_per_cta, int* ctas_per_sm) {
    if (!h) return RMDEC_EINVAL;
    rmdec_status st = ensure_device(h);
    if (st == RMDEC_OK) st = configure_shape(h);
    if (st != RMDEC_OK) return st;
    if (warps_per_cta) *warps_per_cta = h->warps;
    if (ctas_per_sm) *ctas_per_sm = h->blocks_per_sm;
    return RMDEC_OK;
}

rmdec_status rmdec_autotune(rmdec_t h, int64_t n_frames, const char* cache_path, void* stream) {
    if (!h) return RMDEC_EINVAL;
    if (n_frames < 1) return h->fail(RMDEC_EINVAL, "n_frames must be positive");
    rmdec_status st = ensure_device(h);
    if (st != RMDEC_OK) return st;
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, h->device);
    char key[512];
    snprintf(key, sizeof key, "%.200s|algo%d|m%d|r%d|P%d|L%d|dt%d|ppt%d", prop.name, h->algo, h->m, h->r, h->P, h->L,
             (int)h->dtype, h->kern.frames_per_warp ? 1 : 0);
    for (char* c = key; *c; c++)
        if (*c == ' ') *c = '_';
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            // one "key warps ctas" entry per line; the last entry for this key wins
            char k[512];
            int w = 0, c = 0, found = 0, fw = 0, fc = 0;
            while (fscanf(f, "%511s %d %d", k, &w, &c) == 3)
                if (!strcmp(k, key)) {
                    found = 1;
                    fw = w;
                    fc = c;
                }
            fclose(f);
            if (found) {
                h->req_warps = std::max(0, std::min(rmdec_dev::kMaxWarps, fw));
                h->req_ctas = std::max(0, std::min(32, fc));
                h->shape_dirty = true;
                return configure_shape(h);
            }
        }
    }
    // synthetic frames: BPSK-like LLRs (+-2 plus uniform noise) from a fixed xorshift stream
    const size_t eb = llr_elem_bytes(h->dtype);
    const size_t in_b = (size_t)n_frames * h->n * eb, out_b = (size_t)n_frames * ((h->k + 31) / 32) * 4;
    std::vector<uint8_t> host(in_b);
    uint64_t x = 0x9E3779B97F4A7C15ull;
    for (size_t i = 0; i < (size_t)n_frames * h->n; i++) {
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        const float v = ((x & 1) ? 2.f : -2.f) + (float)((x >> 11) % 4096) / 1024.f - 2.f;
        if (h->dtype == RMDEC_LLR_F32) memcpy(&host[i * 4], &v, 4);
        else if (h->dtype == RMDEC_LLR_I8) host[i] = (uint8_t)(int8_t)(v * 4.f);
        else if (h->dtype == RMDEC_LLR_I16) {
            const int16_t q = (int16_t)(v * 256.f);
            memcpy(&host[i * 2], &q, 2);
        } else {
            const __half hv = __float2half(v);
            memcpy(&host[i * 2], &hv, 2);
        }
    }
    void* d = nullptr;
    cudaError_t e = rmdec_host::device_alloc(&d, in_b + out_b + 256);
    if (e != cudaSuccess) return h->fail(RMDEC_ENOMEM, "autotune buffers: %s", cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t* din = static_cast<uint8_t*>(d);
    uint32_t* dout = reinterpret_cast<uint32_t*>(din + (in_b + 255) / 256 * 256);
    cudaMemcpy(din, host.data(), in_b, cudaMemcpyHostToDevice);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    int best_w = 0;
    const int wmax = max_warps_per_cta(h, h->kern);
    for (int w = 1; w <= wmax; w++) {
        h->req_warps = w;
        h->req_ctas = 0;
        h->shape_dirty = true;
        if (configure_shape(h) != RMDEC_OK) continue;
        launch(h, din, n_frames, dout, nullptr, nullptr, nullptr, s);  // warm-up
        cudaEventRecord(e0, s);
        for (int rep = 0; rep < 3; rep++) launch(h, din, n_frames, dout, nullptr, nullptr, nullptr, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best_w = w;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d);
    if ((e = cudaGetLastError()) != cudaSuccess) return h->cuda_fail(e, "autotune");
    if (!best_w) return h->fail(RMDEC_EINVAL, "no launch shape fits");
    h->req_warps = best_w;
    h->req_ctas = 0;
    h->shape_dirty = true;
    st = configure_shape(h);
    if (st == RMDEC_OK && cache_path) {
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "%s %d %d\n", key, best_w, 0);
            fclose(f);
        }
    }
    return st;
}

}  // extern "C"

struct rmdec_graph {
    rmdec_ctx* h = nullptr;
    void* dbuf = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

rmdec_status rmdec_graph_create(rmdec_t h, const void* llr_host, int64_t n_frames, uint32_t* bits_out_host,
                                rmdec_graph_t* out) {
    if (!h || !out) return RMDEC_EINVAL;
    *out = nullptr;
    if (n_frames < 1 || !llr_host || !bits_out_host) return h->fail(RMDEC_EINVAL, "bad graph buffers");
    rmdec_status st = ensure_device(h);
    if (st == RMDEC_OK) st = configure_shape(h);
    if (st != RMDEC_OK) return st;
    rmdec_graph* g = new (std::nothrow) rmdec_graph;
    if (!g) return RMDEC_ENOMEM;
    g->h = h;
    const size_t in_b = (size_t)n_frames * h->n * llr_elem_bytes(h->dtype), in_pad = (in_b + 255) / 256 * 256;
    const size_t out_b = (size_t)n_frames * ((h->k + 31) / 32) * 4;
    cudaError_t e = rmdec_host::device_alloc(&g->dbuf, in_pad + out_b);
    if (e != cudaSuccess) {
        delete g;
        return h->fail(RMDEC_ENOMEM, "graph buffers: %s", cudaGetErrorString(e));
    }
    uint8_t* din = static_cast<uint8_t*>(g->dbuf);
    uint32_t* dout = reinterpret_cast<uint32_t*>(din + in_pad);
    cudaStream_t cs;
    cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemcpyAsync(din, llr_host, in_b, cudaMemcpyHostToDevice, cs);
        st = launch(h, din, n_frames, dout, nullptr, nullptr, nullptr, cs);
        cudaMemcpyAsync(bits_out_host, dout, out_b, cudaMemcpyDeviceToHost, cs);
        e = cudaStreamEndCapture(cs, &g->graph);
    }
    if (e == cudaSuccess && st == RMDEC_OK) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess || st != RMDEC_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        cudaFree(g->dbuf);
        delete g;
        return st != RMDEC_OK ? st : h->cuda_fail(e, "graph capture");
    }
    *out = g;
    return RMDEC_OK;
}

rmdec_status rmdec_graph_launch(rmdec_graph_t g, void* stream) {
    if (!g) return RMDEC_EINVAL;
    const cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? RMDEC_OK : g->h->cuda_fail(e, "graph launch");
}

void rmdec_graph_destroy(rmdec_graph_t g) {
    if (!g) return;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    cudaFree(g->dbuf);
    delete g;
}

rmdec_status rmdec_debug_fail_device_allocs(int64_t n) {
    if (n < 0) return RMDEC_EINVAL;
    g_failing_allocs.store(n);
    return RMDEC_OK;
}

const char* rmdec_last_error(rmdec_t h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

}  // extern "C"

// ------------------------------------------------------ decoding without allocation ---
// rmdec_decode_noalloc reads the permutation maps and information positions from a table
// that the library holds in a fixed device array, instead of from the handle's own
// cudaMalloc'd tables, so that callers who must not allocate device memory can still decode.
constexpr size_t kNoAllocTableBytes = 128 * 1024;  // tables of P decoders + K positions
constexpr int kNoAllocMaxDevices = 64;

// The device copy of the tables: one per GPU that loads the library, held until exit.
static __device__ __align__(256) uint16_t g_noalloc_tables[kNoAllocTableBytes / 2];

namespace {

// The host image the tables are uploaded from. Every rmdec_decode_noalloc call overwrites
// it and the device copy.
uint16_t g_noalloc_host[kNoAllocTableBytes / 2];
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};  // device address of g_noalloc_tables per device

// The layout device_records() builds (per decoder its maps, then their inverses), written
// into a caller buffer of at least rec_words(h) elements.
size_t noalloc_rec_words(const rmdec_ctx* h) {
    if (h->algo == 1) return h->perms.size();
    return (size_t)h->P * 2 * n_perm_levels(h->m, h->r) * 2 * h->L * kRec;
}

void noalloc_write_records(const rmdec_ctx* h, uint16_t* out) {
    if (h->algo == 1) {
        memcpy(out, h->perms.data(), h->perms.size() * sizeof(uint16_t));
        return;
    }
    const int rpd = h->records_per_decoder(), nlev = n_perm_levels(h->m, h->r), L = h->L;
    const size_t nrec = (size_t)nlev * 2 * L;
    for (int p = 0; p < h->P; p++) {
        const uint16_t* base = h->perms.data() + (size_t)p * rpd * kRec;
        uint16_t* dst = out + (size_t)p * 2 * nrec * kRec;
        for (int lev = 0; lev < nlev; lev++)
            for (int c = 0; c < 2 * L; c++) {
                const uint16_t* cand = base + (size_t)(L + lev * 2 * L + c) * kRec;
                const size_t q = (size_t)lev * 2 * L + c;
                uint16_t* o = dst + q * kRec;
                if (lev == 0) compose(base + (size_t)(c % L) * kRec, cand, h->m, o);
                else memcpy(o, cand, sizeof(uint16_t) * kRec);
                invert(o, h->m - lev, dst + (nrec + q) * kRec);
            }
    }
}

}  // namespace

extern "C" rmdec_status rmdec_decode_noalloc(rmdec_t h, const void* llr_dev, int64_t n_frames,
                                             uint32_t* bits_out_dev, void* stream) {
    if (!h) return RMDEC_EINVAL;
    if (n_frames < 0) return h->fail(RMDEC_EINVAL, "n_frames < 0");
    if (n_frames == 0) return RMDEC_OK;
    if (!llr_dev || !bits_out_dev) return h->fail(RMDEC_EINVAL, "null llr or output pointer");
    if (reinterpret_cast<uintptr_t>(llr_dev) % 16) return h->fail(RMDEC_EINVAL, "llr buffer must be 16-byte aligned");
    const size_t rec_words = noalloc_rec_words(h);
    const size_t info_off = (rec_words + 7) / 8 * 8;  // 16-byte aligned start of the positions
    const size_t words = info_off + (size_t)h->k;
    if (words * sizeof(uint16_t) > kNoAllocTableBytes)
        return h->fail(RMDEC_EINVAL,
                       "rmdec_decode_noalloc: this decoder's tables need %zu bytes, above the fixed %zu-byte "
                       "table (use fewer decoders P or a smaller list size, or rmdec_decode)",
                       words * sizeof(uint16_t), kNoAllocTableBytes);
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return h->fail(RMDEC_EDEVICE, "no CUDA device: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return h->fail(RMDEC_EDEVICE, "device %d beyond the supported %d", dev, kNoAllocMaxDevices);
    rmdec_host::KernelEntry kern;
    if (!lookup_kernel(h, &kern)) return h->fail(RMDEC_EINVAL, "no kernel for m=%d r=%d L=%d", h->m, h->r, h->L);
    {
        rmdec_host::KernelEntry kp;  // the same kernel choice as rmdec_decode's
        if (lookup_path_alternative(h, &kp) && n_frames >= kp.min_frames) kern = kp;
    }
    int sms = 0, max_optin = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return h->cuda_fail(e, "cudaDeviceGetAttribute");
    if ((e = cudaFuncSetAttribute(kern.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin)) != cudaSuccess)
        return h->cuda_fail(e, "cudaFuncSetAttribute");
    // launch shape: the handle's requested one, else the default rule of rmdec_set_tuning
    const int wmax = max_warps_per_cta(h, kern);
    auto smem_for = [&](int W) { return (size_t)kern.fixed_bytes(h->P, h->k, W) + 16 + (size_t)W * kern.warp_bytes; };
    auto occ_for = [&](int W) {
        int o = 0;
        if (smem_for(W) > (size_t)max_optin) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern.fn, 32 * W, smem_for(W)) != cudaSuccess) return 0;
        return o;
    };
    int W = std::max(0, std::min(wmax, h->req_warps));
    if (!W) W = default_warps(h, kern, wmax, occ_for);
    const int occ = occ_for(W);
    if (occ < 1) return h->fail(RMDEC_EINVAL, "kernel cannot be resident with %d warps per CTA", W);
    const int per_sm = h->req_ctas ? std::min(h->req_ctas, occ) : occ;

    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        // once per device, with that device current: the device address of the table (the
        // array's name in host code is only a host-side stand-in for it)
        void* p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_noalloc_tables)) != cudaSuccess) return h->cuda_fail(e, "cudaGetSymbolAddress");
        g_noalloc_addr[dev] = p;
    }
    uint16_t* d_tab = static_cast<uint16_t*>(g_noalloc_addr[dev]);
    noalloc_write_records(h, g_noalloc_host);
    for (int i = 0; i < h->k; i++) g_noalloc_host[info_off + i] = (uint16_t)h->info[i];
    // a pageable source: the call returns once the driver has taken the bytes, so the host
    // image may be rewritten by the next call
    if ((e = cudaMemcpyAsync(d_tab, g_noalloc_host, words * sizeof(uint16_t), cudaMemcpyHostToDevice,
                             (cudaStream_t)stream)) != cudaSuccess)
        return h->cuda_fail(e, "table upload");
    rmdec_dev::LaunchArgs a;
    a.llr = llr_dev;
    a.dtype = (int)h->dtype;
    a.qclamp = (float)((1 << (24 - h->m)) - 1);
    a.n_frames = n_frames;
    a.P = h->P;
    a.recs = d_tab;
    a.info = d_tab + info_off;
    a.K = h->k;
    a.info_out = bits_out_dev;
    a.cw_out = nullptr;
    a.pm_out = nullptr;
    a.best_out = nullptr;
    a.single_start = h->single_start ? 1 : 0;
    const unsigned grid = (unsigned)std::min<int64_t>(n_frames, (int64_t)sms * per_sm);
    void* args[] = {&a};
    e = cudaLaunchKernel(kern.fn, dim3(grid), dim3(32 * W), args, smem_for(W), (cudaStream_t)stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "kernel launch");
    return RMDEC_OK;
}
