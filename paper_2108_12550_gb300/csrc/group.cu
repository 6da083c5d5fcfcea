// Host side of grouped multi-code decoding (see include/rmdec_group.h and group_kernel.cuh).
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/rmdec.h"
#include "../../include/rmdec_group.h"
#include "group_kernel.cuh"
#include "rmdec_internal.h"

namespace {
thread_local std::string g_group_create_error;

const void* group_fn(int L) {
    switch (L) {
        case 1: return rmdec_host::group_kernel_l1();
        case 2: return rmdec_host::group_kernel_l2();
        case 4: return rmdec_host::group_kernel_l4();
        case 8: return rmdec_host::group_kernel_l8();
    }
    return nullptr;
}
}  // namespace

struct rmdec_group {
    std::vector<rmdec_t> decs;
    int L = 0;
    const void* fn = nullptr;
    int device = -1;  // device the kernel attributes were set for
    int sm_count = 0, max_optin = 0;
    int req_warps = 0, req_ctas = 0;
    int64_t min_alone = 0;  // 0: half a wave of the decoder's own launch; < 0: never alone
    // resident CTAs per SM for 0..kMaxWarps warps (-1: not computed yet) at the footprint
    // (rec_cap, k_cap, n_cap, warp stride) of the last launch; occupancy queries cost host
    // time on every small launch otherwise
    int occ_key[4] = {-1, -1, -1, -1};
    int occ_cache[rmdec_dev::kMaxWarps + 1];
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
};

namespace {
// One or more group_kernel launches over the segments `order` (all non-empty).
rmdec_status launch_grouped(rmdec_group* g, const rmdec_segment* segs, std::vector<int>& order,
                            const std::vector<rmdec_host::MemberInfo>& mi, int dev, cudaStream_t st) {
    using namespace rmdec_dev;
    cudaError_t e;
    const int nd = (int)g->decs.size();
    std::vector<char> used(nd, 0);
    for (int i : order) used[segs[i].decoder] = 1;
    int rec_cap = 0, k_cap = 0, n_cap = 0, stride = 0;
    for (int d = 0; d < nd; d++) {
        if (!used[d]) continue;
        rec_cap = std::max(rec_cap, mi[d].P * mi[d].nrec * kRec);
        k_cap = std::max(k_cap, mi[d].k);
        n_cap = std::max(n_cap, mi[d].n);
        stride = std::max(stride, mi[d].warp_bytes);
    }
    auto cost = [&](int i) {
        const auto& m = mi[segs[i].decoder];
        return (double)m.P * m.L * m.n * (m.m + m.r);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });

    if (g->device != dev) {
        if ((e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&g->max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
            return g->fail(RMDEC_ECUDA, "device attributes: %s", cudaGetErrorString(e));
        if ((e = cudaFuncSetAttribute(g->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, g->max_optin)) != cudaSuccess)
            return g->fail(RMDEC_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        g->device = dev;
        std::fill(g->occ_key, g->occ_key + 4, -1);  // occupancies are per device
    }
    auto smem_for = [&](int W) { return (size_t)frame_fixed_bytes(rec_cap, k_cap, n_cap, W) + 16 + (size_t)W * stride; };
    const int key[4] = {rec_cap, k_cap, n_cap, stride};
    if (!std::equal(key, key + 4, g->occ_key)) {
        std::copy(key, key + 4, g->occ_key);
        std::fill(g->occ_cache, g->occ_cache + kMaxWarps + 1, -1);
    }
    auto occ_for = [&](int W) {
        int& o = g->occ_cache[W];
        if (o < 0) {
            o = 0;
            if (smem_for(W) <= (size_t)g->max_optin &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, g->fn, 32 * W, smem_for(W)) != cudaSuccess)
                o = 0;
        }
        return o;
    };
    int W = g->req_warps;
    if (!W) {
        int best = -1;
        for (int c = 1; c <= 4; c++) {
            const int warps = occ_for(c) * c;
            if (warps >= best) {
                best = warps;
                W = c;
            }
        }
    }
    // Launches of at most one wave of that shape take the shape that minimises the busiest
    // CTA's work instead: frames go round-robin over the grid, so a CTA decodes at most
    // ceil(n_s / grid) frames of segment s, each in ceil(P / W) rounds of one decoder of that
    // code. (Measured on four codes at 50 frames each: 0.072 against 0.113 ms in four
    // launches; at two or more waves the CTAs that finish early speed up the busiest one,
    // which this count ignores, and the default shape measured faster.)
    int64_t total_all = 0;
    for (int i : order) total_all += segs[i].n_frames;
    if (!g->req_warps && !g->req_ctas && total_all <= (int64_t)g->sm_count * occ_for(W)) {
        auto busiest = [&](int c) {
            const int o = occ_for(c);
            if (o < 1) return 1e300;
            const int64_t grid = std::min<int64_t>(total_all, (int64_t)g->sm_count * o);
            double t = 0;
            for (int i : order) {
                const auto& m = mi[segs[i].decoder];
                t += (double)((segs[i].n_frames + grid - 1) / grid) * ((m.P + c - 1) / c) * ((double)m.L * m.n * (m.m + m.r));
            }
            return t;
        };
        double best = busiest(W);
        for (int c = 1; c <= kMaxWarps; c++) {
            const double v = busiest(c);
            if (v < best) {
                best = v;
                W = c;
            }
        }
    }
    const int occ = occ_for(W);
    if (occ < 1) return g->fail(RMDEC_EINVAL, "group launch cannot be resident (%zu B shared memory)", smem_for(W));
    const int per_sm = g->req_ctas ? std::min(g->req_ctas, occ) : occ;

    static_assert(sizeof(GroupArgs) <= 32000, "kernel parameter space");
    GroupArgs a;
    memset(&a, 0, sizeof a);
    for (int d = 0; d < nd; d++) {
        if (!used[d]) continue;
        GroupDec& gd = a.dec[d];
        gd.recs = mi[d].d_recs;
        gd.info = mi[d].d_info;
        gd.cfg = group_cfg_index(mi[d].m, mi[d].r);
        gd.P = mi[d].P;
        gd.K = mi[d].k;
        gd.rec_elems = mi[d].nrec * kRec;
        gd.dtype = mi[d].dtype;
        gd.qclamp = (float)((1 << (24 - mi[d].m)) - 1);
        gd.single = mi[d].single;
    }
    a.rec_cap = rec_cap;
    a.k_cap = k_cap;
    a.n_cap = n_cap;
    a.warp_stride = stride;
    for (size_t lo = 0; lo < order.size(); lo += kGroupMaxSeg) {
        const size_t hi = std::min(order.size(), lo + (size_t)kGroupMaxSeg);
        int64_t total = 0;
        for (size_t q = lo; q < hi; q++) {
            const rmdec_segment& s = segs[order[q]];
            GroupSeg& gs = a.seg[q - lo];
            gs.llr = s.llr_dev;
            gs.info_out = s.bits_out_dev;
            gs.first = total;
            gs.dec = s.decoder;
            total += s.n_frames;
        }
        a.n_seg = (int)(hi - lo);
        a.total = total;
        const unsigned grid = (unsigned)std::min<int64_t>(total, (int64_t)g->sm_count * per_sm);
        void* args[] = {&a};
        nvtxRangePushA("rmdec_group_decode");
        e = cudaLaunchKernel(g->fn, dim3(grid), dim3(32 * W), args, smem_for(W), st);
        nvtxRangePop();
        if (e != cudaSuccess) return g->fail(RMDEC_ECUDA, "group kernel launch: %s", cudaGetErrorString(e));
    }
    return RMDEC_OK;
}
}  // namespace

extern "C" {

rmdec_status rmdec_group_create(rmdec_group_t* out, const rmdec_t* decoders, int n_decoders) {
    if (!out) {
        g_group_create_error = "null output pointer";
        return RMDEC_EINVAL;
    }
    *out = nullptr;
    if (!decoders || n_decoders < 1 || n_decoders > rmdec_dev::kGroupMaxDec) {
        g_group_create_error = "need 1..16 decoder handles";
        return RMDEC_EINVAL;
    }
    int L = 0;
    for (int i = 0; i < n_decoders; i++) {
        rmdec_host::MemberInfo mi;
        if (!decoders[i] || rmdec_host::member_info(decoders[i], false, &mi) != RMDEC_OK) {
            g_group_create_error = "null decoder handle at index " + std::to_string(i);
            return RMDEC_EINVAL;
        }
        if (mi.algo != 0) {
            g_group_create_error = "decoder " + std::to_string(i) + " is not a p-FHT-FSCL decoder";
            return RMDEC_EINVAL;
        }
        if (mi.hadamard != 0) {
            g_group_create_error = "decoder " + std::to_string(i) + ": tensor-core Hadamard decoders are not supported in groups";
            return RMDEC_EINVAL;
        }
        if (mi.r > 3) {
            g_group_create_error = "decoder " + std::to_string(i) + ": RM(4, m) decoders are not supported in groups";
            return RMDEC_EINVAL;
        }
        if (mi.m > 9) {
            g_group_create_error = "decoder " + std::to_string(i) + ": codes longer than 512 are not supported in groups";
            return RMDEC_EINVAL;
        }
        if (!group_fn(mi.L)) {
            g_group_create_error = "decoder " + std::to_string(i) + ": list size " + std::to_string(mi.L) +
                                   " is not supported in groups (L in {1, 2, 4, 8})";
            return RMDEC_EINVAL;
        }
        if (i == 0) L = mi.L;
        if (mi.L != L) {
            g_group_create_error = "decoders of one group need the same list size";
            return RMDEC_EINVAL;
        }
    }
    rmdec_group* g = new (std::nothrow) rmdec_group;
    if (!g) {
        g_group_create_error = "host allocation failed";
        return RMDEC_ENOMEM;
    }
    g->decs.assign(decoders, decoders + n_decoders);
    g->L = L;
    g->fn = group_fn(L);
    *out = g;
    return RMDEC_OK;
}

rmdec_status rmdec_group_decode(rmdec_group_t g, const rmdec_segment* segs, int n_segs, void* stream) {
    using namespace rmdec_dev;
    if (!g) return RMDEC_EINVAL;
    if (n_segs < 0 || (n_segs > 0 && !segs)) return g->fail(RMDEC_EINVAL, "bad segment list");
    const int nd = (int)g->decs.size();
    for (int i = 0; i < n_segs; i++) {
        const rmdec_segment& s = segs[i];
        if (s.decoder < 0 || s.decoder >= nd) return g->fail(RMDEC_EINVAL, "segment %d: unknown decoder %d", i, s.decoder);
        if (s.n_frames < 0) return g->fail(RMDEC_EINVAL, "segment %d: n_frames < 0", i);
        if (s.n_frames == 0) continue;
        if (!s.llr_dev || !s.bits_out_dev) return g->fail(RMDEC_EINVAL, "segment %d: null buffer", i);
        if (reinterpret_cast<uintptr_t>(s.llr_dev) % 16) return g->fail(RMDEC_EINVAL, "segment %d: llr buffer must be 16-byte aligned", i);
    }
    // the members' current tables on this device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return g->fail(RMDEC_EDEVICE, "no CUDA device: %s", cudaGetErrorString(e));
    std::vector<rmdec_host::MemberInfo> mi(nd);
    std::vector<char> used(nd, 0);
    for (int i = 0; i < n_segs; i++)
        if (segs[i].n_frames > 0) used[segs[i].decoder] = 1;
    for (int d = 0; d < nd; d++) {
        if (!used[d]) continue;
        const rmdec_status st = rmdec_host::member_info(g->decs[d], true, &mi[d]);
        if (st != RMDEC_OK) return g->fail(st, "decoder %d: %s", d, rmdec_last_error(g->decs[d]));
        if (mi[d].device != dev) return g->fail(RMDEC_EINVAL, "decoder %d was prepared on device %d, current is %d", d, mi[d].device, dev);
        if (mi[d].L != g->L || mi[d].algo != 0) return g->fail(RMDEC_EINVAL, "decoder %d no longer fits the group", d);
    }
    // Segments that fill at least min_alone frames (default: half a wave of their decoder's
    // own launch) run in their decoder's own kernel, which keeps its own register and
    // shared-memory footprint, and so do the segments that their decoder's own launch would give
    // to the path-per-thread kernel (the grouped kernel is the warp-per-decoder one, whose FP32
    // results may differ from it in rounding ties); the rest share grouped launches, most work
    // per frame first
    // (stable, so equal costs keep the caller's order). Measured on four codes at 600 frames
    // each (0.2 to 1.3 waves): a one-wave threshold 0.335 ms, half a wave 0.280 ms, a quarter
    // 0.274 ms but 20% slower at 200 frames each; separate launches 0.262 ms.
    std::vector<int> order, alone;
    for (int i = 0; i < n_segs; i++) {
        if (segs[i].n_frames == 0) continue;
        const int64_t thr = g->min_alone > 0 ? g->min_alone : (mi[segs[i].decoder].wave + 1) / 2;
        const int64_t pmin = mi[segs[i].decoder].path_min_frames;
        if ((pmin >= 0 && segs[i].n_frames >= pmin) || (g->min_alone >= 0 && segs[i].n_frames >= thr)) alone.push_back(i);
        else order.push_back(i);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!order.empty()) {
        const rmdec_status gs = launch_grouped(g, segs, order, mi, dev, st);
        if (gs != RMDEC_OK) return gs;
    }
    for (int i : alone) {
        const rmdec_segment& s = segs[i];
        const rmdec_status ds = rmdec_decode(g->decs[s.decoder], s.llr_dev, s.n_frames, s.bits_out_dev, st);
        if (ds != RMDEC_OK) return g->fail(ds, "decoder %d: %s", s.decoder, rmdec_last_error(g->decs[s.decoder]));
    }
    return RMDEC_OK;
}

rmdec_status rmdec_group_set_split(rmdec_group_t g, int64_t min_frames_alone) {
    if (!g) return RMDEC_EINVAL;
    g->min_alone = min_frames_alone < 0 ? -1 : min_frames_alone;
    return RMDEC_OK;
}

rmdec_status rmdec_group_set_tuning(rmdec_group_t g, int warps_per_cta, int ctas_per_sm) {
    if (!g) return RMDEC_EINVAL;
    if (warps_per_cta < 0 || warps_per_cta > rmdec_dev::kMaxWarps || ctas_per_sm < 0)
        return g->fail(RMDEC_EINVAL, "warps_per_cta must be 0..%d and ctas_per_sm >= 0", rmdec_dev::kMaxWarps);
    g->req_warps = warps_per_cta;
    g->req_ctas = ctas_per_sm;
    return RMDEC_OK;
}

void rmdec_group_destroy(rmdec_group_t g) { delete g; }

const char* rmdec_group_last_error(rmdec_group_t g) {
    if (!g) return g_group_create_error.c_str();
    return g->err.c_str();
}

}  // extern "C"
