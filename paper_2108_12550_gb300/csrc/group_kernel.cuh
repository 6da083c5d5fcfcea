// One persistent launch that decodes frames of several RM codes, p-FHT-FSCL decoders and LLR
// types at once (the method of each frame is the same as pfht_kernel's: Algorithms 2-5 of
// arXiv 2108.12550).
//
// Work is a list of segments, each a run of frames of one decoder. The host orders segments
// by decreasing cost per frame and numbers their frames consecutively; CTA b takes global
// frames b, b + grid, b + 2 grid, ... A decoder's work per frame does not depend on the
// received values, so this static round-robin spreads every segment evenly over all CTAs
// (each CTA gets at most one frame more of any segment than another) and keeps all SMs in
// the same code at the same time (one instruction working set per phase). Descriptors travel
// in the kernel parameters (__grid_constant__), so the launch reads no device tables beyond
// each decoder's own permutation records and can be captured in a CUDA graph as is.
//
// One kernel instance serves one list size L and every (m, r) with 4 <= m <= 9, r in {2, 3},
// r <= m - 2 (the family index is (m - 4) * 2 + (r - 2)). Shared memory is sized for the
// largest member of the launch: records and information positions of the decoder in use are
// reloaded when a CTA moves to the next decoder's segment.
#pragma once

#include "pfht_kernel.cuh"

namespace rmdec_dev {

constexpr int kGroupMaxDec = 16;   // decoders referenced by one launch
constexpr int kGroupMaxSeg = 224;  // segments per launch (the host splits longer lists)

__host__ __device__ constexpr int group_cfg_index(int m, int r) { return (m - 4) * 2 + (r - 2); }

struct GroupDec {
    const uint16_t* recs;  // device table: per decoder NREC maps, then their inverses
    const uint16_t* info;  // K information positions
    int cfg;               // group_cfg_index(m, r)
    int P, K;
    int rec_elems;         // SMEM_NREC * kRec: forward map elements per decoder in shared memory
    int dtype;
    float qclamp;
    int single;
    int pad;
};

struct GroupSeg {
    const void* llr;       // [n][N] LLRs of the decoder's dtype
    uint32_t* info_out;    // [n][ceil(K/32)]
    int64_t first;         // global index of the segment's first frame
    int dec;               // index into GroupArgs::dec
    int pad;
};

struct GroupArgs {
    GroupDec dec[kGroupMaxDec];
    GroupSeg seg[kGroupMaxSeg];
    int n_seg;
    int rec_cap, k_cap;    // shared-memory capacity for records and positions
    int n_cap;             // and for the frame LLRs (the longest member code)
    int warp_stride;       // largest warp area of the members
    int64_t total;         // frames over all segments
};

// Members' P need not be multiples of the block's warps, so no leaf barriers here (LOCK false).
template <int L>
__device__ __forceinline__ void group_dispatch(int cfg, const FrameJob& j, const FrameSmem& sm, int64_t f) {
    switch (cfg) {
        case group_cfg_index(4, 2): decode_frame<4, 2, L, false>(j, sm, f); break;
        case group_cfg_index(5, 2): decode_frame<5, 2, L, false>(j, sm, f); break;
        case group_cfg_index(5, 3): decode_frame<5, 3, L, false>(j, sm, f); break;
        case group_cfg_index(6, 2): decode_frame<6, 2, L, false>(j, sm, f); break;
        case group_cfg_index(6, 3): decode_frame<6, 3, L, false>(j, sm, f); break;
        case group_cfg_index(7, 2): decode_frame<7, 2, L, false>(j, sm, f); break;
        case group_cfg_index(7, 3): decode_frame<7, 3, L, false>(j, sm, f); break;
        case group_cfg_index(8, 2): decode_frame<8, 2, L, false>(j, sm, f); break;
        case group_cfg_index(8, 3): decode_frame<8, 3, L, false>(j, sm, f); break;
        case group_cfg_index(9, 2): decode_frame<9, 2, L, false>(j, sm, f); break;
        case group_cfg_index(9, 3): decode_frame<9, 3, L, false>(j, sm, f); break;
        default: break;  // rejected on the host
    }
}

// Up to kMaxWarps warps per CTA (the host takes wide CTAs for launches of a few waves), with
// the same per-thread register budget as pfht_kernel.
template <int L>
__global__ void __launch_bounds__(32 * kMaxWarps, 1) group_kernel(const __grid_constant__ GroupArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const FrameSmem sm = carve_smem(smem, a.rec_cap, a.k_cap, a.warp_stride, a.n_cap, blockDim.x >> 5);
    int seg = 0, loaded = -1;
    for (int64_t g = blockIdx.x; g < a.total; g += gridDim.x) {
        // segments are non-empty and in increasing order of first frame
        while (seg + 1 < a.n_seg && g >= a.seg[seg + 1].first) seg++;
        const GroupSeg& sg = a.seg[seg];
        const GroupDec& d = a.dec[sg.dec];
        if (sg.dec != loaded) {
            __syncthreads();  // every warp is done with the previous decoder's tables
            copy_maps(sm.rec, d.recs, d.P, d.rec_elems);
            for (int i = threadIdx.x; i < d.K; i += blockDim.x) sm.info[i] = d.info[i];
            loaded = sg.dec;  // decode_frame's first barrier publishes the tables
        }
        FrameJob j;
        j.recs = d.recs;
        j.llr = sg.llr;
        j.dtype = d.dtype;
        j.qclamp = d.qclamp;
        j.P = d.P;
        j.K = d.K;
        j.single = d.single;
        j.info_out = sg.info_out;
        j.cw_out = nullptr;
        j.pm_out = nullptr;
        j.best_out = nullptr;
        group_dispatch<L>(d.cfg, j, sm, g - sg.first);
    }
}

}  // namespace rmdec_dev
