// The kernel-table entry of a path-per-thread kernel instance (inst_ppt*.cu).
#pragma once

#include "ppt_kernel.cuh"
#include "rmdec_internal.h"

namespace rmdec_host {

// Decoders per frame P for which the default choice gives large launches to this kernel: the
// P where it decoded 16,384 FP32 frames at least 10% faster than the warp-per-decoder kernel,
// measured at P = 1, 4, 8, 16, 20, 32, 64 and 128 (P between two measured values counts as
// outside unless both were inside). Outside, either the frame's lane group holds too few paths
// (P = 1 for m >= 7: one path in 4 or 8 lanes), or the decoders' tables in shared memory leave
// few CTAs per SM (large P), or the L = 8 candidate lists cost more than the warp kernel's
// selection (RM(2,8), and RM(2,7) or RM(3,7) beyond P = 8 or 4).
struct PptAutoRange {
    int pmin, pmax;  // pmin > pmax: never
};
constexpr PptAutoRange ppt_auto_range(int M, int R, int L) {
    if (R == 2 && M <= 6) return {1, L <= 4 ? 128 : 32};
    if (R == 3 && M <= 6) return {1, L <= 2 ? 128 : (L == 4 ? 64 : (M == 5 ? 20 : 16))};
    if (R == 2 && M == 7) return {4, L <= 2 ? 128 : (L == 4 ? 64 : 8)};
    if (R == 3 && M == 7) return L <= 2 ? PptAutoRange{4, 128} : (L == 4 ? PptAutoRange{1, 32} : PptAutoRange{4, 4});
    if (R == 2 && M == 8) return {4, L <= 2 ? 128 : (L == 4 ? 20 : 0)};
    return {1, 0};
}

template <int M, int R, int L>
bool ppt_entry(int P, KernelEntry* e) {
    using D = rmdec_dev::Ppt<M, R, L>;
    const int fw = rmdec_dev::ppt_frame_lanes(M, L, P);
    e->fn = reinterpret_cast<const void*>(&rmdec_dev::ppt_kernel<M, R, L>);
    e->frames_per_warp = 32 / fw;  // frames a CTA stages at a time
    const int per_batch = fw / D::DL;
    e->batches = (P + per_batch - 1) / per_batch;
    e->warp_bytes = D::PEND_FLOATS * 4 + 32 + rmdec_dev::kPptSlotWords * 4;
    e->nrec = 0;  // the maps sit in the fixed part
    e->fixed_bytes = [](int P2, int K, int) {
        const int fpw = 32 / rmdec_dev::ppt_frame_lanes(M, L, P2);
        const int tables = ((P2 * 2 * rmdec_dev::Ppt<M, R, L>::NREC * rmdec_dev::kRec * 2 + K * 2) + 15) / 16 * 16;
        return tables + ((fpw * rmdec_dev::ppt_frame_stride(M, fpw) * 4) + 15) / 16 * 16;
    };
    // Smallest launch this kernel takes by default (the warp-per-decoder kernel takes smaller
    // ones): where it overtook that kernel, measured with CUDA events over 64..65,536 frames
    // (FP32, L = 4 unless stated): RM(2,5) P=4 L=2 from 512 frames, RM(2,6) P=8 and RM(2,7) P=8
    // INT8 / P=20 from 2,048, RM(2,8) P=8 / P=20 from 8,192; RM(3,5) P=4 L=2, RM(3,6) P=8,
    // RM(3,7) P=8 / P=20 between 512 and 2,048.
    e->min_frames = R == 3 ? 2048 : (M <= 5 ? 512 : (M <= 7 ? 2048 : 8192));
    constexpr PptAutoRange ar = ppt_auto_range(M, R, L);
    e->auto_ok = P >= ar.pmin && P <= ar.pmax;
    return true;
}

template <int M, int R>
bool ppt_case(int L, int P, KernelEntry* e) {
    switch (L) {
        case 1: return ppt_entry<M, R, 1>(P, e);
        case 2: return ppt_entry<M, R, 2>(P, e);
        case 4: return ppt_entry<M, R, 4>(P, e);
        case 8: return ppt_entry<M, R, 8>(P, e);
    }
    return false;
}

}  // namespace rmdec_host
