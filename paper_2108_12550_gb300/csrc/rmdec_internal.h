// Internal interfaces between the C-ABI layer and the kernel instantiation units.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/rmdec.h"

struct rmdec_ctx;

namespace rmdec_host {

// Every device allocation of the library goes through here, so that tests can make it fail
// (rmdec_debug_fail_device_allocs).
cudaError_t device_alloc(void** p, size_t bytes);

// Bytes per LLR element of a handle's current input type.
size_t llr_elem_bytes_of(rmdec_ctx* h);

// One compiled decoder configuration (a kernel template instance).
struct KernelEntry {
    const void* fn = nullptr;  // __global__ function
    int warp_bytes = 0;        // shared memory per warp
    int nrec = 0;              // permutation maps per decoder held in block shared memory
    int (*fixed_bytes)(int P, int K, int W) = nullptr;
    int frames_per_warp = 0;   // path-per-thread kernels: frames a CTA decodes at once (else 0)
    int batches = 0;           // path-per-thread kernels: decoder batches per frame
    int64_t min_frames = 0;    // path-per-thread kernels: smallest launch they take by default
    bool auto_ok = true;       // path-per-thread kernels: faster than the warp-per-decoder
                               // kernel for this P (the default choice may take it)
};

// p-FHT-FSCL kernels: one lookup per code length m (instantiated in inst_m<m>.cu).
bool lookup_pfht_m4(int r, int L, KernelEntry* e);
bool lookup_pfht_m5(int r, int L, KernelEntry* e);
bool lookup_pfht_m6(int r, int L, KernelEntry* e);
bool lookup_pfht_m7(int r, int L, KernelEntry* e);
bool lookup_pfht_m8(int r, int L, KernelEntry* e);
bool lookup_pfht_m9(int r, int L, KernelEntry* e);
bool lookup_pfht_m10(int r, int L, KernelEntry* e);
// RM(4, m): three permuted levels (inst_r4_*.cu)
bool lookup_pfht_r4_small(int m, int L, KernelEntry* e);  // m = 6, 7, 8
bool lookup_pfht_r4_m9(int L, KernelEntry* e);
// list size L = 32 (inst_l32_*.cu)
bool lookup_pfht_l32_small(int m, int r, KernelEntry* e);  // m = 4 .. 7
bool lookup_pfht_l32_m8(int r, KernelEntry* e);
bool lookup_pfht_l32_m9(int r, KernelEntry* e);

// Path-per-thread kernels for RM(2, m), 4 <= m <= 8, and RM(3, m), 5 <= m <= 7, with L in
// {1, 2, 4, 8} (inst_ppt.cu, inst_ppt3.cu); the entry's shared-memory sizes depend on the
// decoder count P.
bool lookup_pfht_ppt(int m, int r, int L, int P, KernelEntry* e);
bool lookup_pfht_ppt3(int m, int L, int P, KernelEntry* e);

// p-FHT-FSCL kernels whose FHTL nodes use the tensor cores (inst_tc.cu).
bool lookup_pfht_tc(int m, int r, int L, KernelEntry* e);

// Aut-SSC baseline kernels (autssc.cu).
bool lookup_autssc(int m, int r, KernelEntry* e);

// p-FHT-FSCL of RM(1, m) and RM(m-1, m), whose root is an FHTL or SPCL node (mlroot.cu).
bool lookup_mlroot(int m, int r, KernelEntry* e);

// What a grouped launch needs to know about one decoder handle.
struct MemberInfo {
    int algo = 0;  // 0: p-FHT-FSCL (and FHT-FSCL), 1: Aut-SSC, 2: RM(1, m) / RM(m-1, m) roots
    int m = 0, r = 0, L = 0, P = 0, n = 0, k = 0;
    int single = 0;
    int dtype = 0;
    int hadamard = 0;  // rmdec_hadamard of the handle
    const uint16_t* d_recs = nullptr;  // valid after prepare
    const uint16_t* d_info = nullptr;
    int warp_bytes = 0;
    int nrec = 0;  // permutation maps per decoder held in block shared memory
    int device = -1;
    int64_t wave = 0;  // CTAs of the handle's own launch resident at once (valid after prepare)
    int64_t path_min_frames = -1;  // launches of at least this many frames use the
                                   // path-per-thread kernel (-1: none; valid after prepare)
};
// Fills *out from the handle; with prepare = true first uploads the handle's tables to the
// current device and fixes its own launch shape (errors are recorded on the handle, see
// rmdec_last_error).
rmdec_status member_info(rmdec_ctx* h, bool prepare, MemberInfo* out);

// Grouped multi-code kernels (group_l<L>.cu), one per supported list size.
const void* group_kernel_l1();
const void* group_kernel_l2();
const void* group_kernel_l4();
const void* group_kernel_l8();

}  // namespace rmdec_host

#define RMDEC_PFHT_ENTRY(M, R, L)                                                        \
    do {                                                                                 \
        e->fn = reinterpret_cast<const void*>(&rmdec_dev::pfht_kernel<M, R, L>);         \
        e->warp_bytes = rmdec_dev::Cfg<M, R, L>::WARP_BYTES;                             \
        e->nrec = rmdec_dev::Cfg<M, R, L>::SMEM_NREC;                                    \
        e->fixed_bytes = [](int P, int K, int W) {                                       \
            return rmdec_dev::Cfg<M, R, L>::fixed_bytes(P, K, W);                        \
        };                                                                               \
        return true;                                                                     \
    } while (0)

#define RMDEC_PFHT_CASE(M, R)                                                            \
    if (r == R) {                                                                        \
        if (L == 1) RMDEC_PFHT_ENTRY(M, R, 1);                                           \
        if (L == 2) RMDEC_PFHT_ENTRY(M, R, 2);                                           \
        if (L == 4) RMDEC_PFHT_ENTRY(M, R, 4);                                           \
        if (L == 8) RMDEC_PFHT_ENTRY(M, R, 8);                                           \
        if (L == 16) RMDEC_PFHT_ENTRY(M, R, 16);                                         \
    }
