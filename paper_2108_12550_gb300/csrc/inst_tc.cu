// Kernel instances whose FHTL nodes compute their spectra on the tensor cores
// (rmdec_set_hadamard(h, RMDEC_HADAMARD_TENSOR)): RM(2,9) and RM(3,9) with L = 4 and 8.
#include "pfht_kernel.cuh"
#include "rmdec_internal.h"

#define RMDEC_PFHT_TC_ENTRY(M, R, L)                                                     \
    do {                                                                                 \
        e->fn = reinterpret_cast<const void*>(&rmdec_dev::pfht_kernel<M, R, L, true>);   \
        e->warp_bytes = rmdec_dev::Cfg<M, R, L>::WARP_BYTES;                             \
        e->nrec = rmdec_dev::Cfg<M, R, L>::SMEM_NREC;                                    \
        e->fixed_bytes = [](int P, int K, int W) {                                       \
            return rmdec_dev::Cfg<M, R, L>::fixed_bytes(P, K, W);                        \
        };                                                                               \
        return true;                                                                     \
    } while (0)

namespace rmdec_host {
bool lookup_pfht_tc(int m, int r, int L, KernelEntry* e) {
    if (m != 9) return false;
    if (r == 2 && L == 4) RMDEC_PFHT_TC_ENTRY(9, 2, 4);
    if (r == 2 && L == 8) RMDEC_PFHT_TC_ENTRY(9, 2, 8);
    if (r == 3 && L == 4) RMDEC_PFHT_TC_ENTRY(9, 3, 4);
    if (r == 3 && L == 8) RMDEC_PFHT_TC_ENTRY(9, 3, 8);
    return false;
}
}  // namespace rmdec_host
