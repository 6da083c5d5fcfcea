// Kernel instances for code length 2^7.
#include "pfht_kernel.cuh"
#include "rmdec_internal.h"

namespace rmdec_host {
bool lookup_pfht_m7(int r, int L, KernelEntry* e) {
    RMDEC_PFHT_CASE(7, 2)
    RMDEC_PFHT_CASE(7, 3)
    return false;
}
}  // namespace rmdec_host
