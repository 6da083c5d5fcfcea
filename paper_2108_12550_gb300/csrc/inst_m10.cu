// Kernel instances for code length 2^10.
#include "pfht_kernel.cuh"
#include "rmdec_internal.h"

namespace rmdec_host {
bool lookup_pfht_m10(int r, int L, KernelEntry* e) {
    RMDEC_PFHT_CASE(10, 2)
    RMDEC_PFHT_CASE(10, 3)
    return false;
}
}  // namespace rmdec_host
