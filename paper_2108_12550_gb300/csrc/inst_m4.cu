// Kernel instances for code length 2^4.
#include "pfht_kernel.cuh"
#include "rmdec_internal.h"

namespace rmdec_host {
bool lookup_pfht_m4(int r, int L, KernelEntry* e) {
    RMDEC_PFHT_CASE(4, 2)
    return false;
}
}  // namespace rmdec_host
