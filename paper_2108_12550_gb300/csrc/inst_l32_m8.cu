// Kernel instances with list size L = 32 for code length 2^8.
#include "pfht_kernel.cuh"
#include "rmdec_internal.h"

namespace rmdec_host {
bool lookup_pfht_l32_m8(int r, KernelEntry* e) {
    if (r == 2) RMDEC_PFHT_ENTRY(8, 2, 32);
    if (r == 3) RMDEC_PFHT_ENTRY(8, 3, 32);
    if (r == 4) RMDEC_PFHT_ENTRY(8, 4, 32);
    return false;
}
}  // namespace rmdec_host
