// Kernel instances with list size L = 32 for code lengths 2^4 to 2^7.
#include "pfht_kernel.cuh"
#include "rmdec_internal.h"

namespace rmdec_host {
bool lookup_pfht_l32_small(int m, int r, KernelEntry* e) {
    if (m == 4 && r == 2) RMDEC_PFHT_ENTRY(4, 2, 32);
    if (m == 5 && r == 2) RMDEC_PFHT_ENTRY(5, 2, 32);
    if (m == 5 && r == 3) RMDEC_PFHT_ENTRY(5, 3, 32);
    if (m == 6 && r == 2) RMDEC_PFHT_ENTRY(6, 2, 32);
    if (m == 6 && r == 3) RMDEC_PFHT_ENTRY(6, 3, 32);
    if (m == 6 && r == 4) RMDEC_PFHT_ENTRY(6, 4, 32);
    if (m == 7 && r == 2) RMDEC_PFHT_ENTRY(7, 2, 32);
    if (m == 7 && r == 3) RMDEC_PFHT_ENTRY(7, 3, 32);
    if (m == 7 && r == 4) RMDEC_PFHT_ENTRY(7, 4, 32);
    return false;
}
}  // namespace rmdec_host
