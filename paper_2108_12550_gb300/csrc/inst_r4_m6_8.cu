// Kernel instances for RM(4, m), m = 6, 7, 8 (three permuted levels).
#include "pfht_kernel.cuh"
#include "rmdec_internal.h"

namespace rmdec_host {
bool lookup_pfht_r4_small(int m, int L, KernelEntry* e) {
    const int r = 4;
    if (m == 6) { RMDEC_PFHT_CASE(6, 4) }
    if (m == 7) { RMDEC_PFHT_CASE(7, 4) }
    if (m == 8) { RMDEC_PFHT_CASE(8, 4) }
    return false;
}
}  // namespace rmdec_host
