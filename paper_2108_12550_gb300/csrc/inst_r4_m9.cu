// Kernel instances for RM(4, 9) (three permuted levels).
#include "pfht_kernel.cuh"
#include "rmdec_internal.h"

namespace rmdec_host {
bool lookup_pfht_r4_m9(int L, KernelEntry* e) {
    const int r = 4;
    RMDEC_PFHT_CASE(9, 4)
    return false;
}
}  // namespace rmdec_host
