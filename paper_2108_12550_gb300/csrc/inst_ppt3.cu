// Kernel instances of the path-per-thread decoder for RM(3, m), 5 <= m <= 7 (ppt_kernel.cuh).
#include "ppt_entry.cuh"

namespace rmdec_host {

bool lookup_pfht_ppt3(int m, int L, int P, KernelEntry* e) {
    switch (m) {
        case 5: return ppt_case<5, 3>(L, P, e);
        case 6: return ppt_case<6, 3>(L, P, e);
        case 7: return ppt_case<7, 3>(L, P, e);
    }
    return false;
}

}  // namespace rmdec_host
