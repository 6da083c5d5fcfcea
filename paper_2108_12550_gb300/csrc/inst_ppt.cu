// Kernel instances of the path-per-thread decoder for RM(2, m), 4 <= m <= 8 (ppt_kernel.cuh);
// RM(3, m) in inst_ppt3.cu.
#include "ppt_entry.cuh"

namespace rmdec_host {

bool lookup_pfht_ppt(int m, int r, int L, int P, KernelEntry* e) {
    if (r == 3) return lookup_pfht_ppt3(m, L, P, e);
    if (r != 2) return false;
    switch (m) {
        case 4: return ppt_case<4, 2>(L, P, e);
        case 5: return ppt_case<5, 2>(L, P, e);
        case 6: return ppt_case<6, 2>(L, P, e);
        case 7: return ppt_case<7, 2>(L, P, e);
        case 8: return ppt_case<8, 2>(L, P, e);
    }
    return false;
}

}  // namespace rmdec_host
