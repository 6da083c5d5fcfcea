// Grouped multi-code kernel instance for list size L = 2.
#include "group_kernel.cuh"
#include "rmdec_internal.h"

namespace rmdec_host {
const void* group_kernel_l2() { return reinterpret_cast<const void*>(&rmdec_dev::group_kernel<2>); }
}  // namespace rmdec_host
