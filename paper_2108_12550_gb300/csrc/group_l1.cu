// Grouped multi-code kernel instance for list size L = 1.
#include "group_kernel.cuh"
#include "rmdec_internal.h"

namespace rmdec_host {
const void* group_kernel_l1() { return reinterpret_cast<const void*>(&rmdec_dev::group_kernel<1>); }
}  // namespace rmdec_host
