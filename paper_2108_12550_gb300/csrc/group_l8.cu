// Grouped multi-code kernel instance for list size L = 8.
#include "group_kernel.cuh"
#include "rmdec_internal.h"

namespace rmdec_host {
const void* group_kernel_l8() { return reinterpret_cast<const void*>(&rmdec_dev::group_kernel<8>); }
}  // namespace rmdec_host
