// Instantiations of the fused size-level kernels for one word per trace.
#include "ltl_level_fused.cuh"

namespace ltl {
const void *fused_kernel_ptr_w1(int C, int op) {
    switch (C) {
    case 1: return fused_fn<1, 1>(op);
    case 2: return fused_fn<1, 2>(op);
    case 4: return fused_fn<1, 4>(op);
    case 8: return fused_fn<1, 8>(op);
    default: return nullptr;
    }
}
}  // namespace ltl
