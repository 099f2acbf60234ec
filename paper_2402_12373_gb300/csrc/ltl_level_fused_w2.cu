// Instantiations of the fused size-level kernels for two words per trace.
#include "ltl_level_fused.cuh"

namespace ltl {
const void *fused_kernel_ptr_w2(int C, int op) {
    switch (C) {
    case 1: return fused_fn<2, 1>(op);
    case 2: return fused_fn<2, 2>(op);
    case 4: return fused_fn<2, 4>(op);
    default: return nullptr;
    }
}
}  // namespace ltl
