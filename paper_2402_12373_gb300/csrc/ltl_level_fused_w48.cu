// Instantiations of the fused size-level kernels for four and eight words per
// trace.
#include "ltl_level_fused.cuh"

namespace ltl {
const void *fused_kernel_ptr_w48(int W, int C, int op) {
    switch (W * 16 + C) {
    case 4 * 16 + 1: return fused_fn<4, 1>(op);
    case 4 * 16 + 2: return fused_fn<4, 2>(op);
    case 8 * 16 + 1: return fused_fn<8, 1>(op);
    default: return nullptr;
    }
}
}  // namespace ltl
