// Instantiations of the warp-specialised size-level kernels for one word per
// trace.
#include "ltl_level_ws.cuh"

namespace ltl {
const void *ws_kernel_ptr_w1(int C, int op) {
    switch (C) {
    case 1: return ws_fn<1, 1>(op);
    case 2: return ws_fn<1, 2>(op);
    case 4: return ws_fn<1, 4>(op);
    case 8: return ws_fn<1, 8>(op);
    default: return nullptr;
    }
}
}  // namespace ltl
