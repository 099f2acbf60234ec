// Instantiations of the warp-specialised size-level kernels for two, four
// and eight words per trace and for the narrow layout (two traces of at most
// 32 positions per word).
#include "ltl_level_ws.cuh"

namespace ltl {
const void *ws_kernel_ptr_wn(int W, int C, int op) {
    switch (W * 16 + C) {
    case 2 * 16 + 1: return ws_fn<2, 1>(op);
    case 2 * 16 + 2: return ws_fn<2, 2>(op);
    case 2 * 16 + 4: return ws_fn<2, 4>(op);
    case 4 * 16 + 1: return ws_fn<4, 1>(op);
    case 4 * 16 + 2: return ws_fn<4, 2>(op);
    case 8 * 16 + 1: return ws_fn<8, 1>(op);
    default: return nullptr;
    }
}

// Candidates per batch of the warp-specialised kernel compiled for (W, C, narrow).
int ws_kernel_batch(int W, int C, bool narrow) {
    if (narrow) return WsNB<1, 1, true>::value;
    return W * C >= 8 ? WsNB<1, 8, false>::value : WsNB<1, 1, false>::value;
}

const void *ws_kernel_ptr_narrow(int C, int op) {
    switch (C) {
    case 1: return ws_fn<1, 1, true>(op);
    case 2: return ws_fn<1, 2, true>(op);
    case 4: return ws_fn<1, 4, true>(op);
    default: return nullptr;
    }
}
}  // namespace ltl
