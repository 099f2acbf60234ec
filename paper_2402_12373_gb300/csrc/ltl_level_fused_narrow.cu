// Instantiations of the fused size-level kernels for the narrow layout (two
// traces of at most 32 positions per uint64 word).
#include "ltl_level_fused.cuh"

namespace ltl {
const void *fused_kernel_ptr_narrow(int C, int op) {
    switch (C) {
    case 1: return fused_fn<1, 1, true>(op);
    case 2: return fused_fn<1, 2, true>(op);
    case 4: return fused_fn<1, 4, true>(op);
    default: return nullptr;
    }
}

// Candidates per batch of the fused kernel compiled for (W, C, narrow).
int fused_kernel_batch(int W, int C, bool narrow) {
    if (narrow) {
        if (W != 1) return -1;
        return C == 1 ? FusedNB<1, 1, true>::value : C == 2 ? FusedNB<1, 2, true>::value : FusedNB<1, 4, true>::value;
    }
    if (W * C >= 8) return FusedNB<1, 8, false>::value;
    return FusedNB<1, 1, false>::value;
}
}  // namespace ltl
