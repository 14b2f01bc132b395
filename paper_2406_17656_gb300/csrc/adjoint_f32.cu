// adjoint_f32.cu -- the adjoint kernel (adjoint_core.cuh) with the FP32
// register tiles of size classes 0-4, R recomputed: its own translation
// unit, compiled in parallel with the others.
#include "adjoint_core.cuh"

namespace sam {

cudaError_t launch_adjoint_f32_bin(sam_handle h, const LsqArgs &args, int bin) {
    switch (bin) {
        case 0: return launch_one<F0, false>(h, args, 0);
        case 1: return launch_one<F1, false>(h, args, 1);
        case 2: return launch_one<F2, false>(h, args, 2);
        case 3: return launch_one<F3, false>(h, args, 3);
        default: return launch_one<F4, false>(h, args, 4);
    }
}

}  // namespace sam
