// adjoint_tape.cu -- the adjoint kernel (adjoint_core.cuh) with the lean
// shapes of size classes 2-4, R read from the forward build's factor tape
// (FP32 or FP64): its own translation unit, compiled in parallel.
#include "adjoint_core.cuh"

namespace sam {

cudaError_t launch_adjoint_tape_bin(sam_handle h, int precision, const LsqArgs &args, int bin) {
    if (precision == SAM_FP64) {
        switch (bin) {
            case 2: return launch_one<D2L, true>(h, args, 2);
            case 3: return launch_one<D3L, true>(h, args, 3);
            default: return launch_one<D4L, true>(h, args, 4);
        }
    }
    switch (bin) {
        case 2: return launch_one<F2L, false>(h, args, 2);
        case 3: return launch_one<F3L, false>(h, args, 3);
        default: return launch_one<F4L, false>(h, args, 4);
    }
}

}  // namespace sam
