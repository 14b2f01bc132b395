// lsq_fp64.cu -- the register-tile least-squares kernel (lsq_kernel.cuh)
// with FP64 tiles, for SAM_FP64 builds: its own translation unit, so that
// the FP32 and FP64 instantiations compile in parallel.
#include "lsq_kernel.cuh"

namespace sam {

cudaError_t launch_lsq_fp64_bin(sam_handle h, const LsqArgs &args, int bin) {
    switch (bin) {
        case 0: return launch_one<D0, true>(h, args, 0);
        case 1: return launch_one<D1, true>(h, args, 1);
        case 2: return launch_one<D2, true>(h, args, 2);
        case 3: return launch_one<D3, true>(h, args, 3);
        default: return launch_one<D4, true>(h, args, 4);
    }
}

}  // namespace sam
