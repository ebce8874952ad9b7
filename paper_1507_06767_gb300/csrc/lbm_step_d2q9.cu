// D2Q9 instantiations of the fused step.
#include "lbm_internal.h"
#include "lbm_step.cuh"

namespace lbm {

cudaError_t step_d2q9(int dtype, const void *fin, void *fout, const StepParams &p, int mode,
                      void *tile_max, void *k_field, cudaStream_t s) {
    switch (dtype) {
        case 0: return launch_fused_step<D2Q9, 0>(fin, fout, p, mode, tile_max, k_field, s);
        case 1: return launch_fused_step<D2Q9, 1>(fin, fout, p, mode, tile_max, k_field, s);
        case 2: return launch_fused_step<D2Q9, 2>(fin, fout, p, mode, tile_max, k_field, s);
        case 3: return launch_fused_step<D2Q9, 3>(fin, fout, p, mode, tile_max, k_field, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
