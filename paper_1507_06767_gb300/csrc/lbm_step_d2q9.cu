// D2Q9 instantiations of the fused step: the one-cell kernel (lbm_step.cuh) by default, the two-cell
// packed kernel (lbm_step_pair.cuh) on request.
#include "lbm_internal.h"
#include "lbm_step_pair.cuh"

namespace lbm {

cudaError_t step_d2q9(int dtype, const void *fin, void *fout, const StepParams &p, int mode,
                      void *tile_max, void *k_field, cudaStream_t s, int variant) {
    // automatic choice, from GB300 measurements at 256^3 / 512^3: the one-cell kernel for FP32
    // and FP64, the two-cell packed kernel for 16-bit storage
    const bool pair_ok = dtype != 0 && pair_applicable<D2Q9>(p);
    const bool pair = pair_ok && (variant == KERNEL_PAIR || (variant == KERNEL_AUTO && dtype >= 2));
    if ((variant == KERNEL_PAIR && !pair_ok) || variant == KERNEL_TMA) return cudaErrorInvalidValue;
    switch (dtype) {
        case 0: return launch_fused_step<D2Q9, 0>(fin, fout, p, mode, tile_max, k_field, s);
        case 1:
            return pair ? launch_fused_step_pair<D2Q9, 1>(fin, fout, p, mode, tile_max, k_field, s)
                        : launch_fused_step<D2Q9, 1>(fin, fout, p, mode, tile_max, k_field, s);
        case 2:
            return pair ? launch_fused_step_pair<D2Q9, 2>(fin, fout, p, mode, tile_max, k_field, s)
                        : launch_fused_step<D2Q9, 2>(fin, fout, p, mode, tile_max, k_field, s);
        case 3:
            return pair ? launch_fused_step_pair<D2Q9, 3>(fin, fout, p, mode, tile_max, k_field, s)
                        : launch_fused_step<D2Q9, 3>(fin, fout, p, mode, tile_max, k_field, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
