// D2Q9 instantiations of the fused step: the one-cell kernel (lbm_step.cuh) and the two-cell packed
// kernel (lbm_step_pair.cuh), with the automatic choice between them.
#include "lbm_internal.h"
#include "lbm_step_pair.cuh"

namespace lbm {

cudaError_t step_d2q9(int dtype, const void *fin, void *fout, const StepParams &p, int mode,
                      void *tile_max, void *k_field, cudaStream_t s, int variant) {
    // automatic choice, from GB300 measurements (D2Q9 cavity, FP32, two-cell against one-cell
    // time per step): 256^2 plain steps 2.41 against 2.10 us, sensor steps 4.12 against 4.11 us;
    // 384^2 2.83 against 2.84 and 6.03 against 6.18 us; 1024^2 8.04 against 9.96 and 12.3 against
    // 16.4 us; 4096^2 173 against 175 and 200 against 230 us.  So the two-cell kernel from 2^17
    // cells with FP32 storage, at every size with 16-bit storage, never with FP64.
    const bool pair_ok = dtype != 0 && pair_applicable<D2Q9>(p);
    const bool big = (long long)p.nx * p.ny >= AUTO_PAIR_MIN_CELLS_D2Q9_F32;
    const bool pair = pair_ok && (variant == KERNEL_PAIR ||
                                  (variant == KERNEL_AUTO && (dtype >= 2 || big)));
    if ((variant == KERNEL_PAIR && !pair_ok) || variant == KERNEL_TMA) return cudaErrorInvalidValue;
    if (has_halo(p)) {
        if (variant != KERNEL_AUTO && variant != KERNEL_CELL) return cudaErrorInvalidValue;
        switch (dtype) {
            case 0: return launch_fused_step<D2Q9, 0, true>(fin, fout, p, mode, tile_max, k_field, s);
            case 1: return launch_fused_step<D2Q9, 1, true>(fin, fout, p, mode, tile_max, k_field, s);
            case 2: return launch_fused_step<D2Q9, 2, true>(fin, fout, p, mode, tile_max, k_field, s);
            case 3: return launch_fused_step<D2Q9, 3, true>(fin, fout, p, mode, tile_max, k_field, s);
            default: return cudaErrorInvalidValue;
        }
    }
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
