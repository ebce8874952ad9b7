// D3Q19 instantiations of the fused step: the TMA-staged kernel (lbm_step_tma.cuh), the one-cell
// kernel (lbm_step.cuh), the two-cell packed kernel (lbm_step_pair.cuh) and the TMA-staged
// two-cell kernel for 16-bit storage (lbm_step_tma_pair.cuh), chosen by `variant`.
#include <cudaTypedefs.h>

#include <mutex>

#include "lbm_internal.h"
#include "lbm_step_pair.cuh"
#include "lbm_step_tma.cuh"
#include "lbm_step_tma_pair.cuh"

namespace lbm {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cache[dev] = n;
    }
    return cache[dev];
}

// Tensor map of a population buffer as a 4-D tensor (x, y, z, direction) with box (w, 1, 1, 1).
template <int DT>
bool encode_populations(CUtensorMap *map, const void *base, const StepParams &p, int w) {
    using T = typename Storage<DT>::T;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t es = sizeof(T);
    const cuuint64_t dims[4] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, (cuuint64_t)p.nz, 19};
    const cuuint64_t strides[3] = {(cuuint64_t)p.nx * es, (cuuint64_t)p.nx * p.ny * es,
                                   (cuuint64_t)p.nx * p.ny * p.nz * es};
    const cuuint32_t box[4] = {(cuuint32_t)w, 1, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType t = DT == 1   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                  : DT == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                            : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    return enc(map, t, 4, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               (CUtensorMapL2promotion)LBM_TMA_L2_PROMO, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <int DT, int MODE>
cudaError_t launch_tma_mode(const CUtensorMap &main_map, const CUtensorMap &halo_map,
                            const void *fin, void *fout, const StepParams &p, void *tile_max,
                            void *k_field, cudaStream_t s) {
    using T = typename Storage<DT>::T;
    using C = TmaCfg<DT>;
    // the shared-memory opt-in is a per-device attribute of the kernel: set once per device
    static std::mutex mu;
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev < 0 || dev >= 64 || !attr[dev]) {
            e = cudaFuncSetAttribute(fused_step_tma_kernel<DT, MODE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
            if (e != cudaSuccess) return e;
            if (dev >= 0 && dev < 64) attr[dev] = true;
        }
    }
    const long long units = (long long)((p.nx + TMA_CHUNK - 1) / TMA_CHUNK) * p.ny *
                            ((p.nz + TMA_UNIT_Z - 1) / TMA_UNIT_Z);
    const int nsm = sm_count();
    long long grid = (long long)TMA_CTAS_PER_SM * (nsm > 0 ? nsm : 1);
    if (grid > units) grid = units;
    fused_step_tma_kernel<DT, MODE><<<(unsigned)grid, TMA_THREADS, C::SMEM_BYTES, s>>>(
        main_map, halo_map, static_cast<const T *>(fin), static_cast<T *>(fout), p,
        static_cast<float *>(tile_max), static_cast<float *>(p.tile_zero),
        static_cast<float *>(k_field));
    return cudaGetLastError();
}

template <int DT>
cudaError_t launch_fused_step_tma(const void *fin, void *fout, const StepParams &p, int mode,
                                  void *tile_max, void *k_field, cudaStream_t s) {
    CUtensorMap main_map, halo_map;
    if (!encode_populations<DT>(&main_map, fin, p, TMA_CHUNK) ||
        !encode_populations<DT>(&halo_map, fin, p, TmaCfg<DT>::H))
        return cudaErrorInvalidValue;
    if (mode == 0) return launch_tma_mode<DT, 0>(main_map, halo_map, fin, fout, p, tile_max, k_field, s);
    if (mode == 1) return launch_tma_mode<DT, 1>(main_map, halo_map, fin, fout, p, tile_max, k_field, s);
    return launch_tma_mode<DT, 2>(main_map, halo_map, fin, fout, p, tile_max, k_field, s);
}

// Tensor map of a 16-bit population buffer as a 4-D tensor (x, y, z, direction) with box
// (bx, by, 1, 1); out-of-range elements read as zero.
bool encode_u16(CUtensorMap *map, const void *base, const StepParams &p, int bx, int by) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, (cuuint64_t)p.nz, 19};
    const cuuint64_t strides[3] = {(cuuint64_t)p.nx * 2, (cuuint64_t)p.nx * p.ny * 2,
                                   (cuuint64_t)p.nx * p.ny * p.nz * 2};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<void *>(base), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               (CUtensorMapL2promotion)LBM_TMA_L2_PROMO, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <int DT, int MODE>
cudaError_t launch_tma_pair_mode(const TpMaps &maps, const void *fin, void *fout,
                                 const StepParams &p, void *tile_max, void *k_field,
                                 cudaStream_t s) {
    using T = typename Storage<DT>::T;
    static std::mutex mu;
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev < 0 || dev >= 64 || !attr[dev]) {
            e = cudaFuncSetAttribute(fused_step_tma_pair_kernel<DT, MODE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     TpLayout::SMEM_BYTES);
            if (e != cudaSuccess) return e;
            if (dev >= 0 && dev < 64) attr[dev] = true;
        }
    }
    const long long units = (long long)((p.nx + TP_TX - 1) / TP_TX) *
                            ((p.ny + TP_TY - 1) / TP_TY) * ((p.nz + TP_TZ - 1) / TP_TZ);
    const int nsm = sm_count();
    long long grid = (long long)TP_CTAS_PER_SM * (nsm > 0 ? nsm : 1);
    if (grid > units) grid = units;
    fused_step_tma_pair_kernel<DT, MODE><<<(unsigned)grid, TP_THREADS, TpLayout::SMEM_BYTES, s>>>(
        maps, static_cast<const T *>(fin), static_cast<T *>(fout), p,
        static_cast<float *>(tile_max), static_cast<float *>(k_field));
    return cudaGetLastError();
}

template <int DT>
cudaError_t launch_fused_step_tma_pair(const void *fin, void *fout, const StepParams &p, int mode,
                                       void *tile_max, void *k_field, cudaStream_t s) {
    if (!tma_pair_applicable(DT, p)) return cudaErrorInvalidValue;
    TpMaps maps;
    if (!encode_u16(&maps.narrow, fin, p, TP_TX, TP_TY) ||
        !encode_u16(&maps.wide, fin, p, TP_WIDE, TP_TY) || !encode_u16(&maps.face, fin, p, 8, 8))
        return cudaErrorInvalidValue;
    if (mode == 0) return launch_tma_pair_mode<DT, 0>(maps, fin, fout, p, tile_max, k_field, s);
    if (mode == 1) return launch_tma_pair_mode<DT, 1>(maps, fin, fout, p, tile_max, k_field, s);
    return launch_tma_pair_mode<DT, 2>(maps, fin, fout, p, tile_max, k_field, s);
}

}  // namespace

cudaError_t step_d3q19(int dtype, const void *fin, void *fout, const StepParams &p, int mode,
                       void *tile_max, void *k_field, cudaStream_t s, int variant) {
    // automatic choice, from GB300 measurements (D3Q19 cavity, two-cell against one-cell time):
    // with 16-bit storage the two-cell kernel at every size and step kind measured (sensor steps
    // 128^3 0.046 against 0.057 ms, 256^3 0.247 against 0.370 ms, 512^3 1.89 against 2.86 ms;
    // plain steps 0.041 / 0.045, 0.236 / 0.310, 1.90 / 2.42 ms); with FP32 storage the one-cell
    // kernel (sensor steps 128^3 0.0644 against 0.0575 ms, 256^3 0.387 against 0.383 ms, 512^3
    // 3.034 against 3.027 ms; plain steps 0.0607 / 0.0545, 0.385 / 0.379, 3.039 / 3.025 ms);
    // FP64: the one-cell kernel
    const bool pair_ok = dtype != 0 && pair_applicable<D3Q19>(p);
    const bool pair = pair_ok && (variant == KERNEL_PAIR || (variant == KERNEL_AUTO && dtype >= 2));
    const bool tma = tma_applicable(dtype, p.nx) && variant == KERNEL_TMA;
    const bool tma_pair = variant == KERNEL_TMA_PAIR && tma_pair_applicable(dtype, p);
    if ((variant == KERNEL_PAIR && !pair_ok) || (variant == KERNEL_TMA && !tma) ||
        (variant == KERNEL_TMA_PAIR && !tma_pair))
        return cudaErrorInvalidValue;
    if (has_halo(p)) {  // a slab with cut faces: the one-cell kernel with the halo gather
        if (variant != KERNEL_AUTO && variant != KERNEL_CELL) return cudaErrorInvalidValue;
        switch (dtype) {
            case 0: return launch_fused_step<D3Q19, 0, true>(fin, fout, p, mode, tile_max, k_field, s);
            case 1: return launch_fused_step<D3Q19, 1, true>(fin, fout, p, mode, tile_max, k_field, s);
            case 2: return launch_fused_step<D3Q19, 2, true>(fin, fout, p, mode, tile_max, k_field, s);
            case 3: return launch_fused_step<D3Q19, 3, true>(fin, fout, p, mode, tile_max, k_field, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (tma_pair) {
        if (dtype == 2) return launch_fused_step_tma_pair<2>(fin, fout, p, mode, tile_max, k_field, s);
        return launch_fused_step_tma_pair<3>(fin, fout, p, mode, tile_max, k_field, s);
    }
    switch (dtype) {
        case 0: return launch_fused_step<D3Q19, 0>(fin, fout, p, mode, tile_max, k_field, s);
        case 1:
            if (tma) return launch_fused_step_tma<1>(fin, fout, p, mode, tile_max, k_field, s);
            return pair ? launch_fused_step_pair<D3Q19, 1>(fin, fout, p, mode, tile_max, k_field, s)
                        : launch_fused_step<D3Q19, 1>(fin, fout, p, mode, tile_max, k_field, s);
        case 2:
            if (tma) return launch_fused_step_tma<2>(fin, fout, p, mode, tile_max, k_field, s);
            return pair ? launch_fused_step_pair<D3Q19, 2>(fin, fout, p, mode, tile_max, k_field, s)
                        : launch_fused_step<D3Q19, 2>(fin, fout, p, mode, tile_max, k_field, s);
        case 3:
            if (tma) return launch_fused_step_tma<3>(fin, fout, p, mode, tile_max, k_field, s);
            return pair ? launch_fused_step_pair<D3Q19, 3>(fin, fout, p, mode, tile_max, k_field, s)
                        : launch_fused_step<D3Q19, 3>(fin, fout, p, mode, tile_max, k_field, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
