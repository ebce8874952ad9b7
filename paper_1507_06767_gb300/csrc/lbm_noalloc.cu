// lbm_step_noalloc: one fused step + block sensor maxima that allocates no device memory.
//
// Some callers cannot call cudaMalloc: applications that hand every byte of device memory out of
// their own pool and forbid libraries to allocate behind their back, and latency-critical loops
// where a cudaMalloc (which may synchronise the device) is not acceptable once set-up is over.
// For them this entry point keeps its only scratch -- the per-tile sensor maxima and the block
// maxima in the step's arithmetic type -- in one file-scope device array of fixed size, so a call
// needs nothing but the caller's own input, output and maxima buffers.
//
// The array belongs to the library's module: every GPU that loads the library holds it (4 MiB)
// until the process exits.  Every call shares it, so two calls whose kernels overlap on the GPU
// (different streams or devices sharing nothing else) race on it; issue them on one stream.  Its
// contents survive from call to call; nothing in it has to start at zero, because each call writes
// every tile maximum it later reads.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

// tile maxima (first half) and block maxima (second half), as doubles or floats
static __device__ __align__(256) double g_noalloc_scratch[2 * LBM_NOALLOC_MAX_TILES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The host-side name of the array is
// only a stand-in; its device address is looked up once per device, with that device current.
int scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices)
        return lbm::report_error(LBM_EINVAL, "device ordinal out of range for lbm_step_noalloc");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return lbm::report_cuda_error(e, "cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" LBM_API int lbm_step_noalloc(int lattice, int dtype, int nx, int ny, int nz, double tau,
                                        double lid_x, double lid_z, int periodic,
                                        const void *f_in_dev, void *f_out_dev, int block,
                                        double *block_max_dev, void *stream) {
    lbm::clear_error();
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19)
        return lbm::report_error(LBM_EINVAL, "lattice must be LBM_D2Q9 or LBM_D3Q19");
    if (dtype < LBM_F64 || dtype > LBM_BF16S)
        return lbm::report_error(LBM_EINVAL, "unknown storage type");
    if (nx < 1 || ny < 1 || nz < 1 || (lattice == LBM_D2Q9 && nz != 1))
        return lbm::report_error(LBM_EINVAL, "bad lattice dimensions");
    if ((unsigned long long)nx * ny * nz > 2147483647ull)
        return lbm::report_error(LBM_EINVAL, "lattice exceeds 2^31 - 1 cells");
    if (!(tau > 0.5) || !isfinite(tau) || !isfinite(lid_x) || !isfinite(lid_z))
        return lbm::report_error(LBM_EINVAL, "tau must be > 1/2 and the lid velocity finite");
    if (lattice == LBM_D2Q9 && lid_z != 0.0)
        return lbm::report_error(LBM_EINVAL, "D2Q9 lid has no z component");
    if (periodic & ~7) return lbm::report_error(LBM_EINVAL, "unknown periodic bits");
    if (block < LBM_TILE || block % LBM_TILE != 0)
        return lbm::report_error(LBM_EINVAL, "block edge must be a positive multiple of LBM_TILE");
    if (!f_in_dev || !f_out_dev || !block_max_dev || f_in_dev == f_out_dev)
        return lbm::report_error(LBM_EINVAL, "need distinct input and output buffers and maxima");
    const int dim = (lattice == LBM_D2Q9) ? 2 : 3;
    const int ntx = (nx + LBM_TILE - 1) / LBM_TILE, nty = (ny + LBM_TILE - 1) / LBM_TILE;
    const int ntz = (dim == 3) ? (nz + LBM_TILE - 1) / LBM_TILE : 1;
    const long long ntiles = (long long)ntx * nty * ntz;
    if (ntiles > LBM_NOALLOC_MAX_TILES) {
        char msg[160];
        snprintf(msg, sizeof(msg),
                 "lattice needs %lld sensor tiles; lbm_step_noalloc holds at most %d "
                 "(LBM_NOALLOC_MAX_TILES)", ntiles, LBM_NOALLOC_MAX_TILES);
        return lbm::report_error(LBM_EINVAL, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lbm::report_cuda_error(e, "cudaGetDevice");
    void *scratch = nullptr;
    int st = scratch_address(dev, &scratch);
    if (st != LBM_OK) return st;
    double *tiles = static_cast<double *>(scratch);
    double *blocks = tiles + LBM_NOALLOC_MAX_TILES;

    lbm::StepParams p;
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.periodic = (dim == 2) ? (periodic & 3) : periodic;
    p.ntx = ntx;
    p.nty = nty;
    p.ntz = ntz;
    p.omega = 1.0 / tau;
    p.lid_x = lid_x;
    p.lid_z = lid_z;
    lbm::finish_params(p);
    p.err = nullptr;
    p.tile_zero = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the automatic kernel choice (the same as lbm_step's default) only picks kernels that write
    // every tile maximum with a plain store, so the scratch needs no clearing between calls
    e = (lattice == LBM_D2Q9)
            ? lbm::step_d2q9(dtype, f_in_dev, f_out_dev, p, 1, tiles, nullptr, s, lbm::KERNEL_AUTO)
            : lbm::step_d3q19(dtype, f_in_dev, f_out_dev, p, 1, tiles, nullptr, s,
                              lbm::KERNEL_AUTO);
    if (e != cudaSuccess) return lbm::report_cuda_error(e, "fused step launch");
    const int m = block / LBM_TILE, mz = (dim == 3) ? m : 1;
    const int nbx = (nx + block - 1) / block, nby = (ny + block - 1) / block;
    const int nbz = (dim == 3) ? (nz + block - 1) / block : 1;
    const int rtype = (dtype == LBM_F64) ? LBM_F64 : LBM_F32;
    e = lbm::tiles_to_blocks(rtype, tiles, ntx, nty, ntz, m, mz, blocks, nbx, nby, nbz, s);
    if (e != cudaSuccess) return lbm::report_cuda_error(e, "tiles_to_blocks");
    e = lbm::to_f64(rtype, blocks, block_max_dev, (size_t)nbx * nby * nbz, s);
    if (e != cudaSuccess) return lbm::report_cuda_error(e, "to_f64");
    return LBM_OK;
}
