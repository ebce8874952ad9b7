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
#include <cudaTypedefs.h>
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

// tile maxima (first half) and block maxima (second half), as doubles or floats
static __device__ __align__(256) double g_noalloc_scratch[2 * LBM_NOALLOC_MAX_TILES];

// The device address of the array is a property of the CUDA context the module is loaded in, not
// of the device ordinal: after cudaDeviceReset, or under a caller's own (non-primary) context, the
// same ordinal has a new context and a new address.  Addresses are therefore cached per context,
// keyed by the driver's context ID, which is unique over the life of the process (a context created
// after a reset never reuses the ID of the one it replaces).
constexpr int kMaxContexts = 64;
struct Entry {
    unsigned long long ctx_id;
    void *addr;
};
std::mutex g_mu;
Entry g_cache[kMaxContexts] = {};
int g_cache_used = 0;
int g_cache_next = 0;  // next slot to overwrite once the table is full

struct DriverFns {
    PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    PFN_cuCtxGetId_v12000 get_id = nullptr;
};

const DriverFns &driver_fns() {
    static DriverFns fns;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fns.get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fns.get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f);
    });
    return fns;
}

// ID of the calling thread's current context (0 if there is none yet).
int current_context_id(unsigned long long *id) {
    const DriverFns &fns = driver_fns();
    if (!fns.get_current || !fns.get_id)
        return lbm::report_error(LBM_ECUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId "
                                            "unavailable");
    CUcontext ctx = nullptr;
    if (fns.get_current(&ctx) != CUDA_SUCCESS)
        return lbm::report_error(LBM_ECUDA, "cuCtxGetCurrent failed");
    *id = 0;
    if (ctx && fns.get_id(ctx, id) != CUDA_SUCCESS)
        return lbm::report_error(LBM_ECUDA, "cuCtxGetId failed");
    return LBM_OK;
}

// Device address of the scratch array in the calling thread's current context.  The host-side
// name of the array is only a stand-in; its device address is looked up with cudaGetSymbolAddress
// the first time a context calls, and cached under that context's ID.
int scratch_address(void **out) {
    unsigned long long id = 0;
    int st = current_context_id(&id);
    if (st != LBM_OK) return st;
    std::lock_guard<std::mutex> lock(g_mu);
    if (id != 0)
        for (int k = 0; k < g_cache_used; ++k)
            if (g_cache[k].ctx_id == id) {
                *out = g_cache[k].addr;
                return LBM_OK;
            }
    // first call in this context (or no context yet: the lookup makes the device's primary
    // context current, and its ID is read afterwards)
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return lbm::report_cuda_error(e, "cudaGetSymbolAddress");
    if (id == 0) {
        st = current_context_id(&id);
        if (st != LBM_OK) return st;
    }
    if (id != 0) {
        int slot;
        if (g_cache_used < kMaxContexts) {
            slot = g_cache_used++;
        } else {  // full: replace the oldest entry
            slot = g_cache_next;
            g_cache_next = (g_cache_next + 1) % kMaxContexts;
        }
        g_cache[slot] = Entry{id, p};
    }
    *out = p;
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
    // an error left pending by earlier work on this thread is reported as such, not as this
    // call's launch failure
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return lbm::report_cuda_error(e, "error pending before lbm_step_noalloc");
    void *scratch = nullptr;
    int st = scratch_address(&scratch);
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
