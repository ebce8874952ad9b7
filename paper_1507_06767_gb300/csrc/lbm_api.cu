// C-ABI layer of the library (declared in include/lbm.h): handle state, argument checking, device
// buffers, stream ordering, CUDA-graph replay of step runs, and the launches of the kernels in
// lbm_step_*.cu / lbm_aux.cu.  Host code only; every step of the computation runs in the kernels.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using lbm::StepParams;

namespace {

thread_local int g_err = LBM_OK;
thread_local char g_msg[512] = "";

int fail(int code, const char *fmt, ...) {
    g_err = code;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(LBM_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, (what)); \
    } while (0)

size_t elem_size(int dtype) {
    switch (dtype) {
        case LBM_F64: return 8;
        case LBM_F32: return 4;
        case LBM_F16S:
        case LBM_BF16S: return 2;
        default: return 0;
    }
}

}  // namespace

struct lbm_s {
    int q = 0, dim = 0;
    int nx = 0, ny = 0, nz = 0;
    size_t N = 0;
    double tau = 1.0;
    double lid_x = 0.1, lid_z = 0.0;
    int periodic = 0;
    int dtype = LBM_F32;
    int device = 0;
    cudaStream_t stream = nullptr;
    int sensor_every = 0;
    int sensor_field = 0;
    int block = 16;
    int graphs = 1;
    int variant = 0;  // LBM_KERNEL_*

    // population buffers
    void *buf[2] = {nullptr, nullptr};
    bool owned = false;
    int cur = 0;

    // sensor scratch: tile maxima of the last sensor step, block maxima, flags
    int ntx = 0, nty = 0, ntz = 0;
    size_t ntiles = 0;
    void *tiles = nullptr;        // tile maxima of the most recent sensor step (one of tilebuf)
    void *tilebuf[2] = {nullptr, nullptr};
    int tile_next = 0;            // buffer the next sensor step writes; it clears the other
    void *blocks = nullptr;
    double *blocks_f64 = nullptr;
    int8_t *flags = nullptr;
    void *kfield = nullptr;
    double *cons_partial = nullptr;
    double *cons_result = nullptr;
    // error word of the kernels' bounded waits: pinned host memory mapped into the device
    int *err_host = nullptr;
    int *err_dev = nullptr;
    double *staging = nullptr;  // staging_cap >= max(N, 64) doubles, for host transfers in double
    size_t staging_cap = 0;
    bool scratch_ready = false;

    long long t = 0;
    bool have_sensor = false;
    bool have_kfield = false;

    // time average of the tile maxima over sensor steps
    bool averaging = false;
    long long avg_count = 0;
    double *tile_sum = nullptr;
    double *tile_avg = nullptr;

    // halo planes of a slab cut along the slowest axis (lbm_set_halo): q x plane values each, and
    // a compact message buffer for host transfers
    void *halo[2] = {nullptr, nullptr};
    void *halo_msg = nullptr;
    int halo_faces = 0;

    // profiling
    int profiling = 0;
    unsigned long long wait_ns = 0;  // lbm_debug_set_wait_limit (0: the kernels' default)
    int hold_copies = 0;             // lbm_debug_hold_copies
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;

    // multi-level block mesh of lbm_blocks_step (built on first use)
    lbm::ml::Mesh *mesh = nullptr;
    int blocks_fusion = 0;  // LBM_FUSION_* for the next mesh build
    int blocks_step_form = 0;  // LBM_STEP_FORM_* for the next mesh build
    int blocks_schedule = 0;   // LBM_SCHEDULE_* for the next mesh build

    // graph cache: runs of RUN_LEN[k] plain steps (k = 0: 2 steps, 1: 16 steps), by starting
    // buffer
    cudaGraphExec_t pair_exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaStream_t pair_stream[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    bool pair_valid = false;

    int rtype() const { return dtype == LBM_F64 ? LBM_F64 : LBM_F32; }
    size_t rsize() const { return dtype == LBM_F64 ? 8 : 4; }
    size_t pop_bytes() const { return (size_t)q * N * elem_size(dtype); }
    // the slab axis is the slowest one: z for D3Q19, y for D2Q9
    int slab_axis_bit() const { return dim == 3 ? 4 : 2; }
    size_t halo_plane() const { return dim == 3 ? (size_t)nx * ny : (size_t)nx; }
    int slab_extent() const { return dim == 3 ? nz : ny; }
};

namespace {

constexpr int RUN_LEN[2] = {2, 16};  // plain steps per cached graph (even: parity is kept)

void drop_graphs(lbm_t *h) {
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) {
            if (h->pair_exec[j][k]) cudaGraphExecDestroy(h->pair_exec[j][k]);
            h->pair_exec[j][k] = nullptr;
        }
    h->pair_valid = false;
}

StepParams params_of(const lbm_t *h) {
    StepParams p;
    p.nx = h->nx;
    p.ny = h->ny;
    p.nz = h->nz;
    p.periodic = h->periodic;
    p.ntx = h->ntx;
    p.nty = h->nty;
    p.ntz = h->ntz;
    p.omega = 1.0 / h->tau;
    p.lid_x = h->lid_x;
    p.lid_z = h->lid_z;
    lbm::finish_params(p);
    p.err = h->err_dev;
    p.tile_zero = nullptr;
    p.wait_ns = h->wait_ns;
    p.hold_copies = h->hold_copies;
    p.halo_lo = (h->halo_faces & LBM_HALO_LO) ? h->halo[0] : nullptr;
    p.halo_hi = (h->halo_faces & LBM_HALO_HI) ? h->halo[1] : nullptr;
    return p;
}

int ensure_scratch(lbm_t *h) {
    if (h->scratch_ready) return LBM_OK;
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    // each buffer is allocated only if it does not exist yet: after a failed allocation the
    // handle keeps what it got (lbm_destroy frees it) and the next call continues from there
    if (!h->tilebuf[0]) CK(lbm::dev_alloc(&h->tilebuf[0], h->ntiles * h->rsize()), "cudaMalloc(tiles)");
    if (!h->tilebuf[1]) CK(lbm::dev_alloc(&h->tilebuf[1], h->ntiles * h->rsize()), "cudaMalloc(tiles)");
    CK(cudaMemset(h->tilebuf[0], 0, h->ntiles * h->rsize()), "cudaMemset(tiles)");
    CK(cudaMemset(h->tilebuf[1], 0, h->ntiles * h->rsize()), "cudaMemset(tiles)");
    h->tiles = h->tilebuf[0];
    h->tile_next = 0;
    if (!h->blocks) CK(lbm::dev_alloc(&h->blocks, h->ntiles * h->rsize()), "cudaMalloc(blocks)");
    if (!h->blocks_f64)
        CK(lbm::dev_alloc(&h->blocks_f64, h->ntiles * sizeof(double)), "cudaMalloc(blocks_f64)");
    if (!h->flags) CK(lbm::dev_alloc(&h->flags, h->ntiles), "cudaMalloc(flags)");
    if (!h->cons_partial)
        CK(lbm::dev_alloc(&h->cons_partial, lbm::CONS_PARTS * 5 * sizeof(double)),
           "cudaMalloc(partial)");
    if (!h->cons_result) CK(lbm::dev_alloc(&h->cons_result, 8 * sizeof(double)), "cudaMalloc(result)");
    if (!h->err_host)
        CK(cudaHostAlloc((void **)&h->err_host, sizeof(int), cudaHostAllocMapped),
           "cudaHostAlloc(err)");
    *h->err_host = 0;
    CK(cudaHostGetDevicePointer((void **)&h->err_dev, h->err_host, 0), "cudaHostGetDevicePointer");
    h->scratch_ready = true;
    return LBM_OK;
}

int ensure_buffers(lbm_t *h) {
    int st = ensure_scratch(h);
    if (st != LBM_OK) return st;
    if (h->buf[0]) return LBM_OK;
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    const size_t bytes = h->pop_bytes();
    cudaError_t e = lbm::dev_alloc(&h->buf[0], bytes);
    if (e != cudaSuccess) {
        h->buf[0] = nullptr;
        return cuda_fail(e, "cudaMalloc(populations A)");
    }
    e = lbm::dev_alloc(&h->buf[1], bytes);
    if (e != cudaSuccess) {
        cudaFree(h->buf[0]);
        h->buf[0] = nullptr;
        h->buf[1] = nullptr;
        return cuda_fail(e, "cudaMalloc(populations B)");
    }
    h->owned = true;
    h->cur = 0;
    CK(lbm::init_rest(h->q, h->dtype, h->buf[0], h->N, h->stream), "init_rest");
    h->t = 0;
    h->have_sensor = false;
    return LBM_OK;
}

int ensure_staging(lbm_t *h) {
    if (h->staging) return LBM_OK;
    const size_t cap = h->N > 64 ? h->N : 64;
    CK(lbm::dev_alloc((void **)&h->staging, cap * sizeof(double)), "cudaMalloc(staging)");
    h->staging_cap = cap;
    return LBM_OK;
}

int ensure_kfield(lbm_t *h) {
    if (h->kfield) return LBM_OK;
    CK(lbm::dev_alloc(&h->kfield, h->N * h->rsize()), "cudaMalloc(k field)");
    return LBM_OK;
}

cudaError_t launch_step(lbm_t *h, int src, int mode) {
    StepParams p = params_of(h);
    void *tiles = mode ? h->tilebuf[h->tile_next] : nullptr;
    if (mode) p.tile_zero = h->tilebuf[h->tile_next ^ 1];
    void *kf = (mode == 2) ? h->kfield : nullptr;
    if (h->q == LBM_D2Q9)
        return lbm::step_d2q9(h->dtype, h->buf[src], h->buf[src ^ 1], p, mode, tiles, kf, h->stream,
                              h->variant);
    return lbm::step_d3q19(h->dtype, h->buf[src], h->buf[src ^ 1], p, mode, tiles, kf, h->stream,
                           h->variant);
}

int timed_step(lbm_t *h, int mode) {
    if (h->profiling) {
        if (h->events_used + 2 > h->events.size()) {
            for (int k = 0; k < 64; ++k) {
                cudaEvent_t ev;
                CK(cudaEventCreate(&ev), "cudaEventCreate");
                h->events.push_back(ev);
            }
        }
        CK(cudaEventRecord(h->events[h->events_used], h->stream), "cudaEventRecord");
    }
    CK(launch_step(h, h->cur, mode), "fused step launch");
    if (h->profiling) {
        CK(cudaEventRecord(h->events[h->events_used + 1], h->stream), "cudaEventRecord");
        h->events_used += 2;
    }
    h->cur ^= 1;
    h->t += 1;
    if (mode) {
        h->tiles = h->tilebuf[h->tile_next];
        h->tile_next ^= 1;
        h->have_sensor = true;
        h->have_kfield = (mode == 2);
        if (h->averaging) {
            CK(lbm::accumulate_tiles(h->rtype(), h->tiles, h->tile_sum, h->ntiles, h->stream),
               "accumulate_tiles");
            h->avg_count += 1;
        }
    }
    return LBM_OK;
}

// Capture (once per stream and starting buffer) a graph of two plain steps: src -> other -> src.
// The cached graph of RUN_LEN[len] plain steps starting from buffer src (captured on first use).
int pair_graph(lbm_t *h, int src, int len, cudaGraphExec_t *out) {
    cudaGraphExec_t &slot = h->pair_exec[len][src];
    if (h->pair_valid && slot && h->pair_stream[len][src] == h->stream) {
        *out = slot;
        return LBM_OK;
    }
    if (slot) {
        cudaGraphExecDestroy(slot);
        slot = nullptr;
    }
    cudaStream_t cap;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const StepParams p = params_of(h);
        for (int k = 0; k < RUN_LEN[len] && e == cudaSuccess; ++k) {
            const int s = src ^ (k & 1);
            if (h->q == LBM_D2Q9)
                e = lbm::step_d2q9(h->dtype, h->buf[s], h->buf[s ^ 1], p, 0, nullptr, nullptr, cap,
                                   h->variant);
            else
                e = lbm::step_d3q19(h->dtype, h->buf[s], h->buf[s ^ 1], p, 0, nullptr, nullptr, cap,
                                    h->variant);
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&slot, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        slot = nullptr;
        return cuda_fail(e, "graph capture");
    }
    h->pair_stream[len][src] = h->stream;
    h->pair_valid = true;
    *out = slot;
    return LBM_OK;
}

int check_block(const lbm_t *h, int block, int *nbx, int *nby, int *nbz, int *m, int *mz) {
    if (block < LBM_TILE || block % LBM_TILE != 0)
        return fail(LBM_EINVAL, "block edge %d is not a positive multiple of %d", block, LBM_TILE);
    *m = block / LBM_TILE;
    *mz = (h->dim == 3) ? *m : 1;
    *nbx = (h->nx + block - 1) / block;
    *nby = (h->ny + block - 1) / block;
    *nbz = (h->dim == 3) ? (h->nz + block - 1) / block : 1;
    return LBM_OK;
}

// Block maxima (native type) of the last sensor step into h->blocks; returns the block count.
int reduce_blocks(lbm_t *h, int block, int *nb_out) {
    if (!h->have_sensor) return fail(LBM_ESTATE, "no sensor step since the last reset");
    int nbx, nby, nbz, m, mz;
    int st = check_block(h, block, &nbx, &nby, &nbz, &m, &mz);
    if (st != LBM_OK) return st;
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    CK(lbm::tiles_to_blocks(h->rtype(), h->tiles, h->ntx, h->nty, h->ntz, m, mz, h->blocks, nbx,
                            nby, nbz, h->stream),
       "tiles_to_blocks");
    *nb_out = nbx * nby * nbz;
    return LBM_OK;
}

int top_count(double frac, int n) {
    double k = ceil(frac * (double)n);
    if (k < 0) k = 0;
    if (k > n) k = n;
    return (int)k;
}

int sync(lbm_t *h) {
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (h->err_host && *(volatile int *)h->err_host)
        return fail(LBM_ETIMEOUT, "a bounded wait in the fused step kernel ran out; results of the "
                                  "steps since the last reset are not valid");
    return LBM_OK;
}

#define CHECK_H(h)                                                 \
    do {                                                           \
        if (!(h)) return fail(LBM_EINVAL, "NULL handle");          \
    } while (0)

// An error left pending on the thread by earlier CUDA work (the caller's or ours) is reported as
// such before a call launches anything, and is not cleared; otherwise the launch's own status check
// (cudaGetLastError after the launch) would report, and clear, it as this call's failure.
#define CHECK_PENDING(where)                                                              \
    do {                                                                                  \
        cudaError_t pe_ = cudaPeekAtLastError();                                          \
        if (pe_ != cudaSuccess)                                                           \
            return fail(LBM_ECUDA, "error pending before %s (left by earlier CUDA work on " \
                                   "this thread): %s", (where), cudaGetErrorString(pe_)); \
    } while (0)

}  // namespace

namespace lbm {
// Failure injection of lbm_debug_fail_alloc: the number of further allocations that succeed before
// one fails (-1: disarmed).
std::atomic<long long> g_fail_alloc_after{-1};

cudaError_t dev_alloc(void **p, size_t bytes) {
    long long c = g_fail_alloc_after.load();
    while (c >= 0) {
        if (g_fail_alloc_after.compare_exchange_weak(c, c - 1)) {
            if (c == 0) {  // this is the allocation that fails; the hook is disarmed now
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

// Error reporting for the other C-ABI translation units (same thread-local state as this file).
int report_error(int code, const char *msg) { return fail(code, "%s", msg); }
int report_cuda_error(cudaError_t e, const char *what) { return cuda_fail(e, what); }
void clear_error() { g_err = LBM_OK; }
}  // namespace lbm

extern "C" {

LBM_API int lbm_last_error(void) { return g_err; }
LBM_API const char *lbm_last_message(void) { return g_msg; }
LBM_API int lbm_version(void) { return 100; }

LBM_API const char *lbm_strerror(int status) {
    switch (status) {
        case LBM_OK: return "ok";
        case LBM_EINVAL: return "invalid argument";
        case LBM_ENOMEM: return "out of device memory";
        case LBM_ECUDA: return "CUDA error";
        case LBM_ENUMERIC: return "non-finite populations";
        case LBM_ETIMEOUT: return "device wait timed out";
        case LBM_ENOTSUP: return "not supported";
        case LBM_ESTATE: return "not allowed in the current state";
        case LBM_EIO: return "checkpoint file error";
        default: return "unknown status";
    }
}

LBM_API lbm_t *lbm_create(int lattice, int nx, int ny, int nz, double tau) {
    g_err = LBM_OK;
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19) {
        fail(LBM_EINVAL, "lattice must be LBM_D2Q9 (9) or LBM_D3Q19 (19), got %d", lattice);
        return nullptr;
    }
    if (nx < 1 || ny < 1 || nz < 1) {
        fail(LBM_EINVAL, "lattice dimensions must be >= 1 (got %d x %d x %d)", nx, ny, nz);
        return nullptr;
    }
    if (lattice == LBM_D2Q9 && nz != 1) {
        fail(LBM_EINVAL, "D2Q9 needs nz == 1 (got %d)", nz);
        return nullptr;
    }
    if (!(tau > 0.5) || !isfinite(tau)) {
        fail(LBM_EINVAL, "tau must be a finite value > 1/2 (got %g)", tau);
        return nullptr;
    }
    const unsigned long long cells = (unsigned long long)nx * ny * nz;
    if (cells > (unsigned long long)INT_MAX) {
        fail(LBM_EINVAL, "lattice of %llu cells exceeds 2^31 - 1", cells);
        return nullptr;
    }
    int dev = 0;
    lbm_t *h = new (std::nothrow) lbm_t();
    if (!h) {
        fail(LBM_ENOMEM, "host allocation failed");
        return nullptr;
    }
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    h->q = lattice;
    h->dim = (lattice == LBM_D2Q9) ? 2 : 3;
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->N = (size_t)cells;
    h->tau = tau;
    h->device = dev;
    h->ntx = (nx + LBM_TILE - 1) / LBM_TILE;
    h->nty = (ny + LBM_TILE - 1) / LBM_TILE;
    h->ntz = (h->dim == 3) ? (nz + LBM_TILE - 1) / LBM_TILE : 1;
    h->ntiles = (size_t)h->ntx * h->nty * h->ntz;
    return h;
}

LBM_API int lbm_destroy(lbm_t *h) {
    CHECK_H(h);
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    for (cudaEvent_t ev : h->events) cudaEventDestroy(ev);
    if (h->owned) {
        cudaFree(h->buf[0]);
        cudaFree(h->buf[1]);
    }
    cudaFree(h->tilebuf[0]);
    cudaFree(h->tilebuf[1]);
    cudaFree(h->blocks);
    cudaFree(h->blocks_f64);
    cudaFree(h->flags);
    cudaFree(h->kfield);
    cudaFree(h->cons_partial);
    cudaFree(h->cons_result);
    cudaFree(h->staging);
    cudaFree(h->tile_sum);
    cudaFree(h->tile_avg);
    cudaFree(h->halo[0]);
    cudaFree(h->halo[1]);
    cudaFree(h->halo_msg);
    if (h->err_host) cudaFreeHost(h->err_host);
    lbm::ml::destroy(h->mesh);
    delete h;
    return LBM_OK;
}

LBM_API int lbm_set_dtype(lbm_t *h, int dtype) {
    CHECK_H(h);
    if (elem_size(dtype) == 0) return fail(LBM_EINVAL, "unknown storage type %d", dtype);
    if (h->buf[0] || h->scratch_ready || h->halo[0] || h->halo[1])
        return fail(LBM_ESTATE, "storage type must be set before the buffers exist");
    h->dtype = dtype;
    return LBM_OK;
}

LBM_API int lbm_set_lid(lbm_t *h, double ux, double uz) {
    CHECK_H(h);
    if (!isfinite(ux) || !isfinite(uz)) return fail(LBM_EINVAL, "lid velocity must be finite");
    if (h->dim == 2 && uz != 0.0) return fail(LBM_EINVAL, "D2Q9 lid has no z component");
    h->lid_x = ux;
    h->lid_z = uz;
    drop_graphs(h);
    return LBM_OK;
}

LBM_API int lbm_set_periodic(lbm_t *h, int axis_mask) {
    CHECK_H(h);
    if (axis_mask & ~7) return fail(LBM_EINVAL, "periodic mask %d has unknown bits", axis_mask);
    if (h->halo_faces && (axis_mask & h->slab_axis_bit()))
        return fail(LBM_EINVAL, "the slab axis has halo faces: it cannot also be periodic");
    h->periodic = (h->dim == 2) ? (axis_mask & 3) : axis_mask;
    drop_graphs(h);
    return LBM_OK;
}

LBM_API int lbm_set_tau(lbm_t *h, double tau) {
    CHECK_H(h);
    if (!(tau > 0.5) || !isfinite(tau)) return fail(LBM_EINVAL, "tau must be > 1/2 (got %g)", tau);
    h->tau = tau;
    drop_graphs(h);
    return LBM_OK;
}

LBM_API int lbm_set_stream(lbm_t *h, void *stream) {
    CHECK_H(h);
    h->stream = static_cast<cudaStream_t>(stream);
    return LBM_OK;
}

LBM_API int lbm_set_sensor_every(lbm_t *h, int k) {
    CHECK_H(h);
    if (k < 0) return fail(LBM_EINVAL, "sensor period must be >= 0 (got %d)", k);
    h->sensor_every = k;
    return LBM_OK;
}

LBM_API int lbm_set_sensor_field(lbm_t *h, int on) {
    CHECK_H(h);
    h->sensor_field = on ? 1 : 0;
    return LBM_OK;
}

LBM_API int lbm_set_block(lbm_t *h, int block) {
    CHECK_H(h);
    if (block < LBM_TILE || block % LBM_TILE != 0)
        return fail(LBM_EINVAL, "block edge %d is not a positive multiple of %d", block, LBM_TILE);
    h->block = block;
    return LBM_OK;
}

LBM_API int lbm_set_profiling(lbm_t *h, int on) {
    CHECK_H(h);
    h->profiling = on ? 1 : 0;
    h->events_used = 0;
    return LBM_OK;
}

LBM_API int lbm_set_kernel_variant(lbm_t *h, int variant) {
    CHECK_H(h);
    if (variant < LBM_KERNEL_AUTO || variant > LBM_KERNEL_TMA_PAIR)
        return fail(LBM_EINVAL, "unknown kernel variant %d", variant);
    if (variant == LBM_KERNEL_TMA_PAIR &&
        (h->q != LBM_D3Q19 || (h->dtype != LBM_F16S && h->dtype != LBM_BF16S) || h->nx % 8 != 0 ||
         20ULL * ((unsigned long long)h->nx * h->ny * h->nz) >= (1ULL << 32)))
        return fail(LBM_EINVAL,
                    "the TMA two-cell kernel needs D3Q19, 16-bit storage, nx a multiple of 8 and "
                    "20 * cells < 2^32");
    if (variant == LBM_KERNEL_PAIR &&
        (h->dtype == LBM_F64 || h->nx % 2 != 0 ||
         (unsigned long long)(h->q + 1) * ((unsigned long long)h->nx * h->ny * h->nz) >=
             (1ULL << 32)))
        return fail(LBM_EINVAL,
                    "the two-cell kernel needs FP32 arithmetic, an even nx and (q + 1) * cells "
                    "< 2^32");
    if (variant == LBM_KERNEL_TMA &&
        (h->q != LBM_D3Q19 || h->dtype == LBM_F64 ||
         (long long)h->nx * (h->dtype == LBM_F32 ? 4 : 2) % 16 != 0))
        return fail(LBM_EINVAL,
                    "the TMA kernel needs D3Q19, 16- or 32-bit storage and rows of a multiple of "
                    "16 bytes");
    if (h->halo_faces && variant != LBM_KERNEL_AUTO && variant != LBM_KERNEL_CELL)
        return fail(LBM_EINVAL, "a slab with halo faces runs the one-cell kernel only");
    h->variant = variant;
    drop_graphs(h);
    return LBM_OK;
}

LBM_API int lbm_set_graphs(lbm_t *h, int on) {
    CHECK_H(h);
    h->graphs = on ? 1 : 0;
    return LBM_OK;
}

LBM_API int lbm_attach(lbm_t *h, void *a_dev, void *b_dev, size_t bytes) {
    CHECK_H(h);
    if (!a_dev || !b_dev || a_dev == b_dev) return fail(LBM_EINVAL, "need two distinct buffers");
    if (bytes < h->pop_bytes())
        return fail(LBM_EINVAL, "buffers of %zu bytes are smaller than %zu", bytes, h->pop_bytes());
    if (((uintptr_t)a_dev | (uintptr_t)b_dev) & 15)
        return fail(LBM_EINVAL, "buffers must be 16-byte aligned");
    int st = ensure_scratch(h);
    if (st != LBM_OK) return st;
    drop_graphs(h);
    if (h->owned) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->buf[0]);
        cudaFree(h->buf[1]);
    }
    h->buf[0] = a_dev;
    h->buf[1] = b_dev;
    h->owned = false;
    h->cur = 0;
    h->t = 0;
    h->have_sensor = false;
    return LBM_OK;
}

LBM_API size_t lbm_population_bytes(const lbm_t *h) { return h ? h->pop_bytes() : 0; }

LBM_API int lbm_nblocks(const lbm_t *h, int block) {
    if (!h || block < LBM_TILE || block % LBM_TILE != 0) return 0;
    int nbx = (h->nx + block - 1) / block, nby = (h->ny + block - 1) / block;
    int nbz = (h->dim == 3) ? (h->nz + block - 1) / block : 1;
    return nbx * nby * nbz;
}

LBM_API long long lbm_steps_done(const lbm_t *h) { return h ? h->t : -1; }

LBM_API int lbm_reset(lbm_t *h) {
    CHECK_H(h);
    if (h->mesh) {
        cudaStreamSynchronize(h->stream);
        lbm::ml::destroy(h->mesh);
        h->mesh = nullptr;
    }
    int st = ensure_buffers(h);
    if (st != LBM_OK) return st;
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    CK(lbm::init_rest(h->q, h->dtype, h->buf[h->cur], h->N, h->stream), "init_rest");
    h->t = 0;
    h->have_sensor = false;
    h->have_kfield = false;
    CK(cudaMemsetAsync(h->tilebuf[0], 0, h->ntiles * h->rsize(), h->stream), "memset(tiles)");
    CK(cudaMemsetAsync(h->tilebuf[1], 0, h->ntiles * h->rsize(), h->stream), "memset(tiles)");
    h->tiles = h->tilebuf[0];
    h->tile_next = 0;
    CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    *h->err_host = 0;
    return LBM_OK;
}

LBM_API int lbm_step(lbm_t *h, int n) {
    CHECK_H(h);
    if (n < 0) return fail(LBM_EINVAL, "step count must be >= 0 (got %d)", n);
    CHECK_PENDING("lbm_step");
    int st = ensure_buffers(h);
    if (st != LBM_OK) return st;
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    if (h->sensor_field) {
        st = ensure_kfield(h);
        if (st != LBM_OK) return st;
    }
    const int sensor_mode = h->sensor_field ? 2 : 1;
    int s = 0;
    while (s < n) {
        const long long t1 = h->t + 1;
        const bool sensor = (h->sensor_every > 0) ? (t1 % h->sensor_every == 0) : (s == n - 1);
        if (!sensor && !h->profiling && h->graphs) {
            // length of the run of plain steps starting here
            int run = 0;
            while (s + run < n) {
                const long long tt = h->t + 1 + run;
                const bool sen =
                    (h->sensor_every > 0) ? (tt % h->sensor_every == 0) : (s + run == n - 1);
                if (sen) break;
                ++run;
            }
            if (run >= 4) {
                // whole runs of 16 steps, then pairs; every graph keeps the buffer parity
                for (int len = 1; len >= 0; --len) {
                    const int count = run / RUN_LEN[len];
                    if (count == 0) continue;
                    cudaGraphExec_t ge;
                    st = pair_graph(h, h->cur, len, &ge);
                    if (st != LBM_OK) return st;
                    for (int k = 0; k < count; ++k)
                        CK(cudaGraphLaunch(ge, h->stream), "cudaGraphLaunch");
                    h->t += (long long)count * RUN_LEN[len];
                    s += count * RUN_LEN[len];
                    run -= count * RUN_LEN[len];
                }
                continue;
            }
        }
        st = timed_step(h, sensor ? sensor_mode : 0);
        if (st != LBM_OK) return st;
        ++s;
    }
    return LBM_OK;
}

LBM_API int lbm_sensor(lbm_t *h, int block, double *out_host) {
    CHECK_H(h);
    if (!out_host) return fail(LBM_EINVAL, "NULL output");
    int nb = 0;
    int st = reduce_blocks(h, block, &nb);
    if (st != LBM_OK) return st;
    CK(lbm::to_f64(h->rtype(), h->blocks, h->blocks_f64, (size_t)nb, h->stream), "to_f64");
    CK(cudaMemcpyAsync(out_host, h->blocks_f64, (size_t)nb * sizeof(double),
                       cudaMemcpyDeviceToHost, h->stream),
       "cudaMemcpyAsync");
    return sync(h);
}

LBM_API int lbm_sensor_dev(lbm_t *h, int block, double *out_dev) {
    CHECK_H(h);
    if (!out_dev) return fail(LBM_EINVAL, "NULL output");
    int nb = 0;
    int st = reduce_blocks(h, block, &nb);
    if (st != LBM_OK) return st;
    CK(lbm::to_f64(h->rtype(), h->blocks, out_dev, (size_t)nb, h->stream), "to_f64");
    return LBM_OK;
}

static int flag_common(lbm_t *h, int rule, double param, int8_t *out, bool host) {
    CHECK_H(h);
    if (!out) return fail(LBM_EINVAL, "NULL output");
    if (rule == LBM_FLAG_THRESHOLD && !isfinite(param))
        return fail(LBM_EINVAL, "threshold must be finite");
    if (rule == LBM_FLAG_TOP && !(param >= 0.0 && param <= 1.0))
        return fail(LBM_EINVAL, "fraction must be in [0, 1] (got %g)", param);
    if (!h->have_sensor) return fail(LBM_ESTATE, "no sensor step since the last reset");
    int nbx, nby, nbz, m, mz;
    int st = check_block(h, h->block, &nbx, &nby, &nbz, &m, &mz);
    if (st != LBM_OK) return st;
    CHECK_PENDING("lbm_flag");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    const int nb = nbx * nby * nbz;
    int8_t *dst = host ? h->flags : out;
    // block maxima (kept in h->blocks, as reduce_blocks leaves them) and flags
    CK(lbm::flags_from_tiles(h->rtype(), h->tiles, h->ntx, h->nty, h->ntz, m, mz, h->blocks, nbx,
                             nby, nbz, rule == LBM_FLAG_THRESHOLD ? 0 : 1, param,
                             rule == LBM_FLAG_TOP ? top_count(param, nb) : 0, dst, h->stream),
       "flags");
    if (host) {
        CK(cudaMemcpyAsync(out, h->flags, (size_t)nb, cudaMemcpyDeviceToHost, h->stream),
           "cudaMemcpyAsync");
        return sync(h);
    }
    return LBM_OK;
}

LBM_API int lbm_flag(lbm_t *h, double threshold, int8_t *out_host) {
    return flag_common(h, LBM_FLAG_THRESHOLD, threshold, out_host, true);
}
LBM_API int lbm_flag_dev(lbm_t *h, double threshold, int8_t *out_dev) {
    return flag_common(h, LBM_FLAG_THRESHOLD, threshold, out_dev, false);
}
LBM_API int lbm_flag_top(lbm_t *h, double frac, int8_t *out_host) {
    return flag_common(h, LBM_FLAG_TOP, frac, out_host, true);
}
LBM_API int lbm_flag_top_dev(lbm_t *h, double frac, int8_t *out_dev) {
    return flag_common(h, LBM_FLAG_TOP, frac, out_dev, false);
}

LBM_API int lbm_flags_from_maxima(const void *maxima_dev, int maxima_dtype, int n, int rule,
                                  double param, int8_t *out_dev, void *stream) {
    g_err = LBM_OK;
    if (n < 0) return fail(LBM_EINVAL, "n must be >= 0");
    if (n > 0 && (!maxima_dev || !out_dev)) return fail(LBM_EINVAL, "NULL pointer");
    if (maxima_dtype != LBM_F32 && maxima_dtype != LBM_F64)
        return fail(LBM_EINVAL, "maxima type must be LBM_F32 or LBM_F64");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (rule == LBM_FLAG_THRESHOLD) {
        if (!isfinite(param)) return fail(LBM_EINVAL, "threshold must be finite");
        if (n == 0) return LBM_OK;
        CK(lbm::flags_threshold(maxima_dtype, maxima_dev, n, param, out_dev, s), "flags");
    } else if (rule == LBM_FLAG_TOP) {
        if (!(param >= 0.0 && param <= 1.0)) return fail(LBM_EINVAL, "fraction must be in [0, 1]");
        if (n == 0) return LBM_OK;
        CK(lbm::flags_top(maxima_dtype, maxima_dev, n, top_count(param, n), out_dev, s), "flags");
    } else {
        return fail(LBM_EINVAL, "unknown flag rule %d", rule);
    }
    return LBM_OK;
}

LBM_API int lbm_get_populations(lbm_t *h, double *out_host) {
    CHECK_H(h);
    if (!out_host) return fail(LBM_EINVAL, "NULL output");
    int st = ensure_buffers(h);
    if (st == LBM_OK) st = ensure_staging(h);
    if (st != LBM_OK) return st;
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    const size_t es = elem_size(h->dtype);
    for (int i = 0; i < h->q; ++i) {
        const char *src = static_cast<const char *>(h->buf[h->cur]) + (size_t)i * h->N * es;
        CK(lbm::storage_to_f64(h->q, h->dtype, i, 1, src, h->staging, h->N, h->stream), "to_f64");
        CK(cudaMemcpyAsync(out_host + (size_t)i * h->N, h->staging, h->N * sizeof(double),
                           cudaMemcpyDeviceToHost, h->stream),
           "cudaMemcpyAsync");
    }
    return sync(h);
}

LBM_API int lbm_set_populations(lbm_t *h, const double *in_host) {
    CHECK_H(h);
    if (!in_host) return fail(LBM_EINVAL, "NULL input");
    int st = ensure_buffers(h);
    if (st == LBM_OK) st = ensure_staging(h);
    if (st != LBM_OK) return st;
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    const size_t es = elem_size(h->dtype);
    for (int i = 0; i < h->q; ++i) {
        char *dst = static_cast<char *>(h->buf[h->cur]) + (size_t)i * h->N * es;
        CK(cudaMemcpyAsync(h->staging, in_host + (size_t)i * h->N, h->N * sizeof(double),
                           cudaMemcpyHostToDevice, h->stream),
           "cudaMemcpyAsync");
        CK(lbm::f64_to_storage(h->q, h->dtype, i, 1, h->staging, dst, h->N, h->stream), "from_f64");
    }
    return sync(h);
}

LBM_API int lbm_get_raw(lbm_t *h, void *out_host, size_t bytes) {
    CHECK_H(h);
    if (!out_host) return fail(LBM_EINVAL, "NULL output");
    if (bytes != h->pop_bytes())
        return fail(LBM_EINVAL, "raw size %zu != population bytes %zu", bytes, h->pop_bytes());
    int st = ensure_buffers(h);
    if (st != LBM_OK) return st;
    CK(cudaMemcpyAsync(out_host, h->buf[h->cur], bytes, cudaMemcpyDeviceToHost, h->stream),
       "cudaMemcpyAsync");
    return sync(h);
}

LBM_API int lbm_set_raw(lbm_t *h, const void *in_host, size_t bytes) {
    CHECK_H(h);
    if (!in_host) return fail(LBM_EINVAL, "NULL input");
    if (bytes != h->pop_bytes())
        return fail(LBM_EINVAL, "raw size %zu != population bytes %zu", bytes, h->pop_bytes());
    int st = ensure_buffers(h);
    if (st != LBM_OK) return st;
    CK(cudaMemcpyAsync(h->buf[h->cur], in_host, bytes, cudaMemcpyHostToDevice, h->stream),
       "cudaMemcpyAsync");
    return sync(h);
}

// ------------------------------------------------------------------------------ slab halos
namespace {

// directions whose velocity component along the slab axis is `sign`, in index order
lbm::HaloDirs slab_dirs(const lbm_t *h, int sign) {
    lbm::HaloDirs d{};
    d.k = 0;
    for (int i = 0; i < h->q; ++i) {
        const int c = (h->q == LBM_D3Q19) ? lbm::D3Q19::cz(i) : lbm::D2Q9::cy(i);
        if (c == sign) d.dir[d.k++] = i;
    }
    return d;
}

int check_face(const lbm_t *h, int face) {
    if (face != LBM_HALO_LO && face != LBM_HALO_HI)
        return fail(LBM_EINVAL, "face must be LBM_HALO_LO or LBM_HALO_HI (got %d)", face);
    if (!(h->halo_faces & face)) return fail(LBM_ESTATE, "face %d has no halo (lbm_set_halo)", face);
    return LBM_OK;
}

int ensure_halo_msg(lbm_t *h) {
    if (h->halo_msg) return LBM_OK;
    const size_t bytes = (size_t)slab_dirs(h, 1).k * h->halo_plane() * elem_size(h->dtype);
    CK(lbm::dev_alloc(&h->halo_msg, bytes), "cudaMalloc(halo message)");
    return LBM_OK;
}

}  // namespace

LBM_API int lbm_set_halo(lbm_t *h, int faces) {
    CHECK_H(h);
    if (faces & ~(LBM_HALO_LO | LBM_HALO_HI))
        return fail(LBM_EINVAL, "halo faces %d have unknown bits", faces);
    if (faces && (h->periodic & h->slab_axis_bit()))
        return fail(LBM_EINVAL, "the slab axis is periodic: it cannot have halo faces");
    if (faces && h->variant != lbm::KERNEL_AUTO && h->variant != lbm::KERNEL_CELL)
        return fail(LBM_EINVAL, "halo faces need the one-cell kernel (LBM_KERNEL_AUTO or _CELL)");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    const size_t plane = h->halo_plane();
    const size_t bytes = (size_t)h->q * plane * elem_size(h->dtype);
    for (int f = 0; f < 2; ++f) {
        if (!((faces >> f) & 1) || h->halo[f]) continue;
        CK(lbm::dev_alloc(&h->halo[f], bytes), "cudaMalloc(halo)");
        // until the first import the halo holds fluid at rest
        CK(lbm::init_rest(h->q, h->dtype, h->halo[f], plane, h->stream), "init_rest(halo)");
    }
    h->halo_faces = faces;
    drop_graphs(h);
    return LBM_OK;
}

LBM_API int lbm_halo_size(const lbm_t *h, long long *elems, long long *bytes) {
    CHECK_H(h);
    const long long n = (long long)slab_dirs(h, 1).k * (long long)h->halo_plane();
    if (elems) *elems = n;
    if (bytes) *bytes = n * (long long)elem_size(h->dtype);
    return LBM_OK;
}

LBM_API int lbm_halo_export(lbm_t *h, int face, void *out, int on_device) {
    CHECK_H(h);
    int st = check_face(h, face);
    if (st != LBM_OK) return st;
    if (!out) return fail(LBM_EINVAL, "NULL output");
    CHECK_PENDING("lbm_halo_export");
    st = ensure_buffers(h);
    if (st == LBM_OK && !on_device) st = ensure_halo_msg(h);
    if (st != LBM_OK) return st;
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    // the populations leaving the slab through the face: velocity component -1 along the slab
    // axis on the low face, +1 on the high face, from the boundary plane of the current state
    const lbm::HaloDirs d = slab_dirs(h, face == LBM_HALO_LO ? -1 : 1);
    const size_t plane = h->halo_plane();
    const size_t off = (face == LBM_HALO_LO) ? 0 : (size_t)(h->slab_extent() - 1) * plane;
    const int elem = (int)elem_size(h->dtype);
    void *dst = on_device ? out : h->halo_msg;
    CK(lbm::halo_pack(elem, h->buf[h->cur], h->N, off, plane, d, dst, h->stream), "halo_pack");
    if (on_device) return LBM_OK;
    CK(cudaMemcpyAsync(out, h->halo_msg, (size_t)d.k * plane * elem, cudaMemcpyDeviceToHost,
                       h->stream),
       "cudaMemcpyAsync");
    return sync(h);
}

LBM_API int lbm_halo_import(lbm_t *h, int face, const void *in, int on_device) {
    CHECK_H(h);
    int st = check_face(h, face);
    if (st != LBM_OK) return st;
    if (!in) return fail(LBM_EINVAL, "NULL input");
    CHECK_PENDING("lbm_halo_import");
    if (!on_device) {
        st = ensure_halo_msg(h);
        if (st != LBM_OK) return st;
    }
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    // the populations arriving through the face: velocity component +1 along the slab axis on
    // the low face, -1 on the high face
    const lbm::HaloDirs d = slab_dirs(h, face == LBM_HALO_LO ? 1 : -1);
    const size_t plane = h->halo_plane();
    const int elem = (int)elem_size(h->dtype);
    const void *src = in;
    if (!on_device) {
        CK(cudaMemcpyAsync(h->halo_msg, in, (size_t)d.k * plane * elem, cudaMemcpyHostToDevice,
                           h->stream),
           "cudaMemcpyAsync");
        src = h->halo_msg;
    }
    CK(lbm::halo_unpack(elem, src, plane, d, h->halo[face == LBM_HALO_LO ? 0 : 1], h->stream),
       "halo_unpack");
    if (on_device) return LBM_OK;
    return sync(h);
}

LBM_API int lbm_get_moments(lbm_t *h, double *rho_host, double *u_host) {
    CHECK_H(h);
    if (!rho_host || !u_host) return fail(LBM_EINVAL, "NULL output");
    int st = ensure_buffers(h);
    if (st == LBM_OK) st = ensure_staging(h);
    if (st != LBM_OK) return st;
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    // staging holds staging_cap doubles: cells go in chunks of staging_cap / 4 (rho + 3 velocity
    // components)
    const size_t chunk = h->staging_cap / 4;
    for (size_t c0 = 0; c0 < h->N; c0 += chunk) {
        const size_t nc = (h->N - c0 < chunk) ? h->N - c0 : chunk;
        double *rho_d = h->staging;
        double *u_d = h->staging + nc;
        CK(lbm::moments_f64(h->q, h->dtype, h->buf[h->cur], h->N, c0, nc, rho_d, u_d, h->stream),
           "moments");
        CK(cudaMemcpyAsync(rho_host + c0, rho_d, nc * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream),
           "cudaMemcpyAsync");
        for (int a = 0; a < 3; ++a)
            CK(cudaMemcpyAsync(u_host + (size_t)a * h->N + c0, u_d + (size_t)a * nc,
                               nc * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
               "cudaMemcpyAsync");
        st = sync(h);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
}

LBM_API int lbm_get_sensor_field(lbm_t *h, double *out_host) {
    CHECK_H(h);
    if (!out_host) return fail(LBM_EINVAL, "NULL output");
    if (!h->have_kfield || !h->kfield)
        return fail(LBM_ESTATE, "no per-cell sensor recorded (lbm_set_sensor_field before stepping)");
    int st = ensure_staging(h);
    if (st != LBM_OK) return st;
    CK(lbm::to_f64(h->rtype(), h->kfield, h->staging, h->N, h->stream), "to_f64");
    CK(cudaMemcpyAsync(out_host, h->staging, h->N * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream),
       "cudaMemcpyAsync");
    return sync(h);
}

LBM_API int lbm_conservation(lbm_t *h, double *mass, double *mom3) {
    CHECK_H(h);
    if (!mass || !mom3) return fail(LBM_EINVAL, "NULL output");
    int st = ensure_buffers(h);
    if (st != LBM_OK) return st;
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    CK(lbm::conservation(h->q, h->dtype, h->buf[h->cur], h->N, h->cons_partial, h->cons_result,
                         h->stream),
       "conservation");
    double r[5];
    CK(cudaMemcpyAsync(r, h->cons_result, sizeof(r), cudaMemcpyDeviceToHost, h->stream),
       "cudaMemcpyAsync");
    st = sync(h);
    if (st != LBM_OK) return st;
    *mass = r[0];
    mom3[0] = r[1];
    mom3[1] = r[2];
    mom3[2] = r[3];
    if (r[4] != 0.0 || !isfinite(r[0]))
        return fail(LBM_ENUMERIC, "%.0f non-finite populations", r[4]);
    return LBM_OK;
}

LBM_API int lbm_kernel_time(lbm_t *h, double *ms_total, long long *launches) {
    CHECK_H(h);
    if (!ms_total || !launches) return fail(LBM_EINVAL, "NULL output");
    int st = sync(h);
    if (st != LBM_OK) return st;
    double total = 0.0;
    for (size_t k = 0; k + 1 < h->events_used; k += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->events[k], h->events[k + 1]), "cudaEventElapsedTime");
        total += ms;
    }
    *ms_total = total;
    *launches = (long long)(h->events_used / 2);
    h->events_used = 0;
    return LBM_OK;
}

LBM_API int lbm_set_sensor_average(lbm_t *h, int on) {
    CHECK_H(h);
    int st = ensure_scratch(h);
    if (st != LBM_OK) return st;
    if (on) {
        if (!h->tile_sum) {
            CK(lbm::dev_alloc((void **)&h->tile_sum, h->ntiles * sizeof(double)), "cudaMalloc(sum)");
            CK(lbm::dev_alloc((void **)&h->tile_avg, h->ntiles * sizeof(double)), "cudaMalloc(avg)");
        }
        CK(cudaMemsetAsync(h->tile_sum, 0, h->ntiles * sizeof(double), h->stream), "memset");
        h->avg_count = 0;
    }
    h->averaging = on != 0;
    return LBM_OK;
}

// Block maxima of the time-averaged tile maxima into h->blocks_f64.
static int average_blocks(lbm_t *h, int block, int *nb_out) {
    if (!h->tile_sum || h->avg_count == 0)
        return fail(LBM_ESTATE, "no sensor step averaged (lbm_set_sensor_average, then step)");
    int nbx, nby, nbz, m, mz;
    int st = check_block(h, block, &nbx, &nby, &nbz, &m, &mz);
    if (st != LBM_OK) return st;
    CK(lbm::scale_f64(h->tile_sum, 1.0 / (double)h->avg_count, h->tile_avg, h->ntiles, h->stream),
       "scale");
    CK(lbm::tiles_to_blocks(LBM_F64, h->tile_avg, h->ntx, h->nty, h->ntz, m, mz, h->blocks_f64,
                            nbx, nby, nbz, h->stream),
       "tiles_to_blocks");
    *nb_out = nbx * nby * nbz;
    return LBM_OK;
}

LBM_API int lbm_sensor_average(lbm_t *h, int block, double *out_host, long long *count) {
    CHECK_H(h);
    if (!out_host) return fail(LBM_EINVAL, "NULL output");
    int nb = 0;
    int st = average_blocks(h, block, &nb);
    if (st != LBM_OK) return st;
    CK(cudaMemcpyAsync(out_host, h->blocks_f64, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream),
       "cudaMemcpyAsync");
    if (count) *count = h->avg_count;
    return sync(h);
}

static int levels_common(lbm_t *h, int block, bool fit, double a, double b, int lmin, int lmax,
                         int source, int8_t *out_host) {
    CHECK_H(h);
    if (!out_host) return fail(LBM_EINVAL, "NULL output");
    if (lmin < -128 || lmax > 127 || lmin > lmax)
        return fail(LBM_EINVAL, "need -128 <= lmin <= lmax <= 127");
    if (!fit && (!(a > 0.0) || !isfinite(a) || !isfinite(b)))
        return fail(LBM_EINVAL, "scale a must be finite and > 0, offset b finite");
    if (source != LBM_SENSOR_LAST && source != LBM_SENSOR_AVERAGE)
        return fail(LBM_EINVAL, "unknown sensor source %d", source);
    int nb = 0, st;
    const void *maxima;
    int rtype;
    if (source == LBM_SENSOR_LAST) {
        st = reduce_blocks(h, block, &nb);
        maxima = h->blocks;
        rtype = h->rtype();
    } else {
        st = average_blocks(h, block, &nb);
        maxima = h->blocks_f64;
        rtype = LBM_F64;
    }
    if (st != LBM_OK) return st;
    if (fit)
        CK(lbm::levels_fit(rtype, maxima, nb, lmin, lmax, h->flags, h->stream), "levels_fit");
    else
        CK(lbm::levels_affine(rtype, maxima, nb, a, b, lmin, lmax, h->flags, h->stream), "levels");
    CK(cudaMemcpyAsync(out_host, h->flags, (size_t)nb, cudaMemcpyDeviceToHost, h->stream),
       "cudaMemcpyAsync");
    return sync(h);
}

LBM_API int lbm_levels(lbm_t *h, int block, double a, double b, int lmin, int lmax, int source,
                       int8_t *out_host) {
    return levels_common(h, block, false, a, b, lmin, lmax, source, out_host);
}

LBM_API int lbm_levels_fit(lbm_t *h, int block, int lmin, int lmax, int source, int8_t *out_host) {
    return levels_common(h, block, true, 0.0, 0.0, lmin, lmax, source, out_host);
}

LBM_API int lbm_blocks_step(lbm_t *h, const lbm_level_batch *batch) {
    CHECK_H(h);
    if (!batch || !batch->leaf) return fail(LBM_EINVAL, "NULL batch or leaf levels");
    if (h->q != LBM_D3Q19) return fail(LBM_ENOTSUP, "multi-level meshes are D3Q19 only");
    if (h->dtype != LBM_F32) return fail(LBM_ENOTSUP, "multi-level meshes use FP32 storage");
    if (batch->cycles < 0) return fail(LBM_EINVAL, "cycles must be >= 0");
    const int nb[3] = {batch->nbx, batch->nby, batch->nbz};
    if (batch->nbx < 1 || batch->nby < 1 || batch->nbz < 1 || batch->edge < 1)
        return fail(LBM_EINVAL, "bad block grid");
    if ((long long)batch->nbx * batch->edge != h->nx || (long long)batch->nby * batch->edge != h->ny ||
        (long long)batch->nbz * batch->edge != h->nz)
        return fail(LBM_EINVAL, "block grid x edge must equal the handle's lattice (%d x %d x %d)",
                    h->nx, h->ny, h->nz);
    CHECK_PENDING("lbm_blocks_step");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    if (h->mesh && !lbm::ml::same_layout(h->mesh, nb, batch->edge, batch->lmax, batch->leaf)) {
        CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        lbm::ml::destroy(h->mesh);
        h->mesh = nullptr;
    }
    // the error word of the persistent cycle's bounded waits
    int st = ensure_scratch(h);
    if (st != LBM_OK) return st;
    if (!h->mesh) {
        const double lid[3] = {h->lid_x, 0.0, h->lid_z};
        st = lbm::ml::build(&h->mesh, nb, batch->edge, batch->lmax, batch->leaf, h->tau, lid,
                            h->periodic, h->blocks_fusion, h->blocks_step_form - 1,
                            h->blocks_schedule, h->stream);
        if (st != LBM_OK) return st;
    }
    st = lbm::ml::run_cycles(h->mesh, batch->cycles, h->stream, h->graphs != 0, h->err_dev,
                             h->wait_ns, h->hold_copies);
    if (st != LBM_OK) return st;
    if (batch->block_max) {
        st = lbm::ml::block_max(h->mesh, batch->block_max, h->stream);  // synchronises
        if (st != LBM_OK) return st;
        if (*(volatile int *)h->err_host)
            return fail(LBM_ETIMEOUT, "a bounded wait of the persistent cycle ran out; the mesh "
                                      "state is not valid (rebuild it)");
    }
    return LBM_OK;
}

LBM_API int lbm_blocks_set_schedule(lbm_t *h, int mode) {
    CHECK_H(h);
    if (mode < LBM_SCHEDULE_AUTO || mode > LBM_SCHEDULE_PERSISTENT_LEAN)
        return fail(LBM_EINVAL, "schedule must be LBM_SCHEDULE_AUTO, _GRAPH, _PERSISTENT, "
                                "_PERSISTENT_BRICK or _PERSISTENT_LEAN");
    if (h->mesh) {  // applies to the next build
        CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        lbm::ml::destroy(h->mesh);
        h->mesh = nullptr;
    }
    h->blocks_schedule = mode;
    return LBM_OK;
}

LBM_API int lbm_blocks_cycle_form(lbm_t *h) {
    CHECK_H(h);
    if (!h->mesh) return fail(LBM_ESTATE, "no multi-level mesh (call lbm_blocks_step first)");
    return lbm::ml::uses_persistent(h->mesh) ? LBM_SCHEDULE_PERSISTENT : LBM_SCHEDULE_GRAPH;
}

LBM_API int lbm_blocks_get(lbm_t *h, int level, int block, double *out_host) {
    CHECK_H(h);
    if (!h->mesh) return fail(LBM_ESTATE, "no multi-level mesh (call lbm_blocks_step first)");
    if (!out_host) return fail(LBM_EINVAL, "NULL output");
    const int st = lbm::ml::get_block(h->mesh, level, block, out_host, h->stream);  // synchronises
    if (st == LBM_OK && h->err_host && *(volatile int *)h->err_host)
        return fail(LBM_ETIMEOUT, "a bounded wait of the persistent cycle ran out; the mesh state "
                                  "is not valid (rebuild it)");
    return st;
}

LBM_API int lbm_blocks_set(lbm_t *h, int level, int block, const double *in_host) {
    CHECK_H(h);
    if (!h->mesh) return fail(LBM_ESTATE, "no multi-level mesh (call lbm_blocks_step first)");
    if (!in_host) return fail(LBM_EINVAL, "NULL input");
    return lbm::ml::set_block(h->mesh, level, block, in_host, h->stream);
}

LBM_API int lbm_blocks_info(lbm_t *h, int level, int *n, double *tau, int *nblocks, int *threads,
                            int *cells_per_thread, long long *cell_updates_per_cycle) {
    CHECK_H(h);
    if (!h->mesh) return fail(LBM_ESTATE, "no multi-level mesh (call lbm_blocks_step first)");
    if (cell_updates_per_cycle) *cell_updates_per_cycle = lbm::ml::cells_per_cycle(h->mesh);
    return lbm::ml::info(h->mesh, level, n, tau, nblocks, threads, cells_per_thread);
}

LBM_API int lbm_block_features(lbm_t *h, int block, float *out_dev) {
    CHECK_H(h);
    if (block < 1 || !out_dev) return fail(LBM_EINVAL, "lbm_block_features: block >= 1, out_dev");
    int st = ensure_buffers(h);
    if (st != LBM_OK) return st;
    CK(lbm::block_features(h->q, h->dtype, h->buf[h->cur], h->nx, h->ny, h->nz, block, out_dev,
                           h->stream),
       "block features");
    return LBM_OK;
}

LBM_API int lbm_blocks_set_fusion(lbm_t *h, int mode) {
    CHECK_H(h);
    if (mode < LBM_FUSION_AUTO || mode > LBM_FUSION_BRICK)
        return fail(LBM_EINVAL, "fusion mode must be LBM_FUSION_AUTO, _SEPARATE, _FUSED or _BRICK");
    if (h->mesh) {  // applies to the next build
        CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        lbm::ml::destroy(h->mesh);
        h->mesh = nullptr;
    }
    h->blocks_fusion = mode;
    return LBM_OK;
}

LBM_API int lbm_blocks_set_step_form(lbm_t *h, int form) {
    CHECK_H(h);
    if (form < LBM_STEP_FORM_AUTO || form > LBM_STEP_FORM_PAIR)
        return fail(LBM_EINVAL, "step form must be one of LBM_STEP_FORM_*");
    if (h->mesh) {  // applies to the next build
        CK(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        lbm::ml::destroy(h->mesh);
        h->mesh = nullptr;
    }
    h->blocks_step_form = form;
    return LBM_OK;
}

LBM_API int lbm_blocks_schedule(lbm_t *h, int level, int *form, int *planes, int *fused) {
    CHECK_H(h);
    if (!h->mesh) return fail(LBM_ESTATE, "no multi-level mesh (call lbm_blocks_step first)");
    return lbm::ml::schedule(h->mesh, level, form, planes, fused);
}

LBM_API int lbm_regrid(lbm_t *h, const double *field_dev, const lbm_regrid_params *p,
                       lbm_box *boxes, int max_boxes, int *nboxes, long long *ntagged,
                       uint8_t *tags_out) {
    CHECK_H(h);
    if (!p || !nboxes) return fail(LBM_EINVAL, "lbm_regrid: NULL params or nboxes");
    if (max_boxes < 0 || (max_boxes > 0 && !boxes))
        return fail(LBM_EINVAL, "lbm_regrid: boxes is NULL or max_boxes < 0");
    if (p->coarsen < 1 || p->buffer < 0 || p->nest < 0 || p->min_width < 1 ||
        !(p->efficiency >= 0.0 && p->efficiency <= 1.0))
        return fail(LBM_EINVAL,
                    "lbm_regrid: need coarsen >= 1, buffer >= 0, nest >= 0, min_width >= 1 and "
                    "efficiency in [0, 1]");
    const void *field = field_dev;
    int ftype = LBM_F64;
    if (!field) {
        if (!h->have_kfield || !h->kfield)
            return fail(LBM_ESTATE,
                        "no per-cell sensor recorded (lbm_set_sensor_field before stepping)");
        field = h->kfield;
        ftype = h->rtype();
    }
    lbm::rg::Params rp;
    rp.coarsen = p->coarsen;
    rp.threshold = p->threshold;
    rp.buffer = p->buffer;
    rp.nest = p->nest;
    rp.efficiency = p->efficiency;
    rp.min_width = p->min_width;
    std::vector<int> out;
    long long nt = 0;
    int st = lbm::rg::regrid(field, ftype, h->nx, h->ny, h->nz, h->periodic, rp, p->allowed, &out,
                             &nt, tags_out, h->stream);
    if (st != LBM_OK) return st;
    const int n = (int)(out.size() / 6);
    *nboxes = n;
    if (ntagged) *ntagged = nt;
    if (n > max_boxes)
        return fail(LBM_EINVAL, "lbm_regrid: %d boxes, more than max_boxes = %d", n, max_boxes);
    for (int k = 0; k < n; ++k)
        for (int a = 0; a < 3; ++a) {
            boxes[k].lo[a] = out[6 * k + a];
            boxes[k].hi[a] = out[6 * k + 3 + a];
        }
    return LBM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------ failure injection
LBM_API int lbm_debug_fail_alloc(int after) {
    g_err = LBM_OK;
    lbm::g_fail_alloc_after.store(after < 0 ? -1 : (long long)after);
    return LBM_OK;
}

LBM_API int lbm_debug_set_wait_limit(lbm_t *h, long long ns) {
    CHECK_H(h);
    if (ns < 0) return fail(LBM_EINVAL, "wait limit must be >= 0 (0: the default)");
    h->wait_ns = (unsigned long long)ns;
    drop_graphs(h);  // captured launches carry the old limit
    return LBM_OK;
}

LBM_API int lbm_debug_hold_copies(lbm_t *h, int on) {
    CHECK_H(h);
    h->hold_copies = on ? 1 : 0;
    drop_graphs(h);
    return LBM_OK;
}

// ------------------------------------------------------------------------------ checkpoints
namespace {

struct CkptHeader {
    char magic[8];          // "LBMCKPT\0"
    int32_t version;        // 1
    int32_t lattice;        // LBM_D2Q9 / LBM_D3Q19
    int32_t nx, ny, nz;
    int32_t dtype;          // storage type of the payload
    int32_t periodic;
    int32_t reserved;
    double tau, lid_x, lid_z;
    int64_t step;           // steps taken since the last reset
    uint64_t payload_bytes; // q * N * element size, the layout of lbm_get_raw
    uint64_t checksum;      // FNV-1a (64-bit) of the payload
};
static_assert(sizeof(CkptHeader) == 88, "checkpoint header layout");
const char kCkptMagic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '\0'};

uint64_t fnv1a(const unsigned char *p, size_t n, uint64_t h = 1469598103934665603ull) {
    for (size_t k = 0; k < n; ++k) {
        h ^= p[k];
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace

LBM_API int lbm_checkpoint_save(lbm_t *h, const char *path) {
    CHECK_H(h);
    if (!path) return fail(LBM_EINVAL, "NULL path");
    const size_t bytes = h->pop_bytes();
    std::vector<unsigned char> buf;
    try {
        buf.resize(bytes);
    } catch (...) {
        return fail(LBM_ENOMEM, "host buffer of %zu bytes for the checkpoint", bytes);
    }
    int st = lbm_get_raw(h, buf.data(), bytes);
    if (st != LBM_OK) return st;
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, kCkptMagic, 8);
    hd.version = 1;
    hd.lattice = h->q;
    hd.nx = h->nx;
    hd.ny = h->ny;
    hd.nz = h->nz;
    hd.dtype = h->dtype;
    hd.periodic = h->periodic;
    hd.tau = h->tau;
    hd.lid_x = h->lid_x;
    hd.lid_z = h->lid_z;
    hd.step = h->t;
    hd.payload_bytes = bytes;
    hd.checksum = fnv1a(buf.data(), bytes);
    FILE *f = fopen(path, "wb");
    if (!f) return fail(LBM_EIO, "cannot open %s for writing", path);
    const bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 && fwrite(buf.data(), 1, bytes, f) == bytes;
    const bool closed = fclose(f) == 0;
    if (!ok || !closed) return fail(LBM_EIO, "writing %s failed", path);
    return LBM_OK;
}

LBM_API int lbm_checkpoint_load(lbm_t *h, const char *path) {
    CHECK_H(h);
    if (!path) return fail(LBM_EINVAL, "NULL path");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(LBM_EIO, "cannot open %s", path);
    CkptHeader hd;
    if (fread(&hd, sizeof(hd), 1, f) != 1 || memcmp(hd.magic, kCkptMagic, 8) != 0 ||
        hd.version != 1) {
        fclose(f);
        return fail(LBM_EIO, "%s is not a checkpoint of this library (bad header)", path);
    }
    if (hd.lattice != h->q || hd.nx != h->nx || hd.ny != h->ny || hd.nz != h->nz ||
        hd.dtype != h->dtype || hd.payload_bytes != h->pop_bytes()) {
        fclose(f);
        return fail(LBM_EINVAL, "checkpoint %s holds a %d-velocity %d x %d x %d lattice of storage "
                                "type %d; the handle is %d-velocity %d x %d x %d of type %d",
                    path, hd.lattice, hd.nx, hd.ny, hd.nz, hd.dtype, h->q, h->nx, h->ny, h->nz,
                    h->dtype);
    }
    if (!(hd.tau > 0.5) || !isfinite(hd.tau) || !isfinite(hd.lid_x) || !isfinite(hd.lid_z) ||
        (hd.periodic & ~7) || hd.step < 0) {
        fclose(f);
        return fail(LBM_EIO, "checkpoint %s has invalid parameters", path);
    }
    std::vector<unsigned char> buf;
    try {
        buf.resize(hd.payload_bytes);
    } catch (...) {
        fclose(f);
        return fail(LBM_ENOMEM, "host buffer of %llu bytes for the checkpoint",
                    (unsigned long long)hd.payload_bytes);
    }
    const bool ok = fread(buf.data(), 1, buf.size(), f) == buf.size();
    fclose(f);
    if (!ok) return fail(LBM_EIO, "checkpoint %s is truncated", path);
    if (fnv1a(buf.data(), buf.size()) != hd.checksum)
        return fail(LBM_EIO, "checkpoint %s fails its checksum", path);
    // parameters first (they validate), then the state; the step counter last
    int st = lbm_set_tau(h, hd.tau);
    if (st == LBM_OK) st = lbm_set_lid(h, hd.lid_x, hd.lid_z);
    if (st == LBM_OK) st = lbm_set_periodic(h, hd.periodic);
    if (st == LBM_OK) st = lbm_set_raw(h, buf.data(), buf.size());
    if (st != LBM_OK) return st;
    h->t = hd.step;
    return LBM_OK;
}
