// Multi-level block-structured lattice Boltzmann step (D3Q19, FP32) on the GPU.
//
// The paper (Sec. 2.1, Sec. 5.2) drives cell-centred block-structured refinement with ratio 2
// under acoustic scaling: levels are sub-cycled and coupled by linear temporal and second-order
// spatial interpolation with the non-equilibrium part of the populations rescaled between levels.
// This file implements the same reading as the FP64 checker of this repository:
//
//   * physical blocks of edge E finest cells carry a leaf level 0..lmax; level l exists on every
//     block whose leaf level is >= l, with n_l = E / 2^(lmax - l) cells per block edge; touching
//     blocks differ by at most one level;
//   * acoustic scaling: tau_l = 3 nu_lmax / 2^(lmax - l) + 1/2, level l takes 2^l steps per
//     level-0 step (a cycle);
//   * a level step is the fused pull step of every block of the level (moving-wall bounce-back at
//     the domain walls, moments, equilibrium, Knudsen sensor, BGK collision) reading a one-cell
//     ghost layer;
//   * a population pulled from another block of the same level is read from that block directly
//     (a 27-entry neighbour table per block); one pulled from where the level does not exist is
//     read from the block's own ghost layer, filled by trilinear (3/4, 1/4 per axis; 5/4, -1/4
//     extrapolation at a wall) interpolation of the coarser level, linear in time between its
//     states before and after its step, with f^neq rescaled by (tau_f - 1) / (2 (tau_c - 1));
//   * after the two sub-steps of level l + 1, the level-l cells under it become the average of
//     their 8 fine cells with f^neq rescaled by 2 (tau_c - 1) / (tau_f - 1).
//
// Device layout of a level: one buffer of nslot blocks x 19 populations x (n + 2)^3 ghosted cells
// (block-major, then population, then z, y, x), two buffers (ping-pong); only the ghost cells that
// face a coarser neighbour are used.  The interpolation and restriction work is precomputed on the
// host as task lists (flat element offsets; for the interpolation, chunks of ghost cells with the
// coarse cells their stencils touch, which a CTA stages in shared memory).  A cycle is captured
// once per level-0 buffer parity as a CUDA graph and replayed.  The launch shape of each level's step kernel (threads per CTA and cells per
// thread) is chosen by timing the candidates once when the mesh is built.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <unordered_set>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"
#include "lbm_step_pair.cuh"

namespace lbm {
namespace ml {

constexpr int Q = 19;
constexpr int MAXL = 3;

// neighbour table entries besides a slot number
constexpr int NB_GHOST = -1;  // the neighbouring block exists only on a coarser level
constexpr int NB_WALL = -2;   // the neighbouring block lies outside the (non-periodic) domain
constexpr int NB_TOP = 16;    // index of the (0, +1, 0) neighbour: (dx+1) + 3 (dy+1) + 9 (dz+1)
// Block layout of one population: (n + 2) planes z = -1..n of (n + 2) rows y = -1..n of n cells
// x = 0..n-1 (interior rows contiguous, no padding), then the two x-ghost columns x = -1 and x = n
// as (n + 2) x (n + 2) arrays over (z, y); G = that size rounded up to 32 floats, so every block and
// population starts on a 128-byte line.  Whole planes are contiguous, so a level of 8^3 or 16^3
// blocks streams without the partly used lines a padded row pitch leaves (ncu: 3x and 2x DRAM
// over-fetch on those levels with padded 128-byte-aligned rows).
__host__ __device__ __forceinline__ int side_base(int n, int side) {  // side 0: x = -1, 1: x = n
    return (n + 2) * (n + 2) * (n + side);
}
// offset of cell (x, y, z), -1 <= x, y, z <= n, within one population of a block
__host__ __device__ __forceinline__ int cell_index(int n, int x, int y, int z) {
    if (x < 0) return side_base(n, 0) + (z + 1) * (n + 2) + (y + 1);
    if (x >= n) return side_base(n, 1) + (z + 1) * (n + 2) + (y + 1);
    return ((z + 1) * (n + 2) + (y + 1)) * n + x;
}

// Brick forms of the fused step + restriction: the 19 sums in registers (BRICK_REG) or in a
// shared-memory column per thread (BRICK_SMEM)
constexpr int BRICK_REG = 0, BRICK_SMEM = 1;

// Forms of a level's step kernel (also the values lbm_blocks_schedule reports):
constexpr int FORM_FLAT = 0;    // k_step: one cell per thread, x-fastest
constexpr int FORM_TILED = 1;   // k_step_tiled: bricks of whole rows walking z planes
constexpr int FORM_SELECT = 2;  // k_step<XSEL>: flat, address-select gather for y/z-inner rows
constexpr int FORM_PAIR = 3;    // k_step_pair: two cells per thread, packed FP32 arithmetic

// Coarse -> fine ghost fill, in chunks.  The ghost cells of a level that face a coarser level are
// grouped (host side) into chunks of at most IC_TASKS cells whose trilinear stencils together touch
// at most IC_WIN coarse cells, the chunk's window.  A CTA copies the window's 19 populations into
// shared memory in one round of independent loads, then each thread fills one ghost cell from it:
// one round of memory latency per chunk instead of one per population and thread.
constexpr int IC_TASKS = 128;
constexpr int IC_WIN = 320;
struct InterpChunk {
    int task0, ntask;  // ghost cells [task0, task0 + ntask) of the level's task list
    int win0, nwin;    // coarse cells [win0, win0 + nwin) of the level's window list
};
// A ghost cell's task is two words, read with vector loads: its flat offset (population 0) in the
// fine level's buffer, and its stencil's 8 coarse cells as 16-bit indices into the chunk's window
// (cell k = x bit 0, y bit 1, z bit 2 of k; low half of a word first), whose bit 15 in the entries
// of cells 0, 1, 2 says that axis 0, 1, 2 extrapolates (weights 5/4, -1/4 instead of 3/4, 1/4).
constexpr unsigned IC_EXTRAP = 0x8000u;
struct RestrictTask {
    int dst;   // coarse cell, population 0
    int fine;  // fine cell (2x, 2y, 2z), population 0
};

struct Level {
    int n = 0, G = 0;      // cells per block edge, values per population per block (ghosted)
    int P = 0, plane = 0;  // row pitch (n) and plane size n (n + 2) of the interior rows
    double tau = 1.0;
    int nslot = 0;
    std::vector<int> slot;  // physical block -> slot or -1
    int cells[3] = {0, 0, 0};
    float *buf[2] = {nullptr, nullptr};
    int cur = 0;
    int *nbr = nullptr;  // device: 27 entries per slot (slot, NB_GHOST or NB_WALL)
    InterpChunk *ichunks = nullptr;  // ghost fill from level - 1: chunks, tasks, window cells
    int *idst = nullptr;
    uint4 *isrc = nullptr;
    int *iwin = nullptr;
    int ninterp = 0, nichunk = 0;
    RestrictTask *restricts = nullptr;  // level cells under level + 1
    int nrestrict = 0;
    float *kmax = nullptr;  // device: per-slot sensor max of the level's last step (int bits)
    // step launch shape (autotuned): the form (FORM_*), `threads` per CTA and `cpt` cells (pairs
    // for FORM_PAIR) per thread of the flat kernels, `zc` planes of the tiled one
    int form = 0;
    int threads = 256, cpt = 1, zc = 1;
    // finest level only: its second sub-step also restricts onto the next coarser level (tiled
    // brick kernel walking fuse_zc planes); the coarser level then skips k_restrict
    bool fuse = false;
    int fuse_zc = 2;
    // or the two-cell brick form (k_step_pair_restrict) with its own launch shape
    bool fuse_brick = false;
    int brick_threads = 256, brick_cpt = 1;
    int brick_mode = 0;  // BRICK_*
    int *cslot = nullptr;  // device: per slot, the slot of the same block one level coarser
};

struct Mesh {
    int nb[3] = {0, 0, 0}, edge = 0, lmax = 0, nblk = 0;
    std::vector<int8_t> leaf;
    double lid[3] = {0, 0, 0};
    int periodic = 0;
    Level lv[MAXL];
    int fusion = 0;  // 0 timed, 1 separate restriction, 2 tiled fused form, 3 brick fused form
    int step_form = -1;  // FORM_* forced on every level where it applies, -1: autotuned
    // a cycle runs level l's work on stream ss[l] (level 0 on the caller's stream, the finer
    // levels on the mesh's own streams), ordered by events: ev_pre[l] before level l's step,
    // ev_post[l] after it, ev_done[l] after the restriction onto it
    cudaStream_t lst[MAXL] = {};
    cudaEvent_t ev_pre[MAXL] = {}, ev_post[MAXL] = {}, ev_done[MAXL] = {}, ev_join[MAXL] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // by level-0 buffer parity
    long long cycles = 0;
    // persistent form of a cycle (one k_cycle launch): phase table and dependency lists per
    // level-0 buffer parity, the counters, the launch width, and whether cycles use it
    struct Plan {
        void *phases = nullptr;  // device PPhase[nph]
        int *deps = nullptr;
        int nph = 0, ntask = 0;
    } plan[2];
    int *pctr = nullptr;  // device: 2 + phases counters
    int pctr_len = 0;
    int pk_grid = 0;
    bool persistent = false;
    // lean persistent form: no brick phase (the finest level's second sub-step is a plain step and
    // the restriction a phase of its own), so that the cycle kernel fits 3 CTAs per SM instead of 2
    bool pk_lean = false;
    int schedule = 0;  // LBM_SCHEDULE_* of the build
    // error word and wait settings the persistent graphs were captured with
    int *err = nullptr;
    unsigned long long wait_ns = 0;
    int hold = 0;
};

// ---------------------------------------------------------------------------------- kernels
__device__ __forceinline__ void moments19(const float *f, float &rho, float &ux, float &uy,
                                          float &uz) {
    float r = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        r += f[i];
        jx += (float)D3Q19::cx(i) * f[i];
        jy += (float)D3Q19::cy(i) * f[i];
        jz += (float)D3Q19::cz(i) * f[i];
    }
    rho = r;
    const float inv = 1.f / r;
    ux = jx * inv;
    uy = jy * inv;
    uz = jz * inv;
}

__device__ __forceinline__ float feq19(int i, float rho, float ux, float uy, float uz) {
    const float cu = (float)D3Q19::cx(i) * ux + (float)D3Q19::cy(i) * uy + (float)D3Q19::cz(i) * uz;
    const float uu = ux * ux + uy * uy + uz * uz;
    return weight<D3Q19, float>(i) * rho * (1.f + 3.f * cu + 4.5f * cu * cu - 1.5f * uu);
}

// How the level kernels read populations.  LdPlain leaves the load form to the compiler: in the
// graph form of a cycle each launch only reads buffers that no CTA of the same launch writes.  LdL2
// reads through L2 (ld.global.cg), the point of coherence: the persistent cycle kernel reads
// buffers that other CTAs of the same launch wrote, which neither the read-only path nor an L1
// line filled earlier in the launch may serve.
struct LdPlain {
    __device__ __forceinline__ float operator()(const float *p) const { return *p; }
    __device__ __forceinline__ float2 pair(const float *p) const {
        return *reinterpret_cast<const float2 *>(p);
    }
};
struct LdL2 {
    __device__ __forceinline__ float operator()(const float *p) const { return __ldcg(p); }
    __device__ __forceinline__ float2 pair(const float *p) const {
        return __ldcg(reinterpret_cast<const float2 *>(p));
    }
};

// Linear blend in time of a coarse population before (p) and after (c) its step, rounded the same
// way on every path that fills ghosts.
__device__ __forceinline__ float time_blend(float p, float c, float theta) {
    return __fmaf_rn(theta, c, __fmul_rn(1.f - theta, p));
}

__device__ __forceinline__ void cp_async4(float *sdst, const float *gsrc) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Ghost fills of a chunk: FILL_PREV the state before the coarse step (theta 0) into fine0;
// FILL_BLEND the blend at theta into fine1; FILL_BOTH both, from one copy of the window (the graph
// form fills the ghosts of both fine sub-steps once the coarse step is done).
constexpr int FILL_PREV = 0, FILL_BLEND = 1, FILL_BOTH = 2;

// The trilinear weights of a task from its extrapolation bits, as products in axis order.
__device__ __forceinline__ void stencil(const uint4 sv, int src[8], float w[8]) {
    const unsigned h[8] = {sv.x & 0xffffu, sv.x >> 16, sv.y & 0xffffu, sv.y >> 16,
                           sv.z & 0xffffu, sv.z >> 16, sv.w & 0xffffu, sv.w >> 16};
    float f0[3], f1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const bool ex = h[a] & IC_EXTRAP;
        f0[a] = ex ? 1.25f : 0.75f;
        f1[a] = ex ? -0.25f : 0.25f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        src[k] = (int)(h[k] & (IC_EXTRAP - 1u));
        float wt = 1.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) wt *= ((k >> a) & 1) ? f1[a] : f0[a];
        w[k] = wt;
    }
}

// Interpolate one ghost cell from a staged window (sw: population i at sw[i * IC_WIN + cell]),
// rescale the non-equilibrium part and store its 19 populations at fine + dst.
__device__ __forceinline__ void fill_ghost(const float *sw, const int src[8], const float w[8],
                                           float *fine, int dst, int Gf, float scale) {
    float acc[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float a = 0.f;
#pragma unroll
        for (int s = 0; s < 8; ++s) a = __fmaf_rn(w[s], sw[i * IC_WIN + src[s]], a);
        acc[i] = a;
    }
    float rho, ux, uy, uz;
    moments19(acc, rho, ux, uy, uz);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float fe = feq19(i, rho, ux, uy, uz);
        fine[dst + (size_t)i * Gf] = fe + scale * (acc[i] - fe);
    }
}

// One chunk of the coarse -> fine ghost fill: interpolate in space (the chunk's window staged in
// shared memory) and linearly in time, rescale the non-equilibrium part.  FILL (above) says which
// states are read and written.  ASYNC: the window is copied with cp.async (buffers no CTA of the
// launch writes; sw2 receives the second state); otherwise by loads through L2 (the persistent
// cycle, whose other CTAs wrote the coarse level earlier in the launch; FILL_PREV or FILL_BLEND
// only).  NTH threads, all of which must call this; with FILL_BOTH a thread fills one of the two
// states of a ghost cell.
template <int FILL, bool ASYNC, int NTH>
__device__ __forceinline__ void interp_chunk(const InterpChunk &c, const int *__restrict__ idst,
                                             const uint4 *__restrict__ isrc,
                                             const int *__restrict__ win, float *fine0,
                                             float *fine1, int Gf, const float *cprev,
                                             const float *ccur, int Gc, float theta, float scale,
                                             float *sw, float *sw2) {
    static_assert(ASYNC || FILL != FILL_BOTH, "the L2 path fills one state");
    constexpr int R = (IC_WIN + NTH - 1) / NTH;
    const int tid = threadIdx.x, nw = c.nwin;
    int off[R];  // the window cells this thread copies, loaded before any copy is issued
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = tid + r * NTH;
        off[r] = j < nw ? win[c.win0 + j] : 0;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = tid + r * NTH;
        if (j >= nw) break;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const size_t e = (size_t)off[r] + (size_t)i * Gc;
            if (ASYNC) {
                cp_async4(sw + i * IC_WIN + j, cprev + e);
                if (FILL != FILL_PREV) cp_async4(sw2 + i * IC_WIN + j, ccur + e);
            } else {
                float v = __ldcg(cprev + e);
                if (FILL == FILL_BLEND) v = time_blend(v, __ldcg(ccur + e), theta);
                sw[i * IC_WIN + j] = v;
            }
        }
    }
    if (ASYNC) {
        cp_async_wait_all();  // this thread's copies; it blends the same elements it copied
        if (FILL != FILL_PREV)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int j = tid + r * NTH;
                if (j >= nw) break;
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    sw2[i * IC_WIN + j] =
                        time_blend(sw[i * IC_WIN + j], sw2[i * IC_WIN + j], theta);
            }
    }
    __syncthreads();
    constexpr int NF = FILL == FILL_BOTH ? 2 : 1;
    for (int e = tid; e < NF * c.ntask; e += NTH) {
        const bool second = NF == 2 && e >= c.ntask;
        const int k = second ? e - c.ntask : e;
        int src[8];
        float w[8];
        stencil(isrc[c.task0 + k], src, w);
        const int dst = idst[c.task0 + k];
        if (FILL == FILL_PREV)
            fill_ghost(sw, src, w, fine0, dst, Gf, scale);
        else if (FILL == FILL_BLEND)
            fill_ghost(ASYNC ? sw2 : sw, src, w, fine1, dst, Gf, scale);
        else
            fill_ghost(second ? sw2 : sw, src, w, second ? fine1 : fine0, dst, Gf, scale);
    }
}

// one CTA per chunk, a thread per ghost cell and state; dynamic shared memory: the window, twice
// unless FILL_PREV
template <int FILL>
__global__ void __launch_bounds__(FILL == FILL_BOTH ? 2 * IC_TASKS : IC_TASKS)
    k_interp(const InterpChunk *__restrict__ ch, const int *__restrict__ idst,
             const uint4 *__restrict__ isrc, const int *__restrict__ win, float *fine0,
             float *fine1, int Gf, const float *cprev, const float *ccur, int Gc, float theta,
             float scale) {
    extern __shared__ float sw[];
    interp_chunk<FILL, true, FILL == FILL_BOTH ? 2 * IC_TASKS : IC_TASKS>(
        ch[blockIdx.x], idst, isrc, win, fine0, fine1, Gf, cprev, ccur, Gc, theta, scale, sw,
        sw + Q * IC_WIN);
}
constexpr int interp_threads(int fill) { return fill == FILL_BOTH ? 2 * IC_TASKS : IC_TASKS; }
constexpr size_t interp_smem(int fill) {
    return (fill == FILL_PREV ? 1 : 2) * sizeof(float) * Q * IC_WIN;
}

// level cells under the finer level: average of 8 fine cells, non-equilibrium part rescaled
template <class LD = LdPlain>
__device__ __forceinline__ void restrict_one(const RestrictTask &r, float *coarse, int Gc,
                                             const float *fine, int pf, int planef, int Gf,
                                             float scale) {
    const LD ld;
    const int row = pf, plane = planef;
    float avg[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float *f = fine + r.fine + i * Gf;
        avg[i] = 0.125f * (ld(f) + ld(f + 1) + ld(f + row) + ld(f + row + 1) + ld(f + plane) +
                           ld(f + plane + 1) + ld(f + plane + row) + ld(f + plane + row + 1));
    }
    float rho, ux, uy, uz;
    moments19(avg, rho, ux, uy, uz);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float fe = feq19(i, rho, ux, uy, uz);
        coarse[r.dst + i * Gc] = fe + scale * (avg[i] - fe);
    }
}

__global__ void k_restrict(const RestrictTask *t, int n, float *coarse, int Gc, const float *fine,
                           int pf, int planef, int Gf, float scale) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    restrict_one(t[k], coarse, Gc, fine, pf, planef, Gf, scale);
}

struct StepArgs {
    int n, G, P, plane;  // cells per edge, values per population, row pitch, plane size
    float omega;
    float lid_x, lid_z;
};

// One cell of a level step (pull, bounce-back at walls, moments, equilibrium, sensor, collision);
// returns its sensor value.  src / dst: the block's slot in the two buffers; also(i, v) sees every
// stored post-collision population.
struct NoVisit {
    __device__ __forceinline__ void operator()(int, float) const {}
};
// XSEL: cells whose y and z neighbours lie inside the block (whole rows for 32-cell rows, so
// the branch is warp-uniform) take a gather where a pull along x that leaves the block selects its
// address (x-neighbour block, interpolated x-ghost column or the wall's bounce-back) instead of
// branching on it, so the two face lanes of a row do not split the warp.
template <int NT, bool XSEL = false, class LD = LdPlain, class Also = NoVisit>
__device__ __forceinline__ float step_cell(const float *__restrict__ in, const float *src,
                                           float *dst, const int *snb, bool top,
                                           const StepArgs &a, int x, int y, int z,
                                           Also &&also = NoVisit()) {
    using L = D3Q19;
    const int n = NT ? NT : a.n;
    const int G = a.G, row = n, plane = n * (n + 2);
    const int g = (z + 1) * plane + (y + 1) * row + x;
    // a pull along +c leaves the block at the low face, along -c at the high face
    const bool xl = x == 0, xh = x == n - 1, yl = y == 0, yh = y == n - 1;
    const bool zl = z == 0, zh = z == n - 1;
    float df[Q];
    if (XSEL && !(yl | yh | zl | zh)) {
        const int nbm = snb[12], nbp = snb[14];  // the x - 1 and x + 1 neighbours
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
            const int off = cz * plane + cy * row + cx;
            const float *p = src + (size_t)i * G + (g - off);
            if (cx != 0) {
                const int nb = cx == 1 ? nbm : nbp;
                const float *q =
                    nb >= 0 ? in + (size_t)nb * Q * G + (size_t)i * G + (g - off + cx * n)
                    : nb == NB_GHOST
                        ? src + (size_t)i * G +
                              (side_base(n, cx < 0) + (z - cz + 1) * (n + 2) + (y - cy + 1))
                        : src + (size_t)L::opp(i) * G + g;
                p = (cx == 1 ? xl : xh) ? q : p;
            }
            df[i] = LD()(p) - weight<L, float>(i);
        }
        return relax_cell<L, 1, 1>(df, a.omega, [&](int i, float d) {
            const float v = d + weight<L, float>(i);
            dst[(size_t)i * G + g] = v;
            also(i, v);
        });
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const int dx = (cx == 1 && xl) ? -1 : ((cx == -1 && xh) ? 1 : 0);
        const int dy = (cy == 1 && yl) ? -1 : ((cy == -1 && yh) ? 1 : 0);
        const int dz = (cz == 1 && zl) ? -1 : ((cz == -1 && zh) ? 1 : 0);
        float v;
        if ((dx | dy | dz) == 0) {
            v = LD()(src + (i * G + g - (cz * plane + cy * row + cx)));
        } else {
            const int nb = snb[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)];
            if (nb >= 0) {
                v = LD()(in + ((size_t)nb * Q * G + i * G + (z - cz - dz * n + 1) * plane +
                               (y - cy - dy * n + 1) * row + (x - cx - dx * n)));
            } else if (nb == NB_GHOST) {
                // interpolated ghost: an x-ghost column, or a ghost row / plane of the block
                v = LD()(src + (i * G + (dx != 0 ? side_base(n, dx > 0) + (z - cz + 1) * (n + 2) +
                                                       (y - cy + 1)
                                                 : g - (cz * plane + cy * row + cx))));
            } else {
                v = LD()(src + (L::opp(i) * G + g));
                if (dy == 1 && top)
                    v += 6.f * weight<L, float>(i) * ((float)cx * a.lid_x + (float)cz * a.lid_z);
            }
        }
        df[i] = v - weight<L, float>(i);
    }
    return relax_cell<L, 1, 1>(df, a.omega, [&](int i, float d) {
        const float v = d + weight<L, float>(i);
        dst[(size_t)i * G + g] = v;
        also(i, v);
    });
}

// Row r (0 <= r < n^2) of a block in the order interior rows first, then face rows: rows with
// 1 <= y, z <= n - 2 (y fastest), then the planes z = 0 and z = n - 1, then the rows y = 0 and
// y = n - 1 of the planes in between.
template <int n>
__device__ __forceinline__ void face_row_order(int r, int &y, int &z) {
    constexpr int ni = (n - 2) * (n - 2);
    if (r < ni) {
        y = 1 + r % (n - 2);
        z = 1 + r / (n - 2);
        return;
    }
    const int f = r - ni;
    if (f < 2 * n) {
        z = f < n ? 0 : n - 1;
        y = f < n ? f : f - n;
        return;
    }
    const int k = f - 2 * n;
    z = 1 + (k >> 1);
    y = (k & 1) ? n - 1 : 0;
}

// warp max of the sensor bits, one atomic per warp (every lane of the warp must call this)
__device__ __forceinline__ void block_max_flush(int km, float *kmax, int slot, int lane) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) km = max(km, __shfl_xor_sync(~0u, km, off));
    if (lane == 0) atomicMax(reinterpret_cast<int *>(kmax) + slot, km);
}

// Flat mapping: grid (slot, chunk), cells of a block in x-fastest order, each thread `cpt` cells;
// with XSEL the rows come interior rows first (face_row_order).  NT is the block edge when it is
// one of the compiled sizes (shifts instead of divisions), 0 otherwise (never with XSEL).
template <int NT, bool XSEL = false>
__global__ void k_step(const float *__restrict__ in, float *__restrict__ out,
                       const int *__restrict__ nbr, const StepArgs a, int cpt, float *kmax) {
    __shared__ int snb[27];
    const int slot = blockIdx.x;
    if (threadIdx.x < 27) snb[threadIdx.x] = nbr[27 * slot + threadIdx.x];
    __syncthreads();
    const int n = NT ? NT : a.n;
    const int ncell = n * n * n;
    const bool top = snb[NB_TOP] == NB_WALL;  // the block touches the lid wall
    const float *src = in + (size_t)slot * Q * a.G;
    float *dst = out + (size_t)slot * Q * a.G;
    int km = 0;
    for (int r = 0; r < cpt; ++r) {
        const int c = (blockIdx.y * cpt + r) * blockDim.x + threadIdx.x;
        if (c >= ncell) break;
        int y, z;
        if (XSEL) {  // interior rows first, so that a warp's rows take one gather only
            face_row_order<(NT ? NT : 16)>(c / n, y, z);
        } else {
            y = (c / n) % n;
            z = c / (n * n);
        }
        const float K = step_cell<NT, XSEL>(in, src, dst, snb, top, a, c % n, y, z);
        km = max(km, __float_as_int(K));
    }
    block_max_flush(km, kmax, slot, threadIdx.x & 31);
}

// Tiled mapping for NT = 8, 16, 32, 64: a CTA of 256 threads is a TX x TY x TZ brick of cells
// (whole rows in x) that walks through `zc` planes of the block, so the planes pulled from along z
// were read by the same CTA just before (L1 reuse, as in the uniform step).
template <int NT>
struct Tile {
    static constexpr int TX = NT;
    static constexpr int TY = NT >= 16 ? 256 / NT : NT;
    static constexpr int TZ = 256 / (TX * TY);
};

template <int NT>
__global__ void __launch_bounds__(256, 4) k_step_tiled(const float *__restrict__ in,
                                                    float *__restrict__ out,
                                                    const int *__restrict__ nbr, const StepArgs a,
                                                    int zc, float *kmax) {
    using T = Tile<NT>;
    __shared__ int snb[27];
    const int slot = blockIdx.x;
    const int tid = (threadIdx.z * T::TY + threadIdx.y) * T::TX + threadIdx.x;
    if (tid < 27) snb[tid] = nbr[27 * slot + tid];
    __syncthreads();
    const bool top = snb[NB_TOP] == NB_WALL;
    const float *src = in + (size_t)slot * Q * a.G;
    float *dst = out + (size_t)slot * Q * a.G;
    constexpr int ytiles = NT / T::TY;
    const int y = (blockIdx.y % ytiles) * T::TY + threadIdx.y;
    const int z0 = (blockIdx.y / ytiles) * zc;
    int km = 0;
    for (int zz = threadIdx.z; zz < zc; zz += T::TZ) {
        const float K = step_cell<NT>(in, src, dst, snb, top, a, threadIdx.x, y, z0 + zz);
        km = max(km, __float_as_int(K));
    }
    block_max_flush(km, kmax, slot, tid & 31);
}

// Two x-adjacent cells per thread (x0 even) for NT = 8, 16, 32, 64: the moments, equilibrium,
// sensor and collision of both cells in packed FP32 pairs (relax_pair of the uniform two-cell
// kernel), 8-byte loads and stores for the directions with c_x = 0.  Rows inside the block in y
// and z take the address-select gather (a face lane pulling along x reads the x-neighbour block,
// the interpolated x-ghost column or its own opposite population at a wall); rows on a y or z
// face take the per-cell gather of step_cell.  Flat mapping: grid (slot, chunk), `cpt` pairs per
// thread, x fastest; the rows of a block are ordered interior rows first ((n - 2)^2 rows, y
// fastest), then the rows on a y or z face, so that a warp holds rows of one kind only (except one
// warp for n = 8) and does not run both the select gather and the per-cell one.
// One row pair-step of k_step_pair: cells (x0, y, z) and (x0 + 1, y, z) of the block, their
// post-collision populations stored and shown to also(i, float2) (the per-cell gather of a face
// row shows each cell's value as (v, 0)); returns both sensors.
struct NoVisit2 {
    __device__ __forceinline__ void operator()(int, float2) const {}
};
template <int NT, class LD = LdPlain, class Also = NoVisit2>
__device__ __forceinline__ float2 pair_row_step(const float *__restrict__ in, const float *src,
                                                float *dst, const int *snb, bool top,
                                                const StepArgs &a, int x0, int y, int z,
                                                Also &&also = NoVisit2()) {
    using L = D3Q19;
    constexpr int n = NT, row = n, plane = n * (n + 2);
    const int G = a.G;
    const int nbm = snb[12], nbp = snb[14];  // the x - 1 and x + 1 neighbours
    const int g = (z + 1) * plane + (y + 1) * row + x0;
    const bool lo = x0 == 0, hi = x0 + 2 == n;
    if (y == 0 || y == n - 1 || z == 0 || z == n - 1) {
        const float K0 = step_cell<NT, false, LD>(in, src, dst, snb, top, a, x0, y, z,
                                                  [&](int i, float v) { also(i, make_float2(v, 0.f)); });
        const float K1 = step_cell<NT, false, LD>(in, src, dst, snb, top, a, x0 + 1, y, z,
                                                  [&](int i, float v) { also(i, make_float2(v, 0.f)); });
        return make_float2(K0, K1);
    }
    // the pull of direction i for a row whose y and z sources lie in this block (or its ghost
    // rows): the x-face lanes select their x neighbour
    const auto inner = [&](int i) -> float2 {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const int off = cz * plane + cy * row;
        const float *base = src + (i * G + g - off);
        if (cx == 0) return LD().pair(base);
        const int ghost = (z - cz + 1) * (n + 2) + (y - cy + 1);
        if (cx == 1) {  // cell x0 pulls from x0 - 1, cell x0 + 1 from x0
            const float *alt = nbm >= 0 ? in + ((size_t)nbm * Q * G + (i * G + g - off - 1 + n))
                               : nbm == NB_GHOST ? src + (i * G + side_base(n, 0) + ghost)
                                                 : src + (L::opp(i) * G + g);
            return make_float2(LD()(lo ? alt : base - 1), LD()(base));
        }
        // cell x0 pulls from x0 + 1, cell x0 + 1 from x0 + 2
        const float *alt = nbp >= 0 ? in + ((size_t)nbp * Q * G + (i * G + g - off + 2 - n))
                           : nbp == NB_GHOST ? src + (i * G + side_base(n, 1) + ghost)
                                             : src + (L::opp(i) * G + g + 1);
        return make_float2(LD()(base + 1), LD()(hi ? alt : base + 2));
    };
    float2 df[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] = __fadd2_rn(inner(i), f2(-weight<L, float>(i)));
    return relax_pair<L, 1, 1>([&](int i) { return df[i]; }, [&](int i) { return df[i]; },
                               a.omega, [&](int i, float2 v) {
                                   *reinterpret_cast<float2 *>(dst + (i * G + g)) = v;
                                   also(i, v);
                               });
}

template <int NT>
__global__ void __launch_bounds__(256, 3) k_step_pair(const float *__restrict__ in,
                                                   float *__restrict__ out,
                                                   const int *__restrict__ nbr, const StepArgs a,
                                                   int cpt, float *kmax) {
    __shared__ int snb[27];
    const int slot = blockIdx.x;
    if (threadIdx.x < 27) snb[threadIdx.x] = nbr[27 * slot + threadIdx.x];
    __syncthreads();
    constexpr int n = NT, half = NT / 2, npair = NT * NT * NT / 2;
    const bool top = snb[NB_TOP] == NB_WALL;
    const float *src = in + (size_t)slot * Q * a.G;
    float *dst = out + (size_t)slot * Q * a.G;
    int km = 0;
    for (int r = 0; r < cpt; ++r) {
        const int pidx = (blockIdx.y * cpt + r) * blockDim.x + threadIdx.x;
        if (pidx >= npair) break;
        const int x0 = 2 * (pidx % half);
        int y, z;
        face_row_order<n>(pidx / half, y, z);
        const float2 K = pair_row_step<NT>(in, src, dst, snb, top, a, x0, y, z);
        km = max(km, max(__float_as_int(K.x), __float_as_int(K.y)));
    }
    block_max_flush(km, kmax, slot, threadIdx.x & 31);
}


// Where the fused restriction writes: the coarser level's current buffer, the coarse slot of every
// fine block, and the rescaling of the non-equilibrium part 2 (tau_c - 1) / (tau_f - 1).
struct RestrictArgs {
    float *coarse;
    const int *cslot;
    int Gc;
    float scale;
};

// The finest level's second sub-step with the restriction onto the next coarser level fused, for
// NT = 8, 16, 32, 64: one thread owns a 2 x 2 x 2 brick of fine cells (an x pair in two rows and
// two planes), steps its four row pairs as k_step_pair does and sums each population's
// post-collision values in registers; the coarse cell under the brick becomes their average with
// f^neq rescaled, as in k_restrict (summed in another order), so the restriction's second pass
// over the fine level is not needed and no thread waits for another.  Bricks come in the coarse
// block's interior-rows-first order, so that most warps take one kind of gather.
// One brick of k_step_pair_restrict: brick b (coarse-block order) of the fine block whose source
// and destination are src / dst, its coarse cell written to `coarse` (the coarse block); returns
// the largest sensor bits of its 8 cells.
// SACC: the 19 sums in this thread's column of a shared-memory array, sacc[i * stride] (fewer
// registers, so more CTAs per SM), instead of registers.
template <int NT, class LD = LdPlain, bool SACC = false>
__device__ __forceinline__ int brick_one(const float *__restrict__ in, const float *src, float *dst,
                                         const int *snb, bool top, const StepArgs &a, int b,
                                         float *coarse, int Gc, float scale,
                                         float *sacc = nullptr, int stride = 0) {
    constexpr int NC = NT / 2;
    const int xc = b % NC;
    int yc, zc;
    face_row_order<NC>(b / NC, yc, zc);
    float acc[Q];
    int km = 0;
    if constexpr (SACC) {
#pragma unroll 1
        for (int q4 = 0; q4 < 4; ++q4) {
            const float2 K = pair_row_step<NT, LD>(
                in, src, dst, snb, top, a, 2 * xc, 2 * yc + (q4 & 1), 2 * zc + (q4 >> 1),
                [&](int i, float2 v) {
                    float &c = sacc[i * stride];
                    c = q4 ? c + (v.x + v.y) : v.x + v.y;
                });
            km = max(km, max(__float_as_int(K.x), __float_as_int(K.y)));
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) acc[i] = sacc[i * stride];
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) acc[i] = 0.f;
#pragma unroll 1
        for (int q4 = 0; q4 < 4; ++q4) {
            const float2 K = pair_row_step<NT, LD>(
                in, src, dst, snb, top, a, 2 * xc, 2 * yc + (q4 & 1), 2 * zc + (q4 >> 1),
                [&](int i, float2 v) { acc[i] += v.x + v.y; });
            km = max(km, max(__float_as_int(K.x), __float_as_int(K.y)));
        }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) acc[i] *= 0.125f;
    float rho, ux, uy, uz;
    moments19(acc, rho, ux, uy, uz);
    const int gc = ((zc + 1) * (NC + 2) + (yc + 1)) * NC + xc;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float fe = feq19(i, rho, ux, uy, uz);
        coarse[i * Gc + gc] = fe + scale * (acc[i] - fe);
    }
    return km;
}

template <int NT>
__global__ void __launch_bounds__(256, 2)
    k_step_pair_restrict(const float *__restrict__ in, float *__restrict__ out,
                         const int *__restrict__ nbr, const StepArgs a, int cpt, float *kmax,
                         const RestrictArgs r) {
    __shared__ int snb[27];
    const int slot = blockIdx.x;
    if (threadIdx.x < 27) snb[threadIdx.x] = nbr[27 * slot + threadIdx.x];
    __syncthreads();
    constexpr int NC = NT / 2, nbrick = NC * NC * NC;
    const bool top = snb[NB_TOP] == NB_WALL;
    const float *src = in + (size_t)slot * Q * a.G;
    float *dst = out + (size_t)slot * Q * a.G;
    float *coarse = r.coarse + (size_t)r.cslot[slot] * Q * r.Gc;
    int km = 0;
    for (int k = 0; k < cpt; ++k) {
        const int b = (blockIdx.y * cpt + k) * blockDim.x + threadIdx.x;
        if (b >= nbrick) break;
        km = max(km, brick_one<NT>(in, src, dst, snb, top, a, b, coarse, r.Gc, r.scale));
    }
    block_max_flush(km, kmax, slot, threadIdx.x & 31);
}

// The same with the 19 sums of each brick in shared memory (19 x blockDim floats), so that three
// CTAs of 256 threads fit an SM without spilling.
template <int NT>
__global__ void __launch_bounds__(256, 3)
    k_step_pair_restrict_s(const float *__restrict__ in, float *__restrict__ out,
                           const int *__restrict__ nbr, const StepArgs a, int cpt, float *kmax,
                           const RestrictArgs r) {
    __shared__ int snb[27];
    extern __shared__ float sacc[];
    const int slot = blockIdx.x;
    if (threadIdx.x < 27) snb[threadIdx.x] = nbr[27 * slot + threadIdx.x];
    __syncthreads();
    constexpr int NC = NT / 2, nbrick = NC * NC * NC;
    const bool top = snb[NB_TOP] == NB_WALL;
    const float *src = in + (size_t)slot * Q * a.G;
    float *dst = out + (size_t)slot * Q * a.G;
    float *coarse = r.coarse + (size_t)r.cslot[slot] * Q * r.Gc;
    int km = 0;
    for (int k = 0; k < cpt; ++k) {
        const int b = (blockIdx.y * cpt + k) * blockDim.x + threadIdx.x;
        if (b >= nbrick) break;
        km = max(km, brick_one<NT, LdPlain, true>(in, src, dst, snb, top, a, b, coarse, r.Gc,
                                                  r.scale, sacc + threadIdx.x, blockDim.x));
    }
    block_max_flush(km, kmax, slot, threadIdx.x & 31);
}

// The tiled step of the finest level's second sub-step fused with the restriction onto the next
// coarser level (NT = 16, 32, 64: bricks one plane deep; zc even).  Each 2 x 2 x 2 group of fine
// cells is summed in a fixed order: x pairs by a lane shuffle, then the z pair in the owning
// thread, then the y pair from shared memory; the coarse cell is the average with its f^neq
// rescaled, as in k_restrict, so the restriction kernel and its re-read of the fine level are
// skipped.
template <int NT>
__global__ void __launch_bounds__(256, 4)
    k_step_tiled_restrict(const float *__restrict__ in, float *__restrict__ out,
                          const int *__restrict__ nbr, const StepArgs a, int zc, float *kmax,
                          const RestrictArgs r) {
    using T = Tile<NT>;
    static_assert(T::TZ == 1 && T::TY % 2 == 0, "one-plane bricks with row pairs");
    constexpr int NC = NT / 2, CX = NT / 2, CY = T::TY / 2;
    __shared__ int snb[27];
    __shared__ float part[2][Q][CY][CX];  // [y parity][population][coarse row][coarse x]
    const int slot = blockIdx.x;
    const int tid = threadIdx.y * T::TX + threadIdx.x;
    if (tid < 27) snb[tid] = nbr[27 * slot + tid];
    __syncthreads();
    const bool top = snb[NB_TOP] == NB_WALL;
    const float *src = in + (size_t)slot * Q * a.G;
    float *dst = out + (size_t)slot * Q * a.G;
    constexpr int ytiles = NT / T::TY;
    const int y = (blockIdx.y % ytiles) * T::TY + threadIdx.y;
    const int z0 = (blockIdx.y / ytiles) * zc;
    const int x = threadIdx.x;
    const int ypar = threadIdx.y & 1, yc = threadIdx.y >> 1, xc = x >> 1;
    const bool owner = (x & 1) == 0;
    float *coarse = r.coarse + (size_t)r.cslot[slot] * Q * r.Gc;
    int km = 0;
    for (int zz = 0; zz < zc; ++zz) {
        const bool second = zz & 1;
        const float K = step_cell<NT>(in, src, dst, snb, top, a, x, y, z0 + zz, [&](int i, float v) {
            const float pair = v + __shfl_xor_sync(0xffffffffu, v, 1);
            if (owner) {
                float &acc = part[ypar][i][yc][xc];
                acc = second ? acc + pair : pair;
            }
        });
        km = max(km, __float_as_int(K));
        if (second) {
            __syncthreads();
            if (tid < CY * CX) {
                const int cy = tid / CX, cx = tid % CX;
                float avg[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) avg[i] = 0.125f * (part[0][i][cy][cx] + part[1][i][cy][cx]);
                float rho, ux, uy, uz;
                moments19(avg, rho, ux, uy, uz);
                const int gx = cx, gy = (y - threadIdx.y) / 2 + cy, gz = (z0 + zz) / 2;
                const int gc = ((gz + 1) * (NC + 2) + (gy + 1)) * NC + gx;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const float fe = feq19(i, rho, ux, uy, uz);
                    coarse[i * r.Gc + gc] = fe + r.scale * (avg[i] - fe);
                }
            }
            __syncthreads();
        }
    }
    block_max_flush(km, kmax, slot, tid & 31);
}

// ------------------------------------------------------------------ persistent cycle kernel
// One launch runs a whole cycle: the work of the graph form (ghost fills, level steps, restrictions,
// the zeroing of each level's sensor maxima) as a list of phases in the order the graph enqueues
// them, each split into tasks (a ghost-fill chunk, or several units of 256 threads of a step,
// brick or restriction).  Persistent CTAs claim tasks in index order with an atomic counter; a
// task first waits until every phase it depends on has completed all its tasks
// (per-phase counters, read with acquire), then runs, then counts itself complete (fence, atomic
// add).  The dependencies are those of the graph form: each level's phases in order (its stream)
// and the cross-level waits on a coarser level's state before or after its step and on the
// restriction onto a finer level.  Every dependency points to an earlier phase, so when a CTA
// claims task t every task before t is held by a running CTA and finishes: no co-residency is
// needed.  Populations are read through L2 (LdL2), as buffers written by other CTAs of the same
// launch are read.  Every wait is bounded: one that runs out raises the abort flag and the error
// word, and every CTA then stops claiming tasks.
constexpr int PH_ZERO = 0;      // zero the level's per-slot sensor maxima
constexpr int PH_INTERP0 = 1;   // ghost fill from the coarser level before its step (theta 0)
constexpr int PH_INTERPB = 2;   // ghost fill blended in time (theta 1/2)
constexpr int PH_STEP = 3;      // level step
constexpr int PH_BRICK = 4;     // finest level's second sub-step with the restriction fused
constexpr int PH_RESTRICT = 5;  // restriction onto the level from the next finer one
constexpr int PK_THREADS = 256;
constexpr int PK_TASKS_PER_CTA = 8, PK_MAX_PER = 32;
constexpr unsigned long long PK_WAIT_NS = 1000000000ull;

struct PPhase {
    int kind, level, ntask, task0, dep0, ndep;
    int nunit, per, nbig;  // step / brick / restriction: work units (chunks of 256 threads); the
                           // first nbig tasks take per units each (a task outlasts the claim and
                           // the waits), the rest one unit each (a short tail before the next
                           // phase may start)
    int chunks;          // step / brick: units per slot
    int nslot;           // zero: slots
    const float *in;     // step / brick: source buffer; ghost fill: coarse state before its step;
                         // restriction: the finer level's state
    float *out;          // step / brick: destination; ghost fill: the fine level's buffer;
                         // restriction: the level's current buffer
    const float *aux;    // ghost fill: the coarse state after its step
    const int *nbr;      // step / brick: neighbour table
    float *kmax;         // step / brick / zero: per-slot sensor maxima
    const void *items;   // ghost fill: chunks; restriction: task list
    int nitems;
    const int *idst;     // ghost fill: the chunks' tasks and window cells
    const uint4 *isrc;
    const int *iwin;
    int G2, P2, plane2;  // ghost fill: coarse G; restriction: finer G, row pitch, plane size
    float theta, scale;
    StepArgs a;          // the level's step arguments (a.G: the level's G)
    float *coarse;       // brick: the coarser level's current buffer, its slots and G
    const int *cslot;
    int Gc;
};

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_gpu(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long pk_now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int NT>
__device__ __forceinline__ void pk_step(const PPhase &P, int slot, int chunk, const int *snb) {
    const bool top = snb[NB_TOP] == NB_WALL;
    const float *src = P.in + (size_t)slot * Q * P.a.G;
    float *dst = P.out + (size_t)slot * Q * P.a.G;
    int km = 0;
    if constexpr (NT == 0) {
        const int n = P.a.n, c = chunk * PK_THREADS + threadIdx.x;
        if (c < n * n * n) {
            const float K = step_cell<0, false, LdL2>(P.in, src, dst, snb, top, P.a, c % n,
                                                      (c / n) % n, c / (n * n));
            km = __float_as_int(K);
        }
    } else {
        constexpr int half = NT / 2, npair = NT * NT * NT / 2;
        const int pidx = chunk * PK_THREADS + threadIdx.x;
        if (pidx < npair) {
            int y, z;
            face_row_order<NT>(pidx / half, y, z);
            const float2 K =
                pair_row_step<NT, LdL2>(P.in, src, dst, snb, top, P.a, 2 * (pidx % half), y, z);
            km = max(__float_as_int(K.x), __float_as_int(K.y));
        }
    }
    block_max_flush(km, P.kmax, slot, threadIdx.x & 31);
}

template <int NT>
__device__ __forceinline__ void pk_brick(const PPhase &P, int slot, int chunk, const int *snb) {
    const bool top = snb[NB_TOP] == NB_WALL;
    const float *src = P.in + (size_t)slot * Q * P.a.G;
    float *dst = P.out + (size_t)slot * Q * P.a.G;
    float *coarse = P.coarse + (size_t)P.cslot[slot] * Q * P.Gc;
    const int b = chunk * PK_THREADS + threadIdx.x;
    int km = 0;
    if (b < (NT / 2) * (NT / 2) * (NT / 2))
        km = brick_one<NT, LdL2>(P.in, src, dst, snb, top, P.a, b, coarse, P.Gc, P.scale);
    block_max_flush(km, P.kmax, slot, threadIdx.x & 31);
}

// the units [u0, u1) of task k of a step, brick or restriction phase
__device__ __forceinline__ void task_units(const PPhase &P, int k, int &u0, int &u1) {
    if (k < P.nbig) {
        u0 = k * P.per;
        u1 = u0 + P.per;
    } else {
        u0 = P.nbig * P.per + (k - P.nbig);
        u1 = u0 + 1;
    }
    u1 = min(u1, P.nunit);
}

template <bool BRICK>
__device__ __forceinline__ void pk_run(const PPhase &P, int k, int *snb, float *swin) {
    const int tid = threadIdx.x;
    if (P.kind == PH_ZERO) {
        for (int i = tid; i < P.nslot; i += PK_THREADS) P.kmax[i] = 0.f;
        return;
    }
    if (P.kind == PH_INTERP0 || P.kind == PH_INTERPB) {  // one chunk per task
        const InterpChunk c = static_cast<const InterpChunk *>(P.items)[k];
        if (P.kind == PH_INTERPB)
            interp_chunk<FILL_BLEND, false, PK_THREADS>(c, P.idst, P.isrc, P.iwin, nullptr, P.out, P.a.G,
                                            P.in, P.aux, P.G2, P.theta, P.scale, swin, nullptr);
        else
            interp_chunk<FILL_PREV, false, PK_THREADS>(c, P.idst, P.isrc, P.iwin, P.out, nullptr, P.a.G, P.in,
                                           P.aux, P.G2, P.theta, P.scale, swin, nullptr);
        return;
    }
    if (P.kind == PH_RESTRICT) {
        int u0, u1;
        task_units(P, k, u0, u1);
        for (int kk = u0; kk < u1; ++kk) {
            const int j = kk * PK_THREADS + tid;
            if (j >= P.nitems) break;
            restrict_one<LdL2>(static_cast<const RestrictTask *>(P.items)[j], P.out, P.a.G, P.in,
                               P.P2, P.plane2, P.G2, P.scale);
        }
        return;
    }
    // step or brick: units in slot-major order, the block's neighbour table in shared memory
    int last = -1;
    int u0, u1;
    task_units(P, k, u0, u1);
    for (int kk = u0; kk < u1; ++kk) {
        const int slot = kk / P.chunks, chunk = kk - slot * P.chunks;
        if (slot != last) {
            if (last >= 0) __syncthreads();  // every thread is done with the previous table
            if (tid < 27) snb[tid] = P.nbr[27 * slot + tid];
            __syncthreads();
            last = slot;
        }
        if (P.kind == PH_STEP) {
            switch (P.a.n) {
                case 8: pk_step<8>(P, slot, chunk, snb); break;
                case 16: pk_step<16>(P, slot, chunk, snb); break;
                case 32: pk_step<32>(P, slot, chunk, snb); break;
                case 64: pk_step<64>(P, slot, chunk, snb); break;
                default: pk_step<0>(P, slot, chunk, snb); break;
            }
        } else if constexpr (BRICK) {  // a lean plan has no brick phase
            switch (P.a.n) {
                case 8: pk_brick<8>(P, slot, chunk, snb); break;
                case 16: pk_brick<16>(P, slot, chunk, snb); break;
                case 32: pk_brick<32>(P, slot, chunk, snb); break;
                default: pk_brick<64>(P, slot, chunk, snb); break;
            }
        }
    }
}

// ctr: [0] next task, [1] abort flag, [2 + p] completed tasks of phase p (zeroed before a launch).
// hold != 0 (a test hook) makes every dependency unreachable, so the first wait runs out.
template <bool BRICK>
__global__ void __launch_bounds__(PK_THREADS, BRICK ? 2 : 3)
    k_cycle(const PPhase *__restrict__ ph, int nph, const int *__restrict__ deps, int ntask,
            int *ctr, int *err, unsigned long long wait_ns, int hold) {
    __shared__ int s_task, s_phase;
    __shared__ int snb[27];
    __shared__ float swin[Q * IC_WIN];  // a ghost-fill chunk's window
    int *next = ctr, *abort_flag = ctr + 1, *done = ctr + 2;
    // thread 0: the phase of the last task (tasks of a CTA come in increasing order, so the phase
    // search resumes there)
    int plast = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(next, 1);
            int p = -1;
            if (t < ntask && !ld_relaxed_gpu(abort_flag)) {
                p = plast;
                while (p + 1 < nph && ph[p + 1].task0 <= t) ++p;
                plast = p;
                const int dep0 = ph[p].dep0, ndep = ph[p].ndep;
                for (int k = 0; k < ndep && p >= 0; ++k) {
                    const int d = deps[dep0 + k];
                    const int target = hold ? 0x7fffffff : ph[d].ntask;
                    if (ld_acquire_gpu(done + d) >= target) continue;
                    const unsigned long long t0 = pk_now_ns();
                    while (ld_acquire_gpu(done + d) < target) {
                        if (ld_acquire_gpu(abort_flag)) {
                            p = -1;
                            break;
                        }
                        if (pk_now_ns() - t0 > wait_ns) {
                            atomicExch(abort_flag, 1);
                            if (err) atomicOr(err, 1);
                            p = -1;
                            break;
                        }
                        __nanosleep(128);
                    }
                }
            }
            s_task = t;
            s_phase = p;
        }
        __syncthreads();
        const int p = s_phase;
        if (p < 0) break;
        pk_run<BRICK>(ph[p], s_task - ph[p].task0, snb, swin);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();  // this task's stores before its count
            atomicAdd(done + p, 1);
        }
    }
}

__global__ void k_fill_rest(float *buf, int nslot, int G) {
    const size_t total = (size_t)nslot * Q * G;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)((k / G) % Q);
        buf[k] = weight<D3Q19, float>(i);
    }
}

// per physical block: the sensor max of its leaf level
__global__ void k_leaf_max(const int *leaf_slot, const int *leaf_level, int nblk,
                           const float *k0, const float *k1, const float *k2, double *out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    const int l = leaf_level[b], s = leaf_slot[b];
    const float *k = l == 0 ? k0 : (l == 1 ? k1 : k2);
    out[b] = (double)k[s];
}

// ------------------------------------------------------------------------------ host side
inline int wrap(int g, int n, bool per) {
    if (g >= 0 && g < n) return g;
    if (per) return ((g % n) + n) % n;
    return -1;
}

}  // namespace ml
}  // namespace lbm

namespace lbm {
namespace ml {
namespace {

#define MLCK(call, what)                                          \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return report_cuda_error(e_, what); \
    } while (0)

int gidx(const Level &L, int x, int y, int z) { return cell_index(L.n, x, y, z); }

bool balanced(const Mesh &m) {
    for (int z = 0; z < m.nb[2]; ++z)
        for (int y = 0; y < m.nb[1]; ++y)
            for (int x = 0; x < m.nb[0]; ++x) {
                const int b = (z * m.nb[1] + y) * m.nb[0] + x;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int c[3] = {x + dx, y + dy, z + dz};
                            bool ok = true;
                            for (int a = 0; a < 3; ++a) {
                                const int w = wrap(c[a], m.nb[a], m.periodic & (1 << a));
                                if (w < 0) ok = false;
                                c[a] = w;
                            }
                            if (!ok) continue;
                            const int o = (c[2] * m.nb[1] + c[1]) * m.nb[0] + c[0];
                            if (abs(m.leaf[b] - m.leaf[o]) > 1) return false;
                        }
            }
    return true;
}

template <class T>
int upload(T **dev, const std::vector<T> &v) {
    *dev = nullptr;
    if (v.empty()) return LBM_OK;
    MLCK(lbm::dev_alloc((void **)dev, v.size() * sizeof(T)), "cudaMalloc(tasks)");
    MLCK(cudaMemcpy(*dev, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "cudaMemcpy");
    return LBM_OK;
}

// flat offset (population 0) of a level-l global cell already wrapped into the domain
int cell_offset(const Mesh &m, int l, const int g[3], int *slot_out) {
    const Level &L = m.lv[l];
    int b[3], loc[3];
    for (int a = 0; a < 3; ++a) {
        b[a] = g[a] / L.n;
        loc[a] = g[a] - b[a] * L.n;
    }
    const int blk = (b[2] * m.nb[1] + b[1]) * m.nb[0] + b[0];
    const int s = L.slot[blk];
    *slot_out = s;
    if (s < 0) return -1;
    return s * Q * L.G + gidx(L, loc[0], loc[1], loc[2]);
}

// One ghost cell's trilinear stencil in the coarser level, before chunking: flat offsets
// (population 0) of the 8 coarse cells.  face orders the ghost cells of a block by the face they lie
// on (x low / high, then y, then z), then z, y, x within it, so that consecutive cells of a chunk
// are neighbours on one face and share most of their coarse cells.
struct GhostStencil {
    int dst, src[8];
    int extrap;     // bit a: axis a extrapolates (weights 5/4, -1/4)
    long long key;  // slot, face, z, y, x
};

// Group consecutive stencils into chunks of at most IC_TASKS ghost cells touching at most IC_WIN
// coarse cells; the window of a chunk lists those cells by ascending offset (rows of a coarse block
// are contiguous, so the copy of a window coalesces).
void chunk_stencils(const std::vector<GhostStencil> &gs, std::vector<InterpChunk> &ch,
                    std::vector<int> &dst, std::vector<uint4> &src, std::vector<int> &win) {
    size_t k = 0;
    std::vector<int> cells;
    std::unordered_set<int> inwin;
    while (k < gs.size()) {
        inwin.clear();
        size_t e = k;
        while (e < gs.size() && e - k < (size_t)IC_TASKS) {
            int fresh[8], nf = 0;
            for (int s = 0; s < 8; ++s) {
                const int o = gs[e].src[s];
                if (inwin.count(o) || std::find(fresh, fresh + nf, o) != fresh + nf) continue;
                fresh[nf++] = o;
            }
            if (inwin.size() + nf > (size_t)IC_WIN) break;  // this cell starts the next chunk
            inwin.insert(fresh, fresh + nf);
            ++e;
        }
        cells.assign(inwin.begin(), inwin.end());
        std::sort(cells.begin(), cells.end());
        InterpChunk c = {(int)dst.size(), (int)(e - k), (int)win.size(), (int)cells.size()};
        for (size_t t = k; t < e; ++t) {
            unsigned h[8];
            for (int s = 0; s < 8; ++s)
                h[s] = (unsigned)(std::lower_bound(cells.begin(), cells.end(), gs[t].src[s]) -
                                  cells.begin());
            for (int a = 0; a < 3; ++a)
                if (gs[t].extrap & (1 << a)) h[a] |= IC_EXTRAP;
            dst.push_back(gs[t].dst);
            src.push_back(make_uint4(h[0] | h[1] << 16, h[2] | h[3] << 16, h[4] | h[5] << 16,
                                     h[6] | h[7] << 16));
        }
        win.insert(win.end(), cells.begin(), cells.end());
        ch.push_back(c);
        k = e;
    }
}

int build_tasks(Mesh &m, int l) {
    Level &L = m.lv[l];
    std::vector<int> nbr;
    std::vector<GhostStencil> stencils;
    const int n = L.n;
    for (int b = 0; b < m.nblk; ++b) {
        const int s = L.slot[b];
        if (s < 0) continue;
        const int bz = b / (m.nb[0] * m.nb[1]), by = (b / m.nb[0]) % m.nb[1], bx = b % m.nb[0];
        for (int z = -1; z <= n; ++z)
            for (int y = -1; y <= n; ++y)
                for (int x = -1; x <= n; ++x) {
                    const int out = (x < 0 || x >= n) + (y < 0 || y >= n) + (z < 0 || z >= n);
                    if (out == 0 || out == 3) continue;  // interior, or a corner (unused)
                    int g[3] = {bx * n + x, by * n + y, bz * n + z};
                    bool inside = true;
                    for (int a = 0; a < 3; ++a) {
                        const int w = wrap(g[a], L.cells[a], m.periodic & (1 << a));
                        if (w < 0) inside = false;
                        g[a] = w;
                    }
                    if (!inside) continue;  // a wall: the step bounces back
                    const int dst = s * Q * L.G + gidx(L, x, y, z);
                    int ns;
                    cell_offset(m, l, g, &ns);
                    if (ns >= 0) continue;  // the step reads the neighbouring block directly
                    if (l == 0) return report_error(LBM_EINVAL, "level-0 ghost without a source");
                    // ghost centre (g + 1/2) h_l lies at g/2 + 1/4 coarse cells: coarse cell
                    // g >> 1, offset -1/4 (g even) or +1/4 (g odd)
                    const Level &C = m.lv[l - 1];
                    int c0[3], c1[3], extrap = 0;
                    for (int a = 0; a < 3; ++a) {
                        const int c = g[a] >> 1;
                        const int dir = (g[a] & 1) ? 1 : -1;
                        const bool per = m.periodic & (1 << a);
                        const int nbr = wrap(c + dir, C.cells[a], per);
                        if (nbr >= 0) {
                            c0[a] = c;
                            c1[a] = nbr;
                        } else {
                            c0[a] = c;
                            c1[a] = wrap(c - dir, C.cells[a], per);
                            extrap |= 1 << a;
                        }
                    }
                    GhostStencil it;
                    it.dst = dst;
                    it.extrap = extrap;
                    {
                        const int face = x < 0 ? 0 : x >= n ? 1 : y < 0 ? 2 : y >= n ? 3
                                                                  : z < 0 ? 4 : 5;
                        it.key = ((((long long)s * 6 + face) * (n + 2) + (z + 1)) * (n + 2) +
                                  (y + 1)) * (n + 2) + (x + 1);
                    }
                    for (int k = 0; k < 8; ++k) {
                        int cc[3];
                        for (int a = 0; a < 3; ++a) cc[a] = ((k >> a) & 1) ? c1[a] : c0[a];
                        int cs;
                        it.src[k] = cell_offset(m, l - 1, cc, &cs);
                        if (cs < 0)
                            return report_error(LBM_EINVAL,
                                                "interpolation stencil outside the coarser level");
                    }
                    stencils.push_back(it);
                }
    }
    // neighbour table: for each slot and each of the 27 offsets, the slot of the neighbouring
    // block at this level, NB_GHOST if that block exists only coarser, NB_WALL outside the domain
    nbr.assign((size_t)27 * std::max(L.nslot, 1), NB_WALL);
    for (int b = 0; b < m.nblk; ++b) {
        const int s = L.slot[b];
        if (s < 0) continue;
        const int bc[3] = {b % m.nb[0], (b / m.nb[0]) % m.nb[1], b / (m.nb[0] * m.nb[1])};
        for (int k = 0; k < 27; ++k) {
            const int d[3] = {k % 3 - 1, (k / 3) % 3 - 1, k / 9 - 1};
            int c[3];
            bool inside = true;
            for (int a = 0; a < 3; ++a) {
                c[a] = wrap(bc[a] + d[a], m.nb[a], m.periodic & (1 << a));
                if (c[a] < 0) inside = false;
            }
            if (!inside) continue;
            const int o = L.slot[(c[2] * m.nb[1] + c[1]) * m.nb[0] + c[0]];
            nbr[(size_t)27 * s + k] = o >= 0 ? o : NB_GHOST;
        }
    }
    int st = upload(&L.nbr, nbr);
    if (st != LBM_OK) return st;
    if (l > 0) {  // the same physical block one level coarser (levels nest per block)
        std::vector<int> cs(std::max(L.nslot, 1), 0);
        for (int b = 0; b < m.nblk; ++b)
            if (L.slot[b] >= 0) cs[L.slot[b]] = m.lv[l - 1].slot[b];
        st = upload(&L.cslot, cs);
        if (st != LBM_OK) return st;
    }
    std::stable_sort(stencils.begin(), stencils.end(),
                     [](const GhostStencil &a, const GhostStencil &b) { return a.key < b.key; });
    std::vector<InterpChunk> chunks;
    std::vector<int> idst, win;
    std::vector<uint4> isrc;
    chunk_stencils(stencils, chunks, idst, isrc, win);
    st = upload(&L.ichunks, chunks);
    if (st == LBM_OK) st = upload(&L.idst, idst);
    if (st == LBM_OK) st = upload(&L.isrc, isrc);
    if (st == LBM_OK) st = upload(&L.iwin, win);
    if (st != LBM_OK) return st;
    L.ninterp = (int)idst.size();
    L.nichunk = (int)chunks.size();
    if (l < m.lmax) {
        const Level &F = m.lv[l + 1];
        std::vector<RestrictTask> rs;
        for (int b = 0; b < m.nblk; ++b) {
            const int sf = F.slot[b];
            if (sf < 0) continue;
            const int sc = L.slot[b];
            for (int z = 0; z < n; ++z)
                for (int y = 0; y < n; ++y)
                    for (int x = 0; x < n; ++x)
                        rs.push_back({sc * Q * L.G + gidx(L, x, y, z),
                                      sf * Q * F.G + gidx(F, 2 * x, 2 * y, 2 * z)});
        }
        st = upload(&L.restricts, rs);
        if (st != LBM_OK) return st;
        L.nrestrict = (int)rs.size();
    }
    return LBM_OK;
}

StepArgs step_args(const Mesh &m, int l) {
    const Level &L = m.lv[l];
    StepArgs a;
    a.n = L.n;
    a.G = L.G;
    a.P = L.P;
    a.plane = L.plane;
    a.omega = (float)(1.0 / L.tau);
    a.lid_x = (float)m.lid[0];
    a.lid_z = (float)m.lid[2];
    return a;
}

bool has_tiled(int n) { return n == 8 || n == 16 || n == 32 || n == 64; }

template <int NT>
cudaError_t launch_tiled(const Level &L, const StepArgs &a, int zc, cudaStream_t s, int src) {
    using T = Tile<NT>;
    const dim3 block(T::TX, T::TY, T::TZ);
    const dim3 grid(L.nslot, (NT / T::TY) * (NT / zc));
    k_step_tiled<NT><<<grid, block, 0, s>>>(L.buf[src], L.buf[src ^ 1], L.nbr, a, zc, L.kmax);
    return cudaGetLastError();
}

// FORM_TILED: zc planes per CTA (a multiple of the brick depth dividing n); else a flat kernel
// with threads x cpt cells (pairs for FORM_PAIR) per CTA
cudaError_t launch_step(const Mesh &m, int l, int form, int threads, int cpt, int zc,
                        cudaStream_t s, int src) {
    const Level &L = m.lv[l];
    const StepArgs a = step_args(m, l);
    if (form == FORM_TILED) {
        switch (L.n) {
            case 8: return launch_tiled<8>(L, a, zc, s, src);
            case 16: return launch_tiled<16>(L, a, zc, s, src);
            case 32: return launch_tiled<32>(L, a, zc, s, src);
            case 64: return launch_tiled<64>(L, a, zc, s, src);
            default: return cudaErrorInvalidValue;
        }
    }
    const int ncell = L.n * L.n * L.n;
    const int units = form == FORM_PAIR ? ncell / 2 : ncell;
    const int chunks = (units + threads * cpt - 1) / (threads * cpt);
    dim3 grid(L.nslot, chunks);
    const float *fin = L.buf[src];
    float *fout = L.buf[src ^ 1];
    if (form == FORM_PAIR) {
        switch (L.n) {
            case 8: k_step_pair<8><<<grid, threads, 0, s>>>(fin, fout, L.nbr, a, cpt, L.kmax); break;
            case 16: k_step_pair<16><<<grid, threads, 0, s>>>(fin, fout, L.nbr, a, cpt, L.kmax); break;
            case 32: k_step_pair<32><<<grid, threads, 0, s>>>(fin, fout, L.nbr, a, cpt, L.kmax); break;
            case 64: k_step_pair<64><<<grid, threads, 0, s>>>(fin, fout, L.nbr, a, cpt, L.kmax); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    if (form == FORM_SELECT) {
        switch (L.n) {
            case 16: k_step<16, true><<<grid, threads, 0, s>>>(fin, fout, L.nbr, a, cpt, L.kmax); break;
            case 32: k_step<32, true><<<grid, threads, 0, s>>>(fin, fout, L.nbr, a, cpt, L.kmax); break;
            case 64: k_step<64, true><<<grid, threads, 0, s>>>(fin, fout, L.nbr, a, cpt, L.kmax); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (L.n) {
        case 4: k_step<4><<<grid, threads, 0, s>>>(fin, fout, L.nbr, a, cpt, L.kmax); break;
        case 8: k_step<8><<<grid, threads, 0, s>>>(fin, fout, L.nbr, a, cpt, L.kmax); break;
        case 16: k_step<16><<<grid, threads, 0, s>>>(fin, fout, L.nbr, a, cpt, L.kmax); break;
        case 32: k_step<32><<<grid, threads, 0, s>>>(fin, fout, L.nbr, a, cpt, L.kmax); break;
        case 64: k_step<64><<<grid, threads, 0, s>>>(fin, fout, L.nbr, a, cpt, L.kmax); break;
        default: k_step<0><<<grid, threads, 0, s>>>(fin, fout, L.nbr, a, cpt, L.kmax); break;
    }
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_fused(const Mesh &m, int l, int zc, cudaStream_t s, int src) {
    const Level &L = m.lv[l], &C = m.lv[l - 1];
    using T = Tile<NT>;
    RestrictArgs r;
    r.coarse = C.buf[C.cur];
    r.cslot = L.cslot;
    r.Gc = C.G;
    r.scale = (float)(2.0 * (C.tau - 1.0) / (L.tau - 1.0));
    const dim3 block(T::TX, T::TY, T::TZ);
    const dim3 grid(L.nslot, (NT / T::TY) * (NT / zc));
    k_step_tiled_restrict<NT><<<grid, block, 0, s>>>(L.buf[src], L.buf[src ^ 1], L.nbr,
                                                     step_args(m, l), zc, L.kmax, r);
    return cudaGetLastError();
}

// The fused step + restriction of level l onto l - 1 (n = 16, 32 or 64; zc even, dividing n).
cudaError_t launch_step_restrict(const Mesh &m, int l, int zc, cudaStream_t s, int src) {
    switch (m.lv[l].n) {
        case 16: return launch_fused<16>(m, l, zc, s, src);
        case 32: return launch_fused<32>(m, l, zc, s, src);
        case 64: return launch_fused<64>(m, l, zc, s, src);
        default: return cudaErrorInvalidValue;
    }
}

template <int NT>
cudaError_t launch_brick(const Mesh &m, int l, int threads, int cpt, int mode, cudaStream_t s,
                         int src) {
    const Level &L = m.lv[l], &C = m.lv[l - 1];
    RestrictArgs r;
    r.coarse = C.buf[C.cur];
    r.cslot = L.cslot;
    r.Gc = C.G;
    r.scale = (float)(2.0 * (C.tau - 1.0) / (L.tau - 1.0));
    const int nbrick = (NT / 2) * (NT / 2) * (NT / 2);
    const dim3 grid(L.nslot, (nbrick + threads * cpt - 1) / (threads * cpt));
    if (mode == BRICK_SMEM)
        k_step_pair_restrict_s<NT><<<grid, threads, sizeof(float) * Q * threads, s>>>(
            L.buf[src], L.buf[src ^ 1], L.nbr, step_args(m, l), cpt, L.kmax, r);
    else
        k_step_pair_restrict<NT><<<grid, threads, 0, s>>>(L.buf[src], L.buf[src ^ 1], L.nbr,
                                                           step_args(m, l), cpt, L.kmax, r);
    return cudaGetLastError();
}

// The brick form of the fused step + restriction of level l onto l - 1 (n = 8, 16, 32, 64).
cudaError_t launch_step_restrict_brick(const Mesh &m, int l, int threads, int cpt, int mode,
                                       cudaStream_t s, int src) {
    switch (m.lv[l].n) {
        case 8: return launch_brick<8>(m, l, threads, cpt, mode, s, src);
        case 16: return launch_brick<16>(m, l, threads, cpt, mode, s, src);
        case 32: return launch_brick<32>(m, l, threads, cpt, mode, s, src);
        case 64: return launch_brick<64>(m, l, threads, cpt, mode, s, src);
        default: return cudaErrorInvalidValue;
    }
}

bool can_fuse_brick(const Mesh &m, int l) {
    return l == m.lmax && l > 0 && has_tiled(m.lv[l].n) && m.lv[l - 1].nrestrict > 0;
}

bool can_fuse(const Mesh &m, int l) {
    const int n = m.lv[l].n;
    return l == m.lmax && l > 0 && (n == 16 || n == 32 || n == 64) && m.lv[l - 1].nrestrict > 0;
}

int brick_depth(int n) {
    switch (n) {
        case 8: return Tile<8>::TZ;
        case 16: return Tile<16>::TZ;
        case 32: return Tile<32>::TZ;
        case 64: return Tile<64>::TZ;
        default: return 0;
    }
}

inline unsigned blocks_for(int n, int t) { return (unsigned)((n + t - 1) / t); }

// One level-l step (the first of a pair, theta 0, also fills the ghosts of both), then the two
// sub-steps of the finer level and the restriction onto this one.  Level l's work goes to stream
// ss[l].  Dependencies between levels are events: a finer level's ghost fill waits for the
// coarser step (its first sub-step's ghosts come from the coarser state before that step, its
// second's from the blend of before and after); the restriction onto level l waits for the finer
// level's second sub-step and the restriction onto the finer level.  The coarser level's next
// step waits for that restriction, which covers every read of the buffer it overwrites.
int advance(Mesh &m, int l, float theta, cudaStream_t *ss) {
    Level &L = m.lv[l];
    if (L.nslot == 0) return LBM_OK;  // no block reaches this level (nor a finer one)
    cudaStream_t s = ss[l];
    if (l > 0) {
        // the ghosts of both sub-steps are filled once the coarser step is done, from one copy of
        // the coarse window: theta 0 into this buffer and theta 1/2 into the other, which the
        // first sub-step writes only inside the blocks
        MLCK(cudaStreamWaitEvent(s, m.ev_post[l - 1], 0), "cudaStreamWaitEvent");
        if (L.ninterp && theta == 0.f) {
            const Level &C = m.lv[l - 1];
            const float scale = (float)((L.tau - 1.0) / (2.0 * (C.tau - 1.0)));
            k_interp<FILL_BOTH><<<L.nichunk, interp_threads(FILL_BOTH), interp_smem(FILL_BOTH),
                                   s>>>(
                L.ichunks, L.idst, L.isrc, L.iwin, L.buf[L.cur], L.buf[L.cur ^ 1], L.G,
                C.buf[C.cur ^ 1], C.buf[C.cur], C.G, 0.5f, scale);
        }
    }
    MLCK(cudaGetLastError(), "ghost fill");
    MLCK(cudaMemsetAsync(L.kmax, 0, sizeof(float) * L.nslot, s), "memset(kmax)");
    MLCK(cudaEventRecord(m.ev_pre[l], s), "cudaEventRecord");
    if (L.fuse_brick && theta > 0.f)  // the finest level's second sub-step restricts as it steps
        MLCK(launch_step_restrict_brick(m, l, L.brick_threads, L.brick_cpt, L.brick_mode, s, L.cur),
             "level step + restriction");
    else if (L.fuse && theta > 0.f)
        MLCK(launch_step_restrict(m, l, L.fuse_zc, s, L.cur), "level step + restriction");
    else
        MLCK(launch_step(m, l, L.form, L.threads, L.cpt, L.zc, s, L.cur), "level step");
    L.cur ^= 1;
    MLCK(cudaEventRecord(m.ev_post[l], s), "cudaEventRecord");
    if (l < m.lmax) {
        int st = advance(m, l + 1, 0.f, ss);
        if (st == LBM_OK) st = advance(m, l + 1, 0.5f, ss);
        if (st != LBM_OK) return st;
        const Level &F = m.lv[l + 1];
        if (F.nslot > 0) MLCK(cudaStreamWaitEvent(s, m.ev_done[l + 1], 0), "cudaStreamWaitEvent");
        if (L.nrestrict && !F.fuse && !F.fuse_brick) {
            const float scale = (float)(2.0 * (L.tau - 1.0) / (F.tau - 1.0));
            k_restrict<<<blocks_for(L.nrestrict, 128), 128, 0, s>>>(
                L.restricts, L.nrestrict, L.buf[L.cur], L.G, F.buf[F.cur], F.P, F.plane, F.G,
                scale);
            MLCK(cudaGetLastError(), "restriction");
        }
    }
    MLCK(cudaEventRecord(m.ev_done[l], s), "cudaEventRecord");
    return LBM_OK;
}

// One level-0 cycle on stream s: the finer levels' streams join s at the start and s waits for
// them at the end.
int cycle(Mesh &m, cudaStream_t s) {
    cudaStream_t ss[MAXL];
    ss[0] = s;
    MLCK(cudaEventRecord(m.ev_fork, s), "cudaEventRecord");
    for (int l = 1; l <= m.lmax; ++l) {
        ss[l] = m.lst[l];
        MLCK(cudaStreamWaitEvent(ss[l], m.ev_fork, 0), "cudaStreamWaitEvent");
    }
    int st = advance(m, 0, 0.f, ss);
    for (int l = 1; l <= m.lmax; ++l) {
        MLCK(cudaEventRecord(m.ev_join[l], ss[l]), "cudaEventRecord");
        MLCK(cudaStreamWaitEvent(s, m.ev_join[l], 0), "cudaStreamWaitEvent");
    }
    return st;
}

// Time each launch shape of the level step once and keep the fastest: the flat kernel with
// (threads, cells per thread) in {128, 256, 512} x {1, 2, 4}, and the tiled kernel with every depth
// of planes it can walk.  The trial steps write the level's other buffer; the caller re-fills both
// buffers afterwards.
int autotune(Mesh &m, int l, cudaStream_t s) {
    Level &L = m.lv[l];
    if (L.nslot == 0) return LBM_OK;
    const int ncell = L.n * L.n * L.n;
    struct Cand {
        int form, threads, cpt, zc;
    };
    std::vector<Cand> cand;
    const int flat[][2] = {{128, 1}, {128, 2}, {256, 1}, {256, 2}, {256, 4}, {512, 1}, {512, 2}};
    const bool select_ok = L.n == 16 || L.n == 32 || L.n == 64;
    const bool pair_ok = has_tiled(L.n);  // edges 8, 16, 32, 64
    for (int form : {FORM_FLAT, FORM_SELECT})
        if (form == FORM_FLAT || select_ok)
            for (const auto &c : flat)
                if (c[0] * c[1] <= 2 * ncell || (c[0] == 128 && c[1] == 1))
                    cand.push_back({form, c[0], c[1], 1});
    if (pair_ok)
        for (const auto &c : flat)  // k_step_pair takes at most 256 threads per CTA
            if (c[0] <= 256 && (c[0] * c[1] <= ncell || (c[0] == 128 && c[1] == 1)))
                cand.push_back({FORM_PAIR, c[0], c[1], 1});
    if (has_tiled(L.n))
        for (int zc = brick_depth(L.n); zc <= L.n; zc *= 2)
            cand.push_back({FORM_TILED, 256, zc / brick_depth(L.n), zc});
    // a forced form keeps only its own candidates, where it applies to this level's edge
    if (m.step_form >= 0) {
        std::vector<Cand> keep;
        for (const Cand &c : cand)
            if (c.form == m.step_form) keep.push_back(c);
        if (!keep.empty()) cand.swap(keep);
    }
    cudaEvent_t e0, e1;
    MLCK(cudaEventCreate(&e0), "cudaEventCreate");
    MLCK(cudaEventCreate(&e1), "cudaEventCreate");
    float best = 1e30f;
    for (const Cand &c : cand) {
        for (int k = 0; k < 2; ++k)
            MLCK(launch_step(m, l, c.form, c.threads, c.cpt, c.zc, s, L.cur), "autotune");
        MLCK(cudaEventRecord(e0, s), "cudaEventRecord");
        for (int k = 0; k < 3; ++k)
            MLCK(launch_step(m, l, c.form, c.threads, c.cpt, c.zc, s, L.cur), "autotune");
        MLCK(cudaEventRecord(e1, s), "cudaEventRecord");
        MLCK(cudaEventSynchronize(e1), "cudaEventSynchronize");
        float ms = 0.f;
        MLCK(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
        if (ms < best) {
            best = ms;
            L.form = c.form;
            L.threads = c.threads;
            L.cpt = c.cpt;
            L.zc = c.zc;
        }
    }
    // finest level: the restriction onto the next coarser level as a separate kernel after the
    // second sub-step, or fused into that sub-step -- the tiled form (forced only: measured slower
    // on the benchmark mesh, 3.45 against 2.65 ms per cycle) or the brick form, timed against the
    // separate step + restriction unless a setting forces one
    L.fuse = false;
    L.fuse_brick = false;
    if (can_fuse(m, l) && m.fusion == 2) {
        L.fuse = true;
        L.fuse_zc = 4;
    }
    if (can_fuse_brick(m, l) && (m.fusion == 0 || m.fusion == 3)) {
        const Level &C = m.lv[l - 1];
        const float scale = (float)(2.0 * (C.tau - 1.0) / (L.tau - 1.0));
        const auto time_it = [&](auto &&launch, float *ms) -> int {
            for (int k = 0; k < 2; ++k) MLCK(launch(), "autotune");
            MLCK(cudaEventRecord(e0, s), "cudaEventRecord");
            for (int k = 0; k < 3; ++k) MLCK(launch(), "autotune");
            MLCK(cudaEventRecord(e1, s), "cudaEventRecord");
            MLCK(cudaEventSynchronize(e1), "cudaEventSynchronize");
            MLCK(cudaEventElapsedTime(ms, e0, e1), "cudaEventElapsedTime");
            return LBM_OK;
        };
        float sep = 0.f;
        int st = time_it([&]() -> cudaError_t {
            cudaError_t e = launch_step(m, l, L.form, L.threads, L.cpt, L.zc, s, L.cur);
            if (e != cudaSuccess) return e;
            k_restrict<<<blocks_for(C.nrestrict, 128), 128, 0, s>>>(
                C.restricts, C.nrestrict, C.buf[C.cur], C.G, L.buf[L.cur ^ 1], L.P, L.plane, L.G,
                scale);
            return cudaGetLastError();
        }, &sep);
        if (st != LBM_OK) return st;
        float bestb = 1e30f;
        const int nbrick = (L.n / 2) * (L.n / 2) * (L.n / 2);
        const int shapes[][2] = {{128, 1}, {128, 2}, {256, 1}, {256, 2}};
        for (int sm = BRICK_REG; sm <= BRICK_SMEM; ++sm)
            for (const auto &c : shapes) {
                if (c[0] * c[1] > 2 * nbrick && !(c[0] == 128 && c[1] == 1)) continue;
                float ms = 0.f;
                st = time_it(
                    [&]() {
                        return launch_step_restrict_brick(m, l, c[0], c[1], sm, s, L.cur);
                    },
                    &ms);
                if (st != LBM_OK) return st;
                if (ms < bestb) {
                    bestb = ms;
                    L.brick_threads = c[0];
                    L.brick_cpt = c[1];
                    L.brick_mode = sm;
                }
            }
        L.fuse_brick = m.fusion == 3 || bestb < sep;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return LBM_OK;
}

int capture(Mesh &m, cudaGraphExec_t *out) {
    cudaStream_t cap;
    MLCK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int st = LBM_OK;
    if (e == cudaSuccess) {
        st = cycle(m, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e2 != cudaSuccess && st == LBM_OK) st = report_cuda_error(e2, "graph capture");
    } else {
        st = report_cuda_error(e, "graph capture");
    }
    if (st == LBM_OK) {
        e = cudaGraphInstantiate(out, g, 0);
        if (e != cudaSuccess) st = report_cuda_error(e, "cudaGraphInstantiate");
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    return st;
}


}  // namespace
int run_cycles(Mesh *m, int cycles, cudaStream_t s, bool graphs, int *err, unsigned long long wait_ns,
               int hold);
namespace {

// --------------------------------------------------------- persistent cycle: the phase plan
// The phases of one cycle and their dependencies, built by walking the cycle exactly as advance()
// enqueues it: each level is a stream whose phases depend on the one before (stream order), and
// the cross-level event waits of advance() become dependencies on the phase recorded there.
struct PlanBuilder {
    std::vector<PPhase> ph;
    std::vector<std::vector<int>> dl;
    int last[MAXL];
    // what a stream's next phase waits for besides the stream's last phase
    std::vector<int> pend[MAXL];
    // the events of advance(): the phases a wait on them covers (a stream's last phase and the
    // waits pending on it when the event was recorded, as a CUDA event recorded after a
    // cudaStreamWaitEvent covers the awaited work)
    std::vector<int> pre[MAXL], post[MAXL], done[MAXL];
    PlanBuilder() {
        for (int l = 0; l < MAXL; ++l) last[l] = -1;
    }
    std::vector<int> record(int s) const {
        std::vector<int> e = pend[s];
        if (last[s] >= 0) e.push_back(last[s]);
        return e;
    }
    void wait(int s, const std::vector<int> &ev) { pend[s].insert(pend[s].end(), ev.begin(), ev.end()); }
    void add(int s, PPhase p) {
        std::vector<int> d = pend[s];
        pend[s].clear();
        if (last[s] >= 0) d.push_back(last[s]);
        std::sort(d.begin(), d.end());
        d.erase(std::unique(d.begin(), d.end()), d.end());
        ph.push_back(p);
        dl.push_back(d);
        last[s] = (int)ph.size() - 1;
    }
};

// Units of 256 threads per task of a step, brick or restriction phase: claiming a task and waiting
// for its dependencies cost a few microseconds of one thread's latency, which a single unit's work
// does not cover, so a task takes several; about PK_TASKS_PER_CTA tasks per CTA of the launch keep
// the phase's tail short.
int units_per_task(const Mesh &m, int nunit) {
    return std::max(1, std::min(PK_MAX_PER, nunit / (PK_TASKS_PER_CTA * std::max(m.pk_grid, 1))));
}

// Tasks of a phase of nunit units: about three quarters of the units in tasks of
// units_per_task units, the rest in one-unit tasks, which CTAs finishing early pick up while the
// last large tasks run, so that the phase ends soon after its last large task.
void split_tasks(const Mesh &m, PPhase &p) {
    p.per = units_per_task(m, p.nunit);
    p.nbig = p.per > 1 ? (3 * p.nunit / 4) / p.per : 0;
    p.ntask = p.nbig + (p.nunit - p.nbig * p.per);
}

int step_chunks(int n) {
    return has_tiled(n) ? (n * n * n / 2 + PK_THREADS - 1) / PK_THREADS
                        : (n * n * n + PK_THREADS - 1) / PK_THREADS;
}

void plan_advance(Mesh &m, PlanBuilder &b, int l, float theta) {
    Level &L = m.lv[l];
    if (L.nslot == 0) return;
    if (l > 0) {
        b.wait(l, theta > 0.f ? b.post[l - 1] : b.pre[l - 1]);
        if (L.ninterp) {
            const Level &C = m.lv[l - 1];
            PPhase p = {};
            p.kind = theta > 0.f ? PH_INTERPB : PH_INTERP0;
            p.level = l;
            p.items = L.ichunks;
            p.nitems = L.nichunk;
            p.idst = L.idst;
            p.isrc = L.isrc;
            p.iwin = L.iwin;
            p.ntask = L.nichunk;
            p.out = L.buf[L.cur];
            p.in = C.buf[C.cur ^ 1];
            p.aux = C.buf[C.cur];
            p.a = step_args(m, l);
            p.G2 = C.G;
            p.theta = theta;
            p.scale = (float)((L.tau - 1.0) / (2.0 * (C.tau - 1.0)));
            b.add(l, p);
        }
    }
    PPhase z = {};
    z.kind = PH_ZERO;
    z.level = l;
    z.ntask = 1;
    z.kmax = L.kmax;
    z.nslot = L.nslot;
    b.add(l, z);
    b.pre[l] = b.record(l);
    PPhase st = {};
    st.level = l;
    st.in = L.buf[L.cur];
    st.out = L.buf[L.cur ^ 1];
    st.nbr = L.nbr;
    st.kmax = L.kmax;
    st.a = step_args(m, l);
    if (L.fuse_brick && theta > 0.f && !m.pk_lean) {
        const Level &C = m.lv[l - 1];
        st.kind = PH_BRICK;
        st.chunks = ((L.n / 2) * (L.n / 2) * (L.n / 2) + PK_THREADS - 1) / PK_THREADS;
        st.coarse = C.buf[C.cur];
        st.cslot = L.cslot;
        st.Gc = C.G;
        st.scale = (float)(2.0 * (C.tau - 1.0) / (L.tau - 1.0));
    } else {
        st.kind = PH_STEP;
        st.chunks = step_chunks(L.n);
    }
    st.nunit = L.nslot * st.chunks;
    split_tasks(m, st);
    b.add(l, st);
    L.cur ^= 1;
    b.post[l] = b.record(l);
    if (l < m.lmax) {
        plan_advance(m, b, l + 1, 0.f);
        plan_advance(m, b, l + 1, 0.5f);
        const Level &F = m.lv[l + 1];
        if (F.nslot > 0) b.wait(l, b.done[l + 1]);
        if (L.nrestrict && !F.fuse && (!F.fuse_brick || m.pk_lean)) {
            PPhase r = {};
            r.kind = PH_RESTRICT;
            r.level = l;
            r.items = L.restricts;
            r.nitems = L.nrestrict;
            r.nunit = (L.nrestrict + PK_THREADS - 1) / PK_THREADS;
            split_tasks(m, r);
            r.out = L.buf[L.cur];
            r.in = F.buf[F.cur];
            r.a = step_args(m, l);
            r.G2 = F.G;
            r.P2 = F.P;
            r.plane2 = F.plane;
            r.scale = (float)(2.0 * (L.tau - 1.0) / (F.tau - 1.0));
            b.add(l, r);
        }
    }
    b.done[l] = b.record(l);
}

// Build and upload the plan of a cycle starting at the current buffer parities (restored after).
int build_plan(Mesh &m, Mesh::Plan *out) {
    int saved[MAXL];
    for (int l = 0; l <= m.lmax; ++l) saved[l] = m.lv[l].cur;
    PlanBuilder b;
    plan_advance(m, b, 0, 0.f);
    for (int l = 0; l <= m.lmax; ++l) m.lv[l].cur = saved[l];
    std::vector<int> flat;
    int task = 0;
    for (size_t k = 0; k < b.ph.size(); ++k) {
        b.ph[k].task0 = task;
        task += b.ph[k].ntask;
        b.ph[k].dep0 = (int)flat.size();
        b.ph[k].ndep = (int)b.dl[k].size();
        for (int d : b.dl[k]) flat.push_back(d);
    }
    out->nph = (int)b.ph.size();
    out->ntask = task;
    if (flat.empty()) flat.push_back(0);
    MLCK(lbm::dev_alloc(&out->phases, sizeof(PPhase) * b.ph.size()), "cudaMalloc(plan)");
    MLCK(cudaMemcpy(out->phases, b.ph.data(), sizeof(PPhase) * b.ph.size(), cudaMemcpyHostToDevice),
         "cudaMemcpy(plan)");
    MLCK(lbm::dev_alloc(&out->deps, sizeof(int) * flat.size()), "cudaMalloc(plan deps)");
    MLCK(cudaMemcpy(out->deps, flat.data(), sizeof(int) * flat.size(), cudaMemcpyHostToDevice),
         "cudaMemcpy(plan deps)");
    if (2 + out->nph > m.pctr_len) {
        cudaFree(m.pctr);
        m.pctr = nullptr;
        m.pctr_len = 0;
        MLCK(lbm::dev_alloc(&m.pctr, sizeof(int) * (2 + out->nph)), "cudaMalloc(plan counters)");
        m.pctr_len = 2 + out->nph;
    }
    return LBM_OK;
}

// The plan of the current level-0 parity and the launch width, made before any stream capture
// (they allocate and copy).
int ensure_plan(Mesh &m) {
    if (!m.pk_grid) {  // the launch width, which also sizes the plan's tasks
        int per_sm = 0, dev = 0, nsm = 0;
        if (m.pk_lean)
            MLCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cycle<false>, PK_THREADS,
                                                               0),
                 "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        else
            MLCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cycle<true>, PK_THREADS,
                                                               0),
                 "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        MLCK(cudaGetDevice(&dev), "cudaGetDevice");
        MLCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "sm count");
        m.pk_grid = std::max(1, per_sm * nsm);
    }
    Mesh::Plan &P = m.plan[m.lv[0].cur];
    if (!P.phases) {
        const int st = build_plan(m, &P);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
}

// The persistent form of one cycle at the current level-0 parity: clear the counters, one launch.
int persistent_cycle(Mesh &m, cudaStream_t s) {
    const int st = ensure_plan(m);
    if (st != LBM_OK) return st;
    Mesh::Plan &P = m.plan[m.lv[0].cur];
    MLCK(cudaMemsetAsync(m.pctr, 0, sizeof(int) * (2 + P.nph), s), "memset(plan counters)");
    const unsigned grid = (unsigned)std::min(m.pk_grid, std::max(P.ntask, 1));
    if (m.pk_lean)
        k_cycle<false><<<grid, PK_THREADS, 0, s>>>(static_cast<const PPhase *>(P.phases), P.nph,
                                                   P.deps, P.ntask, m.pctr, m.err,
                                                   m.wait_ns ? m.wait_ns : PK_WAIT_NS, m.hold);
    else
        k_cycle<true><<<grid, PK_THREADS, 0, s>>>(static_cast<const PPhase *>(P.phases), P.nph,
                                                  P.deps, P.ntask, m.pctr, m.err,
                                                  m.wait_ns ? m.wait_ns : PK_WAIT_NS, m.hold);
    MLCK(cudaGetLastError(), "persistent cycle");
    // the launch covers a whole cycle: level 0 flips once, the finer levels an even number of times
    m.lv[0].cur ^= 1;
    return LBM_OK;
}

int capture_persistent(Mesh &m, cudaGraphExec_t *out) {
    const int pst = ensure_plan(m);
    if (pst != LBM_OK) return pst;
    cudaStream_t cap;
    MLCK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int st = LBM_OK;
    if (e == cudaSuccess) {
        const int cur0 = m.lv[0].cur;
        st = persistent_cycle(m, cap);
        m.lv[0].cur = cur0;
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e2 != cudaSuccess && st == LBM_OK) st = report_cuda_error(e2, "graph capture");
    } else {
        st = report_cuda_error(e, "graph capture");
    }
    if (st == LBM_OK) {
        e = cudaGraphInstantiate(out, g, 0);
        if (e != cudaSuccess) st = report_cuda_error(e, "cudaGraphInstantiate");
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    return st;
}

void drop_cycle_graphs(Mesh &m) {
    for (int k = 0; k < 2; ++k) {
        if (m.graph[k]) cudaGraphExecDestroy(m.graph[k]);
        m.graph[k] = nullptr;
    }
}

// Switch the persistent form between the cycle kernel with brick phases and the lean one; the
// plans and the launch width belong to the form, so they are made again when it changes.
void set_persistent_form(Mesh &m, bool lean) {
    if (m.pk_lean == lean) return;
    m.pk_lean = lean;
    m.pk_grid = 0;
    for (int k = 0; k < 2; ++k) {
        cudaFree(m.plan[k].phases);
        cudaFree(m.plan[k].deps);
        m.plan[k] = Mesh::Plan();
    }
    drop_cycle_graphs(m);
}

// Time a few cycles in each form (graph of separate launches; persistent kernel with the brick
// phases of the finest level, or lean: plain steps and restriction phases at 3 CTAs per SM) and
// keep the fastest, unless the schedule setting forces the graph (LBM_SCHEDULE_GRAPH), the
// persistent kernel (LBM_SCHEDULE_PERSISTENT: the faster of its two forms) or one of its forms
// (LBM_SCHEDULE_PERSISTENT_BRICK, _LEAN).  The persistent form
// needs a restriction that is a separate kernel or the brick form (not the tiled fused form).
int choose_schedule(Mesh &m, cudaStream_t s) {
    bool can = true, brick = false;
    for (int l = 0; l <= m.lmax; ++l) {
        if (m.lv[l].fuse) can = false;
        if (m.lv[l].fuse_brick) brick = true;
    }
    if (m.schedule == LBM_SCHEDULE_GRAPH || !can) {
        m.persistent = false;
        return LBM_OK;
    }
    if (m.schedule == LBM_SCHEDULE_PERSISTENT_BRICK || m.schedule == LBM_SCHEDULE_PERSISTENT_LEAN) {
        m.persistent = true;
        set_persistent_form(m, m.schedule == LBM_SCHEDULE_PERSISTENT_LEAN);
        return LBM_OK;
    }
    cudaEvent_t e0, e1;
    MLCK(cudaEventCreate(&e0), "cudaEventCreate");
    MLCK(cudaEventCreate(&e1), "cudaEventCreate");
    float ms[3] = {1e30f, 1e30f, 1e30f};  // graph, persistent with bricks, lean persistent
    int st = LBM_OK;
    for (int form = m.schedule == LBM_SCHEDULE_PERSISTENT ? 1 : 0; form < 3 && st == LBM_OK;
         ++form) {
        if (form == 2 && !brick) continue;  // without brick phases both plans are the same
        m.persistent = form >= 1;
        if (form >= 1) set_persistent_form(m, form == 2);
        drop_cycle_graphs(m);
        for (int k = 0; k < 5 && st == LBM_OK; ++k) {
            if (k == 2) MLCK(cudaEventRecord(e0, s), "cudaEventRecord");
            st = run_cycles(&m, 1, s, true, nullptr, 0, 0);
        }
        if (st != LBM_OK) break;
        MLCK(cudaEventRecord(e1, s), "cudaEventRecord");
        MLCK(cudaEventSynchronize(e1), "cudaEventSynchronize");
        MLCK(cudaEventElapsedTime(&ms[form], e0, e1), "cudaEventElapsedTime");
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LBM_OK) return st;
    const int best = (int)(std::min_element(ms, ms + 3) - ms);
    m.persistent = best >= 1;
    if (m.persistent) set_persistent_form(m, best == 2);
    drop_cycle_graphs(m);
    return LBM_OK;
}
}  // namespace

void destroy(Mesh *m) {
    if (!m) return;
    for (int k = 0; k < 2; ++k) {
        cudaFree(m->plan[k].phases);
        cudaFree(m->plan[k].deps);
    }
    cudaFree(m->pctr);
    for (int k = 0; k < 2; ++k)
        if (m->graph[k]) cudaGraphExecDestroy(m->graph[k]);
    if (m->ev_fork) cudaEventDestroy(m->ev_fork);
    for (int l = 0; l < MAXL; ++l) {
        for (cudaEvent_t e : {m->ev_pre[l], m->ev_post[l], m->ev_done[l], m->ev_join[l]})
            if (e) cudaEventDestroy(e);
        if (m->lst[l]) cudaStreamDestroy(m->lst[l]);
        Level &L = m->lv[l];
        cudaFree(L.buf[0]);
        cudaFree(L.buf[1]);
        cudaFree(L.nbr);
        cudaFree(L.cslot);
        cudaFree(L.ichunks);
        cudaFree(L.idst);
        cudaFree(L.isrc);
        cudaFree(L.iwin);
        cudaFree(L.restricts);
        cudaFree(L.kmax);
    }
    delete m;
}

bool same_layout(const Mesh *m, const int nb[3], int edge, int lmax, const int8_t *leaf) {
    if (!m || m->edge != edge || m->lmax != lmax) return false;
    for (int a = 0; a < 3; ++a)
        if (m->nb[a] != nb[a]) return false;
    return memcmp(m->leaf.data(), leaf, m->leaf.size()) == 0;
}

int build(Mesh **out, const int nb[3], int edge, int lmax, const int8_t *leaf, double tau_fine,
          const double lid[3], int periodic, int fusion, int step_form, int schedule,
          cudaStream_t s) {
    *out = nullptr;
    if (lmax < 0 || lmax >= MAXL) return report_error(LBM_EINVAL, "lmax must be 0, 1 or 2");
    if (edge < 1 || edge % (1 << lmax) != 0 || edge / (1 << lmax) < 2)
        return report_error(LBM_EINVAL,
                            "block edge must be a multiple of 2^lmax with >= 2 coarse cells");
    for (int a = 0; a < 3; ++a)
        if (nb[a] < 1) return report_error(LBM_EINVAL, "need at least one block per axis");
    Mesh *m = new Mesh();
    for (int a = 0; a < 3; ++a) m->nb[a] = nb[a];
    m->edge = edge;
    m->lmax = lmax;
    m->fusion = fusion;
    m->step_form = step_form;
    m->nblk = nb[0] * nb[1] * nb[2];
    m->leaf.assign(leaf, leaf + m->nblk);
    for (int a = 0; a < 3; ++a) m->lid[a] = lid[a];
    m->periodic = periodic;
    // streams of the finer levels and the events that order a cycle (see advance)
    bool ok = cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int l = 0; l < MAXL && ok; ++l) {
        ok = cudaEventCreateWithFlags(&m->ev_pre[l], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&m->ev_post[l], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&m->ev_done[l], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&m->ev_join[l], cudaEventDisableTiming) == cudaSuccess;
        if (ok && l > 0) ok = cudaStreamCreateWithFlags(&m->lst[l], cudaStreamNonBlocking) == cudaSuccess;
    }
    if (!ok) {
        destroy(m);
        return report_error(LBM_ECUDA, "cannot create the mesh's streams and events");
    }
    for (int b = 0; b < m->nblk; ++b)
        if (leaf[b] < 0 || leaf[b] > lmax) {
            destroy(m);
            return report_error(LBM_EINVAL, "leaf level outside 0..lmax");
        }
    if (!balanced(*m)) {
        destroy(m);
        return report_error(LBM_EINVAL, "touching blocks differ by more than one level");
    }
    const double nu_fine = (tau_fine - 0.5) / 3.0;
    int st = LBM_OK;
    for (int l = 0; l <= lmax && st == LBM_OK; ++l) {
        Level &L = m->lv[l];
        const int h = 1 << (lmax - l);
        L.n = edge / h;
        L.P = L.n;
        L.plane = L.n * (L.n + 2);
        L.G = ((L.n + 2) * (L.n + 2) * (L.n + 2) + 31) / 32 * 32;
        for (int a = 0; a < 3; ++a) L.cells[a] = nb[a] * L.n;
        L.tau = 3.0 * nu_fine / h + 0.5;
        if (lmax > 0 && fabs(L.tau - 1.0) < 1e-3) {
            st = report_error(LBM_EINVAL, "a level's tau is 1: the rescaling divides by tau - 1");
            break;
        }
        L.slot.assign(m->nblk, -1);
        for (int b = 0; b < m->nblk; ++b)
            if (leaf[b] >= l) L.slot[b] = L.nslot++;
        if ((long long)L.nslot * Q * L.G >= (1LL << 31)) {
            st = report_error(LBM_ENOTSUP, "a level exceeds 2^31 population values");
            break;
        }
        const size_t bytes = (size_t)L.nslot * Q * L.G * sizeof(float);
        cudaError_t e = lbm::dev_alloc((void **)&L.buf[0], bytes);
        if (e == cudaSuccess) e = lbm::dev_alloc((void **)&L.buf[1], bytes);
        if (e == cudaSuccess)
            e = lbm::dev_alloc((void **)&L.kmax, sizeof(float) * std::max(L.nslot, 1));
        if (e != cudaSuccess) {
            st = report_cuda_error(e, "cudaMalloc(level)");
            break;
        }
    }
    for (int l = 0; l <= lmax && st == LBM_OK; ++l) st = build_tasks(*m, l);
    for (int l = 0; l <= lmax && st == LBM_OK; ++l) st = autotune(*m, l, s);
    if (st == LBM_OK) {
        m->schedule = schedule;
        st = choose_schedule(*m, s);
    }
    if (st == LBM_OK) {
        // the state at build time is rest, f_i = w_i everywhere (the trial steps are overwritten)
        for (int l = 0; l <= lmax; ++l) {
            if (m->lv[l].nslot == 0) continue;
            for (int k = 0; k < 2; ++k)
                k_fill_rest<<<1024, 256, 0, s>>>(m->lv[l].buf[k], m->lv[l].nslot, m->lv[l].G);
            cudaMemsetAsync(m->lv[l].kmax, 0, sizeof(float) * std::max(m->lv[l].nslot, 1), s);
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = report_cuda_error(e, "mesh set-up");
    }
    if (st != LBM_OK) {
        destroy(m);
        return st;
    }
    *out = m;
    return LBM_OK;
}

int run_cycles(Mesh *m, int cycles, cudaStream_t s, bool graphs, int *err, unsigned long long wait_ns,
               int hold) {
    if (err != m->err || wait_ns != m->wait_ns || hold != m->hold) {
        // the persistent kernel takes these as launch arguments: captured graphs are stale
        m->err = err;
        m->wait_ns = wait_ns;
        m->hold = hold;
        if (m->persistent) drop_cycle_graphs(*m);
    }
    for (int c = 0; c < cycles; ++c) {
        if (graphs) {
            const int par = m->lv[0].cur;
            if (!m->graph[par]) {
                int saved[MAXL];
                for (int l = 0; l <= m->lmax; ++l) saved[l] = m->lv[l].cur;
                const int st = m->persistent ? capture_persistent(*m, &m->graph[par])
                                             : capture(*m, &m->graph[par]);
                for (int l = 0; l <= m->lmax; ++l) m->lv[l].cur = saved[l];
                if (st != LBM_OK) return st;
            }
            MLCK(cudaGraphLaunch(m->graph[par], s), "cudaGraphLaunch");
            // a cycle flips level 0 once; finer levels step an even number of times
            m->lv[0].cur ^= 1;
        } else {
            const int st = m->persistent ? persistent_cycle(*m, s) : cycle(*m, s);
            if (st != LBM_OK) return st;
        }
        m->cycles += 1;
    }
    return LBM_OK;
}

bool uses_persistent(const Mesh *m) { return m->persistent; }

int block_max(Mesh *m, double *out_host, cudaStream_t s) {
    std::vector<int> ls(m->nblk), ll(m->nblk);
    for (int b = 0; b < m->nblk; ++b) {
        ll[b] = m->leaf[b];
        ls[b] = m->lv[ll[b]].slot[b];
    }
    int *dls = nullptr, *dll = nullptr;
    double *dout = nullptr;
    int st = upload(&dls, ls);
    if (st == LBM_OK) st = upload(&dll, ll);
    if (st == LBM_OK && lbm::dev_alloc((void **)&dout, sizeof(double) * m->nblk) != cudaSuccess)
        st = report_error(LBM_ENOMEM, "cudaMalloc(block max)");
    if (st == LBM_OK) {
        const float *k1 = m->lmax >= 1 ? m->lv[1].kmax : m->lv[0].kmax;
        const float *k2 = m->lmax >= 2 ? m->lv[2].kmax : k1;
        k_leaf_max<<<blocks_for(m->nblk, 256), 256, 0, s>>>(dls, dll, m->nblk, m->lv[0].kmax, k1,
                                                            k2, dout);
        cudaError_t e = cudaMemcpyAsync(out_host, dout, sizeof(double) * m->nblk,
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = report_cuda_error(e, "block max");
    }
    cudaFree(dls);
    cudaFree(dll);
    cudaFree(dout);
    return st;
}

// interior populations of physical block b at level l, f[i][z][y][x] as doubles (host)
int get_block(Mesh *m, int l, int b, double *out, cudaStream_t s) {
    if (l < 0 || l > m->lmax || b < 0 || b >= m->nblk || m->lv[l].slot[b] < 0)
        return report_error(LBM_EINVAL, "no such block at that level");
    const Level &L = m->lv[l];
    std::vector<float> tmp((size_t)Q * L.G);
    MLCK(cudaMemcpyAsync(tmp.data(), L.buf[L.cur] + (size_t)L.slot[b] * Q * L.G,
                         tmp.size() * sizeof(float), cudaMemcpyDeviceToHost, s),
         "cudaMemcpyAsync");
    MLCK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    const int n = L.n;
    for (int i = 0; i < Q; ++i)
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x)
                    out[(((size_t)i * n + z) * n + y) * n + x] =
                        tmp[(size_t)i * L.G + gidx(L, x, y, z)];
    return LBM_OK;
}

int set_block(Mesh *m, int l, int b, const double *in, cudaStream_t s) {
    if (l < 0 || l > m->lmax || b < 0 || b >= m->nblk || m->lv[l].slot[b] < 0)
        return report_error(LBM_EINVAL, "no such block at that level");
    Level &L = m->lv[l];
    std::vector<float> tmp((size_t)Q * L.G);
    float *dst = L.buf[L.cur] + (size_t)L.slot[b] * Q * L.G;
    MLCK(cudaMemcpyAsync(tmp.data(), dst, tmp.size() * sizeof(float), cudaMemcpyDeviceToHost, s),
         "cudaMemcpyAsync");
    MLCK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    const int n = L.n;
    for (int i = 0; i < Q; ++i)
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x)
                    tmp[(size_t)i * L.G + gidx(L, x, y, z)] =
                        (float)in[(((size_t)i * n + z) * n + y) * n + x];
    MLCK(cudaMemcpyAsync(dst, tmp.data(), tmp.size() * sizeof(float), cudaMemcpyHostToDevice, s),
         "cudaMemcpyAsync");
    MLCK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return LBM_OK;
}

int info(const Mesh *m, int l, int *n, double *tau, int *nslot, int *threads, int *cpt) {
    if (l < 0 || l > m->lmax) return report_error(LBM_EINVAL, "no such level");
    const Level &L = m->lv[l];
    if (n) *n = L.n;
    if (tau) *tau = L.tau;
    if (nslot) *nslot = L.nslot;
    if (threads) *threads = L.threads;
    if (cpt) *cpt = L.cpt;
    return LBM_OK;
}

int schedule(const Mesh *m, int l, int *form, int *planes, int *fused) {
    if (l < 0 || l > m->lmax) return report_error(LBM_EINVAL, "no such level");
    const Level &L = m->lv[l];
    if (form) *form = L.form;
    if (planes) *planes = L.form == FORM_TILED ? L.zc : 0;
    if (fused) *fused = L.fuse ? L.fuse_zc : (L.fuse_brick ? 1 : 0);
    return LBM_OK;
}

long long cells_per_cycle(const Mesh *m) {
    long long c = 0;
    for (int l = 0; l <= m->lmax; ++l)
        c += (long long)m->lv[l].nslot * m->lv[l].n * m->lv[l].n * m->lv[l].n * (1LL << l);
    return c;
}

}  // namespace ml
}  // namespace lbm
