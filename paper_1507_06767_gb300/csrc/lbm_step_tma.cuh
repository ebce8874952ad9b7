// Fused lattice Boltzmann step (D3Q19), populations staged through shared memory by TMA.
//
// Same computation as fused_step_kernel (lbm_step.cuh), cell for cell, sharing its relax_store_cell
// (moments, Eqs. rho/u; equilibrium, Eq. feq_i; Knudsen sensor, Eq. sensor/kkn; BGK collision,
// Sec. 2.2) and, for cells on the lattice boundary, its gather_cell (pull-stream with moving-wall
// bounce-back, Sec. 4.1).  What differs is how the gathered populations reach the registers.
//
// The one-cell kernel keeps its q loads in registers while they are in flight, and on GB300 its
// bandwidth follows the bytes in flight per SM that the register file allows.  Here a producer warp
// drives the TMA engine: for every (row y, plane z) a CTA works on it copies the 19 rows the pull
// needs -- population i comes from row (y - c_iy, z - c_iz) -- into a ring of shared-memory
// stages.  Copies hold no registers, so a CTA keeps several stages (19 rows each) in flight while
// its 8 consumer warps compute on an earlier one.  Stages are handed over with mbarriers: `full`
// (TMA byte count) and `empty` (one arrival per consumer warp); there is no CTA-wide barrier in the
// loop.
//
// Rows: a CTA covers a chunk of 256 cells along x.  The main copy of a population row is the
// 256-element chunk itself, aligned, so no DRAM segment is fetched for a neighbour's benefit; the
// one element a shifted population (c_ix = +-1) needs from the next chunk comes from a 16-byte halo
// copy into a slot of its own, issued only where that chunk exists (for nx <= 256 never).  Every
// shared-memory destination of a copy starts on a 128-byte boundary.  Out-of-range parts of a copy
// read as zero and are never used: cells on the lattice boundary gather from global memory.
//
// Work units are (x chunk, row y, 8-plane z chunk), taken round-robin by persistent CTAs.  A unit
// holds one row of eight 8^3 sensor tiles, so tile maxima are combined across units with an
// integer atomicMax (K >= 0 orders like its bit pattern; a positive NaN wins) into a buffer that
// the previous sensor step cleared; this kernel clears the other buffer for the next one.
//
// Every wait is bounded (about one second of %globaltimer).  A warp whose wait runs out raises the
// CTA's abort flag and *err; the others stop at their next wait, the producer waits (bounded) for
// the copies it still has in flight, and the CTA exits.
#pragma once

#include <cuda.h>

#include "lbm_step.cuh"

namespace lbm {

constexpr int TMA_CHUNK = 256;  // cells along x per CTA (8 consumer warps x 32 lanes)
constexpr int TMA_UNIT_Z = 8;   // planes per work unit
constexpr int TMA_CONSUMER_WARPS = TMA_CHUNK / 32;
constexpr int TMA_THREADS = TMA_CHUNK + 32;  // + one producer warp
#ifndef LBM_TMA_CTAS_PER_SM
#define LBM_TMA_CTAS_PER_SM 3
#endif
#ifndef LBM_TMA_STAGES_32
#define LBM_TMA_STAGES_32 3
#endif
#ifndef LBM_TMA_STAGES_16
#define LBM_TMA_STAGES_16 6
#endif
#ifndef LBM_TMA_L2_PROMO
#define LBM_TMA_L2_PROMO 2  // 0 none, 1 64 B, 2 128 B, 3 256 B
#endif
constexpr int TMA_CTAS_PER_SM = LBM_TMA_CTAS_PER_SM;
constexpr unsigned long long TMA_WAIT_NS = 1000000000ull;

// Shared memory of a stage: 19 main rows of TMA_CHUNK elements, then 19 halo slots of 128 bytes
// (a 16-byte halo copy each).  Every TMA destination starts on a 128-byte boundary.
template <int DT>
struct TmaCfg {
    using T = typename Storage<DT>::T;
    static constexpr int H = 16 / (int)sizeof(T);                // halo copy width (16 bytes)
    static constexpr int MAIN_BYTES = TMA_CHUNK * (int)sizeof(T);  // multiple of 128
    static constexpr int HALO_SLOT = 128;
    static constexpr int HALO_OFF = 19 * MAIN_BYTES;
    static constexpr int STAGE_BYTES = 19 * (MAIN_BYTES + HALO_SLOT);
    static constexpr int STAGES = (sizeof(T) == 4) ? LBM_TMA_STAGES_32 : LBM_TMA_STAGES_16;
    static constexpr int HEADER = 128;  // mbarriers and the abort flag
    // + 128 so that the ring can start on a 128-byte boundary whatever the base alignment
    static constexpr int SMEM_BYTES = HEADER + 128 + STAGES * STAGE_BYTES;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of parity `parity` to complete.  Returns 1 when it did, 0 when the wait ran out
// of time, -1 when the CTA's abort flag was raised meanwhile.
__device__ __forceinline__ int mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                 const volatile int *abort_flag,
                                                 unsigned long long limit_ns = TMA_WAIT_NS) {
    if (mbar_try_wait(bar, parity)) return 1;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (abort_flag && *abort_flag) return -1;
        if (global_ns() - t0 > limit_ns) return 0;
    }
    return 1;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Work unit u of the lattice: x chunk, row, first plane and plane count.
struct TmaUnit {
    int x0, y, z0, nzu;
};

__device__ __forceinline__ TmaUnit tma_unit(int u, int uxc, int ny, int nz) {
    TmaUnit t;
    const int xc = u % uxc;
    const int r = u / uxc;
    t.x0 = xc * TMA_CHUNK;
    t.y = r % ny;
    t.z0 = (r / ny) * TMA_UNIT_Z;
    t.nzu = min(TMA_UNIT_Z, nz - t.z0);
    return t;
}

template <int DT, int MODE>
__global__ void __launch_bounds__(TMA_THREADS, TMA_CTAS_PER_SM)
    fused_step_tma_kernel(const __grid_constant__ CUtensorMap tmain,
                          const __grid_constant__ CUtensorMap thalo,
                          const typename Storage<DT>::T *__restrict__ fin,
                          typename Storage<DT>::T *__restrict__ fout, const StepParams p,
                          float *__restrict__ tile_max, float *__restrict__ tile_zero,
                          float *__restrict__ k_field) {
    using L = D3Q19;
    using S = Storage<DT>;
    using T = typename S::T;
    using C = TmaCfg<DT>;
    constexpr int Q = L::Q;
    constexpr int NS = C::STAGES;

    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t full0 = smem_addr(smem);   // NS barriers
    const uint32_t empty0 = full0 + 8 * NS;   // NS barriers
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 16 * NS);
    // ring on the first 128-byte boundary after the header
    const uint32_t ring0 = (full0 + C::HEADER + 127u) & ~127u;
    const unsigned char *ring_bytes = smem + (ring0 - full0);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const size_t N = (size_t)nx * ny * nz;
    const int uxc = (nx + TMA_CHUNK - 1) / TMA_CHUNK;
    // limit of the waits between the producer and the consumers; the producer's final wait for its
    // copies in flight keeps the full default, so no CTA exits while a copy into it is pending
    const unsigned long long wait_ns = p.wait_ns ? p.wait_ns : TMA_WAIT_NS;
    const int U = uxc * ny * ((nz + TMA_UNIT_Z - 1) / TMA_UNIT_Z);

    // clear the other tile buffer for the next sensor step
    if (MODE != 0 && tile_zero) {
        const size_t nt = (size_t)p.ntx * p.nty * p.ntz;
        for (size_t k = (size_t)blockIdx.x * blockDim.x + tid; k < nt;
             k += (size_t)gridDim.x * blockDim.x)
            tile_zero[k] = 0.f;
    }

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, TMA_CONSUMER_WARPS);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == TMA_CONSUMER_WARPS) {
        // ---------------------------------------------------------------- producer warp
        if (lane != 0 || p.hold_copies) return;
        int g = 0;
        bool stop = false;
        for (int u = blockIdx.x; u < U && !stop; u += gridDim.x) {
            const TmaUnit w = tma_unit(u, uxc, ny, nz);
            const bool left = w.x0 > 0, right = w.x0 + TMA_CHUNK < nx;
            const uint32_t bytes = (uint32_t)(19 * TMA_CHUNK * sizeof(T)) +
                                   (uint32_t)(((left ? 5 : 0) + (right ? 5 : 0)) * 16);
            for (int j = 0; j < w.nzu; ++j, ++g) {
                const int s = g % NS;
                if (g >= NS) {
                    const int r =
                        mbar_wait_bounded(empty0 + 8 * s, ((g / NS) - 1) & 1, abort_flag, wait_ns);
                    if (r != 1) {
                        if (r == 0) {
                            *abort_flag = 1;
                            if (p.err) atomicOr(p.err, 1);
                        }
                        stop = true;
                        break;
                    }
                }
                const int z = w.z0 + j;
                const uint32_t bar = full0 + 8 * s;
                const uint32_t stage = ring0 + (uint32_t)(s * C::STAGE_BYTES);
                mbar_arrive_expect_tx(bar, bytes);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int ys = w.y - L::cy(i), zs = z - L::cz(i);
                    tma_load_4d(stage + (uint32_t)(i * C::MAIN_BYTES), &tmain, w.x0, ys, zs, i, bar);
                    const uint32_t halo = stage + (uint32_t)(C::HALO_OFF + i * C::HALO_SLOT);
                    if (L::cx(i) == 1 && left) tma_load_4d(halo, &thalo, w.x0 - C::H, ys, zs, i, bar);
                    if (L::cx(i) == -1 && right)
                        tma_load_4d(halo, &thalo, w.x0 + TMA_CHUNK, ys, zs, i, bar);
                }
            }
        }
        // wait (bounded) for the copies still in flight: the last NS issued stages
        for (int g2 = max(0, g - NS); g2 < g; ++g2) {
            const int s = g2 % NS;
            mbar_wait_bounded(full0 + 8 * s, (g2 / NS) & 1, nullptr, TMA_WAIT_NS);
        }
        return;
    }

    // -------------------------------------------------------------------- consumer warps
    const float omega = p.omega_f;
    int g = 0;
    for (int u = blockIdx.x; u < U; u += gridDim.x) {
        const TmaUnit w = tma_unit(u, uxc, ny, nz);
        const int x = w.x0 + tid;
        const int y = w.y;
        int kmax = 0;
        bool quit = false;
        for (int j = 0; j < w.nzu; ++j, ++g) {
            const int s = g % NS;
            const int r = mbar_wait_bounded(full0 + 8 * s, (g / NS) & 1, abort_flag, wait_ns);
            if (r == 0) {
                *abort_flag = 1;
                if (p.err) atomicOr(p.err, 1);
            }
            // the lanes poll on their own: the warp stops as one if any of them stopped
            if (__any_sync(0xffffffffu, r != 1)) {
                quit = true;
                break;
            }
            const int z = w.z0 + j;
            if (x < nx) {
                float df[Q];
                const bool boundary =
                    x == 0 || x == nx - 1 || y == 0 || y == ny - 1 || z == 0 || z == nz - 1;
                if (boundary) {
                    gather_cell<L, DT>(fin, p, N, x, y, z, df);
                } else {
                    const unsigned char *st = ring_bytes + (size_t)s * C::STAGE_BYTES;
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const T *row = reinterpret_cast<const T *>(st + i * C::MAIN_BYTES);
                        const T *halo = reinterpret_cast<const T *>(st + C::HALO_OFF + i * C::HALO_SLOT);
                        const int col = tid - L::cx(i);  // -1 or TMA_CHUNK only at chunk edges
                        T raw;
                        if (L::cx(i) == 1)
                            raw = (col >= 0) ? row[col] : halo[C::H - 1];
                        else if (L::cx(i) == -1)
                            raw = (col < TMA_CHUNK) ? row[col] : halo[0];
                        else
                            raw = row[col];
                        float v = S::to_r(raw);
                        if (!S::SHIFTED) v -= weight<L, float>(i);
                        df[i] = v;
                    }
                }
                const int idx = (z * ny + y) * nx + x;
                const float K = relax_store_cell<L, DT, MODE>(df, omega, fout, N, idx);
                if (MODE != 0) {
                    kmax = max(kmax, __float_as_int(K));
                    if (MODE == 2) k_field[idx] = K;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty0 + 8 * s);
        }
        if (quit) return;
        if (MODE != 0) {
            // this unit's row of 8 tiles per warp: max over 8-lane groups, atomically into the tile
#pragma unroll
            for (int off = 4; off >= 1; off >>= 1) kmax = max(kmax, __shfl_xor_sync(~0u, kmax, off));
            const int tx = x >> 3;
            if ((lane & (TILE - 1)) == 0 && x < nx) {
                const size_t t = ((size_t)(w.z0 / TILE) * p.nty + (y / TILE)) * p.ntx + tx;
                atomicMax(reinterpret_cast<int *>(tile_max) + t, kmax);
            }
        }
    }
}

// Whether the TMA kernel applies: FP32 arithmetic on 16- or 32-bit storage and rows whose length
// in bytes is a multiple of 16 (TMA stride rule).
inline bool tma_applicable(int dtype, int nx) {
    if (dtype < 1 || dtype > 3) return false;
    const int es = (dtype == 1) ? 4 : 2;
    return ((long long)nx * es) % 16 == 0;
}

}  // namespace lbm
