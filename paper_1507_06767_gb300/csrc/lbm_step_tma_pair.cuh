// Fused lattice Boltzmann step for 16-bit shifted storage (f - w_i in FP16 or BF16, FP32
// arithmetic), D3Q19, with every population staged in shared memory by TMA.
//
// Same computation as fused_step_pair_kernel (lbm_step_pair.cuh): pull-stream with moving-wall
// bounce-back (Sec. 2.2 streaming, Sec. 4.1 lid), moments (Eqs. rho, u), equilibrium (Eq. feq_i),
// Knudsen sensor (Eq. sensor / kkn) with per-tile max, BGK collision (Sec. 2.2), two x-adjacent
// cells per thread with the packed-pair relaxation relax_pair.  What changes is how the
// populations arrive: with 16-bit storage the register-loaded two-cell kernel holds too few bytes
// in flight (its 64 registers per thread allow 4 CTAs of 256 threads per SM) and spends a fifth of
// its instructions on 64-bit address arithmetic.  Here
//   * persistent CTAs of 8 consumer warps and one producer warp walk work units of 64 (x) x 8 (y)
//     cells x 8 planes, x fastest, then y, then z; a unit owns eight whole 8^3 sensor tiles, so
//     tile maxima are written with plain stores (no atomics, no cleared buffer);
//   * for every plane z the producer lane copies, per direction i, the box of the previous
//     post-collision state the tile pulls from -- rows y - c_y, plane z - c_z -- into a stage of a
//     ring in shared memory: 64 cells wide for c_x = 0, 72 wide for c_x = +-1 (the 64 sources
//     x - c_x plus the alignment to 16 bytes that TMA requires); out-of-lattice parts read as zero;
//   * a consumer warp is one row of 64 cells, a lane two cells; it reads each population pair with
//     one or two 32-bit shared loads at constant offsets (plus one byte permute for c_x = +-1),
//     releases the stage, relaxes the pair and stores it with one 32-bit global store per
//     direction;
//   * at an x face, the lane holding the face cell takes the population that would come from
//     outside the lattice from a small face box: the cell's own opposite population (bounce-back
//     at a resting wall) or the wrapped column (periodic x);
//   * rows on a y face (the lid, y = ny - 1, and y = 0) and planes on a z face take the general
//     gather from global memory (gather_cell), as the other kernels do.
// Every wait is bounded (StepParams::wait_ns, default one second).  A warp whose wait runs out
// raises the CTA's abort flag and *err; the others stop at their next wait; the producer waits,
// with the full default limit, for the copies it still has in flight, and the CTA exits.
//
// Needs D3Q19, 16-bit storage, nx a multiple of 8 (TMA rows are multiples of 16 bytes) and
// (q + 1) * cells < 2^32 (32-bit element offsets of the stores).
#pragma once

#include <cuda.h>

#include "lbm_step_pair.cuh"
#include "lbm_step_tma.cuh"

namespace lbm {

constexpr int TP_TX = 64;         // cells along x per unit (32 lanes x 2 cells)
constexpr int TP_TY = 8;          // rows per unit (one consumer warp each)
constexpr int TP_TZ = 8;          // planes per unit
constexpr int TP_WARPS = TP_TY;   // consumer warps
constexpr int TP_THREADS = 32 * (TP_WARPS + 1);
constexpr int TP_WIDE = TP_TX + 8;  // box width for c_x = +-1
#ifndef LBM_TP_STAGES
#define LBM_TP_STAGES 3
#endif
#ifndef LBM_TP_CTAS_PER_SM
#define LBM_TP_CTAS_PER_SM 3
#endif
constexpr int TP_STAGES = LBM_TP_STAGES;
constexpr int TP_CTAS_PER_SM = LBM_TP_CTAS_PER_SM;

// Layout of one stage (bytes; every TMA destination on a 128-byte boundary): direction i's box at
// tp_box_off(i) -- rows of 64 (c_x = 0) or 72 (c_x = +-1) 16-bit values, 8 rows -- then the face
// boxes (8 x 8 values): five for the left face (the directions with c_x = +1, in index order),
// five for the right face (c_x = -1).
struct TpLayout {
    __host__ __device__ static constexpr int row_elems(int i) { return D3Q19::cx(i) ? TP_WIDE : TP_TX; }
    __host__ __device__ static constexpr int box_bytes(int i) { return row_elems(i) * TP_TY * 2; }
    __host__ __device__ static constexpr int box_off(int i) {
        int o = 0;
        for (int k = 0; k < i; ++k) o += box_bytes(k);
        return o;
    }
    static constexpr int FACE_BYTES = 8 * 8 * 2;
    static constexpr int FACE_OFF = 9 * TP_TX * TP_TY * 2 + 10 * TP_WIDE * TP_TY * 2;
    static constexpr int STAGE_BYTES = FACE_OFF + 10 * FACE_BYTES;
    static constexpr int HEADER = 128;  // full / empty barriers, abort flag
    static constexpr int TILE_PART_BYTES = 2 * TP_WARPS * (TP_TX / TILE) * 4;
    static constexpr int SMEM_BYTES = HEADER + TILE_PART_BYTES + 128 + TP_STAGES * STAGE_BYTES;
    // rank of direction i among the directions with the same c_x != 0 (face-box slot)
    __host__ __device__ static constexpr int face_rank(int i) {
        int r = 0;
        for (int k = 0; k < i; ++k)
            if (D3Q19::cx(k) == D3Q19::cx(i)) ++r;
        return r;
    }
};
static_assert(TpLayout::FACE_OFF % 128 == 0 && TpLayout::STAGE_BYTES % 128 == 0, "alignment");
static_assert(TpLayout::box_off(18) + TpLayout::box_bytes(18) == TpLayout::FACE_OFF, "layout");

struct TpMaps {
    CUtensorMap narrow;  // box (64, 8, 1, 1)
    CUtensorMap wide;    // box (72, 8, 1, 1)
    CUtensorMap face;    // box (8, 8, 1, 1)
};

struct TpUnit {
    int x0, y0, z0;
};

__device__ __forceinline__ TpUnit tp_unit(int u, int utx, int uty) {
    TpUnit w;
    w.x0 = (u % utx) * TP_TX;
    w.y0 = ((u / utx) % uty) * TP_TY;
    w.z0 = (u / (utx * uty)) * TP_TZ;
    return w;
}

__device__ __forceinline__ void named_barrier_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ unsigned lds32(uint32_t addr) {
    unsigned v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ unsigned lds16(uint32_t addr) {
    unsigned short v;
    asm volatile("ld.shared.b16 %0, [%1];" : "=h"(v) : "r"(addr));
    return v;
}

template <int DT, int MODE>
__global__ void __launch_bounds__(TP_THREADS, TP_CTAS_PER_SM)
    fused_step_tma_pair_kernel(const __grid_constant__ TpMaps maps,
                               const typename Storage<DT>::T *__restrict__ fin,
                               typename Storage<DT>::T *__restrict__ fout, const StepParams p,
                               float *__restrict__ tile_max, float *__restrict__ k_field) {
    using L = D3Q19;
    using S = Storage<DT>;
    using T = typename S::T;
    using RG = PairReg<DT>;
    using V = typename RG::V;
    using LY = TpLayout;
    constexpr int Q = L::Q;
    constexpr int NS = TP_STAGES;

    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t full0 = smem_addr(smem);  // NS barriers
    const uint32_t empty0 = full0 + 8 * NS;  // NS barriers
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 16 * NS);
    int *part = reinterpret_cast<int *>(smem + LY::HEADER);  // [2][TP_WARPS][8] tile maxima
    const uint32_t ring0 = (full0 + LY::HEADER + LY::TILE_PART_BYTES + 127u) & ~127u;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int utx = (nx + TP_TX - 1) / TP_TX, uty = (ny + TP_TY - 1) / TP_TY;
    const int U = utx * uty * ((nz + TP_TZ - 1) / TP_TZ);
    const unsigned long long wait_ns = p.wait_ns ? p.wait_ns : TMA_WAIT_NS;
    const bool perx = p.periodic & 1;

    if (MODE != 0 && p.tile_zero) {
        const size_t nt = (size_t)p.ntx * p.nty * p.ntz;
        for (size_t k = (size_t)blockIdx.x * blockDim.x + tid; k < nt;
             k += (size_t)gridDim.x * blockDim.x)
            static_cast<float *>(p.tile_zero)[k] = 0.f;
    }
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, TP_WARPS);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == TP_WARPS) {
        // ------------------------------------------------------------------ producer lane
        if (lane != 0 || p.hold_copies) return;
        int g = 0;
        bool stop = false;
        for (int u = blockIdx.x; u < U && !stop; u += gridDim.x) {
            const TpUnit w = tp_unit(u, utx, uty);
            const bool left = w.x0 == 0, right = w.x0 + TP_TX >= nx;
            const uint32_t bytes = (uint32_t)LY::FACE_OFF +
                                   (uint32_t)((left ? 5 : 0) + (right ? 5 : 0)) * LY::FACE_BYTES;
            for (int dz = 0; dz < TP_TZ; ++dz, ++g) {
                const int z = w.z0 + dz;
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
                const uint32_t bar = full0 + 8 * s;
                const uint32_t stage = ring0 + (uint32_t)(s * LY::STAGE_BYTES);
                mbar_arrive_expect_tx(bar, bytes);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int cx = L::cx(i);
                    const int ys = w.y0 - L::cy(i), zs = z - L::cz(i);
                    const uint32_t dst = stage + (uint32_t)LY::box_off(i);
                    if (cx == 0)
                        tma_load_4d(dst, &maps.narrow, w.x0, ys, zs, i, bar);
                    else  // the wide box starts 8 cells left of x0 (c_x = +1) or at x0 (c_x = -1)
                        tma_load_4d(dst, &maps.wide, cx == 1 ? w.x0 - 8 : w.x0, ys, zs, i, bar);
                    // face boxes: the population a face cell pulls from outside the lattice
                    if (cx == 1 && left) {
                        const uint32_t fd = stage + LY::FACE_OFF + LY::face_rank(i) * LY::FACE_BYTES;
                        if (perx)  // wrapped: column nx - 1 (element 7 of a box at nx - 8)
                            tma_load_4d(fd, &maps.face, nx - 8, ys, zs, i, bar);
                        else       // bounce-back: the face cell's own opposite population
                            tma_load_4d(fd, &maps.face, 0, w.y0, z, L::opp(i), bar);
                    }
                    if (cx == -1 && right) {
                        const uint32_t fd =
                            stage + LY::FACE_OFF + (5 + LY::face_rank(i)) * LY::FACE_BYTES;
                        if (perx)  // wrapped: column 0 (element 0)
                            tma_load_4d(fd, &maps.face, 0, ys, zs, i, bar);
                        else       // bounce-back: element 7 of a box at nx - 8 is column nx - 1
                            tma_load_4d(fd, &maps.face, nx - 8, w.y0, z, L::opp(i), bar);
                    }
                }
            }
        }
        // wait (bounded, full default) for the copies still in flight: the last NS issued stages
        for (int g2 = max(0, g - NS); g2 < g; ++g2)
            mbar_wait_bounded(full0 + 8 * (g2 % NS), (g2 / NS) & 1, nullptr, TMA_WAIT_NS);
        return;
    }

    // ------------------------------------------------------------------------ consumer warps
    const unsigned N = (unsigned)nx * (unsigned)ny * (unsigned)nz;
    int g = 0;
    // a warp whose wait ran out (or saw the abort flag) is `dead`: it neither waits nor computes
    // any more, but keeps walking the units so that every consumer warp reaches the named barrier
    // of every unit (a warp that returned would leave the others waiting there)
    bool dead = false;
    for (int u = blockIdx.x; u < U; u += gridDim.x) {
        const TpUnit w = tp_unit(u, utx, uty);
        const int x0 = w.x0 + 2 * lane;
        const int y = w.y0 + warp;
        const bool active = x0 < nx && y < ny;
        const bool yface = y == 0 || y == ny - 1;
        const bool left_lane = w.x0 == 0 && lane == 0;
        const bool right_lane = x0 + 2 == nx;
        int kmax = 0;
        for (int dz = 0; dz < TP_TZ; ++dz, ++g) {
            const int z = w.z0 + dz;
            const int s = g % NS;
            if (!dead) {
                const int r = mbar_wait_bounded(full0 + 8 * s, (g / NS) & 1, abort_flag, wait_ns);
                if (r == 0) {
                    *abort_flag = 1;
                    if (p.err) atomicOr(p.err, 1);
                }
                // the lanes poll on their own: the warp stops as one if any of them stopped
                dead = __any_sync(0xffffffffu, r != 1);
            }
            if (dead) continue;
            const bool general = yface || z == 0 || z == nz - 1;  // warp-uniform
            const uint32_t stage = ring0 + (uint32_t)(s * LY::STAGE_BYTES);
            V raw[Q];
            if (active && !general && z < nz) {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int cx = L::cx(i);
                    const uint32_t row = stage + (uint32_t)LY::box_off(i) +
                                         (uint32_t)(warp * LY::row_elems(i) * 2);
                    if (cx == 0) {
                        raw[i] = lds32(row + 4u * lane);
                    } else if (cx == 1) {
                        // sources x0 - 1, x0: elements 2 lane + 7, 2 lane + 8 of the box at x0 - 8
                        unsigned a = lds32(row + 4u * lane + 12u);
                        const unsigned b = lds32(row + 4u * lane + 16u);
                        if (left_lane) {
                            const uint32_t fb = stage + LY::FACE_OFF +
                                                LY::face_rank(i) * LY::FACE_BYTES + warp * 16;
                            a = lds16(fb + (perx ? 14u : 0u)) << 16;
                        }
                        raw[i] = __byte_perm(a, b, 0x5432);
                    } else {
                        // sources x0 + 1, x0 + 2: elements 2 lane + 1, 2 lane + 2 of the box at x0
                        const unsigned a = lds32(row + 4u * lane);
                        unsigned b = lds32(row + 4u * lane + 4u);
                        if (right_lane) {
                            const uint32_t fb = stage + LY::FACE_OFF +
                                                (5 + LY::face_rank(i)) * LY::FACE_BYTES + warp * 16;
                            b = lds16(fb + (perx ? 0u : 14u));
                        }
                        raw[i] = __byte_perm(a, b, 0x5432);
                    }
                }
            }
            // the stage is in registers (or not needed): release it to the producer
            __syncwarp();
            if (lane == 0) mbar_arrive(empty0 + 8 * s);
            if (!active || z >= nz) continue;
            const unsigned idx0 = ((unsigned)z * ny + y) * nx + x0;
            float2 K;
            if (!general) {
                T *C = fout + idx0;
                K = relax_pair<L, DT, MODE>([&](int i) { return RG::widen_a(raw[i]); },
                                            [&](int i) { return RG::widen_b(raw[i]); }, p.omega_f,
                                            [&](int i, float2 v) { RG::store2(C + (unsigned)i * N, v); });
            } else {
                float kc[2];
#pragma unroll 1
                for (int c = 0; c < 2; ++c) {
                    float df[Q];
                    gather_cell<L, DT>(fin, p, N, x0 + c, y, z, df);
                    kc[c] = relax_store_cell<L, DT, MODE>(df, p.omega_f, fout, N, idx0 + c);
                }
                K = make_float2(kc[0], kc[1]);
            }
            if (MODE != 0) {
                kmax = max(kmax, max(__float_as_int(K.x), __float_as_int(K.y)));
                if (MODE == 2) {
                    k_field[idx0] = K.x;
                    k_field[idx0 + 1] = K.y;
                }
            }
        }
        if (MODE != 0) {
            // the unit's 8 tiles: max over the 4 lanes of a tile, then over the 8 rows
#pragma unroll
            for (int off = 2; off >= 1; off >>= 1) kmax = max(kmax, __shfl_xor_sync(~0u, kmax, off));
            const int par = (g / TP_TZ) & 1;
            int *pp = part + par * (TP_WARPS * 8);
            if ((lane & 3) == 0) pp[warp * 8 + (lane >> 2)] = kmax;
            named_barrier_sync(1, 32 * TP_WARPS);
            if (warp == 0 && lane < 8) {
                int m = pp[lane];
#pragma unroll
                for (int r2 = 1; r2 < TP_WARPS; ++r2) m = max(m, pp[r2 * 8 + lane]);
                const int tx = (w.x0 >> 3) + lane;
                if (tx < p.ntx) {
                    const size_t t =
                        ((size_t)(w.z0 >> 3) * p.nty + (size_t)(w.y0 >> 3)) * p.ntx + tx;
                    tile_max[t] = __int_as_float(m);
                }
            }
        }
    }
}

// Whether the kernel applies: D3Q19 with 16-bit storage, nx a multiple of 8 and (q + 1) * cells
// below 2^32.
inline bool tma_pair_applicable(int dtype, const StepParams &p) {
    const unsigned long long cells = (unsigned long long)p.nx * p.ny * p.nz;
    return (dtype == 2 || dtype == 3) && p.nx % 8 == 0 && 20ull * cells < (1ull << 32);
}

}  // namespace lbm
