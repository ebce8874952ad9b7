// Fused lattice Boltzmann step: pull-stream + moving-wall bounce-back + moments + equilibrium +
// Knudsen sensor + per-tile sensor max + BGK collision, one pass over HBM.
//
// Paper (arXiv 1507.06767): streaming and collision of Sec. 2.2 (Eq. bgklb, collide-and-stream
// split), equilibrium Eq. (feq_i), moments Eqs. (rho), (u), sensor Eq. (sensor) / (kkn) of
// Sec. 3.2-3.3, moving bounce-back of Sec. 4.1.
//
// Thread mapping: a CTA of 32 x 8 threads covers 32 cells along x and 8 rows along y; in 3-D it
// walks 8 planes along z.  A CTA therefore owns whole 8^d base tiles (4 of them), so the tile maxima
// are written with plain stores: no atomics, no zeroing pass.  Each thread issues its q gathers
// before any arithmetic, so a warp keeps q independent coalesced loads in flight.
//
// Arithmetic is done on deviations from the rest state, df_i = f_i - w_i: rho - 1 = sum df_i and
// rho u = sum c_i df_i lose no digits to the large w_i, and f^neq = df_i - (f^eq_i - w_i) is formed
// without cancelling against w_i.
#pragma once

#include "lbm_traits.cuh"

namespace lbm {

constexpr int CTA_X = 32;
constexpr int CTA_Y = 8;
constexpr int TILE = 8;

// Tuning knobs (compile-time): resident CTAs per SM requested from the register allocator (one-cell
// kernel: 4 -> at most 64 registers, 1024 threads per SM; the two-cell kernel with 16-bit storage:
// 4, no spills, measured at 512^3 FP16 1.91 ms against 2.00 ms with 3; with FP32 storage: 3 -> at
// most 80 registers, no spills, 3.03 ms against 3.15 ms with 4), and cache hints of the population
// loads / stores (0: default, 1: read-only path / streaming store, 2: evict-first load, 3:
// read-only path asking L2 for the 256-byte group around each address: 512^3 FP16 two-cell 1.912
// -> 1.887 ms, FP32 one-cell 3.109 -> 3.074 ms, FP32 two-cell unchanged).  Measured on GB300 at
// 256^3 D3Q19 FP32: without a minimum the allocator takes 140 registers and the one-cell kernel
// runs at half speed.
#ifndef LBM_STEP_MIN_BLOCKS
#define LBM_STEP_MIN_BLOCKS 4
#endif
#ifndef LBM_PAIR_MIN_BLOCKS
#define LBM_PAIR_MIN_BLOCKS 4
#endif
#ifndef LBM_PAIR_MIN_BLOCKS_F32
#define LBM_PAIR_MIN_BLOCKS_F32 3
#endif
#ifndef LBM_LOAD_HINT
#define LBM_LOAD_HINT 3
#endif
#ifndef LBM_STORE_HINT
#define LBM_STORE_HINT 0
#endif
// 1: CTAs whose cells and all their pull sources lie inside the lattice take a gather without
// wall or wrap logic (one address offset per direction)
#ifndef LBM_INTERIOR_FAST
#define LBM_INTERIOR_FAST 1
#endif
// 1: rows inside in y and z but at an x face take gather_xsel (address selects, no branches)
#ifndef LBM_XSEL_PATH
#define LBM_XSEL_PATH 1
#endif

template <class T>
__device__ __forceinline__ T load_pop(const T *p) {
#if LBM_LOAD_HINT == 1 || LBM_LOAD_HINT == 3
    return __ldg(p);
#elif LBM_LOAD_HINT == 2
    return __ldcs(p);
#else
    return *p;
#endif
}

#if LBM_LOAD_HINT == 3
// read-only loads that also ask L2 to fetch the whole 256-byte sector group around the address
template <>
__device__ __forceinline__ float load_pop<float>(const float *p) {
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
template <>
__device__ __forceinline__ float2 load_pop<float2>(const float2 *p) {
    float2 v;
    asm("ld.global.nc.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
template <>
__device__ __forceinline__ unsigned load_pop<unsigned>(const unsigned *p) {
    unsigned v;
    asm("ld.global.nc.L2::256B.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
template <>
__device__ __forceinline__ unsigned short load_pop<unsigned short>(const unsigned short *p) {
    unsigned short v;
    asm("ld.global.nc.L2::256B.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}
#endif

template <class T>
__device__ __forceinline__ void store_pop(T *p, T v) {
#if LBM_STORE_HINT == 1
    __stcs(p, v);
#else
    *p = v;
#endif
}

// Pull-gather of cell (x, y, z) in the general case (walls with moving-lid bounce-back, periodic
// wrap): writes the deviations from rest df_i = f_i - w_i of the populations arriving at the cell
// to df[i * STRIDE] (STRIDE 2 fills one lane of an array of pairs).  HALO: the faces of the slowest
// axis (z in 3-D, y in 2-D) may be cuts of a slab (StepParams::halo_lo / halo_hi); a source beyond
// such a face and inside the lattice along the other axes (or wrapped) is the neighbouring slab's
// cell, whose population i sits in the halo plane.  A source outside along another axis stays a
// wall ghost, and a 2-D slab whose high y face is a cut has no lid there.  The kernels without
// halos are instantiated with HALO = false and do not carry this code.
template <class L, int DT, int STRIDE = 1, bool HALO = false>
__device__ __forceinline__ void gather_cell(const typename Storage<DT>::T *__restrict__ fin,
                                            const StepParams &p, size_t N, int x, int y, int z,
                                            typename Storage<DT>::R *df) {
    using S = Storage<DT>;
    using R = typename S::R;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const bool perx = p.periodic & 1, pery = p.periodic & 2, perz = p.periodic & 4;
    // source coordinates x - c for c = +1 (xm) and c = -1 (xp), with their validity
    const int xm = (x == 0) ? nx - 1 : x - 1;
    const int xp = (x == nx - 1) ? 0 : x + 1;
    const bool vxm = (x > 0) || perx;
    const bool vxp = (x < nx - 1) || perx;
    const int ym = (y == 0) ? ny - 1 : y - 1;
    const int yp = (y == ny - 1) ? 0 : y + 1;
    const bool vym = (y > 0) || pery;
    const bool vyp = (y < ny - 1) || pery;  // false <=> the y+1 ghost is the lid
    int zm = z, zp = z;
    bool vzm = true, vzp = true;
    if (L::D == 3) {
        zm = (z == 0) ? nz - 1 : z - 1;
        zp = (z == nz - 1) ? 0 : z + 1;
        vzm = (z > 0) || perz;
        vzp = (z < nz - 1) || perz;
    }
    const int idx = (z * ny + y) * nx + x;
    const R lidx = param_lid_x<R>(p), lidz = param_lid_z<R>(p);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const int sx = cx == 1 ? xm : (cx == -1 ? xp : x);
        const int sy = cy == 1 ? ym : (cy == -1 ? yp : y);
        const int sz = cz == 1 ? zm : (cz == -1 ? zp : z);
        const bool valid = (cx == 1 ? vxm : (cx == -1 ? vxp : true)) &&
                           (cy == 1 ? vym : (cy == -1 ? vyp : true)) &&
                           (cz == 1 ? vzm : (cz == -1 ? vzp : true));
        size_t src = valid ? (size_t)i * N + (size_t)((sz * ny + sy) * nx + sx)
                           : (size_t)L::opp(i) * N + (size_t)idx;
        const typename S::T *from = fin;
        bool lid = cy == -1 && !vyp;
        if constexpr (HALO) {
            const bool okx = cx == 1 ? vxm : (cx == -1 ? vxp : true);
            const bool oky = cy == 1 ? vym : (cy == -1 ? vyp : true);
            const bool okz = cz == 1 ? vzm : (cz == -1 ? vzp : true);
            const int cs = (L::D == 3) ? cz : cy;  // component along the slab axis
            const bool beyond = (L::D == 3) ? (cz != 0 && !okz && okx && oky)
                                            : (cy != 0 && !oky && okx);
            const void *hv = cs == 1 ? p.halo_lo : (cs == -1 ? p.halo_hi : nullptr);
            if (beyond && hv != nullptr) {
                from = static_cast<const typename S::T *>(hv);
                src = (L::D == 3) ? (size_t)i * ((size_t)nx * ny) + (size_t)(sy * nx + sx)
                                  : (size_t)i * nx + (size_t)sx;
            }
            if (L::D == 2 && p.halo_hi != nullptr) lid = false;
        }
        R v = S::to_r(load_pop(from + src));
        if (!S::SHIFTED) v -= weight<L, R>(i);  // w_opp(i) == w_i
        if (lid) {
            // moving lid: + 2 w_i (c_i . u_lid) / c_s^2, wall density 1
            v += R(6) * weight<L, R>(i) * (R(cx) * lidx + R(cz) * lidz);
        }
        df[i * STRIDE] = v;
    }
}

// Pull-gather of a cell whose q sources all lie inside the lattice (no wall, no wrap): population i
// comes from idx - (c_z plane + c_y nx + c_x) of population i's array.
template <class L, int DT>
__device__ __forceinline__ void gather_interior(const typename Storage<DT>::T *__restrict__ fin,
                                                size_t N, int nx, int plane, size_t idx,
                                                typename Storage<DT>::R *df) {
    using S = Storage<DT>;
    using R = typename S::R;
    const typename S::T *base = fin + idx;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const long long off =
            (long long)i * (long long)N - (long long)(L::cz(i) * plane + L::cy(i) * nx + L::cx(i));
        R v = S::to_r(load_pop(base + off));
        if (!S::SHIFTED) v -= weight<L, R>(i);
        df[i] = v;
    }
}

// Pull-gather of a cell whose y and z sources lie inside the lattice: as gather_interior, except
// that a pull along x that leaves the lattice (x = 0 pulling along +x, x = nx - 1 along -x)
// selects its address instead of branching: the wrapped cell on a periodic x axis, else the
// cell's own opposite population (bounce-back at a resting wall; the lid is a y wall).
template <class L, int DT>
__device__ __forceinline__ void gather_xsel(const typename Storage<DT>::T *__restrict__ fin,
                                            size_t N, int nx, int plane, size_t idx, int x,
                                            bool perx, typename Storage<DT>::R *df) {
    using S = Storage<DT>;
    using R = typename S::R;
    const typename S::T *base = fin + idx;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int cx = L::cx(i);
        const long long off =
            (long long)i * (long long)N - (long long)(L::cz(i) * plane + L::cy(i) * nx + cx);
        const typename S::T *src = base + off;
        if (cx != 0) {
            const bool face = cx == 1 ? x == 0 : x == nx - 1;
            const typename S::T *alt = perx ? src + cx * nx : fin + (size_t)L::opp(i) * N + idx;
            src = face ? alt : src;
        }
        R v = S::to_r(load_pop(src));
        if (!S::SHIFTED) v -= weight<L, R>(i);
        df[i] = v;
    }
}

// Approximate FP32 reciprocal (PTX rcp.approx, max relative error about 1 ulp; inputs here are
// equilibrium populations, far from zero and from the subnormal range).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Moments, equilibrium, sensor and BGK collision of one cell from its gathered deviations df;
// emit(i, d) receives the post-collision deviation d = f*_i - w_i of every population.  Returns
// the sensor K (MODE != 0).
template <class L, int DT, int MODE, class Emit>
__device__ __forceinline__ typename Storage<DT>::R relax_cell(const typename Storage<DT>::R *df,
                                                              typename Storage<DT>::R omega,
                                                              Emit &&emit) {
    using S = Storage<DT>;
    using R = typename S::R;
    constexpr int Q = L::Q;
    // moments as deviations from rest
    R drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += df[i];
        if (L::cx(i)) jx += R(L::cx(i)) * df[i];
        if (L::cy(i)) jy += R(L::cy(i)) * df[i];
        if (L::cz(i)) jz += R(L::cz(i)) * df[i];
    }
    const R rho = R(1) + drho;
    const R inv_rho = R(1) / rho;
    const R ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
    const R usq15 = R(1.5) * (ux * ux + uy * uy + uz * uz);

    R ksum = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R cu = R(L::cx(i)) * ux + R(L::cy(i)) * uy + R(L::cz(i)) * uz;
        // P_i = c.u / cs2 + ((c.u)^2 - cs2 u.u) / (2 cs2^2)
        const R P = R(3) * cu + R(4.5) * cu * cu - usq15;
        const R w = weight<L, R>(i);
        const R dfeq = w * (drho + rho * P);  // f^eq_i - w_i
        const R fneq = df[i] - dfeq;
        if (MODE != 0) {
            if constexpr (sizeof(R) == 4) {
                // f^eq_i = (f^eq_i - w_i) + w_i: one add, one reciprocal, one fused multiply-add
                ksum = fmaf(fabsf(fneq), rcp_approx(dfeq + w), ksum);
            } else {
                const R feq = w * rho * (R(1) + P);
                ksum += fabs(fneq) / feq;
            }
        }
        emit(i, df[i] - omega * fneq);
    }
    return ksum * (R(1) / R(Q));
}

// relax_cell with the store of the post-collision populations at linear index idx.
template <class L, int DT, int MODE>
__device__ __forceinline__ typename Storage<DT>::R relax_store_cell(
    const typename Storage<DT>::R *df, typename Storage<DT>::R omega,
    typename Storage<DT>::T *__restrict__ fout, size_t N, int idx) {
    using S = Storage<DT>;
    using R = typename S::R;
    return relax_cell<L, DT, MODE>(df, omega, [&](int i, R dnew) {
        store_pop(fout + (size_t)i * N + idx,
                  S::from_r(S::SHIFTED ? dnew : dnew + weight<L, R>(i)));
    });
}

// MODE 0: no sensor.  MODE 1: sensor and per-tile max.  MODE 2: MODE 1 plus per-cell K.  HALO:
// the faces of the slowest axis may be cuts of a slab (gather_cell).
template <class L, int DT, int MODE, bool HALO = false>
__global__ void __launch_bounds__(CTA_X *CTA_Y, LBM_STEP_MIN_BLOCKS)
    fused_step_kernel(const typename Storage<DT>::T *__restrict__ fin,
                      typename Storage<DT>::T *__restrict__ fout, const StepParams p,
                      typename Storage<DT>::R *__restrict__ tile_max,
                      typename Storage<DT>::R *__restrict__ k_field) {
    using S = Storage<DT>;
    using R = typename S::R;
    using B = typename Bits<R>::type;
    constexpr int Q = L::Q;
    constexpr int ZT = (L::D == 3) ? TILE : 1;

    const int lane = threadIdx.x;
    const int x = blockIdx.x * CTA_X + lane;
    const int y = blockIdx.y * CTA_Y + threadIdx.y;
    const int z0 = blockIdx.z * ZT;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const bool active = (x < nx) && (y < ny);
    const size_t N = (size_t)nx * ny * nz;
    const R omega = param_omega<R>(p);

    // clear the other tile buffer for the next sensor step (kernels that combine tiles across
    // CTAs with atomics need it zeroed)
    if (MODE != 0 && p.tile_zero) {
        const size_t nt = (size_t)p.ntx * p.nty * p.ntz;
        const size_t nthreads = (size_t)gridDim.x * gridDim.y * gridDim.z * blockDim.x * blockDim.y;
        const size_t me = (((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) *
                              (blockDim.x * blockDim.y) +
                          threadIdx.y * blockDim.x + threadIdx.x;
        for (size_t k = me; k < nt; k += nthreads) static_cast<R *>(p.tile_zero)[k] = R(0);
    }

    B kmax = 0;
    // a warp is one row of 32 cells: when the row and all its pull sources lie inside the lattice
    // (a warp-uniform test) the gather needs no wall or wrap logic
    const bool inner_x = blockIdx.x * CTA_X >= 1 && (blockIdx.x + 1) * CTA_X <= nx - 1;
    const bool inner_y = y >= 1 && y <= ny - 2;

    for (int dz = 0; dz < ZT; ++dz) {
        const int z = z0 + dz;
        if (z >= nz) break;
        if (active) {
            const int idx = (z * ny + y) * nx + x;
            R df[Q];
            const bool inner_yz = inner_y && (L::D == 2 || (z >= 1 && z <= nz - 2));
            if (LBM_INTERIOR_FAST && inner_yz && inner_x)
                gather_interior<L, DT>(fin, N, nx, nx * ny, (size_t)idx, df);
            else if (LBM_XSEL_PATH && inner_yz)
                gather_xsel<L, DT>(fin, N, nx, nx * ny, (size_t)idx, x, p.periodic & 1, df);
            else
                gather_cell<L, DT, 1, HALO>(fin, p, N, x, y, z, df);
            const R K = relax_store_cell<L, DT, MODE>(df, omega, fout, N, idx);
            if (MODE != 0) {
                const B kb = max_bits(K);
                kmax = kb > kmax ? kb : kmax;
                if (MODE == 2) k_field[idx] = K;
            }
        }
    }

    if (MODE != 0) {
        // max over the 8 lanes of each x-tile of this row, then over the 8 rows via shared memory
#pragma unroll
        for (int off = 4; off >= 1; off >>= 1) {
            const B o = __shfl_xor_sync(0xffffffffu, kmax, off);
            kmax = o > kmax ? o : kmax;
        }
        __shared__ B part[CTA_Y][CTA_X / TILE];
        if ((lane & (TILE - 1)) == 0) part[threadIdx.y][lane / TILE] = kmax;
        __syncthreads();
        if (threadIdx.y == 0 && lane < CTA_X / TILE) {
            B m = part[0][lane];
#pragma unroll
            for (int r = 1; r < CTA_Y; ++r) m = part[r][lane] > m ? part[r][lane] : m;
            const int tx = blockIdx.x * (CTA_X / TILE) + lane;
            if (tx < p.ntx) {
                const size_t t = ((size_t)blockIdx.z * p.nty + blockIdx.y) * p.ntx + tx;
                tile_max[t] = from_bits(m, R(0));
            }
        }
    }
}

template <class L, int DT, bool HALO = false>
cudaError_t launch_fused_step(const void *fin, void *fout, const StepParams &p, int mode,
                              void *tile_max, void *k_field, cudaStream_t stream) {
    using T = typename Storage<DT>::T;
    using R = typename Storage<DT>::R;
    const int zt = (L::D == 3) ? TILE : 1;
    dim3 block(CTA_X, CTA_Y, 1);
    dim3 grid((p.nx + CTA_X - 1) / CTA_X, (p.ny + CTA_Y - 1) / CTA_Y, (p.nz + zt - 1) / zt);
    const T *a = static_cast<const T *>(fin);
    T *b = static_cast<T *>(fout);
    R *tm = static_cast<R *>(tile_max);
    R *kf = static_cast<R *>(k_field);
    if (mode == 0)
        fused_step_kernel<L, DT, 0, HALO><<<grid, block, 0, stream>>>(a, b, p, tm, kf);
    else if (mode == 1)
        fused_step_kernel<L, DT, 1, HALO><<<grid, block, 0, stream>>>(a, b, p, tm, kf);
    else
        fused_step_kernel<L, DT, 2, HALO><<<grid, block, 0, stream>>>(a, b, p, tm, kf);
    return cudaGetLastError();
}

// A slab with halo faces (StepParams::halo_lo / halo_hi) runs the one-cell kernel with the halo
// gather; the other kernels do not take halos.
inline bool has_halo(const StepParams &p) { return p.halo_lo != nullptr || p.halo_hi != nullptr; }

}  // namespace lbm
