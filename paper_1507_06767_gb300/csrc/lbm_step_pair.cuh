// Fused lattice Boltzmann step, two x-adjacent cells per thread, FP32 arithmetic in packed pairs.
//
// Same computation as fused_step_kernel (lbm_step.cuh): pull-stream with moving-wall bounce-back
// (Sec. 2.2 streaming, Sec. 4.1 lid), moments (Eqs. rho, u), equilibrium (Eq. feq_i), Knudsen
// sensor (Eq. sensor / kkn) with per-tile max, BGK collision (Sec. 2.2).  Differences, all for
// instruction economy (the one-cell kernel issues ~800 instructions per cell and is bound by issue
// rate, not by HBM):
//   * each thread owns the cells (x0, x0 + 1), x0 even, so every population is loaded and stored
//     as one aligned pair (8 bytes in FP32, 4 bytes in FP16/BF16) for the directions with c_x = 0,
//     and as two scalar loads for c_x = +-1; the address arithmetic is shared by the two cells;
//   * the arithmetic of both cells runs in packed FP32 pairs (FFMA2 / FADD2 / FMUL2 of sm_100+);
//   * a warp whose cells are all at least one cell away from every wall takes a path without the
//     wall tests (warp-uniform vote); the general path is the per-cell one of the scalar kernel.
// Needs nx even; odd nx uses the one-cell kernel.
#pragma once

#include "lbm_step.cuh"

namespace lbm {

constexpr int PAIR_CTA_CELLS_X = 2 * CTA_X;  // 64 cells along x per CTA

template <int DT>
struct PairIO;
template <>
struct PairIO<1> {  // float pair
    __device__ static float2 load2(const float *p) {
        return load_pop(reinterpret_cast<const float2 *>(p));
    }
    __device__ static void store2(float *p, float2 v) { store_pop(reinterpret_cast<float2 *>(p), v); }
};
template <>
struct PairIO<2> {  // half pair, shifted storage
    __device__ static float2 load2(const __half *p) {
        return __half22float2(load_pop(reinterpret_cast<const __half2 *>(p)));
    }
    __device__ static void store2(__half *p, float2 v) {
        store_pop(reinterpret_cast<__half2 *>(p), __float22half2_rn(v));
    }
};
template <>
struct PairIO<3> {  // bfloat16 pair, shifted storage
    __device__ static float2 load2(const __nv_bfloat16 *p) {
        return __bfloat1622float2(load_pop(reinterpret_cast<const __nv_bfloat162 *>(p)));
    }
    __device__ static void store2(__nv_bfloat16 *p, float2 v) {
        store_pop(reinterpret_cast<__nv_bfloat162 *>(p), __float22bfloat162_rn(v));
    }
};

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// Moments, equilibrium, Knudsen sensor and BGK collision of two cells at once in packed FP32
// pairs (FFMA2 / FADD2 / FMUL2 of sm_100+), from their gathered deviations df_i = f_i - w_i.
// Calls store(i, v) with the post-collision value of direction i in the storage convention of DT
// (f* for plain storage, f* - w_i for shifted storage) and returns the two sensors (MODE != 0).
template <class L, int DT, int MODE, class Store>
__device__ __forceinline__ float2 relax_pair(const float2 *df, float omega_s, Store &&store) {
    using S = Storage<DT>;
    constexpr int Q = L::Q;
    const float2 one = f2(1.f);
    float2 drho = df[0], jx = f2(0.f), jy = f2(0.f), jz = f2(0.f);
#pragma unroll
    for (int i = 1; i < Q; ++i) drho = __fadd2_rn(drho, df[i]);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (L::cx(i) == 1) jx = __fadd2_rn(jx, df[i]);
        if (L::cx(i) == -1) jx = __fadd2_rn(jx, make_float2(-df[i].x, -df[i].y));
        if (L::cy(i) == 1) jy = __fadd2_rn(jy, df[i]);
        if (L::cy(i) == -1) jy = __fadd2_rn(jy, make_float2(-df[i].x, -df[i].y));
        if (L::cz(i) == 1) jz = __fadd2_rn(jz, df[i]);
        if (L::cz(i) == -1) jz = __fadd2_rn(jz, make_float2(-df[i].x, -df[i].y));
    }
    const float2 rho = __fadd2_rn(one, drho);
    const float2 inv_rho = make_float2(__frcp_rn(rho.x), __frcp_rn(rho.y));
    const float2 ux = __fmul2_rn(jx, inv_rho), uy = __fmul2_rn(jy, inv_rho),
                 uz = __fmul2_rn(jz, inv_rho);
    float2 usq = __fmul2_rn(ux, ux);
    usq = __ffma2_rn(uy, uy, usq);
    if (L::D == 3) usq = __ffma2_rn(uz, uz, usq);
    const float2 neg_usq15 = __fmul2_rn(f2(-1.5f), usq);
    const float2 neg_omega = f2(-omega_s);

    float2 ksum = f2(0.f);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        // c.u with the constant components folded
        float2 cu = f2(0.f);
        if (cx == 1) cu = ux;
        if (cx == -1) cu = make_float2(-ux.x, -ux.y);
        if (cy != 0) cu = (cx == 0) ? (cy == 1 ? uy : make_float2(-uy.x, -uy.y))
                                    : __ffma2_rn(f2((float)cy), uy, cu);
        if (cz != 0) cu = (cx == 0 && cy == 0) ? (cz == 1 ? uz : make_float2(-uz.x, -uz.y))
                                               : __ffma2_rn(f2((float)cz), uz, cu);
        // P = c.u/cs2 + ((c.u)^2 - cs2 u.u)/(2 cs2^2) = cu (3 + 4.5 cu) - 1.5 u.u
        const float2 t = __ffma2_rn(f2(4.5f), cu, f2(3.f));
        const float2 P = __ffma2_rn(cu, t, neg_usq15);
        const float w = weight<L, float>(i);
        const float2 A = __ffma2_rn(rho, P, drho);       // (f^eq_i - w_i) / w_i
        const float2 fneq = __ffma2_rn(f2(-w), A, df[i]);  // f_i - f^eq_i
        if (MODE != 0) {
            const float2 feqw = __ffma2_rn(rho, P, rho);   // f^eq_i / w_i
            const float2 r = make_float2(fabsf(fneq.x) * __frcp_rn(feqw.x),
                                         fabsf(fneq.y) * __frcp_rn(feqw.y));
            ksum = __ffma2_rn(r, f2(1.f / w), ksum);
        }
        float2 v = __ffma2_rn(neg_omega, fneq, df[i]);
        if (!S::SHIFTED) v = __fadd2_rn(v, f2(w));
        store(i, v);
    }
    return __fmul2_rn(ksum, f2(1.f / (float)Q));
}

template <class L, int DT, int MODE>
__global__ void __launch_bounds__(CTA_X *CTA_Y, LBM_PAIR_MIN_BLOCKS)
    fused_step_pair_kernel(const typename Storage<DT>::T *__restrict__ fin,
                           typename Storage<DT>::T *__restrict__ fout, const StepParams p,
                           float *__restrict__ tile_max, float *__restrict__ k_field) {
    using S = Storage<DT>;
    using T = typename S::T;
    constexpr int Q = L::Q;
    constexpr int ZT = (L::D == 3) ? TILE : 1;

    const int lane = threadIdx.x;
    const int x0 = (blockIdx.x * CTA_X + lane) * 2;
    const int y = blockIdx.y * CTA_Y + threadIdx.y;
    const int z0 = blockIdx.z * ZT;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const bool active = (x0 < nx) && (y < ny);
    const size_t N = (size_t)nx * ny * nz;
    const size_t nxy = (size_t)nx * ny;

    int kmax = 0;

    if (MODE != 0 && p.tile_zero) {
        const size_t nt = (size_t)p.ntx * p.nty * p.ntz;
        const size_t nthreads = (size_t)gridDim.x * gridDim.y * gridDim.z * blockDim.x * blockDim.y;
        const size_t me = (((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) *
                              (blockDim.x * blockDim.y) +
                          threadIdx.y * blockDim.x + threadIdx.x;
        for (size_t k = me; k < nt; k += nthreads) static_cast<float *>(p.tile_zero)[k] = 0.f;
    }

    for (int dz = 0; dz < ZT; ++dz) {
        const int z = z0 + dz;
        if (z >= nz) break;
        const bool interior = (x0 > 0) && (x0 + 2 < nx) && (y > 0) && (y < ny - 1) &&
                              (L::D == 2 || ((z > 0) && (z < nz - 1)));
        const bool fast = __all_sync(0xffffffffu, !active || interior);
        if (!active) continue;
        const int idx0 = (z * ny + y) * nx + x0;

        float2 df[Q];
        if (fast) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
                const T *base = fin + (size_t)i * N + (size_t)idx0 -
                                (ptrdiff_t)((ptrdiff_t)cz * (ptrdiff_t)nxy + (ptrdiff_t)cy * nx);
                float2 v;
                if (cx == 0) {
                    v = PairIO<DT>::load2(base);
                } else if (cx == 1) {
                    v = make_float2(S::to_r(load_pop(base - 1)), S::to_r(load_pop(base)));
                } else {
                    v = make_float2(S::to_r(load_pop(base + 1)), S::to_r(load_pop(base + 2)));
                }
                if (!S::SHIFTED) v = __fadd2_rn(v, f2(-weight<L, float>(i)));
                df[i] = v;
            }
        } else {
            // each cell of the pair straight into its lane of df (no staging array)
            gather_cell<L, DT, 2>(fin, p, N, x0, y, z, reinterpret_cast<float *>(df));
            gather_cell<L, DT, 2>(fin, p, N, x0 + 1, y, z, reinterpret_cast<float *>(df) + 1);
        }

        T *out0 = fout + idx0;
        const float2 K = relax_pair<L, DT, MODE>(df, p.omega_f, [&](int i, float2 v) {
            PairIO<DT>::store2(out0 + (size_t)i * N, v);
        });
        if (MODE != 0) {
            const int kb = max(__float_as_int(K.x), __float_as_int(K.y));
            kmax = kb > kmax ? kb : kmax;
            if (MODE == 2) {
                k_field[idx0] = K.x;
                k_field[idx0 + 1] = K.y;
            }
        }
    }

    if (MODE != 0) {
        // a warp row covers 64 cells = 8 tiles of 8 cells = 4 lanes per tile
#pragma unroll
        for (int off = 2; off >= 1; off >>= 1) {
            const int o = __shfl_xor_sync(0xffffffffu, kmax, off);
            kmax = o > kmax ? o : kmax;
        }
        constexpr int TPR = PAIR_CTA_CELLS_X / TILE;  // tiles per row of the CTA
        __shared__ int part[CTA_Y][TPR];
        if ((lane & 3) == 0) part[threadIdx.y][lane >> 2] = kmax;
        __syncthreads();
        if (threadIdx.y == 0 && lane < TPR) {
            int m = part[0][lane];
#pragma unroll
            for (int r = 1; r < CTA_Y; ++r) m = part[r][lane] > m ? part[r][lane] : m;
            const int tx = blockIdx.x * TPR + lane;
            if (tx < p.ntx) {
                const size_t t = ((size_t)blockIdx.z * p.nty + blockIdx.y) * p.ntx + tx;
                tile_max[t] = __int_as_float(m);
            }
        }
    }
}

template <class L, int DT>
cudaError_t launch_fused_step_pair(const void *fin, void *fout, const StepParams &p, int mode,
                                   void *tile_max, void *k_field, cudaStream_t stream) {
    using T = typename Storage<DT>::T;
    const int zt = (L::D == 3) ? TILE : 1;
    dim3 block(CTA_X, CTA_Y, 1);
    dim3 grid((p.nx + PAIR_CTA_CELLS_X - 1) / PAIR_CTA_CELLS_X, (p.ny + CTA_Y - 1) / CTA_Y,
              (p.nz + zt - 1) / zt);
    const T *a = static_cast<const T *>(fin);
    T *b = static_cast<T *>(fout);
    float *tm = static_cast<float *>(tile_max);
    float *kf = static_cast<float *>(k_field);
    if (mode == 0)
        fused_step_pair_kernel<L, DT, 0><<<grid, block, 0, stream>>>(a, b, p, tm, kf);
    else if (mode == 1)
        fused_step_pair_kernel<L, DT, 1><<<grid, block, 0, stream>>>(a, b, p, tm, kf);
    else
        fused_step_pair_kernel<L, DT, 2><<<grid, block, 0, stream>>>(a, b, p, tm, kf);
    return cudaGetLastError();
}

}  // namespace lbm
