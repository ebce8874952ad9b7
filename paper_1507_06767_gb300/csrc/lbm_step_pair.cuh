// Fused lattice Boltzmann step, two x-adjacent cells per thread, FP32 arithmetic in packed pairs.
//
// Same computation as fused_step_kernel (lbm_step.cuh): pull-stream with moving-wall bounce-back
// (Sec. 2.2 streaming, Sec. 4.1 lid), moments (Eqs. rho, u), equilibrium (Eq. feq_i), Knudsen
// sensor (Eq. sensor / kkn) with per-tile max, BGK collision (Sec. 2.2).  Differences, all for
// instruction economy (the one-cell kernel issues ~725 instructions per cell, most of them integer
// address work; with 16-bit storage it is bound by issue rate, not by HBM):
//   * each thread owns the cells (x0, x0 + 1), x0 even, so every population is loaded and stored
//     as one aligned pair (8 bytes in FP32, 4 bytes in FP16/BF16) for the directions with c_x = 0,
//     and as two scalar loads for c_x = +-1;
//   * addresses are a per-thread pointer plus a 32-bit per-direction element offset (one
//     wide multiply-add each), which needs (q + 1) * cells < 2^32 (checked by the caller);
//   * 16-bit populations stay packed in one 32-bit register per direction until they are used,
//     and are widened twice (moments, then relaxation) instead of holding 2q floats;
//   * the arithmetic of both cells runs in packed FP32 pairs (FFMA2 / FADD2 / FMUL2 of sm_100+);
//     signed sums are split into positive and negative parts, so no operand needs a negation;
//   * a warp whose cells are all at least one cell away from every wall takes a path without the
//     wall tests (warp-uniform vote), a row inside in y and z one whose x-face lanes select their
//     source address; the general path takes the two cells one after the other through the
//     one-cell kernel's gather and relaxation;
//   * the sensor uses the approximate reciprocal (relative error ~1 ulp) of the one-cell kernel's
//     approximate division.
// Needs nx even; odd nx uses the one-cell kernel.
#pragma once

#include "lbm_step.cuh"

namespace lbm {

constexpr int PAIR_CTA_CELLS_X = 2 * CTA_X;  // 64 cells along x per CTA


__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// The populations of the two cells of one direction as held in registers between the gather and
// the relaxation (PairReg<DT>::V), how they are loaded, widened to FP32 and stored.
//   FP32 storage: a float2.  FP16 / BF16 shifted storage: the two 16-bit values in one 32-bit word
//   (low half: cell x0).  widen_a and widen_b compute the same value; they are written as distinct
//   inline PTX so that the compiler keeps the packed word, not two floats, alive in between.
template <int DT>
struct PairReg;
template <>
struct PairReg<1> {
    using V = float2;
    __device__ static V load2(const float *p) { return load_pop(reinterpret_cast<const float2 *>(p)); }
    __device__ static V load_split(const float *a, const float *b) {
        return make_float2(load_pop(a), load_pop(b));
    }
    __device__ static float2 widen_a(V v) { return v; }
    __device__ static float2 widen_b(V v) { return v; }
    __device__ static void store2(float *p, float2 v) { store_pop(reinterpret_cast<float2 *>(p), v); }
};
template <>
struct PairReg<2> {
    using V = unsigned;
    __device__ static V load2(const __half *p) {
        return load_pop(reinterpret_cast<const unsigned *>(p));
    }
    __device__ static V load_split(const __half *a, const __half *b) {
        const unsigned lo = load_pop(reinterpret_cast<const unsigned short *>(a));
        const unsigned hi = load_pop(reinterpret_cast<const unsigned short *>(b));
        return __byte_perm(lo, hi, 0x5410);
    }
    __device__ static float2 widen_a(V v) {
        float a, b;
        asm("{.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;}"
            : "=f"(a), "=f"(b) : "r"(v));
        return make_float2(a, b);
    }
    __device__ static float2 widen_b(V v) {
        float a, b;
        asm("{.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %1, h;\n\tcvt.f32.f16 %0, l;}"
            : "=f"(a), "=f"(b) : "r"(v));
        return make_float2(a, b);
    }
    __device__ static void store2(__half *p, float2 v) {
        store_pop(reinterpret_cast<__half2 *>(p), __float22half2_rn(v));
    }
};
template <>
struct PairReg<3> {
    using V = unsigned;
    __device__ static V load2(const __nv_bfloat16 *p) {
        return load_pop(reinterpret_cast<const unsigned *>(p));
    }
    __device__ static V load_split(const __nv_bfloat16 *a, const __nv_bfloat16 *b) {
        const unsigned lo = load_pop(reinterpret_cast<const unsigned short *>(a));
        const unsigned hi = load_pop(reinterpret_cast<const unsigned short *>(b));
        return __byte_perm(lo, hi, 0x5410);
    }
    // a BF16 value is the high half of the FP32 value with the same bits
    __device__ static float2 widen_a(V v) {
        unsigned a, b;
        asm("shl.b32 %0, %2, 16;\n\tand.b32 %1, %2, 0xffff0000;" : "=r"(a), "=r"(b) : "r"(v));
        return make_float2(__uint_as_float(a), __uint_as_float(b));
    }
    __device__ static float2 widen_b(V v) {
        unsigned a, b;
        asm("and.b32 %1, %2, 0xffff0000;\n\tshl.b32 %0, %2, 16;" : "=r"(a), "=r"(b) : "r"(v));
        return make_float2(__uint_as_float(a), __uint_as_float(b));
    }
    __device__ static void store2(__nv_bfloat16 *p, float2 v) {
        store_pop(reinterpret_cast<__nv_bfloat162 *>(p), __float22bfloat162_rn(v));
    }
};

// Component of velocity i along axis a (0 x, 1 y, 2 z).
template <class L>
__host__ __device__ constexpr int comp(int a, int i) {
    return a == 0 ? L::cx(i) : a == 1 ? L::cy(i) : L::cz(i);
}
// First direction (lowest index) whose component along axis a equals s.
template <class L>
__host__ __device__ constexpr int first_dir(int a, int s) {
    for (int i = 1; i < L::Q; ++i)
        if (comp<L>(a, i) == s) return i;
    return -1;
}
// First axis along which velocity i has a non-zero component (-1 for the rest velocity).
template <class L>
__host__ __device__ constexpr int lead_axis(int i) {
    return L::cx(i) ? 0 : L::cy(i) ? 1 : L::cz(i) ? 2 : -1;
}

// Moments, equilibrium, Knudsen sensor and BGK collision of two cells at once in packed FP32
// pairs, from their deviations df_i = f_i - w_i: moments(i) and relax(i) return df_i (the same
// value; see PairReg).  Calls store(i, v) with the post-collision value of direction i in the
// storage convention of DT (f* for plain storage, f* - w_i for shifted storage) and returns the
// two sensors (MODE != 0).
template <class L, int DT, int MODE, class Get1, class Get2, class Store>
__device__ __forceinline__ float2 relax_pair(Get1 &&moments, Get2 &&relax, float omega_s,
                                             Store &&store) {
    using S = Storage<DT>;
    constexpr int Q = L::Q;
    // rho - 1 and the positive / negative parts of rho u along each axis
    float2 drho = moments(0);
    float2 jp[3], jn[3];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float2 v = moments(i);
        drho = __fadd2_rn(drho, v);
#pragma unroll
        for (int a = 0; a < L::D; ++a) {
            if (comp<L>(a, i) == 1) jp[a] = (i == first_dir<L>(a, 1)) ? v : __fadd2_rn(jp[a], v);
            if (comp<L>(a, i) == -1) jn[a] = (i == first_dir<L>(a, -1)) ? v : __fadd2_rn(jn[a], v);
        }
    }
    const float2 rho = __fadd2_rn(f2(1.f), drho);
    const float2 inv_rho = make_float2(__frcp_rn(rho.x), __frcp_rn(rho.y));
    float2 u[3];
#pragma unroll
    for (int a = 0; a < L::D; ++a) u[a] = __fmul2_rn(__ffma2_rn(jn[a], f2(-1.f), jp[a]), inv_rho);
    float2 usq = __fmul2_rn(u[0], u[0]);
#pragma unroll
    for (int a = 1; a < L::D; ++a) usq = __ffma2_rn(u[a], u[a], usq);
    const float2 neg_usq15 = __fmul2_rn(f2(-1.5f), usq);
    const float2 neg_omega = f2(-omega_s);

    float2 ksum = f2(0.f);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        // c.u = s g with s the sign of the first non-zero component and g = u_a + (c_a c_b) u_b,
        // shared by i and its opposite; P = c.u/cs2 + ((c.u)^2 - cs2 u.u)/(2 cs2^2)
        //   = g (3 s + 4.5 g) - 1.5 u.u
        float2 P = neg_usq15;
        if (i != 0) {
            const int a = lead_axis<L>(i);
            const int s = comp<L>(a, i);
            float2 g = u[a];
#pragma unroll
            for (int b = a + 1; b < L::D; ++b)
                if (comp<L>(b, i) != 0)
                    g = (s * comp<L>(b, i) == 1) ? __fadd2_rn(g, u[b]) : __ffma2_rn(u[b], f2(-1.f), g);
            P = __ffma2_rn(g, __ffma2_rn(f2(4.5f), g, f2(3.f * s)), neg_usq15);
        }
        const float w = weight<L, float>(i);
        const float2 d = relax(i);
        const float2 A = __ffma2_rn(rho, P, drho);  // (f^eq_i - w_i) / w_i
        const float2 fneq = __ffma2_rn(f2(-w), A, d);  // f_i - f^eq_i
        if (MODE != 0) {
            // f^eq_i = w_i rho (1 + P) = w_i (A + 1)
            const float2 feq = __ffma2_rn(f2(w), A, f2(w));
            ksum.x = fmaf(fabsf(fneq.x), rcp_approx(feq.x), ksum.x);
            ksum.y = fmaf(fabsf(fneq.y), rcp_approx(feq.y), ksum.y);
        }
        float2 v = __ffma2_rn(neg_omega, fneq, d);
        if (!S::SHIFTED) v = __fadd2_rn(v, f2(w));
        store(i, v);
    }
    return __fmul2_rn(ksum, f2(1.f / (float)Q));
}

template <class L, int DT, int MODE>
__global__ void __launch_bounds__(CTA_X *CTA_Y, DT == 1 ? LBM_PAIR_MIN_BLOCKS_F32 : LBM_PAIR_MIN_BLOCKS)
    fused_step_pair_kernel(const typename Storage<DT>::T *__restrict__ fin,
                           typename Storage<DT>::T *__restrict__ fout, const StepParams p,
                           float *__restrict__ tile_max, float *__restrict__ k_field) {
    using S = Storage<DT>;
    using T = typename S::T;
    using RG = PairReg<DT>;
    using V = typename RG::V;
    constexpr int Q = L::Q;
    constexpr int ZT = (L::D == 3) ? TILE : 1;

    const int lane = threadIdx.x;
    const int x0 = (blockIdx.x * CTA_X + lane) * 2;
    const int y = blockIdx.y * CTA_Y + threadIdx.y;
    const int z0 = blockIdx.z * ZT;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const bool active = (x0 < nx) && (y < ny);
    // element offsets fit in 32 bits: (q + 1) * cells < 2^32
    const unsigned N = (unsigned)nx * (unsigned)ny * (unsigned)nz;
    const unsigned nxy = (unsigned)nx * (unsigned)ny;

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
        // y and z are warp-uniform (a warp is one row); x0 is not
        const bool inner_yz = (y > 0) && (y < ny - 1) && (L::D == 2 || ((z > 0) && (z < nz - 1)));
        const bool interior = inner_yz && (x0 > 0) && (x0 + 2 < nx);
        const bool fast = __all_sync(0xffffffffu, !active || interior);
        if (!active) continue;
        const unsigned idx0 = ((unsigned)z * ny + y) * nx + x0;
        const T *B = fin + idx0;
        T *C = fout + idx0;
        const auto store = [&](int i, float2 v) { RG::store2(C + (unsigned)i * N, v); };

        float2 K;
        if (fast || (LBM_XSEL_PATH && inner_yz)) {
            // rows inside in y and z: only a pull along x can leave the lattice, at x0 = 0 (cell
            // x0 along +x) or x0 + 2 = nx (cell x0 + 1 along -x); there the source address is
            // selected: the wrapped cell on a periodic x axis, else the cell's own opposite
            // population (bounce-back at a resting wall)
            V raw[Q];
            if (fast) {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int cx = L::cx(i);
                    const T *src = B + ((unsigned)i * N - (unsigned)(L::cz(i) * (int)nxy +
                                                                     L::cy(i) * nx));
                    raw[i] = cx == 0 ? RG::load2(src)
                                     : RG::load_split(src - cx, src + 1 - cx);
                }
            } else {
                const bool lo_face = x0 == 0, hi_face = x0 + 2 == nx;
                const bool perx = p.periodic & 1;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int cx = L::cx(i);
                    const T *src = B + ((unsigned)i * N - (unsigned)(L::cz(i) * (int)nxy +
                                                                     L::cy(i) * nx));
                    if (cx == 0) {
                        raw[i] = RG::load2(src);
                    } else if (cx == 1) {
                        const T *a = src - 1;
                        const T *alt = perx ? a + nx : B + (unsigned)L::opp(i) * N;
                        raw[i] = RG::load_split(lo_face ? alt : a, src);
                    } else {
                        const T *b = src + 2;
                        const T *alt = perx ? b - nx : B + ((unsigned)L::opp(i) * N + 1u);
                        raw[i] = RG::load_split(src + 1, hi_face ? alt : b);
                    }
                }
            }
            if constexpr (!S::SHIFTED) {
                // plain storage holds f_i: the relaxation works on f_i - w_i
#pragma unroll
                for (int i = 0; i < Q; ++i) raw[i] = __fadd2_rn(raw[i], f2(-weight<L, float>(i)));
            }
            K = relax_pair<L, DT, MODE>([&](int i) { return RG::widen_a(raw[i]); },
                                        [&](int i) { return RG::widen_b(raw[i]); }, p.omega_f,
                                        store);
        } else {
            // one cell after the other, with the one-cell kernel's gather and relaxation (fewer
            // live registers than a pair of gathered cells)
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

// The two-cell kernel applies to an even nx and (q + 1) * cells < 2^32 (32-bit element offsets).
template <class L>
inline bool pair_applicable(const StepParams &p) {
    const unsigned long long cells = (unsigned long long)p.nx * p.ny * p.nz;
    return p.nx % 2 == 0 && (unsigned long long)(L::Q + 1) * cells < (1ULL << 32);
}

template <class L, int DT>
cudaError_t launch_fused_step_pair(const void *fin, void *fout, const StepParams &p, int mode,
                                   void *tile_max, void *k_field, cudaStream_t stream) {
    using T = typename Storage<DT>::T;
    if (!pair_applicable<L>(p)) return cudaErrorInvalidValue;
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
