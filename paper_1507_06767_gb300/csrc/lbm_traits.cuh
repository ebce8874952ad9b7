// Lattice and storage traits shared by the CUDA kernels of the library.
//
// Velocity sets (Sec. 2.2 of the paper uses D2Q9; D3Q19 is the 3-D instance of the same BGK model).
// The direction order is this library's own: rest, axis directions, then diagonals, with the
// opposite of each direction tabulated.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

struct D2Q9 {
    static constexpr int Q = 9;
    static constexpr int D = 2;
    // the tables are returned by constexpr functions so that device code can index them; in the
    // kernels every index is a compile-time constant after unrolling
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) {
        constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
        return t[i];
    }
    // weights as exact rationals num / 36
    __host__ __device__ static constexpr int w36(int i) {
        constexpr int t[9] = {16, 4, 4, 4, 4, 1, 1, 1, 1};
        return t[i];
    }
};

struct D3Q19 {
    static constexpr int Q = 19;
    static constexpr int D = 3;
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i) {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int opp(int i) {
        constexpr int t[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
        return t[i];
    }
    __host__ __device__ static constexpr int w36(int i) {
        constexpr int t[19] = {12, 2, 2, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
        return t[i];
    }
};

template <class L, class R>
__host__ __device__ constexpr R weight(int i) {
    return R(L::w36(i)) / R(36);
}

// Storage: T = element type in HBM, R = arithmetic type, SHIFTED = stores f - w_i.
template <int DT>
struct Storage;

template <>
struct Storage<0> {  // LBM_F64
    using T = double;
    using R = double;
    static constexpr bool SHIFTED = false;
    __device__ static R to_r(T v) { return v; }
    __device__ static T from_r(R v) { return v; }
};
template <>
struct Storage<1> {  // LBM_F32
    using T = float;
    using R = float;
    static constexpr bool SHIFTED = false;
    __device__ static R to_r(T v) { return v; }
    __device__ static T from_r(R v) { return v; }
};
template <>
struct Storage<2> {  // LBM_F16S
    using T = __half;
    using R = float;
    static constexpr bool SHIFTED = true;
    __device__ static R to_r(T v) { return __half2float(v); }
    __device__ static T from_r(R v) { return __float2half_rn(v); }
};
template <>
struct Storage<3> {  // LBM_BF16S
    using T = __nv_bfloat16;
    using R = float;
    static constexpr bool SHIFTED = true;
    __device__ static R to_r(T v) { return __bfloat162float(v); }
    __device__ static T from_r(R v) { return __float2bfloat16_rn(v); }
};

// Order-preserving integer image of a non-negative-or-NaN value, used for max reductions:
// for K >= 0 the bit pattern orders like the value, and a (positive) NaN beats every finite value
// and +inf, so a NaN in a tile poisons its maximum.
__device__ __forceinline__ int max_bits(float v) { return __float_as_int(v); }
__device__ __forceinline__ long long max_bits(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ float from_bits(int b, float) { return __int_as_float(b); }
__device__ __forceinline__ double from_bits(long long b, double) { return __longlong_as_double(b); }

template <class R>
struct Bits;
template <>
struct Bits<float> {
    using type = int;
};
template <>
struct Bits<double> {
    using type = long long;
};

struct StepParams {
    int nx, ny, nz;
    int periodic;      // bit 0 x, bit 1 y, bit 2 z
    int ntx, nty, ntz; // base tiles per axis
    double omega;      // 1 / tau
    double lid_x, lid_z;
    float omega_f, lid_x_f, lid_z_f;  // the same in float (no FP64 conversion in FP32 kernels)
    int *err;          // device-visible error word for bounded waits (may be null)
    void *tile_zero;   // tile-maxima buffer a sensor step clears for the next one (may be null)
    // limit (ns) of the bounded waits between a kernel's own warps; 0 = the kernel's default.  A
    // kernel waiting for its copies in flight before it exits always uses its default.
    unsigned long long wait_ns = 0;
    // test hook: the producer warps of the TMA-staged kernels issue no copies, so the consumers'
    // first wait can only run out (no copy is in flight when they give up)
    int hold_copies = 0;
    // halo planes of a slab cut along the slowest axis (z for D3Q19, y for D2Q9), or null for a
    // wall: the neighbouring slab's boundary plane of the previous post-collision state, as q
    // population planes of nx (D2Q9) or nx * ny (D3Q19) values in the storage type.  A cell on the
    // low face pulls the populations with a velocity component +1 along that axis from halo_lo,
    // one on the high face those with -1 from halo_hi, wherever the other coordinates of the pull
    // source lie inside the lattice (else the source is a wall ghost, as without a halo).
    const void *halo_lo = nullptr;
    const void *halo_hi = nullptr;
};

// The relaxation rate and lid velocity in the kernel's arithmetic type.
template <class R>
__device__ __forceinline__ R param_omega(const StepParams &p);
template <>
__device__ __forceinline__ double param_omega<double>(const StepParams &p) { return p.omega; }
template <>
__device__ __forceinline__ float param_omega<float>(const StepParams &p) { return p.omega_f; }
template <class R>
__device__ __forceinline__ R param_lid_x(const StepParams &p);
template <>
__device__ __forceinline__ double param_lid_x<double>(const StepParams &p) { return p.lid_x; }
template <>
__device__ __forceinline__ float param_lid_x<float>(const StepParams &p) { return p.lid_x_f; }
template <class R>
__device__ __forceinline__ R param_lid_z(const StepParams &p);
template <>
__device__ __forceinline__ double param_lid_z<double>(const StepParams &p) { return p.lid_z; }
template <>
__device__ __forceinline__ float param_lid_z<float>(const StepParams &p) { return p.lid_z_f; }

// Fill the float copies of the double parameters (host side, after omega and the lid are set).
inline void finish_params(StepParams &p) {
    p.omega_f = (float)p.omega;
    p.lid_x_f = (float)p.lid_x;
    p.lid_z_f = (float)p.lid_z;
}

}  // namespace lbm
