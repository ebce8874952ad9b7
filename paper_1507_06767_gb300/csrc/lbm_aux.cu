// Helper kernels around the fused step: population conversion, moments, FP64 conservation sums,
// tile-to-block sensor maxima and the refine / coarsen flag builders.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int EW_THREADS = 256;

inline dim3 ew_grid(size_t N, int q) {
    size_t b = (N + EW_THREADS - 1) / EW_THREADS;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return dim3((unsigned)b, (unsigned)q, 1);
}

template <class L, int DT>
__device__ __forceinline__ double stored_to_f64(typename Storage<DT>::T v, int i) {
    double d = (double)Storage<DT>::to_r(v);
    return Storage<DT>::SHIFTED ? weight<L, double>(i) + d : d;
}

// direction tables in device-readable form for kernels indexed by a runtime direction
template <class L>
__device__ __forceinline__ double w_of(int i) {
    double w = 0;
#pragma unroll
    for (int j = 0; j < L::Q; ++j)
        if (j == i) w = weight<L, double>(j);
    return w;
}

template <class L, int DT>
__global__ void k_init_rest(typename Storage<DT>::T *f, size_t N) {
    const int i = blockIdx.y;
    const double w = w_of<L>(i);
    const auto v = Storage<DT>::SHIFTED ? Storage<DT>::from_r(0) : Storage<DT>::from_r(
        (typename Storage<DT>::R)w);
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
         c += (size_t)gridDim.x * blockDim.x)
        f[(size_t)i * N + c] = v;
}

template <class T>
__device__ __forceinline__ T from_double(double v);
template <>
__device__ __forceinline__ double from_double<double>(double v) { return v; }
template <>
__device__ __forceinline__ float from_double<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __half from_double<__half>(double v) { return __double2half(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double v) {
    return __double2bfloat16(v);
}

// in / out point at population i0; blockIdx.y selects population i0 + blockIdx.y
template <class L, int DT>
__global__ void k_from_f64(const double *in, typename Storage<DT>::T *out, size_t N, int i0) {
    using T = typename Storage<DT>::T;
    const int j = blockIdx.y;
    const double w = w_of<L>(i0 + j);
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
         c += (size_t)gridDim.x * blockDim.x) {
        double v = in[(size_t)j * N + c];
        if (Storage<DT>::SHIFTED) v -= w;
        out[(size_t)j * N + c] = from_double<T>(v);
    }
}

template <class L, int DT>
__global__ void k_to_f64(const typename Storage<DT>::T *in, double *out, size_t N, int i0) {
    const int j = blockIdx.y;
    const double w = w_of<L>(i0 + j);
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
         c += (size_t)gridDim.x * blockDim.x) {
        double d = (double)Storage<DT>::to_r(in[(size_t)j * N + c]);
        out[(size_t)j * N + c] = Storage<DT>::SHIFTED ? w + d : d;
    }
}

// moments of cells [c0, c0 + nc): rho[nc], u[3][nc]
template <class L, int DT>
__global__ void k_moments(const typename Storage<DT>::T *f, size_t N, size_t c0, size_t nc,
                          double *rho, double *u) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < nc;
         k += (size_t)gridDim.x * blockDim.x) {
        const size_t c = c0 + k;
        double r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const double v = stored_to_f64<L, DT>(f[(size_t)i * N + c], i);
            r += v;
            jx += L::cx(i) * v;
            jy += L::cy(i) * v;
            jz += L::cz(i) * v;
        }
        rho[k] = r;
        u[k] = jx / r;
        u[nc + k] = jy / r;
        u[2 * nc + k] = jz / r;
    }
}

// Block means of the cell moments: one CTA per block of edge b (partial blocks at the high ends),
// out[c][block] for c = rho, u_x, u_y (, u_z) with blocks in x-fastest order.  Sums in double for
// FP64 lattices; in float for the others, whose populations carry no more digits (the outputs
// are floats feeding a BF16 network; the slow FP64 pipe of this GPU made the double form take
// 0.18 ms per 1024^2 D2Q9 lattice).  The block sums go through warp shuffles.
constexpr int FEAT_THREADS = 256;

template <class L, int DT>
__global__ void __launch_bounds__(FEAT_THREADS)
    k_block_features(const typename Storage<DT>::T *f, int nx, int ny, int nz, int b, int bz,
                     int nbx, int nby, int nblocks, float *out) {
    using A = typename std::conditional<DT == 0, double, float>::type;
    using S = Storage<DT>;
    const int blk = blockIdx.x;
    const int bx = blk % nbx, by = (blk / nbx) % nby, bzi = blk / (nbx * nby);
    const int x0 = bx * b, y0 = by * b, z0 = bzi * bz;
    const int ex = min(b, nx - x0), ey = min(b, ny - y0), ez = min(bz, nz - z0);
    const int ncell = ex * ey * ez;
    const size_t N = (size_t)nx * ny * nz;
    A acc[4] = {0, 0, 0, 0};
    for (int k = threadIdx.x; k < ncell; k += blockDim.x) {
        const int x = x0 + k % ex, y = y0 + (k / ex) % ey, z = z0 + k / (ex * ey);
        const size_t c = ((size_t)z * ny + y) * nx + x;
        A r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const A d = (A)S::to_r(f[(size_t)i * N + c]);
            const A v = S::SHIFTED ? weight<L, A>(i) + d : d;
            r += v;
            if (L::cx(i)) jx += (A)L::cx(i) * v;
            if (L::cy(i)) jy += (A)L::cy(i) * v;
            if (L::cz(i)) jz += (A)L::cz(i) * v;
        }
        const A inv = A(1) / r;
        acc[0] += r;
        acc[1] += jx * inv;
        acc[2] += jy * inv;
        acc[3] += jz * inv;
    }
    __shared__ A sh[4][FEAT_THREADS / 32];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
        if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = acc[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nch = L::D == 3 ? 4 : 3;
        for (int k = 0; k < nch; ++k) {
            A t = sh[k][0];
            for (int w = 1; w < FEAT_THREADS / 32; ++w) t += sh[k][w];
            out[(size_t)k * nblocks + blk] = (float)(t / (A)ncell);
        }
    }
}

constexpr int CONS_THREADS = 256;

template <class L, int DT>
__global__ void __launch_bounds__(CONS_THREADS)
    k_cons_partial(const typename Storage<DT>::T *f, size_t N, double *partial) {
    double acc[5] = {0, 0, 0, 0, 0};
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N;
         c += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const double v = stored_to_f64<L, DT>(f[(size_t)i * N + c], i);
            if (!isfinite(v)) acc[4] += 1.0;
            acc[0] += v;
            acc[1] += L::cx(i) * v;
            acc[2] += L::cy(i) * v;
            acc[3] += L::cz(i) * v;
        }
    }
    __shared__ double sh[5][CONS_THREADS];
#pragma unroll
    for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = CONS_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 5; ++k) partial[(size_t)blockIdx.x * 5 + k] = sh[k][0];
}

__global__ void __launch_bounds__(1024) k_cons_final(const double *partial, int nparts,
                                                     double *result) {
    __shared__ double sh[5][1024];
    for (int k = 0; k < 5; ++k)
        sh[k][threadIdx.x] = (threadIdx.x < nparts) ? partial[(size_t)threadIdx.x * 5 + k] : 0.0;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 5) result[threadIdx.x] = sh[threadIdx.x][0];
}

// Block maximum of K over the tiles of block b (tile maxima compared as order-preserving bits, so
// a NaN tile makes the block NaN).
template <class R>
__device__ __forceinline__ R block_of_tiles(const R *tiles, int ntx, int nty, int ntz, int m, int mz,
                                            int nbx, int nby, long long b) {
    using B = typename Bits<R>::type;
    const int bx = (int)(b % nbx);
    const int by = (int)((b / nbx) % nby);
    const int bz = (int)(b / ((long long)nbx * nby));
    B mx = 0;
    if (m == 2 && mz <= 2) {
        // blocks of 2 x 2 (x 2) tiles (the 16-cell block on 8-cell tiles): the tile loads are
        // independent, so they are issued together
        B v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int tx = 2 * bx + (j & 1), ty = 2 * by + ((j >> 1) & 1);
            const int tz = bz * mz + (j >> 2);
            const bool ok = tx < ntx && ty < nty && (j >> 2) < mz && tz < ntz;
            v[j] = ok ? max_bits(tiles[((size_t)tz * nty + ty) * ntx + tx]) : B(0);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) mx = v[j] > mx ? v[j] : mx;
        return from_bits(mx, R(0));
    }
    for (int tz = bz * mz; tz < min(bz * mz + mz, ntz); ++tz)
        for (int ty = by * m; ty < min(by * m + m, nty); ++ty)
            for (int tx = bx * m; tx < min(bx * m + m, ntx); ++tx) {
                const B v = max_bits(tiles[((size_t)tz * nty + ty) * ntx + tx]);
                mx = v > mx ? v : mx;
            }
    return from_bits(mx, R(0));
}

template <class R>
__global__ void k_tiles_to_blocks(const R *tiles, int ntx, int nty, int ntz, int m, int mz,
                                  R *blocks, int nbx, int nby, int nbz) {
    const long long nb = (long long)nbx * nby * nbz;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x)
        blocks[b] = block_of_tiles(tiles, ntx, nty, ntz, m, mz, nbx, nby, b);
}

template <class R>
__global__ void k_to_f64_plain(const R *in, double *out, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        out[k] = (double)in[k];
}

template <class R>
__global__ void k_flags_threshold(const R *m, int n, double T, double half_T, int8_t *out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double v = (double)m[k];
        out[k] = (isnan(v) || v > T) ? int8_t(1) : (v < half_T ? int8_t(-1) : int8_t(0));
    }
}

// Order-preserving unsigned keys; NaN maps to the key of +inf.
__device__ __forceinline__ uint32_t sort_key(float v) {
    if (isnan(v)) v = INFINITY;
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ unsigned long long sort_key(double v) {
    if (isnan(v)) v = INFINITY;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

constexpr int TOP_THREADS = 1024;

// Single-CTA radix select of the k-th largest key (1 <= k <= n), then flags: keys above it refine,
// keys equal to it refine in block-index order until k blocks are taken.
template <class R, class K>
__global__ void __launch_bounds__(TOP_THREADS) k_flags_top(const R *m, int n, int k, int8_t *out) {
    __shared__ unsigned hist[256];
    __shared__ int s_digit, s_remaining;
    __shared__ int scan[TOP_THREADS];
    const int tid = threadIdx.x;
    K prefix = 0, mask = 0;
    int remaining = k;
    for (int shift = 8 * (int)sizeof(K) - 8; shift >= 0; shift -= 8) {
        for (int b = tid; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        for (int e = tid; e < n; e += blockDim.x) {
            const K key = sort_key(m[e]);
            if ((key & mask) == prefix) atomicAdd(&hist[(unsigned)(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (tid < 32) {
            const int hi = 255 - 8 * tid;  // this lane's bins: hi, hi-1, ..., hi-7
            unsigned sum8 = 0;
            for (int j = 0; j < 8; ++j) sum8 += hist[hi - j];
            unsigned incl = sum8;
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned o = __shfl_up_sync(0xffffffffu, incl, off);
                if (tid >= off) incl += o;
            }
            const unsigned ballot = __ballot_sync(0xffffffffu, incl >= (unsigned)remaining);
            const int first = __ffs(ballot) - 1;
            if (tid == first) {
                unsigned c = incl - sum8;
                for (int j = 0; j < 8; ++j) {
                    const unsigned h = hist[hi - j];
                    if (c + h >= (unsigned)remaining) {
                        s_digit = hi - j;
                        s_remaining = remaining - (int)c;
                        break;
                    }
                    c += h;
                }
            }
        }
        __syncthreads();
        prefix |= (K)s_digit << shift;
        mask |= (K)0xFF << shift;
        remaining = s_remaining;
        __syncthreads();
    }
    // prefix is the k-th largest key; `remaining` equal keys are taken, lowest indices first
    const int chunk = (n + TOP_THREADS - 1) / TOP_THREADS;
    const int start = min(tid * chunk, n), end = min(start + chunk, n);
    int eq = 0;
    for (int e = start; e < end; ++e) eq += (sort_key(m[e]) == prefix);
    scan[tid] = eq;
    __syncthreads();
    for (int off = 1; off < TOP_THREADS; off <<= 1) {
        const int v = (tid >= off) ? scan[tid - off] : 0;
        __syncthreads();
        scan[tid] += v;
        __syncthreads();
    }
    int before = scan[tid] - eq;
    for (int e = start; e < end; ++e) {
        const K key = sort_key(m[e]);
        int8_t fl = 0;
        if (key > prefix) {
            fl = 1;
        } else if (key == prefix) {
            fl = (before < remaining) ? int8_t(1) : int8_t(0);
            ++before;
        }
        out[e] = fl;
    }
}

// Threshold flags straight from the tile maxima: the block maxima (also written to `blocks`) and
// their flags (+1 refine if max > T or NaN, -1 coarsen if max < T/2, else 0) in one pass.
template <class R>
__global__ void k_flags_threshold_tiles(const R *tiles, int ntx, int nty, int ntz, int m, int mz,
                                        R *blocks, int nbx, int nby, int nbz, double T,
                                        double half_T, int8_t *out) {
    const long long nb = (long long)nbx * nby * nbz;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        const R mx = block_of_tiles(tiles, ntx, nty, ntz, m, mz, nbx, nby, b);
        blocks[b] = mx;
        const double v = (double)mx;
        out[b] = (isnan(v) || v > T) ? int8_t(1) : (v < half_T ? int8_t(-1) : int8_t(0));
    }
}

// Top-k flags of n block maxima in one CTA with their order-preserving keys held in shared memory
// for the 8-bit radix passes that find the k-th largest key (the global-memory form, k_flags_top,
// reads the maxima again on every pass); keys above it are flagged, and of the keys equal to it
// the lowest indices, as many as remain.  Needs n * sizeof(K) bytes of dynamic shared memory (at
// most TOP_SMEM_BYTES) and 0 < k < n.
constexpr int TOP_SMEM_BYTES = 64 * 1024;

template <class R, class K>
__global__ void __launch_bounds__(TOP_THREADS) k_flags_top_keys(const R *maxima, int n, int k,
                                                               int8_t *out) {
    extern __shared__ __align__(16) unsigned char top_smem[];
    K *keys = reinterpret_cast<K *>(top_smem);
    __shared__ unsigned hist[256];
    __shared__ int s_digit, s_remaining;
    __shared__ int wsum[TOP_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int b = tid; b < n; b += TOP_THREADS) keys[b] = sort_key(maxima[b]);
    K prefix = 0, mask = 0;
    int remaining = k;
    for (int shift = 8 * (int)sizeof(K) - 8; shift >= 0; shift -= 8) {
        for (int b = tid; b < 256; b += TOP_THREADS) hist[b] = 0;
        __syncthreads();  // also orders the key writes above before the first pass
        for (int e = tid; e < n; e += TOP_THREADS) {
            const K key = keys[e];
            if ((key & mask) == prefix) atomicAdd(&hist[(unsigned)(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (tid < 32) {
            const int hi = 255 - 8 * tid;  // this lane's bins: hi, hi-1, ..., hi-7
            unsigned sum8 = 0;
            for (int j = 0; j < 8; ++j) sum8 += hist[hi - j];
            unsigned incl = sum8;
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned o = __shfl_up_sync(0xffffffffu, incl, off);
                if (tid >= off) incl += o;
            }
            const unsigned ballot = __ballot_sync(0xffffffffu, incl >= (unsigned)remaining);
            const int first = __ffs(ballot) - 1;
            if (tid == first) {
                unsigned c = incl - sum8;
                for (int j = 0; j < 8; ++j) {
                    const unsigned h = hist[hi - j];
                    if (c + h >= (unsigned)remaining) {
                        s_digit = hi - j;
                        s_remaining = remaining - (int)c;
                        break;
                    }
                    c += h;
                }
            }
        }
        __syncthreads();
        prefix |= (K)s_digit << shift;
        mask |= (K)0xFF << shift;
        remaining = s_remaining;
        __syncthreads();
    }
    // keys equal to the k-th largest: exclusive count over the threads' contiguous chunks
    const int chunk = (n + TOP_THREADS - 1) / TOP_THREADS;
    const int start = min(tid * chunk, n), end = min(start + chunk, n);
    int eq = 0;
    for (int e = start; e < end; ++e) eq += (keys[e] == prefix);
    int incl = eq;
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = wsum[lane];
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += o;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int before = (warp > 0 ? wsum[warp - 1] : 0) + incl - eq;
    for (int e = start; e < end; ++e) {
        const K key = keys[e];
        int8_t fl = 0;
        if (key > prefix) {
            fl = 1;
        } else if (key == prefix) {
            fl = (before < remaining) ? int8_t(1) : int8_t(0);
            ++before;
        }
        out[e] = fl;
    }
}

// Refinement level of one block maximum (Sec. 3.4): phi = log2 K, l = clamp(floor(a phi + b)).
__device__ __forceinline__ int8_t level_of(double v, double a, double b, int lmin, int lmax) {
    if (isnan(v)) return (int8_t)lmax;
    if (!(v > 0.0)) return (int8_t)lmin;
    double t = floor(a * log2(v) + b);
    t = fmin(fmax(t, (double)lmin), (double)lmax);
    return (int8_t)(int)t;
}

template <class R>
__global__ void k_levels_affine(const R *m, int n, double a, double b, int lmin, int lmax,
                                int8_t *out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        out[k] = level_of((double)m[k], a, b, lmin, lmax);
}

// Fit a, b to the range of phi over the blocks with a finite K > 0, then map.  phi = log2 K is
// monotone, so its range is log2 of the range of K: every CTA finds the extreme maxima itself
// (a scan of all n values, no logarithms), takes two logarithms and maps its own share of the
// blocks (one logarithm each; double precision runs at a small fraction of the FP32 rate on this
// GPU, so the logarithms are spread over the whole grid).
template <class R>
__global__ void __launch_bounds__(256) k_levels_fit(const R *m, int n, int lmin, int lmax,
                                                    int8_t *out) {
    // smallest and largest positive finite maximum, compared in the maxima's own type (exact: the
    // conversion to double is monotonic), reduced by warp shuffles
    __shared__ R slo[8], shi[8];
    R lo = R(INFINITY), hi = R(-INFINITY);
#pragma unroll 4
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const R v = m[k];
        if (v > R(0) && isfinite(v)) {
            lo = v < lo ? v : lo;
            hi = v > hi ? v : hi;
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const R ol = __shfl_xor_sync(0xffffffffu, lo, off), oh = __shfl_xor_sync(0xffffffffu, hi, off);
        lo = ol < lo ? ol : lo;
        hi = oh > hi ? oh : hi;
    }
    if ((threadIdx.x & 31) == 0) {
        slo[threadIdx.x >> 5] = lo;
        shi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    // the fit (two double logarithms and a division) once per CTA, shared with its threads
    __shared__ double s_a, s_b;
    __shared__ bool s_scale;
    if (threadIdx.x == 0) {
        lo = slo[0];
        hi = shi[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = slo[w] < lo ? slo[w] : lo;
            hi = shi[w] > hi ? shi[w] : hi;
        }
        const bool any = lo <= hi;
        const double plo = any ? log2((double)lo) : 0.0, phi = any ? log2((double)hi) : 0.0;
        s_scale = phi > plo;
        s_a = s_scale ? (double)(lmax - lmin + 1) / (phi - plo) : 0.0;
        s_b = s_scale ? (double)lmin - s_a * plo : 0.0;
    }
    __syncthreads();
    const bool scale = s_scale;
    const double a = s_a, b = s_b;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double v = (double)m[k];
        out[k] = scale ? level_of(v, a, b, lmin, lmax)
                       : (isnan(v) ? (int8_t)lmax : (int8_t)lmin);
    }
}

__global__ void k_accumulate_tiles_f(const float *t, double *sum, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        sum[k] += (double)t[k];
}
__global__ void k_accumulate_tiles_d(const double *t, double *sum, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        sum[k] += t[k];
}
__global__ void k_scale(const double *sum, double inv, double *out, size_t n) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        out[k] = sum[k] * inv;
}

__global__ void k_fill_i8(int8_t *out, int n, int8_t v) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        out[k] = v;
}

inline unsigned small_grid(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

#define LBM_DISPATCH(q, dtype, CALL)                                         \
    do {                                                                     \
        if ((q) == 9) {                                                      \
            using L = D2Q9;                                                  \
            switch (dtype) {                                                 \
                case 0: { constexpr int DT = 0; CALL; } break;               \
                case 1: { constexpr int DT = 1; CALL; } break;               \
                case 2: { constexpr int DT = 2; CALL; } break;               \
                case 3: { constexpr int DT = 3; CALL; } break;               \
                default: return cudaErrorInvalidValue;                       \
            }                                                                \
        } else if ((q) == 19) {                                              \
            using L = D3Q19;                                                 \
            switch (dtype) {                                                 \
                case 0: { constexpr int DT = 0; CALL; } break;               \
                case 1: { constexpr int DT = 1; CALL; } break;               \
                case 2: { constexpr int DT = 2; CALL; } break;               \
                case 3: { constexpr int DT = 3; CALL; } break;               \
                default: return cudaErrorInvalidValue;                       \
            }                                                                \
        } else {                                                             \
            return cudaErrorInvalidValue;                                    \
        }                                                                    \
    } while (0)

cudaError_t init_rest(int q, int dtype, void *f, size_t N, cudaStream_t s) {
    LBM_DISPATCH(q, dtype, (k_init_rest<L, DT><<<ew_grid(N, q), EW_THREADS, 0, s>>>(
                               static_cast<typename Storage<DT>::T *>(f), N)));
    return cudaGetLastError();
}

namespace {

// Halo messages: plain copies of whole population planes, by element size (the storage types
// are copied bit for bit).
template <class E>
__global__ void k_halo_pack(const E *__restrict__ f, size_t N, size_t plane_off, size_t plane,
                            HaloDirs d, E *__restrict__ msg) {
    const int j = blockIdx.y;
    const E *src = f + (size_t)d.dir[j] * N + plane_off;
    E *dst = msg + (size_t)j * plane;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < plane;
         c += (size_t)gridDim.x * blockDim.x)
        dst[c] = src[c];
}

template <class E>
__global__ void k_halo_unpack(const E *__restrict__ msg, size_t plane, HaloDirs d,
                              E *__restrict__ halo) {
    const int j = blockIdx.y;
    const E *src = msg + (size_t)j * plane;
    E *dst = halo + (size_t)d.dir[j] * plane;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < plane;
         c += (size_t)gridDim.x * blockDim.x)
        dst[c] = src[c];
}

template <class E>
cudaError_t halo_pack_t(const void *f, size_t N, size_t plane_off, size_t plane, const HaloDirs &d,
                        void *msg, cudaStream_t s) {
    k_halo_pack<E><<<ew_grid(plane, d.k), EW_THREADS, 0, s>>>(static_cast<const E *>(f), N,
                                                               plane_off, plane, d,
                                                               static_cast<E *>(msg));
    return cudaGetLastError();
}

template <class E>
cudaError_t halo_unpack_t(const void *msg, size_t plane, const HaloDirs &d, void *halo,
                          cudaStream_t s) {
    k_halo_unpack<E><<<ew_grid(plane, d.k), EW_THREADS, 0, s>>>(static_cast<const E *>(msg), plane,
                                                                 d, static_cast<E *>(halo));
    return cudaGetLastError();
}

}  // namespace

cudaError_t halo_pack(int elem, const void *f, size_t N, size_t plane_off, size_t plane,
                      const HaloDirs &d, void *msg, cudaStream_t s) {
    if (d.k < 1 || d.k > HALO_MAX_DIRS || plane == 0) return cudaErrorInvalidValue;
    switch (elem) {
        case 2: return halo_pack_t<unsigned short>(f, N, plane_off, plane, d, msg, s);
        case 4: return halo_pack_t<unsigned>(f, N, plane_off, plane, d, msg, s);
        case 8: return halo_pack_t<unsigned long long>(f, N, plane_off, plane, d, msg, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t halo_unpack(int elem, const void *msg, size_t plane, const HaloDirs &d, void *halo,
                        cudaStream_t s) {
    if (d.k < 1 || d.k > HALO_MAX_DIRS || plane == 0) return cudaErrorInvalidValue;
    switch (elem) {
        case 2: return halo_unpack_t<unsigned short>(msg, plane, d, halo, s);
        case 4: return halo_unpack_t<unsigned>(msg, plane, d, halo, s);
        case 8: return halo_unpack_t<unsigned long long>(msg, plane, d, halo, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t f64_to_storage(int q, int dtype, int i0, int nq, const double *in, void *out, size_t N,
                           cudaStream_t s) {
    LBM_DISPATCH(q, dtype, (k_from_f64<L, DT><<<ew_grid(N, nq), EW_THREADS, 0, s>>>(
                               in, static_cast<typename Storage<DT>::T *>(out), N, i0)));
    return cudaGetLastError();
}

cudaError_t storage_to_f64(int q, int dtype, int i0, int nq, const void *in, double *out, size_t N,
                           cudaStream_t s) {
    LBM_DISPATCH(q, dtype, (k_to_f64<L, DT><<<ew_grid(N, nq), EW_THREADS, 0, s>>>(
                               static_cast<const typename Storage<DT>::T *>(in), out, N, i0)));
    return cudaGetLastError();
}

cudaError_t moments_f64(int q, int dtype, const void *f, size_t N, size_t c0, size_t nc,
                        double *rho, double *u, cudaStream_t s) {
    LBM_DISPATCH(q, dtype, (k_moments<L, DT><<<ew_grid(nc, 1), EW_THREADS, 0, s>>>(
                               static_cast<const typename Storage<DT>::T *>(f), N, c0, nc, rho, u)));
    return cudaGetLastError();
}

cudaError_t block_features(int q, int dtype, const void *f, int nx, int ny, int nz, int b,
                          float *out, cudaStream_t s) {
    const int bz = nz > 1 ? b : 1;
    const int nbx = (nx + b - 1) / b, nby = (ny + b - 1) / b, nbz = (nz + bz - 1) / bz;
    const int nblocks = nbx * nby * nbz;
    LBM_DISPATCH(q, dtype, (k_block_features<L, DT><<<nblocks, FEAT_THREADS, 0, s>>>(
                               static_cast<const typename Storage<DT>::T *>(f), nx, ny, nz, b, bz,
                               nbx, nby, nblocks, out)));
    return cudaGetLastError();
}

cudaError_t conservation(int q, int dtype, const void *f, size_t N, double *partial, double *result,
                         cudaStream_t s) {
    LBM_DISPATCH(q, dtype, (k_cons_partial<L, DT><<<CONS_PARTS, CONS_THREADS, 0, s>>>(
                               static_cast<const typename Storage<DT>::T *>(f), N, partial)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_cons_final<<<1, 1024, 0, s>>>(partial, CONS_PARTS, result);
    return cudaGetLastError();
}

cudaError_t tiles_to_blocks(int rtype, const void *tiles, int ntx, int nty, int ntz, int m, int mz,
                            void *blocks, int nbx, int nby, int nbz, cudaStream_t s) {
    const long long nb = (long long)nbx * nby * nbz;
    const unsigned g = small_grid(nb, 256);
    if (rtype == 0)
        k_tiles_to_blocks<double><<<g, 256, 0, s>>>(static_cast<const double *>(tiles), ntx, nty,
                                                    ntz, m, mz, static_cast<double *>(blocks), nbx,
                                                    nby, nbz);
    else
        k_tiles_to_blocks<float><<<g, 256, 0, s>>>(static_cast<const float *>(tiles), ntx, nty, ntz,
                                                   m, mz, static_cast<float *>(blocks), nbx, nby,
                                                   nbz);
    return cudaGetLastError();
}

cudaError_t to_f64(int rtype, const void *in, double *out, size_t n, cudaStream_t s) {
    const unsigned g = small_grid((long long)n, 256);
    if (rtype == 0)
        k_to_f64_plain<double><<<g, 256, 0, s>>>(static_cast<const double *>(in), out, n);
    else
        k_to_f64_plain<float><<<g, 256, 0, s>>>(static_cast<const float *>(in), out, n);
    return cudaGetLastError();
}

cudaError_t flags_threshold(int rtype, const void *maxima, int n, double T, int8_t *out,
                            cudaStream_t s) {
    const unsigned g = small_grid(n, 256);
    if (rtype == 0)
        k_flags_threshold<double><<<g, 256, 0, s>>>(static_cast<const double *>(maxima), n, T,
                                                    T / 2.0, out);
    else
        k_flags_threshold<float><<<g, 256, 0, s>>>(static_cast<const float *>(maxima), n, T,
                                                   T / 2.0, out);
    return cudaGetLastError();
}

// Block maxima of the last sensor step's tiles and their flags (rule 0: threshold `param`, one
// launch; 1: the k largest: the block maxima, then the one-CTA select over shared-memory keys, or
// over global memory where the keys do not fit).
cudaError_t flags_from_tiles(int rtype, const void *tiles, int ntx, int nty, int ntz, int m, int mz,
                             void *blocks, int nbx, int nby, int nbz, int rule, double param, int k,
                             int8_t *out, cudaStream_t s) {
    const long long nb = (long long)nbx * nby * nbz;
    if (nb <= 0) return cudaSuccess;
    if (rule == 0) {
        const unsigned g = small_grid(nb, 256);
        if (rtype == 0)
            k_flags_threshold_tiles<double><<<g, 256, 0, s>>>(
                static_cast<const double *>(tiles), ntx, nty, ntz, m, mz,
                static_cast<double *>(blocks), nbx, nby, nbz, param, param / 2.0, out);
        else
            k_flags_threshold_tiles<float><<<g, 256, 0, s>>>(
                static_cast<const float *>(tiles), ntx, nty, ntz, m, mz,
                static_cast<float *>(blocks), nbx, nby, nbz, param, param / 2.0, out);
        return cudaGetLastError();
    }
    cudaError_t e = tiles_to_blocks(rtype, tiles, ntx, nty, ntz, m, mz, blocks, nbx, nby, nbz, s);
    if (e != cudaSuccess) return e;
    const size_t key_bytes = rtype == 0 ? sizeof(unsigned long long) : sizeof(uint32_t);
    if (k <= 0 || k >= nb || (size_t)nb * key_bytes > (size_t)TOP_SMEM_BYTES)
        return flags_top(rtype, blocks, (int)nb, k, out, s);
    // the dynamic shared memory above 48 KB is granted per function and device, once
    static std::atomic<bool> granted[2][64] = {};  // setting the attribute twice is harmless
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!granted[rtype == 0][dev].load(std::memory_order_acquire)) {
        e = rtype == 0 ? cudaFuncSetAttribute(k_flags_top_keys<double, unsigned long long>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              TOP_SMEM_BYTES)
                       : cudaFuncSetAttribute(k_flags_top_keys<float, uint32_t>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              TOP_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        granted[rtype == 0][dev].store(true, std::memory_order_release);
    }
    const size_t smem = (size_t)nb * key_bytes;
    if (rtype == 0)
        k_flags_top_keys<double, unsigned long long><<<1, TOP_THREADS, smem, s>>>(
            static_cast<const double *>(blocks), (int)nb, k, out);
    else
        k_flags_top_keys<float, uint32_t><<<1, TOP_THREADS, smem, s>>>(
            static_cast<const float *>(blocks), (int)nb, k, out);
    return cudaGetLastError();
}

cudaError_t flags_top(int rtype, const void *maxima, int n, int k, int8_t *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (k <= 0 || k >= n) {
        k_fill_i8<<<small_grid(n, 256), 256, 0, s>>>(out, n, k <= 0 ? int8_t(0) : int8_t(1));
        return cudaGetLastError();
    }
    // keys in shared memory where they fit the default 48 KB of a launch, else the select that
    // reads the maxima from global memory on every pass
    const size_t key_bytes = rtype == 0 ? sizeof(unsigned long long) : sizeof(uint32_t);
    if ((size_t)n * key_bytes <= 48 * 1024) {
        const size_t smem = (size_t)n * key_bytes;
        if (rtype == 0)
            k_flags_top_keys<double, unsigned long long><<<1, TOP_THREADS, smem, s>>>(
                static_cast<const double *>(maxima), n, k, out);
        else
            k_flags_top_keys<float, uint32_t><<<1, TOP_THREADS, smem, s>>>(
                static_cast<const float *>(maxima), n, k, out);
        return cudaGetLastError();
    }
    if (rtype == 0)
        k_flags_top<double, unsigned long long><<<1, TOP_THREADS, 0, s>>>(
            static_cast<const double *>(maxima), n, k, out);
    else
        k_flags_top<float, uint32_t><<<1, TOP_THREADS, 0, s>>>(static_cast<const float *>(maxima),
                                                              n, k, out);
    return cudaGetLastError();
}

cudaError_t levels_affine(int rtype, const void *maxima, int n, double a, double b, int lmin,
                          int lmax, int8_t *out, cudaStream_t s) {
    const unsigned g = small_grid(n, 256);
    if (rtype == 0)
        k_levels_affine<double><<<g, 256, 0, s>>>(static_cast<const double *>(maxima), n, a, b, lmin,
                                                  lmax, out);
    else
        k_levels_affine<float><<<g, 256, 0, s>>>(static_cast<const float *>(maxima), n, a, b, lmin,
                                                 lmax, out);
    return cudaGetLastError();
}

cudaError_t levels_fit(int rtype, const void *maxima, int n, int lmin, int lmax, int8_t *out,
                       cudaStream_t s) {
    // each CTA scans all n values once: keep the grid to about one CTA per SM
    const unsigned g = (unsigned)std::min<long long>(((long long)n + 255) / 256, 152);
    if (rtype == 0)
        k_levels_fit<double><<<g, 256, 0, s>>>(static_cast<const double *>(maxima), n, lmin, lmax,
                                               out);
    else
        k_levels_fit<float><<<g, 256, 0, s>>>(static_cast<const float *>(maxima), n, lmin, lmax,
                                              out);
    return cudaGetLastError();
}

cudaError_t accumulate_tiles(int rtype, const void *tiles, double *sum, size_t n, cudaStream_t s) {
    const unsigned g = small_grid((long long)n, 256);
    if (rtype == 0)
        k_accumulate_tiles_d<<<g, 256, 0, s>>>(static_cast<const double *>(tiles), sum, n);
    else
        k_accumulate_tiles_f<<<g, 256, 0, s>>>(static_cast<const float *>(tiles), sum, n);
    return cudaGetLastError();
}

cudaError_t scale_f64(const double *in, double factor, double *out, size_t n, cudaStream_t s) {
    k_scale<<<small_grid((long long)n, 256), 256, 0, s>>>(in, factor, out, n);
    return cudaGetLastError();
}

}  // namespace lbm
