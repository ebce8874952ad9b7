// Learned predictor of the block sensor maxima: three 3x3 convolutions (cin -> H -> H -> 1, ReLU
// after the first two, zero padding), trained with a mean-square loss and Adam.  Not part of the
// paper: it lets a dynamic regrid (Sec. 5.2) refine ahead of the flow, with the Knudsen sensor as
// the judge of its flags.
//
// Precision: weights, biases and activations are stored in BF16; every product is accumulated in
// FP32; the master copy of the parameters, their gradients and the Adam moments are FP32, as are
// the gradients of the activations and the network output.  The layers are small (at most 16 x 16
// x 9 weights), so each kernel keeps its weights in shared memory; the forward pass gives a CTA a
// row tile of pixels with its input window staged in shared memory, the input gradient one
// thread one pixel, and the weight gradient one CTA one (out, in) channel pair (reduced in a
// fixed order so that a training step is deterministic).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace lbm {
namespace net {
namespace {

using bf16 = __nv_bfloat16;
constexpr int NT = 256;           // threads of the pixel kernels
constexpr int LOSS_PARTS = 256;   // CTAs of the loss reduction
constexpr int MAX_CIN = 8;

struct Norm {
    float shift[MAX_CIN], scale[MAX_CIN];
};

__global__ void k_normalise(const float *__restrict__ x, int cin, size_t hw, size_t total, Norm nm,
                            bf16 *__restrict__ x0) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)((k / hw) % cin);
        x0[k] = __float2bfloat16_rn((x[k] - nm.shift[c]) * nm.scale[c]);
    }
}

template <class T>
__device__ __forceinline__ void store_out(T *p, float v);
template <>
__device__ __forceinline__ void store_out<float>(float *p, float v) { *p = v; }
template <>
__device__ __forceinline__ void store_out<bf16>(bf16 *p, float v) { *p = __float2bfloat16_rn(v); }

// out[b, o, y, x] = bias[o] + sum_{c,i,j} W[o, c, i, j] in[b, c, y+i-1, x+j-1] (ReLU if RELU)
//
// One CTA computes FWD_TX consecutive pixels of one row of one batch item.  It stages the
// 3 x (FWD_TX + 2) input window of every channel in shared memory once (one round of independent
// loads instead of 9 dependent rounds per channel), with the weights transposed to [c][tap][o] so
// that a thread reads its output channels' weights as one vector.  Each of the FWD_WARPS warps
// takes a quarter of the work: COUT / 4 output channels, or, for the one-channel output layer, a
// quarter of the input channels, whose partial sums are added in a fixed order (deterministic).
constexpr int FWD_TX = 32;
constexpr int FWD_WARPS = 4;

template <int N>
__device__ __forceinline__ void fma_row(const float *__restrict__ wp, float v, float (&acc)[N]) {
    if constexpr (N == 4) {
        const float4 w = *reinterpret_cast<const float4 *>(wp);
        acc[0] = fmaf(w.x, v, acc[0]);
        acc[1] = fmaf(w.y, v, acc[1]);
        acc[2] = fmaf(w.z, v, acc[2]);
        acc[3] = fmaf(w.w, v, acc[3]);
    } else if constexpr (N == 2) {
        const float2 w = *reinterpret_cast<const float2 *>(wp);
        acc[0] = fmaf(w.x, v, acc[0]);
        acc[1] = fmaf(w.y, v, acc[1]);
    } else {
#pragma unroll
        for (int o = 0; o < N; ++o) acc[o] = fmaf(wp[o], v, acc[o]);
    }
}

template <int CIN, int COUT, bool RELU, class OutT>
__global__ void __launch_bounds__(FWD_TX * FWD_WARPS)
    k_conv_fwd(const bf16 *__restrict__ in, const bf16 *__restrict__ W, const bf16 *__restrict__ bias,
               int B, int H, int Wd, OutT *__restrict__ out) {
    constexpr bool SPLIT = COUT < FWD_WARPS;
    static_assert(SPLIT ? (COUT == 1 && CIN % FWD_WARPS == 0) : COUT % FWD_WARPS == 0,
                  "unsupported layer shape");
    constexpr int OPT = SPLIT ? 1 : COUT / FWD_WARPS;  // output channels per thread
    constexpr int CPT = SPLIT ? CIN / FWD_WARPS : CIN;  // input channels per thread
    constexpr int TW = FWD_TX + 2;
    __shared__ __align__(16) float ws[CIN * 9 * COUT];
    __shared__ float xs[CIN][3][TW];
    __shared__ float part[FWD_WARPS][FWD_TX];
    const int tiles_x = (Wd + FWD_TX - 1) / FWD_TX;
    const long long t = blockIdx.x;
    const int tx = (int)(t % tiles_x), y = (int)((t / tiles_x) % H), b = (int)(t / ((long long)tiles_x * H));
    const int x0 = tx * FWD_TX;
    const size_t hw = (size_t)H * Wd;
    for (int k = threadIdx.x; k < COUT * CIN * 9; k += blockDim.x) {
        const int o = k / (CIN * 9), r = k % (CIN * 9);  // W is [o][c][tap]
        ws[r * COUT + o] = __bfloat162float(W[k]);
    }
    for (int k = threadIdx.x; k < CIN * 3 * TW; k += blockDim.x) {
        const int c = k / (3 * TW), i = (k / TW) % 3, col = k % TW;
        const int yy = y + i - 1, xx = x0 + col - 1;
        xs[c][i][col] = (yy >= 0 && yy < H && xx >= 0 && xx < Wd)
                            ? __bfloat162float(in[((size_t)b * CIN + c) * hw + (size_t)yy * Wd + xx])
                            : 0.f;
    }
    __syncthreads();
    const int lane = threadIdx.x % FWD_TX, g = threadIdx.x / FWD_TX;
    const int x = x0 + lane;
    const int c0 = SPLIT ? g * CPT : 0, o0 = SPLIT ? 0 : g * OPT;
    float acc[OPT];
#pragma unroll
    for (int o = 0; o < OPT; ++o) acc[o] = SPLIT ? 0.f : __bfloat162float(bias[o0 + o]);
#pragma unroll 4
    for (int cc = 0; cc < CPT; ++cc) {
        const int c = c0 + cc;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                fma_row<OPT>(ws + (c * 9 + i * 3 + j) * COUT + o0, xs[c][i][lane + j], acc);
    }
    if constexpr (SPLIT) {
        part[g][lane] = acc[0];
        __syncthreads();
        if (g == 0 && x < Wd) {
            float v = __bfloat162float(bias[0]);
#pragma unroll
            for (int k = 0; k < FWD_WARPS; ++k) v += part[k][lane];
            store_out<OutT>(out + (size_t)b * hw + (size_t)y * Wd + x, RELU ? fmaxf(v, 0.f) : v);
        }
    } else if (x < Wd) {
#pragma unroll
        for (int o = 0; o < OPT; ++o)
            store_out<OutT>(out + ((size_t)b * COUT + o0 + o) * hw + (size_t)y * Wd + x,
                            RELU ? fmaxf(acc[o], 0.f) : acc[o]);
    }
}

// dY = 2 (Y - T) / n and per-CTA partial sums of (Y - T)^2 (fixed grid: deterministic)
__global__ void __launch_bounds__(NT)
    k_loss_grad(const float *__restrict__ y, const float *__restrict__ t, long long n, float two_n,
                float *__restrict__ dy, double *__restrict__ part) {
    double acc = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const float d = y[k] - t[k];
        dy[k] = two_n * d;
        acc += (double)d * (double)d;
    }
    __shared__ double sh[NT];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_loss_final(const double *__restrict__ part, int nparts, long long n,
                             double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < nparts; ++k) s += part[k];
        *out = s / (double)n;
    }
}

// dA[b, c, y, x] = (A > 0) * sum_{o,i,j} W[o, c, i, j] dO[b, o, y-i+1, x-j+1]
template <int CIN, int COUT>
__global__ void __launch_bounds__(NT)
    k_conv_bwd_data(const float *__restrict__ dO, const bf16 *__restrict__ W,
                    const bf16 *__restrict__ A, int B, int H, int Wd, float *__restrict__ dA) {
    __shared__ float ws[COUT * CIN * 9];
    for (int k = threadIdx.x; k < COUT * CIN * 9; k += blockDim.x) ws[k] = __bfloat162float(W[k]);
    __syncthreads();
    const int hw = H * Wd;
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= (long long)B * hw) return;
    const int b = (int)(pix / hw), p = (int)(pix % hw), y = p / Wd, x = p % Wd;
    float acc[CIN];
#pragma unroll
    for (int c = 0; c < CIN; ++c) acc[c] = 0.f;
    for (int o = 0; o < COUT; ++o) {
        const float *plane = dO + ((size_t)b * COUT + o) * hw;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int yy = y - i + 1;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int xx = x - j + 1;
                const float d = (yy >= 0 && yy < H && xx >= 0 && xx < Wd) ? plane[yy * Wd + xx] : 0.f;
#pragma unroll
                for (int c = 0; c < CIN; ++c) acc[c] = fmaf(ws[(o * CIN + c) * 9 + i * 3 + j], d, acc[c]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < CIN; ++c) {
        const size_t k = ((size_t)b * CIN + c) * hw + p;
        dA[k] = __bfloat162float(A[k]) > 0.f ? acc[c] : 0.f;
    }
}

// CTA (o, c): gW[o, c, i, j] = sum_{b,y,x} dO[b, o, y, x] A[b, c, y+i-1, x+j-1]; with c == 0 also
// gb[o] = sum dO[b, o, ...].  Fixed-order tree reduction.
template <int CIN, int COUT>
__global__ void __launch_bounds__(NT)
    k_conv_bwd_weight(const float *__restrict__ dO, const bf16 *__restrict__ A, int B, int H,
                      int Wd, float *__restrict__ gW, float *__restrict__ gb) {
    const int o = blockIdx.x, c = blockIdx.y;
    const int hw = H * Wd;
    const long long n = (long long)B * hw;
    float acc[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = 0.f;
    for (long long pix = threadIdx.x; pix < n; pix += blockDim.x) {
        const int b = (int)(pix / hw), p = (int)(pix % hw), y = p / Wd, x = p % Wd;
        const float d = dO[((size_t)b * COUT + o) * hw + p];
        const bf16 *plane = A + ((size_t)b * CIN + c) * hw;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int yy = y + i - 1;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int xx = x + j - 1;
                const float a = (yy >= 0 && yy < H && xx >= 0 && xx < Wd)
                                    ? __bfloat162float(plane[yy * Wd + xx])
                                    : 0.f;
                acc[i * 3 + j] = fmaf(d, a, acc[i * 3 + j]);
            }
        }
        acc[9] += d;
    }
    __shared__ float sh[10][NT];
#pragma unroll
    for (int k = 0; k < 10; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < 10; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 9) gW[((size_t)o * CIN + c) * 9 + threadIdx.x] = sh[threadIdx.x][0];
    if (threadIdx.x == 9 && c == 0) gb[o] = sh[9][0];
}

__global__ void k_adam(float *__restrict__ theta, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2, bf16 *__restrict__ theta_b) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float th = theta[k] - lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
    theta[k] = th;
    theta_b[k] = __float2bfloat16_rn(th);
}

__global__ void k_to_bf16(const float *__restrict__ in, int n, bf16 *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = __float2bfloat16_rn(in[k]);
}

__global__ void k_log_targets(const double *__restrict__ kmax, long long n, float offset,
                              float floor_k, float *__restrict__ t) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double K = kmax[k];
    if (K != K) {  // a NaN maximum stays visible in the targets
        t[k] = __int_as_float(0x7fc00000);
        return;
    }
    t[k] = (float)(log10(K > (double)floor_k ? K : (double)floor_k)) - offset;
}

__global__ void k_to_maxima(const float *__restrict__ y, long long n, float offset,
                            double *__restrict__ out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    out[k] = exp10((double)y[k] + (double)offset);
}

// Residual form: targets are the change of log10 K over the horizon, predictions are added to
// the log of the maximum now.  NaN in either maximum gives NaN.
__global__ void k_log_residual(const double *__restrict__ next, const double *__restrict__ now,
                               long long n, float floor_k, float *__restrict__ t) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double a = next[k], b = now[k], f = (double)floor_k;
    if (a != a || b != b) {
        t[k] = __int_as_float(0x7fc00000);
        return;
    }
    t[k] = (float)(log10(a > f ? a : f) - log10(b > f ? b : f));
}

__global__ void k_to_maxima_residual(const float *__restrict__ y, const double *__restrict__ now,
                                     long long n, float floor_k, double *__restrict__ out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double b = now[k], f = (double)floor_k;
    out[k] = (b != b) ? b : exp10((double)y[k] + log10(b > f ? b : f));
}

// Fraction of equal flags, counted by one CTA of 1024 threads (the flag arrays of a regrid hold a
// few thousand blocks).
constexpr int JUDGE_THREADS = 1024;

__device__ __forceinline__ double cta_agreement(const int8_t *a, const int8_t *b, int n,
                                                int *red) {
    int c = 0;
    for (int k = threadIdx.x; k < n; k += JUDGE_THREADS) c += a[k] == b[k];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        c = red[threadIdx.x];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
        if (threadIdx.x == 0) red[0] = c;
    }
    __syncthreads();
    const double r = n > 0 ? (double)red[0] / (double)n : 1.0;
    __syncthreads();  // red is reused by the caller
    return r;
}

__global__ void __launch_bounds__(JUDGE_THREADS)
    k_flags_agreement(const int8_t *a, const int8_t *b, int n, double *out) {
    __shared__ int red[JUDGE_THREADS / 32];
    const double r = cta_agreement(a, b, n, red);
    if (threadIdx.x == 0) *out = r;
}

// The judge and fallback of a predicted regrid: the agreement of the previous regrid's predicted
// flags with the exact flags now decides the flags used now -- the prediction for the next
// interval if it reached min_agree (or if there is no previous prediction), else the exact flags.
__global__ void __launch_bounds__(JUDGE_THREADS)
    k_judge_select(const int8_t *pred_prev, const int8_t *exact_now, const int8_t *pred_next,
                   int n, double min_agree, int8_t *used, double *agree_out, int *fell_out) {
    __shared__ int red[JUDGE_THREADS / 32];
    double r = __longlong_as_double(0x7ff8000000000000ll);  // no previous prediction: NaN
    if (pred_prev) r = cta_agreement(pred_prev, exact_now, n, red);
    const bool exact = pred_prev && !(r >= min_agree);
    for (int k = threadIdx.x; k < n; k += JUDGE_THREADS) used[k] = exact ? exact_now[k] : pred_next[k];
    if (threadIdx.x == 0) {
        if (agree_out) *agree_out = r;
        if (fell_out) *fell_out = exact ? 1 : 0;
    }
}

// dst row k = src row idx[k] (rows of `words` 32-bit words)
__global__ void k_gather_rows(const uint32_t *__restrict__ src, size_t words,
                              const int *__restrict__ idx, int count, long long nrows,
                              uint32_t *__restrict__ dst, int *bad) {
    const size_t total = words * (size_t)count;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (size_t)gridDim.x * blockDim.x) {
        const size_t row = k / words, w = k % words;
        const int r = idx[row];
        if (r < 0 || r >= nrows) {  // an index outside the source: flagged, nothing read
            if (w == 0) atomicOr(bad, 1);
            continue;
        }
        dst[k] = src[(size_t)r * words + w];
    }
}

inline unsigned grid_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

#define NETCK(call, what)                                          \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return lbm::report_cuda_error(e_, what); \
    } while (0)

}  // namespace
}  // namespace net
}  // namespace lbm

struct lbm_net_s {
    int cin = 0, hid = 0, nparam = 0;
    int off[6] = {0, 0, 0, 0, 0, 0};  // W1, b1, W2, b2, W3, b3 in the flat parameter vector
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *theta_b = nullptr;
    lbm::net::Norm norm;
    long long t = 0;  // Adam steps taken
    cudaStream_t stream = nullptr;
    long long cap = 0;  // positions (batch x h x w) the activation buffers hold
    __nv_bfloat16 *x0 = nullptr, *a1 = nullptr, *a2 = nullptr;
    float *y = nullptr, *dy = nullptr, *dz1 = nullptr, *dz2 = nullptr;
    double *loss_part = nullptr, *loss_dev = nullptr;
    long long last_pos = 0;  // positions of the last forward / backward call (0: none yet)
};

namespace {

using namespace lbm::net;

void free_acts(lbm_net *n) {
    cudaFree(n->x0);
    cudaFree(n->a1);
    cudaFree(n->a2);
    cudaFree(n->y);
    cudaFree(n->dy);
    cudaFree(n->dz1);
    cudaFree(n->dz2);
    n->x0 = n->a1 = n->a2 = nullptr;
    n->y = n->dy = n->dz1 = n->dz2 = nullptr;
    n->cap = 0;
}

int ensure_acts(lbm_net *n, long long pos) {
    if (pos <= n->cap) return LBM_OK;
    free_acts(n);
    const size_t P = (size_t)pos;
    cudaError_t e = lbm::dev_alloc(&n->x0, P * n->cin * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = lbm::dev_alloc(&n->a1, P * n->hid * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = lbm::dev_alloc(&n->a2, P * n->hid * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = lbm::dev_alloc(&n->y, P * sizeof(float));
    if (e == cudaSuccess) e = lbm::dev_alloc(&n->dy, P * sizeof(float));
    if (e == cudaSuccess) e = lbm::dev_alloc(&n->dz1, P * n->hid * sizeof(float));
    if (e == cudaSuccess) e = lbm::dev_alloc(&n->dz2, P * n->hid * sizeof(float));
    if (e != cudaSuccess) {
        free_acts(n);
        return lbm::report_cuda_error(e, "cudaMalloc(network activations)");
    }
    n->cap = pos;
    return LBM_OK;
}

#define NET_DISPATCH(cin, hid, CALL)                                      \
    do {                                                                  \
        if ((cin) == 3 && (hid) == 16) {                                  \
            constexpr int CI = 3, HD = 16;                                \
            CALL;                                                         \
        } else if ((cin) == 4 && (hid) == 16) {                           \
            constexpr int CI = 4, HD = 16;                                \
            CALL;                                                         \
        } else if ((cin) == 3 && (hid) == 8) {                            \
            constexpr int CI = 3, HD = 8;                                 \
            CALL;                                                         \
        } else if ((cin) == 4 && (hid) == 8) {                            \
            constexpr int CI = 4, HD = 8;                                 \
            CALL;                                                         \
        } else {                                                          \
            return lbm::report_error(LBM_EINVAL, "unsupported network shape"); \
        }                                                                 \
    } while (0)

template <int CI, int HD>
int run_forward(lbm_net *n, const float *x, int B, int H, int W, float *y_out) {
    const long long pos = (long long)B * H * W;
    const __nv_bfloat16 *tb = n->theta_b;
    cudaStream_t s = n->stream;
    const size_t total = (size_t)pos * CI;
    unsigned gn = grid_for((long long)total, NT);
    if (gn > 4096) gn = 4096;
    k_normalise<<<gn, NT, 0, s>>>(x, CI, (size_t)H * W, total, n->norm, n->x0);
    const long long rows = (long long)B * H * ((W + FWD_TX - 1) / FWD_TX);
    if (rows > 0x7fffffffLL) return lbm::report_error(LBM_EINVAL, "network input too large");
    const unsigned g = (unsigned)rows, nt = FWD_TX * FWD_WARPS;
    k_conv_fwd<CI, HD, true, __nv_bfloat16><<<g, nt, 0, s>>>(n->x0, tb + n->off[0], tb + n->off[1],
                                                             B, H, W, n->a1);
    k_conv_fwd<HD, HD, true, __nv_bfloat16><<<g, nt, 0, s>>>(n->a1, tb + n->off[2], tb + n->off[3],
                                                             B, H, W, n->a2);
    k_conv_fwd<HD, 1, false, float><<<g, nt, 0, s>>>(n->a2, tb + n->off[4], tb + n->off[5], B, H, W,
                                                     y_out);
    NETCK(cudaGetLastError(), "network forward");
    return LBM_OK;
}

template <int CI, int HD>
int run_backward(lbm_net *n, const float *x, const float *target, int B, int H, int W) {
    int st = run_forward<CI, HD>(n, x, B, H, W, n->y);
    if (st != LBM_OK) return st;
    const long long pos = (long long)B * H * W;
    cudaStream_t s = n->stream;
    const __nv_bfloat16 *tb = n->theta_b;
    float *gr = n->grad;
    k_loss_grad<<<LOSS_PARTS, NT, 0, s>>>(n->y, target, pos, (float)(2.0 / (double)pos), n->dy,
                                          n->loss_part);
    k_loss_final<<<1, 32, 0, s>>>(n->loss_part, LOSS_PARTS, pos, n->loss_dev);
    const unsigned g = grid_for(pos, NT);
    // layer 3 (H -> 1)
    k_conv_bwd_weight<HD, 1><<<dim3(1, HD), NT, 0, s>>>(n->dy, n->a2, B, H, W, gr + n->off[4],
                                                         gr + n->off[5]);
    k_conv_bwd_data<HD, 1><<<g, NT, 0, s>>>(n->dy, tb + n->off[4], n->a2, B, H, W, n->dz2);
    // layer 2 (H -> H)
    k_conv_bwd_weight<HD, HD><<<dim3(HD, HD), NT, 0, s>>>(n->dz2, n->a1, B, H, W, gr + n->off[2],
                                                           gr + n->off[3]);
    k_conv_bwd_data<HD, HD><<<g, NT, 0, s>>>(n->dz2, tb + n->off[2], n->a1, B, H, W, n->dz1);
    // layer 1 (cin -> H); no input gradient
    k_conv_bwd_weight<CI, HD><<<dim3(HD, CI), NT, 0, s>>>(n->dz1, n->x0, B, H, W, gr + n->off[0],
                                                           gr + n->off[1]);
    NETCK(cudaGetLastError(), "network backward");
    return LBM_OK;
}

#define CHECK_NET(n)                                                             \
    do {                                                                         \
        lbm::clear_error();                                                      \
        if (!(n)) return lbm::report_error(LBM_EINVAL, "NULL network handle");   \
    } while (0)

int check_shape(int B, int H, int W) {
    if (B < 1 || H < 1 || W < 1 || (long long)B * H * W > (1LL << 30))
        return lbm::report_error(LBM_EINVAL, "batch, h, w must be >= 1 (and their product <= 2^30)");
    return LBM_OK;
}

}  // namespace

extern "C" {

LBM_API lbm_net *lbm_net_create(int cin, int hidden) {
    lbm::clear_error();
    if (!((cin == 3 || cin == 4) && (hidden == 8 || hidden == 16))) {
        lbm::report_error(LBM_EINVAL, "lbm_net_create: cin must be 3 or 4, hidden 8 or 16");
        return nullptr;
    }
    lbm_net *n = new (std::nothrow) lbm_net_s();
    if (!n) {
        lbm::report_error(LBM_ENOMEM, "lbm_net_create: out of host memory");
        return nullptr;
    }
    n->cin = cin;
    n->hid = hidden;
    const int sizes[6] = {hidden * cin * 9, hidden, hidden * hidden * 9, hidden, hidden * 9, 1};
    int o = 0;
    for (int k = 0; k < 6; ++k) {
        n->off[k] = o;
        o += sizes[k];
    }
    n->nparam = o;
    for (int c = 0; c < MAX_CIN; ++c) {
        n->norm.shift[c] = 0.f;
        n->norm.scale[c] = 1.f;
    }
    cudaError_t e = lbm::dev_alloc(&n->theta, sizeof(float) * o);
    if (e == cudaSuccess) e = lbm::dev_alloc(&n->grad, sizeof(float) * o);
    if (e == cudaSuccess) e = lbm::dev_alloc(&n->m, sizeof(float) * o);
    if (e == cudaSuccess) e = lbm::dev_alloc(&n->v, sizeof(float) * o);
    if (e == cudaSuccess) e = lbm::dev_alloc(&n->theta_b, sizeof(__nv_bfloat16) * o);
    if (e == cudaSuccess) e = lbm::dev_alloc(&n->loss_part, sizeof(double) * LOSS_PARTS);
    if (e == cudaSuccess) e = lbm::dev_alloc(&n->loss_dev, sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(n->theta, 0, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMemset(n->grad, 0, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMemset(n->theta_b, 0, sizeof(__nv_bfloat16) * o);
    if (e != cudaSuccess) {
        lbm::report_cuda_error(e, "lbm_net_create");
        lbm_net_destroy(n);
        return nullptr;
    }
    return n;
}

LBM_API void lbm_net_destroy(lbm_net *n) {
    if (!n) return;
    free_acts(n);
    cudaFree(n->theta);
    cudaFree(n->grad);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->theta_b);
    cudaFree(n->loss_part);
    cudaFree(n->loss_dev);
    delete n;
}

LBM_API int lbm_net_set_stream(lbm_net *n, void *stream) {
    CHECK_NET(n);
    n->stream = (cudaStream_t)stream;
    return LBM_OK;
}

LBM_API int lbm_net_param_count(lbm_net *n) {
    CHECK_NET(n);
    return n->nparam;
}

LBM_API int lbm_net_set_normalisation(lbm_net *n, const float *shift, const float *scale) {
    CHECK_NET(n);
    if (!shift || !scale) return lbm::report_error(LBM_EINVAL, "NULL shift or scale");
    for (int c = 0; c < n->cin; ++c) {
        n->norm.shift[c] = shift[c];
        n->norm.scale[c] = scale[c];
    }
    return LBM_OK;
}

LBM_API int lbm_net_set_params(lbm_net *n, const float *host) {
    CHECK_NET(n);
    if (!host) return lbm::report_error(LBM_EINVAL, "NULL parameters");
    NETCK(cudaMemcpyAsync(n->theta, host, sizeof(float) * n->nparam, cudaMemcpyHostToDevice,
                          n->stream),
          "parameters upload");
    k_to_bf16<<<grid_for(n->nparam, NT), NT, 0, n->stream>>>(n->theta, n->nparam, n->theta_b);
    NETCK(cudaMemsetAsync(n->m, 0, sizeof(float) * n->nparam, n->stream), "memset");
    NETCK(cudaMemsetAsync(n->v, 0, sizeof(float) * n->nparam, n->stream), "memset");
    n->t = 0;
    NETCK(cudaStreamSynchronize(n->stream), "lbm_net_set_params");
    return LBM_OK;
}

LBM_API int lbm_net_get_params(lbm_net *n, float *host) {
    CHECK_NET(n);
    if (!host) return lbm::report_error(LBM_EINVAL, "NULL output");
    NETCK(cudaMemcpyAsync(host, n->theta, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost,
                          n->stream),
          "parameters download");
    NETCK(cudaStreamSynchronize(n->stream), "lbm_net_get_params");
    return LBM_OK;
}

LBM_API int lbm_net_get_grads(lbm_net *n, float *host) {
    CHECK_NET(n);
    if (!host) return lbm::report_error(LBM_EINVAL, "NULL output");
    NETCK(cudaMemcpyAsync(host, n->grad, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost,
                          n->stream),
          "gradients download");
    NETCK(cudaStreamSynchronize(n->stream), "lbm_net_get_grads");
    return LBM_OK;
}

LBM_API int lbm_net_set_grads(lbm_net *n, const float *host) {
    CHECK_NET(n);
    if (!host) return lbm::report_error(LBM_EINVAL, "NULL gradients");
    NETCK(cudaMemcpyAsync(n->grad, host, sizeof(float) * n->nparam, cudaMemcpyHostToDevice,
                          n->stream),
          "gradients upload");
    NETCK(cudaStreamSynchronize(n->stream), "lbm_net_set_grads");
    return LBM_OK;
}

LBM_API int lbm_net_forward(lbm_net *n, const float *x_dev, int batch, int h, int w,
                            float *y_dev) {
    CHECK_NET(n);
    if (!x_dev || !y_dev) return lbm::report_error(LBM_EINVAL, "NULL input or output");
    int st = check_shape(batch, h, w);
    if (st != LBM_OK) return st;
    st = ensure_acts(n, (long long)batch * h * w);
    if (st != LBM_OK) return st;
    NET_DISPATCH(n->cin, n->hid, (st = run_forward<CI, HD>(n, x_dev, batch, h, w, y_dev)));
    if (st == LBM_OK) n->last_pos = (long long)batch * h * w;
    return st;
}

LBM_API int lbm_net_backward(lbm_net *n, const float *x_dev, const float *target_dev, int batch,
                             int h, int w, double *loss_host) {
    CHECK_NET(n);
    if (!x_dev || !target_dev) return lbm::report_error(LBM_EINVAL, "NULL input or target");
    int st = check_shape(batch, h, w);
    if (st != LBM_OK) return st;
    st = ensure_acts(n, (long long)batch * h * w);
    if (st != LBM_OK) return st;
    NET_DISPATCH(n->cin, n->hid, (st = run_backward<CI, HD>(n, x_dev, target_dev, batch, h, w)));
    if (st != LBM_OK) return st;
    n->last_pos = (long long)batch * h * w;
    if (loss_host) {
        NETCK(cudaMemcpyAsync(loss_host, n->loss_dev, sizeof(double), cudaMemcpyDeviceToHost,
                              n->stream),
              "loss download");
        NETCK(cudaStreamSynchronize(n->stream), "lbm_net_backward");
    }
    return LBM_OK;
}

LBM_API int lbm_net_get_buffer(lbm_net *n, int which, void *out_host, size_t bytes) {
    CHECK_NET(n);
    if (!out_host) return lbm::report_error(LBM_EINVAL, "NULL output");
    const size_t P = (size_t)n->last_pos;
    const void *src = nullptr;
    size_t need = 0;
    switch (which) {
        case LBM_NET_BUF_PARAMS_BF16:
            src = n->theta_b;
            need = (size_t)n->nparam * sizeof(__nv_bfloat16);
            break;
        case LBM_NET_BUF_X0: src = n->x0; need = P * n->cin * sizeof(__nv_bfloat16); break;
        case LBM_NET_BUF_A1: src = n->a1; need = P * n->hid * sizeof(__nv_bfloat16); break;
        case LBM_NET_BUF_A2: src = n->a2; need = P * n->hid * sizeof(__nv_bfloat16); break;
        case LBM_NET_BUF_Y: src = n->y; need = P * sizeof(float); break;
        case LBM_NET_BUF_DY: src = n->dy; need = P * sizeof(float); break;
        case LBM_NET_BUF_DZ2: src = n->dz2; need = P * n->hid * sizeof(float); break;
        case LBM_NET_BUF_DZ1: src = n->dz1; need = P * n->hid * sizeof(float); break;
        default: return lbm::report_error(LBM_EINVAL, "unknown network buffer");
    }
    if (which != LBM_NET_BUF_PARAMS_BF16 && n->last_pos == 0)
        return lbm::report_error(LBM_ESTATE, "no forward or backward pass yet");
    if (bytes != need) return lbm::report_error(LBM_EINVAL, "bytes must equal the buffer's size");
    NETCK(cudaMemcpyAsync(out_host, src, need, cudaMemcpyDeviceToHost, n->stream),
          "buffer download");
    NETCK(cudaStreamSynchronize(n->stream), "lbm_net_get_buffer");
    return LBM_OK;
}

LBM_API int lbm_net_adam(lbm_net *n, float lr, float beta1, float beta2, float eps) {
    CHECK_NET(n);
    if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
        !(eps > 0.f))
        return lbm::report_error(LBM_EINVAL, "Adam needs lr >= 0, beta in [0, 1), eps > 0");
    n->t += 1;
    const double bc1 = 1.0 - pow((double)beta1, (double)n->t);
    const double bc2 = 1.0 - pow((double)beta2, (double)n->t);
    k_adam<<<grid_for(n->nparam, NT), NT, 0, n->stream>>>(n->theta, n->grad, n->m, n->v, n->nparam,
                                                          lr, beta1, beta2, eps, (float)bc1,
                                                          (float)bc2, n->theta_b);
    NETCK(cudaGetLastError(), "lbm_net_adam");
    return LBM_OK;
}

LBM_API int lbm_net_train_step(lbm_net *n, const float *x_dev, const float *target_dev, int batch,
                               int h, int w, float lr, double *loss_host) {
    int st = lbm_net_backward(n, x_dev, target_dev, batch, h, w, nullptr);
    if (st != LBM_OK) return st;
    st = lbm_net_adam(n, lr, 0.9f, 0.999f, 1e-8f);
    if (st != LBM_OK) return st;
    if (loss_host) {
        NETCK(cudaMemcpyAsync(loss_host, n->loss_dev, sizeof(double), cudaMemcpyDeviceToHost,
                              n->stream),
              "loss download");
        NETCK(cudaStreamSynchronize(n->stream), "lbm_net_train_step");
    }
    return LBM_OK;
}

LBM_API int lbm_net_log_targets(const double *kmax_dev, long long n, float offset, float floor_k,
                                float *t_dev, void *stream) {
    lbm::clear_error();
    if (!kmax_dev || !t_dev || n < 0 || !(floor_k > 0.f))
        return lbm::report_error(LBM_EINVAL, "lbm_net_log_targets: bad arguments");
    if (n == 0) return LBM_OK;
    k_log_targets<<<grid_for(n, NT), NT, 0, (cudaStream_t)stream>>>(kmax_dev, n, offset, floor_k,
                                                                     t_dev);
    NETCK(cudaGetLastError(), "lbm_net_log_targets");
    return LBM_OK;
}

LBM_API int lbm_flags_agreement(const int8_t *a_dev, const int8_t *b_dev, int n, double *out_dev,
                                void *stream) {
    lbm::clear_error();
    if (n < 0 || (n > 0 && (!a_dev || !b_dev)) || !out_dev)
        return lbm::report_error(LBM_EINVAL, "lbm_flags_agreement: bad arguments");
    k_flags_agreement<<<1, JUDGE_THREADS, 0, (cudaStream_t)stream>>>(a_dev, b_dev, n, out_dev);
    NETCK(cudaGetLastError(), "lbm_flags_agreement");
    return LBM_OK;
}

LBM_API int lbm_flags_judge_select(const int8_t *pred_prev_dev, const int8_t *exact_now_dev,
                                   const int8_t *pred_next_dev, int n, double min_agreement,
                                   int8_t *used_dev, double *agreement_dev, int *fell_back_dev,
                                   void *stream) {
    lbm::clear_error();
    if (n < 0 || (n > 0 && (!exact_now_dev || !pred_next_dev || !used_dev)) ||
        !(min_agreement >= 0.0 && min_agreement <= 1.0))
        return lbm::report_error(LBM_EINVAL, "lbm_flags_judge_select: bad arguments");
    k_judge_select<<<1, JUDGE_THREADS, 0, (cudaStream_t)stream>>>(
        pred_prev_dev, exact_now_dev, pred_next_dev, n, min_agreement, used_dev, agreement_dev,
        fell_back_dev);
    NETCK(cudaGetLastError(), "lbm_flags_judge_select");
    return LBM_OK;
}

LBM_API int lbm_gather_rows(const void *src_dev, long long nrows, size_t row_bytes,
                            const int *idx_dev, int count, void *dst_dev, int *bad_dev,
                            void *stream) {
    lbm::clear_error();
    if (nrows < 0 || count < 0 || row_bytes % 4 != 0 ||
        (count > 0 && (!src_dev || !idx_dev || !dst_dev || !bad_dev)))
        return lbm::report_error(LBM_EINVAL, "lbm_gather_rows: bad arguments (rows of a multiple "
                                             "of 4 bytes)");
    if (count == 0 || row_bytes == 0) return LBM_OK;
    const size_t words = row_bytes / 4;
    long long total = (long long)words * count;
    unsigned g = grid_for(total, NT);
    if (g > 4096) g = 4096;
    k_gather_rows<<<g, NT, 0, (cudaStream_t)stream>>>(static_cast<const uint32_t *>(src_dev), words,
                                                       idx_dev, count, nrows,
                                                       static_cast<uint32_t *>(dst_dev), bad_dev);
    NETCK(cudaGetLastError(), "lbm_gather_rows");
    return LBM_OK;
}

LBM_API int lbm_net_log_residual(const double *kmax_next_dev, const double *kmax_now_dev,
                                 long long n, float floor_k, float *t_dev, void *stream) {
    lbm::clear_error();
    if (!kmax_next_dev || !kmax_now_dev || !t_dev || n < 0 || !(floor_k > 0.f))
        return lbm::report_error(LBM_EINVAL, "lbm_net_log_residual: bad arguments");
    if (n == 0) return LBM_OK;
    k_log_residual<<<grid_for(n, NT), NT, 0, (cudaStream_t)stream>>>(kmax_next_dev, kmax_now_dev, n,
                                                                      floor_k, t_dev);
    NETCK(cudaGetLastError(), "lbm_net_log_residual");
    return LBM_OK;
}

LBM_API int lbm_net_to_maxima_residual(const float *y_dev, const double *kmax_now_dev, long long n,
                                       float floor_k, double *kmax_dev, void *stream) {
    lbm::clear_error();
    if (!y_dev || !kmax_now_dev || !kmax_dev || n < 0 || !(floor_k > 0.f))
        return lbm::report_error(LBM_EINVAL, "lbm_net_to_maxima_residual: bad arguments");
    if (n == 0) return LBM_OK;
    k_to_maxima_residual<<<grid_for(n, NT), NT, 0, (cudaStream_t)stream>>>(y_dev, kmax_now_dev, n,
                                                                            floor_k, kmax_dev);
    NETCK(cudaGetLastError(), "lbm_net_to_maxima_residual");
    return LBM_OK;
}

LBM_API int lbm_net_to_maxima(const float *y_dev, long long n, float offset, double *kmax_dev,
                              void *stream) {
    lbm::clear_error();
    if (!y_dev || !kmax_dev || n < 0)
        return lbm::report_error(LBM_EINVAL, "lbm_net_to_maxima: bad arguments");
    if (n == 0) return LBM_OK;
    k_to_maxima<<<grid_for(n, NT), NT, 0, (cudaStream_t)stream>>>(y_dev, n, offset, kmax_dev);
    NETCK(cudaGetLastError(), "lbm_net_to_maxima");
    return LBM_OK;
}

}  // extern "C"
