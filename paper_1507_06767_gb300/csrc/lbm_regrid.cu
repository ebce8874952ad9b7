// Regridding of one refinement level from the Knudsen sensor (Sec. 5.2): tags, buffer cells,
// proper nesting, Berger-Rigoutsos point clustering.
//
// The per-cell work runs on the GPU: tagging (max of the sensor over a tag cell against the
// threshold), the buffer (a Chebyshev-ball dilation, done as three 1-D passes since the ball is a
// product of segments), the nesting mask (the dual erosion, positions beyond a non-periodic edge
// counting as covered) and, for every round of candidate boxes, the slab counts (signatures)
// along each axis.  The cut decisions need only the signatures, so the host makes them between
// rounds: shrink to the tags' bounding box, accept at the efficiency, else cut at the hole nearest
// the centre, else at the strongest inflection of the signature, else bisect the longest axis;
// cuts leaving a piece narrower than min_width are not admissible.  Boxes of one round are
// disjoint, so a round costs one pass over at most the tag grid.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace lbm {
namespace rg {

namespace {

constexpr int SIG_XCHUNK = 1024;  // x extent of one signature work item
constexpr int SIG_CELLS = 16384;  // cells of one signature work item (at most)
constexpr int SIG_THREADS = 256;

struct SigItem {
    int box, z, y0, y1, x0, x1;
};
struct SigBox {
    int lo[3];
    int w, h, off;  // sig x at off, y at off + w, z at off + w + h
};

template <class T>
__global__ void k_tag(const T *__restrict__ K, int nx, int ny, int nz, int r, int rz, int tx,
                      int ty, long long ntag, double thr, uint8_t *__restrict__ tags) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntag) return;
    const int x = (int)(t % tx), y = (int)((t / tx) % ty), z = (int)(t / ((long long)tx * ty));
    const int x0 = x * r, y0 = y * r, z0 = z * rz;
    const int x1 = min(x0 + r, nx), y1 = min(y0 + r, ny), z1 = min(z0 + rz, nz);
    uint8_t hit = 0;
    for (int cz = z0; cz < z1 && !hit; ++cz)
        for (int cy = y0; cy < y1 && !hit; ++cy) {
            const T *row = K + ((size_t)cz * ny + cy) * nx;
            for (int cx = x0; cx < x1; ++cx) {
                const double v = (double)row[cx];
                if (v > thr || v != v) {
                    hit = 1;
                    break;
                }
            }
        }
    tags[t] = hit;
}

// The same for FP32 fields whose tag cells span whole groups of 4 cells along x (r % 4 == 0,
// nx % 4 == 0): 16-byte loads, all of a row's loads issued before any test.  thr_f is the largest
// float not above the double threshold, so v > thr_f decides exactly as (double)v > thr, without
// the FP64 pipe (a small fraction of the FP32 rate on this GPU).
__global__ void k_tag_f4(const float *__restrict__ K, int nx, int ny, int nz, int r, int rz,
                         int tx, int ty, long long ntag, float thr_f, uint8_t *__restrict__ tags) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntag) return;
    const int x = (int)(t % tx), y = (int)((t / tx) % ty), z = (int)(t / ((long long)tx * ty));
    const int x0 = x * r, y0 = y * r, z0 = z * rz;
    const int x1 = min(x0 + r, nx), y1 = min(y0 + r, ny), z1 = min(z0 + rz, nz);
    int hit = 0;
    for (int cz = z0; cz < z1; ++cz)
        for (int cy = y0; cy < y1; ++cy) {
            const float4 *row = reinterpret_cast<const float4 *>(K + ((size_t)cz * ny + cy) * nx);
            for (int c4 = x0 / 4; c4 < x1 / 4; ++c4) {
                const float4 v = __ldg(row + c4);
                // NaN fails every comparison: !(v <= thr_f) is true for v > thr_f and for NaN
                hit |= !(v.x <= thr_f) | !(v.y <= thr_f) | !(v.z <= thr_f) | !(v.w <= thr_f);
            }
        }
    tags[t] = (uint8_t)(hit != 0);
}

// One 1-D pass along an axis of extent n and element stride `stride`: dilation (op 0: OR over the
// segment, nothing beyond a non-periodic edge) or erosion (op 1: AND over the segment, covered
// beyond a non-periodic edge).  Periodic axes wrap.
__global__ void k_morph(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, long long total,
                        int n, long long stride, int radius, int periodic, int op) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int c = (int)((t / stride) % n);
    int acc = op;  // OR starts at 0, AND at 1
    for (int k = -radius; k <= radius; ++k) {
        int cc = c + k;
        if (cc < 0 || cc >= n) {
            if (!periodic) continue;  // beyond the edge: 0 for OR, 1 for AND, neither changes acc
            cc = ((cc % n) + n) % n;
        }
        const int v = in[t + (long long)(cc - c) * stride] != 0;
        acc = op ? (acc & v) : (acc | v);
    }
    out[t] = (uint8_t)acc;
}

__global__ void k_and(uint8_t *__restrict__ tags, const uint8_t *__restrict__ mask,
                      long long total) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < total) tags[t] = (uint8_t)(tags[t] && mask[t]);
}

__global__ void k_normalise(uint8_t *m, long long total) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < total) m[t] = (uint8_t)(m[t] != 0);
}

// Slab counts of one work item (a z plane, a run of rows, a run of x) of one box: one warp per
// row, x counts in shared memory, row counts written directly (each row belongs to one warp), the
// plane count added once per CTA.
__global__ void __launch_bounds__(SIG_THREADS)
    k_signatures(const uint8_t *__restrict__ tags, int tx, int ty, const SigItem *__restrict__ items,
                 const SigBox *__restrict__ boxes, int *__restrict__ sig) {
    __shared__ int sx[SIG_XCHUNK];
    __shared__ int sy[SIG_XCHUNK];
    __shared__ int plane;
    const SigItem it = items[blockIdx.x];
    const SigBox b = boxes[it.box];
    const int cw = it.x1 - it.x0, ch = it.y1 - it.y0;
    for (int i = threadIdx.x; i < SIG_XCHUNK; i += blockDim.x) sx[i] = 0;
    if (threadIdx.x == 0) plane = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int cnt = 0;
    for (int y = warp; y < ch; y += nw) {
        const uint8_t *row = tags + ((size_t)it.z * ty + it.y0 + y) * tx + it.x0;
        int rc = 0;
        for (int x = lane; x < cw; x += 32) {
            const int v = row[x];
            if (v) atomicAdd(&sx[x], 1);
            rc += v;
        }
        rc = __reduce_add_sync(0xffffffffu, rc);
        if (lane == 0) sy[y] = rc;
        cnt += rc;
    }
    if (lane == 0 && cnt) atomicAdd(&plane, cnt);
    __syncthreads();
    for (int i = threadIdx.x; i < cw; i += blockDim.x)
        if (sx[i]) atomicAdd(&sig[b.off + it.x0 - b.lo[0] + i], sx[i]);
    for (int i = threadIdx.x; i < ch; i += blockDim.x)
        if (sy[i]) atomicAdd(&sig[b.off + b.w + it.y0 - b.lo[1] + i], sy[i]);
    if (threadIdx.x == 0 && plane) atomicAdd(&sig[b.off + b.w + b.h + it.z - b.lo[2]], plane);
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// The largest float whose value does not exceed t (t itself if it is a float; NaN stays NaN).
inline float float_at_most(double t) {
    float f = (float)t;
    if ((double)f > t) f = nextafterf(f, -INFINITY);
    return f;
}

struct HBox {
    int lo[3], hi[3];
};

// Host side of one box: trim to the tags, then accept or cut.  Returns 0 (drop), 1 (accept,
// `box` trimmed) or 2 (cut into lower / upper).
int decide(HBox &box, const int *sx, const int *sy, const int *sz, double efficiency, int wmin,
           HBox *lower, HBox *upper) {
    const int *s[3] = {sx, sy, sz};
    int len[3];
    int first[3], last[3];
    long long total = 0;
    for (int a = 0; a < 3; ++a) {
        len[a] = box.hi[a] - box.lo[a];
        first[a] = -1;
        last[a] = -1;
        for (int i = 0; i < len[a]; ++i)
            if (s[a][i]) {
                if (first[a] < 0) first[a] = i;
                last[a] = i;
            }
    }
    for (int i = 0; i < len[0]; ++i) total += s[0][i];
    if (total == 0) return 0;
    const int *sig[3];
    for (int a = 0; a < 3; ++a) {
        sig[a] = s[a] + first[a];
        box.hi[a] = box.lo[a] + last[a] + 1;
        box.lo[a] += first[a];
        len[a] = last[a] - first[a] + 1;
    }
    const double vol = (double)len[0] * (double)len[1] * (double)len[2];
    if ((double)total >= efficiency * vol) return 1;

    int cut_axis = -1, cut_at = 0;
    // holes: least |2p - L|, then longer axis, lower axis, lower p
    long long bd = 0;
    int bl = 0;
    for (int a = 0; a < 3; ++a)
        for (int p = wmin; p <= len[a] - wmin; ++p) {
            if (p >= len[a] || sig[a][p] != 0) continue;
            const long long d = llabs(2LL * p - len[a]);
            const bool better = cut_axis < 0 || d < bd || (d == bd && len[a] > bl);
            if (better) {  // equal d and length: the earlier (axis, p) stays
                cut_axis = a;
                cut_at = p;
                bd = d;
                bl = len[a];
            }
        }
    if (cut_axis < 0) {
        // inflections: strongest |D[i+1] - D[i]| at a strict sign change, then as for holes
        long long bs = -1;
        for (int a = 0; a < 3; ++a) {
            const int *q = sig[a];
            for (int i = 1; i <= len[a] - 3; ++i) {
                const long long d0 = (long long)q[i - 1] - 2LL * q[i] + q[i + 1];
                const long long d1 = (long long)q[i] - 2LL * q[i + 1] + q[i + 2];
                if (!((d0 < 0 && d1 > 0) || (d0 > 0 && d1 < 0))) continue;
                const int p = i + 1;
                if (p < wmin || len[a] - p < wmin) continue;
                const long long st = llabs(d1 - d0);
                const long long d = llabs(2LL * p - len[a]);
                const bool better = cut_axis < 0 || st > bs ||
                                    (st == bs && (d < bd || (d == bd && len[a] > bl)));
                if (better) {
                    cut_axis = a;
                    cut_at = p;
                    bs = st;
                    bd = d;
                    bl = len[a];
                }
            }
        }
    }
    if (cut_axis < 0) {
        // bisection of the longest admissible axis (ties: lower axis)
        for (int a = 0; a < 3; ++a) {
            const int p = len[a] / 2;
            if (p < wmin || len[a] - p < wmin) continue;
            if (cut_axis < 0 || len[a] > bl) {
                cut_axis = a;
                cut_at = p;
                bl = len[a];
            }
        }
    }
    if (cut_axis < 0) return 1;
    *lower = box;
    *upper = box;
    lower->hi[cut_axis] = box.lo[cut_axis] + cut_at;
    upper->lo[cut_axis] = box.lo[cut_axis] + cut_at;
    return 2;
}

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    ~DevBuf() { cudaFree(p); }
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap) return cudaSuccess;
        cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = lbm::dev_alloc(&p, bytes);
        if (e == cudaSuccess) cap = bytes;
        return e;
    }
};

#define RGCK(call, what)                                          \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return report_cuda_error(e_, what); \
    } while (0)

}  // namespace

int regrid(const void *field, int field_type, int nx, int ny, int nz, int periodic,
           const Params &p, const uint8_t *allowed_host, std::vector<int> *boxes_out,
           long long *ntagged, uint8_t *tags_out, cudaStream_t s) {
    const int r = p.coarsen, rz = nz > 1 ? p.coarsen : 1;
    const int tx = (nx + r - 1) / r, ty = (ny + r - 1) / r, tz = (nz + rz - 1) / rz;
    const long long ntag = (long long)tx * ty * tz;
    DevBuf tagbuf[2], maskbuf, sigbuf, itembuf, boxbuf;
    RGCK(tagbuf[0].ensure(ntag), "cudaMalloc(tags)");
    RGCK(tagbuf[1].ensure(ntag), "cudaMalloc(tags)");
    uint8_t *ta = (uint8_t *)tagbuf[0].p, *tb = (uint8_t *)tagbuf[1].p;

    // 1. tags
    if (field_type == LBM_F64)
        k_tag<double><<<nblk(ntag, 256), 256, 0, s>>>((const double *)field, nx, ny, nz, r, rz, tx,
                                                      ty, ntag, p.threshold, ta);
    else if (r % 4 == 0 && nx % 4 == 0 && ((uintptr_t)field & 15) == 0)
        k_tag_f4<<<nblk(ntag, 256), 256, 0, s>>>((const float *)field, nx, ny, nz, r, rz, tx, ty,
                                                  ntag, float_at_most(p.threshold), ta);
    else
        k_tag<float><<<nblk(ntag, 256), 256, 0, s>>>((const float *)field, nx, ny, nz, r, rz, tx,
                                                     ty, ntag, p.threshold, ta);
    RGCK(cudaGetLastError(), "tag kernel");
    const int ext[3] = {tx, ty, tz};
    const long long stride[3] = {1, tx, (long long)tx * ty};
    // 2. buffer: three 1-D dilations
    if (p.buffer > 0) {
        for (int a = 0; a < 3; ++a) {
            k_morph<<<nblk(ntag, 256), 256, 0, s>>>(ta, tb, ntag, ext[a], stride[a], p.buffer,
                                                    (periodic >> a) & 1, 0);
            std::swap(ta, tb);
        }
        RGCK(cudaGetLastError(), "buffer kernel");
    }
    // 3. proper nesting: erode the covered mask, keep the tags inside it
    if (allowed_host) {
        RGCK(maskbuf.ensure(2 * ntag), "cudaMalloc(mask)");
        uint8_t *ma = (uint8_t *)maskbuf.p, *mb = ma + ntag;
        RGCK(cudaMemcpyAsync(ma, allowed_host, ntag, cudaMemcpyHostToDevice, s), "mask upload");
        k_normalise<<<nblk(ntag, 256), 256, 0, s>>>(ma, ntag);
        if (p.nest > 0)
            for (int a = 0; a < 3; ++a) {
                k_morph<<<nblk(ntag, 256), 256, 0, s>>>(ma, mb, ntag, ext[a], stride[a], p.nest,
                                                        (periodic >> a) & 1, 1);
                std::swap(ma, mb);
            }
        k_and<<<nblk(ntag, 256), 256, 0, s>>>(ta, ma, ntag);
        RGCK(cudaGetLastError(), "nesting kernel");
    }
    if (tags_out) RGCK(cudaMemcpyAsync(tags_out, ta, ntag, cudaMemcpyDeviceToHost, s), "tags");

    // 4. clustering: rounds of signature passes over the pending boxes
    std::vector<HBox> pending(1), accepted;
    pending[0] = HBox{{0, 0, 0}, {tx, ty, tz}};
    std::vector<SigItem> items;
    std::vector<SigBox> sboxes;
    std::vector<int> sig;
    bool first_round = true;
    while (!pending.empty()) {
        items.clear();
        sboxes.clear();
        int off = 0;
        for (size_t k = 0; k < pending.size(); ++k) {
            const HBox &b = pending[k];
            SigBox sb;
            for (int a = 0; a < 3; ++a) sb.lo[a] = b.lo[a];
            sb.w = b.hi[0] - b.lo[0];
            sb.h = b.hi[1] - b.lo[1];
            sb.off = off;
            off += sb.w + sb.h + (b.hi[2] - b.lo[2]);
            sboxes.push_back(sb);
            for (int z = b.lo[2]; z < b.hi[2]; ++z)
                for (int x0 = b.lo[0]; x0 < b.hi[0]; x0 += SIG_XCHUNK) {
                    const int x1 = std::min(x0 + SIG_XCHUNK, b.hi[0]);
                    const int rows = std::max(1, std::min(SIG_XCHUNK, SIG_CELLS / (x1 - x0)));
                    for (int y0 = b.lo[1]; y0 < b.hi[1]; y0 += rows)
                        items.push_back({(int)k, z, y0, std::min(y0 + rows, b.hi[1]), x0, x1});
                }
        }
        RGCK(sigbuf.ensure(sizeof(int) * off), "cudaMalloc(signatures)");
        RGCK(itembuf.ensure(sizeof(SigItem) * items.size()), "cudaMalloc(items)");
        RGCK(boxbuf.ensure(sizeof(SigBox) * sboxes.size()), "cudaMalloc(boxes)");
        RGCK(cudaMemcpyAsync(itembuf.p, items.data(), sizeof(SigItem) * items.size(),
                             cudaMemcpyHostToDevice, s),
             "items upload");
        RGCK(cudaMemcpyAsync(boxbuf.p, sboxes.data(), sizeof(SigBox) * sboxes.size(),
                             cudaMemcpyHostToDevice, s),
             "boxes upload");
        RGCK(cudaMemsetAsync(sigbuf.p, 0, sizeof(int) * off, s), "memset(signatures)");
        k_signatures<<<(unsigned)items.size(), SIG_THREADS, 0, s>>>(
            ta, tx, ty, (const SigItem *)itembuf.p, (const SigBox *)boxbuf.p, (int *)sigbuf.p);
        RGCK(cudaGetLastError(), "signature kernel");
        sig.resize(off);
        RGCK(cudaMemcpyAsync(sig.data(), sigbuf.p, sizeof(int) * off, cudaMemcpyDeviceToHost, s),
             "signatures download");
        RGCK(cudaStreamSynchronize(s), "regrid round");
        std::vector<HBox> next;
        for (size_t k = 0; k < pending.size(); ++k) {
            HBox b = pending[k], lo, hi;
            const SigBox &sb = sboxes[k];
            const int *sx = sig.data() + sb.off;
            if (first_round && ntagged) {
                long long t = 0;
                for (int i = 0; i < sb.w; ++i) t += sx[i];
                *ntagged = t;
            }
            const int d = decide(b, sx, sx + sb.w, sx + sb.w + sb.h, p.efficiency, p.min_width,
                                 &lo, &hi);
            if (d == 1) accepted.push_back(b);
            if (d == 2) {
                next.push_back(lo);
                next.push_back(hi);
            }
        }
        first_round = false;
        pending.swap(next);
    }
    std::sort(accepted.begin(), accepted.end(), [](const HBox &a, const HBox &b) {
        if (a.lo[2] != b.lo[2]) return a.lo[2] < b.lo[2];
        if (a.lo[1] != b.lo[1]) return a.lo[1] < b.lo[1];
        return a.lo[0] < b.lo[0];
    });
    const int scale[3] = {r, r, rz}, lat[3] = {nx, ny, nz};
    boxes_out->clear();
    for (const HBox &b : accepted) {
        for (int a = 0; a < 3; ++a) boxes_out->push_back(b.lo[a] * scale[a]);
        for (int a = 0; a < 3; ++a)
            boxes_out->push_back((int)std::min<long long>((long long)b.hi[a] * scale[a], lat[a]));
    }
    return LBM_OK;
}

}  // namespace rg
}  // namespace lbm
