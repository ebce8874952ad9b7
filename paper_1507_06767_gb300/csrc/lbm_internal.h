// Internal launch interface between the C-ABI layer (lbm_api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "lbm_traits.cuh"

namespace lbm {

// Fused step (lbm_step_d2q9.cu / lbm_step_d3q19.cu).  mode: 0 no sensor, 1 tile max, 2 + field.
// variant: KERNEL_CELL: the one-cell kernel; KERNEL_PAIR: the two-cell packed one; KERNEL_TMA: the
// TMA-staged one (D3Q19 only); KERNEL_TMA_PAIR: the TMA-staged two-cell one (D3Q19, 16-bit
// storage); the last three are errors where they do not apply.  KERNEL_AUTO picks
// the two-cell kernel where it applies (even nx, (q + 1) * cells < 2^32) for 16-bit storage and
// for FP32 storage on D2Q9 lattices of at least AUTO_PAIR_MIN_CELLS_D2Q9_F32 cells, else the
// one-cell kernel (FP64, FP32 D3Q19, small FP32 D2Q9).  It never picks the TMA kernel, whose tile
// maxima need a cleared buffer (lbm_step_noalloc relies on this).
constexpr long long AUTO_PAIR_MIN_CELLS_D2Q9_F32 = 1LL << 17;
constexpr int KERNEL_AUTO = 0;
constexpr int KERNEL_CELL = 1;
constexpr int KERNEL_PAIR = 2;
constexpr int KERNEL_TMA = 3;
constexpr int KERNEL_TMA_PAIR = 4;
cudaError_t step_d2q9(int dtype, const void *fin, void *fout, const StepParams &p, int mode,
                      void *tile_max, void *k_field, cudaStream_t s, int variant = KERNEL_AUTO);
cudaError_t step_d3q19(int dtype, const void *fin, void *fout, const StepParams &p, int mode,
                       void *tile_max, void *k_field, cudaStream_t s, int variant = KERNEL_AUTO);

// Population helpers (lbm_aux.cu).
cudaError_t init_rest(int q, int dtype, void *f, size_t N, cudaStream_t s);
// Halo planes of a slab (StepParams::halo_lo / halo_hi).  A halo message holds k population
// planes of `plane` values in the storage type (elem bytes each), for the directions dirs[0..k).
// halo_pack: message[j] = population dirs[j] of the lattice plane starting at cell plane_off
// (N cells per population); halo_unpack: halo plane dirs[j] (of a q x plane halo) = message[j].
constexpr int HALO_MAX_DIRS = 8;
struct HaloDirs {
    int k;
    int dir[HALO_MAX_DIRS];
};
cudaError_t halo_pack(int elem, const void *f, size_t N, size_t plane_off, size_t plane,
                      const HaloDirs &d, void *msg, cudaStream_t s);
cudaError_t halo_unpack(int elem, const void *msg, size_t plane, const HaloDirs &d, void *halo,
                        cudaStream_t s);
// Conversions of populations [i0, i0 + nq); in / out point at population i0 (N values each).
cudaError_t f64_to_storage(int q, int dtype, int i0, int nq, const double *in, void *out, size_t N,
                           cudaStream_t s);
cudaError_t storage_to_f64(int q, int dtype, int i0, int nq, const void *in, double *out, size_t N,
                           cudaStream_t s);
// rho[nc] and u[3][nc] of cells [c0, c0 + nc).
cudaError_t moments_f64(int q, int dtype, const void *f, size_t N, size_t c0, size_t nc,
                        double *rho, double *u, cudaStream_t s);
// Block means of rho, u_x, u_y (, u_z for D3Q19) over blocks of edge b (b along z only for 3-D
// lattices): out[c * nblocks + block], blocks x fastest.
cudaError_t block_features(int q, int dtype, const void *f, int nx, int ny, int nz, int b,
                           float *out, cudaStream_t s);
// Deterministic FP64 sums: result[0] = mass, [1..3] = momentum, [4] = number of non-finite
// populations.  partial must hold CONS_PARTS * 5 doubles.
constexpr int CONS_PARTS = 608;
cudaError_t conservation(int q, int dtype, const void *f, size_t N, double *partial, double *result,
                         cudaStream_t s);

// Sensor reductions (lbm_aux.cu).  rtype: LBM_F64 (double maxima) or LBM_F32 (float maxima).
cudaError_t tiles_to_blocks(int rtype, const void *tiles, int ntx, int nty, int ntz, int m, int mz,
                            void *blocks, int nbx, int nby, int nbz, cudaStream_t s);
cudaError_t to_f64(int rtype, const void *in, double *out, size_t n, cudaStream_t s);
cudaError_t flags_threshold(int rtype, const void *maxima, int n, double T, int8_t *out,
                            cudaStream_t s);
cudaError_t flags_top(int rtype, const void *maxima, int n, int k, int8_t *out, cudaStream_t s);
// block maxima from the tile maxima (written to blocks) and their flags: rule 0 threshold
// `param` in one launch; rule 1 the k largest (block maxima, then a one-CTA select with the keys
// in shared memory where they fit)
cudaError_t flags_from_tiles(int rtype, const void *tiles, int ntx, int nty, int ntz, int m, int mz,
                             void *blocks, int nbx, int nby, int nbz, int rule, double param, int k,
                             int8_t *out, cudaStream_t s);

// Level map (Sec. 3.4) of n block maxima, affine (a, b given) or fitted to their range.
cudaError_t levels_affine(int rtype, const void *maxima, int n, double a, double b, int lmin,
                          int lmax, int8_t *out, cudaStream_t s);
cudaError_t levels_fit(int rtype, const void *maxima, int n, int lmin, int lmax, int8_t *out,
                       cudaStream_t s);
// Time average of the tile maxima: sum += tiles; out = sum * factor.
cudaError_t accumulate_tiles(int rtype, const void *tiles, double *sum, size_t n, cudaStream_t s);
cudaError_t scale_f64(const double *in, double factor, double *out, size_t n, cudaStream_t s);

// Multi-level block mesh (lbm_multilevel.cu).
namespace ml {
struct Mesh;
// fusion: 0 automatic (separate), 1 separate restriction, 2 fused into the finest level's step;
// step_form: -1 autotuned, else the step kernel form forced where it applies (LBM_STEP_FORM_*
// minus one)
// schedule: 0 timed, 1 graph of separate launches, 2 one persistent launch per cycle
int build(Mesh **out, const int nb[3], int edge, int lmax, const int8_t *leaf, double tau_fine,
          const double lid[3], int periodic, int fusion, int step_form, int schedule,
          cudaStream_t s);
void destroy(Mesh *m);
bool same_layout(const Mesh *m, const int nb[3], int edge, int lmax, const int8_t *leaf);
// err: device-visible error word set when a bounded wait of the persistent kernel runs out (may
// be null); wait_ns: that wait's limit (0: one second); hold: test hook (every wait runs out)
int run_cycles(Mesh *m, int cycles, cudaStream_t s, bool graphs, int *err, unsigned long long wait_ns,
               int hold);
bool uses_persistent(const Mesh *m);
int block_max(Mesh *m, double *out_host, cudaStream_t s);
int get_block(Mesh *m, int l, int b, double *out, cudaStream_t s);
int set_block(Mesh *m, int l, int b, const double *in, cudaStream_t s);
int info(const Mesh *m, int l, int *n, double *tau, int *nslot, int *threads, int *cpt);
int schedule(const Mesh *m, int l, int *form, int *planes, int *fused);
long long cells_per_cycle(const Mesh *m);
}  // namespace ml

// Regridding of one level (lbm_regrid.cu).  field: nx * ny * nz values of field_type (LBM_F64:
// double, LBM_F32: float) on the device; boxes_out receives 6 ints per box (lo x y z, hi x y z).
namespace rg {
struct Params {
    int coarsen;
    double threshold;
    int buffer;
    int nest;
    double efficiency;
    int min_width;
};
int regrid(const void *field, int field_type, int nx, int ny, int nz, int periodic,
           const Params &p, const uint8_t *allowed_host, std::vector<int> *boxes_out,
           long long *ntagged, uint8_t *tags_out, cudaStream_t s);
}  // namespace rg

// Every device allocation of the library goes through dev_alloc (lbm_api.cu): cudaMalloc, except
// that the failure injection of lbm_debug_fail_alloc can make one call report
// cudaErrorMemoryAllocation without allocating.
cudaError_t dev_alloc(void **p, size_t bytes);
template <class T>
inline cudaError_t dev_alloc(T **p, size_t bytes) {
    return dev_alloc(reinterpret_cast<void **>(p), bytes);
}

// Error state shared by the C-ABI translation units (lbm_api.cu).
int report_error(int code, const char *msg);
int report_cuda_error(cudaError_t e, const char *what);
void clear_error();

}  // namespace lbm
