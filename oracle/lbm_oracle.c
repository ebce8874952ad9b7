/*
 * Plain FP64 CPU oracle for the lattice Boltzmann step with the Knudsen refinement sensor.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA path is measured against.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may load it; the product
 * library never links or calls it, and it shares no source, header or table with the CUDA code.
 *
 * What it computes (paper: "Local mesh refinement sensor for the lattice Boltzmann method"):
 *   - velocity sets D2Q9 and D3Q19 with their standard weights (Sec. 2.2: the paper uses D2Q9;
 *     D3Q19 is another instance of the same discrete-velocity BGK model),
 *   - the truncated Maxwellian equilibrium of Eq. (feq_i) with c_s^2 = 1/3,
 *   - the moments rho and rho*u of Eqs. (rho), (u),
 *   - the BGK lattice equation of Eq. (bgklb), split into the collision f_out = f - (f - feq)/tau and
 *     the streaming f(x + c_i, t + 1) = f_out(x, t) (Sec. 2.2, "collide-and-stream"),
 *   - moving-wall half-way bounce-back for the cavity walls (Sec. 4.1: no-slip walls, the top wall at
 *     y = N moves with the lid velocity),
 *   - the Knudsen sensor K = (1/q) sum_i |f_i^neq / f_i^eq| of Eqs. (sensor) and (kkn), evaluated for
 *     every cell (Sec. 3.2, step 3).
 * Everything is written the plain way: one loop over cells, one over directions, no blocking, no
 * fusion beyond what the step itself states.
 *
 * Readings taken where the paper is silent (each is listed in the design notes):
 *   - nodes sit at integer positions 0..n-1 on every axis; walls are half way, at -1/2 and n-1/2;
 *   - the lid is the ghost plane y = ny; every ghost node with y == ny (edge and corner ghosts
 *     included) moves with the lid velocity, every other ghost node is at rest;
 *   - the wall density in the moving bounce-back term is the reference density rho_w = 1;
 *   - the sensor is evaluated on the pre-collision populations of the step (after streaming and
 *     bounce-back), with the rho and u of those populations;
 *   - the solver variable is the bar-f of Eq. (lbm) (the paper drops the bar), so the sensor is taken
 *     on it directly.
 *
 * An optional constant body force (Guo's forcing, the scheme Sec. 4.5 cites) exists only so that a
 * test can pin the oracle against the Poiseuille closed form; the cavity never uses it.
 *
 * Layout: f[i][z][y][x], x fastest, i slowest, double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXQ 19

/* D2Q9: rest, 4 axis, 4 diagonal. */
static const int C9[9][3] = {
    {0, 0, 0},  {1, 0, 0},   {0, 1, 0},  {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0},  {-1, 1, 0},  {-1, -1, 0}, {1, -1, 0}};
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* D3Q19: rest, 6 axis, 12 edge directions. */
static const int C19[19][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W19[19] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static const double CS2 = 1.0 / 3.0; /* c_s^2, Sec. 2.2 */

typedef struct {
    int q;           /* 9 or 19 */
    int nx, ny, nz;  /* nz == 1 for D2Q9 */
    double tau;      /* lattice relaxation time, > 1/2 */
    double lid[3];   /* lid velocity; y component must be 0 */
    int periodic;    /* bit 0: x, bit 1: y, bit 2: z */
    double force[3]; /* Guo body force (oracle only; zero for the cavity) */
} orc_params;

/* Error codes of the oracle. */
#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_EFEQ -2 /* an equilibrium population <= 0 (the sensor divides by it) */

typedef struct {
    int q;
    int c[ORC_MAXQ][3];
    double w[ORC_MAXQ];
    int opp[ORC_MAXQ];
} lattice_t;

static int get_lattice(int q, lattice_t *L) {
    const int(*c)[3];
    const double *w;
    if (q == 9) {
        c = C9;
        w = W9;
    } else if (q == 19) {
        c = C19;
        w = W19;
    } else {
        return ORC_EINVAL;
    }
    L->q = q;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) L->c[i][a] = c[i][a];
        L->w[i] = w[i];
    }
    /* the opposite direction is found by search, not tabulated */
    for (int i = 0; i < q; ++i) {
        L->opp[i] = -1;
        for (int j = 0; j < q; ++j)
            if (c[j][0] == -c[i][0] && c[j][1] == -c[i][1] && c[j][2] == -c[i][2]) L->opp[i] = j;
    }
    return ORC_OK;
}

static int check_params(const orc_params *p, lattice_t *L) {
    if (get_lattice(p->q, L) != ORC_OK) return ORC_EINVAL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return ORC_EINVAL;
    if (p->q == 9 && p->nz != 1) return ORC_EINVAL;
    if (!(p->tau > 0.5)) return ORC_EINVAL;
    if (p->lid[1] != 0.0) return ORC_EINVAL;
    return ORC_OK;
}

/* Copy the lattice tables out (used by the tests to pin them against the isotropy conditions). */
int orc_lattice(int q, int *c_out, double *w_out, int *opp_out) {
    lattice_t L;
    if (get_lattice(q, &L) != ORC_OK) return ORC_EINVAL;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) c_out[3 * i + a] = L.c[i][a];
        w_out[i] = L.w[i];
        opp_out[i] = L.opp[i];
    }
    return ORC_OK;
}

static size_t cell_index(const orc_params *p, int x, int y, int z) {
    return ((size_t)z * (size_t)p->ny + (size_t)y) * (size_t)p->nx + (size_t)x;
}

static size_t ncells(const orc_params *p) { return (size_t)p->nx * p->ny * p->nz; }

/* Equilibrium of Eq. (feq_i): w_i rho (1 + c.u / cs2 + Q_i:uu / (2 cs2^2)), Q_i = c_i c_i - cs2 I. */
static double feq_i(const lattice_t *L, int i, double rho, const double u[3]) {
    double cu = 0.0, uu = 0.0;
    for (int a = 0; a < 3; ++a) {
        cu += L->c[i][a] * u[a];
        uu += u[a] * u[a];
    }
    double Quu = cu * cu - CS2 * uu;
    return L->w[i] * rho * (1.0 + cu / CS2 + Quu / (2.0 * CS2 * CS2));
}

/* Moments of Eqs. (rho), (u); with a body force the velocity carries the half-force shift of
 * Guo's scheme. */
static void moments(const lattice_t *L, const double *f, const double F[3], double *rho, double u[3]) {
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L->q; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) j[a] += L->c[i][a] * f[i];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / r;
}

/* Sensor of Eq. (sensor): K = (1/q) sum_i |f_i - feq_i| / feq_i.  Returns ORC_EFEQ if an equilibrium
 * population is not positive. */
static int sensor_cell(const lattice_t *L, const double *f, double rho, const double u[3], double *K) {
    double s = 0.0;
    for (int i = 0; i < L->q; ++i) {
        double fe = feq_i(L, i, rho, u);
        if (!(fe > 0.0)) return ORC_EFEQ;
        s += fabs(f[i] - fe) / fe;
    }
    *K = s / L->q;
    return ORC_OK;
}

/* BGK collision of one cell, f_out = f - (f - feq) / tau, plus Guo's source term when a force is
 * given. */
static void collide_cell(const lattice_t *L, const orc_params *p, const double *f, double rho,
                         const double u[3], double *fout) {
    const double *F = p->force;
    for (int i = 0; i < L->q; ++i) {
        double fe = feq_i(L, i, rho, u);
        double out = f[i] - (f[i] - fe) / p->tau;
        if (F[0] != 0.0 || F[1] != 0.0 || F[2] != 0.0) {
            double cu = 0.0, s = 0.0;
            for (int a = 0; a < 3; ++a) cu += L->c[i][a] * u[a];
            for (int a = 0; a < 3; ++a)
                s += ((L->c[i][a] - u[a]) / CS2 + cu * L->c[i][a] / (CS2 * CS2)) * F[a];
            out += (1.0 - 0.5 / p->tau) * L->w[i] * s;
        }
        fout[i] = out;
    }
}

/* Lid term of the moving bounce-back: 2 w_i rho_w (c_i . u_w) / cs2, rho_w = 1. */
static double wall_term(const lattice_t *L, int i, const double uw[3]) {
    double cu = 0.0;
    for (int a = 0; a < 3; ++a) cu += L->c[i][a] * uw[a];
    return 2.0 * L->w[i] * 1.0 * cu / CS2;
}

/* Map a coordinate along an axis; returns 1 when it lies inside the lattice (after wrapping on a
 * periodic axis), 0 when it is a wall ghost. */
static int map_axis(int s, int n, int periodic, int *out) {
    if (periodic) {
        s = ((s % n) + n) % n;
        *out = s;
        return 1;
    }
    *out = s;
    return s >= 0 && s < n;
}

/* Ghost node velocity: the lid velocity for ghosts on the plane y == ny, rest otherwise. */
static void ghost_velocity(const orc_params *p, int sy, double uw[3]) {
    int lid = !(p->periodic & 2) && sy == p->ny;
    for (int a = 0; a < 3; ++a) uw[a] = lid ? p->lid[a] : 0.0;
}

/* Pull form: populations arriving at (x,y,z) for step t -> t+1 from the post-collision field fs. */
static void pull_cell(const lattice_t *L, const orc_params *p, const double *fs, int x, int y, int z,
                      double *f) {
    size_t N = ncells(p);
    for (int i = 0; i < L->q; ++i) {
        int sx, sy, sz;
        int in = map_axis(x - L->c[i][0], p->nx, p->periodic & 1, &sx);
        in &= map_axis(y - L->c[i][1], p->ny, p->periodic & 2, &sy);
        in &= map_axis(z - L->c[i][2], p->nz, p->periodic & 4, &sz);
        if (in) {
            f[i] = fs[(size_t)i * N + cell_index(p, sx, sy, sz)];
        } else {
            double uw[3];
            ghost_velocity(p, sy, uw);
            f[i] = fs[(size_t)L->opp[i] * N + cell_index(p, x, y, z)] + wall_term(L, i, uw);
        }
    }
}

/*
 * One full time step in pull form: stream (with bounce-back) from fs_in, then sensor, then collide
 * into fs_out.  Optional outputs (NULL to skip): K[cell] (sensor), rho[cell], u[3][cell] of the
 * pre-collision state.  fs_in and fs_out must not alias.
 */
int orc_step(const orc_params *p, const double *fs_in, double *fs_out, double *K, double *rho_out,
             double *u_out) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK) return ORC_EINVAL;
    size_t N = ncells(p);
    int status = ORC_OK;
    /* cells are independent within a step, so the planes may be shared among threads; the
     * arithmetic of each cell is unchanged */
#pragma omp parallel for schedule(static) reduction(min : status)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double f[ORC_MAXQ], fout[ORC_MAXQ], rho, u[3];
                size_t c = cell_index(p, x, y, z);
                pull_cell(&L, p, fs_in, x, y, z, f);
                moments(&L, f, p->force, &rho, u);
                if (K) {
                    double k;
                    if (sensor_cell(&L, f, rho, u, &k) != ORC_OK) status = ORC_EFEQ;
                    K[c] = k;
                }
                if (rho_out) rho_out[c] = rho;
                if (u_out)
                    for (int a = 0; a < 3; ++a) u_out[(size_t)a * N + c] = u[a];
                collide_cell(&L, p, f, rho, u, fout);
                for (int i = 0; i < L.q; ++i) fs_out[(size_t)i * N + c] = fout[i];
            }
    return status;
}

/*
 * The same step evaluated only at the listed cells (linear indices (z*ny + y)*nx + x): f_out[k*q + i]
 * receives the post-collision population i of cell cells[k], K[k] its sensor (K may be NULL).
 * Used to check sampled outputs of lattices too large to step in full.
 */
int orc_step_cells(const orc_params *p, const double *fs_in, long long ncell, const long long *cells,
                   double *f_out, double *K) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK || ncell < 0) return ORC_EINVAL;
    const long long N = (long long)ncells(p);
    int status = ORC_OK;
    for (long long k = 0; k < ncell; ++k)
        if (cells[k] < 0 || cells[k] >= N) return ORC_EINVAL;
#pragma omp parallel for schedule(static) reduction(min : status)
    for (long long k = 0; k < ncell; ++k) {
        const long long c = cells[k];
        const int x = (int)(c % p->nx);
        const int y = (int)((c / p->nx) % p->ny);
        const int z = (int)(c / ((long long)p->nx * p->ny));
        double f[ORC_MAXQ], fout[ORC_MAXQ], rho, u[3];
        pull_cell(&L, p, fs_in, x, y, z, f);
        moments(&L, f, p->force, &rho, u);
        if (K) {
            double kk;
            if (sensor_cell(&L, f, rho, u, &kk) != ORC_OK) status = ORC_EFEQ;
            K[k] = kk;
        }
        collide_cell(&L, p, f, rho, u, fout);
        for (int i = 0; i < L.q; ++i) f_out[k * L.q + i] = fout[i];
    }
    return status;
}

/* Number of threads the oracle's parallel loops use. */
int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the number of threads of the oracle's parallel loops (n >= 1); returns the previous count. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    const int old = omp_get_max_threads();
    if (n >= 1) omp_set_num_threads(n);
    return old;
#else
    (void)n;
    return 1;
#endif
}

/* Run n pull steps in place on fs (scratch holds the other buffer).  K (if given) receives the
 * sensor of the last step. */
int orc_run(const orc_params *p, double *fs, double *scratch, int n, double *K) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK || n < 0) return ORC_EINVAL;
    size_t bytes = (size_t)p->q * ncells(p) * sizeof(double);
    for (int t = 0; t < n; ++t) {
        int st = orc_step(p, fs, scratch, (t == n - 1) ? K : NULL, NULL, NULL);
        if (st != ORC_OK) return st;
        memcpy(fs, scratch, bytes);
    }
    return ORC_OK;
}

/* Push form, part 1: collide a pre-collision field f into f_out, with the sensor in K (optional). */
int orc_collide(const orc_params *p, const double *f, double *f_out, double *K) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK) return ORC_EINVAL;
    size_t N = ncells(p);
    int status = ORC_OK;
    for (size_t c = 0; c < N; ++c) {
        double fc[ORC_MAXQ], fo[ORC_MAXQ], rho, u[3];
        for (int i = 0; i < L.q; ++i) fc[i] = f[(size_t)i * N + c];
        moments(&L, fc, p->force, &rho, u);
        if (K) {
            double k;
            if (sensor_cell(&L, fc, rho, u, &k) != ORC_OK) status = ORC_EFEQ;
            K[c] = k;
        }
        collide_cell(&L, p, fc, rho, u, fo);
        for (int i = 0; i < L.q; ++i) f_out[(size_t)i * N + c] = fo[i];
    }
    return status;
}

/*
 * Push form, part 2: stream f_out(x) to x + c_i.  A population leaving towards a wall ghost comes
 * back to x in the opposite direction, minus the moving-wall term (Krueger's moving bounce-back).
 */
int orc_stream_push(const orc_params *p, const double *f_out, double *f_next) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK) return ORC_EINVAL;
    size_t N = ncells(p);
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t c = cell_index(p, x, y, z);
                for (int i = 0; i < L.q; ++i) {
                    int dx, dy, dz;
                    int in = map_axis(x + L.c[i][0], p->nx, p->periodic & 1, &dx);
                    in &= map_axis(y + L.c[i][1], p->ny, p->periodic & 2, &dy);
                    in &= map_axis(z + L.c[i][2], p->nz, p->periodic & 4, &dz);
                    double v = f_out[(size_t)i * N + c];
                    if (in) {
                        f_next[(size_t)i * N + cell_index(p, dx, dy, dz)] = v;
                    } else {
                        double uw[3];
                        ghost_velocity(p, dy, uw);
                        f_next[(size_t)L.opp[i] * N + c] = v - wall_term(&L, i, uw);
                    }
                }
            }
    return ORC_OK;
}

/* Sensor and moments of a given pre-collision field (no streaming, no collision). */
int orc_sensor(const orc_params *p, const double *f, double *K, double *rho_out, double *u_out) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK) return ORC_EINVAL;
    size_t N = ncells(p);
    int status = ORC_OK;
    for (size_t c = 0; c < N; ++c) {
        double fc[ORC_MAXQ], rho, u[3];
        for (int i = 0; i < L.q; ++i) fc[i] = f[(size_t)i * N + c];
        moments(&L, fc, p->force, &rho, u);
        if (K) {
            double k;
            if (sensor_cell(&L, fc, rho, u, &k) != ORC_OK) status = ORC_EFEQ;
            K[c] = k;
        }
        if (rho_out) rho_out[c] = rho;
        if (u_out)
            for (int a = 0; a < 3; ++a) u_out[(size_t)a * N + c] = u[a];
    }
    return status;
}

/* Equilibrium field f_i = feq_i(rho, u) for given rho[cell], u[3][cell]. */
int orc_equilibrium(const orc_params *p, const double *rho, const double *u, double *f) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK) return ORC_EINVAL;
    size_t N = ncells(p);
    for (size_t c = 0; c < N; ++c) {
        double uc[3] = {u[c], u[N + c], u[2 * N + c]};
        for (int i = 0; i < L.q; ++i) f[(size_t)i * N + c] = feq_i(&L, i, rho[c], uc);
    }
    return ORC_OK;
}

/*
 * Block maximum of a per-cell field K[nz][ny][nx] over blocks of edge b (2-D lattices: b x b,
 * nz == 1), starting at the origin; partial blocks at the high ends take the max of the cells they
 * have.  out has ceil(nx/b)*ceil(ny/b)*ceil(nz/b) entries, x fastest.  A NaN in a block makes that
 * block's max NaN.
 */
int orc_block_max(const double *K, int nx, int ny, int nz, int b, double *out) {
    if (nx < 1 || ny < 1 || nz < 1 || b < 1) return ORC_EINVAL;
    int bx = (nx + b - 1) / b, by = (ny + b - 1) / b, bz = (nz + b - 1) / b;
    for (int k = 0; k < bx * by * bz; ++k) out[k] = -INFINITY;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double v = K[((size_t)z * ny + y) * nx + x];
                int k = ((z / b) * by + (y / b)) * bx + (x / b);
                if (isnan(v) || isnan(out[k]))
                    out[k] = NAN;
                else if (v > out[k])
                    out[k] = v;
            }
    return ORC_OK;
}

/* Total mass sum_x sum_i f_i and momentum sum_x sum_i c_i f_i of a field. */
int orc_conservation(const orc_params *p, const double *f, double *mass, double *mom) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK) return ORC_EINVAL;
    size_t N = ncells(p);
    double m = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L.q; ++i)
        for (size_t c = 0; c < N; ++c) {
            double v = f[(size_t)i * N + c];
            m += v;
            for (int a = 0; a < 3; ++a) j[a] += L.c[i][a] * v;
        }
    *mass = m;
    for (int a = 0; a < 3; ++a) mom[a] = j[a];
    return ORC_OK;
}
