/*
 * Plain FP64 CPU oracle of the multi-level block-structured lattice Boltzmann step (D3Q19).
 *
 * TEST INFRASTRUCTURE ONLY: the checker of the CUDA multi-level path; it shares no code with it.
 *
 * The paper (Sec. 2.1 and Sec. 5.2) runs its refined meshes in cell-centred block-structured AMR
 * with refinement ratio 2 and acoustic scaling (dx/dt the same on every level): levels are
 * sub-cycled, coupled at their interfaces by linear temporal and second-order spatial
 * interpolation, with the non-equilibrium part of the populations rescaled between levels
 * (Dupuis & Chopard).  The paper prints no formulas for these steps; this file fixes one reading
 * of them, written the plain way:
 *
 *   - the domain is a grid of physical blocks of edge E (finest cells); every block has a leaf
 *     level 0..Lmax; level l exists on every block whose leaf level is >= l (levels nest, level 0
 *     covers the domain), with cells of edge h_l = 2^(Lmax - l) finest cells;
 *   - blocks whose leaf levels differ by more than one may not touch (faces, edges or corners);
 *   - acoustic scaling: level l steps with dt_l = h_l, so it takes 2^l steps per level-0 step
 *     (a "cycle"); the lattice viscosity follows nu_l = nu_Lmax / h_l (nu = c_s^2 (tau - 1/2),
 *     Eq. nu_omega), so tau_l = 3 nu_Lmax / h_l + 1/2;
 *   - a level step is the uniform pull step (streaming with moving-wall bounce-back, moments,
 *     equilibrium, sensor, BGK collision) of every block of the level, reading a one-cell ghost
 *     layer;
 *   - ghost cells inside another block of the same level are copies of that block's cells; ghost
 *     cells outside the level's region are interpolated from the next coarser level at the fine
 *     level's time: trilinear in space (the eight coarse cells around the ghost cell centre,
 *     weights 3/4 and 1/4 per axis; linear extrapolation with 5/4 and -1/4 where a neighbour lies
 *     outside the domain) and linear in time between the coarse level's states before and after
 *     its step;
 *   - interpolated post-collision populations are split into equilibrium (from their own rho, u)
 *     and non-equilibrium parts, the latter multiplied by (tau_f - 1) / (2 (tau_c - 1)) going
 *     coarse -> fine: the post-collision f^neq is (1 - 1/tau) f^neq_pre and f^neq_pre scales like
 *     tau dt (Chapman-Enskog, Eq. generalf1);
 *   - after the two sub-steps of level l + 1, the level-l cells under level l + 1 are replaced by
 *     the average of their 2^3 fine cells, the non-equilibrium part rescaled by
 *     2 (tau_c - 1) / (tau_f - 1);
 *   - the sensor of a block is the maximum of K over its leaf-level cells at that level's last
 *     sub-step of the cycle.
 *
 * Layout of a block's level array: f[i][k][j][i_x] over the (n + 2)^3 cells including the ghost
 * layer (ghost index -1 stored at 0), n = E / h_l.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MLQ 19
static const int MC[MLQ][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double MW[MLQ] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double MCS2 = 1.0 / 3.0;

#define ML_MAXL 3

typedef struct {
    int nb[3];        /* physical blocks per axis */
    int edge;         /* block edge in finest cells */
    int lmax;         /* finest level (0..2) */
    double tau_fine;  /* relaxation time of level lmax */
    double lid[3];    /* lid velocity (y component 0) */
    int periodic;     /* bit 0 x, bit 1 y, bit 2 z */
} ml_desc;

typedef struct {
    ml_desc d;
    int nblk;
    int8_t *leaf;               /* leaf level per physical block */
    int opp[MLQ];
    /* per level */
    int n[ML_MAXL];             /* cells per block edge */
    int cells[ML_MAXL][3];      /* cells per domain axis */
    double tau[ML_MAXL];
    int *slot[ML_MAXL];         /* physical block -> slot in the level, or -1 */
    int nslot[ML_MAXL];
    double *cur[ML_MAXL];       /* post-collision state, ghosted, per slot */
    double *prev[ML_MAXL];      /* state before the level's last step (time interpolation) */
    double *K[ML_MAXL];         /* sensor per cell of the last step, per slot, n^3 */
    long long steps[ML_MAXL];
    int frozen_time;            /* test hook: 1 = theta 0 on both sub-steps (a planted mistake) */
} ml_mesh;

#define ML_OK 0
#define ML_EINVAL -1
#define ML_ENOMEM -2

static size_t gsize(int n) { return (size_t)(n + 2) * (n + 2) * (n + 2); }
static size_t blk_len(int n) { return (size_t)MLQ * gsize(n); }
/* index of population i at ghosted local cell (x, y, z) in [-1, n] */
static size_t gidx(int n, int i, int x, int y, int z) {
    return (size_t)i * gsize(n) + (((size_t)(z + 1) * (n + 2) + (y + 1)) * (n + 2) + (x + 1));
}

static double feq(int i, double rho, const double u[3]) {
    double cu = 0.0, uu = 0.0;
    for (int a = 0; a < 3; ++a) {
        cu += MC[i][a] * u[a];
        uu += u[a] * u[a];
    }
    return MW[i] * rho * (1.0 + cu / MCS2 + (cu * cu - MCS2 * uu) / (2.0 * MCS2 * MCS2));
}

static void moments(const double *f, double *rho, double u[3]) {
    double r = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < MLQ; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) j[a] += MC[i][a] * f[i];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = j[a] / r;
}

/* physical block of a level-l global cell index (after periodic wrapping); -1 outside */
static int wrap_axis(const ml_mesh *m, int l, int a, int g) {
    const int n = m->cells[l][a];
    if (g >= 0 && g < n) return g;
    if (m->d.periodic & (1 << a)) return ((g % n) + n) % n;
    return -1;
}

static int block_of(const ml_mesh *m, int l, const int g[3], int local[3]) {
    int b[3];
    for (int a = 0; a < 3; ++a) {
        b[a] = g[a] / m->n[l];
        local[a] = g[a] - b[a] * m->n[l];
    }
    return (b[2] * m->d.nb[1] + b[1]) * m->d.nb[0] + b[0];
}

void ml_destroy(ml_mesh *m) {
    if (!m) return;
    for (int l = 0; l < ML_MAXL; ++l) {
        free(m->slot[l]);
        free(m->cur[l]);
        free(m->prev[l]);
        free(m->K[l]);
    }
    free(m->leaf);
    free(m);
}

/* Check the 2:1 rule between touching blocks (26-neighbourhood, periodic wrap). */
static int balanced(const ml_desc *d, const int8_t *leaf) {
    for (int z = 0; z < d->nb[2]; ++z)
        for (int y = 0; y < d->nb[1]; ++y)
            for (int x = 0; x < d->nb[0]; ++x) {
                const int b = (z * d->nb[1] + y) * d->nb[0] + x;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int c[3] = {x + dx, y + dy, z + dz}, ok = 1;
                            for (int a = 0; a < 3; ++a) {
                                if (c[a] < 0 || c[a] >= d->nb[a]) {
                                    if (d->periodic & (1 << a))
                                        c[a] = (c[a] + d->nb[a]) % d->nb[a];
                                    else
                                        ok = 0;
                                }
                            }
                            if (!ok) continue;
                            const int nbk = (c[2] * d->nb[1] + c[1]) * d->nb[0] + c[0];
                            if (abs(leaf[b] - leaf[nbk]) > 1) return 0;
                        }
            }
    return 1;
}

/* Build a mesh at rest (f = w_i on every level).  Returns NULL and *status on failure. */
ml_mesh *ml_create(const ml_desc *d, const int8_t *leaf, int *status) {
    *status = ML_EINVAL;
    if (d->lmax < 0 || d->lmax >= ML_MAXL || d->edge < 1) return NULL;
    if (d->edge % (1 << d->lmax) != 0 || d->edge / (1 << d->lmax) < 2) return NULL;
    if (!(d->tau_fine > 0.5) || d->lid[1] != 0.0) return NULL;
    for (int a = 0; a < 3; ++a)
        if (d->nb[a] < 1) return NULL;
    const int nblk = d->nb[0] * d->nb[1] * d->nb[2];
    for (int b = 0; b < nblk; ++b)
        if (leaf[b] < 0 || leaf[b] > d->lmax) return NULL;
    if (!balanced(d, leaf)) return NULL;
    ml_mesh *m = (ml_mesh *)calloc(1, sizeof(ml_mesh));
    if (!m) {
        *status = ML_ENOMEM;
        return NULL;
    }
    m->d = *d;
    m->nblk = nblk;
    m->leaf = (int8_t *)malloc(nblk);
    memcpy(m->leaf, leaf, nblk);
    for (int i = 0; i < MLQ; ++i)
        for (int j = 0; j < MLQ; ++j)
            if (MC[j][0] == -MC[i][0] && MC[j][1] == -MC[i][1] && MC[j][2] == -MC[i][2])
                m->opp[i] = j;
    const double nu_fine = (d->tau_fine - 0.5) / 3.0;
    for (int l = 0; l <= d->lmax; ++l) {
        const int h = 1 << (d->lmax - l);
        m->n[l] = d->edge / h;
        for (int a = 0; a < 3; ++a) m->cells[l][a] = d->nb[a] * m->n[l];
        m->tau[l] = 3.0 * nu_fine / h + 0.5;
        if (d->lmax > 0 && fabs(m->tau[l] - 1.0) < 1e-3) {
            ml_destroy(m);
            return NULL; /* the rescaling factors divide by tau - 1 */
        }
        m->slot[l] = (int *)malloc(sizeof(int) * nblk);
        int ns = 0;
        for (int b = 0; b < nblk; ++b) m->slot[l][b] = (leaf[b] >= l) ? ns++ : -1;
        m->nslot[l] = ns;
        const size_t len = blk_len(m->n[l]) * ns;
        m->cur[l] = (double *)malloc(sizeof(double) * len);
        m->prev[l] = (double *)malloc(sizeof(double) * len);
        m->K[l] = (double *)calloc((size_t)ns * m->n[l] * m->n[l] * m->n[l], sizeof(double));
        if (!m->cur[l] || !m->prev[l] || !m->K[l]) {
            ml_destroy(m);
            *status = ML_ENOMEM;
            return NULL;
        }
        for (int s = 0; s < ns; ++s)
            for (int i = 0; i < MLQ; ++i)
                for (size_t c = 0; c < gsize(m->n[l]); ++c) {
                    m->cur[l][s * blk_len(m->n[l]) + i * gsize(m->n[l]) + c] = MW[i];
                    m->prev[l][s * blk_len(m->n[l]) + i * gsize(m->n[l]) + c] = MW[i];
                }
    }
    *status = ML_OK;
    return m;
}

/* Populations of level l at global cell g (must lie in the level's region), state `which`:
 * 0 = prev, 1 = cur. */
static void level_cell(const ml_mesh *m, int l, const int g[3], int which, double *f) {
    int loc[3];
    const int b = block_of(m, l, g, loc);
    const int s = m->slot[l][b];
    const double *base = (which ? m->cur[l] : m->prev[l]) + (size_t)s * blk_len(m->n[l]);
    for (int i = 0; i < MLQ; ++i) f[i] = base[gidx(m->n[l], i, loc[0], loc[1], loc[2])];
}

/* Fill every face and edge ghost cell of level l at time fraction theta of the parent step. */
static int fill_ghosts(ml_mesh *m, int l, double theta) {
    const int n = m->n[l];
    for (int b = 0; b < m->nblk; ++b) {
        const int s = m->slot[l][b];
        if (s < 0) continue;
        const int bz = b / (m->d.nb[0] * m->d.nb[1]), by = (b / m->d.nb[0]) % m->d.nb[1],
                  bx = b % m->d.nb[0];
        double *dst = m->cur[l] + (size_t)s * blk_len(n);
        for (int z = -1; z <= n; ++z)
            for (int y = -1; y <= n; ++y)
                for (int x = -1; x <= n; ++x) {
                    const int out = (x < 0 || x >= n) + (y < 0 || y >= n) + (z < 0 || z >= n);
                    if (out == 0 || out == 3) continue; /* interior, or a corner (unused) */
                    int g[3] = {bx * n + x, by * n + y, bz * n + z}, inside = 1;
                    for (int a = 0; a < 3; ++a) {
                        const int w = wrap_axis(m, l, a, g[a]);
                        if (w < 0)
                            inside = 0;
                        else
                            g[a] = w;
                    }
                    if (!inside) continue; /* a wall: the step bounces back */
                    double f[MLQ];
                    int loc[3];
                    const int nbk = block_of(m, l, g, loc);
                    if (m->slot[l][nbk] >= 0) {
                        level_cell(m, l, g, 1, f);
                    } else {
                        if (l == 0) return ML_EINVAL;
                        /* interpolate from level l-1: ghost centre (g + 1/2) h_l, in coarse cells
                         * g/2 + 1/4; coarse cell c = g >> 1, offset -1/4 (g even) or +1/4 */
                        const int lc = l - 1;
                        int c0[3], c1[3];
                        double w0[3], w1[3];
                        for (int a = 0; a < 3; ++a) {
                            const int c = g[a] >> 1;
                            const int dir = (g[a] & 1) ? 1 : -1;
                            int nb = c + dir;
                            if (wrap_axis(m, lc, a, nb) >= 0) {
                                c0[a] = c;
                                c1[a] = wrap_axis(m, lc, a, nb);
                                w0[a] = 0.75;
                                w1[a] = 0.25;
                            } else {
                                c0[a] = c;
                                c1[a] = wrap_axis(m, lc, a, c - dir);
                                w0[a] = 1.25;
                                w1[a] = -0.25;
                            }
                        }
                        double acc[MLQ];
                        for (int i = 0; i < MLQ; ++i) acc[i] = 0.0;
                        for (int k = 0; k < 8; ++k) {
                            int cc[3];
                            double wt = 1.0;
                            for (int a = 0; a < 3; ++a) {
                                const int bit = (k >> a) & 1;
                                cc[a] = bit ? c1[a] : c0[a];
                                wt *= bit ? w1[a] : w0[a];
                            }
                            int cl[3];
                            if (m->slot[lc][block_of(m, lc, cc, cl)] < 0) return ML_EINVAL;
                            double fo[MLQ], fn[MLQ];
                            level_cell(m, lc, cc, 0, fo);
                            level_cell(m, lc, cc, 1, fn);
                            for (int i = 0; i < MLQ; ++i)
                                acc[i] += wt * ((1.0 - theta) * fo[i] + theta * fn[i]);
                        }
                        double rho, u[3];
                        moments(acc, &rho, u);
                        const double sc = (m->tau[l] - 1.0) / (2.0 * (m->tau[lc] - 1.0));
                        for (int i = 0; i < MLQ; ++i) {
                            const double fe = feq(i, rho, u);
                            f[i] = fe + sc * (acc[i] - fe);
                        }
                    }
                    for (int i = 0; i < MLQ; ++i) dst[gidx(n, i, x, y, z)] = f[i];
                }
    }
    return ML_OK;
}

/* One pull step of every block of level l (ghosts filled): prev <- cur, cur <- new state. */
static void step_level(ml_mesh *m, int l) {
    const int n = m->n[l];
    const double tau = m->tau[l];
    const size_t len = blk_len(n) * m->nslot[l];
    memcpy(m->prev[l], m->cur[l], sizeof(double) * len);
    for (int b = 0; b < m->nblk; ++b) {
        const int s = m->slot[l][b];
        if (s < 0) continue;
        const int bz = b / (m->d.nb[0] * m->d.nb[1]), by = (b / m->d.nb[0]) % m->d.nb[1],
                  bx = b % m->d.nb[0];
        const double *src = m->prev[l] + (size_t)s * blk_len(n);
        double *dst = m->cur[l] + (size_t)s * blk_len(n);
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x) {
                    double f[MLQ];
                    for (int i = 0; i < MLQ; ++i) {
                        const int sx = x - MC[i][0], sy = y - MC[i][1], sz = z - MC[i][2];
                        const int gs[3] = {bx * n + sx, by * n + sy, bz * n + sz};
                        int wall = 0, lid = 0;
                        for (int a = 0; a < 3; ++a) {
                            if (wrap_axis(m, l, a, gs[a]) < 0) {
                                wall = 1;
                                if (a == 1 && gs[1] == m->cells[l][1]) lid = 1;
                            }
                        }
                        if (!wall) {
                            f[i] = src[gidx(n, i, sx, sy, sz)];
                        } else {
                            /* moving-wall bounce-back; a ghost on the plane y = ny moves with the
                             * lid (edge and corner ghosts included), rho_w = 1 */
                            double cu = 0.0;
                            if (gs[1] == m->cells[l][1] && !(m->d.periodic & 2)) lid = 1;
                            if (lid)
                                for (int a = 0; a < 3; ++a) cu += MC[i][a] * m->d.lid[a];
                            f[i] = src[gidx(n, m->opp[i], x, y, z)] + 2.0 * MW[i] * cu / MCS2;
                        }
                    }
                    double rho, u[3];
                    moments(f, &rho, u);
                    double k = 0.0;
                    for (int i = 0; i < MLQ; ++i) {
                        const double fe = feq(i, rho, u);
                        k += fabs(f[i] - fe) / fe;
                        dst[gidx(n, i, x, y, z)] = f[i] - (f[i] - fe) / tau;
                    }
                    m->K[l][(size_t)s * n * n * n + ((size_t)z * n + y) * n + x] = k / MLQ;
                }
    }
    m->steps[l] += 1;
}

/* Replace the level-l cells under level l + 1 by the restriction of the fine state. */
static void restrict_level(ml_mesh *m, int l) {
    const int n = m->n[l], nf = m->n[l + 1];
    const double sc = 2.0 * (m->tau[l] - 1.0) / (m->tau[l + 1] - 1.0);
    for (int b = 0; b < m->nblk; ++b) {
        const int sf = m->slot[l + 1][b];
        if (sf < 0) continue;
        const int s = m->slot[l][b];
        double *dst = m->cur[l] + (size_t)s * blk_len(n);
        const double *fine = m->cur[l + 1] + (size_t)sf * blk_len(nf);
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x) {
                    double avg[MLQ];
                    for (int i = 0; i < MLQ; ++i) {
                        double a = 0.0;
                        for (int k = 0; k < 8; ++k)
                            a += fine[gidx(nf, i, 2 * x + (k & 1), 2 * y + ((k >> 1) & 1),
                                           2 * z + ((k >> 2) & 1))];
                        avg[i] = a / 8.0;
                    }
                    double rho, u[3];
                    moments(avg, &rho, u);
                    for (int i = 0; i < MLQ; ++i) {
                        const double fe = feq(i, rho, u);
                        dst[gidx(n, i, x, y, z)] = fe + sc * (avg[i] - fe);
                    }
                }
    }
}

static int advance(ml_mesh *m, int l, double theta) {
    int st = fill_ghosts(m, l, theta);
    if (st != ML_OK) return st;
    step_level(m, l);
    if (l < m->d.lmax) {
        /* the fine level's two sub-steps start at the coarse step's start and half-way through
         * it: its ghosts are interpolated linearly in time at theta = 0 and 1/2 */
        st = advance(m, l + 1, 0.0);
        if (st == ML_OK) st = advance(m, l + 1, m->frozen_time ? 0.0 : 0.5);
        if (st != ML_OK) return st;
        restrict_level(m, l);
    }
    return ML_OK;
}

/* Test hook for the pin of the temporal interpolation: mode 1 plants a mistake, filling the
 * ghosts of every second fine sub-step from the coarse state before the coarse step (theta = 0 on
 * both sub-steps, a coarse level frozen in time); mode 0 (the default) is the linear reading. */
int ml_set_time_interp(ml_mesh *m, int mode) {
    if (mode != 0 && mode != 1) return ML_EINVAL;
    m->frozen_time = mode;
    return ML_OK;
}

/* Advance `cycles` level-0 steps. */
int ml_cycles(ml_mesh *m, int cycles) {
    for (int c = 0; c < cycles; ++c) {
        int st = advance(m, 0, 0.0);
        if (st != ML_OK) return st;
    }
    return ML_OK;
}

/* Per physical block: max of K over its leaf-level cells at that level's last step. */
int ml_block_max(const ml_mesh *m, double *out) {
    for (int b = 0; b < m->nblk; ++b) {
        const int l = m->leaf[b], n = m->n[l], s = m->slot[l][b];
        double mx = -INFINITY;
        for (int c = 0; c < n * n * n; ++c) {
            const double k = m->K[l][(size_t)s * n * n * n + c];
            if (isnan(k) || isnan(mx))
                mx = NAN;
            else if (k > mx)
                mx = k;
        }
        out[b] = mx;
    }
    return ML_OK;
}

/* Interior populations of physical block b at level l (n^3 cells, f[i][z][y][x]). */
int ml_get_block(const ml_mesh *m, int l, int b, double *out) {
    if (l < 0 || l > m->d.lmax || b < 0 || b >= m->nblk || m->slot[l][b] < 0) return ML_EINVAL;
    const int n = m->n[l], s = m->slot[l][b];
    const double *src = m->cur[l] + (size_t)s * blk_len(n);
    for (int i = 0; i < MLQ; ++i)
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x)
                    out[(((size_t)i * n + z) * n + y) * n + x] = src[gidx(n, i, x, y, z)];
    return ML_OK;
}

/* Set the interior populations of block b at level l (the ghosts are refilled before use). */
int ml_set_block(ml_mesh *m, int l, int b, const double *in) {
    if (l < 0 || l > m->d.lmax || b < 0 || b >= m->nblk || m->slot[l][b] < 0) return ML_EINVAL;
    const int n = m->n[l], s = m->slot[l][b];
    double *dst = m->cur[l] + (size_t)s * blk_len(n);
    for (int i = 0; i < MLQ; ++i)
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x)
                    dst[gidx(n, i, x, y, z)] = in[(((size_t)i * n + z) * n + y) * n + x];
    return ML_OK;
}

int ml_level_info(const ml_mesh *m, int l, int *n, double *tau) {
    if (l < 0 || l > m->d.lmax) return ML_EINVAL;
    *n = m->n[l];
    *tau = m->tau[l];
    return ML_OK;
}
