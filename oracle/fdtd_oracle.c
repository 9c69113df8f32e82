/*
 * FP64 CPU oracle of the acoustic FDTD path — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this library. It shares no code with the CUDA library; see oracle.h for the
 * scheme. Every routine follows the paper's equations in their order, with no
 * blocking or fusion: one plain pass per term, OpenMP over rows only where the
 * pass is a pure gather (no change of arithmetic order per cell).
 *
 * Readings of what the paper leaves open (the design notes list each one too):
 *  R1 time discretisation: centred 2nd-order leapfrog; the damping term
 *     eta p_t is centred too: eta (p^{n+1} - p^{n-1}) / (2 dt)   (Eq. cerjan_pde)
 *  R2 sponge units: eta_SI = 1e-3 s/m * (c_damp/h) [rho - sin(2 pi rho)/(2 pi)]
 *     (Eq. cerjan_damp is written in km/s and ms units); rho = j/nb for the
 *     j-th absorbing cell outward (j = 1..nb); corner eta = sum over axes.
 *  R3 CPML (the paper uses a sponge; CPML is an added option): unsplit
 *     recursive-convolution form for the second-order equation, kappa = 1,
 *     d = d0 rho^2, d0 = 3 vmax ln(1/R) / (2 nb h), alpha = pi f_ref (1 - rho),
 *     b = exp(-(d + alpha) dt), a = d (b - 1) / (d + alpha);
 *        psi^n  = b psi^{n-1}  + a D1 p^n
 *        zeta^n = b zeta^{n-1} + a (D2 p^n + D1 psi^n)
 *        axis term = D2 p^n + D1 psi^n + zeta^n
 *  R4 free surface (Eq. free_surface): row z = 0 is held at p = 0; ghost rows
 *     above it mirror the field with odd sign, p(-k) = -p(k).
 *  R5 outside the padded grid p = 0 (Dirichlet ghosts).
 *  R6 point source s = w(t_n) delta(x - x_s), discretised as w/h^d spread with
 *     bi/tri-linear weights; injected in the step n -> n+1. Receivers sample
 *     p^n with the same weights (gather row n). A coordinate within 1e-6 cells
 *     of a grid line snaps to it.
 *  R7 velocity in the absorbing layers = nearest interior cell (edge
 *     replication); the velocity gradient folds those cells back onto the
 *     interior edge cells.
 *  R8 misfit J = 1/2 sum_{n,r} (g[n,r] - d[n,r])^2 (no dt weight); gradient is
 *     the exact derivative of the discrete map (discretise, then differentiate).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Central second-derivative weights of order 8 (M = 4), m = 0..4 (App. E.3.1,
 * Fornberg 1988): the unique weights exact on x^{2j}, j <= 4. */
static const double D2W[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0,
                              8.0 / 315.0, -1.0 / 560.0};
/* Central first-derivative weights of order 8, m = 1..4 (CPML reading R3). */
static const double D1W[5] = {0.0, 4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0,
                              -1.0 / 280.0};

typedef struct {
    int NZ, NY, NX;
    long ncell;
} grid_t;

#define IDX(G, z, y, x) ((((long)(z)) * (G)->NY + (y)) * (G)->NX + (x))

static double rpart(real_t v) {
#ifdef ORACLE_COMPLEX
    return creal(v);
#else
    return v;
#endif
}

static int make_grid(const or_params *P, grid_t *G) {
    if (!P || (P->ndim != 2 && P->ndim != 3)) return -1;
    if (P->nz < 1 || P->nx < 1 || P->ny < 1) return -1;
    if (P->ndim == 2 && P->ny != 1) return -1;
    if (!(P->h > 0) || !(P->dt > 0) || P->nt < 0) return -1;
    for (int k = 0; k < 6; k++)
        if (P->nb[k] < 0) return -1;
    if (P->free_surface && P->nb[0] != 0) return -1;
    if (P->bc < 0 || P->bc > 2) return -1;
    G->NZ = P->nb[0] + P->nz + P->nb[1];
    G->NY = P->ndim == 3 ? P->nb[2] + P->ny + P->nb[3] : 1;
    G->NX = P->nb[4] + P->nx + P->nb[5];
    G->ncell = (long)G->NZ * G->NY * G->NX;
    return 0;
}

/* Number of OpenMP threads the passes run on (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int oracle_padded_dims(const or_params *P, int dims[3]) {
    grid_t G;
    if (make_grid(P, &G)) return -1;
    dims[0] = G.NZ;
    dims[1] = G.NY;
    dims[2] = G.NX;
    return 0;
}

static int nsnap_of(const or_params *P) {
    if (P->snap_every <= 0) return 0;
    int end = P->snap_end < P->nt ? P->snap_end : P->nt;
    if (end <= P->snap_begin || P->snap_begin < 0) return 0;
    return (end - P->snap_begin + P->snap_every - 1) / P->snap_every;
}

/* Field value with the ghost rules R4 (odd mirror above a free surface) and
 * R5 (zero outside the padded grid). */
static real_t get(const or_params *P, const grid_t *G, const real_t *p, int z,
                  int y, int x) {
    if (x < 0 || x >= G->NX || y < 0 || y >= G->NY || z >= G->NZ) return 0;
    if (z < 0) {
        if (!P->free_surface) return 0;
        return -get(P, G, p, -z, y, x);
    }
    return p[IDX(G, z, y, x)];
}

/* Unit step along axis: 0 = z, 1 = y, 2 = x. */
static void axis_step(int ax, int m, int *dz, int *dy, int *dx) {
    *dz = ax == 0 ? m : 0;
    *dy = ax == 1 ? m : 0;
    *dx = ax == 2 ? m : 0;
}

/* Second derivative along one axis, 8th order. */
static real_t d2_axis(const or_params *P, const grid_t *G, const real_t *p,
                      int ax, int z, int y, int x) {
    real_t s = D2W[0] * get(P, G, p, z, y, x);
    for (int m = 1; m <= 4; m++) {
        int dz, dy, dx;
        axis_step(ax, m, &dz, &dy, &dx);
        s += D2W[m] * (get(P, G, p, z + dz, y + dy, x + dx) +
                       get(P, G, p, z - dz, y - dy, x - dx));
    }
    return s / (P->h * P->h);
}

/* First derivative along one axis, 8th order. */
static real_t d1_axis(const or_params *P, const grid_t *G, const real_t *p,
                      int ax, int z, int y, int x) {
    real_t s = 0;
    for (int m = 1; m <= 4; m++) {
        int dz, dy, dx;
        axis_step(ax, m, &dz, &dy, &dx);
        s += D1W[m] * (get(P, G, p, z + dz, y + dy, x + dx) -
                       get(P, G, p, z - dz, y - dy, x - dx));
    }
    return s / P->h;
}

static int axis_active(const or_params *P, int ax) {
    return P->ndim == 3 || ax != 1;
}

/* (L p)_i: the Laplacian as the sum of the per-axis second derivatives. */
static real_t lap_at(const or_params *P, const grid_t *G, const real_t *p,
                     int z, int y, int x) {
    real_t s = 0;
    for (int ax = 0; ax < 3; ax++)
        if (axis_active(P, ax)) s += d2_axis(P, G, p, ax, z, y, x);
    return s;
}

/* Axis length and low/high absorbing widths. */
static void axis_layout(const or_params *P, const grid_t *G, int ax, int *N,
                        int *nlo, int *nhi) {
    if (ax == 0) {
        *N = G->NZ;
        *nlo = P->nb[0];
        *nhi = P->nb[1];
    } else if (ax == 1) {
        *N = G->NY;
        *nlo = P->ndim == 3 ? P->nb[2] : 0;
        *nhi = P->ndim == 3 ? P->nb[3] : 0;
    } else {
        *N = G->NX;
        *nlo = P->nb[4];
        *nhi = P->nb[5];
    }
}

/* Normalised depth rho = j/nb into the layer of index i (0 outside). */
static double layer_rho(int N, int nlo, int nhi, int i, int *width) {
    if (i < nlo) {
        *width = nlo;
        return (double)(nlo - i) / nlo;
    }
    if (i >= N - nhi) {
        *width = nhi;
        return (double)(i - (N - nhi) + 1) / nhi;
    }
    *width = 0;
    return 0.0;
}

/* Sponge damping eta(x) of one axis in SI units (Eq. cerjan_damp, reading R2). */
static double sponge_eta(const or_params *P, int N, int nlo, int nhi, int i) {
    int w;
    double rho = layer_rho(N, nlo, nhi, i, &w);
    if (w == 0) return 0.0;
    double cdamp = 1.5 * log(1.0 / P->R) / w;
    return 1e-3 * (cdamp / P->h) * (rho - sin(2.0 * M_PI * rho) / (2.0 * M_PI));
}

/* CPML recursion coefficients of one axis index (reading R3). */
static void cpml_coef(const or_params *P, double vmax, int N, int nlo, int nhi,
                      int i, double *a, double *b) {
    int w;
    double rho = layer_rho(N, nlo, nhi, i, &w);
    if (w == 0) {
        *a = 0.0;
        *b = 0.0;
        return;
    }
    double d0 = 3.0 * vmax * log(1.0 / P->R) / (2.0 * w * P->h);
    double d = d0 * rho * rho;
    double alpha = M_PI * P->f_ref * (1.0 - rho);
    *b = exp(-(d + alpha) * P->dt);
    *a = d * (*b - 1.0) / (d + alpha);
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Padded velocity by edge replication (reading R7). */
static real_t vel_pad(const or_params *P, const real_t *vel, int z, int y, int x) {
    int iz = clampi(z - P->nb[0], 0, P->nz - 1);
    int iy = P->ndim == 3 ? clampi(y - P->nb[2], 0, P->ny - 1) : 0;
    int ix = clampi(x - P->nb[4], 0, P->nx - 1);
    return vel[((long)iz * P->ny + iy) * P->nx + ix];
}

static double model_vmax(const or_params *P, const real_t *vel) {
    double m = 0;
    long n = (long)P->nz * P->ny * P->nx;
    for (long i = 0; i < n; i++)
        if (rpart(vel[i]) > m) m = rpart(vel[i]);
    return m;
}

/* Per-cell c = v^2 dt^2, a = eta v^2 dt / 2 and eta (sponge only). */
static void build_coefficients(const or_params *P, const grid_t *G,
                               const real_t *vel, real_t *c, real_t *a,
                               double *eta) {
    int N[3], lo[3], hi[3];
    for (int ax = 0; ax < 3; ax++) axis_layout(P, G, ax, &N[ax], &lo[ax], &hi[ax]);
    for (int z = 0; z < G->NZ; z++)
        for (int y = 0; y < G->NY; y++)
            for (int x = 0; x < G->NX; x++) {
                long i = IDX(G, z, y, x);
                real_t v = vel_pad(P, vel, z, y, x);
                double e = 0.0;
                if (P->bc == 0) {
                    e += sponge_eta(P, N[0], lo[0], hi[0], z);
                    if (P->ndim == 3) e += sponge_eta(P, N[1], lo[1], hi[1], y);
                    e += sponge_eta(P, N[2], lo[2], hi[2], x);
                }
                c[i] = v * v * P->dt * P->dt;
                a[i] = e * v * v * P->dt / 2.0;
                if (eta) eta[i] = e;
            }
}

/* Linear-interpolation stencil of a point (reading R6). Position order is
 * (x, z) in 2D and (x, y, z) in 3D, metres from the interior origin. */
static int point_stencil(const or_params *P, const grid_t *G, const double *pos,
                         long *cell, double *w) {
    double f[3];
    int lo[3], len[3];
    int ncoord = P->ndim;
    /* axis 0 = z, 1 = y, 2 = x */
    f[2] = pos[0] / P->h + P->nb[4];
    f[0] = pos[ncoord - 1] / P->h + P->nb[0];
    f[1] = P->ndim == 3 ? pos[1] / P->h + P->nb[2] : 0.0;
    lo[0] = P->nb[0];
    lo[1] = P->ndim == 3 ? P->nb[2] : 0;
    lo[2] = P->nb[4];
    len[0] = P->nz;
    len[1] = P->ny;
    len[2] = P->nx;
    int i0[3];
    double t[3];
    for (int ax = 0; ax < 3; ax++) {
        double r = nearbyint(f[ax]);
        if (fabs(f[ax] - r) < 1e-6) f[ax] = r;
        if (!(f[ax] >= lo[ax]) || !(f[ax] <= lo[ax] + len[ax] - 1)) return -1;
        i0[ax] = (int)floor(f[ax]);
        t[ax] = f[ax] - i0[ax];
    }
    int n = 0;
    for (int kz = 0; kz < 2; kz++)
        for (int ky = 0; ky < 2; ky++)
            for (int kx = 0; kx < 2; kx++) {
                double wz = kz ? t[0] : 1.0 - t[0];
                double wy = ky ? t[1] : 1.0 - t[1];
                double wx = kx ? t[2] : 1.0 - t[2];
                double ww = wz * wy * wx;
                if (ww == 0.0) continue;
                cell[n] = IDX(G, i0[0] + kz, i0[1] + ky, i0[2] + kx);
                w[n] = ww;
                n++;
            }
    return n;
}

static int cell_row(const grid_t *G, long i) { return (int)(i / ((long)G->NY * G->NX)); }

typedef struct {
    int ncell_src;
    long src_cell[8];
    double src_w[8];
    int *rec_n;
    long *rec_cell;
    double *rec_w;
} geometry_t;

static int build_geometry(const or_params *P, const grid_t *G, const double *src,
                          int nrec, const double *rec, geometry_t *g) {
    memset(g, 0, sizeof(*g));
    if (src) {
        int n = point_stencil(P, G, src, g->src_cell, g->src_w);
        if (n < 0) return -2;
        /* a free surface overwrites row 0, so a source weight there is void */
        int k = 0;
        for (int j = 0; j < n; j++)
            if (!(P->free_surface && cell_row(G, g->src_cell[j]) == 0)) {
                g->src_cell[k] = g->src_cell[j];
                g->src_w[k] = g->src_w[j];
                k++;
            }
        g->ncell_src = k;
    }
    if (nrec > 0) {
        g->rec_n = calloc(nrec, sizeof(int));
        g->rec_cell = calloc((size_t)nrec * 8, sizeof(long));
        g->rec_w = calloc((size_t)nrec * 8, sizeof(double));
        if (!g->rec_n || !g->rec_cell || !g->rec_w) return -3;
        for (int r = 0; r < nrec; r++) {
            int n = point_stencil(P, G, rec + (size_t)r * P->ndim,
                                  g->rec_cell + (size_t)r * 8, g->rec_w + (size_t)r * 8);
            if (n < 0) return -2;
            g->rec_n[r] = n;
        }
    }
    return 0;
}

static void free_geometry(geometry_t *g) {
    free(g->rec_n);
    free(g->rec_cell);
    free(g->rec_w);
}

static real_t sample(const geometry_t *g, int r, const real_t *p) {
    real_t s = 0;
    for (int k = 0; k < g->rec_n[r]; k++) s += g->rec_w[(size_t)r * 8 + k] * p[g->rec_cell[(size_t)r * 8 + k]];
    return s;
}

static double h_pow_d(const or_params *P) {
    return P->ndim == 3 ? P->h * P->h * P->h : P->h * P->h;
}

static void copy_interior(const or_params *P, const grid_t *G, const real_t *p,
                          real_t *out) {
    int y0 = P->ndim == 3 ? P->nb[2] : 0;
    for (int z = 0; z < P->nz; z++)
        for (int y = 0; y < P->ny; y++)
            for (int x = 0; x < P->nx; x++)
                out[((long)z * P->ny + y) * P->nx + x] =
                    p[IDX(G, z + P->nb[0], y + y0, x + P->nb[4])];
}

/* CPML memory arrays: per active axis psi, zeta over the padded grid and the
 * per-index coefficients a, b. */
typedef struct {
    int on[3];
    real_t *psi[3], *zeta[3];
    double *ca[3], *cb[3];
} cpml_t;

static int cpml_init(const or_params *P, const grid_t *G, const real_t *vel,
                     cpml_t *C) {
    memset(C, 0, sizeof(*C));
    if (P->bc != 1) return 0;
    double vmax = P->cpml_vmax > 0 ? P->cpml_vmax : model_vmax(P, vel);
    for (int ax = 0; ax < 3; ax++) {
        int N, lo, hi;
        axis_layout(P, G, ax, &N, &lo, &hi);
        if (!axis_active(P, ax) || (lo == 0 && hi == 0)) continue;
        C->on[ax] = 1;
        C->psi[ax] = calloc(G->ncell, sizeof(real_t));
        C->zeta[ax] = calloc(G->ncell, sizeof(real_t));
        C->ca[ax] = calloc(N, sizeof(double));
        C->cb[ax] = calloc(N, sizeof(double));
        if (!C->psi[ax] || !C->zeta[ax] || !C->ca[ax] || !C->cb[ax]) return -3;
        for (int i = 0; i < N; i++) cpml_coef(P, vmax, N, lo, hi, i, &C->ca[ax][i], &C->cb[ax][i]);
    }
    return 0;
}

static void cpml_free(cpml_t *C) {
    for (int ax = 0; ax < 3; ax++) {
        free(C->psi[ax]);
        free(C->zeta[ax]);
        free(C->ca[ax]);
        free(C->cb[ax]);
    }
}

static int coord_of(int ax, int z, int y, int x) { return ax == 0 ? z : (ax == 1 ? y : x); }

/* One time step n -> n+1 (Eq. cerjan_pde with reading R1, CPML reading R3,
 * free surface R4). s is the per-cell source density at step n (or NULL). */
static void step(const or_params *P, const grid_t *G, const real_t *c,
                 const real_t *a, cpml_t *C, const real_t *s, const real_t *pprev,
                 const real_t *pcur, real_t *pnext, real_t *cadd) {
    /* CPML pass 1: psi^n = b psi^{n-1} + a D1 p^n on every cell */
    for (int ax = 0; ax < 3; ax++) {
        if (!C->on[ax]) continue;
#pragma omp parallel for schedule(static)
        for (int z = 0; z < G->NZ; z++)
            for (int y = 0; y < G->NY; y++)
                for (int x = 0; x < G->NX; x++) {
                    long i = IDX(G, z, y, x);
                    int k = coord_of(ax, z, y, x);
                    C->psi[ax][i] = C->cb[ax][k] * C->psi[ax][i] +
                                    C->ca[ax][k] * d1_axis(P, G, pcur, ax, z, y, x);
                }
    }
    /* pass 2: zeta and the update of p */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < G->NZ; z++)
        for (int y = 0; y < G->NY; y++)
            for (int x = 0; x < G->NX; x++) {
                long i = IDX(G, z, y, x);
                real_t rhs = 0, add = 0;
                for (int ax = 0; ax < 3; ax++) {
                    if (!axis_active(P, ax)) continue;
                    real_t d2 = d2_axis(P, G, pcur, ax, z, y, x);
                    rhs += d2;
                    if (C->on[ax]) {
                        int k = coord_of(ax, z, y, x);
                        real_t dpsi = d1_axis(P, G, C->psi[ax], ax, z, y, x);
                        C->zeta[ax][i] = C->cb[ax][k] * C->zeta[ax][i] + C->ca[ax][k] * (d2 + dpsi);
                        rhs += dpsi + C->zeta[ax][i];
                        add += dpsi + C->zeta[ax][i];
                    }
                }
                if (cadd) cadd[i] = add;
                if (s) rhs += s[i];
                pnext[i] = (2.0 * pcur[i] - (1.0 - a[i]) * pprev[i] + c[i] * rhs) / (1.0 + a[i]);
            }
    /* free surface: row 0 held at zero */
    if (P->free_surface)
        for (int y = 0; y < G->NY; y++)
            for (int x = 0; x < G->NX; x++) pnext[IDX(G, 0, y, x)] = 0;
}

int oracle_forward(const or_params *P, const real_t *vel, const double *wavelet,
                   const double *src, int nrec, const double *rec, real_t *gather,
                   real_t *snaps, const real_t *init_prev, const real_t *init_cur,
                   real_t *final_prev, real_t *final_cur) {
    grid_t G;
    if (make_grid(P, &G) || !vel) return -1;
    if (src && !wavelet) return -1;
    if (nrec < 0 || (nrec > 0 && (!rec || !gather))) return -1;
    long nc = G.ncell;
    real_t *c = calloc(nc, sizeof(real_t)), *a = calloc(nc, sizeof(real_t));
    real_t *buf[3] = {calloc(nc, sizeof(real_t)), calloc(nc, sizeof(real_t)),
                      calloc(nc, sizeof(real_t))};
    real_t *s = src ? calloc(nc, sizeof(real_t)) : NULL;
    cpml_t C;
    geometry_t geo;
    int rc = 0;
    memset(&C, 0, sizeof(C));
    if (!c || !a || !buf[0] || !buf[1] || !buf[2] || (src && !s)) { rc = -3; goto done_nogeo; }
    if ((rc = cpml_init(P, &G, vel, &C))) goto done_nogeo;
    if ((rc = build_geometry(P, &G, src, nrec, rec, &geo))) goto done;
    build_coefficients(P, &G, vel, c, a, NULL);
    real_t *pprev = buf[0], *pcur = buf[1], *pnext = buf[2];
    if (init_prev) memcpy(pprev, init_prev, nc * sizeof(real_t));
    if (init_cur) memcpy(pcur, init_cur, nc * sizeof(real_t));
    int nsnap = nsnap_of(P);
    long nint = (long)P->nz * P->ny * P->nx;
    double hd = h_pow_d(P);
    for (int n = 0; n < P->nt; n++) {
        for (int r = 0; r < nrec; r++) gather[(size_t)n * nrec + r] = sample(&geo, r, pcur);
        if (snaps && nsnap > 0 && n >= P->snap_begin && (n - P->snap_begin) % P->snap_every == 0) {
            int k = (n - P->snap_begin) / P->snap_every;
            if (k < nsnap) copy_interior(P, &G, pcur, snaps + (size_t)k * nint);
        }
        if (s)
            for (int j = 0; j < geo.ncell_src; j++) s[geo.src_cell[j]] = wavelet[n] * geo.src_w[j] / hd;
        step(P, &G, c, a, &C, s, pprev, pcur, pnext, NULL);
        if (s)
            for (int j = 0; j < geo.ncell_src; j++) s[geo.src_cell[j]] = 0;
        real_t *t = pprev;
        pprev = pcur;
        pcur = pnext;
        pnext = t;
    }
    if (final_prev) memcpy(final_prev, pprev, nc * sizeof(real_t));
    if (final_cur) memcpy(final_cur, pcur, nc * sizeof(real_t));
done:
    free_geometry(&geo);
done_nogeo:
    cpml_free(&C);
    free(c);
    free(a);
    free(buf[0]);
    free(buf[1]);
    free(buf[2]);
    free(s);
    return rc;
}

/* Ghost-rule placement used by the explicit transpose: the adjoint of reading
 * a value through get(). */
static void put(const or_params *P, const grid_t *G, real_t *out, int z, int y,
                int x, real_t v) {
    if (x < 0 || x >= G->NX || y < 0 || y >= G->NY || z >= G->NZ) return;
    if (z < 0) {
        if (!P->free_surface) return;
        put(P, G, out, -z, y, x, -v);
        return;
    }
    out[IDX(G, z, y, x)] += v;
}

/* out = L^T f, written as the scatter that transposes lap_at term by term. */
static void lap_transpose(const or_params *P, const grid_t *G, const real_t *f,
                          real_t *out) {
    memset(out, 0, G->ncell * sizeof(real_t));
    double ih2 = 1.0 / (P->h * P->h);
    for (int z = 0; z < G->NZ; z++)
        for (int y = 0; y < G->NY; y++)
            for (int x = 0; x < G->NX; x++) {
                real_t v = f[IDX(G, z, y, x)] * ih2;
                for (int ax = 0; ax < 3; ax++) {
                    if (!axis_active(P, ax)) continue;
                    put(P, G, out, z, y, x, D2W[0] * v);
                    for (int m = 1; m <= 4; m++) {
                        int dz, dy, dx;
                        axis_step(ax, m, &dz, &dy, &dx);
                        put(P, G, out, z + dz, y + dy, x + dx, D2W[m] * v);
                        put(P, G, out, z - dz, y - dy, x - dx, D2W[m] * v);
                    }
                }
            }
}

/* out += D1^T f and out += D2^T f along one axis: the scatters that transpose
 * d1_axis and d2_axis term by term (ghost rules through put()). */
static void d1_transpose_add(const or_params *P, const grid_t *G, const real_t *f, int ax,
                             real_t *out) {
    for (int z = 0; z < G->NZ; z++)
        for (int y = 0; y < G->NY; y++)
            for (int x = 0; x < G->NX; x++) {
                real_t v = f[IDX(G, z, y, x)] / P->h;
                for (int m = 1; m <= 4; m++) {
                    int dz, dy, dx;
                    axis_step(ax, m, &dz, &dy, &dx);
                    put(P, G, out, z + dz, y + dy, x + dx, D1W[m] * v);
                    put(P, G, out, z - dz, y - dy, x - dx, -D1W[m] * v);
                }
            }
}
static void d2_transpose_add(const or_params *P, const grid_t *G, const real_t *f, int ax,
                             real_t *out) {
    for (int z = 0; z < G->NZ; z++)
        for (int y = 0; y < G->NY; y++)
            for (int x = 0; x < G->NX; x++) {
                real_t v = f[IDX(G, z, y, x)] / (P->h * P->h);
                put(P, G, out, z, y, x, D2W[0] * v);
                for (int m = 1; m <= 4; m++) {
                    int dz, dy, dx;
                    axis_step(ax, m, &dz, &dy, &dx);
                    put(P, G, out, z + dz, y + dy, x + dx, D2W[m] * v);
                    put(P, G, out, z - dz, y - dy, x - dx, D2W[m] * v);
                }
            }
}

int oracle_apply_laplacian(const or_params *P, const real_t *f, real_t *out) {
    grid_t G;
    if (make_grid(P, &G)) return -1;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < G.NZ; z++)
        for (int y = 0; y < G.NY; y++)
            for (int x = 0; x < G.NX; x++) out[IDX(&G, z, y, x)] = lap_at(P, &G, f, z, y, x);
    return 0;
}

int oracle_apply_laplacian_T(const or_params *P, const real_t *f, real_t *out) {
    grid_t G;
    if (make_grid(P, &G)) return -1;
    lap_transpose(P, &G, f, out);
    return 0;
}

int oracle_coefficients(const or_params *P, const real_t *vel, real_t *c,
                        real_t *a, double *cpml_a, double *cpml_b) {
    grid_t G;
    if (make_grid(P, &G)) return -1;
    build_coefficients(P, &G, vel, c, a, NULL);
    if (cpml_a && cpml_b) {
        double vmax = P->cpml_vmax > 0 ? P->cpml_vmax : model_vmax(P, vel);
        int off = 0;
        for (int ax = 0; ax < 3; ax++) {
            int N, lo, hi;
            axis_layout(P, &G, ax, &N, &lo, &hi);
            for (int i = 0; i < N; i++) cpml_coef(P, vmax, N, lo, hi, i, &cpml_a[off + i], &cpml_b[off + i]);
            off += N;
        }
    }
    return 0;
}

/*
 * Misfit and velocity gradient of one shot by the adjoint-state method on the
 * discrete scheme (reading R8). With
 *   F_i^n = (1+a_i) p_i^{n+1} - 2 p_i^n + (1-a_i) p_i^{n-1} - c_i ((L p^n)_i + s_i^n)
 * the multipliers lambda^k (k = nt..1) solve
 *   (1+a) lambda^k = 2 lambda^{k+1} + L^T (c lambda^{k+1}) - (1-a) lambda^{k+2}
 *                    + R^T (R p^k - d^k)
 * and dJ/dv_i = - sum_n lambda_i^{n+1} dF_i^n/dv_i, where
 *   dF_i^n/dv_i = eta_i v_i dt (p_i^{n+1} - p_i^{n-1}) - 2 v_i dt^2 ((L p^n)_i + s_i^n).
 * A free-surface row carries no unknown (p = 0 there), so its multiplier is 0.
 * dJ/dw^n = sum_i lambda_i^{n+1} c_i weight_i / h^d gives the wavelet gradient.
 * All forward states are stored (no checkpointing: this is the plain version).
 *
 * CPML (reading R3) adds, per absorbing axis, the constraints
 *   Psi^n  = psi^n  - b psi^{n-1}  - a D1 p^n
 *   Zeta^n = zeta^n - b zeta^{n-1} - a (D2 p^n + D1 psi^n)
 * and the term D1 psi^n + zeta^n to (L p^n) in F^n. With multipliers mu^k, nu^k
 * (zero for k >= nt), stationarity in zeta^k, psi^k and p^k gives
 *   nu^k = b nu^{k+1} + c lambda^{k+1}
 *   mu^k = b mu^{k+1} + D1^T (c lambda^{k+1} + a nu^k)
 *   and D1^T (a mu^k) + D2^T (a nu^k) added to the right side of lambda^k,
 * and dF/dv gains -2 v dt^2 (D1 psi^n + zeta^n). The CPML coefficients are
 * constants of the map (taken at cpml_vmax, else at the model's maximum).
 */
int oracle_gradient(const or_params *P, const real_t *vel, const double *wavelet,
                    const double *src, int nrec, const double *rec,
                    const double *d_obs, real_t *misfit, real_t *grad,
                    real_t *grad_wavelet, real_t *gather) {
    grid_t G;
    if (make_grid(P, &G) || !vel || !wavelet || !src || nrec < 1 || !rec || !d_obs) return -1;
    long nc = G.ncell;
    int nt = P->nt;
    int rc = 0;
    real_t *c = calloc(nc, sizeof(real_t)), *a = calloc(nc, sizeof(real_t));
    double *eta = calloc(nc, sizeof(double));
    real_t *states = calloc((size_t)(nt + 1) * nc, sizeof(real_t));
    real_t *s = calloc(nc, sizeof(real_t));
    real_t *g = calloc((size_t)nt * nrec, sizeof(real_t));
    real_t *lam[3] = {calloc(nc, sizeof(real_t)), calloc(nc, sizeof(real_t)),
                      calloc(nc, sizeof(real_t))};
    real_t *work = calloc(nc, sizeof(real_t)), *lt = calloc(nc, sizeof(real_t));
    real_t *lp = calloc(nc, sizeof(real_t)), *rt = calloc(nc, sizeof(real_t));
    real_t *gpad = calloc(nc, sizeof(real_t));
    real_t *pm1 = calloc(nc, sizeof(real_t));
    real_t *tadd = NULL, *nu[3] = {NULL, NULL, NULL}, *mu[3] = {NULL, NULL, NULL}, *tmp = NULL;
    cpml_t C;
    memset(&C, 0, sizeof(C));
    geometry_t geo;
    memset(&geo, 0, sizeof(geo));
    if (!c || !a || !eta || !states || !s || !g || !lam[0] || !lam[1] || !lam[2] ||
        !work || !lt || !lp || !rt || !gpad || !pm1) {
        rc = -3;
        goto out_nogeo;
    }
    if ((rc = cpml_init(P, &G, vel, &C))) goto out_nogeo;
    if (P->bc == 1) {
        tadd = calloc((size_t)nt * nc, sizeof(real_t));
        tmp = calloc(nc, sizeof(real_t));
        if (!tadd || !tmp) {
            rc = -3;
            goto out_nogeo;
        }
        for (int ax = 0; ax < 3; ax++) {
            if (!C.on[ax]) continue;
            nu[ax] = calloc(nc, sizeof(real_t));
            mu[ax] = calloc(nc, sizeof(real_t));
            if (!nu[ax] || !mu[ax]) {
                rc = -3;
                goto out_nogeo;
            }
        }
    }
    if ((rc = build_geometry(P, &G, src, nrec, rec, &geo))) goto out;
    build_coefficients(P, &G, vel, c, a, eta);
    double hd = h_pow_d(P);

    /* forward, storing p^0 .. p^nt */
    for (int n = 0; n < nt; n++) {
        real_t *pcur = states + (size_t)n * nc;
        const real_t *pprev = n > 0 ? states + (size_t)(n - 1) * nc : pm1;
        for (int r = 0; r < nrec; r++) g[(size_t)n * nrec + r] = sample(&geo, r, pcur);
        for (int j = 0; j < geo.ncell_src; j++) s[geo.src_cell[j]] = wavelet[n] * geo.src_w[j] / hd;
        step(P, &G, c, a, &C, s, pprev, pcur, states + (size_t)(n + 1) * nc, tadd ? tadd + (size_t)n * nc : NULL);
        for (int j = 0; j < geo.ncell_src; j++) s[geo.src_cell[j]] = 0;
    }
    if (gather) memcpy(gather, g, (size_t)nt * nrec * sizeof(real_t));

    /* residual and misfit */
    real_t J = 0;
    for (size_t k = 0; k < (size_t)nt * nrec; k++) {
        g[k] -= d_obs[k];
        J += 0.5 * g[k] * g[k];
    }
    if (misfit) *misfit = J;

    /* backward recursion, k = nt .. 1 */
    real_t *l1 = lam[0], *l2 = lam[1], *lk = lam[2]; /* lambda^{k+1}, lambda^{k+2}, lambda^k */
    for (int k = nt; k >= 1; k--) {
        for (long i = 0; i < nc; i++) work[i] = c[i] * l1[i];
        lap_transpose(P, &G, work, lt);
        /* CPML multipliers of step k (zero for k = nt) and their terms in lambda^k */
        if (tadd && k <= nt - 1)
            for (int ax = 0; ax < 3; ax++) {
                if (!C.on[ax]) continue;
                for (int z = 0; z < G.NZ; z++)
                    for (int y = 0; y < G.NY; y++)
                        for (int x = 0; x < G.NX; x++) {
                            long i = IDX(&G, z, y, x);
                            int q = coord_of(ax, z, y, x);
                            nu[ax][i] = C.cb[ax][q] * nu[ax][i] + work[i];
                            tmp[i] = work[i] + C.ca[ax][q] * nu[ax][i];
                        }
                memset(rt, 0, nc * sizeof(real_t));
                d1_transpose_add(P, &G, tmp, ax, rt);
                for (int z = 0; z < G.NZ; z++)
                    for (int y = 0; y < G.NY; y++)
                        for (int x = 0; x < G.NX; x++) {
                            long i = IDX(&G, z, y, x);
                            int q = coord_of(ax, z, y, x);
                            mu[ax][i] = C.cb[ax][q] * mu[ax][i] + rt[i];
                        }
                for (int z = 0; z < G.NZ; z++)
                    for (int y = 0; y < G.NY; y++)
                        for (int x = 0; x < G.NX; x++) {
                            long i = IDX(&G, z, y, x);
                            int q = coord_of(ax, z, y, x);
                            tmp[i] = C.ca[ax][q] * mu[ax][i];
                        }
                d1_transpose_add(P, &G, tmp, ax, lt);
                for (int z = 0; z < G.NZ; z++)
                    for (int y = 0; y < G.NY; y++)
                        for (int x = 0; x < G.NX; x++) {
                            long i = IDX(&G, z, y, x);
                            int q = coord_of(ax, z, y, x);
                            tmp[i] = C.ca[ax][q] * nu[ax][i];
                        }
                d2_transpose_add(P, &G, tmp, ax, lt);
            }
        memset(rt, 0, nc * sizeof(real_t));
        if (k <= nt - 1)
            for (int r = 0; r < nrec; r++)
                for (int q = 0; q < geo.rec_n[r]; q++)
                    rt[geo.rec_cell[(size_t)r * 8 + q]] += geo.rec_w[(size_t)r * 8 + q] * g[(size_t)k * nrec + r];
        for (long i = 0; i < nc; i++)
            lk[i] = (2.0 * l1[i] + lt[i] - (1.0 - a[i]) * l2[i] + rt[i]) / (1.0 + a[i]);
        if (P->free_surface)
            for (int y = 0; y < G.NY; y++)
                for (int x = 0; x < G.NX; x++) lk[IDX(&G, 0, y, x)] = 0;

        /* gradient term of F^{k-1}: needs p^k, p^{k-1}, p^{k-2} and L p^{k-1} */
        int n = k - 1;
        const real_t *pn1 = states + (size_t)(n + 1) * nc;
        const real_t *pn = states + (size_t)n * nc;
        const real_t *pnm1 = n > 0 ? states + (size_t)(n - 1) * nc : pm1;
        oracle_apply_laplacian(P, pn, lp);
        for (int j = 0; j < geo.ncell_src; j++) lp[geo.src_cell[j]] += wavelet[n] * geo.src_w[j] / hd;
        if (tadd)
            for (long i = 0; i < nc; i++) lp[i] += tadd[(size_t)n * nc + i];
        for (int z = 0; z < G.NZ; z++) {
            if (P->free_surface && z == 0) continue;
            for (int y = 0; y < G.NY; y++)
                for (int x = 0; x < G.NX; x++) {
                    long i = IDX(&G, z, y, x);
                    real_t v = vel_pad(P, vel, z, y, x);
                    real_t dF = eta[i] * v * P->dt * (pn1[i] - pnm1[i]) -
                                2.0 * v * P->dt * P->dt * lp[i];
                    gpad[i] -= lk[i] * dF;
                }
        }
        if (grad_wavelet) {
            real_t gw = 0;
            for (int j = 0; j < geo.ncell_src; j++)
                gw += lk[geo.src_cell[j]] * c[geo.src_cell[j]] * geo.src_w[j] / hd;
            grad_wavelet[n] = gw;
        }
        real_t *t = l2;
        l2 = l1;
        l1 = lk;
        lk = t;
    }

    /* fold the padding cells onto the interior cells they replicate (R7) */
    if (grad) {
        long nint = (long)P->nz * P->ny * P->nx;
        for (long i = 0; i < nint; i++) grad[i] = 0;
        for (int z = 0; z < G.NZ; z++)
            for (int y = 0; y < G.NY; y++)
                for (int x = 0; x < G.NX; x++) {
                    int iz = clampi(z - P->nb[0], 0, P->nz - 1);
                    int iy = P->ndim == 3 ? clampi(y - P->nb[2], 0, P->ny - 1) : 0;
                    int ix = clampi(x - P->nb[4], 0, P->nx - 1);
                    grad[((long)iz * P->ny + iy) * P->nx + ix] += gpad[IDX(&G, z, y, x)];
                }
    }
out:
    free_geometry(&geo);
out_nogeo:
    free(c);
    free(a);
    free(eta);
    free(states);
    free(s);
    free(g);
    free(lam[0]);
    free(lam[1]);
    free(lam[2]);
    free(work);
    free(lt);
    free(lp);
    free(rt);
    free(gpad);
    free(pm1);
    free(tadd);
    free(tmp);
    for (int ax = 0; ax < 3; ax++) {
        free(nu[ax]);
        free(mu[ax]);
    }
    cpml_free(&C);
    return rc;
}
