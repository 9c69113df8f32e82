/*
 * FP64 CPU oracle of the acoustic FDTD path — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this library. It shares no code, header, table or helper with the CUDA library
 * under paper_2605_30541_gb300/; the two meet only through seeded inputs.
 *
 * The scheme it spells out, step by step (paper App. E.2-E.3, Eq. acoustic_2d,
 * Eq. cerjan_pde, Eq. cerjan_damp, Eq. free_surface; readings of the gaps are
 * listed beside each routine in fdtd_oracle.c):
 *
 *   (1+a_i) p_i^{n+1} = 2 p_i^n - (1-a_i) p_i^{n-1} + c_i ((L p^n)_i + s_i^n)
 *
 * with c = v^2 dt^2, a = eta v^2 dt / 2 (sponge), L the 8th-order Laplacian,
 * s^n the point source w(t_n)/h^d, receivers sampling p^n (gather row n).
 *
 * Build with -DORACLE_COMPLEX to get the same scheme over double complex, used
 * for complex-step derivatives of the forward map.
 */
#ifndef FDTD_ORACLE_H
#define FDTD_ORACLE_H

#ifdef ORACLE_COMPLEX
#include <complex.h>
typedef double complex real_t;
#else
typedef double real_t;
#endif

typedef struct {
    int ndim;            /* 2 or 3 */
    int nz, ny, nx;      /* interior cells (ny = 1 in 2D) */
    double h;            /* grid spacing, m */
    double dt;           /* time step, s */
    int nt;              /* number of time steps; gather rows n = 0..nt-1 */
    int bc;              /* 0 sponge, 1 CPML, 2 none (p = 0 outside) */
    int nb[6];           /* absorbing cells per face: -z,+z,-y,+y,-x,+x */
    int free_surface;    /* 1: row z = 0 held at p = 0, odd mirror above */
    double R;            /* design reflection coefficient of the layer */
    double f_ref;        /* CPML alpha reference frequency, Hz */
    double cpml_vmax;    /* velocity used for the CPML d0; <= 0: model maximum */
    int snap_every, snap_begin, snap_end; /* snapshots at n = begin + k*every < end */
} or_params;

int oracle_num_threads(void);

/* 0 on success, negative on bad arguments. */
int oracle_padded_dims(const or_params *P, int dims[3]);

int oracle_forward(const or_params *P, const real_t *vel,
                   const double *wavelet, const double *src,
                   int nrec, const double *rec, real_t *gather,
                   real_t *snaps,
                   const real_t *init_prev, const real_t *init_cur,
                   real_t *final_prev, real_t *final_cur);

int oracle_gradient(const or_params *P, const real_t *vel,
                    const double *wavelet, const double *src,
                    int nrec, const double *rec, const double *d_obs,
                    real_t *misfit, real_t *grad, real_t *grad_wavelet,
                    real_t *gather);

int oracle_apply_laplacian(const or_params *P, const real_t *f, real_t *out);
int oracle_apply_laplacian_T(const or_params *P, const real_t *f, real_t *out);
int oracle_coefficients(const or_params *P, const real_t *vel,
                        real_t *c, real_t *a, double *cpml_a, double *cpml_b);

#endif
