/*
 * sim.h — C ABI of the GB300 acoustic FDTD library (libsim).
 *
 * The library solves the constant-density acoustic wave equation
 *     (1/v^2) p_tt - lap p (+ eta p_t) = s(x, t)                     (paper Sec. 2, Eq. acoustic;
 *                                                                     App. E.2, Eq. acoustic_2d, Eq. cerjan_pde)
 * on a regular grid with an 8th-order central Laplacian and second-order
 * leapfrog in time (App. E.3, Tab. params), zero initial state (App. E.2),
 * a free surface p = 0 on top (Eq. free_surface), an absorbing layer on the
 * other faces (Cerjan sponge, Eq. cerjan_damp; or a CPML), a point source
 * with a given wavelet (Sec. 2, App. E.4) and receivers that sample the field
 * into a shot gather R p (Sec. 2), plus wavefield snapshots every k steps
 * (App. E.3.3). It also returns the exact gradient of the L2 data misfit with
 * respect to velocity (adjoint-state method on the discrete scheme; the paper
 * names FWI as the consumer of these solves, Sec. 1).
 *
 * The discrete scheme, per padded cell i and step n = 0 .. nt-1:
 *   (1+a_i) p_i^{n+1} = 2 p_i^n - (1-a_i) p_i^{n-1} + c_i ((L p^n)_i + s_i^n)
 *   c = v^2 dt^2, a = eta v^2 dt / 2 (sponge; 0 otherwise),
 *   s^n = w[n] / h^d at the source (bi/tri-linear weights), gather[n] = R p^n.
 *
 * Conventions (all entry points):
 *  - Grids are row-major [z][y][x] (x fastest); 2D problems have ny = 1.
 *    Depth z is the slowest axis; z = 0 is the top of the interior.
 *  - Positions are metres from the interior origin, ordered (x, z) in 2D and
 *    (x, y, z) in 3D, and must lie inside the interior box [0, (n-1) h].
 *  - Data pointers (velocity, wavelet, gathers, snapshots, gradients) may be
 *    device or host memory; the library tells them apart. Host inputs are
 *    copied in; when any output is host memory the call synchronises its
 *    stream before returning. Position arrays are read on the host.
 *  - The element type of every `void*` data array is the handle's precision:
 *    float for SIM_FP32, double for SIM_FP64 (FP16 snapshots are `uint16`
 *    IEEE half with a float scale per snapshot).
 *  - The caller owns every argument buffer. The library owns its padded
 *    fields, coefficients, absorbing-layer memory, checkpoints and staging
 *    buffers, all freed by sim_destroy. The forward buffers are allocated in
 *    sim_create; the adjoint-state buffers (checkpoints, imaging terms,
 *    adjoint fields) by the first sim_adjoint call on the handle, and a
 *    staging buffer for host-memory snapshots by the first call that asks
 *    for them.
 *  - Calls are ordered on the handle's CUDA stream and return after enqueue
 *    (unless an output is host memory). Device-side failures (non-finite
 *    values, a bounded wait that gave up) surface at the next call or at
 *    sim_sync. Errors are sticky per handle; sim_last_error explains them.
 *  - No entry point aborts or throws; every one returns a sim_status.
 */
#ifndef GB300_SIM_H
#define GB300_SIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIM_OK = 0,
    SIM_ERR_ARG = 1,            /* an argument is invalid (message in sim_last_error) */
    SIM_ERR_CFL = 2,            /* v_max dt / h above the stability bound of App. E.3.2 */
    SIM_WARN_DISPERSION = 3,    /* non-fatal: h > v_min / (4 f_max) (App. E.3.1) */
    SIM_ERR_OOM = 4,            /* device or host allocation failed */
    SIM_ERR_CUDA = 5,           /* a CUDA runtime call failed */
    SIM_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
    SIM_ERR_UNSTABLE = 7,       /* non-finite values appeared in the field or outputs */
    SIM_ERR_STATE = 8,          /* call made in the wrong state (e.g. no model set) */
    SIM_ERR_UNSUPPORTED = 9     /* valid request this build does not implement */
} sim_status;

typedef enum { SIM_BC_SPONGE = 0, SIM_BC_CPML = 1, SIM_BC_NONE = 2 } sim_bc;
typedef enum { SIM_FP32 = 0, SIM_FP64 = 1 } sim_precision;

/* Problem description. Zero-initialise, then set the fields you need;
 * sim_desc_init fills the defaults. */
typedef struct {
    int ndim;             /* 2 or 3 */
    int nz, ny, nx;       /* interior cells (ny = 1 in 2D) */
    double h;             /* isotropic grid spacing, m (Tab. params: 10 m) */
    double dt;            /* time step, s (Tab. params: 1 ms) */
    int nt;               /* steps; gather rows and snapshot steps n = 0 .. nt-1 */
    int space_order;      /* 8 (M = 4); 0 means 8 */
    int bc;               /* sim_bc */
    int nb[6];            /* absorbing cells per face: -z,+z,-y,+y,-x,+x */
    int free_surface;     /* 1: row z = 0 held at p = 0 (requires nb[0] = 0) */
    double R;             /* design reflection of the absorbing layer; <= 0 means 1e-3 */
    double f_ref;         /* CPML alpha reference frequency (Hz); <= 0 means 10 */
    double f_max;         /* highest source frequency for the dispersion check; 0 skips it */
    int snap_every;       /* snapshot period k (App. E.3.3); 0: no snapshots */
    int snap_begin;       /* first snapshot step */
    int snap_end;         /* snapshots at n = begin + j*k < min(end, nt) */
    int snap_fp16;        /* 0: snapshots in the handle precision; 1: FP16 + per-snapshot scale */
    int max_shots;        /* most shots one call carries; <= 0 means 1 */
    int max_rec;          /* most receivers one call carries */
    int precision;        /* sim_precision */
    int skip_cfl_check;   /* 1: accept dt above the stability bound (tests only) */
    int pad0;
    long long adj_budget; /* device bytes the gradient's buffers may take (checkpoints,
                             imaging terms, adjoint fields); <= 0: the free device memory
                             at the first sim_adjoint call, less max(2 GiB, 4% of the
                             device). Sets the checkpoint schedule (see sim_adjoint). */
} sim_desc;

/* Host-side facts about a description (no GPU needed). */
typedef struct {
    int NZ, NY, NX;           /* padded grid = interior + absorbing cells */
    int nsnap;                /* snapshots per shot */
    double courant;           /* v_max dt / h (0 if v_max unknown) */
    double courant_limit;     /* paper bound s_max = 1/sqrt(d sum_{m>=1} |a_m|) (App. E.3.2) */
    double courant_exact;     /* von Neumann bound 2/sqrt(d * 6.5016) of this stencil */
    double vmin, vmax;        /* model range (from sim_set_model, or as given to sim_plan) */
    double c_damp[6];         /* sponge c_damp = 1.5 ln(1/R)/nb per face (0 where nb = 0) */
    long long cells_per_shot; /* padded cells updated per shot per step */
    size_t device_bytes;      /* device memory the handle owns (0 from sim_plan) */
    int tile_x, tile_y, tile_z; /* tile of the stencil kernels the autotuner chose */
    int last_path;            /* how the last sim_forward ran: 0 none yet, 1 one kernel launch per
                                 step (captured as a CUDA graph), 2 resident: the whole time loop in
                                 one cooperative launch that keeps the wavefield on chip (2D FP32
                                 runs whose subdomains all fit on the GPU at once), 3 the 3D path,
                                 4 row march: one launch per step in which every warp streams
                                 down a 128-column strip of rows (2D FP32, when not resident) */
    int last_rows;            /* path 2: rows of the tallest resident subdomain (x 128 columns) */
    /* checkpoint schedule of the gradient (0 before the first sim_adjoint call) */
    int adj_levels;           /* 1: one checkpoint level; 2: two */
    int adj_slots;            /* L: imaging-term slots = steps of an innermost segment */
    int adj_inner;            /* m: innermost segments per top segment (1 with one level) */
    int adj_top;              /* top-level checkpoints, every m L steps */
    int adj_sub;              /* second-level checkpoint slots */
    int pad1;
    size_t adj_bytes;         /* device memory of the gradient's buffers */
    int z_variant;            /* 3D: z-march the autotuner chose (1 per-thread cp.async staging, 2 TMA
                                 staging with the x-strip CPML folded in, 3 TMA staging; 4 and 5: 3 and
                                 2 with the plane loop not unrolled; 6: 3 with the loop unrolled by 3) */
    int z_chunk;              /* 3D: planes per CTA of the z-march */
    int batch_sched;          /* schedule of the last sim_batch forward this handle took part in
                                 (0 none yet, 1 row march, 2 two-step row march, 3 stepped tiles,
                                 4 persistent tiles) */
    int batch_tile;           /* its tile height (stepped and persistent schedules) */
} sim_info;

typedef struct sim_s *sim_t;

/* Fill defaults: space_order 8, R 1e-3, f_ref 10 Hz, max_shots 1, FP32. */
void sim_desc_init(sim_desc *d);

/* Validate a description on the host and report its layout. With vmax > 0
 * also applies the CFL check (SIM_ERR_CFL) and, with vmin > 0 and
 * f_max > 0, the dispersion check (SIM_WARN_DISPERSION). Never touches the GPU. */
sim_status sim_plan(const sim_desc *d, double vmin, double vmax, sim_info *out);

/* Create a solver on the current CUDA device. `vel` is the interior velocity
 * [nz][ny][nx] in m/s (host or device, handle precision) or NULL to set it
 * later; `cuda_stream` is a cudaStream_t (NULL: the legacy default stream).
 * Allocates every device buffer the handle needs. On failure *out is NULL. */
sim_status sim_create(const sim_desc *d, const void *vel, void *cuda_stream, sim_t *out);

/* Replace the velocity model (same layout as in sim_create). Recomputes
 * c = v^2 dt^2 and the absorbing-layer coefficients; velocities in the
 * absorbing layers copy the nearest interior cell. Returns SIM_ERR_CFL when
 * v_max dt / h exceeds the bound (unless skip_cfl_check), SIM_WARN_DISPERSION
 * (model still set) when the grid under-samples f_max, SIM_ERR_ARG when a
 * velocity is not finite or not positive. Synchronises the stream. */
sim_status sim_set_model(sim_t s, const void *vel);

/* Forward modelling of `nshots` shots sharing the model and the receivers.
 *   wavelet   [nt]                source time function w(t_n), shared by the shots
 *   src_pos   [nshots][ndim]      source positions (host), metres
 *   rec_pos   [nrec][ndim]        receiver positions (host), metres
 *   gather    [nshots][nt][nrec]  out: R p^n (NULL: not recorded)
 *   snaps     [nshots][nsnap][nz][ny][nx]  out: interior p^n at snapshot steps
 *             (NULL: none); FP16 when desc.snap_fp16, else handle precision
 *   snap_scale [nshots][nsnap]    out (FP16 only): scale s, value = half * s,
 *             s = 2^(floor(log2 max|p|) - 14), 1 for an all-zero snapshot
 * SIM_ERR_ARG for nshots > max_shots, nrec > max_rec or positions outside the
 * interior. */
sim_status sim_forward(sim_t s, int nshots, const void *wavelet, const double *src_pos,
                       int nrec, const double *rec_pos, void *gather, void *snaps,
                       float *snap_scale);

/* Misfit J = 1/2 sum (g - d_obs)^2 over shots, steps and receivers, and its
 * exact gradient with respect to the interior velocity, by the adjoint-state
 * method on the discrete scheme.
 *   d_obs      [nshots][nt][nrec]  observed data
 *   gather_out [nshots][nt][nrec]  out: modelled gather (NULL ok)
 *   misfit_out [1] (host)          out: J, accumulated over shots in FP64
 *   ckpt_fp16  1: checkpoints (2D: and the stored imaging terms) in FP16
 *              with a power-of-two scale per tile (the CPML memory: per row
 *              of its strips); 0: handle precision. On 3D handles the
 *              imaging terms stay FP32.
 *   grad_v     [nz][ny][nx]        out: dJ/dv ACCUMULATED (+=) in handle
 *              precision, after an FP64 sum over the shots
 * 2D and 3D (FP32) handles; sponge, no-absorption and CPML boundaries (for
 * CPML the exact transpose of the psi / zeta recursions, their state kept
 * with every checkpoint, the CPML coefficients, set from the model maximum by
 * sim_set_model, held fixed as constants of the map).
 * Checkpointing (optimal checkpointing is the trade-off the paper names,
 * Sec. 5): the forward sweep keeps the state at the start of each segment
 * and the reverse sweep recomputes the segments. The first call allocates
 * the buffers for the cheapest schedule that fits desc.adj_budget: sqrt(nt)
 * segments (two forward sweeps), else the one-level split needing least
 * memory, else two levels (a top segment is recomputed once keeping inner
 * checkpoints: three forward sweeps); SIM_ERR_OOM when even that does not
 * fit. Each checkpoint holds p^{n-1}, p^n and the CPML memory on its strips
 * only, at the storage precision. A later FP32-storage call on buffers sized
 * for FP16 frees and re-plans them. sim_get_info reports the schedule. */
sim_status sim_adjoint(sim_t s, int nshots, const void *wavelet, const double *src_pos,
                       int nrec, const double *rec_pos, const void *d_obs,
                       void *gather_out, double *misfit_out, int ckpt_fp16, void *grad_v);

/* Vector-Jacobian product of the gather map: grad_v += (dg/dv)^T cot, for a
 * cotangent cot [nshots][nt][nrec] of the gathers g(v) (what a
 * torch.autograd backward pass needs). The same sweeps as sim_adjoint with
 * cot injected directly as the adjoint source, so a cotangent much smaller
 * than the gathers loses no precision to a difference g - d. Arguments and
 * errors as in sim_adjoint (no misfit). */
sim_status sim_adjoint_vjp(sim_t s, int nshots, const void *wavelet, const double *src_pos,
                           int nrec, const double *rec_pos, const void *cot,
                           void *gather_out, int ckpt_fp16, void *grad_v);

/* One entry of a batch: a handle (model + grid) and its shots. */
typedef struct {
    sim_t sim;
    int nshots;
    const void *wavelet;      /* [nt] */
    const double *src_pos;    /* [nshots][ndim] (host) */
    int nrec;
    const double *rec_pos;    /* [nrec][ndim] (host) */
    void *gather;             /* [nshots][nt][nrec] out (NULL: not recorded) */
    /* gradient mode only (NULL in forward mode): */
    const void *d_obs;        /* [nshots][nt][nrec] observed data */
    double *grad_sum_fp64;    /* [nz][ny][nx] DEVICE, += dJ/dv of this item's shots, summed in FP64 */
    double *misfit;           /* [1] host, out: J of this item's shots */
} sim_batch_item;

/* Forward modelling of many shots on many (uneven) 2D FP32 grids in one
 * batch. All handles must share dt and nt. Schedules: the row march, per
 * time step one launch over every (slice, shot, strip) of the batch, warps
 * taking row items from a per-step counter (two launches on two streams when
 * members have CPML: the CPML items and the plain ones); the two-step row
 * march (members without CPML: one launch per two steps, temporal
 * blocking); the stepped tile kernel (one launch per step); one persistent
 * dataflow launch for all steps whose tiles wait on their neighbours with
 * bounded waits (SIM_ERR_TIMEOUT when a wait gives up). On a stream other
 * than the legacy one the launches are captured as one CUDA graph and
 * replayed. The schedule and the tile height are picked by timing on the
 * first call for a batch shape (sim_get_info reports the pick);
 * GSIM_BATCH=march|march2|stepped|persistent forces one. `cuda_stream` as in
 * sim_create. */
sim_status sim_batch(int nitems, const sim_batch_item *items, void *cuda_stream);

/* The batch with a mode: 0 forward (sim_batch); 1 gradient: for each item,
 * the misfit of its shots against d_obs and its velocity gradient (as in
 * sim_adjoint, checkpoints in FP16 when ckpt_fp16) added in FP64 to the
 * item's grad_sum_fp64 (one array per slice; the caller sums slices that
 * share a model). 2D and 3D handles of any precision in mode 1. Items run
 * one after another, ordered on cuda_stream. */
sim_status sim_batch_ex(int nitems, const sim_batch_item *items, int mode, int ckpt_fp16, void *cuda_stream);

/* No counterpart in the paper. A forward solve for callers that cannot
 * allocate device memory at the time they call: processes whose device
 * memory is already reserved in full by a framework's pool (a cudaMalloc
 * there would fail), and latency-critical paths where cudaMalloc / cudaFree,
 * which may synchronise the device, are not acceptable.
 * 2D, FP32, one shot, gather only: vel [nz][nx], wavelet [nt] and
 * gather [nt][nrec] are device pointers; src_pos [2] and rec_pos [nrec][2]
 * are host arrays as in sim_forward. Every intermediate lives in one 32 MiB
 * array built into the library (each GPU that loads the library holds it
 * until the process exits); a problem that does not fit returns SIM_ERR_ARG
 * before any GPU work. Nothing is allocated. Every call reads the velocity
 * range back and waits for cuda_stream, and copies host-built lists in, so
 * no call may be made while that stream (or, in global capture mode, any
 * stream) is being captured. The first call on a device looks up that
 * array's address with the device current and keeps it for the life of the
 * process: do not use the entry point across a cudaDeviceReset. All calls
 * share the array: each clears what must start at zero, and calls whose GPU
 * work overlaps (other streams or threads) race on it. Returns after the
 * solve has completed on cuda_stream (NULL: legacy stream); non-finite values
 * in the final field or the gather give SIM_ERR_UNSTABLE. Errors:
 * sim_last_error(NULL). */
sim_status sim_forward_noalloc(const sim_desc *d, const float *vel, const float *wavelet,
                               const double *src_pos, int nrec, const double *rec_pos, float *gather,
                               void *cuda_stream);

/* Band-passed Ricker source wavelet of the paper's production runs (Sec.
 * "Source Wavelet", Tab. bands): w(t) = Ricker of peak frequency f0 centred at
 * t0 = 1/f0, sampled at t = n dt (n = 0 .. nt-1), filtered by a digital
 * Butterworth band-pass of the given order (2 order poles, edges f_lo < f_hi,
 * bilinear transform with prewarped edges) forward and then backward in time
 * (zero phase; odd reflection of 3 (2 order + 1) samples at each end, every
 * section started in steady state), then divided by its l2 norm and multiplied
 * by sqrt((f_hi - f_lo) / 24 Hz). The paper's five bands use order 4.
 *   precision  SIM_FP32 or SIM_FP64: element type of out
 *   out        [nt], host or device memory, owned by the caller
 *   stream     CUDA stream (NULL: legacy default stream); the call returns
 *              when out is written
 * Runs on the current device; computes in FP64 on the GPU. Errors:
 * SIM_ERR_ARG (nt <= 3 (2 order + 1), dt <= 0, f0 <= 0, not 0 < f_lo < f_hi <
 * 1/(2 dt), order outside [1, 16], or a band so wide that the design has real
 * poles),
 * SIM_ERR_OOM, SIM_ERR_CUDA (text from sim_last_error(NULL)). */
sim_status sim_wavelet_bandpass(int nt, double dt, double f0, double f_lo, double f_hi, int order, int precision,
                                void *out, void *stream);

/* ---------------------------------------------------------------------------
 * Velocity-model builder warps: the pull-sample steps of the paper's model
 * generator modules Squish (Alg. squish), Fault (Alg. fault) and a
 * simplified Deposit (Alg. deposit), App. "Model builder modules". They run
 * on the GPU so generated models feed sim_create / sim_set_model / sim_batch
 * without leaving the device.
 *
 * Grids are (nz, ny, nx) row-major DEVICE arrays owned by the caller (ny = 1
 * for a 2D slice, z the depth index): velocities FP32 (m/s), labels int32
 * (the geologic layer of each voxel). Labels are optional, but on both sides
 * or neither. Outputs must not overlap the inputs. The drawn random fields
 * of the modules (fractal-noise displacements, bed thicknesses and
 * velocities, perturbed bed boundaries, texture) are inputs.
 *
 * Interpolation (the paper says "sinc"; this library's reading): an 8-tap
 * Lanczos-windowed sinc per axis (sinc(x) sinc(x/4), |x| < 4), weights
 * normalised to sum 1, taps beyond the grid taking the edge value; labels by
 * nearest neighbour (round half to even, clamped). A voxel whose pulled depth
 * lies outside [0, nz) takes fill_v / fill_label (Alg. fault; Squish alike);
 * depths down to -1e-6 count as 0. Source positions are computed in FP64,
 * weights and sums in FP32.
 *
 * Calls are stream-ordered on `stream` (NULL: legacy default stream) and
 * return after enqueue. Errors: SIM_ERR_ARG (sizes, NULL or overlapping
 * arrays, parameters out of range), SIM_ERR_CUDA (launch failure); text from
 * sim_last_error(NULL). */

/* Alg. squish: out(z, y, x) = in(z + dz(y, x), y, x).
 *   dz  [ny][nx] device, displacement in cells (a 2D fractal-noise field) */
sim_status sim_model_squish(int nz, int ny, int nx, const float *v_in, const int *lab_in, const float *dz,
                            float fill_v, int fill_label, float *v_out, int *lab_out, void *stream);

/* Alg. fault: a listric normal fault as a rotation about a cylinder whose
 * axis runs along strike. Frame (z down): dip-azimuth direction
 * e_d = (0, cos a, sin a) in (z, y, x), strike e_s = (0, -sin a, cos a);
 * the cylinder centre is c - (R sin dip) e_z - (R cos dip) e_d, so the fault
 * surface (radius R) passes through c with the given dip. Each voxel is
 * rotated about the axis by -chi d w slip/R (chi = +1 outside the cylinder,
 * the footwall, -1 inside; w the product of cosine tapers of
 * |r - R| / d_die, |angle - angle of c| / theta_die and |along-strike
 * offset| / d_perp, zero where any ratio reaches 1) and pulled from
 * 2 p - p_rotated. A 2D slice is the case a = +-pi/2 on ny = 1. */
typedef struct {
    double cz, cy, cx;   /* point on the fault surface, cells */
    double azimuth;      /* a, radians */
    double dip;          /* radians */
    double radius;       /* R, cells (> 0; large: planar fault) */
    double slip;         /* cells of arc along the fault */
    int direction;       /* +1 or -1 */
    int pad;
    double d_die;        /* cells (> 0) */
    double d_perp;       /* cells (> 0) */
    double theta_die;    /* radians (> 0) */
} sim_fault;
sim_status sim_model_fault(int nz, int ny, int nx, const float *v_in, const int *lab_in, const sim_fault *f,
                           float fill_v, int fill_label, float *v_out, int *lab_out, void *stream);

/* Alg. deposit, simplified: a slab of t rows with nbeds beds is laid on top
 * of the model (rows z < t; the model below is pushed down by t rows). In the
 * slab, l = number of bed boundaries above z, S_l = the deepest of them (0 in
 * the first bed), tau(z) = min(z / (f_top t), 1) min((t - z) / (f_base t), 1)
 * (a zero fraction: no taper on that side), vbar = mean bed velocity, and
 *   v = (vbar + beta z) + tau(z) [(vbed_l - vbar) + a_eta eta(z - floor(S_l) + off_l, y, x)]
 * with the texture depth clamped to [0, nzt); label = label0 + l. The final
 * conformance of the slab to an underlying topography is not applied. */
typedef struct {
    int t;               /* slab rows, 1 <= t <= nz */
    int nbeds;           /* 1 .. 128 */
    int nzt;             /* rows of the texture field eta */
    int label0;
    float beta;          /* m/s per row */
    float a_eta;         /* m/s per unit of texture */
    float f_top, f_base; /* taper fractions >= 0 */
} sim_deposit;
/*   bounds   [nbeds - 1][ny][nx] device: bed boundary depths in rows (noise
 *            already applied); may be NULL when nbeds == 1
 *   vbed     [nbeds] HOST bed velocities; offsets [nbeds] HOST texture offsets
 *   eta      [nzt][ny][nx] device texture, or NULL (no texture) */
sim_status sim_model_deposit(int nz, int ny, int nx, const float *v_in, const int *lab_in, const sim_deposit *p,
                             const float *bounds, const float *vbed, const int *offsets, const float *eta,
                             float *v_out, int *lab_out, void *stream);

/* Wait for the handle's stream and report any device-side failure. */
sim_status sim_sync(sim_t s);

/* Layout and model facts of a live handle. */
sim_status sim_get_info(sim_t s, sim_info *out);

/* Human-readable reason of the last failure on this handle (or on this thread
 * when s is NULL). Never NULL. */
const char *sim_last_error(sim_t s);

/* Free every resource of the handle (NULL is a no-op). */
void sim_destroy(sim_t s);

#ifdef __cplusplus
}
#endif
#endif
