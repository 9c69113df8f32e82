// libsim C ABI: descriptor validation, device allocation, model set-up,
// acquisition geometry (receiver and injection lists per tile) and the time
// loop. Host code only; kernels live in the other translation units.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <type_traits>
#include <vector>

#include "sim_internal.h"
#include "stencil.cuh"

using namespace gsim;

namespace {

thread_local std::string t_err;

std::string vfmt(const char *fmt, va_list ap) {
    char buf[1024];
    vsnprintf(buf, sizeof buf, fmt, ap);
    return buf;
}

sim_status thread_fail(sim_status code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    t_err = vfmt(fmt, ap);
    va_end(ap);
    return code;
}

long long roundup(long long v, long long m) { return (v + m - 1) / m * m; }

// 1D profile arrays (sponge E, CPML a/b) live in one buffer per kind: per axis
// z, y, x a block of [kProfAlign zeros | N rounded up to kProfAlign | kProfAlign
// zeros], so tile-wide vector loads just outside [0, N) read zeros in bounds.
long long prof_block(int N) { return kProfAlign + roundup(N, kProfAlign) + kProfAlign; }
long long prof_offset(const Geom &g, int axis) {
    const int N[3] = {g.NZ, g.NY, g.NX};
    long long off = kProfAlign;
    for (int a = 0; a < axis; a++) off += prof_block(N[a]);
    return off;
}
long long prof_total(const Geom &g) { return prof_block(g.NZ) + prof_block(g.NY) + prof_block(g.NX); }

// Stability bounds of the 8th-order scheme (App. E.3.2).
double symbol_sum_abs() { return std::fabs(kC1) + std::fabs(kC2) + std::fabs(kC3) + std::fabs(kC4); }
double courant_paper(int d) { return 1.0 / std::sqrt(d * symbol_sum_abs()); }
double courant_exact(int d) {
    const double sym = -(kC0 - 2 * kC1 + 2 * kC2 - 2 * kC3 + 2 * kC4);  // symbol at theta = pi
    return 2.0 / std::sqrt(d * sym);
}

int nsnap_of(const sim_desc &d) {
    if (d.snap_every <= 0) return 0;
    const int end = std::min(d.snap_end, d.nt);
    if (d.snap_begin < 0 || end <= d.snap_begin) return 0;
    return (end - d.snap_begin + d.snap_every - 1) / d.snap_every;
}

void normalise(sim_desc &d) {
    if (d.space_order == 0) d.space_order = 8;
    if (!(d.R > 0)) d.R = 1e-3;
    if (!(d.f_ref > 0)) d.f_ref = 10.0;
    if (d.max_shots <= 0) d.max_shots = 1;
    if (d.ndim == 2) {
        d.ny = 1;
        d.nb[2] = d.nb[3] = 0;
    }
}

sim_status validate(const sim_desc &d) {
    if (d.ndim != 2 && d.ndim != 3) return thread_fail(SIM_ERR_ARG, "ndim must be 2 or 3 (got %d)", d.ndim);
    if (d.nz < 1 || d.nx < 1 || d.ny < 1) return thread_fail(SIM_ERR_ARG, "grid extents must be >= 1");
    if (!(d.h > 0) || !(d.dt > 0)) return thread_fail(SIM_ERR_ARG, "h and dt must be positive");
    if (d.nt < 1) return thread_fail(SIM_ERR_ARG, "nt must be >= 1");
    if (d.space_order != 8) return thread_fail(SIM_ERR_UNSUPPORTED, "only space_order 8 is built");
    if (d.bc < 0 || d.bc > 2) return thread_fail(SIM_ERR_ARG, "unknown bc %d", d.bc);
    for (int k = 0; k < 6; k++)
        if (d.nb[k] < 0 || d.nb[k] > 4096) return thread_fail(SIM_ERR_ARG, "nb[%d] out of range", k);
    if (d.free_surface && d.nb[0] != 0)
        return thread_fail(SIM_ERR_ARG, "a free surface needs nb[0] = 0 (no absorbing layer on top)");
    if (d.snap_every < 0) return thread_fail(SIM_ERR_ARG, "snap_every must be >= 0");
    if (d.precision != SIM_FP32 && d.precision != SIM_FP64) return thread_fail(SIM_ERR_ARG, "bad precision");
    if (d.snap_fp16 && d.precision != SIM_FP32)
        return thread_fail(SIM_ERR_ARG, "FP16 snapshots need an FP32 handle");
    if (d.max_rec < 0) return thread_fail(SIM_ERR_ARG, "max_rec must be >= 0");
    const long long NZ = (long long)d.nb[0] + d.nz + d.nb[1];
    const long long NY = d.ndim == 3 ? (long long)d.nb[2] + d.ny + d.nb[3] : 1;
    const long long NX = (long long)d.nb[4] + d.nx + d.nb[5];
    if (NZ > (1 << 20) || NY > (1 << 20) || NX > (1 << 20) || NZ * NY * NX > (1LL << 36))
        return thread_fail(SIM_ERR_ARG, "grid too large");
    return SIM_OK;
}

Geom make_geom(const sim_desc &d) {
    Geom g{};
    g.ndim = d.ndim;
    g.nz = d.nz;
    g.ny = d.ndim == 3 ? d.ny : 1;
    g.nx = d.nx;
    g.nbz0 = d.nb[0];
    g.nbz1 = d.nb[1];
    g.nby0 = d.ndim == 3 ? d.nb[2] : 0;
    g.nby1 = d.ndim == 3 ? d.nb[3] : 0;
    g.nbx0 = d.nb[4];
    g.nbx1 = d.nb[5];
    g.NZ = g.nbz0 + g.nz + g.nbz1;
    g.NY = g.nby0 + g.ny + g.nby1;
    g.NX = g.nbx0 + g.nx + g.nbx1;
    g.oz = g.nbz0;
    g.oy = g.nby0;
    g.ox = g.nbx0;
    const int G = kGhost;
    g.P = (int)roundup(G + roundup(g.NX, kRoundX) + G, 32);
    g.PY = d.ndim == 3 ? (int)(G + roundup(g.NY, kRoundY) + G) : 1;
    const long long planes = G + roundup(g.NZ, kRoundZ) + G;
    g.fstride = planes * g.PY * g.P;
    g.org = ((long long)G * g.PY + (d.ndim == 3 ? G : 0)) * g.P + G;
    g.fs = d.free_surface;
    return g;
}

void fill_info(const sim_desc &d, sim_info *out) {
    memset(out, 0, sizeof(*out));
    out->NZ = d.nb[0] + d.nz + d.nb[1];
    out->NY = d.ndim == 3 ? d.nb[2] + d.ny + d.nb[3] : 1;
    out->NX = d.nb[4] + d.nx + d.nb[5];
    out->nsnap = nsnap_of(d);
    out->courant_limit = courant_paper(d.ndim);
    out->courant_exact = courant_exact(d.ndim);
    for (int k = 0; k < 6; k++) out->c_damp[k] = d.nb[k] > 0 ? 1.5 * std::log(1.0 / d.R) / d.nb[k] : 0.0;
    out->cells_per_shot = (long long)out->NZ * out->NY * out->NX;
    out->tile_x = d.precision == SIM_FP32 ? kTileXF : kTileX2;
    out->tile_y = 1;
    out->tile_z = d.precision == SIM_FP32 ? 16 : kTileZ2;
}

sim_status model_checks(const sim_desc &d, double vmin, double vmax, sim_info *info) {
    if (vmax > 0) {
        info->courant = vmax * d.dt / d.h;
        if (info->courant > courant_paper(d.ndim) && !d.skip_cfl_check)
            return thread_fail(SIM_ERR_CFL, "v_max dt / h = %.4f exceeds the stability bound %.4f",
                               info->courant, courant_paper(d.ndim));
    }
    info->vmin = vmin;
    info->vmax = vmax;
    if (vmin > 0 && d.f_max > 0 && d.h > vmin / (4.0 * d.f_max))
        return thread_fail(SIM_WARN_DISPERSION, "h = %g m exceeds v_min / (4 f_max) = %g m", d.h,
                           vmin / (4.0 * d.f_max));
    return SIM_OK;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Interpolation stencil of a point: base cell (padded coordinates) and the
// fractional offsets; a coordinate within 1e-6 cells of a grid line snaps to it.
bool locate(const Geom &g, double h, const double *pos, int i0[3], double t[3]) {
    const int nd = g.ndim;
    double f[3];
    f[2] = pos[0] / h + g.ox;
    f[0] = pos[nd - 1] / h + g.oz;
    f[1] = nd == 3 ? pos[1] / h + g.oy : 0.0;
    const int lo[3] = {g.oz, g.oy, g.ox};
    const int len[3] = {g.nz, g.ny, g.nx};
    for (int a = 0; a < 3; a++) {
        const double r = std::nearbyint(f[a]);
        if (std::fabs(f[a] - r) < 1e-6) f[a] = r;
        if (!(f[a] >= lo[a]) || !(f[a] <= lo[a] + len[a] - 1)) return false;
        i0[a] = (int)std::floor(f[a]);
        t[a] = f[a] - i0[a];
    }
    return true;
}

double corner_weight(const double t[3], int dz, int dy, int dx) {
    return (dz ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) * (dx ? t[2] : 1.0 - t[2]);
}

}  // namespace

void gsim::set_thread_error(const char *msg) { t_err = msg; }

// ============================================================== handle

// Non-uniform 2D tiling (resident path): tile of each (column, row) and the
// first row of each tile. Columns are kTileXF wide.
struct TileMap {
    int NZ = 0, ntiles = 0;
    std::vector<int> tile;  // [bx * NZ + z]
    std::vector<int> z0;    // [tile]
};

// Resident-path decomposition for one shot count (see plan_resident).
struct ResidentPlan {
    int rz = 0;  // 0: the run does not fit on chip
    std::vector<RTile> tiles;
    TileMap map;
};

// Checkpoint schedule of the gradient and the sizes it was planned for
// (see plan_adjoint).
struct AdjPlan {
    int fp16 = 0;      // storage precision the buffers were sized for
    int levels = 1;
    int L = 1;         // imaging-term slots = steps of an innermost segment
    int m = 1;         // innermost segments per top segment (1 with one level)
    int n1 = 1;        // top-level checkpoints
    int n2 = 0;        // second-level checkpoint slots (m - 2: the first inner
                       // segment restarts from the top checkpoint, the last
                       // from the recompute itself)
    size_t ck_bytes = 0, q_bytes = 0, fixed_bytes = 0, total = 0;
};

struct sim_s {
    sim_desc d{};
    Geom g{};
    int dev = 0;
    cudaStream_t st = nullptr;
    size_t esz = 4;
    int ntx = 0, nty = 1, ntz = 0;
    int tile_x = kTileX2, tile_z = kTileZ2;  // tile of the step kernel in use
    int nsnap = 0;
    std::vector<void *> allocs;
    size_t bytes = 0;
    // device buffers
    void *pbuf = nullptr, *ch = nullptr, *vpad = nullptr, *vel = nullptr;
    void *E = nullptr, *ca = nullptr, *cb = nullptr;
    void *psi[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    void *zeta[3] = {nullptr, nullptr, nullptr};
    double *part = nullptr;
    SimIO *io = nullptr;
    unsigned *flags = nullptr;
    unsigned *snap_max = nullptr;
    float *snap_scale = nullptr;
    void *wave = nullptr, *gath = nullptr, *snaps = nullptr;
    size_t snaps_bytes = 0;
    int *rec_start = nullptr;
    void *rec = nullptr;      // RecEntryT<T>
    int *inj_start = nullptr;
    InjGroup *inj_grp = nullptr;
    void *inj_ent = nullptr;  // InjEntryT<T>
    size_t cap_rec = 0, cap_grp = 0, cap_start = 0;
    unsigned *flags_host = nullptr;  // pinned copy of the device flags
    // time loops are captured once per (kind, nshots) and replayed as CUDA graphs
    // on a handle-owned stream, ordered with the caller's stream by events
    cudaStream_t cst = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<std::pair<long long, cudaGraphExec_t>> graphs;
    bool use_graphs = true;
    int tuned_nshots = 0;  // shot count the tile shape was tuned for (0: not yet)
    bool use_march = false; // the autotuner's choice: row march rather than the tiled step kernel
    Pt3 *src3 = nullptr, *rec3 = nullptr;  // 3D point tables
    int *rdone = nullptr;                  // resident path: step counter per (shot, subdomain)
    Inj3 *src3g = nullptr, *res3g = nullptr;  // 3D adjoint: injection groups (sources, residuals)
    InjE3 *src3e = nullptr, *res3e = nullptr;
    RTile *rtiles = nullptr;               // resident path: subdomain descriptors
    const TileMap *tmap = nullptr;         // set while lists are built for a non-uniform tiling
    std::list<std::pair<int, ResidentPlan>> rplans;  // per shot count
    MarchSeg *mseg = nullptr;              // row march: segments, warp ranges, slice arguments
    StepArgs<float> *mslice = nullptr;
    size_t cap_mseg = 0;
    long long march_key = -1;              // (shot count, item rows, tile height) of the plan on the device
    int march_nwarps = 0, march_nitems = 0;
    unsigned *mctr = nullptr;              // row march: per-step item counters
    int last_path = 0, last_rows = 0;      // see sim_info
    int zchunk = 0;                        // z-march chunk of the 3D kernel (planes per CTA)
    int zvariant = kZMarchTma;             // z-march staging (cp.async or TMA), see autotune3d
    int batch_sched = 0, batch_tile = 0;   // schedule and tile of the last batch forward (as sim_info)
    void *pbuf3 = nullptr;                 // two-step row march: third and fourth pressure fields (max_shots shots each)
    int tuned3d = 0;                       // shot count the 3D launch shape was tuned for
    // adjoint-state buffers, allocated by the first sim_adjoint call (on
    // their own list: a call that needs a larger plan frees and re-plans them)
    bool adj_ready = false;
    AdjPlan plan;
    std::vector<void *> adj_allocs;
    size_t adj_bytes = 0;
    void *ubuf = nullptr, *Gbuf = nullptr, *qbuf = nullptr, *ckpt = nullptr, *res = nullptr, *dobs = nullptr;
    // 2D FP32 CPML gradient: multipliers nu [z, x][parity], mu [z, x], the
    // adjoint Laplacian term, and checkpoints of (psi_z, zeta_z, psi_x, zeta_x)
    void *cnu[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}}, *cmu[3] = {nullptr, nullptr, nullptr};
    void *cext = nullptr;
    float *qscale = nullptr;
    double *acc = nullptr, *mpart = nullptr;
    void *gradst = nullptr;
    int *inj2_start = nullptr;
    InjGroup *inj2_grp = nullptr;
    void *inj2_ent = nullptr;
    bool model_set = false;
    double vmin = 0, vmax = 0;
    sim_status sticky = SIM_OK;
    std::string err;

    sim_status fail(sim_status code, const char *fmt, ...) {
        va_list ap;
        va_start(ap, fmt);
        err = vfmt(fmt, ap);
        va_end(ap);
        t_err = err;
        if (code == SIM_ERR_CUDA || code == SIM_ERR_TIMEOUT || code == SIM_ERR_UNSTABLE) sticky = code;
        return code;
    }
    sim_status cuda(cudaError_t e, const char *what) {
        if (e == cudaSuccess) return SIM_OK;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SIM_ERR_OOM : SIM_ERR_CUDA, "%s: %s", what,
                    cudaGetErrorString(e));
    }
    void *alloc(size_t n, sim_status *rc) {
        void *p = nullptr;
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *rc = fail(SIM_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", n, cudaGetErrorString(e));
            return nullptr;
        }
        allocs.push_back(p);
        bytes += n;
        return p;
    }
    template <typename T>
    T *field(void *base, int shot) const {
        return static_cast<T *>(base) + (long long)shot * g.fstride;
    }
};

namespace {

// Surface device-side flags written by earlier work once the stream is idle.
sim_status poll_flags(sim_t s, bool wait) {
    if (s->sticky != SIM_OK) return s->sticky;
    if (wait) {
        if (sim_status r = s->cuda(cudaStreamSynchronize(s->st), "stream synchronize")) return r;
    } else if (cudaStreamQuery(s->st) != cudaSuccess) {
        cudaGetLastError();
        return SIM_OK;
    }
    const unsigned f = *s->flags_host;
    if (f & kFlagTimeout) return s->fail(SIM_ERR_TIMEOUT, "a bounded device wait gave up");
    if (f & kFlagUnstable) return s->fail(SIM_ERR_UNSTABLE, "non-finite values in the wavefield or outputs");
    return SIM_OK;
}

template <typename T>
void host_profiles(const sim_s &s, std::vector<T> &E, std::vector<T> &ca, std::vector<T> &cb) {
    const sim_desc &d = s.d;
    const Geom &g = s.g;
    const int N[3] = {g.NZ, g.NY, g.NX};
    const int lo[3] = {g.nbz0, g.nby0, g.nbx0}, hi[3] = {g.nbz1, g.nby1, g.nbx1};
    E.assign(prof_total(g), T(0));
    ca.assign(E.size(), T(0));
    cb.assign(E.size(), T(0));
    for (int a = 0; a < 3; a++) {
        const long long off = prof_offset(g, a);
        for (int i = 0; i < N[a]; i++) {
            int w = 0;
            double rho = 0;
            if (i < lo[a]) {
                w = lo[a];
                rho = double(lo[a] - i) / lo[a];
            } else if (i >= N[a] - hi[a]) {
                w = hi[a];
                rho = double(i - (N[a] - hi[a]) + 1) / hi[a];
            }
            if (w == 0) continue;
            if (d.bc == SIM_BC_SPONGE) {
                // Eq. cerjan_damp in SI (1e-3 s/m: the printed form uses km/s and ms),
                // stored as eta h^2 / (2 dt) so that a = c_field * E
                const double cdamp = 1.5 * std::log(1.0 / d.R) / w;
                const double eta = 1e-3 * (cdamp / d.h) * (rho - std::sin(2 * M_PI * rho) / (2 * M_PI));
                E[off + i] = T(eta * d.h * d.h / (2.0 * d.dt));
            } else if (d.bc == SIM_BC_CPML) {
                const double d0 = 3.0 * s.vmax * std::log(1.0 / d.R) / (2.0 * w * d.h);
                const double dd = d0 * rho * rho;
                const double alpha = M_PI * d.f_ref * (1.0 - rho);
                const double b = std::exp(-(dd + alpha) * d.dt);
                ca[off + i] = T(dd * (b - 1.0) / (dd + alpha));
                cb[off + i] = T(b);
            }
        }
    }
}

template <typename T>
sim_status set_model_t(sim_t s, const void *vel) {
    const Geom &g = s->g;
    const size_t nint = (size_t)g.nz * g.ny * g.nx;
    const void *src = vel;
    if (!is_device_ptr(vel)) {
        if (sim_status r = s->cuda(cudaMemcpyAsync(s->vel, vel, nint * sizeof(T), cudaMemcpyHostToDevice, s->st),
                                   "velocity upload"))
            return r;
        src = s->vel;
    } else if (vel != s->vel) {
        if (sim_status r = s->cuda(cudaMemcpyAsync(s->vel, vel, nint * sizeof(T), cudaMemcpyDeviceToDevice, s->st),
                                   "velocity copy"))
            return r;
        src = s->vel;
    }
    if (sim_status r = s->cuda(launch_minmax<T>(g, static_cast<const T *>(src), s->part, s->st), "minmax")) return r;
    std::vector<double> part(3 * kMinmaxBlocks);
    if (sim_status r = s->cuda(cudaMemcpyAsync(part.data(), s->part, part.size() * sizeof(double),
                                               cudaMemcpyDeviceToHost, s->st), "minmax readback"))
        return r;
    if (sim_status r = s->cuda(cudaStreamSynchronize(s->st), "minmax sync")) return r;
    double lo = 1e300, hi = -1e300, bad = 0;
    for (int b = 0; b < kMinmaxBlocks; b++) {
        lo = std::min(lo, part[3 * b]);
        hi = std::max(hi, part[3 * b + 1]);
        bad += part[3 * b + 2];
    }
    if (bad > 0) return s->fail(SIM_ERR_ARG, "velocity has %.0f non-finite or non-positive cells", bad);
    sim_info info{};
    sim_status chk = model_checks(s->d, lo, hi, &info);
    if (chk == SIM_ERR_CFL) {
        s->err = t_err;
        return chk;
    }
    s->vmin = lo;
    s->vmax = hi;
    std::vector<T> E, ca, cb;
    host_profiles<T>(*s, E, ca, cb);
    const size_t np = E.size() * sizeof(T);
    if (sim_status r = s->cuda(cudaMemcpyAsync(s->E, E.data(), np, cudaMemcpyHostToDevice, s->st), "profiles")) return r;
    if (sim_status r = s->cuda(cudaMemcpyAsync(s->ca, ca.data(), np, cudaMemcpyHostToDevice, s->st), "profiles")) return r;
    if (sim_status r = s->cuda(cudaMemcpyAsync(s->cb, cb.data(), np, cudaMemcpyHostToDevice, s->st), "profiles")) return r;
    if (sim_status r = s->cuda(launch_setup_model<T>(g, static_cast<const T *>(src), static_cast<T *>(s->ch),
                                                     static_cast<T *>(s->vpad), s->d.dt / s->d.h, s->st),
                               "model set-up"))
        return r;
    if (sim_status r = s->cuda(cudaStreamSynchronize(s->st), "model set-up sync")) return r;
    s->model_set = true;
    if (chk == SIM_WARN_DISPERSION) s->err = t_err;
    return chk;
}

// Tile holding 2D cell (z, x) and the cell's tile-local coordinates, for
// the uniform tiling of the handle or the non-uniform one being listed.
int tiles_of(const sim_s *s) { return s->tmap ? s->tmap->ntiles : s->ntx * s->nty * s->ntz; }
void tile_of(const sim_s *s, int z, int x, int &t, int &lz, int &lx) {
    const int bx = x / s->tile_x;
    if (s->tmap) {
        t = s->tmap->tile[(size_t)bx * s->tmap->NZ + z];
        lz = z - s->tmap->z0[t];
    } else {
        const int bz = z / s->tile_z;
        t = bz * s->ntx + bx;
        lz = z - bz * s->tile_z;
    }
    lx = x - bx * s->tile_x;
}

// Receivers: one entry per receiver, in the list of the tile that holds its
// base cell; the stencil corners lie within that tile's radius-4 halo.
template <typename T>
sim_status build_receivers(sim_t s, int nrec, const double *rec_pos, std::vector<int> &start,
                           std::vector<RecEntryT<T>> &ent) {
    const Geom &g = s->g;
    const int ntiles = tiles_of(s);
    std::vector<std::pair<int, RecEntryT<T>>> tmp;
    tmp.reserve(nrec);
    for (int r = 0; r < nrec; r++) {
        int i0[3];
        double t[3];
        if (!locate(g, s->d.h, rec_pos + (size_t)r * g.ndim, i0, t))
            return s->fail(SIM_ERR_ARG, "receiver %d lies outside the interior", r);
        RecEntryT<T> e{};
        e.rec = r;
        int tl;
        tile_of(s, i0[0], i0[2], tl, e.lz, e.lx);
        e.ly = 0;
        int k = 0;
        for (int dz = 0; dz < 2; dz++)
            for (int dy = 0; dy < (g.ndim == 3 ? 2 : 1); dy++)
                for (int dx = 0; dx < 2; dx++) e.w[k++] = T(corner_weight(t, dz, dy, dx));
        tmp.push_back({tl, e});
    }
    // by tile, then by row within the tile (the row march walks them in order)
    std::stable_sort(tmp.begin(), tmp.end(), [](const auto &a, const auto &b) {
        return a.first != b.first ? a.first < b.first : a.second.lz < b.second.lz;
    });
    start.assign(ntiles + 1, 0);
    ent.clear();
    for (auto &p : tmp) {
        start[p.first + 1]++;
        ent.push_back(p.second);
    }
    for (int i = 0; i < ntiles; i++) start[i + 1] += start[i];
    return SIM_OK;
}

struct InjPoint {
    int tile;   // list index (global tile)
    int cell;   // local linear index
    int pt;
    double w;
};

// Point injection: every stencil corner with a non-zero weight is a target
// cell of the tile that owns it (none on a free-surface row, which is held at
// zero). Targets are grouped per cell so one thread sums each cell in order.
template <typename T>
void group_injection(std::vector<InjPoint> &pts, int nlists, std::vector<int> &start,
                     std::vector<InjGroup> &grp, std::vector<InjEntryT<T>> &ent) {
    std::stable_sort(pts.begin(), pts.end(), [](const InjPoint &a, const InjPoint &b) {
        return a.tile != b.tile ? a.tile < b.tile : a.cell < b.cell;
    });
    start.assign(nlists + 1, 0);
    grp.clear();
    ent.clear();
    for (size_t i = 0; i < pts.size();) {
        size_t j = i;
        InjGroup G{};
        G.cell = pts[i].cell;
        G.e0 = (int)ent.size();
        while (j < pts.size() && pts[j].tile == pts[i].tile && pts[j].cell == pts[i].cell) {
            InjEntryT<T> e{};
            e.pt = pts[j].pt;
            e.w = T(pts[j].w);
            ent.push_back(e);
            j++;
        }
        G.e1 = (int)ent.size();
        grp.push_back(G);
        start[pts[i].tile + 1]++;
        i = j;
    }
    for (int i = 0; i < nlists; i++) start[i + 1] += start[i];
}

sim_status collect_points(sim_t s, int npts, const double *pos, bool per_shot, std::vector<InjPoint> &out,
                          const char *what) {
    const Geom &g = s->g;
    const int ntiles = tiles_of(s);
    for (int q = 0; q < npts; q++) {
        int i0[3];
        double t[3];
        if (!locate(g, s->d.h, pos + (size_t)q * g.ndim, i0, t))
            return s->fail(SIM_ERR_ARG, "%s %d lies outside the interior", what, q);
        for (int dz = 0; dz < 2; dz++)
            for (int dy = 0; dy < (g.ndim == 3 ? 2 : 1); dy++)
                for (int dx = 0; dx < 2; dx++) {
                    const double w = corner_weight(t, dz, dy, dx);
                    if (w == 0.0) continue;
                    const int z = i0[0] + dz, x = i0[2] + dx;
                    if (g.fs && z == 0) continue;
                    int tl, lz, lx;
                    tile_of(s, z, x, tl, lz, lx);
                    InjPoint p;
                    p.tile = (per_shot ? q * ntiles : 0) + tl;
                    p.cell = lz * s->tile_x + lx;
                    p.pt = q;
                    p.w = w;
                    out.push_back(p);
                }
    }
    return SIM_OK;
}

template <typename V>
sim_status upload(sim_t s, V *dst, const std::vector<V> &src, size_t cap, const char *what) {
    if (src.size() > cap) return s->fail(SIM_ERR_ARG, "%s list exceeds its capacity", what);
    if (src.empty()) return SIM_OK;
    return s->cuda(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice, s->st), what);
}

template <typename T>
StepArgs<T> step_args(sim_t s) {
    StepArgs<T> a{};
    a.g = s->g;
    a.pbuf[0] = static_cast<T *>(s->pbuf);
    a.pbuf[1] = static_cast<T *>(s->pbuf) + (long long)s->d.max_shots * s->g.fstride;
    a.ch = static_cast<const T *>(s->ch);
    for (int ax = 0; ax < 3; ax++) {
        const long long off = prof_offset(s->g, ax);
        a.E[ax] = s->d.bc == SIM_BC_SPONGE ? static_cast<const T *>(s->E) + off : nullptr;
        const bool on = s->d.bc == SIM_BC_CPML && s->psi[ax][0] != nullptr;
        a.ca[ax] = on ? static_cast<const T *>(s->ca) + off : nullptr;
        a.cb[ax] = on ? static_cast<const T *>(s->cb) + off : nullptr;
        a.psi[ax][0] = static_cast<T *>(s->psi[ax][0]);
        a.psi[ax][1] = static_cast<T *>(s->psi[ax][1]);
        a.zeta[ax] = static_cast<T *>(s->zeta[ax]);
    }
    a.bc = s->d.bc;
    a.src_scale = T(s->g.ndim == 3 ? 1.0 / s->d.h : 1.0);
    a.ntx = s->ntx;
    a.nty = s->nty;
    a.ntz = s->ntz;
    a.nt = s->d.nt;
    a.nsnap = s->nsnap;
    a.snap_every = s->d.snap_every > 0 ? s->d.snap_every : 1;
    a.snap_begin = s->d.snap_begin;
    a.snap_end = std::min(s->d.snap_end, s->d.nt);
    a.rec_start = s->rec_start;
    a.rec = static_cast<const RecEntryT<T> *>(s->rec);
    a.inj_start = s->inj_start;
    a.inj_grp = s->inj_grp;
    a.inj_ent = static_cast<const InjEntryT<T> *>(s->inj_ent);
    a.io = s->io;
    a.flags = s->flags;
    a.sample = 1;
    a.inj_reverse = 0;
    return a;
}

// Zero the per-run state of `nshots` shots: both pressure buffers, the CPML
// memory and the FP16 snapshot maxima.
cudaError_t reset_state_on(const sim_s *s, int nshots, cudaStream_t st) {
    const size_t fb = (size_t)s->g.fstride * s->esz * nshots;
    const size_t half = (size_t)s->g.fstride * s->esz * s->d.max_shots;
    cudaError_t e = cudaMemsetAsync(s->pbuf, 0, fb, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(static_cast<char *>(s->pbuf) + half, 0, fb, st);
    for (int ax = 0; ax < 3 && e == cudaSuccess; ax++) {
        for (int k = 0; k < 2 && e == cudaSuccess; k++)
            if (s->psi[ax][k]) e = cudaMemsetAsync(s->psi[ax][k], 0, fb, st);
        if (s->zeta[ax] && e == cudaSuccess) e = cudaMemsetAsync(s->zeta[ax], 0, fb, st);
    }
    if (s->nsnap > 0 && e == cudaSuccess) e = cudaMemsetAsync(s->snap_max, 0, sizeof(unsigned) * s->nsnap * nshots, st);
    return e;
}
sim_status reset_state(sim_t s, int nshots) { return s->cuda(reset_state_on(s, nshots, s->st), "reset"); }

// Per-launch facts of step n for the FP32 kernel (see StepTime).
template <typename T>
StepTime step_time(const sim_s *s, const StepArgs<T> &a, int n, int mode, void *qslot, float *qscale) {
    StepTime t{};
    t.n = n;
    t.snap_k = t.max_k = -1;
    auto snap_index = [&](int m) {
        if (a.nsnap <= 0 || m < a.snap_begin || m >= a.snap_end || (m - a.snap_begin) % a.snap_every) return -1;
        return (m - a.snap_begin) / a.snap_every;
    };
    if (mode == kModeForward) {
        t.snap_k = snap_index(n);
        if (s->d.snap_fp16) t.max_k = snap_index(n + 1);
    }
    const int row = a.inj_reverse ? a.nt - n : n;
    t.inj_row = (row >= 0 && row < a.nt) ? row : -1;
    t.qslot = qslot;
    t.qscale = qscale;
    return t;
}

template <typename T>
cudaError_t launch_step(sim_t s, const StepArgs<T> &a, int n, int nshots, int mode, cudaStream_t st,
                        void *qslot = nullptr, float *qscale = nullptr);
template <>
cudaError_t launch_step<float>(sim_t s, const StepArgs<float> &a, int n, int nshots, int mode, cudaStream_t st,
                               void *qslot, float *qscale) {
    return launch_step2d_f32(a, step_time(s, a, n, mode, qslot, qscale), s->tile_z, nshots, mode, st,
                             s->use_graphs);
}
template <>
cudaError_t launch_step<double>(sim_t s, const StepArgs<double> &a, int n, int nshots, int mode, cudaStream_t st,
                                void *qslot, float *qscale) {
    StepArgs<double> b = a;
    b.qslot = qslot;
    b.qscale = qscale;
    return launch_step2d<double>(b, n, nshots, mode, st);
}

// Run `body(stream)` — a sequence of kernel launches whose arguments depend
// only on handle-owned buffers — as a captured CUDA graph keyed by `key`
// (captured on first use, replayed afterwards), ordered after everything
// already queued on the handle's stream and before anything queued later.
template <typename F>
sim_status run_graph(sim_t s, long long key, F body) {
    if (!s->use_graphs) {
        cudaError_t e = body(s->st);
        return s->cuda(e, "time loop");
    }
    cudaGraphExec_t exec = nullptr;
    for (auto &kv : s->graphs)
        if (kv.first == key) exec = kv.second;
    if (!exec) {
        cudaGraph_t graph = nullptr;
        if (sim_status r = s->cuda(cudaStreamBeginCapture(s->cst, cudaStreamCaptureModeThreadLocal), "capture"))
            return r;
        cudaError_t e = body(s->cst);
        cudaError_t e2 = cudaStreamEndCapture(s->cst, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (sim_status r = s->cuda(e, "graph capture")) return r;
        s->graphs.push_back({key, exec});
    }
    if (sim_status r = s->cuda(cudaEventRecord(s->ev_in, s->st), "event")) return r;
    if (sim_status r = s->cuda(cudaStreamWaitEvent(s->cst, s->ev_in, 0), "event")) return r;
    if (sim_status r = s->cuda(cudaGraphLaunch(exec, s->cst), "graph launch")) return r;
    if (sim_status r = s->cuda(cudaEventRecord(s->ev_out, s->cst), "event")) return r;
    return s->cuda(cudaStreamWaitEvent(s->st, s->ev_out, 0), "event");
}

// ---------------------------------------------------------------- autotuner
//
// The FP32 step kernel comes in tile heights 8, 16 and 32 rows (x 128 cells).
// Which is fastest depends on the grid (waves per launch, share of CPML
// tiles) and on the shot count, so the first forward or adjoint call for a
// (grid, boundary, shots) key times a short run of each on this GPU with CUDA
// events and keeps the winner; the choice is cached for the process.
// GSIM_TILE_Z forces a height; GSIM_AUTOTUNE=0 keeps the default (16).
using TuneKey = std::tuple<int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune_cache;

// Most tiles any tuned shape can produce (sizes the per-tile lists).
long long max_tiles(const sim_s *s) {
    if (s->d.precision == SIM_FP32) return (long long)((s->g.NX + kTileXF - 1) / kTileXF) * ((s->g.NZ + 7) / 8);
    return (long long)((s->g.NX + kTileX2 - 1) / kTileX2) * ((s->g.NZ + kTileZ2 - 1) / kTileZ2);
}

void set_tile_z(sim_t s, int tz) {
    s->tile_z = tz;
    s->ntz = (s->g.NZ + tz - 1) / tz;
}

bool march_enabled(const sim_s *s);
sim_status march_prepare(sim_t s, const StepArgs<float> &a, int nshots, MarchArgs &m);

// 2D FP32 forward: the row march (march2d.cu) is one more candidate, timed
// the same way; GSIM_MARCH=1 takes it without timing, GSIM_MARCH=0 never.
int march_forced() {
    const char *f = getenv("GSIM_MARCH");
    return f ? (f[0] == '0' ? 0 : 1) : -1;
}

sim_status autotune(sim_t s, int nshots) {
    if (s->d.precision != SIM_FP32 || s->tuned_nshots == nshots) return SIM_OK;
    s->tuned_nshots = nshots;
    const bool can_march = march_enabled(s);
    const int forced = march_forced();
    s->use_march = can_march && forced != 0;  // untimed default
    if (const char *f = getenv("GSIM_TILE_Z")) {
        const int tz = atoi(f);
        if (tz == 8 || tz == 16 || tz == 32) set_tile_z(s, tz);
        return SIM_OK;
    }
    const char *at = getenv("GSIM_AUTOTUNE");
    if (at && at[0] == '0') return SIM_OK;
    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, s->dev);
    const TuneKey key{s->g.NZ, s->g.NX, s->d.bc, s->d.free_surface, nshots, dev_sms};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        // value: tile height | 256 if the march was faster | 512 if it was timed
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end() && (forced >= 0 || !can_march || (it->second & 512))) {
            set_tile_z(s, it->second & 0xff);
            if (forced < 0) s->use_march = can_march && (it->second & 256) != 0;
            return SIM_OK;
        }
    }
    const int cand[3] = {8, 16, 32};
    float best = 1e30f;
    int best_tz = 16;
    cudaEvent_t e0, e1;
    if (sim_status r = s->cuda(cudaEventCreate(&e0), "tune event")) return r;
    if (sim_status r = s->cuda(cudaEventCreate(&e1), "tune event")) return r;
    sim_status rc = SIM_OK;
    for (int tz : cand) {
        set_tile_z(s, tz);
        const int ntiles = s->ntx * s->ntz;
        std::vector<int> zeros((size_t)nshots * ntiles + 1, 0);
        rc = upload(s, s->rec_start, zeros, s->cap_start, "tune lists");
        if (!rc) rc = upload(s, s->inj_start, zeros, s->cap_start, "tune lists");
        if (!rc) rc = reset_state(s, nshots);
        if (rc) break;
        StepArgs<float> a = step_args<float>(s);
        a.sample = 0;
        a.nsnap = 0;
        const int warm = 3, timed = 12;
        cudaError_t e = cudaSuccess;
        for (int n = 0; n < warm + timed && e == cudaSuccess; n++) {
            if (n == warm) e = cudaEventRecord(e0, s->st);
            if (e == cudaSuccess)
                e = launch_step2d_f32(a, step_time(s, a, n, kModeForward, nullptr, nullptr), tz, nshots,
                                      kModeForward, s->st, false);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s->st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if ((rc = s->cuda(e, "autotune"))) break;
        if (getenv("GSIM_TUNE_LOG"))
            fprintf(stderr, "[gsim autotune] grid %dx%d shots %d tile 128x%d: %.2f us/step\n", s->g.NZ, s->g.NX,
                    nshots, tz, 1e3 * ms / timed);
        if (ms < best) {
            best = ms;
            best_tz = tz;
        }
    }
    bool march_best = false;
    const bool march_timed = !rc && can_march && forced < 0;
    if (march_timed) {  // the row march, with empty lists of the finest tiling
        set_tile_z(s, 8);
        std::vector<int> zeros((size_t)nshots * s->ntx * s->ntz + 1, 0);
        rc = upload(s, s->rec_start, zeros, s->cap_start, "tune lists");
        if (!rc) rc = upload(s, s->inj_start, zeros, s->cap_start, "tune lists");
        if (!rc) rc = reset_state(s, nshots);
        StepArgs<float> a = step_args<float>(s);
        a.sample = 0;
        a.nsnap = 0;
        MarchArgs m{};
        if (!rc) rc = march_prepare(s, a, nshots, m);
        if (!rc) {
            const int warm = 3, timed = 12;
            cudaError_t e = m.ctr ? cudaMemsetAsync(m.ctr, 0, 2 * sizeof(unsigned), s->st) : cudaSuccess;
            for (int n = 0; n < warm + timed && e == cudaSuccess; n++) {
                if (n == warm) e = cudaEventRecord(e0, s->st);
                if (e == cudaSuccess)
                    e = launch_march2d(m, s->d.bc == SIM_BC_CPML, step_time(s, a, n, kModeForward, nullptr, nullptr),
                                       s->st, false);
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, s->st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            rc = s->cuda(e, "autotune");
            if (!rc && getenv("GSIM_TUNE_LOG"))
                fprintf(stderr, "[gsim autotune] grid %dx%d shots %d row march: %.2f us/step\n", s->g.NZ, s->g.NX,
                        nshots, 1e3 * ms / timed);
            if (!rc && ms < best) march_best = true;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_tile_z(s, best_tz);
    if (forced < 0) s->use_march = march_best;
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best_tz | (march_best ? 256 : 0) | (march_timed ? 512 : 0);
    return SIM_OK;
}

// z-chunks of the 3D z-march: enough CTAs for two per SM, at least 64 planes per chunk
int zchunk_for(const sim_s *s, int nshots) {
    const Geom &g = s->g;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->dev);
    const long long cols = (long long)s->ntx * ((g.NY + 7) / 8) * nshots;
    const int chunks = (int)std::max<long long>(1, std::min<long long>((2LL * sms + cols - 1) / cols, g.NZ / 64));
    return (g.NZ + chunks - 1) / chunks;
}

// One forward-type 3D step without its point work: the CPML passes of the
// absorbing axes around the z-march (the x axis first, as the march that
// folds the x strips in adds their term first), skipping the x pass when the
// march takes it over. slot: the record mode's imaging term (else NULL).
cudaError_t step3d_core(const sim_s *s, const StepArgs<float> &a, int n, int variant, int zc, int nshots,
                        cudaStream_t st, bool pdl, int mode, float *slot) {
    const bool cpml = s->d.bc == SIM_BC_CPML;
    const bool on[3] = {s->psi[0][0] != nullptr, s->psi[1][0] != nullptr, s->psi[2][0] != nullptr};
    const bool fx = cpml && zmarch_folds_x(a, variant, mode);
    const int order[3] = {2, 0, 1};
    cudaError_t e = cudaSuccess;
    for (int ax : order)
        if (e == cudaSuccess && cpml && on[ax] && !(ax == 2 && fx)) e = launch_cpml3d(a, n, ax, 0, nshots, st);
    if (e == cudaSuccess) e = launch_step3d(a, n, variant, zc, nshots, st, pdl, mode, slot, nullptr);
    for (int ax : order)
        if (e == cudaSuccess && cpml && on[ax] && !(ax == 2 && fx)) e = launch_cpml3d(a, n, ax, 1, nshots, st, slot);
    return e;
}

// 3D launch shape: the z-march variant (per-thread cp.async or TMA staging)
// and the planes per CTA (z chunk: fewer, longer columns re-read less halo;
// more, shorter ones fill the GPU). The first forward or gradient call for a
// shot count times a few steps of each candidate on this GPU with CUDA
// events (on zeroed fields, before the run resets them) and keeps the
// fastest. GSIM_ZMARCH=async|tma|tma-plain|tma-loop|tma-loop-fold|tma-loop3 fixes the
// variant, GSIM_ZCHUNK the chunk;
// GSIM_AUTOTUNE=0 takes the TMA variant with the default chunk untimed.
sim_status autotune3d(sim_t s, int nshots) {
    if (s->tuned3d == nshots) return SIM_OK;
    s->tuned3d = nshots;
    const int base = zchunk_for(s, nshots), NZ = s->g.NZ;
    std::vector<int> variants = {kZMarchTmaLoop3, kZMarchTmaPlain, kZMarchTmaLoop, kZMarchTma, kZMarchTmaFoldLoop,
                                 kZMarchAsync};
    if (s->d.bc != SIM_BC_CPML)  // no x strips to fold
        variants = {kZMarchTmaLoop3, kZMarchTmaPlain, kZMarchTmaLoop, kZMarchAsync};
    static const char *const names[7] = {"", "async", "tma", "tma-plain", "tma-loop", "tma-loop-fold", "tma-loop3"};
    if (const char *f = getenv("GSIM_ZMARCH"))
        for (int v = 1; v <= 6; v++)
            if (!strcmp(f, names[v])) variants = {v};
    s->zvariant = variants[0];
    s->zchunk = base;
    const char *at = getenv("GSIM_AUTOTUNE");
    if (at && at[0] == '0') return SIM_OK;
    std::vector<int> chunks = {base};
    for (int c : {NZ, (NZ + 1) / 2, (NZ + 3) / 4, (NZ + 7) / 8})
        if (c >= 16 && std::find(chunks.begin(), chunks.end(), c) == chunks.end()) chunks.push_back(c);
    if (const char *f = getenv("GSIM_ZCHUNK")) {  // a fixed chunk (tests)
        chunks = {std::max(1, std::min(NZ, atoi(f)))};
        s->zchunk = chunks[0];
    }
    if (variants.size() == 1 && chunks.size() == 1) return SIM_OK;
    if (sim_status r = reset_state(s, nshots)) return r;
    StepArgs<float> a = step_args<float>(s);
    cudaEvent_t e0, e1;
    if (sim_status r = s->cuda(cudaEventCreate(&e0), "tune event")) return r;
    if (sim_status r = s->cuda(cudaEventCreate(&e1), "tune event")) {
        cudaEventDestroy(e0);
        return r;
    }
    float best = 1e30f;
    cudaError_t e = cudaSuccess;
    for (int v : variants)
        for (int zc : chunks) {
            const int warm = 1, timed = 3;
            for (int n = 0; n < warm + timed && e == cudaSuccess; n++) {
                if (n == warm) e = cudaEventRecord(e0, s->st);
                if (e == cudaSuccess) e = step3d_core(s, a, n, v, zc, nshots, s->st, false, kModeForward, nullptr);
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, s->st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) break;
            if (getenv("GSIM_TUNE_LOG"))
                fprintf(stderr, "[gsim autotune] 3D %dx%dx%d shots %d %s chunk %d: %.1f us/step\n", s->g.NZ, s->g.NY,
                        s->g.NX, nshots, names[v], zc, 1e3 * ms / timed);
            if (ms < best) {
                best = ms;
                s->zvariant = v;
                s->zchunk = zc;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s->cuda(e, "3D autotune");
}

// 3D points: the 8 trilinear corners of each point as field offsets.
sim_status points3d(sim_t s, int npts, const double *pos, std::vector<Pt3> &out, bool drop_surface,
                    const char *what) {
    const Geom &g = s->g;
    out.resize(npts);
    for (int q = 0; q < npts; q++) {
        int i0[3];
        double t[3];
        if (!locate(g, s->d.h, pos + (size_t)q * 3, i0, t))
            return s->fail(SIM_ERR_ARG, "%s %d lies outside the interior", what, q);
        Pt3 &P = out[q];
        int k = 0;
        for (int dz = 0; dz < 2; dz++)
            for (int dy = 0; dy < 2; dy++)
                for (int dx = 0; dx < 2; dx++, k++) {
                    const double w = corner_weight(t, dz, dy, dx);
                    const int z = i0[0] + dz;
                    if (w == 0.0 || (drop_surface && g.fs && z == 0)) {
                        P.cell[k] = -1;
                        P.w[k] = 0.f;
                        continue;
                    }
                    P.cell[k] = cell_off(g, z, i0[1] + dy, i0[2] + dx);
                    P.w[k] = (float)w;
                }
    }
    return SIM_OK;
}

sim_status forward3d(sim_t s, int nshots, const void *wav, const double *src_pos, int nrec, const double *rec_pos,
                     void *gdev, void *sdev, float *scdev) {
    const sim_desc &d = s->d;
    if (d.precision != SIM_FP32) return s->fail(SIM_ERR_UNSUPPORTED, "the 3D path runs in FP32");
    std::vector<Pt3> src, rec;
    if (wav)
        if (sim_status r = points3d(s, nshots, src_pos, src, true, "source")) return r;
    if (sim_status r = points3d(s, nrec, rec_pos, rec, false, "receiver")) return r;
    if (!src.empty())
        if (sim_status r = s->cuda(cudaMemcpyAsync(s->src3, src.data(), src.size() * sizeof(Pt3),
                                                   cudaMemcpyHostToDevice, s->st), "source upload"))
            return r;
    if (!rec.empty())
        if (sim_status r = s->cuda(cudaMemcpyAsync(s->rec3, rec.data(), rec.size() * sizeof(Pt3),
                                                   cudaMemcpyHostToDevice, s->st), "receiver upload"))
            return r;
    SimIO io{};
    io.wavelet = wav;
    io.gather = nrec > 0 ? gdev : nullptr;
    io.snaps = s->nsnap > 0 ? sdev : nullptr;
    io.snap_scale = scdev;
    io.snap_max = s->snap_max;
    io.nrec = nrec;
    io.nshots = nshots;
    io.snap_fp16 = d.snap_fp16;
    if (sim_status r = s->cuda(cudaMemcpyAsync(s->io, &io, sizeof io, cudaMemcpyHostToDevice, s->st), "io upload"))
        return r;
    if (sim_status r = autotune3d(s, nshots)) return r;
    if (sim_status r = reset_state(s, nshots)) return r;
    StepArgs<float> a = step_args<float>(s);
    a.inj_per_shot = 1;
    a.inj_kind = 0;
    a.sample = nrec > 0 && gdev != nullptr;
    const bool has_src = !src.empty(), has_snap = io.snaps != nullptr;
    const Pt3 *s3 = s->src3, *r3 = s->rec3;
    return run_graph(s, ((long long)nshots << 8) | (3 << 2) | 2, [&](cudaStream_t st) {
        cudaError_t e = cudaSuccess;
        for (int n = 0; n < d.nt && e == cudaSuccess; n++) {
            const StepTime t = step_time(s, a, n, kModeForward, nullptr, nullptr);
            if (has_snap && t.snap_k >= 0) e = launch_snap3d(a, t, d.snap_fp16, nshots, st);
            if (e == cudaSuccess && a.sample) e = launch_sample3d(a, t, r3, nrec, nshots, st);
            if (e == cudaSuccess)
                e = step3d_core(s, a, n, s->zvariant, s->zchunk, nshots, st, false, kModeForward, nullptr);
            if (e == cudaSuccess && has_src) e = launch_inject3d(a, t, s3, nshots, st);
        }
        return e;
    });
}

// Polls a dataflow wait makes before it gives up (GSIM_SPIN_LIMIT overrides).
long long spin_limit() {
    long long v = 1LL << 22;
    if (const char *f = getenv("GSIM_SPIN_LIMIT")) v = atoll(f);
    return v;
}

// Resident forward path (resident2d.cu). The slice is cut into columns of
// kTileXF cells and each column into subdomains of at most 16 RZ rows, as
// even in time per step as the GPU allows. Cost model (fitted to per-CTA
// phase timings of this kernel, in units of one interior row): a subdomain
// costs 50 (halo exchange and barriers) plus, per row, 1, plus 0.039 per
// CPML x-strip float4 chunk its column updates, plus 1.34 within 4 rows of a
// CPML z-strip. The smallest target cost whose subdomains (times the shots)
// all fit on the GPU at once is chosen, trying RZ = 1, 2, ... 2D FP32 forward
// runs with FP32 (or no) snapshots only; GSIM_RESIDENT=0 turns the path off.
// CPML x-strip float4 chunks (psi and zeta) a column updates, as the kernel counts them.
int strip_chunks(const Geom &g, int bx) {
    const int x0 = bx * kTileXF;
    int lo = 1 << 30, hi = -(1 << 30);
    auto part = [&](int a, int b) {
        a = std::max(a - x0, -4);
        b = std::min(b - x0, kTileXF + 4);
        if (a < b) lo = std::min(lo, a), hi = std::max(hi, b);
    };
    if (g.nbx0 > 0) part(0, g.nbx0);
    if (g.nbx1 > 0) part(g.NX - g.nbx1, g.NX);
    if (lo >= hi) return 0;
    const int ncx = ((hi + 7) >> 2) - ((lo + 4) >> 2);
    const int nax = ((std::min(kTileXF, hi + 4) + 3) >> 2) - (std::max(0, lo - 4) >> 2);
    return ncx + nax;
}

bool cut_columns(const sim_s *s, int wz, double target, std::vector<RTile> &tiles) {
    const Geom &g = s->g;
    const bool cp = s->d.bc == SIM_BC_CPML;
    const int ntx = (g.NX + kTileXF - 1) / kTileXF, hmin = 8;
    tiles.clear();
    for (int bx = 0; bx < ntx; bx++) {
        const double cx = cp ? 0.039 * strip_chunks(g, bx) : 0.0;
        int z = 0;
        while (z < g.NZ) {
            RTile t{};
            t.bx = bx;
            t.z0 = z;
            double acc = 50.0;
            while (z < g.NZ && t.rows < wz) {
                const bool zs = cp && ((g.nbz0 > 0 && z < g.nbz0 + 4) || (g.nbz1 > 0 && z >= g.NZ - g.nbz1 - 4));
                const double c = 1.0 + cx + (zs ? 1.34 : 0.0);
                if (t.rows >= hmin && acc + c > target) break;
                acc += c;
                t.rows++;
                z++;
            }
            tiles.push_back(t);
        }
        // a short last subdomain joins the one above when both fit in wz rows
        const size_t k = tiles.size();
        if (k >= 2 && tiles[k - 1].bx == bx && tiles[k - 2].bx == bx && tiles[k - 1].rows < hmin &&
            tiles[k - 2].rows + tiles[k - 1].rows <= wz) {
            tiles[k - 2].rows += tiles[k - 1].rows;
            tiles.pop_back();
        }
    }
    for (RTile &t : tiles) t.rpw = (t.rows + kResidentWarps - 1) / kResidentWarps;
    return true;
}

// Neighbours of each subdomain: above and below in its column, and those of
// the adjacent columns whose rows overlap its rows.
bool link_tiles(std::vector<RTile> &tiles) {
    for (size_t i = 0; i < tiles.size(); i++) {
        RTile &t = tiles[i];
        auto add = [&](size_t j) {
            if (t.nnbr >= kResidentMaxNbr) return false;
            t.nbr[t.nnbr++] = (int)j;
            return true;
        };
        for (size_t j = 0; j < tiles.size(); j++) {
            const RTile &u = tiles[j];
            bool nb = false;
            if (u.bx == t.bx) nb = u.z0 + u.rows == t.z0 || t.z0 + t.rows == u.z0;
            else if (u.bx == t.bx - 1 || u.bx == t.bx + 1) nb = u.z0 < t.z0 + t.rows && t.z0 < u.z0 + u.rows;
            if (nb && !add(j)) return false;
        }
    }
    return true;
}

bool plan_resident_uncached(sim_t s, int nshots, ResidentPlan &plan) {
    int sms = 0, coop = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->dev);
    if (!coop || sms <= 0) return false;
    const long long cap_tiles = max_tiles(s);  // step counters and descriptors
    for (int rz = 1; rz <= 4; rz++) {
        const int bps = resident2d_blocks_per_sm(rz, s->d.bc);
        if (bps <= 0) continue;
        const long long cap = std::min((long long)bps * sms / nshots, cap_tiles);
        const int wz = kResidentWarps * rz;
        std::vector<RTile> t;
        // the largest target gives uniform wz-row subdomains (the fewest)
        if (!cut_columns(s, wz, 1e30, t) || (long long)t.size() > cap) continue;
        double lo = 50, hi = 50 + 4.0 * wz;
        for (int it = 0; it < 40; it++) {
            const double mid = 0.5 * (lo + hi);
            if (cut_columns(s, wz, mid, t) && (long long)t.size() <= cap) hi = mid;
            else lo = mid;
        }
        if (!cut_columns(s, wz, hi, t) || (long long)t.size() > cap || !link_tiles(t)) continue;
        plan.rz = rz;
        plan.tiles = t;
        TileMap &m = plan.map;
        m.NZ = s->g.NZ;
        m.ntiles = (int)t.size();
        m.tile.assign((size_t)((s->g.NX + kTileXF - 1) / kTileXF) * m.NZ, -1);
        m.z0.resize(t.size());
        for (size_t i = 0; i < t.size(); i++) {
            m.z0[i] = t[i].z0;
            for (int r = 0; r < t[i].rows; r++) m.tile[(size_t)t[i].bx * m.NZ + t[i].z0 + r] = (int)i;
        }
        return true;
    }
    return false;
}

// The plan depends only on the grid and the shot count: kept per handle.
const ResidentPlan *plan_resident(sim_t s, int nshots) {
    if (s->g.ndim != 2 || s->d.precision != SIM_FP32 || s->d.snap_fp16 || !s->rdone) return nullptr;
    const char *f = getenv("GSIM_RESIDENT");
    if (f && f[0] == '0') return nullptr;
    for (const auto &p : s->rplans)
        if (p.first == nshots) return p.second.rz ? &p.second : nullptr;
    s->rplans.emplace_back(nshots, ResidentPlan{});
    ResidentPlan &p = s->rplans.back().second;
    if (!plan_resident_uncached(s, nshots, p)) p = ResidentPlan{};
    return p.rz ? &p : nullptr;
}

// One cooperative launch for the whole time loop, after zeroing the step
// counters; ordered on the handle's stream like any other work.
template <typename T>
sim_status run_resident(sim_t s, const StepArgs<T> &a, const ResidentPlan &plan, int nshots);
template <>
sim_status run_resident<double>(sim_t s, const StepArgs<double> &, const ResidentPlan &, int) {
    return s->fail(SIM_ERR_UNSUPPORTED, "the resident path is FP32 only");
}
template <>
sim_status run_resident<float>(sim_t s, const StepArgs<float> &a, const ResidentPlan &plan, int nshots) {
    const int nt = (int)plan.tiles.size();
    if (sim_status r = upload(s, s->rtiles, plan.tiles, (size_t)max_tiles(s), "subdomains")) return r;
    if (sim_status r = s->cuda(cudaMemsetAsync(s->rdone, 0, (size_t)nt * nshots * sizeof(int), s->st),
                               "step counters"))
        return r;
    ResidentArgs r{s->rdone, spin_limit(), s->rtiles, nt};
    return s->cuda(launch_resident2d(a, r, plan.rz, nshots, s->st), "resident launch");
}

// ---------------------------------------------------------------- row march plan

struct MarchMember {
    int slice, shot;
    const sim_s *s;
};

// Dynamic schedule: the step's work as items of `item` rows of one strip of
// one member. Items that update CPML memory (their strip within 4 cells of
// an x strip, or a row within 4 rows of a z strip) take the slower CPML
// loop, so they come first; then by member, band of rows and strip, so the
// items taken at about the same time cover neighbouring strips of the same
// rows. Returns the number of warps to launch (one per item at most).
int march_item_rows() {
    int k = 16;
    if (const char *f = getenv("GSIM_MARCH_ITEM")) k = std::max(4, atoi(f));
    return (k + 3) & ~3;
}
int plan_march_items(const std::vector<MarchMember> &mem, long long max_warps, int item, std::vector<MarchSeg> &segs,
                     int *ncpml = nullptr) {
    segs.clear();
    for (int pass = 0; pass < 2; pass++)
        for (const MarchMember &m : mem) {
            const Geom &g = m.s->g;
            const bool cp = m.s->d.bc == SIM_BC_CPML;
            const int NZ = g.NZ, ntx = (g.NX + kMarchW - 1) / kMarchW;
            for (int zc = 0; zc < NZ; zc += item)
                for (int bx = 0; bx < ntx; bx++) {
                    const int x0 = bx * kMarchW, ze = std::min(NZ, zc + item);
                    const bool c = cp && ((g.nbx0 > 0 && x0 - 4 < g.nbx0) ||
                                          (g.nbx1 > 0 && x0 + kMarchW + 4 > g.NX - g.nbx1) ||
                                          (g.nbz0 > 0 && zc < g.nbz0 + 4) || (g.nbz1 > 0 && ze > NZ - g.nbz1 - 4));
                    if (c == (pass == 0)) segs.push_back(MarchSeg{m.slice, m.shot, bx, zc, ze, {0, 0, 0}});
                }
            if (pass == 0 && ncpml) *ncpml = (int)segs.size();
        }
    return (int)std::min<long long>(max_warps, (long long)segs.size());
}

bool march_enabled(const sim_s *s) {
    if (!s->mseg || s->g.ndim != 2 || s->d.precision != SIM_FP32) return false;
    const char *f = getenv("GSIM_MARCH");
    return !(f && f[0] == '0');
}

int device_sms(int dev) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Plan (when the shot count or list tiling changed) and slice arguments of a
// single-handle row march, uploaded to the handle's buffers.
sim_status march_prepare(sim_t s, const StepArgs<float> &a, int nshots, MarchArgs &m) {
    const int item = march_item_rows();
    const long long key = ((long long)nshots << 16) | ((long long)item << 6) | s->tile_z;
    if (key != s->march_key) {
        std::vector<MarchMember> mem;
        for (int k = 0; k < nshots; k++) mem.push_back({0, k, s});
        std::vector<MarchSeg> segs;
        const int maxw = device_sms(s->dev) * std::max(1, march2d_warps_per_sm(s->d.bc == SIM_BC_CPML));
        s->march_nwarps = plan_march_items(mem, maxw, item, segs);
        s->march_nitems = (int)segs.size();
        if (sim_status r = upload(s, s->mseg, segs, s->cap_mseg, "march segments")) return r;
        s->march_key = key;
    }
    if (sim_status r = s->cuda(cudaMemcpyAsync(s->mslice, &a, sizeof a, cudaMemcpyHostToDevice, s->st), "march args"))
        return r;
    m.slices = s->mslice;
    m.segs = s->mseg;
    m.ctr = s->mctr;
    m.nwarps = s->march_nwarps;
    m.nitems = s->march_nitems;
    m.tz = s->tile_z;
    return SIM_OK;
}

// The forward time loop as one row-march launch per step, captured as a graph.
template <typename T>
sim_status run_march(sim_t s, const StepArgs<T> &a, int nshots);
template <>
sim_status run_march<double>(sim_t s, const StepArgs<double> &, int) {
    return s->fail(SIM_ERR_UNSUPPORTED, "the row march is FP32 only");
}
template <>
sim_status run_march<float>(sim_t s, const StepArgs<float> &a, int nshots) {
    MarchArgs m{};
    if (sim_status r = march_prepare(s, a, nshots, m)) return r;
    const bool cpml = s->d.bc == SIM_BC_CPML;
    return run_graph(s, ((long long)nshots << 16) | ((long long)march_item_rows() << 8) | ((long long)s->tile_z << 2) | 3,
                     [&](cudaStream_t st) {
        cudaError_t e0 = cudaMemsetAsync(m.ctr, 0, 2 * sizeof(unsigned), st);
        if (e0 != cudaSuccess) return e0;
        for (int n = 0; n < s->d.nt; n++) {
            cudaError_t e = launch_march2d(m, cpml, step_time(s, a, n, kModeForward, nullptr, nullptr), st,
                                           s->use_graphs);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    });
}

template <typename T>
sim_status forward_t(sim_t s, int nshots, const void *wavelet, const double *src_pos, int nrec,
                     const double *rec_pos, void *gather, void *snaps, float *snap_scale) {
    const sim_desc &d = s->d;
    const Geom &g = s->g;
    const ResidentPlan *plan = std::is_same<T, float>::value ? plan_resident(s, nshots) : nullptr;
    const int rz = plan ? plan->rz : 0;
    if (g.ndim == 2 && !rz)
        if (sim_status r = autotune(s, nshots)) return r;
    const bool march = std::is_same<T, float>::value && g.ndim == 2 && !rz && s->use_march;
    const size_t nt = d.nt;
    // inputs
    const void *wav = wavelet;
    if (wavelet && !is_device_ptr(wavelet)) {
        if (sim_status r = s->cuda(cudaMemcpyAsync(s->wave, wavelet, nt * sizeof(T), cudaMemcpyHostToDevice, s->st),
                                   "wavelet upload"))
            return r;
        wav = s->wave;
    }
    // outputs
    const bool g_host = gather && !is_device_ptr(gather);
    void *gdev = g_host ? s->gath : gather;
    const size_t gbytes = (size_t)nshots * nt * nrec * sizeof(T);
    const bool sn_host = snaps && s->nsnap > 0 && !is_device_ptr(snaps);
    const size_t sesz = d.snap_fp16 ? 2 : sizeof(T);
    const size_t sbytes = (size_t)nshots * s->nsnap * g.nz * g.ny * g.nx * sesz;
    void *sdev = snaps;
    if (sn_host) {
        if (s->snaps_bytes < sbytes) {
            sim_status rc = SIM_OK;
            s->snaps = s->alloc(sbytes, &rc);
            if (!s->snaps) return rc;
            s->snaps_bytes = sbytes;
        }
        sdev = s->snaps;
    }
    const bool sc_host = snap_scale && !is_device_ptr(snap_scale);
    float *scdev = sc_host ? s->snap_scale : snap_scale;
    if (d.snap_fp16 && snaps && s->nsnap > 0 && !snap_scale)
        return s->fail(SIM_ERR_ARG, "FP16 snapshots need a snap_scale array");

    if (g.ndim == 3) {
        s->last_path = 3;
        if (sim_status r = forward3d(s, nshots, wav, src_pos, nrec, rec_pos, gdev, sdev, scdev)) return r;
    } else {
    // geometry lists, per tile of the kernel that runs (the resident
    // subdomains while this scope lasts)
    struct MapScope {
        sim_t s;
        ~MapScope() { s->tmap = nullptr; }
    } map_scope{s};
    s->tmap = rz ? &plan->map : nullptr;
    std::vector<int> rstart, istart;
    std::vector<RecEntryT<T>> rent;
    std::vector<InjGroup> igrp;
    std::vector<InjEntryT<T>> ient;
    if (sim_status r = build_receivers<T>(s, nrec, rec_pos, rstart, rent)) return r;
    std::vector<InjPoint> pts;
    if (wavelet)
        if (sim_status r = collect_points(s, nshots, src_pos, true, pts, "source")) return r;
    group_injection<T>(pts, nshots * tiles_of(s), istart, igrp, ient);
    if (sim_status r = upload(s, s->rec_start, rstart, s->cap_start, "receiver start")) return r;
    if (sim_status r = upload(s, static_cast<RecEntryT<T> *>(s->rec), rent, s->cap_rec, "receiver")) return r;
    if (sim_status r = upload(s, s->inj_start, istart, s->cap_start, "injection start")) return r;
    if (sim_status r = upload(s, s->inj_grp, igrp, s->cap_grp, "injection group")) return r;
    if (sim_status r = upload(s, static_cast<InjEntryT<T> *>(s->inj_ent), ient, s->cap_grp, "injection entry"))
        return r;

    SimIO io{};
    io.wavelet = wav;
    io.gather = nrec > 0 ? gdev : nullptr;
    io.snaps = s->nsnap > 0 ? sdev : nullptr;
    io.snap_scale = scdev;
    io.snap_max = s->snap_max;
    io.nrec = nrec;
    io.nshots = nshots;
    io.snap_fp16 = d.snap_fp16;
    if (sim_status r = s->cuda(cudaMemcpyAsync(s->io, &io, sizeof io, cudaMemcpyHostToDevice, s->st), "io upload"))
        return r;
    if (sim_status r = reset_state(s, nshots)) return r;

    StepArgs<T> a = step_args<T>(s);
    a.inj_per_shot = 1;
    a.inj_kind = 0;
    s->last_path = rz ? 2 : (march ? 4 : 1);
    s->last_rows = 0;
    if (rz)
        for (const RTile &t : plan->tiles) s->last_rows = std::max(s->last_rows, t.rows);
    if (rz) {
        if (sim_status r = run_resident(s, a, *plan, nshots)) return r;
    } else if (march) {
        if (sim_status r = run_march(s, a, nshots)) return r;
    } else if (sim_status r = run_graph(s, ((long long)nshots << 8) | ((long long)s->tile_z << 2) | 1,
                                        [&](cudaStream_t st) {
                                            for (int n = 0; n < d.nt; n++) {
                                                cudaError_t e = launch_step<T>(s, a, n, nshots, kModeForward, st);
                                                if (e != cudaSuccess) return e;
                                            }
                                            return cudaSuccess;
                                        })) {
        return r;
    }
    }
    // the buffer written last holds p^nt
    const T *last = static_cast<const T *>(s->pbuf) + ((d.nt & 1) ? (long long)d.max_shots * g.fstride : 0);
    if (sim_status r = s->cuda(launch_check_finite<T>(g, last, nshots, s->flags, s->st), "finite check"))
        return r;
    if (sim_status r = s->cuda(cudaMemcpyAsync(s->flags_host, s->flags, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                               s->st), "flag readback"))
        return r;
    bool wait = false;
    if (g_host && nrec > 0) {
        if (sim_status r = s->cuda(cudaMemcpyAsync(gather, gdev, gbytes, cudaMemcpyDeviceToHost, s->st), "gather"))
            return r;
        wait = true;
    }
    if (sn_host) {
        if (sim_status r = s->cuda(cudaMemcpyAsync(snaps, sdev, sbytes, cudaMemcpyDeviceToHost, s->st), "snapshots"))
            return r;
        wait = true;
    }
    if (sc_host && d.snap_fp16 && s->nsnap > 0) {
        if (sim_status r = s->cuda(cudaMemcpyAsync(snap_scale, scdev, sizeof(float) * nshots * s->nsnap,
                                                   cudaMemcpyDeviceToHost, s->st), "scales"))
            return r;
        wait = true;
    }
    if (wait) return poll_flags(s, true);
    return SIM_OK;
}


constexpr int kResidBlocks = 1024;

// ---------------------------------------------------------------- adjoint plan
//
// The gradient needs the forward states in reverse order. They are rebuilt
// from checkpoints: the forward sweep keeps the state (p^{n-1}, p^n and the
// CPML memory) at the start of every top segment; in reverse, each top
// segment is restored and recomputed. With one level, the recompute records
// the imaging terms Q' of the whole segment into L slots and the adjoint
// sweep consumes them (two forward sweeps in all). With two levels, a top
// segment of m L steps is first recomputed once keeping a second-level
// checkpoint every L steps, then each inner segment is restored, recorded
// and swept as above (three forward sweeps). Memory: checkpoint slots
// (n1 + n2) x one state at the storage precision, plus L imaging-term slots.
// The plan is the cheapest that fits the device-memory budget: sqrt(nt)
// segments if they fit, else the one-level split that needs least memory,
// else the two-level one that needs least (the trade-off of optimal
// checkpointing; Sec. 5 names it).

// Checkpoint fields of the CPML state: psi and zeta of each absorbing axis.
// Field j of a checkpoint: axis cpml_axes[j / 2], psi (even j) or zeta (odd).
int cpml_ckpt_axes(const sim_s *s, int axes[3]) {
    int k = 0;
    for (int ax = 0; ax < 3; ax++)
        if (s->psi[ax][0]) axes[k++] = ax;
    return k;
}

// The strip boxes of axis ax (where its CPML memory can be non-zero).
CkBoxes strip_boxes(const Geom &g, int ax) {
    CkBoxes B{};
    const int N[3] = {g.NZ, g.NY, g.NX}, lo[3] = {g.nbz0, g.nby0, g.nbx0}, hi[3] = {g.nbz1, g.nby1, g.nbx1};
    const int r0[2] = {0, N[ax] - hi[ax]}, r1[2] = {lo[ax], N[ax]};
    for (int side = 0; side < 2; side++) {
        if (r1[side] <= r0[side]) continue;
        CkBox b{0, g.NZ, 0, g.NY, 0, g.NX};
        if (ax == 0) b.z0 = r0[side], b.z1 = r1[side];
        if (ax == 1) b.y0 = r0[side], b.y1 = r1[side];
        if (ax == 2) b.x0 = r0[side], b.x1 = r1[side];
        B.b[B.n++] = b;
    }
    for (int k = 0; k < B.n; k++) {
        const CkBox &b = B.b[k];
        const long long rows = (long long)(b.z1 - b.z0) * (b.y1 - b.y0);
        B.row0[k + 1] = B.row0[k] + rows;
        B.elem0[k + 1] = B.elem0[k] + rows * (b.x1 - b.x0);
    }
    return B;
}

// Layout of one checkpoint slot (all max_shots shots): the two pressure
// states, their per-tile FP16 scales, then per CPML field its strip boxes
// and per-row scales. Byte offsets within the slot.
struct CkLayout {
    int ckx = 0, ckz = 0;          // store tiles of the pressure states
    size_t state = 0;              // elements of one pressure state (all shots)
    size_t off_scale = 0;          // byte offset of the state scales
    int nf = 0;                    // CPML fields
    int ax[6] = {0, 0, 0, 0, 0, 0};
    CkBoxes box[3];                // per axis (index into ax order)
    size_t off_f[6] = {0, 0, 0, 0, 0, 0}, off_fs[6] = {0, 0, 0, 0, 0, 0};
    size_t bytes = 0;              // per slot
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

CkLayout ck_layout(const sim_s *s, int fp16) {
    const Geom &g = s->g;
    const int ms = s->d.max_shots;
    const size_t es = fp16 ? 2 : s->esz;
    CkLayout c;
    c.ckx = (g.NX + kTileX2 - 1) / kTileX2;
    c.ckz = (g.NZ * g.NY + kTileZ2 - 1) / kTileZ2;
    c.state = (size_t)ms * g.NZ * g.NY * g.NX;
    size_t off = align256(2 * c.state * es);
    c.off_scale = off;
    off += align256((size_t)2 * ms * c.ckx * c.ckz * sizeof(float));
    int axes[3];
    const int na = s->d.bc == SIM_BC_CPML ? cpml_ckpt_axes(s, axes) : 0;
    for (int k = 0; k < na; k++) {
        c.box[k] = strip_boxes(g, axes[k]);
        for (int z = 0; z < 2; z++) {
            const int j = 2 * k + z;
            c.ax[j] = axes[k];
            c.off_f[j] = off;
            off += align256((size_t)ms * c.box[k].elem0[c.box[k].n] * es);
            c.off_fs[j] = off;
            off += align256((size_t)ms * c.box[k].row0[c.box[k].n] * sizeof(float));
        }
    }
    c.nf = 2 * na;
    c.bytes = off;
    return c;
}

// Bytes of one imaging-term slot (all max_shots shots) and its scales.
size_t q_slot_bytes(const sim_s *s, int fp16) {
    const int ms = s->d.max_shots;
    if (s->g.ndim == 3) return align256((size_t)ms * s->g.fstride * sizeof(float));  // 3D slots are FP32
    return align256((size_t)ms * s->g.fstride * (fp16 ? 2 : s->esz));
}
size_t q_scale_bytes(const sim_s *s) { return align256((size_t)s->d.max_shots * max_tiles(s) * sizeof(float)); }

// Buffers of the gradient other than checkpoints and imaging-term slots.
size_t adjoint_fixed_bytes(const sim_s *s) {
    const Geom &g = s->g;
    const sim_desc &d = s->d;
    const size_t fb = align256((size_t)d.max_shots * g.fstride * s->esz);
    const size_t nint = (size_t)g.nz * g.ny * g.nx;
    const size_t nrows = (size_t)d.max_shots * d.nt * std::max(1, d.max_rec);
    size_t b = 3 * fb;  // u (two parities), G
    if (d.bc == SIM_BC_CPML) {
        int axes[3];
        b += (size_t)cpml_ckpt_axes(s, axes) * 3 * fb;  // nu (two parities), mu
        if (g.ndim == 2) b += fb;                       // the bracket
    }
    b += 2 * align256(nrows * s->esz) + align256(nint * sizeof(double)) + align256(nint * s->esz);
    b += align256(kResidBlocks * sizeof(double)) + 3 * align256(s->cap_grp * sizeof(InjEntryT<double>) + s->cap_start * 4);
    if (g.ndim == 3) b += 4 * align256(8 * (size_t)std::max(d.max_shots, std::max(1, d.max_rec)) * sizeof(Inj3));
    return b;
}

sim_status plan_adjoint(sim_t s, int fp16, AdjPlan &P) {
    const int nt = s->d.nt;
    P = AdjPlan{};
    P.fp16 = fp16;
    P.ck_bytes = ck_layout(s, fp16).bytes;
    P.q_bytes = q_slot_bytes(s, fp16) + (s->g.ndim == 2 ? q_scale_bytes(s) : 0);
    P.fixed_bytes = adjoint_fixed_bytes(s);
    long long budget = s->d.adj_budget;
    size_t freeb = 0, totalb = 0;
    if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) {
        cudaGetLastError();
        return s->fail(SIM_ERR_CUDA, "cudaMemGetInfo failed");
    }
    if (budget <= 0) {
        const size_t margin = std::max<size_t>(2ull << 30, totalb / 25);
        budget = freeb > margin ? (long long)(freeb - margin) : 0;
    }
    auto mem = [&](int levels, int L, int m, int &n1, int &n2) {
        n1 = (nt + L * m - 1) / (L * m);
        n2 = levels == 2 ? std::max(0, m - 2) : 0;
        return (double)(n1 + n2) * P.ck_bytes + (double)L * P.q_bytes;
    };
    const double room = (double)budget - (double)P.fixed_bytes;
    auto take = [&](int levels, int L, int m) {
        P.levels = levels;
        P.L = L;
        P.m = m;
        P.total = (size_t)(mem(levels, L, m, P.n1, P.n2) + P.fixed_bytes);
        return SIM_OK;
    };
    int n1, n2;
    const int Ls = (int)std::ceil(std::sqrt((double)nt));
    if (mem(1, Ls, 1, n1, n2) <= room) return take(1, Ls, 1);
    double best = 1e300;
    int bl = 1;
    for (int L = 1; L <= nt; L++) {
        const double v = mem(1, L, 1, n1, n2);
        if (v < best) best = v, bl = L;
    }
    if (best <= room) return take(1, bl, 1);
    best = 1e300;
    int bm = 2;
    for (int L = 1; L <= nt; L++) {
        const int mmax = (nt + L - 1) / L;
        const int mhi = std::min(mmax, 2 * (int)std::ceil(std::sqrt((double)nt / L)) + 2);
        for (int m = 2; m <= mhi; m++) {
            const double v = mem(2, L, m, n1, n2);
            if (v < best) best = v, bl = L, bm = m;
        }
    }
    if (best <= room) return take(2, bl, bm);
    return s->fail(SIM_ERR_OOM,
                   "the gradient needs %.2f GB of device memory at least (%.2f GB of checkpoints and imaging terms "
                   "with two checkpoint levels) and %.2f GB are available",
                   (best + P.fixed_bytes) / 1e9, best / 1e9, (double)budget / 1e9);
}

// Free the adjoint buffers (and every captured graph, which may use them).
void free_adjoint(sim_t s) {
    cudaStreamSynchronize(s->st);
    if (s->cst) cudaStreamSynchronize(s->cst);
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
    s->graphs.clear();
    for (void *p : s->adj_allocs) cudaFree(p);
    s->adj_allocs.clear();
    s->bytes -= s->adj_bytes;
    s->adj_bytes = 0;
    s->adj_ready = false;
    s->ubuf = s->Gbuf = s->qbuf = s->ckpt = s->res = s->dobs = s->cext = s->gradst = nullptr;
    for (int ax = 0; ax < 3; ax++) s->cnu[ax][0] = s->cnu[ax][1] = s->cmu[ax] = nullptr;
    s->qscale = nullptr;
    s->acc = s->mpart = nullptr;
    s->inj2_start = nullptr;
    s->inj2_grp = nullptr;
    s->inj2_ent = nullptr;
    s->src3g = s->res3g = nullptr;
    s->src3e = s->res3e = nullptr;
}

// Zero the CPML multipliers (both parities) and the 2D bracket of `nshots`
// shots before an adjoint sweep.
cudaError_t reset_cpml_adjoint(const sim_s *s, int nshots, cudaStream_t st) {
    const size_t fb = (size_t)nshots * s->g.fstride * s->esz;
    cudaError_t e = cudaSuccess;
    for (int ax = 0; ax < 3 && e == cudaSuccess; ax++) {
        if (!s->cnu[ax][0]) continue;
        e = cudaMemsetAsync(s->cnu[ax][0], 0, fb, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->cnu[ax][1], 0, fb, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->cmu[ax], 0, fb, st);
    }
    if (e == cudaSuccess && s->cext) e = cudaMemsetAsync(s->cext, 0, fb, st);
    return e;
}

// Allocate the adjoint buffers for checkpoints at the requested storage
// precision (re-planned when earlier buffers were sized for FP16 and FP32
// storage is asked for).
sim_status ensure_adjoint(sim_t s, int fp16) {
    if (s->adj_ready && (!s->plan.fp16 || fp16)) return SIM_OK;
    if (s->adj_ready) free_adjoint(s);
    const sim_desc &d = s->d;
    const Geom &g = s->g;
    AdjPlan P;
    if (sim_status r = plan_adjoint(s, fp16, P)) return r;
    const int ms = d.max_shots;
    const size_t nint = (size_t)g.nz * g.ny * g.nx;
    const size_t nrows = (size_t)ms * d.nt * std::max(1, d.max_rec);
    const size_t fb = (size_t)ms * g.fstride * s->esz;
    sim_status rc = SIM_OK;
    const size_t before = s->bytes;
    auto A = [&](size_t n) {
        if (rc != SIM_OK) return (void *)nullptr;
        void *p = s->alloc(n, &rc);
        if (p) {
            s->allocs.pop_back();  // owned by the adjoint list, freed on re-plan
            s->adj_allocs.push_back(p);
        }
        return p;
    };
    s->ubuf = A(2 * fb);
    s->Gbuf = A(fb);
    if (d.bc == SIM_BC_CPML) {
        for (int ax = 0; ax < 3; ax++) {
            if (!s->psi[ax][0]) continue;
            s->cnu[ax][0] = A(fb);
            s->cnu[ax][1] = A(fb);
            s->cmu[ax] = A(fb);
        }
        if (g.ndim == 2) s->cext = A(fb);
    }
    s->ckpt = A((size_t)(P.n1 + P.n2) * P.ck_bytes);
    s->qbuf = A((size_t)P.L * q_slot_bytes(s, fp16));
    if (g.ndim == 2) s->qscale = static_cast<float *>(A((size_t)P.L * q_scale_bytes(s)));
    s->res = A(nrows * s->esz);
    s->dobs = A(nrows * s->esz);
    s->acc = static_cast<double *>(A(nint * sizeof(double)));
    s->gradst = A(nint * s->esz);
    s->mpart = static_cast<double *>(A(kResidBlocks * sizeof(double)));
    s->inj2_start = static_cast<int *>(A(s->cap_start * sizeof(int)));
    s->inj2_grp = static_cast<InjGroup *>(A(s->cap_grp * sizeof(InjGroup)));
    s->inj2_ent = A(s->cap_grp * sizeof(InjEntryT<double>));
    if (g.ndim == 3) {
        s->src3g = static_cast<Inj3 *>(A(8 * (size_t)ms * sizeof(Inj3)));
        s->src3e = static_cast<InjE3 *>(A(8 * (size_t)ms * sizeof(InjE3)));
        s->res3g = static_cast<Inj3 *>(A(8 * (size_t)std::max(1, d.max_rec) * sizeof(Inj3)));
        s->res3e = static_cast<InjE3 *>(A(8 * (size_t)std::max(1, d.max_rec) * sizeof(InjE3)));
    }
    s->adj_bytes = s->bytes - before;
    if (rc != SIM_OK) {
        free_adjoint(s);
        return rc;
    }
    s->plan = P;
    s->adj_ready = true;
    return SIM_OK;
}

// Checkpoint slot k: store (or restore) the state entering step n: p^n,
// p^{n-1} and the CPML memory of every absorbing axis (2D: psi of the
// parity step n reads; 3D: psi kept in place).
template <typename T>
cudaError_t checkpoint(sim_t s, const StepArgs<T> &a, const CkLayout &c, int k, int n, bool store, int fp16,
                       int nshots, cudaStream_t st) {
    const Geom &g = s->g;
    char *slot = static_cast<char *>(s->ckpt) + (size_t)k * s->plan.ck_bytes;
    const size_t es = fp16 ? 2 : sizeof(T);
    float *scale = reinterpret_cast<float *>(slot + c.off_scale);
    const size_t ck_tiles = (size_t)s->d.max_shots * c.ckx * c.ckz;
    const long long ncomp = (long long)g.NZ * g.NY * g.NX;
    cudaError_t e = cudaSuccess;
    for (int w = 0; w < 2 && e == cudaSuccess; w++) {  // w = 1: p^n, w = 0: p^{n-1}
        T *f = a.pbuf[(n + 1 + w) & 1];
        void *dst = slot + w * c.state * es;
        e = store ? launch_store_state<T>(g, f, dst, scale + w * ck_tiles, fp16, nshots, ncomp, c.ckx, c.ckz, st)
                  : launch_load_state<T>(g, f, dst, scale + w * ck_tiles, fp16, nshots, ncomp, c.ckx, c.ckz, st);
    }
    for (int j = 0; j < c.nf && e == cudaSuccess; j++) {
        const int ax = c.ax[j];
        T *f = static_cast<T *>(j % 2 ? s->zeta[ax] : s->psi[ax][g.ndim == 2 ? (n + 1) & 1 : 0]);
        const CkBoxes &B = c.box[j / 2];
        e = store ? launch_store_boxes<T>(g, B, f, slot + c.off_f[j], reinterpret_cast<float *>(slot + c.off_fs[j]),
                                          fp16, nshots, st)
                  : launch_load_boxes<T>(g, B, f, slot + c.off_f[j], reinterpret_cast<const float *>(slot + c.off_fs[j]),
                                         fp16, nshots, st);
    }
    return e;
}

// The reverse schedule of a plan as a sequence of launches:
//   fwd_first(n): forward step n of the first sweep (samples the gather);
//   fwd(n): forward step n of a recompute that keeps checkpoints only;
//   rec(n, slot): forward step n recording its imaging term into slot;
//   adj(k, slot): adjoint step k (the slot recorded by forward step k - 1);
//   ck(slot, n, store): store / restore the state entering step n;
//   mid(): between the forward sweep and the reverse (residual, zeroing).
template <typename F1, typename F2, typename F3, typename F4, typename F5, typename F6>
cudaError_t emit_gradient(const AdjPlan &P, int nt, F1 fwd_first, F2 fwd, F3 rec, F4 adj, F5 ck, F6 mid) {
    const int S1 = P.L * P.m;
    cudaError_t e = cudaSuccess;
    for (int n = 0; n < nt && e == cudaSuccess; n++) {
        if (n % S1 == 0) e = ck(n / S1, n, true);
        if (e == cudaSuccess) e = fwd_first(n);
    }
    if (e == cudaSuccess) e = mid();
    for (int t = (nt + S1 - 1) / S1 - 1; t >= 0 && e == cudaSuccess; t--) {
        const int t0 = t * S1, t1 = std::min(nt, t0 + S1);
        const int msub = (t1 - t0 + P.L - 1) / P.L;
        e = ck(t, t0, false);
        // recompute up to the last inner segment, keeping the inner starts
        // 1 .. msub - 2 (the first restarts from slot t, the last from here)
        for (int n = t0; n < t0 + (msub - 1) * P.L && e == cudaSuccess; n++) {
            if (n > t0 && (n - t0) % P.L == 0 && (n - t0) / P.L <= msub - 2) e = ck(P.n1 + (n - t0) / P.L - 1, n, true);
            if (e == cudaSuccess) e = fwd(n);
        }
        for (int j = msub - 1; j >= 0 && e == cudaSuccess; j--) {
            const int s0 = t0 + j * P.L, s1 = std::min(t1, s0 + P.L);
            if (j < msub - 1) e = ck(j == 0 ? t : P.n1 + j - 1, s0, false);
            for (int n = s0; n < s1 && e == cudaSuccess; n++) e = rec(n, n - s0);
            for (int k = s1; k >= s0 + 1 && e == cudaSuccess; k--) e = adj(k, k - 1 - s0);
        }
    }
    return e;
}

// Injection groups of 3D points (adjoint path): every corner with a non-zero
// weight off the free surface, grouped by target cell in a fixed order;
// shot >= 0 gives each point's groups to that shot, -1 shares them.
void group3d(const std::vector<Pt3> &pts, bool per_shot, std::vector<Inj3> &grp, std::vector<InjE3> &ent) {
    struct C {
        long long cell;
        int shot, pt;
        float w;
    };
    std::vector<C> cs;
    for (size_t q = 0; q < pts.size(); q++)
        for (int k = 0; k < 8; k++)
            if (pts[q].cell[k] >= 0) cs.push_back({pts[q].cell[k], per_shot ? (int)q : -1, (int)q, pts[q].w[k]});
    std::stable_sort(cs.begin(), cs.end(), [](const C &a, const C &b) {
        return a.shot != b.shot ? a.shot < b.shot : a.cell < b.cell;
    });
    grp.clear();
    ent.clear();
    for (size_t i = 0; i < cs.size();) {
        Inj3 G{};
        G.cell = cs[i].cell;
        G.shot = cs[i].shot;
        G.e0 = (int)ent.size();
        size_t j = i;
        while (j < cs.size() && cs[j].cell == cs[i].cell && cs[j].shot == cs[i].shot) {
            ent.push_back(InjE3{cs[j].pt, cs[j].w});
            j++;
        }
        G.e1 = (int)ent.size();
        grp.push_back(G);
        i = j;
    }
}

// Options of one gradient call beyond sim_adjoint's arguments.
struct AdjOpts {
    bool vjp = false;          // d_obs holds the adjoint source itself (the residual): gradient = J^T r
    double *grad_fp64 = nullptr;  // device FP64 accumulator to add the gradient to (instead of grad_v)
};

// After the graph: add the FP64 gradient to the caller's array, check the
// final field, copy outputs and (when an output is host memory or the misfit
// is asked for) wait and report.
template <typename T>
sim_status finish_gradient(sim_t s, const StepArgs<T> &a, int nshots, size_t nrows, void *grad_v, void *grdev,
                           bool gr_host, void *gather_out, bool g_host, double *misfit_out, const AdjOpts &o) {
    const Geom &g = s->g;
    const long long nint = (long long)g.nz * g.ny * g.nx;
    if (o.grad_fp64) {
        if (sim_status r = s->cuda(launch_add_gradient<double>(s->acc, o.grad_fp64, nint, s->st), "gradient add"))
            return r;
    } else if (sim_status r = s->cuda(launch_add_gradient<T>(s->acc, static_cast<T *>(grdev), nint, s->st),
                                      "gradient add"))
        return r;
    if (sim_status r = s->cuda(launch_check_finite<T>(g, a.pbuf[s->d.nt & 1], nshots, s->flags, s->st),
                               "finite check"))
        return r;
    if (sim_status r = s->cuda(cudaMemcpyAsync(s->flags_host, s->flags, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                               s->st), "flag readback"))
        return r;
    if (gr_host)
        if (sim_status r = s->cuda(cudaMemcpyAsync(grad_v, grdev, nint * sizeof(T), cudaMemcpyDeviceToHost, s->st),
                                   "gradient download"))
            return r;
    if (gather_out)
        if (sim_status r = s->cuda(cudaMemcpyAsync(gather_out, s->gath, nrows * sizeof(T), cudaMemcpyDefault, s->st),
                                   "gather copy"))
            return r;
    std::vector<double> part(kResidBlocks);
    const bool want_misfit = misfit_out && !o.vjp;
    if (want_misfit)
        if (sim_status r = s->cuda(cudaMemcpyAsync(part.data(), s->mpart, part.size() * sizeof(double),
                                                   cudaMemcpyDeviceToHost, s->st), "misfit readback"))
            return r;
    if (misfit_out || gr_host || g_host) {
        if (sim_status r = poll_flags(s, true)) return r;
        if (misfit_out) {
            double J = 0;
            if (want_misfit)
                for (double v : part) J += v;
            *misfit_out = J;
        }
    }
    return SIM_OK;
}

// Residual (g - d_obs, with the misfit) or the given adjoint source, then
// zero the adjoint state: the step between the forward sweep and the reverse.
template <typename T>
cudaError_t gradient_mid(sim_t s, int nshots, size_t nrows, bool vjp, cudaStream_t st) {
    cudaError_t e = vjp ? cudaMemcpyAsync(s->res, s->dobs, nrows * sizeof(T), cudaMemcpyDeviceToDevice, st)
                        : launch_residual<T>(static_cast<const T *>(s->gath), static_cast<const T *>(s->dobs),
                                             static_cast<T *>(s->res), (long long)nrows, s->mpart, kResidBlocks, st);
    const size_t ub = (size_t)s->g.fstride * s->esz * nshots;
    if (e == cudaSuccess) e = cudaMemsetAsync(s->ubuf, 0, ub, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(static_cast<char *>(s->ubuf) + (size_t)s->g.fstride * s->esz * s->d.max_shots, 0, ub, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->Gbuf, 0, ub, st);
    if (e == cudaSuccess && s->d.bc == SIM_BC_CPML) e = reset_cpml_adjoint(s, nshots, st);
    return e;
}

// The adjoint-state gradient on the 3D path: the z-march in its record /
// adjoint modes, point injection grouped by cell, the CPML passes of each
// absorbing axis around the update (in the recompute they also take the
// addend off the imaging term) and the transposed CPML recursions after
// each adjoint update. Imaging-term slots are FP32 (checkpoints may be FP16).
sim_status adjoint3d(sim_t s, int nshots, const void *wavelet, const double *src_pos, int nrec,
                     const double *rec_pos, const void *d_obs, void *gather_out, double *misfit_out, int ckpt_fp16,
                     void *grad_v, const AdjOpts &o) {
    const sim_desc &d = s->d;
    const Geom &g = s->g;
    if (sim_status r = ensure_adjoint(s, ckpt_fp16)) return r;
    const size_t nt = d.nt;
    const int ms = d.max_shots;
    const long long nint = (long long)g.nz * g.ny * g.nx;
    const size_t nrows = (size_t)nshots * nt * nrec;
    const void *wav = wavelet;
    if (!is_device_ptr(wavelet)) {
        if (sim_status r = s->cuda(cudaMemcpyAsync(s->wave, wavelet, nt * sizeof(float), cudaMemcpyHostToDevice,
                                                   s->st), "wavelet upload"))
            return r;
        wav = s->wave;
    }
    if (sim_status r = s->cuda(cudaMemcpyAsync(s->dobs, d_obs, nrows * sizeof(float), cudaMemcpyDefault, s->st),
                               "d_obs copy"))
        return r;
    const bool g_host = gather_out && !is_device_ptr(gather_out);
    const bool gr_host = !o.grad_fp64 && !is_device_ptr(grad_v);
    void *grdev = gr_host ? s->gradst : grad_v;
    if (gr_host)
        if (sim_status r = s->cuda(cudaMemcpyAsync(grdev, grad_v, nint * sizeof(float), cudaMemcpyHostToDevice, s->st),
                                   "gradient upload"))
            return r;
    // points: receivers for sampling (all corners), sources and residuals for injection
    std::vector<Pt3> src, rsam, rinj;
    if (sim_status r = points3d(s, nshots, src_pos, src, true, "source")) return r;
    if (sim_status r = points3d(s, nrec, rec_pos, rsam, false, "receiver")) return r;
    if (sim_status r = points3d(s, nrec, rec_pos, rinj, true, "receiver")) return r;
    std::vector<Inj3> sg, rg;
    std::vector<InjE3> se, re;
    group3d(src, true, sg, se);
    group3d(rinj, false, rg, re);
    if (sim_status r = s->cuda(cudaMemcpyAsync(s->rec3, rsam.data(), rsam.size() * sizeof(Pt3),
                                               cudaMemcpyHostToDevice, s->st), "receiver upload"))
        return r;
    if (sim_status r = upload(s, s->src3g, sg, 8 * (size_t)ms, "source group")) return r;
    if (sim_status r = upload(s, s->src3e, se, 8 * (size_t)ms, "source entry")) return r;
    if (sim_status r = upload(s, s->res3g, rg, 8 * (size_t)std::max(1, d.max_rec), "residual group")) return r;
    if (sim_status r = upload(s, s->res3e, re, 8 * (size_t)std::max(1, d.max_rec), "residual entry")) return r;
    SimIO io{};
    io.wavelet = wav;
    io.gather = s->gath;
    io.resid = s->res;
    io.nrec = nrec;
    io.nshots = nshots;
    if (sim_status r = s->cuda(cudaMemcpyAsync(s->io, &io, sizeof io, cudaMemcpyHostToDevice, s->st), "io upload"))
        return r;

    if (sim_status r = autotune3d(s, nshots)) return r;
    const AdjPlan &P = s->plan;
    const int zc = s->zchunk, zv = s->zvariant;
    const CkLayout ckl = ck_layout(s, ckpt_fp16);
    StepArgs<float> a = step_args<float>(s);
    a.sample = 1;
    a.nsnap = 0;
    StepArgs<float> quiet = a;  // recompute: no sampling
    quiet.sample = 0;
    const bool cpml = d.bc == SIM_BC_CPML;
    StepArgs<float> adj = a;
    adj.pbuf[0] = static_cast<float *>(s->ubuf);
    adj.pbuf[1] = static_cast<float *>(s->ubuf) + (long long)ms * g.fstride;
    adj.src_scale = (float)(d.h * d.h);
    float *Gs = static_cast<float *>(s->Gbuf);
    const size_t qstride = q_slot_bytes(s, ckpt_fp16);
    const int nsg = (int)sg.size(), nrg = (int)rg.size();
    const Pt3 *r3 = s->rec3;
    const long long gkey = ((long long)nshots << 40) ^ ((long long)nrec << 16) ^ ((long long)ckpt_fp16 << 3) ^
                           ((long long)o.vjp << 5) ^ 6;
    if (sim_status r = run_graph(s, gkey, [&](cudaStream_t st) {
            cudaError_t e = reset_state_on(s, nshots, st);
            if (e != cudaSuccess) return e;
            auto step = [&](const StepArgs<float> &A, int n, int mode, float *slot, bool sample) {
                cudaError_t e2 = cudaSuccess;
                if (sample) e2 = launch_sample3d(A, step_time(s, A, n, kModeForward, nullptr, nullptr), r3, nrec,
                                                 nshots, st);
                if (e2 == cudaSuccess) e2 = step3d_core(s, A, n, zv, zc, nshots, st, true, mode, slot);
                if (e2 == cudaSuccess)
                    e2 = launch_inj3d(A, n, n, s->src3g, nsg, s->src3e, 0, nshots, mode, slot, nullptr, st);
                return e2;
            };
            auto slot_of = [&](int i) { return reinterpret_cast<float *>(static_cast<char *>(s->qbuf) + (size_t)i * qstride); };
            e = emit_gradient(
                P, d.nt, [&](int n) { return step(a, n, kModeForward, nullptr, true); },
                [&](int n) { return step(quiet, n, kModeForward, nullptr, false); },
                [&](int n, int i) { return step(quiet, n, kModeRecord, slot_of(i), false); },
                [&](int k, int i) {
                    float *slot = slot_of(i);
                    const int n = d.nt - k;
                    cudaError_t e2 = launch_step3d(adj, n, zv, zc, nshots, st, true, kModeAdjoint, slot, Gs);
                    if (e2 == cudaSuccess)
                        e2 = launch_inj3d(adj, n, k, s->res3g, nrg, s->res3e, 1, nshots, kModeAdjoint, slot, Gs, st);
                    if (e2 == cudaSuccess && cpml && k <= d.nt - 1) {  // nu^k, mu^k from u^{k+1}; c [.] into u^k
                        CpmlAdjArgs<float> ca{};
                        ca.u = adj.pbuf[(d.nt - k) & 1];
                        for (int ax = 0; ax < 3; ax++) {
                            ca.nu[ax][0] = static_cast<float *>(s->cnu[ax][0]);
                            ca.nu[ax][1] = static_cast<float *>(s->cnu[ax][1]);
                            ca.mu[ax] = static_cast<float *>(s->cmu[ax]);
                        }
                        ca.uo = adj.pbuf[(n + 1) & 1];
                        ca.q = slot;
                        ca.G = Gs;
                        e2 = launch_cpml_adjoint<float>(a, ca, k & 1, nshots, st);
                    }
                    return e2;
                },
                [&](int k, int n, bool store) { return checkpoint<float>(s, a, ckl, k, n, store, ckpt_fp16, nshots, st); },
                [&]() { return gradient_mid<float>(s, nshots, nrows, o.vjp, st); });
            // FP64 sum over shots and replicated cells
            if (e == cudaSuccess) e = cudaMemsetAsync(s->acc, 0, nint * sizeof(double), st);
            if (e == cudaSuccess)
                e = launch_fold_gradient<float>(g, Gs, g.fstride, nshots, static_cast<const float *>(s->vpad),
                                                1.0 / (d.h * d.h), s->acc, st);
            return e;
        }))
        return r;
    return finish_gradient<float>(s, a, nshots, nrows, grad_v, grdev, gr_host, gather_out, g_host, misfit_out, o);
}

template <typename T>
sim_status adjoint_t(sim_t s, int nshots, const void *wavelet, const double *src_pos, int nrec,
                     const double *rec_pos, const void *d_obs, void *gather_out, double *misfit_out, int ckpt_fp16,
                     void *grad_v, const AdjOpts &o) {
    const sim_desc &d = s->d;
    const Geom &g = s->g;
    if (g.ndim == 3 && d.precision != SIM_FP32) return s->fail(SIM_ERR_UNSUPPORTED, "the 3D path runs in FP32");
    if (ckpt_fp16 && d.precision != SIM_FP32) return s->fail(SIM_ERR_ARG, "FP16 checkpoints need an FP32 handle");
    if (nrec < 1) return s->fail(SIM_ERR_ARG, "the misfit needs receivers");
    if (!d_obs || !wavelet || (!grad_v && !o.grad_fp64))
        return s->fail(SIM_ERR_ARG, "d_obs, wavelet and grad_v are required");
    if (g.ndim == 3)
        return adjoint3d(s, nshots, wavelet, src_pos, nrec, rec_pos, d_obs, gather_out, misfit_out, ckpt_fp16,
                         grad_v, o);
    if (sim_status r = ensure_adjoint(s, ckpt_fp16)) return r;
    if (sim_status r = autotune(s, nshots)) return r;
    const size_t nt = d.nt;
    const int ms = d.max_shots;
    const int ntiles = s->ntx * s->nty * s->ntz;
    const long long nint = (long long)g.nz * g.ny * g.nx;
    const size_t nrows = (size_t)nshots * nt * nrec;

    // inputs
    const void *wav = wavelet;
    if (!is_device_ptr(wavelet)) {
        if (sim_status r = s->cuda(cudaMemcpyAsync(s->wave, wavelet, nt * sizeof(T), cudaMemcpyHostToDevice, s->st),
                                   "wavelet upload"))
            return r;
        wav = s->wave;
    }
    // The time loops run as one captured graph on handle-owned buffers: d_obs
    // is copied into the handle, the gather is recorded in the handle's buffer
    // and copied out afterwards.
    if (sim_status r = s->cuda(cudaMemcpyAsync(s->dobs, d_obs, nrows * sizeof(T), cudaMemcpyDefault, s->st),
                               "d_obs copy"))
        return r;
    const bool g_host = gather_out && !is_device_ptr(gather_out);
    const bool gr_host = !o.grad_fp64 && !is_device_ptr(grad_v);
    void *grdev = gr_host ? s->gradst : grad_v;
    if (gr_host)
        if (sim_status r = s->cuda(cudaMemcpyAsync(grdev, grad_v, nint * sizeof(T), cudaMemcpyHostToDevice, s->st),
                                   "gradient upload"))
            return r;

    // geometry: receivers sample the forward; sources drive the forward and the
    // recompute; receivers inject the residual into the adjoint sweep
    std::vector<int> rstart, istart, jstart;
    std::vector<RecEntryT<T>> rent;
    std::vector<InjGroup> igrp, jgrp;
    std::vector<InjEntryT<T>> ient, jent;
    if (sim_status r = build_receivers<T>(s, nrec, rec_pos, rstart, rent)) return r;
    std::vector<InjPoint> pts, rpts;
    if (sim_status r = collect_points(s, nshots, src_pos, true, pts, "source")) return r;
    group_injection<T>(pts, nshots * ntiles, istart, igrp, ient);
    if (sim_status r = collect_points(s, nrec, rec_pos, false, rpts, "receiver")) return r;
    group_injection<T>(rpts, ntiles, jstart, jgrp, jent);
    if (sim_status r = upload(s, s->rec_start, rstart, s->cap_start, "receiver start")) return r;
    if (sim_status r = upload(s, static_cast<RecEntryT<T> *>(s->rec), rent, s->cap_rec, "receiver")) return r;
    if (sim_status r = upload(s, s->inj_start, istart, s->cap_start, "injection start")) return r;
    if (sim_status r = upload(s, s->inj_grp, igrp, s->cap_grp, "injection group")) return r;
    if (sim_status r = upload(s, static_cast<InjEntryT<T> *>(s->inj_ent), ient, s->cap_grp, "injection entry"))
        return r;
    if (sim_status r = upload(s, s->inj2_start, jstart, s->cap_start, "residual start")) return r;
    if (sim_status r = upload(s, s->inj2_grp, jgrp, s->cap_grp, "residual group")) return r;
    if (sim_status r = upload(s, static_cast<InjEntryT<T> *>(s->inj2_ent), jent, s->cap_grp, "residual entry"))
        return r;

    SimIO io{};
    io.wavelet = wav;
    io.gather = s->gath;
    io.resid = s->res;
    io.nrec = nrec;
    io.nshots = nshots;
    if (sim_status r = s->cuda(cudaMemcpyAsync(s->io, &io, sizeof io, cudaMemcpyHostToDevice, s->st), "io upload"))
        return r;

    const AdjPlan &P = s->plan;
    const CkLayout ckl = ck_layout(s, ckpt_fp16);
    // 1. forward pass, keeping (p^{n-1}, p^n) at every segment start
    StepArgs<T> a = step_args<T>(s);
    a.inj_per_shot = 1;
    a.inj_kind = 0;
    a.nsnap = 0;
    StepArgs<T> quiet = a;  // recompute: no sampling
    quiet.sample = 0;
    StepArgs<T> rcp = quiet;
    rcp.q_fp16 = ckpt_fp16;
    StepArgs<T> adj = a;
    adj.pbuf[0] = static_cast<T *>(s->ubuf);
    adj.pbuf[1] = static_cast<T *>(s->ubuf) + (long long)ms * g.fstride;
    adj.sample = 0;
    adj.inj_start = s->inj2_start;
    adj.inj_grp = s->inj2_grp;
    adj.inj_ent = static_cast<const InjEntryT<T> *>(s->inj2_ent);
    adj.inj_per_shot = 0;
    adj.inj_kind = 1;
    adj.inj_reverse = 1;
    adj.src_scale = T(d.h * d.h);
    adj.q_fp16 = ckpt_fp16;
    adj.G = static_cast<T *>(s->Gbuf);
    // CPML: the sweep runs the plain update of u plus the transposed CPML
    // terms (cpml_adj.cu) it receives through cext
    const bool cpml = d.bc == SIM_BC_CPML;
    if (cpml) {
        adj.bc = SIM_BC_NONE;
        adj.cext = static_cast<const T *>(s->cext);
    }
    const size_t qstride = q_slot_bytes(s, ckpt_fp16), q_tiles = (size_t)ms * ntiles;
    // graph key: everything the captured launches depend on beyond handle buffers
    const long long gkey = ((long long)nshots << 40) ^ ((long long)nrec << 12) ^ ((long long)s->tile_z << 4) ^
                           ((long long)ckpt_fp16 << 3) ^ ((long long)o.vjp << 9) ^ 5;
    if (sim_status r = run_graph(s, gkey, [&](cudaStream_t st) {
            cudaError_t e = reset_state_on(s, nshots, st);
            if (e != cudaSuccess) return e;
            auto slot_of = [&](int i) { return static_cast<void *>(static_cast<char *>(s->qbuf) + (size_t)i * qstride); };
            auto scale_of = [&](int i) { return s->qscale + (size_t)i * (q_scale_bytes(s) / sizeof(float)); };
            (void)q_tiles;
            e = emit_gradient(
                P, d.nt, [&](int n) { return launch_step<T>(s, a, n, nshots, kModeForward, st); },
                [&](int n) { return launch_step<T>(s, quiet, n, nshots, kModeForward, st); },
                [&](int n, int i) { return launch_step<T>(s, rcp, n, nshots, kModeRecord, st, slot_of(i), scale_of(i)); },
                [&](int k, int i) {
                    cudaError_t e2 = cudaSuccess;
                    if (cpml && k <= d.nt - 1) {  // nu^k, mu^k from u^{k+1}, then their term in u^k
                        CpmlAdjArgs<T> ca{};
                        ca.u = adj.pbuf[(d.nt - k) & 1];
                        for (int ax = 0; ax < 3; ax++) {
                            ca.nu[ax][0] = static_cast<T *>(s->cnu[ax][0]);
                            ca.nu[ax][1] = static_cast<T *>(s->cnu[ax][1]);
                            ca.mu[ax] = static_cast<T *>(s->cmu[ax]);
                        }
                        ca.ext = static_cast<T *>(s->cext);
                        e2 = launch_cpml_adjoint<T>(a, ca, k & 1, nshots, st);
                    }
                    if (e2 == cudaSuccess)
                        e2 = launch_step<T>(s, adj, d.nt - k, nshots, kModeAdjoint, st, slot_of(i), scale_of(i));
                    return e2;
                },
                [&](int k, int n, bool store) { return checkpoint<T>(s, a, ckl, k, n, store, ckpt_fp16, nshots, st); },
                [&]() { return gradient_mid<T>(s, nshots, nrows, o.vjp, st); });
            // FP64 sum over shots and replicated cells
            if (e == cudaSuccess) e = cudaMemsetAsync(s->acc, 0, nint * sizeof(double), st);
            if (e == cudaSuccess)
                e = launch_fold_gradient<T>(g, static_cast<const T *>(s->Gbuf), g.fstride, nshots,
                                            static_cast<const T *>(s->vpad), 1.0 / (d.h * d.h), s->acc, st);
            return e;
        }))
        return r;
    return finish_gradient<T>(s, a, nshots, nrows, grad_v, grdev, gr_host, gather_out, g_host, misfit_out, o);
}


// ---------------------------------------------------------------- batch
//
// One persistent launch for many (slice, shot) members (k_batch2d). Members
// are grouped so that a group's fields fit in a share of L2; the device work
// list runs group after group, each through all its steps. The per-device
// context below owns the work-list tables and the captured graph of
// (counter resets + kernel); handles keep owning their fields and lists.
struct BatchCtx {
    int dev = -1;
    void *slices = nullptr, *groups = nullptr, *members = nullptr, *done = nullptr;
    unsigned long long *head = nullptr;
    unsigned *flags = nullptr, *flags_host = nullptr;
    size_t cap_slices = 0, cap_groups = 0, cap_members = 0, cap_done = 0;
    void *msegs = nullptr;  // row march items
    size_t cap_msegs = 0;
    unsigned *mctr = nullptr;                  // row march: per-step item counters (two pairs)
    cudaStream_t st2 = nullptr;                // row march with CPML: the plain items' kernel
    cudaEvent_t evf = nullptr, evj = nullptr;  //   forks to it and joins back each step
    void *tbm = nullptr, *tbs = nullptr;       // two-step march: members, receiver samples
    size_t cap_tbm = 0, cap_tbs = 0;
    cudaGraphExec_t exec = nullptr;
    std::vector<char> key;
    cudaEvent_t ev = nullptr;
};
std::mutex g_batch_mu;
std::vector<BatchCtx> g_batch;

cudaError_t grow(void **p, size_t *cap, size_t need) {
    if (*cap >= need) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(p, need);
    if (e == cudaSuccess) *cap = need;
    return e;
}

// Batch schedules: the row march (one launch per step over every member; two
// concurrent launches when members have CPML: the CPML items and the plain
// ones), the two-step row march (one launch per two steps, no CPML), the
// stepped tile kernel (one launch per step) and the persistent dataflow
// kernel (one launch for all steps).
enum { kBatchMarch = 0, kBatchStepped = 1, kBatchPersistent = 2, kBatchMarch2 = 3 };

// One batch run with a given schedule and list tile height. probe > 0: run
// only that many steps, launched directly (the autotuner's timing probe; no
// graph, no output copies), with pe0 / pe1 recorded around the launches.
sim_status batch_run(int nitems, const sim_batch_item *items, cudaStream_t bst, int sched, int tz_in, int probe,
                     cudaEvent_t pe0 = nullptr, cudaEvent_t pe1 = nullptr) {
    if (nitems < 1 || !items) return thread_fail(SIM_ERR_ARG, "empty batch");
    sim_t s0 = items[0].sim;
    if (!s0) return thread_fail(SIM_ERR_ARG, "batch item 0 has no handle");
    for (int i = 0; i < nitems; i++) {
        sim_t s = items[i].sim;
        if (!s || !s->model_set) return thread_fail(SIM_ERR_STATE, "batch item %d: no handle or no model", i);
        if (s->sticky) return s->sticky;
        if (s->d.ndim != 2 || s->d.precision != SIM_FP32)
            return thread_fail(SIM_ERR_UNSUPPORTED, "batch item %d: the batch runs 2D FP32 handles", i);
        if (s->d.nt != s0->d.nt) return thread_fail(SIM_ERR_ARG, "batch item %d: nt differs", i);
        if (s->dev != s0->dev) return thread_fail(SIM_ERR_ARG, "batch item %d: another device", i);
        if (items[i].nshots < 1 || items[i].nshots > s->d.max_shots)
            return thread_fail(SIM_ERR_ARG, "batch item %d: nshots outside [1, max_shots]", i);
        if (items[i].nrec < 0 || items[i].nrec > s->d.max_rec || (items[i].nrec > 0 && !items[i].rec_pos))
            return thread_fail(SIM_ERR_ARG, "batch item %d: bad receivers", i);
        if (!items[i].wavelet || !items[i].src_pos) return thread_fail(SIM_ERR_ARG, "batch item %d: no source", i);
        for (int j = 0; j < i; j++)
            if (items[j].sim == s) return thread_fail(SIM_ERR_ARG, "batch items %d and %d share a handle", j, i);
    }
    cudaSetDevice(s0->dev);
    const int nt = s0->d.nt;
    const int nsteps = probe > 0 ? std::min(probe, nt) : nt;
    const bool persistent = sched == kBatchPersistent;
    const bool march2 = sched == kBatchMarch2;
    const bool march = sched == kBatchMarch;
    const bool stepped = !persistent && !march2;
    const int tz = tz_in;
    bool any_cpml = false;
    std::vector<StepArgs<float>> slices(nitems);
    std::vector<void *> gdev(nitems, nullptr);
    // per handle: lists, io and a clean state, on the handle's own stream
    for (int i = 0; i < nitems; i++) {
        sim_t s = items[i].sim;
        const sim_batch_item &it = items[i];
        set_tile_z(s, tz);
        any_cpml |= s->d.bc == SIM_BC_CPML;
        if (march2) {  // the two-step march: no CPML; two more pressure fields per handle
            if (s->d.bc == SIM_BC_CPML)
                return thread_fail(SIM_ERR_UNSUPPORTED, "batch item %d: the two-step march takes no CPML", i);
            if (!s->pbuf3) {
                const size_t fb = 2 * (size_t)s->d.max_shots * s->g.fstride * sizeof(float);
                sim_status rc = SIM_OK;
                void *p3 = s->alloc(fb, &rc);
                if (rc != SIM_OK) return rc;
                if (sim_status r = s->cuda(cudaMemsetAsync(p3, 0, fb, s->st), "clear")) return r;
                s->pbuf3 = p3;
            }
        }
        const void *wav = it.wavelet;
        if (!is_device_ptr(wav)) {
            if (sim_status r = s->cuda(cudaMemcpyAsync(s->wave, wav, (size_t)nt * sizeof(float),
                                                       cudaMemcpyHostToDevice, s->st), "wavelet upload"))
                return r;
            wav = s->wave;
        }
        gdev[i] = it.gather && is_device_ptr(it.gather) ? it.gather : (it.gather ? s->gath : nullptr);
        std::vector<int> rstart, istart;
        std::vector<RecEntryT<float>> rent;
        std::vector<InjGroup> igrp;
        std::vector<InjEntryT<float>> ient;
        std::vector<InjPoint> pts;
        if (sim_status r = build_receivers<float>(s, it.nrec, it.rec_pos, rstart, rent)) return r;
        if (sim_status r = collect_points(s, it.nshots, it.src_pos, true, pts, "source")) return r;
        const int ntiles = s->ntx * s->ntz;
        group_injection<float>(pts, it.nshots * ntiles, istart, igrp, ient);
        if (sim_status r = upload(s, s->rec_start, rstart, s->cap_start, "receiver start")) return r;
        if (sim_status r = upload(s, static_cast<RecEntryT<float> *>(s->rec), rent, s->cap_rec, "receiver")) return r;
        if (sim_status r = upload(s, s->inj_start, istart, s->cap_start, "injection start")) return r;
        if (sim_status r = upload(s, s->inj_grp, igrp, s->cap_grp, "injection group")) return r;
        if (sim_status r = upload(s, static_cast<InjEntryT<float> *>(s->inj_ent), ient, s->cap_grp,
                                  "injection entry"))
            return r;
        SimIO io{};
        io.wavelet = wav;
        io.gather = it.nrec > 0 ? gdev[i] : nullptr;
        io.nrec = it.nrec;
        io.nshots = it.nshots;
        if (sim_status r = s->cuda(cudaMemcpyAsync(s->io, &io, sizeof io, cudaMemcpyHostToDevice, s->st), "io"))
            return r;
        if (sim_status r = reset_state(s, it.nshots)) return r;
        StepArgs<float> a = step_args<float>(s);
        a.inj_per_shot = 1;
        a.inj_kind = 0;
        a.nsnap = 0;
        a.sample = it.nrec > 0 && gdev[i] != nullptr;
        slices[i] = a;
    }
    // members and L2-sized groups
    int l2 = 0, sms = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, s0->dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s0->dev);
    double budget = 0.6 * l2;
    if (const char *f = getenv("GSIM_BATCH_GROUP_MB")) budget = atof(f) * 1048576.0;
    std::vector<BatchMember> members;
    std::vector<BatchGroup> groups;
    long long total = 0, done_total = 0;
    BatchGroup cur{0, 0, 0, 0};
    double bytes = 0;
    int last_slice = -1;
    for (int i = 0; i < nitems; i++) {
        sim_t s = items[i].sim;
        const Geom &g = s->g;
        const int ntiles = s->ntx * s->ntz;
        const double cells = (double)g.NZ * g.NX;
        const double strip = s->d.bc == SIM_BC_CPML ? (double)(g.nbx0 + g.nbx1) * g.NZ + (double)(g.nbz0 + g.nbz1) * g.NX : 0;
        for (int k = 0; k < items[i].nshots; k++) {
            double mb = 8.0 * cells + 12.0 * strip + (last_slice != i ? 4.0 * cells : 0.0);
            if (cur.T > 0 && bytes + mb > budget) {
                cur.m1 = (int)members.size();
                groups.push_back(cur);
                total += (long long)nt * cur.T;
                cur = BatchGroup{total, 0, (int)members.size(), 0};
                bytes = 0;
                mb = 12.0 * cells + 12.0 * strip;
            }
            BatchMember m{i, k, cur.T, (int)(done_total + (long long)k * ntiles)};
            members.push_back(m);
            cur.T += ntiles;
            bytes += mb;
            last_slice = i;
        }
        done_total += (long long)items[i].nshots * ntiles;
    }
    cur.m1 = (int)members.size();
    groups.push_back(cur);
    total += (long long)nt * cur.T;

    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchCtx *ctx = nullptr;
    for (auto &c : g_batch)
        if (c.dev == s0->dev) ctx = &c;
    if (!ctx) {
        g_batch.emplace_back();
        ctx = &g_batch.back();
        ctx->dev = s0->dev;
    }
    auto fail = [&](cudaError_t e, const char *what) {
        cudaGetLastError();
        return thread_fail(e == cudaErrorMemoryAllocation ? SIM_ERR_OOM : SIM_ERR_CUDA, "batch %s: %s", what,
                           cudaGetErrorString(e));
    };
    cudaError_t e = cudaSuccess;
    if (!ctx->head) {
        e = cudaMalloc(&ctx->head, sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->flags, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMallocHost(&ctx->flags_host, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(e, "allocation");
    }
    if ((e = grow(&ctx->slices, &ctx->cap_slices, slices.size() * sizeof(StepArgs<float>))) ||
        (e = grow(&ctx->groups, &ctx->cap_groups, groups.size() * sizeof(BatchGroup))) ||
        (e = grow(&ctx->members, &ctx->cap_members, members.size() * sizeof(BatchMember))) ||
        (e = grow(&ctx->done, &ctx->cap_done, (size_t)done_total * sizeof(int)))) {
        if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
        ctx->exec = nullptr;
        return fail(e, "allocation");
    }
    // order the handles' preparation before the batch stream
    for (int i = 0; i < nitems; i++) {
        if ((e = cudaEventRecord(ctx->ev, items[i].sim->st)) || (e = cudaStreamWaitEvent(bst, ctx->ev, 0)))
            return fail(e, "ordering");
    }
    if ((e = cudaMemcpyAsync(ctx->slices, slices.data(), slices.size() * sizeof(StepArgs<float>),
                             cudaMemcpyHostToDevice, bst)) ||
        (e = cudaMemcpyAsync(ctx->groups, groups.data(), groups.size() * sizeof(BatchGroup), cudaMemcpyHostToDevice,
                             bst)) ||
        (e = cudaMemcpyAsync(ctx->members, members.data(), members.size() * sizeof(BatchMember),
                             cudaMemcpyHostToDevice, bst)))
        return fail(e, "upload");
    MarchArgs mb{}, mpl{};
    bool split = false;
    if (march) {  // the row-march plan over all members
        std::vector<MarchMember> mm;
        for (const BatchMember &m : members) mm.push_back({m.slice, m.shot, items[m.slice].sim});
        std::vector<MarchSeg> segs;
        const long long maxw = (long long)sms * std::max(1, march2d_warps_per_sm(any_cpml));
        int ncp = 0;
        const int nw = plan_march_items(mm, maxw, march_item_rows(), segs, &ncp);
        if (!ctx->mctr && (e = cudaMalloc(&ctx->mctr, 4 * sizeof(unsigned)))) return fail(e, "allocation");
        if ((e = grow(&ctx->msegs, &ctx->cap_msegs, segs.size() * sizeof(MarchSeg)))) {
            if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
            ctx->exec = nullptr;
            return fail(e, "allocation");
        }
        if ((e = cudaMemcpyAsync(ctx->msegs, segs.data(), segs.size() * sizeof(MarchSeg), cudaMemcpyHostToDevice,
                                 bst)))
            return fail(e, "upload");
        mb.slices = static_cast<const StepArgs<float> *>(ctx->slices);
        mb.segs = static_cast<const MarchSeg *>(ctx->msegs);
        mb.ctr = ctx->mctr;
        mb.nwarps = nw;
        mb.nitems = (int)segs.size();
        mb.tz = tz;
        // With CPML, the items that take the CPML loop run in the CPML instance
        // of the kernel (2 CTAs per SM) and the plain ones in the plain
        // instance (3 CTAs per SM) on a second stream: launched together each
        // step, the plain kernel's CTAs take each SM as the CPML ones leave it.
        const char *sp = getenv("GSIM_MARCH_SPLIT");
        split = any_cpml && ncp > 0 && ncp < (int)segs.size() && !(sp && sp[0] == '0');
        if (split) {
            if (!ctx->st2 && (e = cudaStreamCreateWithFlags(&ctx->st2, cudaStreamNonBlocking))) return fail(e, "stream");
            if (!ctx->evf && (e = cudaEventCreateWithFlags(&ctx->evf, cudaEventDisableTiming))) return fail(e, "event");
            if (!ctx->evj && (e = cudaEventCreateWithFlags(&ctx->evj, cudaEventDisableTiming))) return fail(e, "event");
            mpl = mb;
            mpl.segs = static_cast<const MarchSeg *>(ctx->msegs) + ncp;
            mpl.nitems = (int)segs.size() - ncp;
            mpl.ctr = ctx->mctr + 2;
            mpl.nwarps = (int)std::min<long long>((long long)sms * std::max(1, march2d_warps_per_sm(false)), mpl.nitems);
            mb.nitems = ncp;
            mb.nwarps = (int)std::min<long long>(maxw, ncp);
        }
    }
    int tb_nwarps = 0;
    TBArgs tb{};
    if (march2) {  // members, receiver samples and items of the two-step march
        std::vector<TBMember> tm;
        std::vector<TBSample> ts;
        std::vector<MarchSeg> segs;
        int rows = 40;  // item height: 40 and 48 measured fastest on the 619 x 1000 production slice
        if (const char *f = getenv("GSIM_TB_ROWS")) rows = std::max(1, atoi(f));
        for (size_t mi = 0; mi < members.size(); mi++) {
            const BatchMember &m = members[mi];
            const sim_batch_item &it = items[m.slice];
            sim_s *s = it.sim;
            const Geom &g = s->g;
            TBMember M{};
            M.slice = m.slice;
            M.shot = m.shot;
            M.p3 = static_cast<float *>(s->pbuf3);
            M.pstride = (long long)s->d.max_shots * g.fstride;
            int i0[3];
            double t[3];
            if (!locate(g, s->d.h, it.src_pos + (size_t)m.shot * 2, i0, t))
                return thread_fail(SIM_ERR_ARG, "batch item %d: source %d lies outside the interior", m.slice, m.shot);
            for (int dz = 0; dz < 2; dz++)
                for (int dx = 0; dx < 2; dx++) {  // the corners the one-step injection lists hold
                    const double w = corner_weight(t, dz, 0, dx);
                    const int z = i0[0] + dz, x = i0[2] + dx;
                    if (w == 0.0 || (g.fs && z == 0)) continue;
                    M.sz[M.nsrc] = z;
                    M.sx[M.nsrc] = x;
                    M.sw[M.nsrc] = (float)w;
                    M.nsrc++;
                }
            tm.push_back(M);
            if (gdev[m.slice] && it.nrec > 0)
                for (int r = 0; r < it.nrec; r++) {
                    if (!locate(g, s->d.h, it.rec_pos + (size_t)r * 2, i0, t))
                        return thread_fail(SIM_ERR_ARG, "batch item %d: receiver %d lies outside the interior", m.slice,
                                           r);
                    TBSample Q{};
                    Q.member = (int)mi;
                    Q.rec = r;
                    Q.z = i0[0];
                    Q.x = i0[2];
                    int k = 0;
                    for (int dz = 0; dz < 2; dz++)
                        for (int dx = 0; dx < 2; dx++) Q.w[k++] = (float)corner_weight(t, dz, 0, dx);
                    ts.push_back(Q);
                }
            const int nstrip = (g.NX + kTBW - 1) / kTBW;
            for (int zc = 0; zc < g.NZ; zc += rows)
                for (int bx = 0; bx < nstrip; bx++)
                    segs.push_back(MarchSeg{(int)mi, m.shot, bx, zc, std::min(g.NZ, zc + rows), {0, 0, 0}});
        }
        if (!ctx->mctr && (e = cudaMalloc(&ctx->mctr, 4 * sizeof(unsigned)))) return fail(e, "allocation");
        if ((e = grow(&ctx->msegs, &ctx->cap_msegs, segs.size() * sizeof(MarchSeg))) ||
            (e = grow(&ctx->tbm, &ctx->cap_tbm, tm.size() * sizeof(TBMember))) ||
            (e = grow(&ctx->tbs, &ctx->cap_tbs, std::max<size_t>(1, ts.size()) * sizeof(TBSample)))) {
            if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
            ctx->exec = nullptr;
            return fail(e, "allocation");
        }
        if ((e = cudaMemcpyAsync(ctx->msegs, segs.data(), segs.size() * sizeof(MarchSeg), cudaMemcpyHostToDevice,
                                 bst)) ||
            (e = cudaMemcpyAsync(ctx->tbm, tm.data(), tm.size() * sizeof(TBMember), cudaMemcpyHostToDevice, bst)) ||
            (!ts.empty() &&
             (e = cudaMemcpyAsync(ctx->tbs, ts.data(), ts.size() * sizeof(TBSample), cudaMemcpyHostToDevice, bst))))
            return fail(e, "upload");
        tb.slices = static_cast<const StepArgs<float> *>(ctx->slices);
        tb.members = static_cast<const TBMember *>(ctx->tbm);
        tb.segs = static_cast<const MarchSeg *>(ctx->msegs);
        tb.samples = static_cast<const TBSample *>(ctx->tbs);
        tb.ctr = ctx->mctr;
        tb.nitems = (int)segs.size();
        tb.nsamples = (long long)ts.size();
        tb_nwarps = (int)std::min<long long>((long long)sms * std::max(1, march2x_warps_per_sm()), tb.nitems);
    }
    if (stepped) {  // members with global tile offsets
        long long t0 = 0;
        for (BatchMember &m : members) {
            m.tile0 = (int)t0;
            t0 += items[m.slice].sim->ntx * items[m.slice].sim->ntz;
        }
        if ((e = cudaMemcpyAsync(ctx->members, members.data(), members.size() * sizeof(BatchMember),
                                 cudaMemcpyHostToDevice, bst)))
            return fail(e, "upload");
    }
    BatchArgs b{};
    b.slices = static_cast<const StepArgs<float> *>(ctx->slices);
    b.groups = static_cast<const BatchGroup *>(ctx->groups);
    b.ngroups = (int)groups.size();
    b.nmembers = (int)members.size();
    b.members = static_cast<const BatchMember *>(ctx->members);
    b.done = static_cast<int *>(ctx->done);
    b.head = ctx->head;
    b.total = total;
    b.spin_limit = spin_limit();
    b.flags = ctx->flags;
    const int grid = sms * std::max(1, batch_blocks_per_sm(tz, any_cpml));
    // counters reset + the persistent kernel, replayed as one graph
    const int kk[4] = {tz, (int)any_cpml | (stepped ? 2 : 0) | (march ? 4 : 0) | (march2 ? 8 : 0) | (split ? 16 : 0), grid,
                       tb_nwarps};
    std::vector<char> key(sizeof b + 2 * sizeof mb + sizeof tb + sizeof kk + sizeof done_total);
    {
        char *k = key.data();
        memcpy(k, &b, sizeof b);
        memcpy(k += sizeof b, &mb, sizeof mb);
        memcpy(k += sizeof mb, &mpl, sizeof mpl);
        memcpy(k += sizeof mpl, &tb, sizeof tb);
        memcpy(k += sizeof tb, kk, sizeof kk);
        memcpy(k + sizeof kk, &done_total, sizeof done_total);
    }
    if (!ctx->exec || key != ctx->key || bst == nullptr) {
        if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
        ctx->exec = nullptr;
    }
    auto body = [&](cudaStream_t st) {
        if (march2) {  // passes of two steps (the last of one step when the count is odd)
            cudaError_t r = cudaMemsetAsync(ctx->flags, 0, sizeof(unsigned), st);
            if (r == cudaSuccess) r = cudaMemsetAsync(tb.ctr, 0, 2 * sizeof(unsigned), st);
            for (int k = 0; 2 * k < nsteps && r == cudaSuccess; k++) {
                TBPass t{};
                t.k = k;
                t.n = 2 * k;
                t.two = t.n + 1 < nsteps;
                t.inj0 = t.n;
                t.inj1 = t.two ? t.n + 1 : -1;
                r = launch_march2x(tb, t, tb_nwarps, st);
            }
            return r;
        }
        if (march) {
            cudaError_t r = cudaMemsetAsync(ctx->flags, 0, sizeof(unsigned), st);
            if (r == cudaSuccess && mb.ctr) r = cudaMemsetAsync(mb.ctr, 0, 4 * sizeof(unsigned), st);
            for (int n = 0; n < nsteps && r == cudaSuccess; n++) {
                StepTime t{};
                t.n = n;
                t.snap_k = t.max_k = -1;
                t.inj_row = n;
                if (!split) {
                    r = launch_march2d(mb, any_cpml, t, st, st != nullptr);
                    continue;
                }
                // fork: the plain items on the second stream; join before the next step
                if (r == cudaSuccess) r = cudaEventRecord(ctx->evf, st);
                if (r == cudaSuccess) r = cudaStreamWaitEvent(ctx->st2, ctx->evf, 0);
                if (r == cudaSuccess) r = launch_march2d(mb, true, t, st, false);
                if (r == cudaSuccess) r = launch_march2d(mpl, false, t, ctx->st2, false);
                if (r == cudaSuccess) r = cudaEventRecord(ctx->evj, ctx->st2);
                if (r == cudaSuccess) r = cudaStreamWaitEvent(st, ctx->evj, 0);
            }
            return r;
        }
        if (stepped) {
            cudaError_t r = cudaMemsetAsync(ctx->flags, 0, sizeof(unsigned), st);
            for (int n = 0; n < nsteps && r == cudaSuccess; n++)
                r = launch_multi2d(b, tz, any_cpml, (int)done_total, n, st, st != nullptr);
            return r;
        }
        cudaError_t r = cudaMemsetAsync(ctx->done, 0, (size_t)done_total * sizeof(int), st);
        if (r == cudaSuccess) r = cudaMemsetAsync(ctx->head, 0, sizeof(unsigned long long), st);
        if (r == cudaSuccess) r = cudaMemsetAsync(ctx->flags, 0, sizeof(unsigned), st);
        if (r == cudaSuccess) r = launch_batch2d(b, tz, any_cpml, grid, st);
        return r;
    };
    if (probe > 0) {  // timing probe: launch directly, leave outputs alone; the events bracket the launches only
        if (pe0 && (e = cudaEventRecord(pe0, bst))) return fail(e, "timing");
        if ((e = body(bst))) return fail(e, "launch");
        if (pe1 && (e = cudaEventRecord(pe1, bst))) return fail(e, "timing");
        return SIM_OK;
    }
    for (int i = 0; i < nitems; i++) {
        items[i].sim->batch_sched = march ? 1 : march2 ? 2 : stepped ? 3 : 4;
        items[i].sim->batch_tile = tz;
    }
    if (bst == nullptr) {  // the legacy stream cannot be captured: launch directly
        if ((e = body(bst))) return fail(e, "launch");
    } else {
        if (!ctx->exec) {
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(bst, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e1 = body(bst);
                e = cudaStreamEndCapture(bst, &graph);
                if (e1 != cudaSuccess) e = e1;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) return fail(e, "graph capture");
            ctx->key = key;
        }
        if ((e = cudaGraphLaunch(ctx->exec, bst))) return fail(e, "graph launch");
    }
    // the handles' later work waits for the batch; outputs to host
    if ((e = cudaEventRecord(ctx->ev, bst))) return fail(e, "ordering");
    bool wait = false;
    for (int i = 0; i < nitems; i++) {
        sim_t s = items[i].sim;
        if ((e = cudaStreamWaitEvent(s->st, ctx->ev, 0))) return fail(e, "ordering");
        const sim_batch_item &it = items[i];
        if (it.gather && gdev[i] == s->gath && it.nrec > 0) {
            if ((e = cudaMemcpyAsync(it.gather, s->gath, (size_t)it.nshots * nt * it.nrec * sizeof(float),
                                     cudaMemcpyDeviceToHost, s->st)))
                return fail(e, "gather download");
            wait = true;
        }
        if ((e = cudaMemcpyAsync(s->flags_host, s->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s->st)))
            return fail(e, "flags");
    }
    if ((e = cudaMemcpyAsync(ctx->flags_host, ctx->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, bst)) ||
        (e = cudaStreamSynchronize(bst)))
        return fail(e, "completion");
    if (*ctx->flags_host & kFlagTimeout) return thread_fail(SIM_ERR_TIMEOUT, "a bounded wait in the batch kernel gave up");
    for (int i = 0; i < nitems; i++)
        if (sim_status r = poll_flags(items[i].sim, wait)) return r;
    return SIM_OK;
}

// Batch autotuner: the schedule (row march, the two-step row march when no
// item has CPML, or the stepped kernel with list tiles of 8, 16 or 32 rows)
// of a batch shape (every item's grid, boundary,
// shot count, receivers; nt) is picked on its first call by timing a short
// probe of each candidate with CUDA events on the batch stream, and cached
// for the process. The persistent kernel (slower wherever measured: every
// item pays a counter, an acquire wait and a release) runs only when forced:
// GSIM_BATCH=march|march2|stepped|persistent fixes the schedule, GSIM_TILE_Z the
// tile height, GSIM_AUTOTUNE=0 takes the row march untimed.
std::mutex g_btune_mu;
std::map<std::vector<long long>, std::pair<int, int>> g_btune;

sim_status batch_impl(int nitems, const sim_batch_item *items, cudaStream_t bst) {
    if (nitems < 1 || !items || !items[0].sim) return batch_run(nitems, items, bst, kBatchMarch, 16, 0);
    int sched = -1, tz = 0;
    if (const char *bm = getenv("GSIM_BATCH")) {
        if (!strcmp(bm, "persistent")) sched = kBatchPersistent;
        else if (!strcmp(bm, "stepped")) sched = kBatchStepped;
        else if (!strcmp(bm, "march")) sched = kBatchMarch;
        else if (!strcmp(bm, "march2")) sched = kBatchMarch2;
    }
    if (const char *f = getenv("GSIM_TILE_Z")) {
        const int v = atoi(f);
        if (v == 8 || v == 16 || v == 32) tz = v;
    }
    const char *at = getenv("GSIM_AUTOTUNE");
    const bool untimed = at && at[0] == '0';
    if (sched >= 0 || untimed) {
        if (sched < 0) sched = kBatchMarch;
        return batch_run(nitems, items, bst, sched, tz ? tz : (sched == kBatchStepped ? 32 : 16), 0);
    }
    std::vector<long long> key = {items[0].sim->dev, items[0].sim->d.nt, tz};
    for (int i = 0; i < nitems; i++) {
        const sim_s *s = items[i].sim;
        if (!s) return batch_run(nitems, items, bst, kBatchMarch, 16, 0);  // reports the bad item
        key.insert(key.end(), {(long long)s->g.NZ, (long long)s->g.NX, (long long)s->d.bc, (long long)s->d.free_surface,
                               (long long)items[i].nshots, (long long)(items[i].nrec > 0 && items[i].gather)});
    }
    {
        std::lock_guard<std::mutex> lk(g_btune_mu);
        auto it = g_btune.find(key);
        if (it != g_btune.end()) return batch_run(nitems, items, bst, it->second.first, it->second.second, 0);
    }
    std::vector<std::pair<int, int>> cand;
    if (tz) cand = {{kBatchMarch, tz}, {kBatchStepped, tz}};
    else cand = {{kBatchMarch, 16}, {kBatchStepped, 8}, {kBatchStepped, 16}, {kBatchStepped, 32}};
    bool cpml = false;
    for (int i = 0; i < nitems; i++) cpml |= items[i].sim->d.bc == SIM_BC_CPML;
    if (!cpml) cand.push_back({kBatchMarch2, tz ? tz : 16});  // two steps per pass
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return thread_fail(SIM_ERR_CUDA, "batch autotune: event creation failed");
    }
    float best = 1e30f, best1 = 1e30f;  // best1: the fastest schedule of one step per launch
    std::pair<int, int> pick = cand[0], pick1 = cand[0];
    sim_status rc = SIM_OK;
    for (const auto &c : cand) {
        const int steps = 6;
        if ((rc = batch_run(nitems, items, bst, c.first, c.second, 2))) break;  // warm-up (and first-use set-up)
        if ((rc = batch_run(nitems, items, bst, c.first, c.second, steps, e0, e1))) break;
        float ms = 0;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            cudaGetLastError();
            rc = thread_fail(SIM_ERR_CUDA, "batch autotune timing failed");
            break;
        }
        if (getenv("GSIM_TUNE_LOG"))
            fprintf(stderr, "[gsim autotune] batch of %d items: %s tile %d: %.1f us/step (probe)\n", nitems,
                    c.first == kBatchMarch ? "march" : c.first == kBatchMarch2 ? "two-step march" : "stepped",
                    c.second, 1e3 * ms / steps);
        if (ms < best) best = ms, pick = c;
        if (c.first != kBatchMarch2 && ms < best1) best1 = ms, pick1 = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    // the two-step march only when it is clearly faster than every schedule
    // of one launch per step (a probe difference within 2% is noise)
    if (pick.first == kBatchMarch2 && best1 < 1.02f * best) pick = pick1;
    {
        std::lock_guard<std::mutex> lk(g_btune_mu);
        g_btune[key] = pick;
    }
    return batch_run(nitems, items, bst, pick.first, pick.second, 0);
}

}  // namespace

// Gradient mode of the batch: for every item, the adjoint-state gradient of
// its shots on its handle (all shots of an item in one call, FP64 fold over
// its shots) added to the item's FP64 accumulator, and its misfit. Items run
// one after another on their handles' streams, ordered after the batch
// stream's earlier work and before its later work.
sim_status batch_gradient(int nitems, const sim_batch_item *items, int ckpt_fp16, cudaStream_t bst) {
    if (nitems < 1 || !items) return thread_fail(SIM_ERR_ARG, "empty batch");
    for (int i = 0; i < nitems; i++) {
        const sim_batch_item &it = items[i];
        sim_t s = it.sim;
        if (!s || !s->model_set) return thread_fail(SIM_ERR_STATE, "batch item %d: no handle or no model", i);
        if (s->sticky) return s->sticky;
        if (s->dev != items[0].sim->dev) return thread_fail(SIM_ERR_ARG, "batch item %d: another device", i);
        if (it.nshots < 1 || it.nshots > s->d.max_shots)
            return thread_fail(SIM_ERR_ARG, "batch item %d: nshots outside [1, max_shots]", i);
        if (it.nrec < 1 || it.nrec > s->d.max_rec || !it.rec_pos)
            return thread_fail(SIM_ERR_ARG, "batch item %d: the gradient needs receivers", i);
        if (!it.wavelet || !it.src_pos || !it.d_obs)
            return thread_fail(SIM_ERR_ARG, "batch item %d: wavelet, sources and d_obs are required", i);
        if (!it.grad_sum_fp64 || !is_device_ptr(it.grad_sum_fp64))
            return thread_fail(SIM_ERR_ARG, "batch item %d: grad_sum_fp64 must be device memory", i);
        for (int j = 0; j < i; j++)
            if (items[j].sim == s) return thread_fail(SIM_ERR_ARG, "batch items %d and %d share a handle", j, i);
    }
    cudaSetDevice(items[0].sim->dev);
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return thread_fail(SIM_ERR_CUDA, "event creation failed");
    }
    sim_status rc = SIM_OK;
    for (int i = 0; i < nitems && rc == SIM_OK; i++) {
        const sim_batch_item &it = items[i];
        sim_t s = it.sim;
        if (cudaEventRecord(ev, bst) != cudaSuccess || cudaStreamWaitEvent(s->st, ev, 0) != cudaSuccess) {
            cudaGetLastError();
            rc = thread_fail(SIM_ERR_CUDA, "batch ordering failed");
            break;
        }
        AdjOpts o;
        o.grad_fp64 = it.grad_sum_fp64;
        double J = 0;
        rc = s->d.precision == SIM_FP64
                 ? adjoint_t<double>(s, it.nshots, it.wavelet, it.src_pos, it.nrec, it.rec_pos, it.d_obs, it.gather,
                                     it.misfit ? &J : nullptr, ckpt_fp16, nullptr, o)
                 : adjoint_t<float>(s, it.nshots, it.wavelet, it.src_pos, it.nrec, it.rec_pos, it.d_obs, it.gather,
                                    it.misfit ? &J : nullptr, ckpt_fp16, nullptr, o);
        if (rc != SIM_OK) {
            t_err = s->err;
            break;
        }
        if (it.misfit) *it.misfit = J;
        if (cudaEventRecord(ev, s->st) != cudaSuccess || cudaStreamWaitEvent(bst, ev, 0) != cudaSuccess) {
            cudaGetLastError();
            rc = thread_fail(SIM_ERR_CUDA, "batch ordering failed");
        }
    }
    cudaEventDestroy(ev);
    return rc;
}

// ============================================================== C ABI

extern "C" {

void sim_desc_init(sim_desc *d) {
    if (!d) return;
    memset(d, 0, sizeof(*d));
    d->space_order = 8;
    d->R = 1e-3;
    d->f_ref = 10.0;
    d->max_shots = 1;
    d->precision = SIM_FP32;
}

sim_status sim_plan(const sim_desc *din, double vmin, double vmax, sim_info *out) {
    if (!din || !out) return thread_fail(SIM_ERR_ARG, "NULL argument");
    sim_desc d = *din;
    normalise(d);
    if (sim_status r = validate(d)) return r;
    fill_info(d, out);
    return model_checks(d, vmin, vmax, out);
}

sim_status sim_create(const sim_desc *din, const void *vel, void *cuda_stream, sim_t *out) {
    if (!din || !out) return thread_fail(SIM_ERR_ARG, "NULL argument");
    *out = nullptr;
    sim_desc d = *din;
    normalise(d);
    if (sim_status r = validate(d)) return r;
    sim_s *s = new (std::nothrow) sim_s();
    if (!s) return thread_fail(SIM_ERR_OOM, "host allocation failed");
    s->d = d;
    s->g = make_geom(d);
    s->st = static_cast<cudaStream_t>(cuda_stream);
    s->esz = d.precision == SIM_FP64 ? 8 : 4;
    s->nsnap = nsnap_of(d);
    if (d.precision == SIM_FP32) {
        s->tile_x = kTileXF;
        s->tile_z = 16;
    }
    s->ntx = (s->g.NX + s->tile_x - 1) / s->tile_x;
    s->ntz = (s->g.NZ + s->tile_z - 1) / s->tile_z;
    s->nty = 1;
    sim_status rc = SIM_OK;
    if (cudaGetDevice(&s->dev) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return thread_fail(SIM_ERR_CUDA, "no CUDA device available");
    }
    const Geom &g = s->g;
    const size_t fb = (size_t)g.fstride * s->esz;
    const int ms = d.max_shots;
    const size_t nint = (size_t)g.nz * g.ny * g.nx;
    const size_t nprof = (size_t)prof_total(g);
    auto A = [&](size_t n) { return rc == SIM_OK ? s->alloc(n, &rc) : nullptr; };
    s->pbuf = A(2 * fb * ms);
    s->ch = A(fb);
    s->vpad = A(fb);
    s->vel = A(nint * s->esz);
    s->E = A(nprof * s->esz);
    s->ca = A(nprof * s->esz);
    s->cb = A(nprof * s->esz);
    if (d.bc == SIM_BC_CPML) {
        const int nbz = d.nb[0] + d.nb[1], nby = d.ndim == 3 ? d.nb[2] + d.nb[3] : 0, nbx = d.nb[4] + d.nb[5];
        const int on[3] = {nbz > 0, nby > 0, nbx > 0};
        for (int ax = 0; ax < 3; ax++)
            if (on[ax]) {
                // 2D kernels keep psi of two parities; 3D passes update psi in place
                s->psi[ax][0] = A(fb * ms);
                if (d.ndim == 2) s->psi[ax][1] = A(fb * ms);
                s->zeta[ax] = A(fb * ms);
            }
    }
    s->part = static_cast<double *>(A(3 * kMinmaxBlocks * sizeof(double)));
    s->io = static_cast<SimIO *>(A(sizeof(SimIO)));
    s->flags = static_cast<unsigned *>(A(sizeof(unsigned)));
    s->snap_max = static_cast<unsigned *>(A(sizeof(unsigned) * std::max(1, s->nsnap * ms)));
    s->snap_scale = static_cast<float *>(A(sizeof(float) * std::max(1, s->nsnap * ms)));
    s->wave = A((size_t)d.nt * s->esz);
    s->gath = A((size_t)ms * d.nt * std::max(1, d.max_rec) * s->esz);
    s->cap_start = (size_t)ms * max_tiles(s) + 1;
    s->cap_rec = std::max(1, d.max_rec);
    s->cap_grp = 8 * (size_t)std::max(ms, std::max(1, d.max_rec));
    s->rec_start = static_cast<int *>(A(s->cap_start * sizeof(int)));
    s->rec = A(s->cap_rec * sizeof(RecEntryT<double>));
    s->inj_start = static_cast<int *>(A(s->cap_start * sizeof(int)));
    s->inj_grp = static_cast<InjGroup *>(A(s->cap_grp * sizeof(InjGroup)));
    s->inj_ent = A(s->cap_grp * sizeof(InjEntryT<double>));
    const char *ge = getenv("GSIM_GRAPHS");
    s->use_graphs = !(ge && ge[0] == '0');
    if (rc == SIM_OK) rc = s->cuda(cudaStreamCreateWithFlags(&s->cst, cudaStreamNonBlocking), "stream");
    if (rc == SIM_OK) rc = s->cuda(cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming), "event");
    if (rc == SIM_OK) rc = s->cuda(cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming), "event");
    if (rc == SIM_OK && d.precision == SIM_FP32) rc = s->cuda(configure_step2d_f32(), "kernel configuration");
    if (rc == SIM_OK && d.precision == SIM_FP32 && d.ndim == 2) {
        rc = s->cuda(configure_resident2d(), "kernel configuration");
        if (rc == SIM_OK) rc = s->cuda(configure_march2d(), "kernel configuration");
        if (rc == SIM_OK) rc = s->cuda(configure_march2x(), "kernel configuration");
        s->rdone = static_cast<int *>(A(sizeof(int) * ms * max_tiles(s)));
        s->rtiles = static_cast<RTile *>(A(sizeof(RTile) * max_tiles(s)));
        // row march: one item per (shot, strip, 4 rows) at most
        s->cap_mseg = (size_t)ms * ((g.NX + kMarchW - 1) / kMarchW) * ((g.NZ + 3) / 4) + 2;
        s->mseg = static_cast<MarchSeg *>(A(sizeof(MarchSeg) * s->cap_mseg));
        s->mslice = static_cast<StepArgs<float> *>(A(sizeof(StepArgs<float>)));
        s->mctr = static_cast<unsigned *>(A(2 * sizeof(unsigned)));
    }
    if (rc == SIM_OK && d.ndim == 3) {
        rc = s->cuda(configure_step3d(), "kernel configuration");
        s->src3 = static_cast<Pt3 *>(A(sizeof(Pt3) * ms));
        s->rec3 = static_cast<Pt3 *>(A(sizeof(Pt3) * std::max(1, d.max_rec)));
    }
    if (rc == SIM_OK && cudaMallocHost(&s->flags_host, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        rc = s->fail(SIM_ERR_OOM, "pinned host allocation failed");
    }
    if (rc == SIM_OK) {
        *s->flags_host = 0;
        // ghost cells of every field must read as zero, forever
        for (void *p : {s->pbuf, s->ch, s->vpad})
            if (rc == SIM_OK)
                rc = s->cuda(cudaMemsetAsync(p, 0, p == s->pbuf ? 2 * fb * ms : fb, s->st), "initial clear");
        if (rc == SIM_OK) rc = s->cuda(cudaMemsetAsync(s->flags, 0, sizeof(unsigned), s->st), "initial clear");
        if (rc == SIM_OK) rc = s->cuda(cudaStreamSynchronize(s->st), "create sync");
    }
    if (rc != SIM_OK) {
        t_err = s->err;
        sim_destroy(s);
        return rc;
    }
    if (vel) {
        rc = sim_set_model(s, vel);
        if (rc != SIM_OK && rc != SIM_WARN_DISPERSION) {
            t_err = s->err;
            sim_destroy(s);
            return rc;
        }
    }
    *out = s;
    return rc;
}

sim_status sim_set_model(sim_t s, const void *vel) {
    if (!s || !vel) return thread_fail(SIM_ERR_ARG, "NULL argument");
    if (s->sticky) return s->sticky;
    cudaSetDevice(s->dev);
    return s->d.precision == SIM_FP64 ? set_model_t<double>(s, vel) : set_model_t<float>(s, vel);
}

sim_status sim_forward(sim_t s, int nshots, const void *wavelet, const double *src_pos, int nrec,
                       const double *rec_pos, void *gather, void *snaps, float *snap_scale) {
    if (!s) return thread_fail(SIM_ERR_ARG, "NULL handle");
    if (sim_status r = poll_flags(s, false)) return r;
    if (!s->model_set) return s->fail(SIM_ERR_STATE, "no velocity model set");
    if (nshots < 1 || nshots > s->d.max_shots)
        return s->fail(SIM_ERR_ARG, "nshots = %d outside [1, %d]", nshots, s->d.max_shots);
    if (nrec < 0 || nrec > s->d.max_rec) return s->fail(SIM_ERR_ARG, "nrec = %d outside [0, %d]", nrec, s->d.max_rec);
    if (nrec > 0 && !rec_pos) return s->fail(SIM_ERR_ARG, "receivers need positions");
    if (wavelet && !src_pos) return s->fail(SIM_ERR_ARG, "a wavelet needs source positions");
    cudaSetDevice(s->dev);
    return s->d.precision == SIM_FP64
               ? forward_t<double>(s, nshots, wavelet, src_pos, nrec, rec_pos, gather, snaps, snap_scale)
               : forward_t<float>(s, nshots, wavelet, src_pos, nrec, rec_pos, gather, snaps, snap_scale);
}

sim_status sim_adjoint(sim_t s, int nshots, const void *wavelet, const double *src_pos, int nrec,
                       const double *rec_pos, const void *d_obs, void *gather_out, double *misfit_out, int ckpt_fp16,
                       void *grad_v) {
    if (!s) return thread_fail(SIM_ERR_ARG, "NULL handle");
    if (sim_status r = poll_flags(s, false)) return r;
    if (!s->model_set) return s->fail(SIM_ERR_STATE, "no velocity model set");
    if (nshots < 1 || nshots > s->d.max_shots)
        return s->fail(SIM_ERR_ARG, "nshots = %d outside [1, %d]", nshots, s->d.max_shots);
    if (nrec < 0 || nrec > s->d.max_rec) return s->fail(SIM_ERR_ARG, "nrec = %d outside [0, %d]", nrec, s->d.max_rec);
    if (!src_pos || !rec_pos) return s->fail(SIM_ERR_ARG, "positions are required");
    cudaSetDevice(s->dev);
    const AdjOpts o;
    return s->d.precision == SIM_FP64
               ? adjoint_t<double>(s, nshots, wavelet, src_pos, nrec, rec_pos, d_obs, gather_out, misfit_out,
                                   ckpt_fp16, grad_v, o)
               : adjoint_t<float>(s, nshots, wavelet, src_pos, nrec, rec_pos, d_obs, gather_out, misfit_out,
                                  ckpt_fp16, grad_v, o);
}

sim_status sim_adjoint_vjp(sim_t s, int nshots, const void *wavelet, const double *src_pos, int nrec,
                           const double *rec_pos, const void *cot, void *gather_out, int ckpt_fp16, void *grad_v) {
    if (!s) return thread_fail(SIM_ERR_ARG, "NULL handle");
    if (sim_status r = poll_flags(s, false)) return r;
    if (!s->model_set) return s->fail(SIM_ERR_STATE, "no velocity model set");
    if (nshots < 1 || nshots > s->d.max_shots)
        return s->fail(SIM_ERR_ARG, "nshots = %d outside [1, %d]", nshots, s->d.max_shots);
    if (nrec < 0 || nrec > s->d.max_rec) return s->fail(SIM_ERR_ARG, "nrec = %d outside [0, %d]", nrec, s->d.max_rec);
    if (!src_pos || !rec_pos) return s->fail(SIM_ERR_ARG, "positions are required");
    cudaSetDevice(s->dev);
    AdjOpts o;
    o.vjp = true;
    return s->d.precision == SIM_FP64
               ? adjoint_t<double>(s, nshots, wavelet, src_pos, nrec, rec_pos, cot, gather_out, nullptr, ckpt_fp16,
                                   grad_v, o)
               : adjoint_t<float>(s, nshots, wavelet, src_pos, nrec, rec_pos, cot, gather_out, nullptr, ckpt_fp16,
                                  grad_v, o);
}

sim_status sim_batch(int nitems, const sim_batch_item *items, void *cuda_stream) {
    return batch_impl(nitems, items, static_cast<cudaStream_t>(cuda_stream));
}

sim_status sim_batch_ex(int nitems, const sim_batch_item *items, int mode, int ckpt_fp16, void *cuda_stream) {
    if (mode == 0) return batch_impl(nitems, items, static_cast<cudaStream_t>(cuda_stream));
    if (mode == 1) return batch_gradient(nitems, items, ckpt_fp16, static_cast<cudaStream_t>(cuda_stream));
    return thread_fail(SIM_ERR_ARG, "batch mode %d is neither 0 (forward) nor 1 (gradient)", mode);
}

sim_status sim_sync(sim_t s) {
    if (!s) return thread_fail(SIM_ERR_ARG, "NULL handle");
    cudaSetDevice(s->dev);
    return poll_flags(s, true);
}

sim_status sim_get_info(sim_t s, sim_info *out) {
    if (!s || !out) return thread_fail(SIM_ERR_ARG, "NULL argument");
    fill_info(s->d, out);
    out->tile_x = s->tile_x;
    out->tile_z = s->tile_z;
    out->last_path = s->last_path;
    out->last_rows = s->last_rows;
    out->vmin = s->vmin;
    out->vmax = s->vmax;
    out->courant = s->vmax * s->d.dt / s->d.h;
    out->device_bytes = s->bytes;
    out->batch_sched = s->batch_sched;
    out->batch_tile = s->batch_tile;
    if (s->g.ndim == 3 && s->tuned3d) {
        out->z_variant = s->zvariant;
        out->z_chunk = s->zchunk;
    }
    if (s->adj_ready) {
        out->adj_levels = s->plan.levels;
        out->adj_slots = s->plan.L;
        out->adj_top = s->plan.n1;
        out->adj_sub = s->plan.n2;
        out->adj_inner = s->plan.m;
        out->adj_bytes = s->adj_bytes;
    }
    return SIM_OK;
}

const char *sim_last_error(sim_t s) {
    if (s) return s->err.c_str();
    return t_err.c_str();
}

void sim_destroy(sim_t s) {
    if (!s) return;
    cudaSetDevice(s->dev);
    cudaStreamSynchronize(s->st);
    if (s->cst) cudaStreamSynchronize(s->cst);
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
    if (s->cst) cudaStreamDestroy(s->cst);
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    if (s->ev_out) cudaEventDestroy(s->ev_out);
    for (void *p : s->allocs) cudaFree(p);
    for (void *p : s->adj_allocs) cudaFree(p);
    if (s->flags_host) cudaFreeHost(s->flags_host);
    cudaGetLastError();
    delete s;
}

}  // extern "C"
