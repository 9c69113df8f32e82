// sim_forward_noalloc: a forward solve that allocates no device memory.
//
// Some callers cannot allocate GPU memory at the moment they need a solve:
// processes whose device memory has been reserved in full up front by a
// framework's pool (a cudaMalloc there fails), and latency-critical paths
// where cudaMalloc / cudaFree, which may synchronise the whole device, are
// not acceptable. For them this entry point takes the caller's inputs and
// outputs and keeps every intermediate (pressure fields, the c field, the
// absorbing-layer profiles, the receiver and source lists, the I/O block) in
// one fixed array, kScratchBytes large, that lives in the library's device
// image: every GPU that loads the library holds it until the process exits.
//
// Contract (also in include/sim.h):
//  - 2D, FP32, one shot, no snapshots; vel, wavelet and gather are device
//    pointers, positions are host arrays.
//  - Problems whose working set exceeds kScratchBytes are rejected with
//    SIM_ERR_ARG before any GPU work.
//  - Every call reads the velocity range back to the host and waits for its
//    stream (twice), and copies host-built lists in; so no call may be made
//    while its stream (or, in global capture mode, any stream) is being
//    captured into a CUDA graph.
//  - The first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current and keeps it for the
//    life of the process; do not use the entry point across a
//    cudaDeviceReset, which reloads the module and moves the array.
//  - Every call reuses the same array and clears what must start at zero;
//    calls whose GPU work overlaps (other streams, other threads) race on
//    it. Calls on one stream are ordered and safe.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "sim_internal.h"
#include "stencil.cuh"

namespace gsim {
namespace {

constexpr size_t kScratchBytes = 32u << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

sim_status nfail(sim_status code, const char *msg) {
    set_thread_error(msg);
    return code;
}

std::mutex g_mu;
std::vector<std::pair<int, unsigned char *>> g_addr;  // device -> address of g_scratch

// Device address of g_scratch on the current device (looked up once per device).
sim_status scratch_address(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nfail(SIM_ERR_CUDA, "no CUDA device available");
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &kv : g_addr)
        if (kv.first == dev) {
            *out = kv.second;
            return SIM_OK;
        }
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nfail(SIM_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    }
    if (configure_step2d_f32() != cudaSuccess) {  // shared-memory opt-in of the step kernel, once per device
        cudaGetLastError();
        return nfail(SIM_ERR_CUDA, "step kernel configuration failed");
    }
    g_addr.push_back({dev, static_cast<unsigned char *>(p)});
    *out = static_cast<unsigned char *>(p);
    return SIM_OK;
}

long long rup(long long v, long long m) { return (v + m - 1) / m * m; }

// Layout of sub-arrays inside the scratch array (256-byte aligned offsets).
struct Carve {
    size_t used = 0;
    bool ok = true;
    size_t take(size_t bytes) {
        const size_t off = (size_t)rup((long long)used, 256);
        if (off + bytes > kScratchBytes) ok = false;
        used = off + bytes;
        return off;
    }
};

}  // namespace
}  // namespace gsim

using namespace gsim;

extern "C" sim_status sim_forward_noalloc(const sim_desc *din, const float *vel, const float *wavelet,
                                          const double *src_pos, int nrec, const double *rec_pos, float *gather,
                                          void *cuda_stream) {
    if (!din || !vel || !wavelet || !src_pos || (nrec > 0 && (!rec_pos || !gather)) || nrec < 0)
        return nfail(SIM_ERR_ARG, "missing argument");
    sim_desc d = *din;
    if (d.space_order == 0) d.space_order = 8;
    if (!(d.R > 0)) d.R = 1e-3;
    if (!(d.f_ref > 0)) d.f_ref = 10.0;
    if (d.ndim != 2 || d.precision != SIM_FP32 || d.space_order != 8)
        return nfail(SIM_ERR_UNSUPPORTED, "sim_forward_noalloc runs 2D FP32 8th-order problems");
    if (d.nz < 1 || d.nx < 1 || !(d.h > 0) || !(d.dt > 0) || d.nt < 1 || d.bc < 0 || d.bc > 2)
        return nfail(SIM_ERR_ARG, "invalid description");
    for (int k = 0; k < 6; k++)
        if (d.nb[k] < 0 || d.nb[k] > 4096) return nfail(SIM_ERR_ARG, "invalid absorbing width");
    if (d.free_surface && d.nb[0] != 0) return nfail(SIM_ERR_ARG, "a free surface needs nb[0] = 0");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // geometry (same layout as the handle path)
    Geom g{};
    g.ndim = 2;
    g.nz = d.nz;
    g.ny = 1;
    g.nx = d.nx;
    g.nbz0 = d.nb[0];
    g.nbz1 = d.nb[1];
    g.nbx0 = d.nb[4];
    g.nbx1 = d.nb[5];
    g.NZ = g.nbz0 + g.nz + g.nbz1;
    g.NY = 1;
    g.NX = g.nbx0 + g.nx + g.nbx1;
    g.oz = g.nbz0;
    g.ox = g.nbx0;
    g.P = (int)rup(kGhost + rup(g.NX, kRoundX) + kGhost, 32);
    g.PY = 1;
    g.fstride = (kGhost + rup(g.NZ, kRoundZ) + kGhost) * (long long)g.P;
    g.org = (long long)kGhost * g.P + kGhost;
    g.fs = d.free_surface;
    const int TZ = 16, ntx = (g.NX + kTileXF - 1) / kTileXF, ntz = (g.NZ + TZ - 1) / TZ, ntiles = ntx * ntz;
    const bool cpml = d.bc == SIM_BC_CPML;
    const int on[3] = {cpml && (g.nbz0 + g.nbz1) > 0, 0, cpml && (g.nbx0 + g.nbx1) > 0};
    const int N[3] = {g.NZ, 1, g.NX};
    long long poff[3], ptot = 0;
    for (int a = 0; a < 3; a++) {
        poff[a] = ptot + kProfAlign;
        ptot += kProfAlign + rup(N[a], kProfAlign) + kProfAlign;
    }
    // layout of the working set inside the scratch array; too large: reject before any GPU work
    Carve cv;
    const size_t o_pb = cv.take((size_t)2 * g.fstride * 4), o_ch = cv.take((size_t)g.fstride * 4),
                 o_vp = cv.take((size_t)g.fstride * 4);
    size_t o_psi[3][2] = {{0, 0}, {0, 0}, {0, 0}}, o_zeta[3] = {0, 0, 0};
    for (int ax = 0; ax < 3; ax += 2)
        if (on[ax]) {
            o_psi[ax][0] = cv.take((size_t)g.fstride * 4);
            o_psi[ax][1] = cv.take((size_t)g.fstride * 4);
            o_zeta[ax] = cv.take((size_t)g.fstride * 4);
        }
    const size_t o_E = cv.take((size_t)ptot * 4), o_ca = cv.take((size_t)ptot * 4), o_cb = cv.take((size_t)ptot * 4);
    const size_t o_rs = cv.take((size_t)(ntiles + 1) * 4);
    const size_t o_rec = cv.take((size_t)std::max(1, nrec) * sizeof(RecEntryT<float>));
    const size_t o_is = cv.take((size_t)(ntiles + 1) * 4);
    const size_t o_ig = cv.take(8 * sizeof(InjGroup)), o_ie = cv.take(8 * sizeof(InjEntryT<float>));
    const size_t o_io = cv.take(sizeof(SimIO)), o_fl = cv.take(sizeof(unsigned));
    const size_t o_part = cv.take(3 * kMinmaxBlocks * sizeof(double));
    if (!cv.ok) return nfail(SIM_ERR_ARG, "problem exceeds the 32 MiB scratch of sim_forward_noalloc");

    unsigned char *base = nullptr;
    if (sim_status r = scratch_address(&base)) return r;
    float *pb = reinterpret_cast<float *>(base + o_pb), *ch = reinterpret_cast<float *>(base + o_ch);
    float *vp = reinterpret_cast<float *>(base + o_vp);
    float *psi[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    float *zeta[3] = {nullptr, nullptr, nullptr};
    for (int ax = 0; ax < 3; ax += 2)
        if (on[ax]) {
            psi[ax][0] = reinterpret_cast<float *>(base + o_psi[ax][0]);
            psi[ax][1] = reinterpret_cast<float *>(base + o_psi[ax][1]);
            zeta[ax] = reinterpret_cast<float *>(base + o_zeta[ax]);
        }
    float *E = reinterpret_cast<float *>(base + o_E), *ca = reinterpret_cast<float *>(base + o_ca);
    float *cb = reinterpret_cast<float *>(base + o_cb);
    int *rec_start = reinterpret_cast<int *>(base + o_rs);
    RecEntryT<float> *rec = reinterpret_cast<RecEntryT<float> *>(base + o_rec);
    int *inj_start = reinterpret_cast<int *>(base + o_is);
    InjGroup *inj_grp = reinterpret_cast<InjGroup *>(base + o_ig);
    InjEntryT<float> *inj_ent = reinterpret_cast<InjEntryT<float> *>(base + o_ie);
    SimIO *io = reinterpret_cast<SimIO *>(base + o_io);
    unsigned *flags = reinterpret_cast<unsigned *>(base + o_fl);
    double *part = reinterpret_cast<double *>(base + o_part);

    auto cuda = [&](cudaError_t e, const char *what) {
        if (e == cudaSuccess) return SIM_OK;
        cudaGetLastError();
        set_thread_error((std::string(what) + ": " + cudaGetErrorString(e)).c_str());
        return SIM_ERR_CUDA;
    };
    // velocity range: CFL check and the CPML d0
    if (sim_status r = cuda(launch_minmax<float>(g, vel, part, st), "velocity range")) return r;
    std::vector<double> hp(3 * kMinmaxBlocks);
    if (sim_status r = cuda(cudaMemcpyAsync(hp.data(), part, hp.size() * 8, cudaMemcpyDeviceToHost, st), "readback"))
        return r;
    if (sim_status r = cuda(cudaStreamSynchronize(st), "readback")) return r;
    double vmax = 0, bad = 0;
    for (int b = 0; b < kMinmaxBlocks; b++) {
        vmax = std::max(vmax, hp[3 * b + 1]);
        bad += hp[3 * b + 2];
    }
    if (bad > 0) return nfail(SIM_ERR_ARG, "velocity has non-finite or non-positive cells");
    const double smax = 1.0 / std::sqrt(2.0 * (std::fabs(kC1) + std::fabs(kC2) + std::fabs(kC3) + std::fabs(kC4)));
    if (vmax * d.dt / d.h > smax && !d.skip_cfl_check) return nfail(SIM_ERR_CFL, "v_max dt / h exceeds the bound");

    // clear what must start at zero: fields (with their ghost cells), CPML memory, flags
    if (sim_status r = cuda(cudaMemsetAsync(base, 0, cv.used, st), "clear")) return r;

    // absorbing-layer profiles (host arithmetic, as in sim_create / sim_set_model)
    std::vector<float> hE(ptot, 0.f), hca(ptot, 0.f), hcb(ptot, 0.f);
    const int lo[3] = {g.nbz0, 0, g.nbx0}, hi[3] = {g.nbz1, 0, g.nbx1};
    for (int a = 0; a < 3; a++)
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
                const double cdamp = 1.5 * std::log(1.0 / d.R) / w;
                const double eta = 1e-3 * (cdamp / d.h) * (rho - std::sin(2 * M_PI * rho) / (2 * M_PI));
                hE[poff[a] + i] = (float)(eta * d.h * d.h / (2.0 * d.dt));
            } else if (cpml) {
                const double d0 = 3.0 * vmax * std::log(1.0 / d.R) / (2.0 * w * d.h);
                const double dd = d0 * rho * rho, alpha = M_PI * d.f_ref * (1.0 - rho);
                const double b = std::exp(-(dd + alpha) * d.dt);
                hca[poff[a] + i] = (float)(dd * (b - 1.0) / (dd + alpha));
                hcb[poff[a] + i] = (float)b;
            }
        }
    if (sim_status r = cuda(cudaMemcpyAsync(E, hE.data(), ptot * 4, cudaMemcpyHostToDevice, st), "profiles")) return r;
    if (sim_status r = cuda(cudaMemcpyAsync(ca, hca.data(), ptot * 4, cudaMemcpyHostToDevice, st), "profiles")) return r;
    if (sim_status r = cuda(cudaMemcpyAsync(cb, hcb.data(), ptot * 4, cudaMemcpyHostToDevice, st), "profiles")) return r;
    if (sim_status r = cuda(launch_setup_model<float>(g, vel, ch, vp, d.dt / d.h, st), "model set-up")) return r;

    // receiver and source lists for 128 x 16 tiles
    auto locate = [&](const double *pos, int i0[2], double t[2]) {
        double f[2] = {pos[1] / d.h + g.oz, pos[0] / d.h + g.ox};
        const int lo2[2] = {g.oz, g.ox}, len[2] = {g.nz, g.nx};
        for (int a = 0; a < 2; a++) {
            const double r = std::nearbyint(f[a]);
            if (std::fabs(f[a] - r) < 1e-6) f[a] = r;
            if (!(f[a] >= lo2[a]) || !(f[a] <= lo2[a] + len[a] - 1)) return false;
            i0[a] = (int)std::floor(f[a]);
            t[a] = f[a] - i0[a];
        }
        return true;
    };
    std::vector<int> rs(ntiles + 1, 0);
    std::vector<std::pair<int, RecEntryT<float>>> tmp;
    for (int r = 0; r < nrec; r++) {
        int i0[2];
        double t[2];
        if (!locate(rec_pos + 2 * r, i0, t)) return nfail(SIM_ERR_ARG, "a receiver lies outside the interior");
        RecEntryT<float> e{};
        e.rec = r;
        const int tz = i0[0] / TZ, tx = i0[1] / kTileXF;
        e.lz = i0[0] - tz * TZ;
        e.lx = i0[1] - tx * kTileXF;
        e.w[0] = (float)((1 - t[0]) * (1 - t[1]));
        e.w[1] = (float)((1 - t[0]) * t[1]);
        e.w[2] = (float)(t[0] * (1 - t[1]));
        e.w[3] = (float)(t[0] * t[1]);
        tmp.push_back({tz * ntx + tx, e});
    }
    std::stable_sort(tmp.begin(), tmp.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
    std::vector<RecEntryT<float>> re;
    for (auto &p : tmp) {
        rs[p.first + 1]++;
        re.push_back(p.second);
    }
    for (int i = 0; i < ntiles; i++) rs[i + 1] += rs[i];
    std::vector<int> is(ntiles + 1, 0);
    std::vector<std::pair<int, int>> cells;  // (tile, local cell) per source corner
    std::vector<float> wts;
    {
        int i0[2];
        double t[2];
        if (!locate(src_pos, i0, t)) return nfail(SIM_ERR_ARG, "the source lies outside the interior");
        for (int dz = 0; dz < 2; dz++)
            for (int dx = 0; dx < 2; dx++) {
                const double w = (dz ? t[0] : 1 - t[0]) * (dx ? t[1] : 1 - t[1]);
                const int z = i0[0] + dz, x = i0[1] + dx;
                if (w == 0.0 || (g.fs && z == 0)) continue;
                const int tz = z / TZ, tx = x / kTileXF;
                cells.push_back({tz * ntx + tx, (z - tz * TZ) * kTileXF + (x - tx * kTileXF)});
                wts.push_back((float)w);
            }
    }
    std::vector<InjGroup> ig;
    std::vector<InjEntryT<float>> ie;
    std::vector<int> order(cells.size());
    for (size_t k = 0; k < order.size(); k++) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cells[a] < cells[b]; });
    for (int k : order) {
        InjGroup G{};
        G.cell = cells[k].second;
        G.e0 = (int)ie.size();
        InjEntryT<float> e{};
        e.pt = 0;
        e.w = wts[k];
        ie.push_back(e);
        G.e1 = (int)ie.size();
        ig.push_back(G);
        is[cells[k].first + 1]++;
    }
    for (int i = 0; i < ntiles; i++) is[i + 1] += is[i];
    if (sim_status r = cuda(cudaMemcpyAsync(rec_start, rs.data(), rs.size() * 4, cudaMemcpyHostToDevice, st), "lists"))
        return r;
    if (!re.empty())
        if (sim_status r = cuda(cudaMemcpyAsync(rec, re.data(), re.size() * sizeof(re[0]), cudaMemcpyHostToDevice, st),
                                "lists"))
            return r;
    if (sim_status r = cuda(cudaMemcpyAsync(inj_start, is.data(), is.size() * 4, cudaMemcpyHostToDevice, st), "lists"))
        return r;
    if (!ig.empty()) {
        if (sim_status r = cuda(cudaMemcpyAsync(inj_grp, ig.data(), ig.size() * sizeof(ig[0]), cudaMemcpyHostToDevice, st),
                                "lists"))
            return r;
        if (sim_status r = cuda(cudaMemcpyAsync(inj_ent, ie.data(), ie.size() * sizeof(ie[0]), cudaMemcpyHostToDevice, st),
                                "lists"))
            return r;
    }
    SimIO hio{};
    hio.wavelet = wavelet;
    hio.gather = nrec > 0 ? gather : nullptr;
    hio.nrec = nrec;
    hio.nshots = 1;
    if (sim_status r = cuda(cudaMemcpyAsync(io, &hio, sizeof hio, cudaMemcpyHostToDevice, st), "io")) return r;

    // the time loop with the FP32 step kernel
    StepArgs<float> a{};
    a.g = g;
    a.pbuf[0] = pb;
    a.pbuf[1] = pb + g.fstride;
    a.ch = ch;
    for (int ax = 0; ax < 3; ax++) {
        a.E[ax] = d.bc == SIM_BC_SPONGE ? E + poff[ax] : nullptr;
        a.ca[ax] = on[ax] ? ca + poff[ax] : nullptr;
        a.cb[ax] = on[ax] ? cb + poff[ax] : nullptr;
        a.psi[ax][0] = psi[ax][0];
        a.psi[ax][1] = psi[ax][1];
        a.zeta[ax] = zeta[ax];
    }
    a.bc = d.bc;
    a.src_scale = 1.f;
    a.ntx = ntx;
    a.nty = 1;
    a.ntz = ntz;
    a.nt = d.nt;
    a.snap_every = 1;
    a.rec_start = rec_start;
    a.rec = rec;
    a.inj_start = inj_start;
    a.inj_grp = inj_grp;
    a.inj_ent = inj_ent;
    a.inj_per_shot = 1;
    a.io = io;
    a.flags = flags;
    a.sample = nrec > 0;
    for (int n = 0; n < d.nt; n++) {
        StepTime t{};
        t.n = n;
        t.snap_k = t.max_k = -1;
        t.inj_row = n;
        if (sim_status r = cuda(launch_step2d_f32(a, t, TZ, 1, kModeForward, st, false), "step kernel")) return r;
    }
    // non-finite values anywhere in the final field (the step kernel only
    // checks the samples it records)
    if (sim_status r = cuda(launch_check_finite<float>(g, a.pbuf[d.nt & 1], 1, flags, st), "finite check")) return r;
    unsigned hflags = 0;
    if (sim_status r = cuda(cudaMemcpyAsync(&hflags, flags, sizeof hflags, cudaMemcpyDeviceToHost, st), "flags"))
        return r;
    if (sim_status r = cuda(cudaStreamSynchronize(st), "completion")) return r;
    if (hflags & kFlagUnstable) return nfail(SIM_ERR_UNSTABLE, "non-finite values in the wavefield or outputs");
    return SIM_OK;
}
