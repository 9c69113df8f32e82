// Velocity-model builder warps (App. "Model builder modules"): the
// pull-sample steps of Squish (Alg. squish), Fault (Alg. fault) and a
// simplified Deposit (Alg. deposit) on (nz, ny, nx) row-major device grids,
// ny = 1 for a 2D slice. One thread per output voxel, x fastest, so reads of
// the source grid by neighbouring threads fall in the same lines.
//
// Interpolation (the paper says "sinc"): an 8-tap Lanczos-windowed sinc per
// axis, sinc(x) sinc(x/4) on |x| < 4, weights normalised to sum 1, taps
// beyond the grid taking the edge value; labels by nearest neighbour (round
// half to even). A voxel whose pulled depth lies outside [0, nz) (depths
// down to -1e-6 counting as 0) takes the fill velocity and label. Source
// positions are computed in FP64, weights and sums in FP32.
#include <algorithm>
#include <cmath>

#include "sim_internal.h"

namespace gsim {
namespace {

constexpr int kTaps = 8;
constexpr int kMaxBeds = 128;

// first tap index and normalised weights of the 8 taps around s
__device__ __forceinline__ int taps(double s, float *w) {
    const double f = floor(s);
    const int i0 = (int)f - 3;
    const float fr = (float)(s - f);  // in [0, 1)
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < kTaps; k++) {
        const float x = fr + 3.f - (float)k;  // s - (i0 + k)
        float v;
        if (x == 0.f) {
            v = 1.f;
        } else if (fabsf(x) >= 4.f) {
            v = 0.f;
        } else {
            const float px = 3.14159265358979f * x;
            v = sinpif(x) / px * (sinpif(0.25f * x) / (0.25f * px));
        }
        w[k] = v;
        sum += v;
    }
    const float inv = 1.f / sum;
#pragma unroll
    for (int k = 0; k < kTaps; k++) w[k] *= inv;
    return i0;
}

__device__ __forceinline__ int clampi(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

__device__ __forceinline__ bool filled(double sz, int nz) { return sz < -1e-6 || sz >= (double)nz; }

__device__ __forceinline__ int nearest(double s, int n) { return clampi((int)rint(s), n); }

// ---------------------------------------------------------------- Squish
// A column's displacement is one number, so its 8 weights are the same at
// every depth: a thread computes them once and walks down kSquishRows rows
// of its column with a sliding window of the 8 taps (each input value read
// once per chunk). Threads: x fastest (coalesced rows), then y, then chunks.
constexpr int kSquishRows = 32;

__global__ void k_squish(int nz, int ny, int nx, const float *__restrict__ v, const int *__restrict__ lab,
                         const float *__restrict__ dz, float fill_v, int fill_label, float *__restrict__ vo,
                         int *__restrict__ lo) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const int z0 = blockIdx.z * kSquishRows, z1 = min(nz, z0 + kSquishRows);
    const long long col = (long long)y * nx + x, plane = (long long)ny * nx;
    const float d = dz[col];
    float w[kTaps];
    const int s0 = taps((double)d, w);  // taps of row z: z + s0 .. z + s0 + 7
    // the pulled depth z + d = (z + di) + fr with di = floor(d), fr in [0, 1)
    // exact in FP32, so the fill test and the nearest row are integer logic
    const int di = s0 + 3;
    const float fr = d - floorf(d);
    const int up = fr > 0.5f ? 1 : (fr < 0.5f ? 0 : -1);  // -1: a tie, rounded to even
    float win[kTaps];
#pragma unroll
    for (int k = 0; k < kTaps - 1; k++) win[k + 1] = v[clampi(z0 + s0 + k, nz) * plane + col];
#pragma unroll 4
    for (int z = z0; z < z1; z++) {
#pragma unroll
        for (int k = 0; k < kTaps - 1; k++) win[k] = win[k + 1];
        win[kTaps - 1] = v[clampi(z + s0 + kTaps - 1, nz) * plane + col];
        const long long o = z * plane + col;
        const int zk = z + di;
        // outside [0, nz) (depths down to -1e-6 count as 0)
        if (zk >= nz || zk <= -2 || (zk == -1 && fr < 1.f - 1e-6f)) {
            vo[o] = fill_v;
            if (lo) lo[o] = fill_label;
            continue;
        }
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < kTaps; k++) acc += w[k] * win[k];
        vo[o] = acc;
        if (lo) lo[o] = lab[clampi(zk + (up >= 0 ? up : (zk & 1)), nz) * plane + col];
    }
}

// ---------------------------------------------------------------- Fault
struct FaultK {
    double ct[3];      // cylinder centre (z, y, x)
    double ed[3], es[3];
    double R, th0, shift, dir, d_die, d_perp, th_die;
};

__global__ void k_fault(int nz, int ny, int nx, const float *__restrict__ v, const int *__restrict__ lab,
                        const FaultK F, float fill_v, int fill_label, float *__restrict__ vo,
                        int *__restrict__ lo) {
    const double hpi = 1.5707963267948966;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const long long i = ((long long)z * ny + y) * nx + x;
    {
        // cylindrical coordinates about the axis through ct along e_s
        const double wz = z - F.ct[0], wy = y - F.ct[1], wx = x - F.ct[2];
        const double u = wy * F.ed[1] + wx * F.ed[2];
        const double as = wy * F.es[1] + wx * F.es[2];
        const double r = hypot(u, wz);
        const double rr = fabs(r - F.R) / F.d_die, rs = fabs(as) / F.d_perp;
        double rt = 2.0, th = 0.0;
        if (rr < 1.0 && rs < 1.0) {
            th = atan2(wz, u);
            rt = fabs(th - F.th0) / F.th_die;
        }
        if (!(rr < 1.0 && rs < 1.0 && rt < 1.0)) {  // outside the die-off region: the voxel does not move
            vo[i] = v[i];
            if (lo) lo[i] = lab[i];
            return;
        }
        const double taper = cos(hpi * rr) * cos(hpi * rt) * cos(hpi * rs);
        const double chi = r >= F.R ? 1.0 : -1.0;
        const double thn = th - chi * F.dir * taper * F.shift;
        double sn, cs;
        sincos(thn, &sn, &cs);
        const double fz = F.ct[0] + r * sn;
        const double fy = F.ct[1] + r * cs * F.ed[1] + as * F.es[1];
        const double fx = F.ct[2] + r * cs * F.ed[2] + as * F.es[2];
        const double sz = 2.0 * z - fz, sy = 2.0 * y - fy, sx = 2.0 * x - fx;
        if (filled(sz, nz)) {
            vo[i] = fill_v;
            if (lo) lo[i] = fill_label;
            return;
        }
        float wzt[kTaps], wxt[kTaps];
        const int iz0 = taps(sz, wzt), ix0 = taps(sx, wxt);
        int xs[kTaps];
#pragma unroll
        for (int c = 0; c < kTaps; c++) xs[c] = clampi(ix0 + c, nx);
        float acc = 0.f;
        if (ny == 1) {
#pragma unroll
            for (int a = 0; a < kTaps; a++) {
                const float *row = v + (long long)clampi(iz0 + a, nz) * nx;
                float ra = 0.f;
#pragma unroll
                for (int c = 0; c < kTaps; c++) ra += wxt[c] * row[xs[c]];
                acc += wzt[a] * ra;
            }
        } else {
            float wyt[kTaps];
            const int iy0 = taps(sy, wyt);
            for (int a = 0; a < kTaps; a++) {
                const long long pz = (long long)clampi(iz0 + a, nz) * ny;
                float pa = 0.f;
                for (int b = 0; b < kTaps; b++) {
                    const float *row = v + (pz + clampi(iy0 + b, ny)) * nx;
                    float rb = 0.f;
#pragma unroll
                    for (int c = 0; c < kTaps; c++) rb += wxt[c] * row[xs[c]];
                    pa += wyt[b] * rb;
                }
                acc += wzt[a] * pa;
            }
        }
        vo[i] = acc;
        if (lo) lo[i] = lab[((long long)nearest(sz, nz) * ny + nearest(sy, ny)) * nx + nearest(sx, nx)];
    }
}

// ---------------------------------------------------------------- Deposit
struct DepositK {
    int t, nbeds, nzt, label0;
    float beta, a_eta, f_top, f_base, vbar;
    float vbed[kMaxBeds];
    int off[kMaxBeds];
};

__global__ void k_deposit(int nz, int ny, int nx, const float *__restrict__ v, const int *__restrict__ lab,
                          const DepositK P, const float *__restrict__ bounds, const float *__restrict__ eta,
                          float *__restrict__ vo, int *__restrict__ lo) {
    const long long plane = (long long)ny * nx;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const long long col = (long long)y * nx + x, i = z * plane + col;
    {
        if (z >= P.t) {  // the model below, pushed down by the slab
            vo[i] = v[i - (long long)P.t * plane];
            if (lo) lo[i] = lab[i - (long long)P.t * plane];
            return;
        }
        int ell = 0;
        float start = 0.f;
        for (int b = 0; b < P.nbeds - 1; b++) {  // beds whose boundary lies above z
            const float h = bounds[b * plane + col];
            if (h < (float)z) {
                ell++;
                start = fmaxf(start, h);
            }
        }
        const float top = P.f_top > 0.f ? fminf((float)z / (P.f_top * P.t), 1.f) : 1.f;
        const float base = P.f_base > 0.f ? fminf((float)(P.t - z) / (P.f_base * P.t), 1.f) : 1.f;
        const float tau = top * base;
        const int zt = clampi(z - (int)floorf(start) + P.off[ell], P.nzt);
        const float tex = eta ? eta[zt * plane + col] : 0.f;
        vo[i] = (P.vbar + P.beta * z) + tau * ((P.vbed[ell] - P.vbar) + P.a_eta * tex);
        if (lo) lo[i] = P.label0 + ell;
    }
}

sim_status finish(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SIM_OK;
    cudaGetLastError();
    set_thread_error((std::string(what) + ": " + cudaGetErrorString(e)).c_str());
    return SIM_ERR_CUDA;
}

bool bad_grid(int nz, int ny, int nx, const float *v, const float *vo, const int *lab, const int *lo) {
    return nz < 1 || ny < 1 || nx < 1 || !v || !vo || v == vo || (!lab) != (!lo) || (lab && lab == lo);
}

}  // namespace
}  // namespace gsim

using namespace gsim;

extern "C" sim_status sim_model_squish(int nz, int ny, int nx, const float *v_in, const int *lab_in, const float *dz,
                                       float fill_v, int fill_label, float *v_out, int *lab_out, void *stream) {
    if (bad_grid(nz, ny, nx, v_in, v_out, lab_in, lab_out) || !dz) {
        set_thread_error("sim_model_squish: need positive sizes, distinct input and output grids, a displacement "
                         "field, and labels on both sides or neither");
        return SIM_ERR_ARG;
    }
    if (ny > 65535 || (nz + kSquishRows - 1) / kSquishRows > 65535) {
        set_thread_error("sim_model_squish: ny and nz / 32 must stay below 65536");
        return SIM_ERR_ARG;
    }
    const dim3 grid((nx + 127) / 128, ny, (nz + kSquishRows - 1) / kSquishRows);
    k_squish<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(nz, ny, nx, v_in, lab_in, dz, fill_v, fill_label,
                                                                  v_out, lab_out);
    return finish(cudaGetLastError(), "sim_model_squish");
}

extern "C" sim_status sim_model_fault(int nz, int ny, int nx, const float *v_in, const int *lab_in,
                                      const sim_fault *f, float fill_v, int fill_label, float *v_out, int *lab_out,
                                      void *stream) {
    if (bad_grid(nz, ny, nx, v_in, v_out, lab_in, lab_out) || !f || !(f->radius > 0) || !(f->d_die > 0) ||
        !(f->d_perp > 0) || !(f->theta_die > 0) || (f->direction != 1 && f->direction != -1)) {
        set_thread_error("sim_model_fault: need positive sizes, distinct grids, labels on both sides or neither, "
                         "radius and die-off extents > 0 and direction +1 or -1");
        return SIM_ERR_ARG;
    }
    FaultK K{};
    K.ed[0] = 0.0;
    K.ed[1] = std::cos(f->azimuth);
    K.ed[2] = std::sin(f->azimuth);
    K.es[0] = 0.0;
    K.es[1] = -std::sin(f->azimuth);
    K.es[2] = std::cos(f->azimuth);
    const double dz = f->radius * std::sin(f->dip), daz = f->radius * std::cos(f->dip);
    K.ct[0] = f->cz - dz;
    K.ct[1] = f->cy - daz * K.ed[1];
    K.ct[2] = f->cx - daz * K.ed[2];
    K.th0 = std::atan2(dz, daz);
    K.R = f->radius;
    K.shift = f->slip / f->radius;
    K.dir = f->direction;
    K.d_die = f->d_die;
    K.d_perp = f->d_perp;
    K.th_die = f->theta_die;
    if (ny > 65535 || nz > 65535) {
        set_thread_error("sim_model_fault: ny and nz must stay below 65536");
        return SIM_ERR_ARG;
    }
    const dim3 grid((nx + 127) / 128, ny, nz);
    k_fault<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(nz, ny, nx, v_in, lab_in, K, fill_v, fill_label,
                                                                 v_out, lab_out);
    return finish(cudaGetLastError(), "sim_model_fault");
}

extern "C" sim_status sim_model_deposit(int nz, int ny, int nx, const float *v_in, const int *lab_in,
                                        const sim_deposit *p, const float *bounds, const float *vbed,
                                        const int *offsets, const float *eta, float *v_out, int *lab_out,
                                        void *stream) {
    if (bad_grid(nz, ny, nx, v_in, v_out, lab_in, lab_out) || !p || p->t < 1 || p->t > nz || p->nbeds < 1 ||
        p->nbeds > kMaxBeds || (p->nbeds > 1 && !bounds) || !vbed || !offsets || (eta && p->nzt < 1) ||
        p->f_top < 0 || p->f_base < 0) {
        set_thread_error("sim_model_deposit: need positive sizes, distinct grids, labels on both sides or neither, "
                         "1 <= t <= nz, 1 <= nbeds <= 128, bed boundaries when nbeds > 1, bed velocities and "
                         "offsets, and non-negative taper fractions");
        return SIM_ERR_ARG;
    }
    DepositK K{};
    K.t = p->t;
    K.nbeds = p->nbeds;
    K.nzt = eta ? p->nzt : 1;
    K.label0 = p->label0;
    K.beta = p->beta;
    K.a_eta = eta ? p->a_eta : 0.f;
    K.f_top = p->f_top;
    K.f_base = p->f_base;
    double sum = 0.0;
    for (int b = 0; b < p->nbeds; b++) {
        K.vbed[b] = vbed[b];
        K.off[b] = offsets[b];
        sum += vbed[b];
    }
    K.vbar = (float)(sum / p->nbeds);
    if (ny > 65535 || nz > 65535) {
        set_thread_error("sim_model_deposit: ny and nz must stay below 65536");
        return SIM_ERR_ARG;
    }
    const dim3 grid((nx + 127) / 128, ny, nz);
    k_deposit<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(nz, ny, nx, v_in, lab_in, K, bounds, eta, v_out,
                                                                   lab_out);
    return finish(cudaGetLastError(), "sim_model_deposit");
}
