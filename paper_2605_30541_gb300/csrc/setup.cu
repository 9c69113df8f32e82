// Model set-up and health checks: padded coefficient fields from the interior
// velocity, the velocity range (for the CFL and dispersion checks of
// App. E.3.1-E.3.2) and a scan for non-finite values.
#include <cfloat>

#include "sim_internal.h"

namespace gsim {
namespace {

// c-field (v dt / h)^2 and the padded velocity; absorbing cells copy the
// nearest interior cell.
template <typename T>
__global__ void k_setup_model(const Geom g, const T *__restrict__ vel, T *ch, T *vpad, double r) {
    const long long total = (long long)g.NZ * g.NY * g.NX;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.NX);
        const long long zy = i / g.NX;
        const int y = (int)(zy % g.NY);
        const int z = (int)(zy / g.NY);
        const int iz = min(max(z - g.oz, 0), g.nz - 1);
        const int iy = min(max(y - g.oy, 0), g.ny - 1);
        const int ix = min(max(x - g.ox, 0), g.nx - 1);
        const double v = (double)vel[((long long)iz * g.ny + iy) * g.nx + ix];
        const long long o = cell_off(g, z, y, x);
        ch[o] = (T)((v * r) * (v * r));
        vpad[o] = (T)v;
    }
}

// Per-block (min, max, #bad) of the interior velocity into part[3 * block].
template <typename T>
__global__ void k_minmax(const T *__restrict__ vel, long long n, double *part) {
    __shared__ double smin[256], smax[256], sbad[256];
    double lo = DBL_MAX, hi = -DBL_MAX, bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = (double)vel[i];
        if (!(v > 0.0) || !(v <= DBL_MAX)) bad += 1;
        else {
            lo = fmin(lo, v);
            hi = fmax(hi, v);
        }
    }
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    sbad[threadIdx.x] = bad;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
            sbad[threadIdx.x] += sbad[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = smin[0];
        part[3 * blockIdx.x + 1] = smax[0];
        part[3 * blockIdx.x + 2] = sbad[0];
    }
}

template <typename T>
__global__ void k_check_finite(const T *__restrict__ f, long long n, unsigned *flags) {
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite((double)f[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, kFlagUnstable);
}

}  // namespace

template <typename T>
cudaError_t launch_setup_model(const Geom &g, const T *vel, T *ch, T *vpad, double dt_over_h,
                               cudaStream_t st) {
    k_setup_model<T><<<1216, 256, 0, st>>>(g, vel, ch, vpad, dt_over_h);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_minmax(const Geom &g, const T *vel, double *part, cudaStream_t st) {
    const long long n = (long long)g.nz * g.ny * g.nx;
    k_minmax<T><<<kMinmaxBlocks, 256, 0, st>>>(vel, n, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_check_finite(const Geom &g, const T *f, int nshots, unsigned *flags,
                                cudaStream_t st) {
    k_check_finite<T><<<1216, 256, 0, st>>>(f, (long long)nshots * g.fstride, flags);
    return cudaGetLastError();
}

#define INST(T)                                                                             \
    template cudaError_t launch_setup_model<T>(const Geom &, const T *, T *, T *, double,   \
                                               cudaStream_t);                               \
    template cudaError_t launch_minmax<T>(const Geom &, const T *, double *, cudaStream_t); \
    template cudaError_t launch_check_finite<T>(const Geom &, const T *, int, unsigned *,   \
                                                cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace gsim
