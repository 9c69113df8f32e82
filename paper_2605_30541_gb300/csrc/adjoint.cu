// Support kernels of the adjoint-state gradient: checkpoint store/restore
// (FP32/FP64 copy or FP16 with a power-of-two scale per tile; the CPML
// memory of an axis only on the boxes of its strips, where it can be
// non-zero, with a scale per row), the data
// residual with its misfit, and the final FP64 fold of the per-shot imaging
// sums onto the interior velocity cells (absorbing cells replicate the
// nearest interior cell, so their contributions land on the edge cells).
#include <cfloat>

#include "sim_internal.h"
#include "stencil.cuh"

namespace gsim {
namespace {

constexpr int TX = kTileX2, TZ = kTileZ2, BX = 32, BY = 8, RZ = TZ / BY, NTH = BX * BY;

__device__ __forceinline__ float tile_max(float v, float *red) {
    const int tid = threadIdx.y * BX + threadIdx.x;
    v = warp_max(v);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    float m = tid < NTH / 32 ? red[tid & 31] : 0.f;
    if (tid < 32) m = warp_max(m);
    __syncthreads();
    if (tid == 0) red[0] = m;
    __syncthreads();
    return red[0];
}

// Rows of the computational grid: r = z NY + y (r = z in 2D), NZ NY rows of NX cells.
__device__ __forceinline__ long long row_off(const Geom &g, int r, int x) {
    return cell_off(g, r / g.NY, r % g.NY, x);
}

// One CTA per (tile of rows x columns, shot); the compact copy of a state is
// [shot][NZ NY NX].
template <typename T>
__global__ void __launch_bounds__(NTH) k_store(const Geom g, const T *__restrict__ field, void *dst, float *scale,
                                               int fp16, long long sstride, int ntx) {
    __shared__ float red[NTH / 32];
    const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ, shot = blockIdx.z, nrow = g.NZ * g.NY;
    const int tile = blockIdx.y * ntx + blockIdx.x, ntiles = ntx * gridDim.y;
    const T *f = field + (long long)shot * g.fstride;
    T v[RZ];
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < RZ; k++) {
        const int gz = z0 + threadIdx.y + k * BY, gx = x0 + threadIdx.x;
        v[k] = (gz < nrow && gx < g.NX) ? f[row_off(g, gz, gx)] : T(0);
        m = fmaxf(m, fabsf((float)v[k]));
    }
    float inv = 1.f;
    if (fp16) {
        const float s = pow2_scale(tile_max(m, red));
        inv = 1.f / s;
        if (threadIdx.x == 0 && threadIdx.y == 0) scale[(long long)shot * ntiles + tile] = s;
    }
#pragma unroll
    for (int k = 0; k < RZ; k++) {
        const int gz = z0 + threadIdx.y + k * BY, gx = x0 + threadIdx.x;
        if (gz >= nrow || gx >= g.NX) continue;
        const long long ci = shot * sstride + (long long)gz * g.NX + gx;
        if (fp16) static_cast<__half *>(dst)[ci] = __float2half_rn((float)v[k] * inv);
        else static_cast<T *>(dst)[ci] = v[k];
    }
}

template <typename T>
__global__ void __launch_bounds__(NTH) k_load(const Geom g, T *field, const void *src, const float *scale, int fp16,
                                              long long sstride, int ntx) {
    const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ, shot = blockIdx.z, nrow = g.NZ * g.NY;
    const int tile = blockIdx.y * ntx + blockIdx.x, ntiles = ntx * gridDim.y;
    T *f = field + (long long)shot * g.fstride;
    const float s = fp16 ? scale[(long long)shot * ntiles + tile] : 1.f;
#pragma unroll
    for (int k = 0; k < RZ; k++) {
        const int gz = z0 + threadIdx.y + k * BY, gx = x0 + threadIdx.x;
        if (gz >= nrow || gx >= g.NX) continue;
        const long long ci = shot * sstride + (long long)gz * g.NX + gx;
        f[row_off(g, gz, gx)] =
            fp16 ? T(__half2float(static_cast<const __half *>(src)[ci]) * s) : static_cast<const T *>(src)[ci];
    }
}

// Boxes of the computational grid (the CPML strips of one axis): one warp per
// (row of a box, shot). A box row is the x run [x0, x1) at one (z, y); the
// compact copy is [shot][rows of box 0, box 1, ...][x] and, in FP16, carries
// one power-of-two scale per (shot, row).
__device__ __forceinline__ int box_of(const CkBoxes &B, long long r) {
    int k = 0;
    while (k + 1 < B.n && B.row0[k + 1] <= r) k++;
    return k;
}

template <typename T, bool STORE>
__global__ void __launch_bounds__(256) k_boxes(const Geom g, const CkBoxes B, T *field, void *cmp, float *scale,
                                               int fp16, int nshots) {
    const int lane = threadIdx.x & 31;
    const long long rows = B.row0[B.n];
    const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (w >= rows * nshots) return;
    const int shot = (int)(w / rows);
    const long long r = w - (long long)shot * rows;
    const int k = box_of(B, r);
    const CkBox &b = B.b[k];
    const long long lr = r - B.row0[k];
    const int ny = b.y1 - b.y0, len = b.x1 - b.x0;
    const int z = b.z0 + (int)(lr / ny), y = b.y0 + (int)(lr % ny);
    T *f = field + (long long)shot * g.fstride + cell_off(g, z, y, b.x0);
    const long long e0 = (long long)shot * B.elem0[B.n] + B.elem0[k] + lr * len;
    const long long si = (long long)shot * rows + r;
    if (STORE) {
        float inv = 1.f;
        if (fp16) {
            float m = 0.f;
            for (int i = lane; i < len; i += 32) m = fmaxf(m, fabsf((float)f[i]));
            const float sc = pow2_scale(warp_max(m));
            inv = 1.f / sc;
            if (lane == 0) scale[si] = sc;
        }
        for (int i = lane; i < len; i += 32) {
            if (fp16) static_cast<__half *>(cmp)[e0 + i] = __float2half_rn((float)f[i] * inv);
            else static_cast<T *>(cmp)[e0 + i] = f[i];
        }
    } else {
        const float sc = fp16 ? scale[si] : 1.f;
        for (int i = lane; i < len; i += 32)
            f[i] = fp16 ? T(__half2float(static_cast<const __half *>(cmp)[e0 + i]) * sc) : static_cast<const T *>(cmp)[e0 + i];
    }
}

template <typename T>
__global__ void k_residual(const T *__restrict__ gath, const T *__restrict__ d, T *res, long long n, double *part) {
    __shared__ double sm[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T r = gath[i] - d[i];
        res[i] = r;
        acc += 0.5 * (double)r * (double)r;
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// Interior cell i gathers every computational cell whose velocity copies it:
// itself, plus the absorbing cells beyond it when it sits on an edge. Per
// cell, the shots' imaging terms are summed first and then scaled by
// -2 / (h^2 v) (one FP64 division per cell, not per cell and shot: FP64
// division is slow on this part, and the edge cells fold whole absorbing
// rows, columns or corner blocks serially).
template <typename T>
__global__ void k_fold(const Geom g, const T *__restrict__ G, long long gshot, int nshots,
                       const T *__restrict__ vpad, double inv_h2, double *acc) {
    const long long nint = (long long)g.nz * g.ny * g.nx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nint; i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % g.nx);
        const long long zy = i / g.nx;
        const int iy = (int)(zy % g.ny), iz = (int)(zy / g.ny);
        const int za = iz == 0 ? 0 : iz + g.oz, zb = iz == g.nz - 1 ? g.NZ : iz + g.oz + 1;
        const int ya = iy == 0 ? 0 : iy + g.oy, yb = iy == g.ny - 1 ? g.NY : iy + g.oy + 1;
        const int xa = ix == 0 ? 0 : ix + g.ox, xb = ix == g.nx - 1 ? g.NX : ix + g.ox + 1;
        double sum = 0.0;
        for (int z = za; z < zb; z++)
            for (int y = ya; y < yb; y++)
                for (int x = xa; x < xb; x++) {
                    const long long o = cell_off(g, z, y, x);
                    double gs = 0.0;
                    for (int s = 0; s < nshots; s++) gs += (double)G[s * gshot + o];
                    sum += -2.0 * inv_h2 / (double)vpad[o] * gs;
                }
        acc[i] += sum;
    }
}

template <typename T>
__global__ void k_add(const double *__restrict__ acc, T *grad, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        grad[i] += (T)acc[i];
}

}  // namespace

template <typename T>
cudaError_t launch_store_state(const Geom &g, const T *field, void *dst, float *scale, int fp16, int nshots,
                               long long shot_stride, int ntx, int ntz, cudaStream_t st) {
    k_store<T><<<dim3(ntx, ntz, nshots), dim3(BX, BY), 0, st>>>(g, field, dst, scale, fp16, shot_stride, ntx);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_load_state(const Geom &g, T *field, const void *src, const float *scale, int fp16, int nshots,
                              long long shot_stride, int ntx, int ntz, cudaStream_t st) {
    k_load<T><<<dim3(ntx, ntz, nshots), dim3(BX, BY), 0, st>>>(g, field, src, scale, fp16, shot_stride, ntx);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_store_boxes(const Geom &g, const CkBoxes &b, const T *field, void *dst, float *scale, int fp16,
                               int nshots, cudaStream_t st) {
    const long long warps = b.row0[b.n] * nshots;
    if (warps == 0) return cudaSuccess;
    k_boxes<T, true><<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(g, b, const_cast<T *>(field), dst, scale, fp16,
                                                                  nshots);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_load_boxes(const Geom &g, const CkBoxes &b, T *field, const void *src, const float *scale,
                              int fp16, int nshots, cudaStream_t st) {
    const long long warps = b.row0[b.n] * nshots;
    if (warps == 0) return cudaSuccess;
    k_boxes<T, false><<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(g, b, field, const_cast<void *>(src),
                                                                   const_cast<float *>(scale), fp16, nshots);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual(const T *g, const T *d, T *res, long long n, double *part, int nblocks, cudaStream_t st) {
    k_residual<T><<<nblocks, 256, 0, st>>>(g, d, res, n, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fold_gradient(const Geom &g, const T *G, long long gshot, int nshots, const T *vpad,
                                 double inv_h2, double *acc, cudaStream_t st) {
    k_fold<T><<<1216, 256, 0, st>>>(g, G, gshot, nshots, vpad, inv_h2, acc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_add_gradient(const double *acc, T *grad, long long n, cudaStream_t st) {
    k_add<T><<<1216, 256, 0, st>>>(acc, grad, n);
    return cudaGetLastError();
}

#define INST(T)                                                                                               \
    template cudaError_t launch_store_state<T>(const Geom &, const T *, void *, float *, int, int, long long,  \
                                               int, int, cudaStream_t);                                       \
    template cudaError_t launch_load_state<T>(const Geom &, T *, const void *, const float *, int, int,        \
                                              long long, int, int, cudaStream_t);                             \
    template cudaError_t launch_store_boxes<T>(const Geom &, const CkBoxes &, const T *, void *, float *, int, int, \
                                               cudaStream_t);                                                \
    template cudaError_t launch_load_boxes<T>(const Geom &, const CkBoxes &, T *, const void *, const float *, int, \
                                              int, cudaStream_t);                                            \
    template cudaError_t launch_residual<T>(const T *, const T *, T *, long long, double *, int, cudaStream_t); \
    template cudaError_t launch_fold_gradient<T>(const Geom &, const T *, long long, int, const T *,      \
                                                 double, double *, cudaStream_t);                             \
    template cudaError_t launch_add_gradient<T>(const double *, T *, long long, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace gsim
