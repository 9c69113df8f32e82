// CPML terms of the 2D adjoint sweep (FP32): the exact transpose of the
// forward CPML recursions of the step kernels, in their scaled variables
// (psi ~ h psi, zeta ~ h^2 zeta, unscaled stencils D1 / D2, c = (v dt / h)^2):
//   psi^n  = b psi^{n-1}  + a D1 p^n
//   zeta^n = b zeta^{n-1} + a (D2 p^n + D1 psi^n),  addend D1 psi^n + zeta^n.
// With the adjoint field u = c lambda and multipliers nu (of zeta) and mu (of
// psi), zero after the last step, step k of the sweep is
//   nu^k = b nu^{k+1} + u^{k+1}
//   mu^k = b mu^{k+1} - D1 (u^{k+1} + a nu^k)
//   u^k  = (the sponge-free update of u) + c [-D1 (a mu^k) + D2 (a nu^k)]
// (D1^T = -D1 and D2^T = D2 on the zero-ghost grid; a free surface never
// meets a z strip, so its odd mirror does not enter). Pass A updates nu and
// mu on the strip cells of each absorbing axis; pass B writes the bracket,
// summed over the axes, on the cells within 4 of a strip into `ext`, which
// the step kernel adds to the Laplacian of u^{k+1}. a = b = 0 outside the
// strips, so nu and mu matter only there and the bracket vanishes beyond 4
// cells from them.
#include "sim_internal.h"
#include "stencil.cuh"

namespace gsim {
namespace {

struct AxisView {
    const float *a, *b;  // profile of the axis (zero margins beyond the grid)
    int N, lo, hi;       // extent and strip widths
    long long stride;    // field elements per step along the axis
};

__device__ __forceinline__ AxisView axis_view(const StepArgs<float> &A, int ax) {
    const Geom &g = A.g;
    AxisView v;
    v.a = A.ca[ax];
    v.b = A.cb[ax];
    if (ax == 0) {
        v.N = g.NZ;
        v.lo = g.nbz0;
        v.hi = g.nbz1;
        v.stride = (long long)g.PY * g.P;
    } else {
        v.N = g.NX;
        v.lo = g.nbx0;
        v.hi = g.nbx1;
        v.stride = 1;
    }
    return v;
}

__device__ __forceinline__ bool in_strip(const AxisView &v, int q, int margin) {
    return (v.lo > 0 && q < v.lo + margin) || (v.hi > 0 && q >= v.N - v.hi - margin);
}

// pass A: nu_new, mu (in place) on the strip cells of axes z (0) and x (2)
__global__ void k_cpml_adj_a(const StepArgs<float> A, CpmlAdjArgs C, int parity) {
    const Geom &g = A.g;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, z = blockIdx.y, shot = blockIdx.z;
    if (x >= g.NX) return;
    const long long o = (long long)shot * g.fstride + cell_off(g, z, 0, x);
    const float *u = C.u;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int ax = k == 0 ? 0 : 2;
        if (!A.ca[ax]) continue;
        const AxisView v = axis_view(A, ax);
        const int q = ax == 0 ? z : x;
        if (!in_strip(v, q, 0)) continue;
        const float *nuo = C.nu[k][parity ^ 1];
        float *nun = C.nu[k][parity];
        float *mu = C.mu[k];
        nun[o] = v.b[q] * nuo[o] + u[o];
        // D1 of w = u + a (b nu_old + u) = u + a nu_new, at the neighbours along the axis
        float d1 = 0.f;
#pragma unroll
        for (int m = 1; m <= 4; m++) {
            const long long op = o + m * v.stride, om = o - m * v.stride;
            const float wp = u[op] + v.a[q + m] * (v.b[q + m] * nuo[op] + u[op]);
            const float wm = u[om] + v.a[q - m] * (v.b[q - m] * nuo[om] + u[om]);
            const float dm = m == 1 ? float(kD1) : (m == 2 ? float(kD2) : (m == 3 ? float(kD3) : float(kD4)));
            d1 += dm * (wp - wm);
        }
        mu[o] = v.b[q] * mu[o] - d1;
    }
}

// pass B: ext = sum over the axes of -D1 (a mu) + D2 (a nu) on the cells
// within 4 of a strip
__global__ void k_cpml_adj_b(const StepArgs<float> A, CpmlAdjArgs C, int parity) {
    const Geom &g = A.g;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, z = blockIdx.y, shot = blockIdx.z;
    if (x >= g.NX) return;
    const long long o = (long long)shot * g.fstride + cell_off(g, z, 0, x);
    float ext = 0.f;
    bool near = false;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int ax = k == 0 ? 0 : 2;
        if (!A.ca[ax]) continue;
        const AxisView v = axis_view(A, ax);
        const int q = ax == 0 ? z : x;
        if (!in_strip(v, q, 4)) continue;
        near = true;
        const float *nu = C.nu[k][parity], *mu = C.mu[k];
        float d1 = 0.f, d2 = float(kC0) * v.a[q] * nu[o];
#pragma unroll
        for (int m = 1; m <= 4; m++) {
            const long long op = o + m * v.stride, om = o - m * v.stride;
            const float dm = m == 1 ? float(kD1) : (m == 2 ? float(kD2) : (m == 3 ? float(kD3) : float(kD4)));
            const float cm = m == 1 ? float(kC1) : (m == 2 ? float(kC2) : (m == 3 ? float(kC3) : float(kC4)));
            d1 += dm * (v.a[q + m] * mu[op] - v.a[q - m] * mu[om]);
            d2 += cm * (v.a[q + m] * nu[op] + v.a[q - m] * nu[om]);
        }
        ext += d2 - d1;
    }
    if (near) C.ext[o] = ext;
}

}  // namespace

cudaError_t launch_cpml_adjoint(const StepArgs<float> &a, const CpmlAdjArgs &c, int parity, int nshots,
                                cudaStream_t st) {
    const dim3 grid((a.g.NX + 127) / 128, a.g.NZ, nshots);
    k_cpml_adj_a<<<grid, 128, 0, st>>>(a, c, parity);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_cpml_adj_b<<<grid, 128, 0, st>>>(a, c, parity);
    return cudaGetLastError();
}

}  // namespace gsim
