// CPML terms of the 2D adjoint sweep (FP32 or FP64): the exact transpose of the
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
#include <algorithm>

#include "sim_internal.h"
#include "stencil.cuh"

namespace gsim {
namespace {

template <typename T>
struct AxisView {
    const T *a, *b;      // profile of the axis (zero margins beyond the grid)
    int N, lo, hi;       // extent and strip widths
    long long stride;    // field elements per step along the axis
};

template <typename T>
__device__ __forceinline__ AxisView<T> axis_view(const StepArgs<T> &A, int ax) {
    const Geom &g = A.g;
    AxisView<T> v;
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

template <typename T>
__device__ __forceinline__ bool in_strip(const AxisView<T> &v, int q, int margin) {
    return (v.lo > 0 && q < v.lo + margin) || (v.hi > 0 && q >= v.N - v.hi - margin);
}

// The launch covers the union of the strips (widened by a margin) as up to 4
// disjoint boxes: the top and bottom row bands over the full width, then the
// left and right column bands of the rows between; thread i -> (box, z, x),
// x fastest.
struct Boxes {
    int n;
    int z0[4], z1[4], x0[4], x1[4];
    long long start[5];
};

__device__ __forceinline__ bool box_cell(const Boxes &B, long long i, int &z, int &x) {
    if (i >= B.start[B.n]) return false;
    int b = 0;
    while (b + 1 < B.n && B.start[b + 1] <= i) b++;
    const long long r = i - B.start[b];
    const int w = B.x1[b] - B.x0[b];
    z = B.z0[b] + (int)(r / w);
    x = B.x0[b] + (int)(r % w);
    return true;
}

// pass A: nu_new, mu (in place) on the strip cells of axes z (0) and x (2)
template <typename T>
__global__ void k_cpml_adj_a(const StepArgs<T> A, CpmlAdjArgs<T> C, int parity, const Boxes B) {
    const Geom &g = A.g;
    const int shot = blockIdx.y;
    int z, x;
    if (!box_cell(B, blockIdx.x * (long long)blockDim.x + threadIdx.x, z, x)) return;
    const long long o = (long long)shot * g.fstride + cell_off(g, z, 0, x);
    const T *u = C.u;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int ax = k == 0 ? 0 : 2;
        if (!A.ca[ax]) continue;
        const AxisView<T> v = axis_view(A, ax);
        const int q = ax == 0 ? z : x;
        if (!in_strip(v, q, 0)) continue;
        const T *nuo = C.nu[k][parity ^ 1];
        T *nun = C.nu[k][parity];
        T *mu = C.mu[k];
        nun[o] = v.b[q] * nuo[o] + u[o];
        // D1 of w = u + a (b nu_old + u) = u + a nu_new, at the neighbours along the axis
        T d1 = T(0);
#pragma unroll
        for (int m = 1; m <= 4; m++) {
            const long long op = o + m * v.stride, om = o - m * v.stride;
            const T wp = u[op] + v.a[q + m] * (v.b[q + m] * nuo[op] + u[op]);
            const T wm = u[om] + v.a[q - m] * (v.b[q - m] * nuo[om] + u[om]);
            const T dm = m == 1 ? T(kD1) : (m == 2 ? T(kD2) : (m == 3 ? T(kD3) : T(kD4)));
            d1 += dm * (wp - wm);
        }
        mu[o] = v.b[q] * mu[o] - d1;
    }
}

// pass B: ext = sum over the axes of -D1 (a mu) + D2 (a nu) on the cells
// within 4 of a strip
template <typename T>
__global__ void k_cpml_adj_b(const StepArgs<T> A, CpmlAdjArgs<T> C, int parity, const Boxes B) {
    const Geom &g = A.g;
    const int shot = blockIdx.y;
    int z, x;
    if (!box_cell(B, blockIdx.x * (long long)blockDim.x + threadIdx.x, z, x)) return;
    const long long o = (long long)shot * g.fstride + cell_off(g, z, 0, x);
    T ext = T(0);
    bool near = false;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int ax = k == 0 ? 0 : 2;
        if (!A.ca[ax]) continue;
        const AxisView<T> v = axis_view(A, ax);
        const int q = ax == 0 ? z : x;
        if (!in_strip(v, q, 4)) continue;
        near = true;
        const T *nu = C.nu[k][parity], *mu = C.mu[k];
        T d1 = T(0), d2 = T(kC0) * v.a[q] * nu[o];
#pragma unroll
        for (int m = 1; m <= 4; m++) {
            const long long op = o + m * v.stride, om = o - m * v.stride;
            const T dm = m == 1 ? T(kD1) : (m == 2 ? T(kD2) : (m == 3 ? T(kD3) : T(kD4)));
            const T cm = m == 1 ? T(kC1) : (m == 2 ? T(kC2) : (m == 3 ? T(kC3) : T(kC4)));
            d1 += dm * (v.a[q + m] * mu[op] - v.a[q - m] * mu[om]);
            d2 += cm * (v.a[q + m] * nu[op] + v.a[q - m] * nu[om]);
        }
        ext += d2 - d1;
    }
    if (near) C.ext[o] = ext;
}

}  // namespace

namespace {
// the strips of the active axes widened by `margin`, as disjoint boxes
template <typename T>
Boxes strip_boxes(const StepArgs<T> &a, int margin) {
    const Geom &g = a.g;
    const bool zon = a.ca[0] != nullptr, xon = a.ca[2] != nullptr;
    const int zt = zon && g.nbz0 > 0 ? std::min(g.NZ, g.nbz0 + margin) : 0;
    const int zb = zon && g.nbz1 > 0 ? std::max(zt, g.NZ - g.nbz1 - margin) : g.NZ;
    const int xl = xon && g.nbx0 > 0 ? std::min(g.NX, g.nbx0 + margin) : 0;
    const int xr = xon && g.nbx1 > 0 ? std::max(xl, g.NX - g.nbx1 - margin) : g.NX;
    Boxes B{};
    auto add = [&](int z0, int z1, int x0, int x1) {
        if (z1 <= z0 || x1 <= x0) return;
        B.z0[B.n] = z0;
        B.z1[B.n] = z1;
        B.x0[B.n] = x0;
        B.x1[B.n] = x1;
        B.start[B.n + 1] = B.start[B.n] + (long long)(z1 - z0) * (x1 - x0);
        B.n++;
    };
    add(0, zt, 0, g.NX);
    add(zb, g.NZ, 0, g.NX);
    add(zt, zb, 0, xl);
    add(zt, zb, xr, g.NX);
    return B;
}
}  // namespace

template <typename T>
cudaError_t launch_cpml_adjoint(const StepArgs<T> &a, const CpmlAdjArgs<T> &c, int parity, int nshots,
                                cudaStream_t st) {
    const Boxes ba = strip_boxes(a, 0), bb = strip_boxes(a, 4);
    if (ba.n > 0) {
        k_cpml_adj_a<T><<<dim3((unsigned)((ba.start[ba.n] + 127) / 128), nshots), 128, 0, st>>>(a, c, parity, ba);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (bb.n > 0)
        k_cpml_adj_b<T><<<dim3((unsigned)((bb.start[bb.n] + 127) / 128), nshots), 128, 0, st>>>(a, c, parity, bb);
    return cudaGetLastError();
}

template cudaError_t launch_cpml_adjoint<float>(const StepArgs<float> &, const CpmlAdjArgs<float> &, int, int,
                                                cudaStream_t);
template cudaError_t launch_cpml_adjoint<double>(const StepArgs<double> &, const CpmlAdjArgs<double> &, int, int,
                                                 cudaStream_t);

}  // namespace gsim
