// CPML terms of the adjoint sweep (2D: FP32 or FP64; 3D: FP32): the exact
// transpose of the forward CPML recursions, in the scaled variables of the
// step kernels (psi ~ h psi, zeta ~ h^2 zeta, unscaled stencils D1 / D2,
// c = (v dt / h)^2), per absorbing axis:
//   psi^n  = b psi^{n-1}  + a D1 p^n
//   zeta^n = b zeta^{n-1} + a (D2 p^n + D1 psi^n),  addend D1 psi^n + zeta^n.
// With the adjoint field u = c lambda and multipliers nu (of zeta) and mu (of
// psi), zero after the last step, step k of the sweep is
//   nu^k = b nu^{k+1} + u^{k+1}
//   mu^k = b mu^{k+1} - D1 (u^{k+1} + a nu^k)
//   u^k  = (the sponge-free update of u) + c [-D1 (a mu^k) + D2 (a nu^k)]
// (D1^T = -D1 and D2^T = D2 on the zero-ghost grid; a free surface never
// meets a z strip, so its odd mirror does not enter). Pass A updates nu and
// mu on the strip cells of each absorbing axis; pass B forms the bracket,
// summed over the axes, on the cells within 4 of a strip. In 2D it goes to
// `ext`, which the step kernel adds to the Laplacian of u^{k+1}; in 3D pass B
// runs after the update and adds c times the bracket to u^k itself and, as
// the update kernel does for the rest of u^k, its product with the recorded
// imaging term to G. a = b = 0 outside the strips, so nu and mu matter only
// there and the bracket vanishes beyond 4 cells from them.
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
    } else if (ax == 1) {
        v.N = g.NY;
        v.lo = g.nby0;
        v.hi = g.nby1;
        v.stride = g.P;
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

// The launch covers the union of the strips (widened by a margin) as up to 6
// disjoint boxes: the top and bottom z bands over all (y, x), then in the z
// range between them the low and high y bands over all x, then in the (z, y)
// range between those the low and high x bands; thread i -> (box, z, y, x),
// x fastest, then y.
struct Boxes {
    int n;
    int z0[6], z1[6], y0[6], y1[6], x0[6], x1[6];
    long long start[7];
};

__device__ __forceinline__ bool box_cell(const Boxes &B, long long i, int &z, int &y, int &x) {
    if (i >= B.start[B.n]) return false;
    int b = 0;
    while (b + 1 < B.n && B.start[b + 1] <= i) b++;
    const long long r = i - B.start[b];
    const int w = B.x1[b] - B.x0[b], h = B.y1[b] - B.y0[b];
    const long long t = r / w;
    x = B.x0[b] + (int)(r - t * w);
    y = B.y0[b] + (int)(t % h);
    z = B.z0[b] + (int)(t / h);
    return true;
}

// pass A: nu_new, mu (in place) on the strip cells of every absorbing axis
template <typename T>
__global__ void k_cpml_adj_a(const StepArgs<T> A, CpmlAdjArgs<T> C, int parity, const Boxes B) {
    const Geom &g = A.g;
    const int shot = blockIdx.y;
    int z, y, x;
    if (!box_cell(B, blockIdx.x * (long long)blockDim.x + threadIdx.x, z, y, x)) return;
    const long long o = (long long)shot * g.fstride + cell_off(g, z, y, x);
    const T *u = C.u;
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        if (!A.ca[ax]) continue;
        const AxisView<T> v = axis_view(A, ax);
        const int q = ax == 0 ? z : (ax == 1 ? y : x);
        if (!in_strip(v, q, 0)) continue;
        const T *nuo = C.nu[ax][parity ^ 1];
        T *nun = C.nu[ax][parity];
        T *mu = C.mu[ax];
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

// pass B: the sum over the axes of -D1 (a mu) + D2 (a nu) on the cells
// within 4 of a strip, into ext (C.uo == NULL) or, times c, into u^k (and
// its product with the imaging term into G)
template <typename T>
__global__ void k_cpml_adj_b(const StepArgs<T> A, CpmlAdjArgs<T> C, int parity, const Boxes B) {
    const Geom &g = A.g;
    const int shot = blockIdx.y;
    int z, y, x;
    if (!box_cell(B, blockIdx.x * (long long)blockDim.x + threadIdx.x, z, y, x)) return;
    const long long cell = cell_off(g, z, y, x), o = (long long)shot * g.fstride + cell;
    T ext = T(0);
    bool near = false;
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        if (!A.ca[ax]) continue;
        const AxisView<T> v = axis_view(A, ax);
        const int q = ax == 0 ? z : (ax == 1 ? y : x);
        if (!in_strip(v, q, 4)) continue;
        near = true;
        const T *nu = C.nu[ax][parity], *mu = C.mu[ax];
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
    if (!near) return;
    if (!C.uo) {
        C.ext[o] = ext;
    } else if (!(g.fs && z == 0)) {  // the free-surface row of u stays zero
        const T du = A.ch[cell] * ext;
        C.uo[o] += du;
        C.G[o] += du * C.q[o];
    }
}

// the strips of the active axes widened by `margin`, as disjoint boxes
template <typename T>
Boxes strip_boxes(const StepArgs<T> &a, int margin) {
    const Geom &g = a.g;
    const int N[3] = {g.NZ, g.NY, g.NX};
    const int lo[3] = {g.nbz0, g.nby0, g.nbx0}, hi[3] = {g.nbz1, g.nby1, g.nbx1};
    int b0[3], b1[3];  // per axis: [0, b0) and [b1, N) are the widened strips
    for (int ax = 0; ax < 3; ax++) {
        const bool on = a.ca[ax] != nullptr;
        b0[ax] = on && lo[ax] > 0 ? std::min(N[ax], lo[ax] + margin) : 0;
        b1[ax] = on && hi[ax] > 0 ? std::max(b0[ax], N[ax] - hi[ax] - margin) : N[ax];
    }
    Boxes B{};
    auto add = [&](int z0, int z1, int y0, int y1, int x0, int x1) {
        if (z1 <= z0 || y1 <= y0 || x1 <= x0) return;
        B.z0[B.n] = z0;
        B.z1[B.n] = z1;
        B.y0[B.n] = y0;
        B.y1[B.n] = y1;
        B.x0[B.n] = x0;
        B.x1[B.n] = x1;
        B.start[B.n + 1] = B.start[B.n] + (long long)(z1 - z0) * (y1 - y0) * (x1 - x0);
        B.n++;
    };
    add(0, b0[0], 0, N[1], 0, N[2]);
    add(b1[0], N[0], 0, N[1], 0, N[2]);
    add(b0[0], b1[0], 0, b0[1], 0, N[2]);
    add(b0[0], b1[0], b1[1], N[1], 0, N[2]);
    add(b0[0], b1[0], b0[1], b1[1], 0, b0[2]);
    add(b0[0], b1[0], b0[1], b1[1], b1[2], N[2]);
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
