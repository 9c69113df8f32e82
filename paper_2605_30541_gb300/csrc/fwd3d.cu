// 3D time step of the acoustic scheme (FP32).
//
// Main kernel: a z-march over (x, y) tiles (2.5D blocking). A CTA of 8 warps
// owns a 128 x TY column of the grid (TY = 8 RY); each lane owns 4
// consecutive x cells in RY y-rows and keeps the 9 planes z-4 .. z+4 of those
// cells in a register queue, so p^n is read from memory once per cell for the
// z-derivative. The planes with their radius-4 x/y halo are staged into a
// shared-memory ring ahead of use: by per-thread cp.async copies (k_step3d)
// or by tensor-memory-accelerator copies that one thread issues (k_step3d_tma,
// the autotuner's usual pick). The update is the leapfrog step with the
// centred sponge term (Eq. cerjan_pde), the free-surface plane z = 0 held at
// zero with an odd mirror above it (Eq. free_surface), and no boundary
// arithmetic outside absorbing tiles.
//
// Side kernels of a step touch only small parts of the grid: the CPML memory
// terms of each axis (one pass after the update on its strips: psi, zeta and
// the D1 psi + zeta addend), point injection of the source, trilinear
// receiver sampling and snapshot output.
#include <cfloat>

#include <cudaTypedefs.h>

#include "sim_internal.h"
#include "stencil.cuh"

namespace gsim {
namespace {

constexpr int TX = kTileXF, NW = 8, NTH = NW * 32, SW3 = TX + 8;

__device__ __forceinline__ float lane4(const float4 &v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}
__device__ __forceinline__ float4 ld4g(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// The four cells of one thread at one plane: x window L, C, R (C the cells),
// the nine y rows yv (yv[4] = C) and the nine z planes z0..z8 (z4 = C) of
// p^n. The second differences run in cell pairs (0, 1) and (2, 3) with the
// pair arithmetic, in d2c's order of roundings; rhs = D2x + D2y + D2z. The
// plain update p^{n+1} = 2 p - p^{n-1} + c rhs is fma(c, rhs, fma(2, p,
// -p^{n-1})), also in pairs; the sponge update (Eq. cerjan_pde) runs per
// cell. Both z-marches call this, so they give the same bits.
struct Cells4 {
    float res[4], rhs[4], d2x[4];
};
__device__ __forceinline__ Cells4 cells4(const float4 &L, const float4 &C, const float4 &R, const float4 (&yv)[9],
                                         const float4 &z0, const float4 &z1, const float4 &z2, const float4 &z3,
                                         const float4 &z5, const float4 &z6, const float4 &z7, const float4 &z8,
                                         const float4 &pp4, const float4 &ch4, bool spg, float es0,
                                         const float4 &Ex4) {
    // x: pairs of the 12-float window; (v3, v4), (v5, v6), (v1, v2), (v7, v8), (v9, v10) straddle float4s
    const float2 v34 = make_float2(L.w, C.x), v56 = make_float2(C.y, C.z), v12 = make_float2(L.y, L.z),
                 v78 = make_float2(C.w, R.x), v910 = make_float2(R.y, R.z);
    const float2 xa = d2c2(lo2(C), v34, v56, hi2(L), hi2(C), v12, v78, lo2(L), lo2(R));
    const float2 xb = d2c2(hi2(C), v56, v78, lo2(C), lo2(R), v34, v910, hi2(L), hi2(R));
    const float2 ya = d2c2(lo2(C), lo2(yv[3]), lo2(yv[5]), lo2(yv[2]), lo2(yv[6]), lo2(yv[1]), lo2(yv[7]),
                           lo2(yv[0]), lo2(yv[8]));
    const float2 yb = d2c2(hi2(C), hi2(yv[3]), hi2(yv[5]), hi2(yv[2]), hi2(yv[6]), hi2(yv[1]), hi2(yv[7]),
                           hi2(yv[0]), hi2(yv[8]));
    const float2 za = d2c2(lo2(C), lo2(z3), lo2(z5), lo2(z2), lo2(z6), lo2(z1), lo2(z7), lo2(z0), lo2(z8));
    const float2 zb = d2c2(hi2(C), hi2(z3), hi2(z5), hi2(z2), hi2(z6), hi2(z1), hi2(z7), hi2(z0), hi2(z8));
    const float2 ra = add2(add2(xa, ya), za), rb = add2(add2(xb, yb), zb);
    Cells4 o;
    o.d2x[0] = xa.x, o.d2x[1] = xa.y, o.d2x[2] = xb.x, o.d2x[3] = xb.y;
    o.rhs[0] = ra.x, o.rhs[1] = ra.y, o.rhs[2] = rb.x, o.rhs[3] = rb.y;
    if (!spg) {
        const float2 two = splat2(2.f);
        const float2 oa = fma2(lo2(ch4), ra, fma2(two, lo2(C), neg2(lo2(pp4))));
        const float2 ob = fma2(hi2(ch4), rb, fma2(two, hi2(C), neg2(hi2(pp4))));
        o.res[0] = oa.x, o.res[1] = oa.y, o.res[2] = ob.x, o.res[3] = ob.y;
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float p = lane4(C, k), chv = lane4(ch4, k), pp = lane4(pp4, k);
            const float a = chv * (es0 + lane4(Ex4, k));
            o.res[k] = (2.f * p - (1.f - a) * pp + chv * o.rhs[k]) / (1.f + a);
        }
    }
    return o;
}
__device__ __forceinline__ void cp16(void *smem, const void *gmem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
// 16-byte copy that writes zeros (reads nothing) when v is false
__device__ __forceinline__ void cp16z(unsigned dst, const void *gmem, bool v) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(gmem), "r"(v ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Staged planes in flight: while plane z is computed, planes z+1 .. z+4 are
// ready or arriving and plane z+5 is being requested. A ring slot holds the
// plane's p^n with its x/y halo, and p^{n-1} and c of the CTA's own cells;
// the register queue takes plane z+4's own cells from its slot, so after the
// prologue every global read of the march is a cp.async issued five planes
// ahead of its use.
constexpr int NS3 = 6;
template <int RY>
constexpr int slot3d() {
    return (NW * RY + 8) * SW3 + 2 * NW * RY * TX;
}

// MODE (kModeForward / kModeRecord / kModeAdjoint) as in the 2D kernel: the
// record sweep also writes the imaging term Q'^n = E (p^{n+1} - p^{n-1}) -
// h^2 L p^n of each cell to qs (the source's share is added by the injection
// kernel), the adjoint sweep adds u^{n+1} Q'^n, read from qs, to Gs.
template <int RY, int MODE>
__global__ void __launch_bounds__(NTH, 2) k_step3d(const StepArgs<float> A, const int n, const int zchunk,
                                                   float *qs, float *Gs) {
    constexpr int TY = NW * RY, NR = TY + 8;  // staged rows per plane
    constexpr int SLOT = slot3d<RY>();
    extern __shared__ float4 sm3[];
    float *const ring = reinterpret_cast<float *>(sm3);

    const Geom &g = A.g;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nchunk = (g.NZ + zchunk - 1) / zchunk;
    const int shot = blockIdx.z / nchunk, zb = (blockIdx.z % nchunk) * zchunk;
    const int ze = min(zb + zchunk, g.NZ);
    const long long PP = (long long)g.PY * g.P;  // plane pitch
    const long long sh = (long long)shot * g.fstride;
    const float *pc = A.pbuf[n & 1] + sh;
    float *pn = A.pbuf[(n + 1) & 1] + sh;
    const int gx0 = x0 + 4 * lane;
    const bool xedge = x0 + TX > g.NX;
    const bool spg = A.bc == SIM_BC_SPONGE &&
                     ((g.nbx0 > 0 && x0 < g.nbx0) || (g.nbx1 > 0 && x0 + TX > g.NX - g.nbx1) ||
                      (g.nby0 > 0 && y0 < g.nby0) || (g.nby1 > 0 && y0 + TY > g.NY - g.nby1) || g.nbz0 > 0 ||
                      g.nbz1 > 0);
    float4 Ex4 = make_float4(0, 0, 0, 0);
    float Ey[RY];
#pragma unroll
    for (int r = 0; r < RY; r++) Ey[r] = 0.f;
    if (spg) {
        Ex4 = __ldg(reinterpret_cast<const float4 *>(A.E[2] + gx0));
#pragma unroll
        for (int r = 0; r < RY; r++) Ey[r] = __ldg(A.E[1] + y0 + w * RY + r);
    }
    // offsets of (z = 0, y0 + w RY, gx0), of the staged plane's corner and of the tile's corner
    const long long own0 = cell_off(g, 0, y0 + w * RY, gx0);
    const long long halo0 = cell_off(g, 0, y0 - 4, x0 - 4);
    const long long tile0 = cell_off(g, 0, y0, x0);

    cudaGridDependencySynchronize();

    // register queue: planes z-4 .. z+4 of this thread's cells
    float4 q[9][RY];
    auto load_plane = [&](int z, int r) -> float4 {
        if (z < 0) {
            if (!g.fs) return make_float4(0, 0, 0, 0);
            const float4 v = *reinterpret_cast<const float4 *>(pc + own0 + (long long)(-z) * PP + r * g.P);
            return make_float4(-v.x, -v.y, -v.z, -v.w);
        }
        return *reinterpret_cast<const float4 *>(pc + own0 + (long long)z * PP + r * g.P);
    };
#pragma unroll
    for (int k = 0; k < 8; k++)
#pragma unroll
        for (int r = 0; r < RY; r++) q[k + 1][r] = load_plane(zb - 4 + k, r);

    // plane z into its slot: p^n with halo, and (for planes this CTA
    // updates) p^{n-1} and c of the own cells
    auto stage = [&](int z) {
        float *dst = ring + (z % NS3) * SLOT;
        const float *src = pc + halo0 + (long long)z * PP;
        for (int rr = w; rr < NR; rr += NW) {
            cp16(dst + rr * SW3 + 4 * lane, src + rr * g.P + 4 * lane);
            if (lane < 2) cp16(dst + rr * SW3 + 128 + 4 * lane, src + rr * g.P + 128 + 4 * lane);
        }
        if (z < ze) {
            float *dpp = dst + NR * SW3, *dch = dpp + TY * TX;
            const long long o = tile0 + (long long)z * PP;
            for (int rr = w; rr < TY; rr += NW) {
                cp16(dpp + rr * TX + 4 * lane, pn + o + rr * g.P + 4 * lane);
                cp16(dch + rr * TX + 4 * lane, A.ch + o + rr * g.P + 4 * lane);
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int k = 0; k < NS3 - 1; k++) stage(zb + k);

    for (int z = zb; z < ze; z++) {
        stage(z + NS3 - 1);
        cp_wait<1>();
        __syncthreads();
        const float *cur = ring + (z % NS3) * SLOT;
        const float *ahead = ring + ((z + 4) % NS3) * SLOT;
#pragma unroll
        for (int k = 0; k < 8; k++)
#pragma unroll
            for (int r = 0; r < RY; r++) q[k][r] = q[k + 1][r];
#pragma unroll
        for (int r = 0; r < RY; r++)
            q[8][r] = *reinterpret_cast<const float4 *>(ahead + (w * RY + r + 4) * SW3 + 4 + 4 * lane);
        const float ez = spg ? __ldg(A.E[0] + z) : 0.f;
#pragma unroll
        for (int r = 0; r < RY; r++) {
            const int ly = w * RY + r, gy = y0 + ly;
            const float *row = cur + (ly + 4) * SW3 + 4 + 4 * lane;  // this thread's float4 in the staged plane
            const float4 L = *reinterpret_cast<const float4 *>(row - 4), C = *reinterpret_cast<const float4 *>(row),
                         R = *reinterpret_cast<const float4 *>(row + 4);
            float4 yv[9];
#pragma unroll
            for (int m = 0; m < 9; m++) yv[m] = *reinterpret_cast<const float4 *>(row + (m - 4) * SW3);
            const float4 pp4 = *reinterpret_cast<const float4 *>(cur + NR * SW3 + ly * TX + 4 * lane);
            const float4 ch4 = *reinterpret_cast<const float4 *>(cur + NR * SW3 + TY * TX + ly * TX + 4 * lane);
            const Cells4 cu = cells4(L, C, R, yv, q[0][r], q[1][r], q[2][r], q[3][r], q[5][r], q[6][r], q[7][r],
                                     q[8][r], pp4, ch4, spg, ez + Ey[r], Ex4);
            float res[4], qk[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                res[k] = cu.res[k];
                const float es = spg ? ez + Ey[r] + lane4(Ex4, k) : 0.f;
                qk[k] = es * (res[k] - lane4(pp4, k)) - cu.rhs[k];
            }
            if (xedge) {
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if (gx0 + k >= g.NX) res[k] = 0.f;
            }
            if (g.fs && z == 0) res[0] = res[1] = res[2] = res[3] = 0.f;
            if (gy < g.NY) {
                const long long o = own0 + (long long)z * PP + r * g.P;
                *reinterpret_cast<float4 *>(pn + o) = make_float4(res[0], res[1], res[2], res[3]);
                if (MODE == kModeRecord)
                    *reinterpret_cast<float4 *>(qs + sh + o) = make_float4(qk[0], qk[1], qk[2], qk[3]);
                if (MODE == kModeAdjoint) {
                    const float4 q4 = *reinterpret_cast<const float4 *>(qs + sh + o);
                    float4 g4 = *reinterpret_cast<const float4 *>(Gs + sh + o);
                    g4.x += res[0] * q4.x;
                    g4.y += res[1] * q4.y;
                    g4.z += res[2] * q4.z;
                    g4.w += res[3] * q4.w;
                    *reinterpret_cast<float4 *>(Gs + sh + o) = g4;
                }
            }
        }
        __syncthreads();  // this slot is restaged at the next plane
    }
    cp_wait<0>();  // no copy into shared memory outlives the block
}

// ---------------------------------------------------------------- x-strip CPML arithmetic
// One float4 of x cells (v: the 12-float window of p^n around it, cells
// v[4..7]); shared by the x-strip pass (k_cpml_row3d) and the z-march that
// folds the x strips in, so both give the same bits.
//   psi^n  = b psi^{n-1} + a D1 p^n
//   zeta^n = b zeta^{n-1} + a (D2 p^n + D1 psi^n),   addend = D1 psi^n + zeta^n
__device__ __forceinline__ float4 xcpml_psi(const float *v, const float4 old, const float4 a4, const float4 b4) {
    float r[4];
#pragma unroll
    for (int k = 0; k < 4; k++)
        r[k] = lane4(b4, k) * lane4(old, k) +
               lane4(a4, k) * (float(kD1) * (v[5 + k] - v[3 + k]) + float(kD2) * (v[6 + k] - v[2 + k]) +
                               float(kD3) * (v[7 + k] - v[1 + k]) + float(kD4) * (v[8 + k] - v[k]));
    return make_float4(r[0], r[1], r[2], r[3]);
}
// w: the 12-float window of psi^n; d2[k]: D2 p^n of the cells
__device__ __forceinline__ void xcpml_zeta(const float *w, const float *d2, const float4 zo, const float4 a4,
                                           const float4 b4, float *zt, float *add) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float dps = float(kD1) * (w[5 + k] - w[3 + k]) + float(kD2) * (w[6 + k] - w[2 + k]) +
                          float(kD3) * (w[7 + k] - w[1 + k]) + float(kD4) * (w[8 + k] - w[k]);
        zt[k] = lane4(b4, k) * lane4(zo, k) + lane4(a4, k) * (d2[k] + dps);
        add[k] = dps + zt[k];
    }
}
// the float4 starting at cell x holds x-strip cells
__device__ __forceinline__ bool xstrip4(const Geom &g, int x) {
    return x + 3 >= 0 && x < g.NX && ((g.nbx0 > 0 && x < g.nbx0) || (g.nbx1 > 0 && x + 3 >= g.NX - g.nbx1));
}

// ---------------------------------------------------------------- z-march with TMA
//
// The same update as k_step3d, with the planes staged by the tensor memory
// accelerator: one thread issues, per plane, three bulk tensor copies (p^n
// with its radius-4 x/y halo, 136 x 16 cells, into the halo ring; p^{n-1} and
// c of the tile's own 128 x 8 cells into the own ring) and arms each slot's
// mbarrier with its byte count; every thread waits on the barriers (bounded)
// instead of issuing its own 16-byte copies. The z loop is unrolled by the 9
// planes of the register queue (the queue rotates by renaming registers) or
// not (it shifts). A wait that gives up sets kFlagTimeout; all threads then
// leave together after the copies already issued have landed (also bounded).
// Two rings: the p^n halo tiles (read four planes ahead of their own update,
// for the register queue, and again at it) and the p^{n-1} / c tiles of the
// own cells (read only at the update). The halo ring stages NSH - 1 planes
// ahead, so the queue's plane z + 4 was requested three planes before its
// use; the own ring stages NSO - 1 planes ahead. 8 x 8704 + 3 x 8192 bytes:
// two CTAs per SM.
constexpr int NSH = 8, NSO = 3;
constexpr int HALO_T = 16 * SW3 * 4, OWN_T = 8 * TX * 4, OSLOT_T = 2 * OWN_T;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned cnt) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity, long long limit) {
    for (long long i = 0; i < limit; i++)
        if (mbar_try(b, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load4(void *dst, const CUtensorMap *m, int x, int y, int z, int w,
                                          unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(m)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *m, int x, int y, int z,
                                          unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(m)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// x strips folded into the march: the float4s overlapping [0, lqb) and
// [rqa, NX) take the x-CPML addend (their psi / zeta where they hold strip
// cells); both ranges lie inside the first / last x tile.
struct XFuse {
    int on, lqb, rqa, pad;
};

__device__ __forceinline__ float4 shfl4w(const float4 v, bool up) {
    float4 r;
    r.x = up ? __shfl_up_sync(0xffffffffu, v.x, 1) : __shfl_down_sync(0xffffffffu, v.x, 1);
    r.y = up ? __shfl_up_sync(0xffffffffu, v.y, 1) : __shfl_down_sync(0xffffffffu, v.y, 1);
    r.z = up ? __shfl_up_sync(0xffffffffu, v.z, 1) : __shfl_down_sync(0xffffffffu, v.z, 1);
    r.w = up ? __shfl_up_sync(0xffffffffu, v.w, 1) : __shfl_down_sync(0xffffffffu, v.w, 1);
    return r;
}

// UN = 9: the plane loop unrolled by the queue's length (the queue rotates by
// renaming); UN = 1: a plain loop that shifts the queue (smaller code); UN =
// 3: unrolled by three, the queue rotated by three after each block.
template <int MODE, int UN>
__global__ void __launch_bounds__(NTH, 2) k_step3d_tma(const StepArgs<float> A, const __grid_constant__ Tma3 M,
                                                       const int n, const int zchunk, const int ms, const XFuse X,
                                                       float *qs, float *Gs, const long long spin) {
    constexpr int TY = NW;
    extern __shared__ __align__(128) unsigned char sm_t[];
    unsigned char *const hring = sm_t, *const oring = sm_t + NSH * HALO_T;
    unsigned long long *const fh = reinterpret_cast<unsigned long long *>(sm_t + NSH * HALO_T + NSO * OSLOT_T);
    unsigned long long *const fo = fh + NSH;

    const Geom &g = A.g;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nchunk = (g.NZ + zchunk - 1) / zchunk;
    const int shot = blockIdx.z / nchunk, zb = (blockIdx.z % nchunk) * zchunk;
    const int ze = min(zb + zchunk, g.NZ);
    const long long PP = (long long)g.PY * g.P;
    const long long sh = (long long)shot * g.fstride;
    const float *pc = A.pbuf[n & 1] + sh;
    float *pn = A.pbuf[(n + 1) & 1] + sh;
    const int gx0 = x0 + 4 * lane;
    const bool xedge = x0 + TX > g.NX;
    const bool spg = A.bc == SIM_BC_SPONGE &&
                     ((g.nbx0 > 0 && x0 < g.nbx0) || (g.nbx1 > 0 && x0 + TX > g.NX - g.nbx1) ||
                      (g.nby0 > 0 && y0 < g.nby0) || (g.nby1 > 0 && y0 + TY > g.NY - g.nby1) || g.nbz0 > 0 ||
                      g.nbz1 > 0);
    float4 Ex4 = make_float4(0, 0, 0, 0);
    float Ey = 0.f;
    if (spg) {
        Ex4 = __ldg(reinterpret_cast<const float4 *>(A.E[2] + gx0));
        Ey = __ldg(A.E[1] + y0 + w);
    }
    const long long own0 = cell_off(g, 0, y0 + w, gx0);
    // this tile holds x-strip cells whose CPML the march takes (block-uniform)
    const bool xtile = MODE != kModeAdjoint && X.on && (x0 < X.lqb || x0 + TX > X.rqa);
    // tensor coordinates of the padded layout: (x, y, z) + kGhost; w = buffer parity * ms + shot
    const int tx = x0 + kGhost, ty = y0 + kGhost;
    const int wcur = (n & 1) * ms + shot, wprev = ((n + 1) & 1) * ms + shot;
    if (tid == 0) {
        for (int k = 0; k < NSH + NSO; k++) mbar_init(fh + k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    cudaGridDependencySynchronize();

    // thread 0 stages: the halo tile of plane z into halo slot (z - zb) % NSH
    // (planes up to ze + 3 feed the queue; beyond the grid the copy fills
    // zeros), the own tiles of plane z < ze into own slot (z - zb) % NSO
    int zlast = zb - 1, olast = zb - 1;  // last planes staged (thread 0)
    auto stage_h = [&](int z, int k) {
        zlast = z;
        mbar_expect(fh + k, HALO_T);
        tma_load4(hring + k * HALO_T, &M.ph, tx - 4, ty - 4, z + kGhost, wcur, fh + k);
    };
    auto stage_o = [&](int z, int k) {
        if (z >= ze) return;
        olast = z;
        unsigned char *dst = oring + k * OSLOT_T;
        mbar_expect(fo + k, OSLOT_T);
        tma_load4(dst, &M.po, tx, ty, z + kGhost, wprev, fo + k);
        tma_load3(dst + OWN_T, &M.c, tx, ty, z + kGhost, fo + k);
    };
    if (tid == 0) {
        for (int k = 0; k < NSH - 1; k++) stage_h(zb + k, k);
        for (int k = 0; k < NSO - 1; k++) stage_o(zb + k, k);
    }

    // register queue of this thread's cells: plane z + m lives in q[(j + m + 4) % 9]
    // at unrolled step j of a block of 9 planes
    float4 q[9];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int z = zb - 4 + k;
        float4 v;
        if (z < 0) {
            if (!g.fs) {
                v = make_float4(0, 0, 0, 0);
            } else {
                const float4 u = *reinterpret_cast<const float4 *>(pc + own0 + (long long)(-z) * PP);
                v = make_float4(-u.x, -u.y, -u.z, -u.w);
            }
        } else {
            v = *reinterpret_cast<const float4 *>(pc + own0 + (long long)z * PP);
        }
        q[k] = v;
    }

    // x-strip CPML memory of the next plane, loaded one plane ahead of its use
    // (the edge tiles would otherwise wait on a DRAM round trip every plane)
    const bool xlane = xtile && y0 + w < g.NY && xstrip4(g, gx0);
    float4 psiN = make_float4(0.f, 0.f, 0.f, 0.f), zetaN = psiN;
    if (xlane) {
        const long long o = sh + own0 + (long long)zb * PP;
        psiN = ld4g(A.psi[2][0] + o);
        zetaN = ld4g(A.zeta[2] + o);
    }
    bool bad = false;
    // halo slots and barrier phases of planes z and z + 4, own slot and phase
    // of plane z, advanced per plane
    int kz = 0, pz = 0, k4 = 4 % NSH, p4 = 4 / NSH, ko = 0, po = 0;
    long long orow = own0 + (long long)zb * PP;  // this thread's float4 of plane z
    for (int zz = zb; zz < ze && !bad; zz += UN) {
#pragma unroll
        for (int j = 0; j < UN; j++) {
            const int z = zz + j;
            if (z >= ze || bad) break;
            if (tid == 0) {  // into the slots plane z - 1 used
                stage_h(z + NSH - 1, kz == 0 ? NSH - 1 : kz - 1);
                stage_o(z + NSO - 1, ko == 0 ? NSO - 1 : ko - 1);
            }
            // plane z's halo arrived before plane z - 4 used it (a completed
            // phase answers at once); plane z + 4's and the own tiles are new
            bool ok = mbar_wait(fh + kz, pz, spin);
            ok = ok && mbar_wait(fh + k4, p4, spin);
            ok = ok && mbar_wait(fo + ko, po, spin);
            ok = __all_sync(0xffffffffu, ok);  // the warp computes (and shuffles) together or not at all
            if (ok) {
                const float *cur = reinterpret_cast<const float *>(hring + kz * HALO_T);
                const float *ahead = reinterpret_cast<const float *>(hring + k4 * HALO_T);
                const float *own = reinterpret_cast<const float *>(oring + ko * OSLOT_T);
                q[(j + 8) % 9] = *reinterpret_cast<const float4 *>(ahead + (w + 4) * SW3 + 4 + 4 * lane);
                const float ez = spg ? __ldg(A.E[0] + z) : 0.f;
                const int gy = y0 + w;
                const float *row = cur + (w + 4) * SW3 + 4 + 4 * lane;
                const float4 L = *reinterpret_cast<const float4 *>(row - 4), C = *reinterpret_cast<const float4 *>(row),
                             R = *reinterpret_cast<const float4 *>(row + 4);
                const float v[12] = {L.x, L.y, L.z, L.w, C.x, C.y, C.z, C.w, R.x, R.y, R.z, R.w};
                float4 yv[9];
#pragma unroll
                for (int m = 0; m < 9; m++) yv[m] = *reinterpret_cast<const float4 *>(row + (m - 4) * SW3);
                const float4 pp4 = *reinterpret_cast<const float4 *>(own + w * TX + 4 * lane);
                const float4 ch4 = *reinterpret_cast<const float4 *>(own + TY * TX + w * TX + 4 * lane);
                const Cells4 cu = cells4(L, C, R, yv, q[j % 9], q[(j + 1) % 9], q[(j + 2) % 9], q[(j + 3) % 9],
                                         q[(j + 5) % 9], q[(j + 6) % 9], q[(j + 7) % 9], q[(j + 8) % 9], pp4, ch4,
                                         spg, ez + Ey, Ex4);
                float res[4], qk[4], d2xs[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    res[k] = cu.res[k];
                    d2xs[k] = cu.d2x[k];
                    const float es = spg ? ez + Ey + lane4(Ex4, k) : 0.f;
                    qk[k] = es * (res[k] - lane4(pp4, k)) - cu.rhs[k];
                }
                if (xtile) {  // x-strip CPML of the row, as k_cpml_row3d computes it after the update
                    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    const long long o = sh + orow;
                    const bool strip = gy < g.NY && xstrip4(g, gx0);
                    const bool inw = gy < g.NY && gx0 < g.NX && (gx0 < X.lqb || gx0 + 3 >= X.rqa);
                    const bool zrow = !(g.fs && z == 0);  // the free-surface row stays zero
                    float4 a4 = zero4, b4 = zero4, old = zero4, zo = zero4;
                    if (strip) {
                        a4 = ld4g(A.ca[2] + gx0);
                        b4 = ld4g(A.cb[2] + gx0);
                        old = psiN;
                        if (zrow) zo = zetaN;
                        if (z + 1 < ze) {  // the next plane's, in flight while this one is computed
                            psiN = ld4g(A.psi[2][0] + o + PP);
                            zetaN = ld4g(A.zeta[2] + o + PP);
                        }
                    }
                    float4 ps = zero4;
                    if (strip) {
                        ps = xcpml_psi(v, old, a4, b4);
                        *reinterpret_cast<float4 *>(A.psi[2][0] + o) = ps;
                    }
                    float4 sL = shfl4w(ps, true), sR = shfl4w(ps, false);
                    if (lane == 0) sL = zero4;
                    if (lane == 31) sR = zero4;
                    if (inw && zrow) {
                        const float wv[12] = {sL.x, sL.y, sL.z, sL.w, ps.x, ps.y, ps.z, ps.w, sR.x, sR.y, sR.z, sR.w};
                        float zt[4], add[4];
                        xcpml_zeta(wv, d2xs, zo, a4, b4, zt, add);
                        if (strip) *reinterpret_cast<float4 *>(A.zeta[2] + o) = make_float4(zt[0], zt[1], zt[2], zt[3]);
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            res[k] += lane4(ch4, k) * add[k];
                            qk[k] -= add[k];
                        }
                    }
                }
                if (xedge) {
#pragma unroll
                    for (int k = 0; k < 4; k++)
                        if (gx0 + k >= g.NX) res[k] = 0.f;
                }
                if (g.fs && z == 0) res[0] = res[1] = res[2] = res[3] = 0.f;
                if (gy < g.NY && gx0 < g.NX) {  // cells past the grid stay zero: no store
                    const long long o = orow;
                    *reinterpret_cast<float4 *>(pn + o) = make_float4(res[0], res[1], res[2], res[3]);
                    if (MODE == kModeRecord)
                        *reinterpret_cast<float4 *>(qs + sh + o) = make_float4(qk[0], qk[1], qk[2], qk[3]);
                    if (MODE == kModeAdjoint) {
                        const float4 q4 = *reinterpret_cast<const float4 *>(qs + sh + o);
                        float4 g4 = *reinterpret_cast<const float4 *>(Gs + sh + o);
                        g4.x += res[0] * q4.x;
                        g4.y += res[1] * q4.y;
                        g4.z += res[2] * q4.z;
                        g4.w += res[3] * q4.w;
                        *reinterpret_cast<float4 *>(Gs + sh + o) = g4;
                    }
                }
            }
            if (UN == 1) {
#pragma unroll
                for (int k = 0; k < 8; k++) q[k] = q[k + 1];
            }
            orow += PP;
            if (++kz == NSH) kz = 0, pz ^= 1;
            if (++k4 == NSH) k4 = 0, p4 ^= 1;
            if (++ko == NSO) ko = 0, po ^= 1;
            // every thread is done with slot kz before it is restaged; a wait
            // that gave up anywhere ends the march for the whole block
            bad = __syncthreads_or(!ok) != 0;
        }
        if (UN == 3) {  // plane zz + 3 + m back to q[(m + 4) % 9] for the next block
            const float4 t0 = q[0], t1 = q[1];
#pragma unroll
            for (int k = 0; k < 6; k++) q[k] = q[k + 3];
            q[6] = t0;
            q[7] = t1;
        }
    }
    // the last planes staged (ahead of the march) may still be in flight:
    // wait for each slot's last phase (a completed phase returns at once) so
    // no copy outlives the block
    if (tid == 0) {
        if (bad) atomicOr(A.flags, kFlagTimeout);
        for (int z = max(zb, zlast - NSH + 1); z <= zlast; z++) {
            const int k = (z - zb) % NSH;
            if (!mbar_wait(fh + k, ((z - zb) / NSH) & 1, spin)) atomicOr(A.flags, kFlagTimeout);
        }
        for (int z = max(zb, olast - NSO + 1); z <= olast; z++) {
            const int k = (z - zb) % NSO;
            if (!mbar_wait(fo + k, ((z - zb) / NSO) & 1, spin)) atomicOr(A.flags, kFlagTimeout);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- CPML (3D)
// psi^n = b psi^{n-1} + a D1 p^n on the cells of one axis' strips.
__device__ __forceinline__ long long axis_stride(const Geom &g, int ax) {
    return ax == 0 ? (long long)g.PY * g.P : (ax == 1 ? (long long)g.P : 1LL);
}

struct Box {
    int z0, z1, y0, y1, x0, x1;
};

// The strip kernels work on float4 columns: a box's x-range is rounded out to
// multiples of 4 (cells so added lie outside the strips, where both
// recursion coefficients are zero, or beyond the grid, where c is zero, so
// they stay zero and add nothing). Item i of a box is float4 column
// i mod C of row i / C, rows ordered (z, y).
__device__ __forceinline__ bool box_item(const Box &b, long long i, int &z, int &y, int &x) {
    const int nc = (b.x1 - b.x0) >> 2, ny = b.y1 - b.y0;
    if (nc <= 0 || ny <= 0) return false;
    const long long row = i / nc;
    x = b.x0 + 4 * (int)(i - row * nc);
    y = b.y0 + (int)(row % ny);
    z = b.z0 + (int)(row / ny);
    return z < b.z1;
}
__device__ __forceinline__ long long box_items(const Box &b) {
    return (long long)(b.z1 - b.z0) * (b.y1 - b.y0) * ((b.x1 - b.x0) >> 2);
}

// D1 of the float4 at o along axis stride s (s > 1), or along x from a
// 12-float window (s == 1)
__device__ __forceinline__ float4 d1_4(const float *f, long long o, long long s) {
    float r[4];
    if (s == 1) {
        const float4 L = ld4g(f + o - 4), C = ld4g(f + o), R = ld4g(f + o + 4);
        const float v[12] = {L.x, L.y, L.z, L.w, C.x, C.y, C.z, C.w, R.x, R.y, R.z, R.w};
#pragma unroll
        for (int k = 0; k < 4; k++)
            r[k] = float(kD1) * (v[5 + k] - v[3 + k]) + float(kD2) * (v[6 + k] - v[2 + k]) +
                   float(kD3) * (v[7 + k] - v[1 + k]) + float(kD4) * (v[8 + k] - v[k]);
    } else {
        float4 a = ld4g(f + o + s), b = ld4g(f + o - s);
        r[0] = float(kD1) * (a.x - b.x); r[1] = float(kD1) * (a.y - b.y);
        r[2] = float(kD1) * (a.z - b.z); r[3] = float(kD1) * (a.w - b.w);
        a = ld4g(f + o + 2 * s), b = ld4g(f + o - 2 * s);
        r[0] += float(kD2) * (a.x - b.x); r[1] += float(kD2) * (a.y - b.y);
        r[2] += float(kD2) * (a.z - b.z); r[3] += float(kD2) * (a.w - b.w);
        a = ld4g(f + o + 3 * s), b = ld4g(f + o - 3 * s);
        r[0] += float(kD3) * (a.x - b.x); r[1] += float(kD3) * (a.y - b.y);
        r[2] += float(kD3) * (a.z - b.z); r[3] += float(kD3) * (a.w - b.w);
        a = ld4g(f + o + 4 * s), b = ld4g(f + o - 4 * s);
        r[0] += float(kD4) * (a.x - b.x); r[1] += float(kD4) * (a.y - b.y);
        r[2] += float(kD4) * (a.z - b.z); r[3] += float(kD4) * (a.w - b.w);
    }
    return make_float4(r[0], r[1], r[2], r[3]);
}
// D2 of the float4 at o along axis stride s (same conventions)
__device__ __forceinline__ float4 d2_4(const float *f, long long o, long long s) {
    float r[4];
    if (s == 1) {
        const float4 L = ld4g(f + o - 4), C = ld4g(f + o), R = ld4g(f + o + 4);
        const float v[12] = {L.x, L.y, L.z, L.w, C.x, C.y, C.z, C.w, R.x, R.y, R.z, R.w};
#pragma unroll
        for (int k = 0; k < 4; k++)
            r[k] = d2c<float>(v[4 + k], v[3 + k], v[5 + k], v[2 + k], v[6 + k], v[1 + k], v[7 + k], v[k], v[8 + k]);
    } else {
        const float4 c = ld4g(f + o);
        const float4 m1 = ld4g(f + o - s), p1 = ld4g(f + o + s), m2 = ld4g(f + o - 2 * s), p2 = ld4g(f + o + 2 * s);
        const float4 m3 = ld4g(f + o - 3 * s), p3 = ld4g(f + o + 3 * s), m4 = ld4g(f + o - 4 * s),
                     p4 = ld4g(f + o + 4 * s);
#pragma unroll
        for (int k = 0; k < 4; k++)
            r[k] = d2c<float>(lane4(c, k), lane4(m1, k), lane4(p1, k), lane4(m2, k), lane4(p2, k), lane4(m3, k),
                              lane4(p3, k), lane4(m4, k), lane4(p4, k));
    }
    return make_float4(r[0], r[1], r[2], r[3]);
}
__device__ __forceinline__ void coef4(const StepArgs<float> &A, int ax, int z, int y, int x, float4 &a4, float4 &b4) {
    if (ax == 2) {
        a4 = ld4g(A.ca[2] + x);
        b4 = ld4g(A.cb[2] + x);
    } else {
        const int k = ax == 0 ? z : y;
        const float a = A.ca[ax][k], b = A.cb[ax][k];
        a4 = make_float4(a, a, a, a);
        b4 = make_float4(b, b, b, b);
    }
}

__global__ void k_psi3d(const StepArgs<float> A, const int n, const int ax, const Box b0, const Box b1) {
    const Geom &g = A.g;
    const long long s = axis_stride(g, ax);
    const long long n0 = box_items(b0), n1 = box_items(b1);
    const int shot = blockIdx.y;
    const long long sh = (long long)shot * g.fstride;
    const float *p = A.pbuf[n & 1] + sh;
    float *psi = A.psi[ax][0] + sh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n0 + n1;
         i += (long long)gridDim.x * blockDim.x) {
        int z, y, x;
        if (!(i < n0 ? box_item(b0, i, z, y, x) : box_item(b1, i - n0, z, y, x))) continue;
        const long long o = cell_off(g, z, y, x);
        float4 a4, b4;
        coef4(A, ax, z, y, x, a4, b4);
        const float4 d = d1_4(p, o, s), old = ld4g(psi + o);
        *reinterpret_cast<float4 *>(psi + o) = make_float4(b4.x * old.x + a4.x * d.x, b4.y * old.y + a4.y * d.y,
                                                           b4.z * old.z + a4.z * d.z, b4.w * old.w + a4.w * d.w);
    }
}

// zeta^n = b zeta^{n-1} + a (D2 p^n + D1 psi^n); p^{n+1} += c (D1 psi^n + zeta^n)
// on the strips of one axis widened by 4 cells (where D1 psi is non-zero).
__global__ void k_cpml_add3d(const StepArgs<float> A, const int n, const int ax, const Box b0, const Box b1,
                             float *qs) {
    const Geom &g = A.g;
    const long long s = axis_stride(g, ax);
    const long long n0 = box_items(b0), n1 = box_items(b1);
    const int shot = blockIdx.y;
    const long long sh = (long long)shot * g.fstride;
    const float *p = A.pbuf[n & 1] + sh;
    float *pn = A.pbuf[(n + 1) & 1] + sh;
    const float *psi = A.psi[ax][0] + sh;
    float *zeta = A.zeta[ax] + sh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n0 + n1;
         i += (long long)gridDim.x * blockDim.x) {
        int z, y, x;
        if (!(i < n0 ? box_item(b0, i, z, y, x) : box_item(b1, i - n0, z, y, x))) continue;
        if (g.fs && z == 0) continue;
        const long long o = cell_off(g, z, y, x);
        float4 d2;
        if (ax == 0 && g.fs && z < 4) {  // z-derivative across the free surface: odd mirror
            float r[4];
            for (int k = 0; k < 4; k++) {
                float c[9];
                for (int m = -4; m <= 4; m++) {
                    const int zz = z + m;
                    c[m + 4] = zz < 0 ? -p[cell_off(g, -zz, y, x + k)] : p[cell_off(g, zz, y, x + k)];
                }
                r[k] = d2c<float>(c[4], c[3], c[5], c[2], c[6], c[1], c[7], c[0], c[8]);
            }
            d2 = make_float4(r[0], r[1], r[2], r[3]);
        } else {
            d2 = d2_4(p, o, s);
        }
        float4 a4, b4;
        coef4(A, ax, z, y, x, a4, b4);
        const float4 dps = d1_4(psi, o, s), zo = ld4g(zeta + o), ch = ld4g(A.ch + o);
        const float4 zt = make_float4(b4.x * zo.x + a4.x * (d2.x + dps.x), b4.y * zo.y + a4.y * (d2.y + dps.y),
                                      b4.z * zo.z + a4.z * (d2.z + dps.z), b4.w * zo.w + a4.w * (d2.w + dps.w));
        *reinterpret_cast<float4 *>(zeta + o) = zt;
        float4 pv = ld4g(pn + o);
        pv.x += ch.x * (dps.x + zt.x);
        pv.y += ch.y * (dps.y + zt.y);
        pv.z += ch.z * (dps.z + zt.z);
        pv.w += ch.w * (dps.w + zt.w);
        *reinterpret_cast<float4 *>(pn + o) = pv;
        if (qs) {  // record mode: the addend is part of the Laplacian in the imaging term
            float4 qv = ld4g(qs + sh + o);
            qv.x -= dps.x + zt.x;
            qv.y -= dps.y + zt.y;
            qv.z -= dps.z + zt.z;
            qv.w -= dps.w + zt.w;
            *reinterpret_cast<float4 *>(qs + sh + o) = qv;
        }
    }
}

// CPML of the z or y axis (stride > 1) in one pass after the update, on
// float4 columns along the axis. A thread owns one column of one strip range
// [s0, s1) (the strip widened by 4 cells towards the interior, where D1 psi
// is non-zero) and marches along it: psi^n at r from p^n at r - 4 .. r + 4
// (a 13-entry register window of p^n, r - 8 .. r + 4), then, 4 positions
// behind, zeta^n and the addend at q = r - 4 from the 9 psi^n values
// q - 4 .. q + 4 (a second window) and D2 p^n at q:
//   psi^n  = b psi^{n-1}  + a D1 p^n          (strip cells; written back)
//   zeta^n = b zeta^{n-1} + a (D2 p^n + D1 psi^n)
//   p^{n+1} += c (D1 psi^n + zeta^n)          (cells of [s0, s1))
// p^n is still intact after the update kernel (which writes p^{n+1} into the
// other buffer). Same arithmetic as k_psi3d + k_cpml_add3d, with every value
// read once. Not used for a z range within reach of a free surface (its D2
// needs the odd mirror; the two-kernel path handles it).

constexpr int CNS = 4;  // positions in a column pass thread's copy ring

struct ColRanges {
    int n;            // ranges (1 or 2)
    int s0[2], s1[2]; // [s0, s1) along the axis
};

__global__ void __launch_bounds__(128) k_cpml_col3d(const StepArgs<float> A, const int n, const int ax,
                                                    const ColRanges R, const int ncols, float *qs) {
    const Geom &g = A.g;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= (long long)R.n * ncols) return;
    const int k = (int)(tid / ncols), col = (int)(tid - (long long)k * ncols);
    const int nx4 = (g.NX + 3) >> 2;
    const int u = col / nx4, x = 4 * (col - u * nx4);  // u: y (z axis) or z (y axis)
    const int N = ax == 0 ? g.NZ : g.NY;
    const int lo = ax == 0 ? g.nbz0 : g.nby0, hi = ax == 0 ? g.nbz1 : g.nby1;
    const long long s = axis_stride(g, ax);
    const int s0 = k == 0 ? R.s0[0] : R.s0[1], s1 = k == 0 ? R.s1[0] : R.s1[1];
    const int shot = blockIdx.y;
    const long long sh = (long long)shot * g.fstride;
    const long long o0 = ax == 0 ? cell_off(g, 0, u, x) : cell_off(g, u, 0, x);  // position 0 of the column
    const float *__restrict__ p = A.pbuf[n & 1] + sh + o0;
    float *__restrict__ pn = A.pbuf[(n + 1) & 1] + sh + o0;
    float *__restrict__ psi = A.psi[ax][0] + sh + o0;
    float *__restrict__ zeta = A.zeta[ax] + sh + o0;
    const float *__restrict__ ch = A.ch + o0;
    float *qcol = qs ? qs + sh + o0 : nullptr;  // record mode: imaging term of the step
    const float *ca = A.ca[ax], *cb = A.cb[ax];
    const bool skip_row = g.fs && ax == 1 && u == 0;  // the free-surface row stays zero
    auto strip = [&](int r) { return (lo > 0 && r >= 0 && r < lo) || (hi > 0 && r >= N - hi && r < N); };
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);

    // The loads of position r (p^n at r + 4, psi^{n-1} at r, and at q = r - 4
    // zeta^{n-1}, c, p^{n+1}) go by cp.async into this thread's slots of a
    // shared-memory ring, CNS - 1 positions ahead of their use; a load that
    // does not apply fills its slot with zeros (source size 0). Slot (k, f) of
    // thread t is float4 (k * 5 + f) * blockDim + t: a warp's 16-byte accesses
    // are consecutive. The thread reads only its own slots, so its own
    // cp.async.wait_group orders them.
    extern __shared__ float4 col_ring[];
    const unsigned ring0 = (unsigned)__cvta_generic_to_shared(col_ring + threadIdx.x);
    const unsigned fstep = 16u * blockDim.x;  // bytes from one field's slot to the next
    auto issue = [&](int r, int slot) {
        const unsigned d = ring0 + (unsigned)(slot * 5) * fstep;
        const int q = r - 4;
        const bool qq = q >= s0 && !skip_row;
        cp16z(d, p + (long long)(r + 4) * s, true);
        cp16z(d + fstep, strip(r) ? psi + (long long)r * s : p, strip(r));
        cp16z(d + 2 * fstep, qq && strip(q) ? zeta + (long long)q * s : p, qq && strip(q));
        cp16z(d + 3 * fstep, qq ? ch + (long long)q * s : p, qq);
        cp16z(d + 4 * fstep, qq ? pn + (long long)q * s : p, qq);
    };
    auto slot_ld = [&](int slot, int f) {
        return col_ring[(slot * 5 + f) * blockDim.x + threadIdx.x];
    };

    float4 P[13], S[9];
#pragma unroll
    for (int m = 0; m < 4; m++) P[m] = zero;
#pragma unroll
    for (int m = 0; m < 8; m++) P[4 + m] = ld4g(p + (long long)(s0 - 8 + m) * s);
#pragma unroll
    for (int m = 0; m < 9; m++) S[m] = zero;
    const int r0 = s0 - 4, r1 = s1 + 4;
#pragma unroll
    for (int k = 0; k < CNS - 1; k++) {
        if (r0 + k < r1) issue(r0 + k, k);
        cp_commit();
    }

    for (int r = r0, slot = 0; r < r1; r++, slot = slot == CNS - 1 ? 0 : slot + 1) {
        // position r + CNS - 1 into the slot position r - 1 used
        if (r + CNS - 1 < r1) issue(r + CNS - 1, slot == 0 ? CNS - 1 : slot - 1);
        cp_commit();
        cp_wait<CNS - 1>();
        struct {
            float4 p, ps, zo, c, pv;
        } cur = {slot_ld(slot, 0), slot_ld(slot, 1), slot_ld(slot, 2), slot_ld(slot, 3), slot_ld(slot, 4)};
        P[12] = cur.p;
        // psi^n at r (zero off the strips)
        float4 ps = zero;
        if (strip(r)) {
            const float a = __ldg(ca + r), b = __ldg(cb + r);
            const float2 da = d1c2(lo2(P[7]), lo2(P[9]), lo2(P[6]), lo2(P[10]), lo2(P[5]), lo2(P[11]), lo2(P[4]),
                                   lo2(P[12]));
            const float2 db = d1c2(hi2(P[7]), hi2(P[9]), hi2(P[6]), hi2(P[10]), hi2(P[5]), hi2(P[11]), hi2(P[4]),
                                   hi2(P[12]));
            const float4 old = cur.ps;
            const float2 pa = fma2(splat2(a), da, mul2(splat2(b), lo2(old)));
            const float2 pb = fma2(splat2(a), db, mul2(splat2(b), hi2(old)));
            ps = make_float4(pa.x, pa.y, pb.x, pb.y);
            *reinterpret_cast<float4 *>(psi + (long long)r * s) = ps;
        }
        S[8] = ps;
        // zeta^n and the addend at q = r - 4
        const int q = r - 4;
        if (q >= s0 && !skip_row) {
            float a = 0.f, b = 0.f;
            const bool in = strip(q);
            if (in) {
                a = __ldg(ca + q);
                b = __ldg(cb + q);
            }
            const float4 zo = cur.zo, c4 = cur.c;
            float4 pv = cur.pv;
            float zt[4], add[4];
            {
                const float2 d2a = d2c2(lo2(P[4]), lo2(P[3]), lo2(P[5]), lo2(P[2]), lo2(P[6]), lo2(P[1]), lo2(P[7]),
                                        lo2(P[0]), lo2(P[8]));
                const float2 d2b = d2c2(hi2(P[4]), hi2(P[3]), hi2(P[5]), hi2(P[2]), hi2(P[6]), hi2(P[1]), hi2(P[7]),
                                        hi2(P[0]), hi2(P[8]));
                const float2 dsa = d1c2(lo2(S[3]), lo2(S[5]), lo2(S[2]), lo2(S[6]), lo2(S[1]), lo2(S[7]), lo2(S[0]),
                                        lo2(S[8]));
                const float2 dsb = d1c2(hi2(S[3]), hi2(S[5]), hi2(S[2]), hi2(S[6]), hi2(S[1]), hi2(S[7]), hi2(S[0]),
                                        hi2(S[8]));
                const float2 za = fma2(splat2(a), add2(d2a, dsa), mul2(splat2(b), lo2(zo)));
                const float2 zb = fma2(splat2(a), add2(d2b, dsb), mul2(splat2(b), hi2(zo)));
                const float2 aa = add2(dsa, za), ab = add2(dsb, zb);
                zt[0] = za.x, zt[1] = za.y, zt[2] = zb.x, zt[3] = zb.y;
                add[0] = aa.x, add[1] = aa.y, add[2] = ab.x, add[3] = ab.y;
            }
            if (in) *reinterpret_cast<float4 *>(zeta + (long long)q * s) = make_float4(zt[0], zt[1], zt[2], zt[3]);
            {
                const float2 va = fma2(lo2(c4), make_float2(add[0], add[1]), lo2(pv));
                const float2 vb = fma2(hi2(c4), make_float2(add[2], add[3]), hi2(pv));
                pv = make_float4(va.x, va.y, vb.x, vb.y);
            }
            *reinterpret_cast<float4 *>(pn + (long long)q * s) = pv;
            if (qcol) {  // the addend is part of the Laplacian in the imaging term
                float4 qv = ld4g(qcol + (long long)q * s);
                qv.x -= add[0];
                qv.y -= add[1];
                qv.z -= add[2];
                qv.w -= add[3];
                *reinterpret_cast<float4 *>(qcol + (long long)q * s) = qv;
            }
        }
#pragma unroll
        for (int m = 0; m < 12; m++) P[m] = P[m + 1];
#pragma unroll
        for (int m = 0; m < 8; m++) S[m] = S[m + 1];
    }
    cp_wait<0>();  // no copy outlives the thread
}

// CPML of the x axis in one pass after the update: a half-warp per (z, y)
// row and strip end. Lane j holds p^n at the 4 cells xa + 4j (lanes
// [0, nq + 4)); the neighbours' float4s come by shuffles. Lanes [1, nq + 3)
// form psi^n (zero off the strip, written back on strip cells), lanes
// [2, nq + 2) cover the strip widened by 4 cells and update zeta^n and
// p^{n+1} += c (D1 psi^n + zeta^n). Same arithmetic as k_psi3d +
// k_cpml_add3d on the x axis.
struct XEnds {
    int ne;            // strip ends (1 or 2)
    int xa[2], nq[2];  // first cell of lane 0 (a multiple of 4), float4 lanes of the widened strip
};

__device__ __forceinline__ float4 shfl4(const float4 v, int d, bool up) {
    float4 r;
    r.x = up ? __shfl_up_sync(0xffffffffu, v.x, d, 16) : __shfl_down_sync(0xffffffffu, v.x, d, 16);
    r.y = up ? __shfl_up_sync(0xffffffffu, v.y, d, 16) : __shfl_down_sync(0xffffffffu, v.y, d, 16);
    r.z = up ? __shfl_up_sync(0xffffffffu, v.z, d, 16) : __shfl_down_sync(0xffffffffu, v.z, d, 16);
    r.w = up ? __shfl_up_sync(0xffffffffu, v.w, d, 16) : __shfl_down_sync(0xffffffffu, v.w, d, 16);
    return r;
}

// Two row ends per half-warp (items 2 hw and 2 hw + 1 of the (end, row)
// list): the loads of both are issued before either's arithmetic, so twice
// the bytes are in flight per thread.
constexpr int XR = 2;
__global__ void __launch_bounds__(128) k_cpml_row3d(const StepArgs<float> A, const int n, const XEnds E,
                                                    const long long nrows, float *qrec) {
    const Geom &g = A.g;
    const long long hw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 4;
    const int j = threadIdx.x & 15;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const long long sh = (long long)blockIdx.y * g.fstride;
    struct It {
        long long o;
        int z, xj;
        bool strip, pl, ss, qs, ql;
        float4 pc, old, a4, b4, zo, c4, pv;
    };
    It it[XR];
#pragma unroll
    for (int u = 0; u < XR; u++) {  // every load of both items first
        It &I = it[u];
        const long long idx = XR * hw + u;
        const bool live = idx < (long long)E.ne * nrows;  // every lane takes part in the shuffles
        const int e = live && idx >= nrows ? 1 : 0;
        const long long row = live ? idx - e * nrows : 0;
        const int z = (int)(row / g.NY), y = (int)(row - (long long)z * g.NY);
        const int xa = e ? E.xa[1] : E.xa[0], nq = e ? E.nq[1] : E.nq[0];
        I.z = z;
        I.xj = xa + 4 * j;
        I.o = cell_off(g, z, y, 0) + I.xj;
        I.strip = xstrip4(g, I.xj);
        I.pl = live && j < nq + 4;
        const bool sl = live && j >= 1 && j < nq + 3;
        I.ql = live && j >= 2 && j < nq + 2;
        I.qs = I.ql && !(g.fs && z == 0);  // the free-surface row stays zero
        I.ss = sl && I.strip;
        I.pc = I.pl ? ld4g(A.pbuf[n & 1] + sh + I.o) : zero;
        I.old = I.ss ? ld4g(A.psi[2][0] + sh + I.o) : zero;
        I.a4 = zero, I.b4 = zero;
        if (I.ss) {
            I.a4 = ld4g(A.ca[2] + I.xj);
            I.b4 = ld4g(A.cb[2] + I.xj);
        }
        I.zo = I.qs && I.strip ? ld4g(A.zeta[2] + sh + I.o) : zero;
        I.c4 = I.qs ? ld4g(A.ch + I.o) : zero;
        I.pv = I.qs ? ld4g(A.pbuf[(n + 1) & 1] + sh + I.o) : zero;
    }
#pragma unroll
    for (int u = 0; u < XR; u++) {
        const It &I = it[u];
        float *__restrict__ psi = A.psi[2][0] + sh + I.o;
        float *__restrict__ zeta = A.zeta[2] + sh + I.o;
        float *__restrict__ pn = A.pbuf[(n + 1) & 1] + sh + I.o;
        const float4 pL = shfl4(I.pc, 1, true), pR = shfl4(I.pc, 1, false);
        const float v[12] = {pL.x, pL.y, pL.z, pL.w, I.pc.x, I.pc.y, I.pc.z, I.pc.w, pR.x, pR.y, pR.z, pR.w};
        // psi^n of the lane's cells
        float4 ps = zero;
        if (I.ss) {
            ps = xcpml_psi(v, I.old, I.a4, I.b4);
            *reinterpret_cast<float4 *>(psi) = ps;
        }
        const float4 sL = shfl4(ps, 1, true), sR = shfl4(ps, 1, false);
        if (!I.qs) continue;
        const float w[12] = {sL.x, sL.y, sL.z, sL.w, ps.x, ps.y, ps.z, ps.w, sR.x, sR.y, sR.z, sR.w};
        float d2[4], zt[4], add[4];
#pragma unroll
        for (int k = 0; k < 4; k++)
            d2[k] = d2c<float>(v[4 + k], v[3 + k], v[5 + k], v[2 + k], v[6 + k], v[1 + k], v[7 + k], v[k], v[8 + k]);
        xcpml_zeta(w, d2, I.zo, I.a4, I.b4, zt, add);
        if (I.strip) *reinterpret_cast<float4 *>(zeta) = make_float4(zt[0], zt[1], zt[2], zt[3]);
        float4 pv = I.pv;
        pv.x += I.c4.x * add[0];
        pv.y += I.c4.y * add[1];
        pv.z += I.c4.z * add[2];
        pv.w += I.c4.w * add[3];
        *reinterpret_cast<float4 *>(pn) = pv;
        if (qrec) {  // record mode: the addend is part of the Laplacian in the imaging term
            float4 qv = ld4g(qrec + sh + I.o);
            qv.x -= add[0];
            qv.y -= add[1];
            qv.z -= add[2];
            qv.w -= add[3];
            *reinterpret_cast<float4 *>(qrec + sh + I.o) = qv;
        }
    }
}

// ---------------------------------------------------------------- points (3D)

// p^{n+1} += c w[n] weight / h / (1 + a) at each source corner (one thread per shot and corner)
__global__ void k_inject3d(const StepArgs<float> A, const StepTime t, const Pt3 *src, int nshots) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * nshots || t.inj_row < 0) return;
    const int shot = i >> 3, c = i & 7;
    const Pt3 P = src[shot];
    const long long o = P.cell[c];
    if (o < 0) return;
    const Geom &g = A.g;
    float *pn = A.pbuf[(t.n + 1) & 1] + (long long)shot * g.fstride;
    const float w = static_cast<const float *>(A.io->wavelet)[t.inj_row];
    float a = 0.f;
    if (A.bc == SIM_BC_SPONGE) {
        const long long r = o - g.org;
        const long long PP = (long long)g.PY * g.P;
        const int z = (int)(r / PP), y = (int)((r % PP) / g.P), x = (int)(r % g.P);
        a = A.ch[o] * (A.E[0][z] + A.E[1][y] + A.E[2][x]);
    }
    pn[o] += A.ch[o] * A.src_scale * P.w[c] * w / (1.f + a);
}

// Point injection into p^{n+1} by target cell (deterministic order of the
// entries of a cell): value = wavelet[row] (kind 0) or the residual of
// receiver pt at row (kind 1). With the record / adjoint modes the cell's
// imaging term gets the source's share / its G the injected part of u^{n+1}.
__global__ void k_inj3d(const StepArgs<float> A, const int n, const int row, const Inj3 *grp, const int ngrp,
                        const InjE3 *ent, const int kind, const int mode, float *qs, float *Gs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ngrp || row < 0 || row >= A.nt) return;
    const Inj3 G = grp[i];
    if (G.shot >= 0 && blockIdx.y != 0) return;
    const int shot = G.shot >= 0 ? G.shot : blockIdx.y;
    const Geom &g = A.g;
    const SimIO *io = A.io;
    float sum = 0.f;
    for (int e = G.e0; e < G.e1; e++) {
        const InjE3 E = ent[e];
        const float val = kind == 0 ? static_cast<const float *>(io->wavelet)[row]
                                    : static_cast<const float *>(io->resid)[((long long)shot * A.nt + row) * io->nrec + E.pt];
        sum += E.w * val;
    }
    const long long o = G.cell, so = (long long)shot * g.fstride + o;
    float es = 0.f;
    if (A.bc == SIM_BC_SPONGE) {
        const long long r = o - g.org, PP = (long long)g.PY * g.P;
        const int z = (int)(r / PP), y = (int)((r % PP) / g.P), x = (int)(r % g.P);
        es = A.E[0][z] + A.E[1][y] + A.E[2][x];
    }
    const float chv = A.ch[o];
    const float d = chv * A.src_scale * sum / (1.f + chv * es);
    A.pbuf[(n + 1) & 1][so] += d;
    if (mode == kModeRecord) qs[so] += es * d - A.src_scale * sum;
    if (mode == kModeAdjoint) Gs[so] += d * qs[so];
}

__global__ void k_sample3d(const StepArgs<float> A, const StepTime t, const Pt3 *rec, int nrec, int nshots) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)nrec * nshots) return;
    const int shot = (int)(i / nrec), r = (int)(i % nrec);
    const Pt3 P = rec[r];
    const float *p = A.pbuf[t.n & 1] + (long long)shot * A.g.fstride;
    float v = 0.f;
#pragma unroll
    for (int c = 0; c < 8; c++)
        if (P.cell[c] >= 0) v += P.w[c] * p[P.cell[c]];
    static_cast<float *>(A.io->gather)[((long long)shot * A.nt + t.n) * nrec + r] = v;
    if (!isfinite(v)) atomicOr(A.flags, kFlagUnstable);
}

// interior of p^n into the snapshot stack (FP32), or its max |p| (FP16 pass 1)
__global__ void k_snap3d(const StepArgs<float> A, const StepTime t, int pass) {
    const Geom &g = A.g;
    const int shot = blockIdx.y;
    const float *p = A.pbuf[t.n & 1] + (long long)shot * g.fstride;
    const long long nint = (long long)g.nz * g.ny * g.nx;
    const SimIO *io = A.io;
    const long long base = ((long long)shot * A.nsnap + t.snap_k) * nint;
    const float s = (pass == 2) ? pow2_scale(__uint_as_float(io->snap_max[shot * A.nsnap + t.snap_k])) : 1.f;
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nint; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx);
        const long long zy = i / g.nx;
        const int y = (int)(zy % g.ny), z = (int)(zy / g.ny);
        const float v = p[cell_off(g, z + g.oz, y + g.oy, x + g.ox)];
        if (pass == 0) static_cast<float *>(io->snaps)[base + i] = v;
        else if (pass == 1) m = fmaxf(m, fabsf(v));
        else static_cast<__half *>(io->snaps)[base + i] = __float2half_rn(v / s);
    }
    if (pass == 1) {
        m = warp_max(m);
        if ((threadIdx.x & 31) == 0) {
            if (!(m <= FLT_MAX)) atomicOr(A.flags, kFlagUnstable);
            else atomicMax(&io->snap_max[shot * A.nsnap + t.snap_k], __float_as_uint(m));
        }
    }
    if (pass == 2 && blockIdx.x == 0 && threadIdx.x == 0) io->snap_scale[shot * A.nsnap + t.snap_k] = s;
}

template <int RY>
size_t smem3d() {
    return (size_t)NS3 * slot3d<RY>() * sizeof(float);
}

}  // namespace

constexpr size_t kSmemTma = (size_t)NSH * HALO_T + NSO * OSLOT_T + (NSH + NSO) * sizeof(unsigned long long);

// Which x-strip pass a CPML step uses: the one-pass kernel k_cpml_row3d when
// each widened strip spans at most 12 float4s and the two ends are apart;
// with the TMA march (forward and record modes) the march takes it over when,
// moreover, each widened strip lies inside the first / last x tile.
bool x_row_pass(const Geom &g, XEnds *E) {
    const int NX = g.NX;
    int qa[2], qb[2], m = 0;  // widened strips [qa, qb)
    if (g.nbx0 > 0) qa[m] = 0, qb[m++] = std::min(NX, g.nbx0 + 4);
    if (g.nbx1 > 0) qa[m] = std::max(0, NX - g.nbx1 - 4), qb[m++] = NX;
    bool ok = m > 0 && (m < 2 || qa[1] - qb[0] >= 16);  // ends apart: no cell's psi formed twice
    XEnds e{};
    for (int k = 0; k < m && ok; k++) {
        const int q4 = qa[k] & ~3, nq = (qb[k] - q4 + 3) >> 2;
        e.xa[k] = q4 - 8;
        e.nq[k] = nq;
        ok = nq + 4 <= 16;
    }
    e.ne = m;
    if (E) *E = e;
    return ok;
}

XFuse x_fuse(const StepArgs<float> &a, int variant, int mode) {
    XFuse X{0, 0, 1 << 30, 0};
    const Geom &g = a.g;
    if ((variant != kZMarchTma && variant != kZMarchTmaFoldLoop) || mode == kModeAdjoint || a.bc != SIM_BC_CPML ||
        !a.ca[2] || !x_row_pass(g, nullptr))
        return X;
    X.lqb = g.nbx0 > 0 ? std::min(g.NX, g.nbx0 + 4) : 0;
    X.rqa = g.nbx1 > 0 ? std::max(0, g.NX - g.nbx1 - 4) : (1 << 30);
    const int last = ((g.NX - 1) / TX) * TX;
    X.on = X.lqb <= TX && (g.nbx1 == 0 || X.rqa >= last);
    return X;
}

bool zmarch_folds_x(const StepArgs<float> &a, int variant, int mode) { return x_fuse(a, variant, mode).on != 0; }

// Tensor maps of one launch (host): the pressure buffers pbuf[0] (both
// parities of max_shots shots, fstride apart) and c, in the padded layout.
cudaError_t make_maps(const StepArgs<float> &a, Tma3 &m) {
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    if (!enc) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return cudaErrorNotSupported;
        enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const Geom &g = a.g;
    const long long ms = (a.pbuf[1] - a.pbuf[0]) / g.fstride;
    const long long planes = g.fstride / ((long long)g.PY * g.P);
    // x extent: the ghost columns left of the grid, the grid and the 4 columns
    // of the last cells' halo; columns past it (the padding of the last x tile,
    // all zeros) come as the copy's zero fill instead of DRAM reads
    const cuuint64_t nxt = std::min<cuuint64_t>((cuuint64_t)g.P, (cuuint64_t)(kGhost + g.NX + 4));
    const cuuint64_t dims[4] = {nxt, (cuuint64_t)g.PY, (cuuint64_t)planes, (cuuint64_t)(2 * ms)};
    const cuuint64_t strides[3] = {(cuuint64_t)g.P * 4, (cuuint64_t)g.PY * g.P * 4, (cuuint64_t)g.fstride * 4};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    const cuuint32_t bh[4] = {TX + 8, 16, 1, 1}, bo[4] = {TX, 8, 1, 1};
    CUresult r = enc(&m.ph, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.pbuf[0], dims, strides, bh, one,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
        r = enc(&m.po, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.pbuf[0], dims, strides, bo, one,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
        r = enc(&m.c, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(a.ch), dims, strides, bo, one,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t configure_step3d() {
    cudaError_t e = cudaSuccess;
    for (auto k : {k_step3d_tma<kModeForward, 9>, k_step3d_tma<kModeRecord, 9>, k_step3d_tma<kModeAdjoint, 9>,
                   k_step3d_tma<kModeForward, 1>, k_step3d_tma<kModeRecord, 1>, k_step3d_tma<kModeAdjoint, 1>,
                   k_step3d_tma<kModeForward, 3>, k_step3d_tma<kModeRecord, 3>, k_step3d_tma<kModeAdjoint, 3>})
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTma);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step3d<1, kModeForward>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem3d<1>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step3d<1, kModeRecord>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem3d<1>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step3d<1, kModeAdjoint>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem3d<1>());
    return e;
}

template <int RY, int MODE>
cudaError_t launch_step3d_mode(cudaLaunchConfig_t &cfg, const StepArgs<float> &a, int n, int zchunk, float *qs,
                               float *Gs) {
    cfg.dynamicSmemBytes = smem3d<RY>();
    return cudaLaunchKernelEx(&cfg, k_step3d<RY, MODE>, a, n, zchunk, qs, Gs);
}

cudaError_t launch_step3d(const StepArgs<float> &a, int n, int variant, int zchunk, int nshots, cudaStream_t st,
                          bool pdl, int mode, float *qs, float *Gs) {
    const int nchunk = (a.g.NZ + zchunk - 1) / zchunk;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.ntx, (a.g.NY + NW - 1) / NW, nchunk * nshots);
    cfg.blockDim = dim3(NTH);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    if (variant >= kZMarchTma && variant <= kZMarchTmaLoop3) {
        Tma3 m;
        if (cudaError_t e = make_maps(a, m)) return e;
        cfg.dynamicSmemBytes = kSmemTma;
        const int ms = (int)((a.pbuf[1] - a.pbuf[0]) / a.g.fstride);
        const long long spin = 1LL << 22;
        const XFuse X = x_fuse(a, variant, mode);
        if (variant == kZMarchTmaLoop || variant == kZMarchTmaFoldLoop) {
            if (mode == kModeRecord)
                return cudaLaunchKernelEx(&cfg, k_step3d_tma<kModeRecord, 1>, a, m, n, zchunk, ms, X, qs, Gs, spin);
            if (mode == kModeAdjoint)
                return cudaLaunchKernelEx(&cfg, k_step3d_tma<kModeAdjoint, 1>, a, m, n, zchunk, ms, X, qs, Gs, spin);
            return cudaLaunchKernelEx(&cfg, k_step3d_tma<kModeForward, 1>, a, m, n, zchunk, ms, X, qs, Gs, spin);
        }
        if (variant == kZMarchTmaLoop3) {
            if (mode == kModeRecord)
                return cudaLaunchKernelEx(&cfg, k_step3d_tma<kModeRecord, 3>, a, m, n, zchunk, ms, X, qs, Gs, spin);
            if (mode == kModeAdjoint)
                return cudaLaunchKernelEx(&cfg, k_step3d_tma<kModeAdjoint, 3>, a, m, n, zchunk, ms, X, qs, Gs, spin);
            return cudaLaunchKernelEx(&cfg, k_step3d_tma<kModeForward, 3>, a, m, n, zchunk, ms, X, qs, Gs, spin);
        }
        if (mode == kModeRecord)
            return cudaLaunchKernelEx(&cfg, k_step3d_tma<kModeRecord, 9>, a, m, n, zchunk, ms, X, qs, Gs, spin);
        if (mode == kModeAdjoint)
            return cudaLaunchKernelEx(&cfg, k_step3d_tma<kModeAdjoint, 9>, a, m, n, zchunk, ms, X, qs, Gs, spin);
        return cudaLaunchKernelEx(&cfg, k_step3d_tma<kModeForward, 9>, a, m, n, zchunk, ms, X, qs, Gs, spin);
    }
    if (variant != kZMarchAsync) return cudaErrorInvalidValue;
    if (mode == kModeRecord) return launch_step3d_mode<1, kModeRecord>(cfg, a, n, zchunk, qs, Gs);
    if (mode == kModeAdjoint) return launch_step3d_mode<1, kModeAdjoint>(cfg, a, n, zchunk, qs, Gs);
    return launch_step3d_mode<1, kModeForward>(cfg, a, n, zchunk, qs, Gs);
}

cudaError_t launch_inj3d(const StepArgs<float> &a, int n, int row, const Inj3 *grp, int ngrp, const InjE3 *ent,
                         int kind, int nshots, int mode, float *qs, float *Gs, cudaStream_t st) {
    if (ngrp <= 0) return cudaSuccess;
    k_inj3d<<<dim3((ngrp + 127) / 128, nshots), 128, 0, st>>>(a, n, row, grp, ngrp, ent, kind, mode, qs, Gs);
    return cudaGetLastError();
}

// CPML of one axis, called with phase 0 before the update kernel and phase 1
// after it; with `qs` (record mode of the gradient) the addend is also taken
// off the step's imaging term, as it is part of the Laplacian there. The one-pass kernels (k_cpml_col3d for z / y, k_cpml_row3d for x)
// run at phase 1 and launch nothing at phase 0; strip layouts they do not
// take use k_psi3d at phase 0 (boxes = the two strips) and k_cpml_add3d at
// phase 1 (the strips widened by 4 cells along the axis).
cudaError_t launch_cpml3d(const StepArgs<float> &a, int n, int ax, int phase, int nshots, cudaStream_t st,
                          float *qs) {
    const Geom &g = a.g;
    const int N[3] = {g.NZ, g.NY, g.NX};
    const int lo[3] = {g.nbz0, g.nby0, g.nbx0}, hi[3] = {g.nbz1, g.nby1, g.nbx1};
    if (ax == 2) {  // x: one pass after the update (phase 1), when each widened strip spans <= 12 float4s
        XEnds E{};
        if (x_row_pass(g, &E)) {
            if (phase == 0) return cudaSuccess;
            const int m = E.ne;
            const long long nrows = (long long)g.NZ * g.NY, th = 16 * ((m * nrows + XR - 1) / XR);
            k_cpml_row3d<<<dim3((unsigned)((th + 127) / 128), nshots), 128, 0, st>>>(a, n, E, nrows, qs);
            return cudaGetLastError();
        }
    }
    if (ax != 2) {  // z or y: one marching pass after the update (phase 1), unless a z range nears a free surface
        ColRanges R{};
        const int l1 = lo[ax] > 0 ? std::min(N[ax], lo[ax] + 4) : 0;
        const int h0 = hi[ax] > 0 ? std::max(0, N[ax] - hi[ax] - 4) : N[ax];
        if (l1 > 0 && h0 < N[ax] && l1 >= h0) {
            R.n = 1;
            R.s0[0] = 0;
            R.s1[0] = N[ax];
        } else {
            if (l1 > 0) R.s0[R.n] = 0, R.s1[R.n++] = l1;
            if (h0 < N[ax]) R.s0[R.n] = h0, R.s1[R.n++] = N[ax];
        }
        const bool mirror = ax == 0 && g.fs && R.n > 0 && R.s0[0] < 4;
        if (!mirror) {
            if (phase == 0 || R.n == 0) return cudaSuccess;
            const int ncols = (ax == 0 ? g.NY : g.NZ) * ((g.NX + 3) >> 2);
            const long long th = (long long)R.n * ncols;
            k_cpml_col3d<<<dim3((unsigned)((th + 127) / 128), nshots), 128, 128 * CNS * 5 * sizeof(float4), st>>>(
                a, n, ax, R, ncols, qs);
            return cudaGetLastError();
        }
    }
    const int widen = phase == 0 ? 0 : 4;
    int a0 = 0, a1 = lo[ax] > 0 ? std::min(N[ax], lo[ax] + widen) : 0;
    int b0 = hi[ax] > 0 ? std::max(0, N[ax] - hi[ax] - widen) : N[ax], b1 = N[ax];
    if (a1 > b0) {  // strips meet: one box
        a1 = b1;
        b0 = b1;
    }
    Box B0{0, g.NZ, 0, g.NY, 0, g.NX}, B1 = B0;
    auto set = [&](Box &b, int s0, int s1) {
        if (ax == 0) { b.z0 = s0; b.z1 = s1; }
        else if (ax == 1) { b.y0 = s0; b.y1 = s1; }
        else { b.x0 = s0; b.x1 = s1; }
    };
    set(B0, a0, a1);
    set(B1, b0, b1);
    // float4 columns: x-ranges rounded out to multiples of 4; boxes that then
    // touch or overlap become one box (so no cell is updated twice)
    auto round4 = [](Box &b) {
        if (b.x1 <= b.x0) return;
        b.x0 = b.x0 & ~3;
        b.x1 = (b.x1 + 3) & ~3;
    };
    round4(B0);
    round4(B1);
    const bool empty0 = B0.z1 <= B0.z0 || B0.y1 <= B0.y0 || B0.x1 <= B0.x0;
    const bool empty1 = B1.z1 <= B1.z0 || B1.y1 <= B1.y0 || B1.x1 <= B1.x0;
    if (ax == 2 && !empty0 && !empty1 && B0.x1 >= B1.x0) {
        B0.x1 = B1.x1;
        B1 = Box{0, 0, 0, 0, 0, 0};
    }
    const long long items = (long long)(B0.z1 - B0.z0) * (B0.y1 - B0.y0) * ((B0.x1 - B0.x0) >> 2) +
                            (long long)(B1.z1 - B1.z0) * (B1.y1 - B1.y0) * ((B1.x1 - B1.x0) >> 2);
    if (items <= 0) return cudaSuccess;
    const int blocks = (int)std::min<long long>((items + 255) / 256, 152 * 16);
    if (phase == 0) k_psi3d<<<dim3(blocks, nshots), 256, 0, st>>>(a, n, ax, B0, B1);
    else k_cpml_add3d<<<dim3(blocks, nshots), 256, 0, st>>>(a, n, ax, B0, B1, qs);
    return cudaGetLastError();
}

cudaError_t launch_sample3d(const StepArgs<float> &a, const StepTime &t, const void *rec, int nrec, int nshots,
                            cudaStream_t st) {
    if (!rec || nrec <= 0) return cudaSuccess;
    const long long tot = (long long)nrec * nshots;
    k_sample3d<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(a, t, static_cast<const Pt3 *>(rec), nrec, nshots);
    return cudaGetLastError();
}

cudaError_t launch_inject3d(const StepArgs<float> &a, const StepTime &t, const void *src, int nshots,
                            cudaStream_t st) {
    if (!src || nshots <= 0) return cudaSuccess;
    k_inject3d<<<(8 * nshots + 63) / 64, 64, 0, st>>>(a, t, static_cast<const Pt3 *>(src), nshots);
    return cudaGetLastError();
}

cudaError_t launch_snap3d(const StepArgs<float> &a, const StepTime &t, int fp16, int nshots, cudaStream_t st) {
    if (fp16) {
        k_snap3d<<<dim3(608, nshots), 256, 0, st>>>(a, t, 1);
        k_snap3d<<<dim3(608, nshots), 256, 0, st>>>(a, t, 2);
    } else {
        k_snap3d<<<dim3(608, nshots), 256, 0, st>>>(a, t, 0);
    }
    return cudaGetLastError();
}

}  // namespace gsim
