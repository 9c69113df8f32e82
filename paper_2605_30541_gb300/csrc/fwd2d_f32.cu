// FP32 2D time step, tuned for GB300: same scheme and outputs as the generic
// kernel in fwd2d.cu (8th-order Laplacian, leapfrog with the centred sponge
// term or CPML memory terms, free surface, point injection, receivers,
// snapshots, imaging-term record/adjoint modes).
//
// Work layout: a CTA of 8 warps owns a 128 x TZ tile (TZ = 8 RZ); each lane
// owns 4 consecutive x cells (one float4) in RZ consecutive rows. p^n and
// its radius-4 halo (radius 8 in CPML tiles) are staged into shared memory by
// cp.async, whole 512-byte rows per warp; the z-derivative slides down a
// register window of RZ + 8 float4 rows, the x-derivative reads the lane's
// float4 and its two neighbours. Per-step facts (snapshot index, injection
// row) arrive resolved from the host, offsets are 32-bit from per-CTA base
// pointers, and edge masks exist only in edge tiles, so the instruction count
// stays close to the stencil arithmetic itself.
//
// Everything that is fixed during a run (c field, profiles, point lists,
// injected values) is read before cudaGridDependencySynchronize(): with
// programmatic dependent launch that overlaps the previous step's tail.
#include <cfloat>

#include "sim_internal.h"
#include "stencil.cuh"

namespace gsim {
namespace {

constexpr int TX = kTileXF, HM = 8, SW = TX + 2 * HM;  // smem row stride (floats)
constexpr int NW = 8, NTH = NW * 32;

__device__ __forceinline__ float lane_of(const float4 &v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ float bmax(float v, float *red) {
    const int tid = threadIdx.x;
    v = warp_max(v);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    float m = tid < NW ? red[tid] : 0.f;
    if (tid < 32) m = warp_max(m);
    if (tid == 0) red[0] = m;
    __syncthreads();
    return red[0];
}

// second difference of the 12-float window v[0..11] at v[4 + k]
__device__ __forceinline__ float d2w(const float *v, int k) {
    return d2c<float>(v[4 + k], v[3 + k], v[5 + k], v[2 + k], v[6 + k], v[1 + k], v[7 + k], v[k], v[8 + k]);
}
// first difference of the 12-float window at v[4 + k]
__device__ __forceinline__ float d1w(const float *v, int k) {
    return float(kD1) * (v[5 + k] - v[3 + k]) + float(kD2) * (v[6 + k] - v[2 + k]) +
           float(kD3) * (v[7 + k] - v[1 + k]) + float(kD4) * (v[8 + k] - v[k]);
}
__device__ __forceinline__ void unpack3(const float4 &a, const float4 &b, const float4 &c, float *v) {
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    v[8] = c.x; v[9] = c.y; v[10] = c.z; v[11] = c.w;
}

template <int TZ>
constexpr size_t smem_floats(bool cpml) {
    return (size_t)(TZ + 2 * HM) * SW + (size_t)TZ * TX + (cpml ? (size_t)TZ * (TX + 8) + (size_t)(TZ + 8) * TX : 0);
}

// One tile of one step: the whole CTA updates the 128 x TZ tile (bx, bz) of
// `shot`. Shared by the per-step kernel (one tile per CTA) and the persistent
// batch kernel (a work list of tiles). With PDL the fields of the previous
// step are touched only after cudaGridDependencySynchronize().
template <int TZ, int MODE, bool PDL>
__device__ __forceinline__ void tile_step(const StepArgs<float> &A, const StepTime &t, const int bx, const int bz,
                                          const int shot, float *S, float *red) {
    constexpr int RZ = TZ / NW;
    float *INJ = S + (TZ + 2 * HM) * SW;           // TZ x TX
    float *PX = INJ + TZ * TX;                     // TZ x (TX + 8), CPML launches only
    float *PZ = PX + TZ * (TX + 8);                // (TZ + 8) x TX

    const Geom &g = A.g;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, tid = threadIdx.x;
    const int x0 = bx * TX, z0 = bz * TZ;
    const int tile = bz * A.ntx + bx;
    const int P = g.P;
    const long long sh = (long long)shot * g.fstride;
    const long long org = cell_off(g, z0, 0, x0);           // tile origin within one field
    const float *pcb = A.pbuf[t.n & 1] + sh + org;          // p^n
    float *pnb = A.pbuf[(t.n + 1) & 1] + sh + org;          // p^{n-1} in, p^{n+1} out
    const float *chb = A.ch + org;

    const bool cpml = A.bc == SIM_BC_CPML;
    const bool cpx = cpml && A.ca[2] &&
                     ((g.nbx0 > 0 && x0 - 4 < g.nbx0) || (g.nbx1 > 0 && x0 + TX + 4 > g.NX - g.nbx1));
    const bool cpz = cpml && A.ca[0] &&
                     ((g.nbz0 > 0 && z0 - 4 < g.nbz0) || (g.nbz1 > 0 && z0 + TZ + 4 > g.NZ - g.nbz1));
    const bool spg = A.bc == SIM_BC_SPONGE &&
                     ((g.nbx0 > 0 && x0 < g.nbx0) || (g.nbx1 > 0 && x0 + TX > g.NX - g.nbx1) ||
                      (g.nbz0 > 0 && z0 < g.nbz0) || (g.nbz1 > 0 && z0 + TZ > g.NZ - g.nbz1));
    const bool xedge = x0 + TX > g.NX;          // last tile column: mask cells beyond NX
    const bool zedge = z0 + TZ > g.NZ;          // last tile row: skip rows beyond NZ
    const bool top = g.fs && z0 == 0;           // free-surface tile
    const int H = (cpx || cpz) ? 8 : 4;
    const int c0 = HM + 4 * lane, gx0 = x0 + 4 * lane, rb = HM + w * RZ;
    const int lo = w * RZ * P + 4 * lane;       // offset of this thread's first float4 from the tile origin

    // ================= run constants: read before waiting for the previous step
    float4 ch4[RZ];
#pragma unroll
    for (int j = 0; j < RZ; j++) ch4[j] = __ldg(reinterpret_cast<const float4 *>(chb + lo + j * P));
    float4 E4 = make_float4(0, 0, 0, 0);
    if (spg) E4 = __ldg(reinterpret_cast<const float4 *>(A.E[2] + gx0));
    const int itile = A.inj_per_shot ? shot * (A.ntx * A.ntz) + tile : tile;
    const int g0 = A.inj_start[itile], g1 = A.inj_start[itile + 1];
    const bool has_inj = g1 > g0 && t.inj_row >= 0;
    if (has_inj) {  // injected values of this step, one thread per target cell
        for (int i = tid; i < TZ * TX / 4; i += NTH) reinterpret_cast<float4 *>(INJ)[i] = make_float4(0, 0, 0, 0);
        __syncthreads();
        const SimIO *io = A.io;
        for (int gi = g0 + tid; gi < g1; gi += NTH) {
            const InjGroup G = A.inj_grp[gi];
            float sum = 0.f;
            for (int e = G.e0; e < G.e1; e++) {
                const InjEntryT<float> E = A.inj_ent[e];
                const float val =
                    A.inj_kind == 0
                        ? static_cast<const float *>(io->wavelet)[t.inj_row]
                        : static_cast<const float *>(io->resid)[((long long)shot * A.nt + t.inj_row) * io->nrec + E.pt];
                sum += E.w * val;
            }
            INJ[G.cell] = sum;
        }
    }
    const int r0 = A.sample ? A.rec_start[tile] : 0, r1 = A.sample ? A.rec_start[tile + 1] : 0;

    // ================= the previous step's fields are needed from here on
    if (PDL) cudaGridDependencySynchronize();

    {   // stage p^n: TZ + 2H rows of TX + 2H floats
        const float *src = pcb - H * g.PY * P - H;
        float *dst = S + (HM - H) * SW + (HM - H);
        const bool wide = H == 8;
        for (int r = w; r < TZ + 2 * H; r += NW) {
            cp_async16(dst + r * SW + 4 * lane, src + r * P + 4 * lane);
            if (lane < (wide ? 4 : 2)) cp_async16(dst + r * SW + 128 + 4 * lane, src + r * P + 128 + 4 * lane);
        }
    }
    float4 pp4[RZ];
#pragma unroll
    for (int j = 0; j < RZ; j++) pp4[j] = ld4(pnb + lo + j * P);
    if (cpx) {  // old psi_x of rows [0, TZ) x cells [-4, TX + 4) into PX
        const float *po = A.psi[2][(t.n + 1) & 1] + sh + org;
#pragma unroll
        for (int j = 0; j < RZ; j++) {
            const int lz = w * RZ + j;
            cp_async16(PX + lz * (TX + 8) + 4 * lane, po + lz * P + 4 * lane - 4);
            if (lane < 2) cp_async16(PX + lz * (TX + 8) + 128 + 4 * lane, po + lz * P + 128 + 4 * lane - 4);
        }
    }
    if (cpz) {  // old psi_z of rows [-4, TZ + 4) x cells [0, TX) into PZ
        const float *po = A.psi[0][(t.n + 1) & 1] + sh + org;
#pragma unroll
        for (int j = 0; j < RZ + 1; j++) {
            const int lzz = -4 + w + NW * j;
            cp_async16(PZ + (lzz + 4) * TX + 4 * lane, po + lzz * P + 4 * lane);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (top) {  // odd mirror above the free surface: p(-k) = -p(k)
        const int nch = (TX + 2 * H) / 4;
        for (int k = 1 + w; k <= H; k += NW) {
            float4 *d = reinterpret_cast<float4 *>(S + (HM - k) * SW + (HM - H));
            const float4 *sr = reinterpret_cast<const float4 *>(S + (HM + k) * SW + (HM - H));
            for (int c = lane; c < nch; c += 32) {
                const float4 v = sr[c];
                d[c] = make_float4(-v.x, -v.y, -v.z, -v.w);
            }
        }
        __syncthreads();
    }

    // ================= CPML: psi^n = b psi^{n-1} + a D1 p^n on the tile +-4 cells (scaled by h)
    if (cpx) {
        float *pw = A.psi[2][t.n & 1] + sh + org;
#pragma unroll
        for (int j = 0; j < RZ; j++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int c = lane + 32 * h, lz = w * RZ + j, gz = z0 + lz, gx = x0 + 4 * c - 4;
                if (c >= (TX + 8) / 4) continue;
                const float *row = S + (HM + lz) * SW + HM + 4 * c - 4;
                float v[12];
                unpack3(ld4(row - 4), ld4(row), ld4(row + 4), v);
                const float4 a4 = __ldg(reinterpret_cast<const float4 *>(A.ca[2] + gx));
                const float4 b4 = __ldg(reinterpret_cast<const float4 *>(A.cb[2] + gx));
                float *px = PX + lz * (TX + 8) + 4 * c;
                const float4 old = ld4(px);
                float o4[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const bool in = gz < g.NZ && gx + k >= 0 && gx + k < g.NX;
                    o4[k] = in ? lane_of(b4, k) * lane_of(old, k) + lane_of(a4, k) * d1w(v, k) : 0.f;
                }
                const float4 o = make_float4(o4[0], o4[1], o4[2], o4[3]);
                st4(px, o);
                if (c >= 1 && c <= TX / 4 && gz < g.NZ) st4(pw + lz * P + 4 * c - 4, o);
            }
    }
    if (cpz) {
        float *pw = A.psi[0][t.n & 1] + sh + org;
#pragma unroll
        for (int j = 0; j < RZ + 1; j++) {
            const int lzz = -4 + w + NW * j, gz = z0 + lzz;
            const float *col = S + (HM + lzz) * SW + c0;
            float4 q[9];
#pragma unroll
            for (int m = 0; m < 9; m++) q[m] = ld4(col + (m - 4) * SW);
            const bool zin = gz >= 0 && gz < g.NZ;
            const float az = zin ? __ldg(A.ca[0] + gz) : 0.f, bz = zin ? __ldg(A.cb[0] + gz) : 0.f;
            float *pz = PZ + (lzz + 4) * TX + 4 * lane;
            const float4 old = ld4(pz);
            float o4[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float d1 = float(kD1) * (lane_of(q[5], k) - lane_of(q[3], k)) +
                                 float(kD2) * (lane_of(q[6], k) - lane_of(q[2], k)) +
                                 float(kD3) * (lane_of(q[7], k) - lane_of(q[1], k)) +
                                 float(kD4) * (lane_of(q[8], k) - lane_of(q[0], k));
                o4[k] = (zin && gx0 + k < g.NX) ? bz * lane_of(old, k) + az * d1 : 0.f;
            }
            const float4 o = make_float4(o4[0], o4[1], o4[2], o4[3]);
            st4(pz, o);
            if (lzz >= 0 && lzz < TZ && zin) st4(pw + lzz * P + 4 * lane, o);
        }
    }
    if (cpx || cpz || has_inj) __syncthreads();

    // CPML phase 2: zeta^n = b zeta^{n-1} + a (D2 p^n + D1 psi^n) on own cells, and
    // the per-cell addend D1 psi^n + zeta^n that the update adds to the Laplacian
    float4 cadd[RZ];
#pragma unroll
    for (int j = 0; j < RZ; j++) cadd[j] = make_float4(0, 0, 0, 0);
    if (cpx || cpz) {
#pragma unroll
        for (int j = 0; j < RZ; j++) {
            const int lz = w * RZ + j, gz = z0 + lz, o = lo + j * P;
            if (zedge && gz >= g.NZ) continue;
            float ad[4] = {0.f, 0.f, 0.f, 0.f};
            if (cpx) {
                float v[12], px[12];
                const float *row = S + (rb + j) * SW + c0;
                unpack3(ld4(row - 4), ld4(row), ld4(row + 4), v);
                const float *pr = PX + lz * (TX + 8) + 4 * lane;
                unpack3(ld4(pr), ld4(pr + 4), ld4(pr + 8), px);
                const float4 a4 = __ldg(reinterpret_cast<const float4 *>(A.ca[2] + gx0));
                const float4 b4 = __ldg(reinterpret_cast<const float4 *>(A.cb[2] + gx0));
                float *zp = A.zeta[2] + sh + org + o;
                const float4 z4 = ld4(zp);
                float zo[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float dps = d1w(px, k);
                    zo[k] = lane_of(b4, k) * lane_of(z4, k) + lane_of(a4, k) * (d2w(v, k) + dps);
                    ad[k] += dps + zo[k];
                }
                st4(zp, make_float4(zo[0], zo[1], zo[2], zo[3]));
            }
            if (cpz) {
                const float *col = S + (rb + j) * SW + c0;
                const float *pzc = PZ + (lz + 4) * TX + 4 * lane;
                const float az = __ldg(A.ca[0] + gz), bz = __ldg(A.cb[0] + gz);
                float *zp = A.zeta[0] + sh + org + o;
                const float4 z4 = ld4(zp);
                float zo[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    float cz[9], pz[9];
#pragma unroll
                    for (int m = 0; m < 9; m++) {
                        cz[m] = col[(m - 4) * SW + k];
                        pz[m] = pzc[(m - 4) * TX + k];
                    }
                    const float d2 = d2c<float>(cz[4], cz[3], cz[5], cz[2], cz[6], cz[1], cz[7], cz[0], cz[8]);
                    const float dps = float(kD1) * (pz[5] - pz[3]) + float(kD2) * (pz[6] - pz[2]) +
                                      float(kD3) * (pz[7] - pz[1]) + float(kD4) * (pz[8] - pz[0]);
                    zo[k] = bz * lane_of(z4, k) + az * (d2 + dps);
                    ad[k] += dps + zo[k];
                }
                st4(zp, make_float4(zo[0], zo[1], zo[2], zo[3]));
            }
            cadd[j] = make_float4(ad[0], ad[1], ad[2], ad[3]);
        }
    }

    // ================= receivers sample p^n
    if (r1 > r0) {
        float *gout = static_cast<float *>(A.io->gather);
        if (gout) {
            const long long rowo = ((long long)shot * A.nt + t.n) * A.io->nrec;
            for (int e = r0 + tid; e < r1; e += NTH) {
                const RecEntryT<float> R = A.rec[e];
                const float *b = S + (HM + R.lz) * SW + HM + R.lx;
                const float val = R.w[0] * b[0] + R.w[1] * b[1] + R.w[2] * b[SW] + R.w[3] * b[SW + 1];
                gout[rowo + R.rec] = val;
                if (!isfinite(val)) atomicOr(A.flags, kFlagUnstable);
            }
        }
    }

    // ================= snapshots: this step writes p^n (index snap_k); the
    // step before a snapshot folds max |p^{n+1}| into its FP16 scale
    void *snaps = nullptr;
    int fp16 = 0;
    float sinv = 1.f;
    long long sbase = 0;
    if (MODE == kModeForward && (t.snap_k >= 0 || t.max_k >= 0)) {
        const SimIO *io = A.io;
        snaps = io->snaps;
        fp16 = io->snap_fp16;
        if (t.snap_k >= 0 && snaps) {
            sbase = ((long long)shot * A.nsnap + t.snap_k) * g.nz * g.nx;
            if (fp16) {
                const float s = pow2_scale(__uint_as_float(io->snap_max[shot * A.nsnap + t.snap_k]));
                sinv = 1.f / s;
                if (bx == 0 && bz == 0 && tid == 0) io->snap_scale[shot * A.nsnap + t.snap_k] = s;
            }
        }
    }
    const bool snap_io = MODE == kModeForward && snaps != nullptr;
    const int ntiles = A.ntx * A.ntz;
    const float qs = (MODE == kModeAdjoint && A.q_fp16) ? t.qscale[shot * ntiles + tile] : 1.f;

    // ================= update
    float4 zw[RZ + 8];
#pragma unroll
    for (int j = 0; j < RZ + 8; j++) zw[j] = ld4(S + (rb - 4 + j) * SW + c0);
    float tmax = 0.f;
    float4 qv[RZ];
#pragma unroll
    for (int j = 0; j < RZ; j++) {
        qv[j] = make_float4(0, 0, 0, 0);
        const int lz = w * RZ + j, gz = z0 + lz;
        if (zedge && gz >= g.NZ) continue;
        const int o = lo + j * P;
        float v[12];
        unpack3(ld4(S + (rb + j) * SW + c0 - 4), zw[j + 4], ld4(S + (rb + j) * SW + c0 + 4), v);
        // second differences in FP32 pairs (the bits of d2w / d2c cell by cell)
        float2 dxa, dxb, dza, dzb;
        {
            const float4 L = ld4(S + (rb + j) * SW + c0 - 4), C = zw[j + 4], R = ld4(S + (rb + j) * SW + c0 + 4);
            const float2 v34 = make_float2(L.w, C.x), v56 = make_float2(C.y, C.z), v12 = make_float2(L.y, L.z),
                         v78 = make_float2(C.w, R.x), v910 = make_float2(R.y, R.z);
            dxa = d2c2(lo2(C), v34, v56, hi2(L), hi2(C), v12, v78, lo2(L), lo2(R));
            dxb = d2c2(hi2(C), v56, v78, lo2(C), lo2(R), v34, v910, hi2(L), hi2(R));
            const float4 *q = zw + j;
            dza = d2c2(lo2(C), lo2(q[3]), lo2(q[5]), lo2(q[2]), lo2(q[6]), lo2(q[1]), lo2(q[7]), lo2(q[0]), lo2(q[8]));
            dzb = d2c2(hi2(C), hi2(q[3]), hi2(q[5]), hi2(q[2]), hi2(q[6]), hi2(q[1]), hi2(q[7]), hi2(q[0]), hi2(q[8]));
        }
        const float d2xs[4] = {dxa.x, dxa.y, dxb.x, dxb.y}, d2zs[4] = {dza.x, dza.y, dzb.x, dzb.y};
        float res[4], qk[4];
        float4 inj4 = make_float4(0, 0, 0, 0), ext4 = make_float4(0, 0, 0, 0);
        if (has_inj) inj4 = ld4(INJ + lz * TX + 4 * lane);
        if (MODE == kModeAdjoint && A.cext) ext4 = ld4(A.cext + sh + org + o);
        const float ez = spg ? A.E[0][gz] : 0.f;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float p = v[4 + k];
            float rhs = d2zs[k] + d2xs[k];
            if (cpx || cpz) rhs += lane_of(cadd[j], k);
            if (MODE == kModeAdjoint && A.cext) rhs += lane_of(ext4, k);
            if (has_inj) rhs += A.src_scale * lane_of(inj4, k);
            const float chv = lane_of(ch4[j], k), pp = lane_of(pp4[j], k);
            float out, es = 0.f;
            if (spg) {
                es = ez + lane_of(E4, k);
                const float a = chv * es;
                out = (2.f * p - (1.f - a) * pp + chv * rhs) / (1.f + a);
            } else {
                out = 2.f * p - pp + chv * rhs;
            }
            res[k] = out;
            qk[k] = es * (out - pp) - rhs;
        }
        if (xedge) {
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (gx0 + k >= g.NX) res[k] = 0.f;
        }
        if (top && lz == 0) res[0] = res[1] = res[2] = res[3] = 0.f;
        st4(pnb + o, make_float4(res[0], res[1], res[2], res[3]));
        if (MODE == kModeRecord) {
            qv[j] = make_float4(qk[0], qk[1], qk[2], qk[3]);
            if (A.q_fp16)
                tmax = fmaxf(tmax, fmaxf(fmaxf(fabsf(qk[0]), fabsf(qk[1])), fmaxf(fabsf(qk[2]), fabsf(qk[3]))));
            else
                st4(static_cast<float *>(t.qslot) + sh + org + o, qv[j]);
        }
        if (MODE == kModeAdjoint) {
            float4 q;
            if (A.q_fp16) {
                const __half2 *hq =
                    reinterpret_cast<const __half2 *>(static_cast<const __half *>(t.qslot) + sh + org + o);
                const float2 a = __half22float2(hq[0]), b = __half22float2(hq[1]);
                q = make_float4(a.x * qs, a.y * qs, b.x * qs, b.y * qs);
            } else {
                q = ld4(static_cast<const float *>(t.qslot) + sh + org + o);
            }
            float *gp = A.G + sh + org + o;
            float4 gv = ld4(gp);
            gv.x += res[0] * q.x;
            gv.y += res[1] * q.y;
            gv.z += res[2] * q.z;
            gv.w += res[3] * q.w;
            st4(gp, gv);
        }
        if (snap_io && gz >= g.oz && gz < g.oz + g.nz) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int gx = gx0 + k;
                if (gx < g.ox || gx >= g.ox + g.nx) continue;
                if (t.max_k >= 0) tmax = fmaxf(tmax, fabsf(res[k]));
                if (t.snap_k >= 0) {
                    const long long si = sbase + (long long)(gz - g.oz) * g.nx + (gx - g.ox);
                    if (fp16) static_cast<__half *>(snaps)[si] = __float2half_rn(v[4 + k] * sinv);
                    else static_cast<float *>(snaps)[si] = v[4 + k];
                }
            }
        }
    }

    // FP16 imaging term: one power-of-two scale per tile and step
    if (MODE == kModeRecord && A.q_fp16) {
        const float s = pow2_scale(bmax(tmax, red)), inv = 1.f / s;
        if (tid == 0) t.qscale[shot * ntiles + tile] = s;
#pragma unroll
        for (int j = 0; j < RZ; j++) {
            if (zedge && z0 + w * RZ + j >= g.NZ) continue;
            __half2 *hq = reinterpret_cast<__half2 *>(static_cast<__half *>(t.qslot) + sh + org + lo + j * P);
            hq[0] = __floats2half2_rn(qv[j].x * inv, qv[j].y * inv);
            hq[1] = __floats2half2_rn(qv[j].z * inv, qv[j].w * inv);
        }
    }

    // block max of p^{n+1} for the next snapshot's FP16 scale
    if (MODE == kModeForward && t.max_k >= 0 && fp16 && snaps) {
        const float m = bmax(tmax, red);
        if (tid == 0) {
            if (!(m <= FLT_MAX)) atomicOr(A.flags, kFlagUnstable);
            else atomicMax(&A.io->snap_max[shot * A.nsnap + t.max_k], __float_as_uint(m));
        }
    }
}

template <int TZ, int MODE>
__global__ void __launch_bounds__(NTH, 2) k_step2d_f32(const StepArgs<float> A, const StepTime t) {
    extern __shared__ float4 smem4[];
    __shared__ float red[NW];
    tile_step<TZ, MODE, true>(A, t, blockIdx.x, blockIdx.y, blockIdx.z, reinterpret_cast<float *>(smem4), red);
}

// ---------------------------------------------------------------- batch
//
// Persistent dataflow execution of many shots on many grids. Work items are
// (group, step, member, tile), taken in order from a global counter; a group
// is a set of (slice, shot) members whose fields fit in L2 together, so a
// group advances through all its steps while resident. An item waits until
// its own tile and the 8 neighbouring tiles of its shot (earlier items, maybe
// on other CTAs) have finished the previous step
// (per-tile step counters, acquire/release), which also guarantees that none
// of them still reads the buffer it is about to overwrite. Every item was
// queued after the items it waits on, so progress never depends on which
// CTAs are resident. Each wait is bounded: on timeout the kernel raises a
// flag and every CTA returns.
__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

template <int TZ>
__global__ void __launch_bounds__(NTH, 2) k_batch2d(const BatchArgs B) {
    extern __shared__ float4 smem4[];
    __shared__ float red[NW];
    __shared__ StepArgs<float> sA;
    __shared__ long long s_item;
    __shared__ int s_abort, s_slice;
    const int tid = threadIdx.x;
    if (tid == 0) s_slice = -1;
    for (;;) {
        if (tid == 0) {
            s_item = (long long)atomicAdd(B.head, 1ULL);
            s_abort = (*reinterpret_cast<volatile unsigned *>(B.flags) & kFlagTimeout) != 0;
        }
        __syncthreads();
        const long long i = s_item;
        if (i >= B.total || s_abort) return;
        int gi = 0;
        while (gi + 1 < B.ngroups && B.groups[gi + 1].base <= i) gi++;
        const BatchGroup G = B.groups[gi];
        const long long r = i - G.base;
        const int n = (int)(r / G.T), ri = (int)(r % G.T);
        int lo = G.m0, hi = G.m1 - 1;  // member whose tile range holds ri
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.members[mid].tile0 <= ri) lo = mid;
            else hi = mid - 1;
        }
        const BatchMember M = B.members[lo];
        if (M.slice != s_slice) {  // the member's grid arguments, once per change of grid
            __syncthreads();
            static_assert(sizeof(StepArgs<float>) % 8 == 0, "copied in 8-byte units");
            const long long *src = reinterpret_cast<const long long *>(B.slices + M.slice);
            long long *dst = reinterpret_cast<long long *>(&sA);
            for (int k = tid; k < (int)(sizeof(StepArgs<float>) / 8); k += NTH) dst[k] = src[k];
            if (tid == 0) s_slice = M.slice;
            __syncthreads();
        }
        const int tile = ri - M.tile0, ntx = sA.ntx, ntz = sA.ntz;
        const int bz = tile / ntx, bx = tile - bz * ntx;
        int *done = B.done + M.done0;
        if (n > 0 && tid < 32) {  // wait for the tile and its 8 neighbours to finish step n-1
            const int dz = tid / 3 - 1, dx = tid % 3 - 1;
            const int nz = bz + dz, nx = bx + dx;
            bool need = tid < 9 && nz >= 0 && nz < ntz && nx >= 0 && nx < ntx;
            long long spins = 0;
            while (__any_sync(0xffffffffu, need)) {
                if (need && ld_acquire(done + nz * ntx + nx) >= n) need = false;
                if (++spins > B.spin_limit) {
                    if (tid == 0) atomicOr(B.flags, kFlagTimeout);
                    break;
                }
                if (need) __nanosleep(32);
                if ((spins & 1023) == 0 && (*reinterpret_cast<volatile unsigned *>(B.flags) & kFlagTimeout)) break;
            }
            if (tid == 0) s_abort = (*reinterpret_cast<volatile unsigned *>(B.flags) & kFlagTimeout) != 0;
        }
        __syncthreads();
        if (s_abort) return;
        StepTime t{};
        t.n = n;
        t.snap_k = t.max_k = -1;
        t.inj_row = n;
        tile_step<TZ, kModeForward, false>(sA, t, bx, bz, M.shot, reinterpret_cast<float *>(smem4), red);
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            st_release(done + tile, n + 1);
        }
    }
}

// ---------------------------------------------------------------- stepped batch
//
// One step of every (slice, shot) member of a batch in one launch: block i
// updates tile i - tile0 of the member whose tile range holds i (members
// sorted by tile0), with that slice's arguments. A kernel boundary per step
// orders the steps, so no waits are needed; launched with programmatic
// dependent launch, the member lookup and the slice's run constants overlap
// the previous step's tail.
template <int TZ>
__global__ void __launch_bounds__(NTH, 2) k_multi2d(const BatchArgs B, const int n) {
    extern __shared__ float4 smem4[];
    __shared__ float red[NW];
    __shared__ StepArgs<float> sA;
    __shared__ int s_m;
    const int tid = threadIdx.x, i = blockIdx.x;
    if (tid == 0) {
        int lo = 0, hi = B.nmembers - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (B.members[mid].tile0 <= i) lo = mid;
            else hi = mid - 1;
        }
        s_m = lo;
    }
    __syncthreads();
    const BatchMember M = B.members[s_m];
    static_assert(sizeof(StepArgs<float>) % 8 == 0, "copied in 8-byte units");
    const long long *src = reinterpret_cast<const long long *>(B.slices + M.slice);
    long long *dst = reinterpret_cast<long long *>(&sA);
    for (int k = tid; k < (int)(sizeof(StepArgs<float>) / 8); k += NTH) dst[k] = src[k];
    __syncthreads();
    const int tile = i - M.tile0, bz = tile / sA.ntx, bx = tile - bz * sA.ntx;
    StepTime t{};
    t.n = n;
    t.snap_k = t.max_k = -1;
    t.inj_row = n;
    tile_step<TZ, kModeForward, true>(sA, t, bx, bz, M.shot, reinterpret_cast<float *>(smem4), red);
}

template <int TZ, int MODE>
cudaError_t launch_mode(const StepArgs<float> &a, const StepTime &t, int nshots, cudaStream_t st, bool pdl) {
    const bool cp = a.bc == SIM_BC_CPML;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.ntx, a.ntz, nshots);
    cfg.blockDim = dim3(NTH);
    cfg.dynamicSmemBytes = smem_floats<TZ>(cp) * sizeof(float);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_step2d_f32<TZ, MODE>, a, t);
}

template <int TZ, int MODE>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(k_step2d_f32<TZ, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(smem_floats<TZ>(true) * sizeof(float)));
}

template <int TZ>
cudaError_t configure_tz() {
    cudaError_t e = configure_one<TZ, kModeForward>();
    if (e == cudaSuccess) e = configure_one<TZ, kModeRecord>();
    if (e == cudaSuccess) e = configure_one<TZ, kModeAdjoint>();
    return e;
}

template <int TZ>
cudaError_t launch_tz(const StepArgs<float> &a, const StepTime &t, int nshots, int mode, cudaStream_t st, bool pdl) {
    if (mode == kModeRecord) return launch_mode<TZ, kModeRecord>(a, t, nshots, st, pdl);
    if (mode == kModeAdjoint) return launch_mode<TZ, kModeAdjoint>(a, t, nshots, st, pdl);
    return launch_mode<TZ, kModeForward>(a, t, nshots, st, pdl);
}

}  // namespace

// Shared-memory opt-in of every instantiation; call once per device before
// any launch (and before any stream capture).
cudaError_t configure_step2d_f32() {
    cudaError_t e = configure_tz<8>();
    if (e == cudaSuccess) e = configure_tz<16>();
    if (e == cudaSuccess) e = configure_tz<32>();
    for (int tz : {8, 16, 32}) {
        if (e != cudaSuccess) break;
        const int bytes = (int)(tz == 8 ? smem_floats<8>(true) : tz == 16 ? smem_floats<16>(true) : smem_floats<32>(true)) *
                          (int)sizeof(float);
        e = tz == 8 ? cudaFuncSetAttribute(k_batch2d<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
            : tz == 16 ? cudaFuncSetAttribute(k_batch2d<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
                       : cudaFuncSetAttribute(k_batch2d<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = tz == 8 ? cudaFuncSetAttribute(k_multi2d<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
                : tz == 16 ? cudaFuncSetAttribute(k_multi2d<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
                           : cudaFuncSetAttribute(k_multi2d<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    }
    return e;
}

cudaError_t launch_multi2d(const BatchArgs &b, int tz, bool cpml, int nblocks, int n, cudaStream_t st, bool pdl) {
    const size_t bytes = (tz == 8 ? smem_floats<8>(cpml) : tz == 16 ? smem_floats<16>(cpml) : smem_floats<32>(cpml)) *
                         sizeof(float);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(NTH);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    if (tz == 8) return cudaLaunchKernelEx(&cfg, k_multi2d<8>, b, n);
    if (tz == 16) return cudaLaunchKernelEx(&cfg, k_multi2d<16>, b, n);
    if (tz == 32) return cudaLaunchKernelEx(&cfg, k_multi2d<32>, b, n);
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch2d(const BatchArgs &b, int tz, bool cpml, int grid, cudaStream_t st) {
    const size_t bytes = (tz == 8 ? smem_floats<8>(cpml) : tz == 16 ? smem_floats<16>(cpml) : smem_floats<32>(cpml)) *
                         sizeof(float);
    if (tz == 8) k_batch2d<8><<<grid, NTH, bytes, st>>>(b);
    else if (tz == 16) k_batch2d<16><<<grid, NTH, bytes, st>>>(b);
    else if (tz == 32) k_batch2d<32><<<grid, NTH, bytes, st>>>(b);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

int batch_blocks_per_sm(int tz, bool cpml) {
    int nb = 0;
    const size_t bytes = (tz == 8 ? smem_floats<8>(cpml) : tz == 16 ? smem_floats<16>(cpml) : smem_floats<32>(cpml)) *
                         sizeof(float);
    if (tz == 8) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch2d<8>, NTH, bytes);
    else if (tz == 16) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch2d<16>, NTH, bytes);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch2d<32>, NTH, bytes);
    return nb;
}

cudaError_t launch_step2d_f32(const StepArgs<float> &a, const StepTime &t, int tz, int nshots, int mode,
                              cudaStream_t st, bool pdl) {
    switch (tz) {
        case 8: return launch_tz<8>(a, t, nshots, mode, st, pdl);
        case 16: return launch_tz<16>(a, t, nshots, mode, st, pdl);
        case 32: return launch_tz<32>(a, t, nshots, mode, st, pdl);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gsim
