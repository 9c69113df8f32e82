// Streaming FP32 2D forward step ("row march"): the same scheme and outputs as
// the tiled step kernel (8th-order Laplacian, leapfrog with the centred sponge
// term or CPML memory terms, free surface, point injection, receivers,
// snapshots), organised so that HBM never waits on arithmetic.
//
// Work layout: a warp owns a strip of 128 columns (lane l: the float4 of
// columns 4l .. 4l+3) and a contiguous range of rows [z0, z1) of one
// (slice, shot) member, and walks down the rows. Each warp keeps its own
// ring of rows in shared memory, filled by cp.async ahead of the output rows:
// p^n rows with their x halo, and per output row p^{n-1}, c (and the CPML
// memory it updates). The z-derivative slides down a register window; the
// x-derivative reads the lane's float4 and its two neighbours from the ring.
// Warps never wait on each other: the only waits are cp.async.wait_group on
// the warp's own copies, so every warp keeps rows in flight at all times.
//
// Two loops:
//  - sponge / no absorption: RB = 4 rows per iteration with a 12-row register
//    window (rows z-4 .. z+7), so the per-row bookkeeping (waits, copies,
//    list checks, window shifts) is shared by 16 cells per lane;
//  - CPML (items within 4 cells of a strip, on CPML slices): one row per
//    iteration with a 9-row window. psi_x is recomputed on the strip's 4-cell
//    chunks within x0-4 .. x0+131 from a halo-8 row (the x-derivative of psi_x
//    needs its neighbours), and psi_z^n at row r needs D1 p^n over rows r-4 .. r+4
//    while the update of row z needs psi_z^n at rows z-4 .. z+4, so psi_z runs
//    4 rows ahead of the output row (p^n staged 8 rows ahead) in a second
//    register window.
//
// Segments (member, strip, rows) are claimed by the warps from a per-step
// counter (16-row items, CPML items first); segment starts are multiples of
// 4 rows.
#include <cfloat>
#include <climits>

#include "f32_tile.cuh"
#include "sim_internal.h"
#include "stencil.cuh"

namespace gsim {
namespace {

using f32::cp_async16;
using f32::d1_pairs;
using f32::d1w;
using f32::d1x_pairs;
using f32::rec2;
using f32::d2_pairs;
using f32::d2w;
using f32::Pairs4;
using f32::plain1;
using f32::plain4;
using f32::lane_of;
using f32::ld4;
using f32::st4;
using f32::unpack3;

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// 16-byte global -> shared copy (shared address a) issued only where p holds,
// as a predicated instruction rather than a branch
__device__ __forceinline__ void cp16(unsigned a, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp16_if(unsigned a, const void *gmem, bool p) {
    asm volatile(
        "{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q cp.async.cg.shared.global [%0], [%1], 16;\n}\n" ::"r"(a),
        "l"(gmem), "r"((int)p)
        : "memory");
}
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ float4 neg4(const float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }

// psi_z^n = b psi_z^{n-1} + a D1_z p^n of the lane's four cells at a row r,
// from p^n at rows r-4 .. r-1 (m4 .. m1) and r+1 .. r+4 (p1 .. p4); zero in
// cells beyond the grid. One function for every row, so each cell gets the
// same arithmetic wherever its segment starts.
__device__ __forceinline__ float4 psi_z_row(const float4 &m4, const float4 &m3, const float4 &m2, const float4 &m1,
                                            const float4 &p1, const float4 &p2, const float4 &p3, const float4 &p4,
                                            const float4 &old, const float az, const float bz, const int gx0,
                                            const int NX) {
    float2 da, db;
    d1_pairs(m4, m3, m2, m1, p1, p2, p3, p4, da, db);
    const float2 a2 = rec2(splat2(az), da, splat2(bz), lo2(old)), b2 = rec2(splat2(az), db, splat2(bz), hi2(old));
    float o[4] = {a2.x, a2.y, b2.x, b2.y};
#pragma unroll
    for (int k = 0; k < 4; k++)
        if (gx0 + k >= NX) o[k] = 0.f;
    return make_float4(o[0], o[1], o[2], o[3]);
}

// ---------------------------------------------------------------- per-row I/O
//
// Receivers and injection groups come in the per-tile lists of the uniform
// 128 x tz tiling, sorted by row within a tile; a segment walks them with two
// cursors, reloaded whenever it enters a new tile row.
struct Lists {
    int tz0 = -1, rp = 0, re = 0, gp = 0, ge = 0;

    __device__ __forceinline__ void at(const StepArgs<float> &A, const MarchSeg &S, int tz, int z, bool rec,
                                       bool inj) {
        if (tz0 >= 0 && z - tz0 < tz) return;
        const int btz = z / tz;
        tz0 = btz * tz;
        const int tile = btz * A.ntx + S.bx, lz = z - tz0;
        // skip the entries of the tile's earlier rows (a segment may start
        // mid tile), 32 at a time: they form a prefix of the sorted list
        if (rec) {
            rp = A.rec_start[tile];
            re = A.rec_start[tile + 1];
            while (rp < re) {
                const int e = rp + (threadIdx.x & 31);
                const unsigned b = __ballot_sync(0xffffffffu, e < re && A.rec[e].lz < lz);
                rp += __popc(b);
                if (b != 0xffffffffu) break;
            }
        }
        if (inj) {
            const int it = A.inj_per_shot ? S.shot * (A.ntx * A.ntz) + tile : tile;
            gp = A.inj_start[it];
            ge = A.inj_start[it + 1];
            while (gp < ge) {
                const int e = gp + (threadIdx.x & 31);
                const unsigned b = __ballot_sync(0xffffffffu, e < ge && (A.inj_grp[e].cell >> 7) < lz);
                gp += __popc(b);
                if (b != 0xffffffffu) break;
            }
        }
    }
};

// receivers whose base cell is on row z sample p^n from the staged rows z
// (r0) and z + 1 (r1), cell x0 at r0[0]
__device__ __forceinline__ void sample_row(const StepArgs<float> &A, const StepTime &t, const MarchSeg &S, Lists &L,
                                           int lz, const float *r0, const float *r1, float *gout, int lane) {
    while (L.rp < L.re) {
        const int e = L.rp + lane;
        bool m = false;
        RecEntryT<float> R;
        if (e < L.re) {
            R = A.rec[e];
            m = R.lz == lz;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, m);
        if (m) {
            const float val = R.w[0] * r0[R.lx] + R.w[1] * r0[R.lx + 1] + R.w[2] * r1[R.lx] + R.w[3] * r1[R.lx + 1];
            gout[((long long)S.shot * A.nt + t.n) * A.io->nrec + R.rec] = val;
            if (!isfinite(val)) atomicOr(A.flags, kFlagUnstable);
        }
        const int cnt = __popc(bal);
        L.rp += cnt;
        if (cnt < 32) break;
    }
}

// injected values of row z, one group per target cell, into the lane's inj
__device__ __forceinline__ bool inject_row(const StepArgs<float> &A, const StepTime &t, const MarchSeg &S, Lists &L,
                                           int lz, float4 &inj, int lane) {
    bool any = false;
    while (L.gp < L.ge) {
        const InjGroup G = A.inj_grp[L.gp];
        if ((G.cell >> 7) != lz) break;
        float sum = 0.f;
        for (int e = G.e0; e < G.e1; e++) {
            const InjEntryT<float> E = A.inj_ent[e];
            const float val =
                A.inj_kind == 0
                    ? static_cast<const float *>(A.io->wavelet)[t.inj_row]
                    : static_cast<const float *>(A.io->resid)[((long long)S.shot * A.nt + t.inj_row) * A.io->nrec + E.pt];
            sum += E.w * val;
        }
        const int lx = G.cell & 127;
        if (lane == (lx >> 2)) {
            const int k = lx & 3;
            inj.x = k == 0 ? sum : inj.x;
            inj.y = k == 1 ? sum : inj.y;
            inj.z = k == 2 ? sum : inj.z;
            inj.w = k == 3 ? sum : inj.w;
        }
        any = true;
        L.gp++;
    }
    return any;
}

// Snapshot of p^n at this step (FP32, or FP16 with the scale of the previous
// step's maximum, published by each member's first segment), and the share of
// the next snapshot's FP16 scale (max |p^{n+1}| over interior cells).
struct Snap {
    void *out = nullptr;
    int fp16 = 0;
    float sinv = 1.f;
    long long base = 0;

    __device__ __forceinline__ void init(const StepArgs<float> &A, const StepTime &t, const MarchSeg &S, int lane) {
        if (t.snap_k < 0 && t.max_k < 0) return;
        const SimIO *io = A.io;
        out = io->snaps;
        fp16 = io->snap_fp16;
        if (t.snap_k >= 0 && out) {
            base = ((long long)S.shot * A.nsnap + t.snap_k) * A.g.nz * A.g.nx;
            if (fp16) {
                const float s = pow2_scale(__uint_as_float(io->snap_max[S.shot * A.nsnap + t.snap_k]));
                sinv = 1.f / s;
                if (S.bx == 0 && S.z0 == 0 && lane == 0) io->snap_scale[S.shot * A.nsnap + t.snap_k] = s;
            }
        }
    }
    __device__ __forceinline__ void row(const Geom &g, const StepTime &t, int z, int gx0, const float *p,
                                        const float *res, float &tmax) const {
        if (!out || z < g.oz || z >= g.oz + g.nz) return;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int gx = gx0 + k;
            if (gx < g.ox || gx >= g.ox + g.nx) continue;
            if (t.max_k >= 0) tmax = fmaxf(tmax, fabsf(res[k]));
            if (t.snap_k >= 0) {
                const long long si = base + (long long)(z - g.oz) * g.nx + (gx - g.ox);
                if (fp16) static_cast<__half *>(out)[si] = __float2half_rn(p[k] * sinv);
                else static_cast<float *>(out)[si] = p[k];
            }
        }
    }
    __device__ __forceinline__ void finish(const StepArgs<float> &A, const StepTime &t, const MarchSeg &S, float tmax,
                                           int lane) const {
        if (t.max_k < 0 || !fp16 || !out) return;
        const float m = warp_max(tmax);
        if (lane == 0) {
            if (!(m <= FLT_MAX)) atomicOr(A.flags, kFlagUnstable);
            else atomicMax(&A.io->snap_max[S.shot * A.nsnap + t.max_k], __float_as_uint(m));
        }
    }
};

// p^n rows z0-4 .. z0-1 of the lane's columns straight from HBM (odd mirror
// above a free surface)
__device__ __forceinline__ void rows_above(const Geom &g, const float *pc, int za, int gx0, float4 *w) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int r = za - 4 + k;
        w[k] = (r < 0 && g.fs) ? neg4(ld4(pc + (long long)(-r) * g.P + gx0)) : ld4(pc + (long long)r * g.P + gx0);
    }
}

// ---------------------------------------------------------------- sponge / none: 4 rows per iteration
struct LeanCfg {
    static constexpr int RB = 4;             // rows per iteration
    static constexpr int DB = 1;             // blocks of copies in flight beyond the two being read
    static constexpr int H = 4;              // x halo of a staged p^n row
    static constexpr int RW = kMarchW + 2 * H;
    static constexpr int NPB = DB + 2;       // p^n ring: blocks b, b+1 and DB in flight
    static constexpr int NOB = DB + 1;       // p^{n-1}, c ring
    static constexpr int PBF = RB * RW;      // floats per p^n block
    static constexpr int OBF = RB * 256;     // floats per output block (p^{n-1} row, c row)
    static constexpr int ARGS = 128;         // floats kept for the warp's copy of the slice arguments
    static constexpr int WF = ARGS + NPB * PBF + NOB * OBF;
    static_assert(NOB == 2, "the output ring alternates between two slots");
};

__device__ __forceinline__ void march_lean(const StepArgs<float> &A, const StepTime &t, const MarchSeg &S, int tz,
                                           float *W, int lane) {
    using C = LeanCfg;
    constexpr int RB = C::RB, DB = C::DB, H = C::H, RW = C::RW, NPB = C::NPB;
    // slice facts in registers: the copies' memory clobbers would otherwise
    // reload them from the shared-memory argument block on every row
    const int P = A.g.P, NX = A.g.NX, fs = A.g.fs;
    const int za = S.z0, zb = S.z1, x0 = S.bx * kMarchW, gx0 = x0 + 4 * lane;
    const int nb = (zb - za + RB - 1) / RB;  // blocks of output rows
    const long long base = (long long)S.shot * A.g.fstride + A.g.org;
    const float *pc = A.pbuf[t.n & 1] + base;  // p^n
    float *pn = A.pbuf[(t.n + 1) & 1] + base;  // p^{n-1} in, p^{n+1} out
    const bool sponge = A.bc == SIM_BC_SPONGE;
    const bool spx = sponge && ((A.g.nbx0 > 0 && x0 < A.g.nbx0) || (A.g.nbx1 > 0 && x0 + kMarchW > NX - A.g.nbx1));
    // rows [zs0, zs1) are free of z-sponge
    const int zs0 = sponge ? A.g.nbz0 : 0, zs1 = sponge ? A.g.NZ - A.g.nbz1 : A.g.NZ;
    const float *E0 = A.E[0];
    const float src_scale = A.src_scale;
    const bool inner = x0 + kMarchW <= NX;  // no lane beyond the grid
    const bool halo_lane = lane < RW / 4 - 32;
    // copy cursors: next p^n block and next output block to issue, and the
    // lane's shared-memory addresses of ring slot 0
    const long long blk = (long long)RB * P;
    const float *psrc = pc + (long long)za * P + x0 - H + 4 * lane;
    const float *osrc = pn + (long long)za * P + gx0;
    const float *csrc = A.ch + A.g.org + (long long)za * P + gx0;
    const unsigned pdst0 = (unsigned)__cvta_generic_to_shared(W) + 16u * lane;
    const unsigned odst0 = pdst0 + 4u * NPB * C::PBF;
    int kp = 0, ko = 0, sp = 0, so = 0;  // blocks issued, slots they go to

    auto issue_p = [&]() {  // the next p^n block (rows with the x halo), if the segment reads it
        if (kp <= nb) {
            const unsigned d = pdst0 + 4u * sp * C::PBF;
#pragma unroll
            for (int j = 0; j < RB; j++) {
                cp16(d + 4u * j * RW, psrc + (long long)j * P);
                cp16_if(d + 4u * (j * RW + 128), psrc + (long long)j * P + 128, halo_lane);
            }
        }
        kp++;
        psrc += blk;
        sp = sp == NPB - 1 ? 0 : sp + 1;
    };
    auto issue_o = [&]() {  // p^{n-1} and c of the next output block
        if (ko < nb) {
            const unsigned d = odst0 + 4u * so * C::OBF;
            const int left = zb - za - RB * ko;
            if (left >= RB) {
#pragma unroll
                for (int j = 0; j < RB; j++) {
                    cp16(d + 4u * j * 256, osrc + (long long)j * P);
                    cp16(d + 4u * (j * 256 + 128), csrc + (long long)j * P);
                }
            } else {
#pragma unroll
                for (int j = 0; j < RB; j++) {
                    cp16_if(d + 4u * j * 256, osrc + (long long)j * P, j < left);
                    cp16_if(d + 4u * (j * 256 + 128), csrc + (long long)j * P, j < left);
                }
            }
        }
        ko++;
        osrc += blk;
        csrc += blk;
        so = so == 1 ? 0 : 1;
    };

    // group 0: p^n blocks 0 and 1, outputs of block 0; group j: p^n block j + 1, outputs of block j
    issue_p();
#pragma unroll
    for (int j = 0; j <= DB; j++) {
        issue_p();
        issue_o();
        cp_commit();
    }
    float4 w[RB + 8];  // p^n rows z-4 .. z+RB+3 of the lane's columns
    rows_above(A.g, pc, za, gx0, w);

    float4 E4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (spx) E4 = __ldg(reinterpret_cast<const float4 *>(A.E[2] + gx0));
    float *gout = A.sample ? static_cast<float *>(A.io->gather) : nullptr;
    const bool has_inj = t.inj_row >= 0;
    Snap snap;
    snap.init(A, t, S, lane);
    float tmax = 0.f;
    Lists L;
    float *out_row = pn + (long long)za * P + gx0;
    const float *sb = W + H, *sn = W + C::PBF + H, *os = W + NPB * C::PBF;  // blocks b, b + 1; outputs of b
    int rb = 0;                                                              // ring slot of block b

    for (int b = 0; b < nb; b++) {
        cp_wait<DB>();
        __syncwarp();
        if (b == 0) {
#pragma unroll
            for (int j = 0; j < RB; j++) w[4 + j] = ld4(sb + j * RW + 4 * lane);
        }
#pragma unroll
        for (int j = 0; j < RB; j++) w[8 + j] = ld4(sn + j * RW + 4 * lane);
        const int z = za + RB * b;
        L.at(A, S, tz, z, gout != nullptr, has_inj);
        const bool lists = (gout && L.rp < L.re) || (has_inj && L.gp < L.ge);
        const bool full = z + RB <= zb;
        const bool spz = z < zs0 || z + RB > zs1;  // block touches a z-sponge row

        if (full && !lists && !snap.out && !spx && !spz && inner && !(fs && z == 0)) {
            // plain block: interior of the absorbing frame, nothing to sample,
            // inject or save; no branch per row
#pragma unroll
            for (int j = 0; j < RB; j++) {
                const float *row = sb + j * RW;
                const Pairs4 d = d2_pairs(ld4(row + 4 * lane - 4), w[4 + j], ld4(row + 4 * lane + 4), w + j);
                const float4 pp4 = ld4(os + j * 256 + 4 * lane), c4 = ld4(os + j * 256 + 128 + 4 * lane);
                st4(out_row, plain4(w[4 + j], pp4, c4, add2(d.za, d.xa), add2(d.zb, d.xb)));
                out_row += P;
            }
        } else {
#pragma unroll
            for (int j = 0; j < RB; j++) {
                const int zr = z + j;
                const bool live = full || zr < zb;
                const float *row = sb + j * RW;
                float v[12];
                unpack3(ld4(row + 4 * lane - 4), w[4 + j], ld4(row + 4 * lane + 4), v);
                const Pairs4 d = d2_pairs(ld4(row + 4 * lane - 4), w[4 + j], ld4(row + 4 * lane + 4), w + j);
                const float2 ra = add2(d.za, d.xa), rb = add2(d.zb, d.xb);
                const float r4[4] = {ra.x, ra.y, rb.x, rb.y};
                float4 inj = make_float4(0.f, 0.f, 0.f, 0.f);
                bool any_inj = false;
                if (lists && live) {
                    const int lz = zr - L.tz0;
                    if (gout) sample_row(A, t, S, L, lz, row, j + 1 < RB ? row + RW : sn, gout, lane);
                    if (has_inj) any_inj = inject_row(A, t, S, L, lz, inj, lane);
                }
                const float4 pp4 = ld4(os + j * 256 + 4 * lane), c4 = ld4(os + j * 256 + 128 + 4 * lane);
                const bool spg = spx || (sponge && (zr < zs0 || zr >= zs1));
                const float ez = spg ? __ldg(E0 + zr) : 0.f;
                float res[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    float rhs = r4[k];
                    if (any_inj) rhs += src_scale * lane_of(inj, k);
                    const float p = v[4 + k], pp = lane_of(pp4, k), chv = lane_of(c4, k);
                    float o;
                    if (spg) {
                        const float a = chv * (ez + lane_of(E4, k));
                        o = __fdividef(2.f * p - (1.f - a) * pp + chv * rhs, 1.f + a);
                    } else {
                        o = plain1(p, pp, chv, rhs);
                    }
                    res[k] = gx0 + k < NX ? o : 0.f;
                }
                if (fs && zr == 0) res[0] = res[1] = res[2] = res[3] = 0.f;
                if (live) {
                    st4(out_row, make_float4(res[0], res[1], res[2], res[3]));
                    snap.row(A.g, t, zr, gx0, v + 4, res, tmax);
                }
                out_row += P;
            }
        }

        // refill the slots this block freed, then slide the window and the ring
        __syncwarp();
        issue_p();
        issue_o();
        cp_commit();
#pragma unroll
        for (int k = 0; k < 8; k++) w[k] = w[k + RB];
        rb = rb == NPB - 1 ? 0 : rb + 1;
        sb = sn;
        sn = W + (rb == NPB - 1 ? 0 : rb + 1) * C::PBF + H;
        os = W + NPB * C::PBF + (os == W + NPB * C::PBF ? C::OBF : 0);
    }
    cp_wait<0>();
    __syncwarp();
    snap.finish(A, t, S, tmax, lane);
}

// ---------------------------------------------------------------- CPML: one row per iteration
struct CpmlCfg {
    static constexpr int LA = 8;   // p^n rows staged ahead of the output row
    static constexpr int D = 2;    // rows of copies in flight (a power of two)
    static constexpr int H = 8;    // x halo of a staged p^n row
    static constexpr int RW = kMarchW + 2 * H;
    static constexpr int NSP = 16;  // p^n ring slots: a power of two >= LA + D
    static_assert((NSP & (NSP - 1)) == 0 && NSP >= LA + D && (D & (D - 1)) == 0, "ring sizes");
    // output-row slot: p^{n-1}, c, psi_x^{n-1} (cells -4 .. 131), zeta_x,
    // zeta_z, psi_z^{n-1} of row z + 4
    static constexpr int O_PP = 0, O_C = 128, O_PSX = 256, O_ZX = 392, O_ZZ = 520, O_PSZ = 648;
    static constexpr int OW = 776;
    static constexpr int ARGS = 128;
    static constexpr int SCR = 136;
    static constexpr int WF = ARGS + NSP * RW + D * OW + SCR;
};

// Runs only on CPML slices (see cpml_segment). Every per-item constant the
// row loop needs (field pointers, strip bounds, the lane's x profile) is
// taken into registers first: the slice arguments live in shared memory and
// the cp.async statements clobber memory, so fields read in the loop would be
// reloaded after every copy.
__device__ __forceinline__ void march_cpml(const StepArgs<float> &A, const StepTime &t, const MarchSeg &S, int tz,
                                           float *W, int lane) {
    using C = CpmlCfg;
    constexpr int LA = C::LA, D = C::D, H = C::H, RW = C::RW, NSP = C::NSP, OW = C::OW;
    float *PR = W;             // NSP x RW
    float *OR = PR + NSP * RW; // D x OW
    float *SC = OR + D * OW;   // psi_x^n of the row, cells -4 .. 131
    const Geom &g = A.g;
    const int P = g.P, NX = g.NX, NZ = g.NZ;
    const bool fs = g.fs;
    const int za = S.z0, zb = S.z1, x0 = S.bx * kMarchW, gx0 = x0 + 4 * lane;
    const long long base = (long long)S.shot * g.fstride + g.org;
    const int par = t.n & 1;
    const float *pc = A.pbuf[par] + base;
    float *pn = A.pbuf[par ^ 1] + base;
    const float *chp = A.ch + g.org;
    const float src_scale = A.src_scale;

    // x strips: cells [0, nbx0) and [NX - nbx1, NX)
    const int nbx0 = g.nbx0, nbx1 = g.nbx1;
    const float *cax = A.ca[2], *cbx = A.cb[2];
    const bool cpx = cax != nullptr && ((nbx0 > 0 && x0 - 4 < nbx0) || (nbx1 > 0 && x0 + kMarchW + 4 > NX - nbx1));
    // psi_x^n is needed on cells x0 - 4 .. x0 + 131 (34 chunks of 4) and is
    // zero off the strips (a = b = 0 there): only chunks [cx0, cx1) meeting a
    // strip are recomputed and streamed, and of the row's own cells only the
    // float4s meeting a strip carry zeta_x
    int cx0 = 34, cx1 = 0;
    if (cpx) {
        if (nbx0 > 0 && x0 - 4 < nbx0) {
            cx0 = 0;
            cx1 = min(34, (nbx0 - 1 - (x0 - 4)) / 4 + 1);
        }
        const int xs = NX - nbx1;
        if (nbx1 > 0 && x0 + kMarchW + 4 > xs) {
            cx0 = min(cx0, max(0, xs - (x0 - 4)) / 4);
            cx1 = max(cx1, min(34, (NX - 1 - (x0 - 4)) / 4 + 1));
        }
    }
    const bool zxl = cpx && ((nbx0 > 0 && gx0 < nbx0) || (nbx1 > 0 && gx0 + 3 >= NX - nbx1));
    const bool cin0 = cx0 <= lane && lane < cx1, cin1 = lane < 2 && cx0 <= lane + 32 && lane + 32 < cx1;
    float *psx_n = nullptr, *zex = nullptr;
    const float *psx_o = nullptr;
    float4 ax4 = make_float4(0.f, 0.f, 0.f, 0.f), bx4 = ax4, ac4 = ax4, bc4 = ax4;
    if (cpx) {
        psx_n = A.psi[2][par] + base;
        psx_o = A.psi[2][par ^ 1] + base;
        zex = A.zeta[2] + base;
        ax4 = __ldg(reinterpret_cast<const float4 *>(cax + gx0));
        bx4 = __ldg(reinterpret_cast<const float4 *>(cbx + gx0));
        if (cx0 + lane < cx1) {  // the lane's chunk of the first recompute pass
            ac4 = __ldg(reinterpret_cast<const float4 *>(cax + x0 - 4 + 4 * (cx0 + lane)));
            bc4 = __ldg(reinterpret_cast<const float4 *>(cbx + x0 - 4 + 4 * (cx0 + lane)));
        }
    }
    // z strips: rows [0, zs0) and [zs1, NZ); zeta_z and the z addend matter
    // on rows < zn0 and >= zn1 (within 4 rows of a strip)
    const float *caz = A.ca[0], *cbz = A.cb[0];
    const bool cpz = caz != nullptr;
    const int zs0 = g.nbz0 > 0 ? g.nbz0 : 0, zs1 = g.nbz1 > 0 ? NZ - g.nbz1 : NZ;
    const int zn0 = zs0 > 0 ? zs0 + 4 : 0, zn1 = zs1 < NZ ? zs1 - 4 : INT_MAX;
    float *psz_n = nullptr, *zez = nullptr;
    const float *psz_o = nullptr;
    if (cpz) {
        psz_n = A.psi[0][par] + base;
        psz_o = A.psi[0][par ^ 1] + base;
        zez = A.zeta[0] + base;
    }
    auto zstrip = [&](int r) { return cpz && r >= 0 && r < NZ && (r < zs0 || r >= zs1); };
    auto znear = [&](int r) { return cpz && (r < zn0 || r >= zn1); };
    const int zlast = zb - 1 + LA;  // last p^n row the segment reads

    auto issue_p = [&](int r) {
        float *dst = PR + ((r - za) & (NSP - 1)) * RW;
        const float *src = pc + (long long)r * P + x0 - H;
        cp_async16(dst + 4 * lane, src + 4 * lane);
        if (lane < RW / 4 - 32) cp_async16(dst + 128 + 4 * lane, src + 128 + 4 * lane);
    };
    auto issue_o = [&](int z) {
        float *o = OR + ((z - za) & (D - 1)) * OW;
        const long long ro = (long long)z * P + gx0;
        cp_async16(o + C::O_PP + 4 * lane, pn + ro);
        cp_async16(o + C::O_C + 4 * lane, chp + ro);
        if (cpx) {
            const float *ps = psx_o + (long long)z * P + x0 - 4;
            cp16_if(smem_u32(o + C::O_PSX + 4 * lane), ps + 4 * lane, cin0);
            cp16_if(smem_u32(o + C::O_PSX + 128 + 4 * lane), ps + 128 + 4 * lane, cin1);
            cp16_if(smem_u32(o + C::O_ZX + 4 * lane), zex + ro, zxl);
        }
        if (zstrip(z)) cp_async16(o + C::O_ZZ + 4 * lane, zez + ro);
        if (zstrip(z + 4)) cp_async16(o + C::O_PSZ + 4 * lane, psz_o + ro + 4LL * P);
    };

    if (cpx) {  // chunks outside [cx0, cx1) read as zero in the psi_x^n row
        st4(SC + 4 * lane, make_float4(0.f, 0.f, 0.f, 0.f));
        if (lane < 2) st4(SC + 128 + 4 * lane, make_float4(0.f, 0.f, 0.f, 0.f));
    }
#pragma unroll
    for (int j = 0; j < D; j++) {
        if (j == 0) {
            for (int r = za; r <= za + LA; r++) issue_p(r);
        } else if (za + LA + j <= zlast) {
            issue_p(za + LA + j);
        }
        if (za + j < zb) issue_o(za + j);
        cp_commit();
    }
    float4 q[9];
    rows_above(g, pc, za, gx0, q);
    cp_wait<D - 1>();
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; k++) q[4 + k] = ld4(PR + k * RW + H + 4 * lane);

    // psi_z^n at rows z0-4 .. z0+3: the window the first update needs
    float4 qz[9];
#pragma unroll
    for (int k = 0; k < 9; k++) qz[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (cpz) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int r = za - 4 + k;
            if (zstrip(r)) {
                float4 pm[9];
#pragma unroll
                for (int m = 0; m < 9; m++) {
                    const int rr = r - 4 + m;
                    pm[m] = rr >= za ? ld4(PR + ((rr - za) & (NSP - 1)) * RW + H + 4 * lane)
                                     : ld4(pc + (long long)rr * P + gx0);
                }
                const float az = __ldg(caz + r), bz = __ldg(cbz + r);
                const float4 old = ld4(psz_o + (long long)r * P + gx0);
                qz[k] = psi_z_row(pm[0], pm[1], pm[2], pm[3], pm[5], pm[6], pm[7], pm[8], old, az, bz, gx0, NX);
                if (r >= za && r < zb) st4(psz_n + (long long)r * P + gx0, qz[k]);
            }
        }
    }

    float *gout = A.sample ? static_cast<float *>(A.io->gather) : nullptr;
    const bool has_inj = t.inj_row >= 0;
    Snap snap;
    snap.init(A, t, S, lane);
    float tmax = 0.f;
    Lists L;

    // psi_x^n of chunk c (cells x0 - 4 + 4c ..) from row z's p^n, into SC and,
    // for the row's own cells, into the field
    auto psi_chunk = [&](const float *rz, const float *pso, float *pw, int c, const float4 &a4, const float4 &b4) {
        const int gx = x0 - 4 + 4 * c;
        const float4 old = ld4(pso + 4 * c);
        float2 da, db;
        d1x_pairs(ld4(rz + 4 * c - 8), ld4(rz + 4 * c - 4), ld4(rz + 4 * c), da, db);
        const float2 pa = rec2(lo2(a4), da, lo2(b4), lo2(old)), pb = rec2(hi2(a4), db, hi2(b4), hi2(old));
        float o[4] = {pa.x, pa.y, pb.x, pb.y};
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (!(gx + k >= 0 && gx + k < NX)) o[k] = 0.f;
        const float4 o4 = make_float4(o[0], o[1], o[2], o[3]);
        st4(SC + 4 * c, o4);
        if (c >= 1 && c <= 32) st4(pw + gx, o4);
    };

    for (int z = za; z < zb; z++) {
        const int i = z - za;
        cp_wait<D - 1>();
        __syncwarp();
        const float *rz = PR + (i & (NSP - 1)) * RW + H;  // row z; cell x0 at rz[0]
        q[8] = ld4(PR + ((i + 4) & (NSP - 1)) * RW + H + 4 * lane);
        const float *os = OR + (i & (D - 1)) * OW;
        const long long ro = (long long)z * P + gx0;
        L.at(A, S, tz, z, gout != nullptr, has_inj);
        const int lzc = z - L.tz0;

        float v[12];
        unpack3(ld4(rz + 4 * lane - 4), q[4], ld4(rz + 4 * lane + 4), v);
        const Pairs4 dp = d2_pairs(ld4(rz + 4 * lane - 4), q[4], ld4(rz + 4 * lane + 4), q);
        const float d2x[4] = {dp.xa.x, dp.xa.y, dp.xb.x, dp.xb.y}, d2z[4] = {dp.za.x, dp.za.y, dp.zb.x, dp.zb.y};

        // CPML memory terms: the per-cell addend D1 psi^n + zeta^n of each axis
        float cadd[4] = {0.f, 0.f, 0.f, 0.f};
        if (cpx) {
            const float *pso = os + C::O_PSX;
            float *pw = psx_n + (long long)z * P;
            if (cx0 + lane < cx1) psi_chunk(rz, pso, pw, cx0 + lane, ac4, bc4);
            for (int c = cx0 + lane + 32; c < cx1; c += 32)
                psi_chunk(rz, pso, pw, c, __ldg(reinterpret_cast<const float4 *>(cax + x0 - 4 + 4 * c)),
                          __ldg(reinterpret_cast<const float4 *>(cbx + x0 - 4 + 4 * c)));
            __syncwarp();
            const float4 z4 = zxl ? ld4(os + C::O_ZX + 4 * lane) : make_float4(0.f, 0.f, 0.f, 0.f);
            float2 da, db;
            d1x_pairs(ld4(SC + 4 * lane), ld4(SC + 4 * lane + 4), ld4(SC + 4 * lane + 8), da, db);
            const float2 za = rec2(lo2(ax4), add2(dp.xa, da), lo2(bx4), lo2(z4));
            const float2 zb = rec2(hi2(ax4), add2(dp.xb, db), hi2(bx4), hi2(z4));
            const float2 ca = add2(da, za), cb = add2(db, zb);
            const float zo[4] = {za.x, za.y, zb.x, zb.y};
            cadd[0] += ca.x, cadd[1] += ca.y, cadd[2] += cb.x, cadd[3] += cb.y;
            if (zxl) st4(zex + ro, make_float4(zo[0], zo[1], zo[2], zo[3]));
        }
        if (cpz) {
            // psi_z^n of row z + 4 enters the window first: D1 over rows z .. z+8
            float4 nz4 = make_float4(0.f, 0.f, 0.f, 0.f);
            const int r = z + 4;
            if (zstrip(r)) {
                const float4 f5 = ld4(PR + ((i + 5) & (NSP - 1)) * RW + H + 4 * lane);
                const float4 f6 = ld4(PR + ((i + 6) & (NSP - 1)) * RW + H + 4 * lane);
                const float4 f7 = ld4(PR + ((i + 7) & (NSP - 1)) * RW + H + 4 * lane);
                const float4 f8 = ld4(PR + ((i + 8) & (NSP - 1)) * RW + H + 4 * lane);
                const float az = __ldg(caz + r), bz = __ldg(cbz + r);
                const float4 old = ld4(os + C::O_PSZ + 4 * lane);
                nz4 = psi_z_row(q[4], q[5], q[6], q[7], f5, f6, f7, f8, old, az, bz, gx0, NX);
                if (r < zb) st4(psz_n + ro + 4LL * P, nz4);
            }
            qz[8] = nz4;
            if (znear(z)) {
                const bool in = zstrip(z);
                float az = 0.f, bz = 0.f;
                float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (in) {
                    az = __ldg(caz + z);
                    bz = __ldg(cbz + z);
                    z4 = ld4(os + C::O_ZZ + 4 * lane);
                }
                float2 da, db;
                d1_pairs(qz[0], qz[1], qz[2], qz[3], qz[5], qz[6], qz[7], qz[8], da, db);
                const float2 za = rec2(splat2(az), add2(dp.za, da), splat2(bz), lo2(z4));
                const float2 zb = rec2(splat2(az), add2(dp.zb, db), splat2(bz), hi2(z4));
                const float2 ca = add2(da, za), cb = add2(db, zb);
                const float zo[4] = {za.x, za.y, zb.x, zb.y};
                cadd[0] += ca.x, cadd[1] += ca.y, cadd[2] += cb.x, cadd[3] += cb.y;
                if (in) st4(zez + ro, make_float4(zo[0], zo[1], zo[2], zo[3]));
            }
        }

        if (gout) sample_row(A, t, S, L, lzc, rz, PR + ((i + 1) & (NSP - 1)) * RW + H, gout, lane);
        float4 inj = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool any_inj = has_inj && inject_row(A, t, S, L, lzc, inj, lane);

        const float4 pp4 = ld4(os + C::O_PP + 4 * lane), c4 = ld4(os + C::O_C + 4 * lane);
        float res[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            float rhs = d2z[k] + d2x[k];
            rhs += cadd[k];
            if (any_inj) rhs += src_scale * lane_of(inj, k);
            const float out = plain1(v[4 + k], lane_of(pp4, k), lane_of(c4, k), rhs);
            res[k] = gx0 + k < NX ? out : 0.f;
        }
        if (fs && z == 0) res[0] = res[1] = res[2] = res[3] = 0.f;
        st4(pn + ro, make_float4(res[0], res[1], res[2], res[3]));
        snap.row(g, t, z, gx0, v + 4, res, tmax);

        __syncwarp();
        if (z + LA + D <= zlast) issue_p(z + LA + D);
        if (z + D < zb) issue_o(z + D);
        cp_commit();
#pragma unroll
        for (int k = 0; k < 8; k++) {
            q[k] = q[k + 1];
            qz[k] = qz[k + 1];
        }
    }
    cp_wait<0>();
    __syncwarp();
    snap.finish(A, t, S, tmax, lane);
}

static_assert(sizeof(StepArgs<float>) <= 4 * LeanCfg::ARGS && sizeof(StepArgs<float>) <= 4 * CpmlCfg::ARGS,
              "slice arguments fit the per-warp copy");
static_assert(sizeof(StepArgs<float>) % 8 == 0, "copied in 8-byte units");

template <bool CPML>
struct KCfg;
template <>
struct KCfg<false> {
    static constexpr int WPB = 4, MINB = 3, WF = LeanCfg::WF, ARGS = LeanCfg::ARGS;
};
template <>
struct KCfg<true> {  // both loops: CPML segments and the plain ones of CPML problems
    static constexpr int WPB = 4, MINB = 2, WF = CpmlCfg::WF > LeanCfg::WF ? CpmlCfg::WF : LeanCfg::WF,
                         ARGS = CpmlCfg::ARGS;
    static_assert(CpmlCfg::ARGS == LeanCfg::ARGS, "one argument block layout");
};

// Does the segment update CPML memory or need its addend? Its strip reaches
// within 4 cells of an x strip, or one of its rows within 4 rows of a z
// strip. Elsewhere psi and zeta are zero and stay zero, and the plain loop
// computes the same update.
__device__ __forceinline__ bool cpml_segment(const StepArgs<float> &A, const MarchSeg &S) {
    if (A.bc != SIM_BC_CPML) return false;
    const Geom &g = A.g;
    const int x0 = S.bx * kMarchW;
    if (A.ca[2] && ((g.nbx0 > 0 && x0 - 4 < g.nbx0) || (g.nbx1 > 0 && x0 + kMarchW + 4 > g.NX - g.nbx1))) return true;
    return A.ca[0] && ((g.nbz0 > 0 && S.z0 < g.nbz0 + 4) || (g.nbz1 > 0 && S.z1 > g.NZ - g.nbz1 - 4));
}

template <bool CPML>
__global__ void __launch_bounds__(KCfg<CPML>::WPB * 32, KCfg<CPML>::MINB) k_march2d(const MarchArgs M,
                                                                                     const StepTime t) {
    extern __shared__ float4 smem4[];
    using K = KCfg<CPML>;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * K::WPB + wib;
    if (gw >= M.nwarps) return;
    float *W = reinterpret_cast<float *>(smem4) + (size_t)wib * K::WF;
    const StepArgs<float> &A = *reinterpret_cast<const StepArgs<float> *>(W);
    int cur = -1;
    auto run = [&](const MarchSeg &S) {
        if (S.slice != cur) {  // the member's slice arguments, once per change of slice
            __syncwarp();
            const long long *src = reinterpret_cast<const long long *>(M.slices + S.slice);
            long long *dst = reinterpret_cast<long long *>(W);
            for (int k = lane; k < (int)(sizeof(StepArgs<float>) / 8); k += 32) dst[k] = src[k];
            __syncwarp();
            cur = S.slice;
        }
        if (CPML && cpml_segment(A, S)) march_cpml(A, t, S, M.tz, W + K::ARGS, lane);
        else march_lean(A, t, S, M.tz, W + K::ARGS, lane);
    };
    // segments in order from this step's counter, the next one claimed while
    // the current one runs; after the previous step is complete (every
    // counter use of it included), zero the next step's
    cudaGridDependencySynchronize();
    unsigned *ctr = M.ctr + (t.n & 1);
    if (gw == 0 && lane == 0) M.ctr[(t.n + 1) & 1] = 0u;
    unsigned next = 0;
    if (lane == 0) next = atomicAdd(ctr, 1u);
    next = __shfl_sync(0xffffffffu, next, 0);
    while (next < (unsigned)M.nitems) {
        const MarchSeg S = M.segs[next];
        if (lane == 0) next = atomicAdd(ctr, 1u);
        run(S);
        next = __shfl_sync(0xffffffffu, next, 0);
    }
}

template <bool CPML>
size_t march_smem() {
    return (size_t)KCfg<CPML>::WPB * KCfg<CPML>::WF * sizeof(float);
}

}  // namespace

cudaError_t configure_march2d() {
    cudaError_t e = cudaFuncSetAttribute(k_march2d<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)march_smem<false>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_march2d<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)march_smem<true>());
    return e;
}

int march2d_warps_per_sm(bool cpml) {
    int nb = 0;
    if (cpml) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_march2d<true>, KCfg<true>::WPB * 32, march_smem<true>());
        return nb * KCfg<true>::WPB;
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_march2d<false>, KCfg<false>::WPB * 32, march_smem<false>());
    return nb * KCfg<false>::WPB;
}

cudaError_t launch_march2d(const MarchArgs &m, bool cpml, const StepTime &t, cudaStream_t st, bool pdl) {
    if (m.nwarps < 1) return cudaSuccess;
    const int wpb = cpml ? KCfg<true>::WPB : KCfg<false>::WPB;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((m.nwarps + wpb - 1) / wpb);
    cfg.blockDim = dim3(wpb * 32);
    cfg.dynamicSmemBytes = cpml ? march_smem<true>() : march_smem<false>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    if (cpml) return cudaLaunchKernelEx(&cfg, k_march2d<true>, m, t);
    return cudaLaunchKernelEx(&cfg, k_march2d<false>, m, t);
}

}  // namespace gsim
