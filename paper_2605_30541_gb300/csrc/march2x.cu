// Temporal blocking of the 2D row march: two time steps per pass over HBM.
//
// The one-step row march reads p^n, p^{n-1} and c and writes p^{n+1}: 16 B
// per cell and step. Here one pass computes p^{n+1} and p^{n+2}: it reads
// p^n, p^{n-1} and c once and writes p^{n+1} and p^{n+2}, 20 B per cell for
// two steps (10 B per cell-step). The price is redundant arithmetic on a
// 4-cell ring around each warp's item: p^{n+1} is computed on the item
// widened by 4 cells in x and z (the stencil radius), so that p^{n+2} on the
// item needs nothing from other warps.
//
// Work layout: a warp owns a strip of 120 output columns x0 .. x0+119 (x0 a
// multiple of 120) and a run of rows [z0, z1) of one member (slice, shot).
// Lane l holds the float4 of columns x0 - 4 + 4l: lanes 1 .. 30 are the
// strip, lanes 0 and 31 its 4-cell x ring. The warp walks down the rows r =
// z0 - 4 .. z1 + 3: p^{n+1} of row r (every lane) from a 9-row register
// window of p^n and the x neighbours of a shared-memory ring (p^n rows with
// an 8-cell x halo, staged by cp.async ahead of use), and 4 rows behind it
// p^{n+2} of row r - 4 (lanes 1 .. 30) from a 9-row register window of
// p^{n+1}, whose x neighbours come from the adjacent lanes by shuffles.
//
// Buffers: four pressure fields per shot, two pairs. Every warp reads p^n
// AND p^{n-1} on its widened item, so a pass may overwrite neither: pass k
// (steps n = 2k, 2k + 1) reads p^n and p^{n-1} from one pair and writes
// p^{n+1} and p^{n+2} into the other (even passes read fields 0, 1 and write
// 3, 2; odd passes read 2, 3 and write 1, 0). A pass with one step (the last
// one when nt is odd) writes p^{n+1} only.
//
// Each cell's arithmetic is the one-step march's (the same expressions in
// the same order: second differences, sponge update, injection, mirror), so
// both give the same bits. Sponge or no absorption, free surface or not,
// point sources; receivers are sampled by a small kernel after each pass
// (rows n and n + 1 from buffers that are still intact). CPML slices and
// snapshots take the one-step march.
#include <cfloat>

#include "f32_tile.cuh"
#include "sim_internal.h"
#include "stencil.cuh"

namespace gsim {
namespace {

using f32::d2_pairs;
using f32::Pairs4;
using f32::plain1;
using f32::plain4;
using f32::lane_of;
using f32::ld4;
using f32::st4;
using f32::unpack3;

constexpr int NW2 = 4;        // warps per CTA
constexpr int NS2 = 8;        // ring rows per field (a power of two: slots are row & (NS2 - 1))
constexpr int D2 = 3;         // rows staged ahead of use
constexpr int PNW = 136;      // staged p^n row: columns x0 - 8 .. x0 + 127
constexpr int OW = 128;       // staged p^{n-1} / c row: columns x0 - 4 .. x0 + 123
constexpr int WARPF = NS2 * (PNW + 2 * OW);  // floats per warp

__device__ __forceinline__ void cp16_if(unsigned a, const void *gmem, bool p) {
    asm volatile(
        "{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q cp.async.cg.shared.global [%0], [%1], 16;\n}\n" ::"r"(a),
        "l"(gmem), "r"((int)p)
        : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ float4 neg4(const float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }
__device__ __forceinline__ float4 shfl4(const float4 v, bool up) {
    float4 r;
    r.x = up ? __shfl_up_sync(0xffffffffu, v.x, 1) : __shfl_down_sync(0xffffffffu, v.x, 1);
    r.y = up ? __shfl_up_sync(0xffffffffu, v.y, 1) : __shfl_down_sync(0xffffffffu, v.y, 1);
    r.z = up ? __shfl_up_sync(0xffffffffu, v.z, 1) : __shfl_down_sync(0xffffffffu, v.z, 1);
    r.w = up ? __shfl_up_sync(0xffffffffu, v.w, 1) : __shfl_down_sync(0xffffffffu, v.w, 1);
    return r;
}

// one leapfrog update of the lane's four cells, as the row march computes it.
// MODE 0: the plain update; 1: plus the injection inj (zeros in cells without
// a source); 2: the sponge update plus the injection, with damping
// a = c (ez + E4) (zero in undamped cells, where it gives the plain update's
// bits). EDGE: cells outside [0, NX) give zeros.
template <int MODE, bool EDGE>
__device__ __forceinline__ float4 update4(const float *v, const float4 *w, const float4 pp4, const float4 c4,
                                          const float4 inj, float src_scale, float ez, const float4 E4, int gx,
                                          int NX) {
    const Pairs4 d = d2_pairs(make_float4(v[0], v[1], v[2], v[3]), w[4], make_float4(v[8], v[9], v[10], v[11]), w);
    const float2 ra = add2(d.za, d.xa), rb = add2(d.zb, d.xb);
    float res[4];
    if (MODE == 0) {
        const float4 o = plain4(w[4], pp4, c4, ra, rb);
        res[0] = o.x, res[1] = o.y, res[2] = o.z, res[3] = o.w;
    } else {
        const float r4[4] = {ra.x, ra.y, rb.x, rb.y};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float rhs = r4[k] + src_scale * lane_of(inj, k);
            const float p = v[4 + k], pp = lane_of(pp4, k), chv = lane_of(c4, k);
            if (MODE == 2) {
                const float a = chv * (ez + lane_of(E4, k));
                res[k] = __fdividef(2.f * p - (1.f - a) * pp + chv * rhs, 1.f + a);
            } else {
                res[k] = plain1(p, pp, chv, rhs);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 4; k++)
        if (EDGE && !(gx + k >= 0 && gx + k < NX)) res[k] = 0.f;
    return make_float4(res[0], res[1], res[2], res[3]);
}

__device__ void march2x_item(const StepArgs<float> &A, const TBMember &M, const MarchSeg &S, const TBPass &T,
                             float *W, int lane) {
    const Geom &g = A.g;
    const int P = g.P, NX = g.NX, NZ = g.NZ, fs = g.fs;
    const int x0 = S.bx * kTBW, xl = x0 - 4 + 4 * lane;  // the lane's first column
    const long long sh = (long long)M.shot * g.fstride + g.org;
    const bool odd = T.k & 1;
    float *const b0 = A.pbuf[0] + sh, *const b1 = A.pbuf[1] + sh, *const b2 = M.p3 + sh, *const b3 = b2 + M.pstride;
    const float *pc = odd ? b2 : b0;  // p^n
    const float *pb = odd ? b3 : b1;  // p^{n-1}
    float *pw = odd ? b1 : b3;        // p^{n+1} out
    float *pw2 = odd ? b0 : b2;       // p^{n+2} out
    const int z0 = S.z0, z1 = S.z1;
    const bool two = T.two;
    // step-1 rows: the item widened by 4 (two steps), or the item itself (one)
    int rs = two ? z0 - 4 : z0;
    if (fs && rs < 0) rs = 0;  // rows above the free surface are mirrors, not computed
    const int re = two ? z1 + 3 : z1 - 1;
    const bool sponge = A.bc == SIM_BC_SPONGE;
    const int zs0 = sponge ? g.nbz0 : 0, zs1 = sponge ? NZ - g.nbz1 : NZ;
    const bool spx = sponge && ((g.nbx0 > 0 && xl < g.nbx0) || (g.nbx1 > 0 && xl + 3 >= NX - g.nbx1));
    float4 E4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (sponge && xl >= -4 && xl < NX) E4 = __ldg(reinterpret_cast<const float4 *>(A.E[2] + xl));
    const float src_scale = A.src_scale;
    const float *const E0 = A.E[0];
    const int colmax = P - kGhost;  // columns of a row: -kGhost .. colmax - 1
    // the member's point source: its corners lie in rows zA and zA + 1; the
    // injection of a row is summed from the member record when a row needs
    // it (the one-step march's injection: weight x wavelet sample, one entry
    // per cell, zeros elsewhere)
    int zA = -(1 << 30);
    bool hit = false;  // a corner in the lane's columns
    for (int q = 0; q < M.nsrc; q++) {
        zA = q == 0 ? M.sz[0] : min(zA, M.sz[q]);
        hit |= M.sx[q] >= xl && M.sx[q] <= xl + 3;
    }
    const float *wav = static_cast<const float *>(A.io->wavelet);
    auto src_row = [&](int r, int row) {  // the injection of row r, wavelet sample row
        float4 inj = make_float4(0.f, 0.f, 0.f, 0.f);
        const float val = wav[row];
        for (int q = 0; q < M.nsrc; q++) {
            const int k = M.sx[q] - xl;
            if (M.sz[q] != r || k < 0 || k > 3) continue;
            const float add = M.sw[q] * val;
            if (k == 0) inj.x = add;
            if (k == 1) inj.y = add;
            if (k == 2) inj.z = add;
            if (k == 3) inj.w = add;
        }
        return inj;
    };
    // warp-uniform facts: rows with a source corner in the item, rows with
    // damping (a sponge lane or a z-sponge row), items with columns outside
    // [0, NX)
    const bool hit_w = __any_sync(0xffffffffu, hit);
    const bool spx_w = __any_sync(0xffffffffu, spx);
    const bool edge_w = x0 - 4 < 0 || x0 + 124 > NX;
    auto damped = [&](int r) { return spx_w || (sponge && (r < zs0 || r >= zs1)); };
    auto src_in = [&](int r) { return hit_w && (r == zA || r == zA + 1); };

    // ring: p^n rows (columns x0 - 8 ..), p^{n-1} rows and c rows (columns x0 - 4 ..)
    float *RPN = W, *RPP = W + NS2 * PNW, *RCC = RPP + NS2 * OW;
    const unsigned spn = (unsigned)__cvta_generic_to_shared(RPN) + 16u * lane,
                   spp = (unsigned)__cvta_generic_to_shared(RPP) + 16u * lane,
                   scc = (unsigned)__cvta_generic_to_shared(RCC) + 16u * lane;
    // the lane's staged columns and whether they lie in the row's memory
    const int c0 = x0 - 8 + 4 * lane;
    const bool in0 = c0 + 3 < colmax, in1 = lane < 2 && x0 + 123 + 4 * lane < colmax, ino = xl + 3 < colmax;
    const long long oP = (long long)P;
    // copy cursors: the next p^n row and the next p^{n-1} / c row to stage
    const float *pn_src = pc + (long long)rs * P + c0;
    const float *pp_src = pb + (long long)rs * P + xl;
    const float *cc_src = A.ch + g.org + (long long)rs * P + xl;
    int pn_row = rs, o_row = rs;
    auto stage_pn = [&]() {  // p^n row pn_row, columns x0 - 8 .. x0 + 127
        const unsigned d = spn + 4u * (pn_row & (NS2 - 1)) * PNW;
        cp16_if(d, pn_src, in0);
        if (!in0) *reinterpret_cast<float4 *>(RPN + (pn_row & (NS2 - 1)) * PNW + 4 * lane) = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane < 2) {
            cp16_if(d + 512u, pn_src + 128, in1);
            if (!in1)
                *reinterpret_cast<float4 *>(RPN + (pn_row & (NS2 - 1)) * PNW + 128 + 4 * lane) =
                    make_float4(0.f, 0.f, 0.f, 0.f);
        }
        pn_src += oP;
        pn_row++;
    };
    auto stage_o = [&]() {  // p^{n-1} and c rows o_row, columns x0 - 4 .. x0 + 123
        const unsigned off = 4u * (o_row & (NS2 - 1)) * OW;
        cp16_if(spp + off, pp_src, ino);
        cp16_if(scc + off, cc_src, ino);
        if (!ino) {
            *reinterpret_cast<float4 *>(RPP + (o_row & (NS2 - 1)) * OW + 4 * lane) = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4 *>(RCC + (o_row & (NS2 - 1)) * OW + 4 * lane) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        pp_src += oP;
        cc_src += oP;
        o_row++;
    };

    // prologue: p^n rows rs .. rs + 3 (the first windows), then D2 groups of
    // the rows iterations rs .. rs + D2 - 1 will read
    for (int r = rs; r < rs + 4; r++) stage_pn();
    cp_commit();
    for (int j = 0; j < D2; j++) {
        if (rs + j <= re) {
            stage_pn();
            stage_o();
        }
        cp_commit();
    }
    // p^n window: rows r-4 .. r+4 of the lane's columns; rows above the
    // free surface mirror with odd sign
    float4 w0[9], w1[9];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int r = rs - 4 + k;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ino) v = (r < 0 && fs) ? neg4(ld4(pc + (long long)(-r) * P + xl)) : ld4(pc + (long long)r * P + xl);
        w0[k] = v;
    }
#pragma unroll
    for (int k = 0; k < 9; k++) w1[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    cp_wait<D2>();
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; k++) w0[4 + k] = ld4(RPN + ((rs + k) & (NS2 - 1)) * PNW + 4 + 4 * lane);
    float *out1 = pw + (long long)(two ? z0 : rs) * P + xl, *out2 = pw2 + (long long)z0 * P + xl;
    const bool st_lane = lane >= 1 && lane <= 30 && xl < NX;

    for (int r = rs; r <= re; r++) {
        // every lane's reads of the slots refilled below (rows r - 1 and
        // r - 5, read in the previous iteration) come before the refill
        __syncwarp();
        if (r + D2 <= re) {  // the rows iteration r + D2 reads
            stage_pn();
            stage_o();
        }
        cp_commit();
        cp_wait<D2>();
        __syncwarp();
        const int slot = r & (NS2 - 1);
        w0[8] = ld4(RPN + ((r + 4) & (NS2 - 1)) * PNW + 4 + 4 * lane);
        // step 1: p^{n+1} at row r
        float4 p1 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r >= 0 && r < NZ && !(fs && r == 0)) {
            const float *row = RPN + slot * PNW;
            float v[12];
            unpack3(ld4(row + 4 * lane), w0[4], ld4(row + 4 * lane + 8), v);
            const float4 pp4 = ld4(RPP + slot * OW + 4 * lane), c4 = ld4(RCC + slot * OW + 4 * lane);
            const bool sr = src_in(r) && T.inj0 >= 0;
            if (damped(r)) {
                const float4 inj = sr ? src_row(r, T.inj0) : make_float4(0.f, 0.f, 0.f, 0.f);
                p1 = update4<2, true>(v, w0, pp4, c4, inj, src_scale, __ldg(E0 + r), E4, xl, NX);
            } else if (sr) {
                p1 = update4<1, true>(v, w0, pp4, c4, src_row(r, T.inj0), src_scale, 0.f, E4, xl, NX);
            } else if (edge_w) {
                p1 = update4<0, true>(v, w0, pp4, c4, pp4, 0.f, 0.f, E4, xl, NX);
            } else {
                p1 = update4<0, false>(v, w0, pp4, c4, pp4, 0.f, 0.f, E4, xl, NX);
            }
        }
        w1[8] = p1;
        if (two && fs && r == 4) {  // the window now holds rows -4 .. 4: rows -4 .. -1 mirror rows 4 .. 1
#pragma unroll
            for (int k = 0; k < 4; k++) w1[k] = neg4(w1[8 - k]);
        }
        if (!two) {  // one step: p^{n+1} of the item's own columns
            if (st_lane) st4(out1, p1);
            out1 += P;
        } else if (r - 4 >= z0) {
            // step 2: p^{n+2} at row r2 = r - 4, from the p^{n+1} window
            const int r2 = r - 4;
            const float4 L = shfl4(w1[4], true), R = shfl4(w1[4], false);
            float4 p2 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r2 < NZ && !(fs && r2 == 0)) {
                float v[12];
                unpack3(L, w1[4], R, v);
                const float4 c4 = ld4(RCC + (r2 & (NS2 - 1)) * OW + 4 * lane);
                const bool sr = src_in(r2) && T.inj1 >= 0;
                if (damped(r2)) {
                    const float4 inj = sr ? src_row(r2, T.inj1) : make_float4(0.f, 0.f, 0.f, 0.f);
                    p2 = update4<2, true>(v, w1, w0[0], c4, inj, src_scale, __ldg(E0 + r2), E4, xl, NX);
                } else if (sr) {
                    p2 = update4<1, true>(v, w1, w0[0], c4, src_row(r2, T.inj1), src_scale, 0.f, E4, xl, NX);
                } else if (edge_w) {
                    p2 = update4<0, true>(v, w1, w0[0], c4, c4, 0.f, 0.f, E4, xl, NX);
                } else {
                    p2 = update4<0, false>(v, w1, w0[0], c4, c4, 0.f, 0.f, E4, xl, NX);
                }
            }
            if (st_lane) {
                st4(out1, w1[4]);
                st4(out2, p2);
            }
            out1 += P;
            out2 += P;
        }
#pragma unroll
        for (int k = 0; k < 8; k++) {
            w0[k] = w0[k + 1];
            w1[k] = w1[k + 1];
        }
    }
    cp_wait<0>();
    __syncwarp();
}

__global__ void __launch_bounds__(NW2 * 32, 4) k_march2x(const TBArgs B, const TBPass T) {
    extern __shared__ float4 smx[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *W = reinterpret_cast<float *>(smx) + (size_t)wib * WARPF;
    // items in order from this pass's counter; the previous pass is complete
    // (stream order), so zeroing the next pass's counter here is safe
    unsigned *ctr = B.ctr + (T.k & 1);
    if (blockIdx.x == 0 && threadIdx.x == 0) B.ctr[(T.k + 1) & 1] = 0u;
    unsigned next = 0;
    if (lane == 0) next = atomicAdd(ctr, 1u);
    next = __shfl_sync(0xffffffffu, next, 0);
    while (next < (unsigned)B.nitems) {
        const MarchSeg S = B.segs[next];
        if (lane == 0) next = atomicAdd(ctr, 1u);
        const TBMember &M = B.members[S.slice];
        march2x_item(B.slices[M.slice], M, S, T, W, lane);
        next = __shfl_sync(0xffffffffu, next, 0);
    }
}

// receivers of every member: row n from p^n, and row n + 1 from p^{n+1} when
// the pass took two steps (both buffers still hold them after the pass)
__global__ void k_sample2x(const TBArgs B, const TBPass T) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int rows = T.two ? 2 : 1;
    if (i >= B.nsamples * rows) return;
    const int which = (int)(i / B.nsamples);
    const long long j = i - (long long)which * B.nsamples;
    const TBSample Q = B.samples[j];
    const TBMember &M = B.members[Q.member];
    const StepArgs<float> &A = B.slices[M.slice];
    const Geom &g = A.g;
    const long long sh = (long long)M.shot * g.fstride + g.org;
    // p^n: field 0 (even pass) or 2 (odd); p^{n+1}: field 3 or 1
    const bool odd = T.k & 1;
    const float *p = which ? (odd ? A.pbuf[1] + sh : M.p3 + M.pstride + sh) : (odd ? M.p3 + sh : A.pbuf[0] + sh);
    const float *r0 = p + (long long)Q.z * g.P, *r1 = r0 + g.P;
    const float val = Q.w[0] * r0[Q.x] + Q.w[1] * r0[Q.x + 1] + Q.w[2] * r1[Q.x] + Q.w[3] * r1[Q.x + 1];
    const int n = T.n + which;
    static_cast<float *>(A.io->gather)[((long long)M.shot * A.nt + n) * A.io->nrec + Q.rec] = val;
    if (!isfinite(val)) atomicOr(A.flags, kFlagUnstable);
}

size_t march2x_smem() { return (size_t)NW2 * WARPF * sizeof(float); }

}  // namespace

cudaError_t configure_march2x() {
    return cudaFuncSetAttribute(k_march2x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)march2x_smem());
}

int march2x_warps_per_sm() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_march2x, NW2 * 32, march2x_smem());
    return nb * NW2;
}

cudaError_t launch_march2x(const TBArgs &b, const TBPass &t, int nwarps, cudaStream_t st) {
    if (nwarps < 1) return cudaSuccess;
    k_march2x<<<(nwarps + NW2 - 1) / NW2, NW2 * 32, march2x_smem(), st>>>(b, t);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || b.nsamples == 0) return e;
    const long long tot = b.nsamples * (t.two ? 2 : 1);
    k_sample2x<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(b, t);
    return cudaGetLastError();
}

}  // namespace gsim
