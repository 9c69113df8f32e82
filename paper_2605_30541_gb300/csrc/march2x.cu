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

using f32::d2w;
using f32::lane_of;
using f32::ld4;
using f32::st4;
using f32::unpack3;

constexpr int NW2 = 4;        // warps per CTA
constexpr int NS2 = 8;        // ring rows per field
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

// second difference along z at cell k of the 9-row window w (centre w[4]):
// the row march's own expression
__device__ __forceinline__ float d2z9(const float4 *w, int k) {
    return d2c<float>(lane_of(w[4], k), lane_of(w[3], k), lane_of(w[5], k), lane_of(w[2], k), lane_of(w[6], k),
                      lane_of(w[1], k), lane_of(w[7], k), lane_of(w[0], k), lane_of(w[8], k));
}

// the point sources of a member injected into row r of the lane's float4
// (columns xl .. xl+3): value = wavelet[row] w summed per cell, as the one-step
// march's injection groups sum their entries
__device__ __forceinline__ bool src_row(const TBMember &M, int r, int xl, float val, float4 &inj) {
    bool any = false;
    for (int s = 0; s < M.nsrc; s++) {
        const int k = M.sx[s] - xl;
        if (M.sz[s] != r || k < 0 || k > 3) continue;
        const float add = M.sw[s] * val;
        if (k == 0) inj.x += add;
        if (k == 1) inj.y += add;
        if (k == 2) inj.z += add;
        if (k == 3) inj.w += add;
        any = true;
    }
    return any;
}

// one leapfrog update of the lane's four cells, as the row march computes it
__device__ __forceinline__ float4 update4(const float *v, const float4 *w, const float4 pp4, const float4 c4,
                                          const float4 inj, bool any_inj, float src_scale, bool spg, float ez,
                                          const float4 E4, int gx, int NX) {
    float res[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        float rhs = d2z9(w, k) + d2w(v, k);
        if (any_inj) rhs += src_scale * lane_of(inj, k);
        const float p = v[4 + k], pp = lane_of(pp4, k), chv = lane_of(c4, k);
        float o;
        if (spg) {
            const float a = chv * (ez + lane_of(E4, k));
            o = __fdividef(2.f * p - (1.f - a) * pp + chv * rhs, 1.f + a);
        } else {
            o = 2.f * p - pp + chv * rhs;
        }
        res[k] = gx + k >= 0 && gx + k < NX ? o : 0.f;
    }
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
    // step-1 rows: the item widened by 4 (two steps), or the item itself (one)
    int rs = T.two ? z0 - 4 : z0;
    if (fs && rs < 0) rs = 0;  // rows above the free surface are mirrors, not computed
    const int re = T.two ? z1 + 3 : z1 - 1;
    const bool sponge = A.bc == SIM_BC_SPONGE;
    const int zs0 = sponge ? g.nbz0 : 0, zs1 = sponge ? NZ - g.nbz1 : NZ;
    const bool spx = sponge && ((g.nbx0 > 0 && xl < g.nbx0) || (g.nbx1 > 0 && xl + 3 >= NX - g.nbx1));
    float4 E4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (sponge && xl >= -4 && xl < NX) E4 = __ldg(reinterpret_cast<const float4 *>(A.E[2] + xl));
    const float src_scale = A.src_scale;
    const float *wav = static_cast<const float *>(A.io->wavelet);
    const int colmax = P - kGhost;  // columns of a row: -kGhost .. colmax - 1

    // ring: p^n rows (columns x0 - 8 ..), p^{n-1} rows and c rows (columns x0 - 4 ..)
    float *RPN = W, *RPP = W + NS2 * PNW, *RCC = RPP + NS2 * OW;
    const unsigned spn = (unsigned)__cvta_generic_to_shared(RPN), spp = (unsigned)__cvta_generic_to_shared(RPP),
                   scc = (unsigned)__cvta_generic_to_shared(RCC);
    auto zero_pn = [&](int slot, int c) {  // a staged p^n float4 beyond the row: zeros
        *reinterpret_cast<float4 *>(RPN + slot * PNW + c - (x0 - 8)) = make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto stage_pn = [&](int row) {  // p^n row with columns x0 - 8 .. x0 + 127
        const int slot = ((row % NS2) + NS2) % NS2;
        const float *src = pc + (long long)row * P;
        const int c0 = x0 - 8 + 4 * lane;
        const bool in0 = c0 + 3 < colmax;
        cp16_if(spn + 4u * (slot * PNW + 4 * lane), src + c0, in0);
        if (!in0) zero_pn(slot, c0);
        if (lane < 2) {
            const int c1 = x0 + 120 + 4 * lane;
            const bool in1 = c1 + 3 < colmax;
            cp16_if(spn + 4u * (slot * PNW + 128 + 4 * lane), src + c1, in1);
            if (!in1) zero_pn(slot, c1);
        }
    };
    auto stage_o = [&](int row) {  // p^{n-1} and c rows, columns x0 - 4 .. x0 + 123
        const int slot = ((row % NS2) + NS2) % NS2;
        const long long o = (long long)row * P + xl;
        const bool in = xl + 3 < colmax;
        cp16_if(spp + 4u * (slot * OW + 4 * lane), pb + o, in);
        cp16_if(scc + 4u * (slot * OW + 4 * lane), A.ch + g.org + o, in);
        if (!in) {
            *reinterpret_cast<float4 *>(RPP + slot * OW + 4 * lane) = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4 *>(RCC + slot * OW + 4 * lane) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };

    // prologue: p^n rows rs .. rs + 3 (the first windows), then D2 groups of
    // the rows iterations rs .. rs + D2 - 1 will read
    for (int r = rs; r < rs + 4; r++) stage_pn(r);
    cp_commit();
    for (int j = 0; j < D2; j++) {
        const int r = rs + j;
        if (r + 4 <= re + 4) stage_pn(r + 4);
        if (r <= re) stage_o(r);
        cp_commit();
    }
    // p^n window: rows r-4 .. r+4 of the lane's columns; rows above the
    // free surface mirror with odd sign
    float4 w0[9], w1[9];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int r = rs - 4 + k;
        const bool in = xl + 3 < colmax;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (in) v = (r < 0 && fs) ? neg4(ld4(pc + (long long)(-r) * P + xl)) : ld4(pc + (long long)r * P + xl);
        w0[k] = v;
    }
#pragma unroll
    for (int k = 0; k < 9; k++) w1[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    cp_wait<D2>();
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; k++) w0[4 + k] = ld4(RPN + (((rs + k) % NS2 + NS2) % NS2) * PNW + 4 + 4 * lane);

    for (int r = rs; r <= re; r++) {
        // every lane's reads of the slots refilled below (rows r - 1 and
        // r - 5, read in the previous iteration) come before the refill
        __syncwarp();
        {  // the rows iteration r + D2 reads
            const int rr = r + D2;
            if (rr <= re) {
                stage_pn(rr + 4);
                stage_o(rr);
            }
            cp_commit();
        }
        cp_wait<D2>();
        __syncwarp();
        const int slot = ((r % NS2) + NS2) % NS2;
        w0[8] = ld4(RPN + (((r + 4) % NS2 + NS2) % NS2) * PNW + 4 + 4 * lane);
        // step 1: p^{n+1} at row r
        float4 p1 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r >= 0 && r < NZ && !(fs && r == 0)) {
            const float *row = RPN + slot * PNW;
            float v[12];
            unpack3(ld4(row + 4 * lane), w0[4], ld4(row + 4 * lane + 8), v);
            const float4 pp4 = ld4(RPP + slot * OW + 4 * lane), c4 = ld4(RCC + slot * OW + 4 * lane);
            float4 inj = make_float4(0.f, 0.f, 0.f, 0.f);
            const bool any = T.inj0 >= 0 && src_row(M, r, xl, wav[T.inj0], inj);
            const bool spg = spx || (sponge && (r < zs0 || r >= zs1));
            const float ez = spg ? __ldg(A.E[0] + r) : 0.f;
            p1 = update4(v, w0, pp4, c4, inj, any, src_scale, spg, ez, E4, xl, NX);
        }
        w1[8] = p1;
        if (T.two && fs && r == 4) {  // the window now holds rows -4 .. 4: rows -4 .. -1 mirror rows 4 .. 1
#pragma unroll
            for (int k = 0; k < 4; k++) w1[k] = neg4(w1[8 - k]);
        }
        if (!T.two) {  // one step: p^{n+1} of the item's own columns
            if (lane >= 1 && lane <= 30 && xl < NX) st4(pw + (long long)r * P + xl, p1);
        } else if (r - 4 >= z0) {
            // step 2: p^{n+2} at row r2 = r - 4, from the p^{n+1} window
            const int r2 = r - 4;
            const float4 L = shfl4(w1[4], true), R = shfl4(w1[4], false);
            if (lane >= 1 && lane <= 30) {
                float4 p2 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (r2 < NZ && !(fs && r2 == 0)) {
                    float v[12];
                    unpack3(L, w1[4], R, v);
                    const int s2 = ((r2 % NS2) + NS2) % NS2;
                    const float4 c4 = ld4(RCC + s2 * OW + 4 * lane);
                    float4 inj = make_float4(0.f, 0.f, 0.f, 0.f);
                    const bool any = T.inj1 >= 0 && src_row(M, r2, xl, wav[T.inj1], inj);
                    const bool spg = spx || (sponge && (r2 < zs0 || r2 >= zs1));
                    const float ez = spg ? __ldg(A.E[0] + r2) : 0.f;
                    p2 = update4(v, w1, w0[0], c4, inj, any, src_scale, spg, ez, E4, xl, NX);
                }
                if (xl < NX) {
                    st4(pw + (long long)r2 * P + xl, w1[4]);
                    st4(pw2 + (long long)r2 * P + xl, p2);
                }
            }
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

__global__ void __launch_bounds__(NW2 * 32) k_march2x(const TBArgs B, const TBPass T) {
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
