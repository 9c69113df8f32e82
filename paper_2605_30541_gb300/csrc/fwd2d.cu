// 2D time step of the acoustic scheme, one fused kernel per step:
//   8th-order Laplacian (App. E.3), leapfrog update with the centred sponge
//   term (Eq. cerjan_pde / cerjan_damp) or CPML memory terms, free surface
//   (Eq. free_surface), point injection, receiver sampling (Sec. 2, R p) and
//   snapshot output (App. E.3.3).
//
// A CTA owns a 32 x 16 tile of the computational grid and stages p^n with a
// radius-4 halo (radius 8 in CPML tiles, which recompute psi^n on the tile
// +-4 cells) in shared memory; a thread updates two cells of one column.
// Tiles are classified per CTA (interior / sponge / CPML / surface) so that
// interior tiles run the plain update with no boundary arithmetic.
//
// The same kernel serves the adjoint-state gradient: with u = c lambda the
// discrete adjoint recursion has the forward update's form, driven by the
// data residual injected at the receivers (MODE kModeAdjoint), and the
// forward recompute records the per-cell imaging term (MODE kModeRecord).
#include <cfloat>

#include "sim_internal.h"
#include "stencil.cuh"

namespace gsim {
namespace {

constexpr int TX = kTileX2, TZ = kTileZ2, HM = 8;
constexpr int BX = 32, BY = 8, RZ = TZ / BY, NTH = BX * BY;

__device__ __forceinline__ float block_max(float v, float *red) {
    const int tid = threadIdx.y * BX + threadIdx.x;
    v = warp_max(v);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    float m = tid < NTH / 32 ? red[tid & 31] : 0.f;
    if (tid < 32) m = warp_max(m);
    if (tid == 0) red[0] = m;
    __syncthreads();
    return red[0];
}

template <typename T, int MODE>
__global__ void __launch_bounds__(NTH) k_step2d(const StepArgs<T> A, const int n) {
    __shared__ T S[TZ + 2 * HM][TX + 2 * HM];
    __shared__ T PX[TZ][TX + 8];
    __shared__ T PZ[TZ + 8][TX];
    __shared__ T INJ[TZ][TX];
    __shared__ float red[NTH / 32];

    const Geom &g = A.g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ, shot = blockIdx.z;
    const int tile = blockIdx.y * A.ntx + blockIdx.x;
    const long long sh = (long long)shot * g.fstride;
    const T *pc = A.pbuf[n & 1] + sh;
    T *pnx = A.pbuf[(n + 1) & 1] + sh;  // holds p^{n-1}, receives p^{n+1}

    const bool cpml = A.bc == SIM_BC_CPML;
    const bool cpx = cpml && A.ca[2] &&
                     ((g.nbx0 > 0 && x0 - 4 < g.nbx0) || (g.nbx1 > 0 && x0 + TX + 4 > g.NX - g.nbx1));
    const bool cpz = cpml && A.ca[0] &&
                     ((g.nbz0 > 0 && z0 - 4 < g.nbz0) || (g.nbz1 > 0 && z0 + TZ + 4 > g.NZ - g.nbz1));
    const bool spg = A.bc == SIM_BC_SPONGE &&
                     ((g.nbx0 > 0 && x0 < g.nbx0) || (g.nbx1 > 0 && x0 + TX > g.NX - g.nbx1) ||
                      (g.nbz0 > 0 && z0 < g.nbz0) || (g.nbz1 > 0 && z0 + TZ > g.NZ - g.nbz1));
    const int H = (cpx || cpz) ? 8 : 4;

    // ---- stage p^n (tile + halo); ghost memory supplies p = 0 outside the grid
    {
        const int W = TX + 2 * H, NR = TZ + 2 * H, o = HM - H;
        for (int i = tid; i < W * NR; i += NTH) {
            const int r = i / W, c = i - r * W;
            S[o + r][o + c] = pc[cell_off(g, z0 - H + r, 0, x0 - H + c)];
        }
    }
    __syncthreads();
    if (g.fs && z0 < H) {  // odd mirror above the free surface: p(-k) = -p(k)
        const int W = TX + 2 * H, o = HM - H;
        for (int i = tid; i < H * W; i += NTH) {
            const int k = i / W + 1, c = i - (k - 1) * W;
            S[HM - k][o + c] = -S[HM + k][o + c];
        }
        __syncthreads();
    }

    // ---- CPML: psi^n = b psi^{n-1} + a D1 p^n on the tile +-4 cells (scaled by h)
    if (cpx) {
        const T *po = A.psi[2][(n + 1) & 1] + sh;
        T *pw = A.psi[2][n & 1] + sh;
        for (int i = tid; i < TZ * (TX + 8); i += NTH) {
            const int lz = i / (TX + 8), lxx = i - lz * (TX + 8) - 4;
            const int gz = z0 + lz, gx = x0 + lxx;
            T v = T(0);
            if (gz < g.NZ && gx >= 0 && gx < g.NX) {
                const long long o = cell_off(g, gz, 0, gx);
                const T d1 = d1_row(&S[HM + lz][HM + lxx], 1);
                v = A.cb[2][gx] * po[o] + A.ca[2][gx] * d1;
                if (lxx >= 0 && lxx < TX) pw[o] = v;
            }
            PX[lz][lxx + 4] = v;
        }
    }
    if (cpz) {
        const T *po = A.psi[0][(n + 1) & 1] + sh;
        T *pw = A.psi[0][n & 1] + sh;
        for (int i = tid; i < (TZ + 8) * TX; i += NTH) {
            const int lzz = i / TX - 4, lx = i - (lzz + 4) * TX;
            const int gz = z0 + lzz, gx = x0 + lx;
            T v = T(0);
            if (gz >= 0 && gz < g.NZ && gx < g.NX) {
                const long long o = cell_off(g, gz, 0, gx);
                const T d1 = d1_row(&S[HM + lzz][HM + lx], TX + 2 * HM);
                v = A.cb[0][gz] * po[o] + A.ca[0][gz] * d1;
                if (lzz >= 0 && lzz < TZ) pw[o] = v;
            }
            PZ[lzz + 4][lx] = v;
        }
    }

    // ---- point injection into this tile (deterministic: one thread per cell)
    const int itile = A.inj_per_shot ? shot * (A.ntx * A.ntz) + tile : tile;
    const int g0 = A.inj_start[itile], g1 = A.inj_start[itile + 1];
    const bool has_inj = g1 > g0;
    if (has_inj) {
        for (int i = tid; i < TZ * TX; i += NTH) (&INJ[0][0])[i] = T(0);
        __syncthreads();
        const SimIO *io = A.io;
        const int row = A.inj_reverse ? A.nt - n : n;
        for (int gi = g0 + tid; gi < g1; gi += NTH) {
            const InjGroup G = A.inj_grp[gi];
            T sum = T(0);
            for (int e = G.e0; e < G.e1; e++) {
                const InjEntryT<T> E = A.inj_ent[e];
                T val = T(0);
                if (A.inj_kind == 0)
                    val = static_cast<const T *>(io->wavelet)[row];
                else if (row < A.nt)
                    val = static_cast<const T *>(io->resid)[((long long)shot * A.nt + row) * io->nrec + E.pt];
                sum += T(E.w) * val;
            }
            (&INJ[0][0])[G.cell] = sum;
        }
    }
    __syncthreads();

    // ---- receivers sample p^n
    if (A.sample) {
        const int r0 = A.rec_start[tile], r1 = A.rec_start[tile + 1];
        if (r1 > r0) {
            const SimIO *io = A.io;
            T *gout = static_cast<T *>(io->gather);
            if (gout) {
                const long long row = ((long long)shot * A.nt + n) * io->nrec;
                for (int e = r0 + tid; e < r1; e += NTH) {
                    const RecEntryT<T> R = A.rec[e];
                    const T *b = &S[HM + R.lz][HM + R.lx];
                    const T val = T(R.w[0]) * b[0] + T(R.w[1]) * b[1] +
                                  T(R.w[2]) * b[TX + 2 * HM] + T(R.w[3]) * b[TX + 2 * HM + 1];
                    gout[row + R.rec] = val;
                    if (!isfinite((double)val)) atomicOr(A.flags, kFlagUnstable);
                }
            }
        }
    }

    // ---- snapshot bookkeeping
    const bool snap_now = MODE == kModeForward && A.nsnap > 0 && n >= A.snap_begin && n < A.snap_end &&
                          (n - A.snap_begin) % A.snap_every == 0;
    const int n1 = n + 1;
    const bool max_next = MODE == kModeForward && A.nsnap > 0 && n1 >= A.snap_begin && n1 < A.snap_end &&
                          (n1 - A.snap_begin) % A.snap_every == 0;
    void *snaps = nullptr;
    int fp16 = 0;
    float sinv = 1.f;
    long long sbase = 0;
    if (snap_now || max_next) {
        const SimIO *io = A.io;
        snaps = io->snaps;
        fp16 = io->snap_fp16;
        if (snap_now && snaps) {
            const int k = (n - A.snap_begin) / A.snap_every;
            sbase = ((long long)shot * A.nsnap + k) * g.nz * g.nx;
            if (fp16) {
                const float m = __uint_as_float(io->snap_max[shot * A.nsnap + k]);
                const float s = pow2_scale(m);
                sinv = 1.f / s;
                if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) io->snap_scale[shot * A.nsnap + k] = s;
            }
        }
    }

    // ---- adjoint sweep: imaging term of this step, recorded by the recompute
    const int ntiles = A.ntx * A.ntz;
    float qs = 1.f;
    if (MODE == kModeAdjoint && A.q_fp16) qs = A.qscale[shot * ntiles + tile];

    // ---- update
    float tmax = 0.f;
    T qv[RZ];
#pragma unroll
    for (int k = 0; k < RZ; k++) {
        qv[k] = T(0);
        const int lz = ty + k * BY, lx = tx;
        const int gz = z0 + lz, gx = x0 + lx;
        if (gz >= g.NZ || gx >= g.NX) continue;
        const int r = HM + lz, c = HM + lx;
        const T p = S[r][c];
        const T d2z = d2_col(&S[r][c], TX + 2 * HM);
        const T d2x = d2_col(&S[r][c], 1);
        T rhs = d2z + d2x;
        const long long o = cell_off(g, gz, 0, gx);
        if (cpx) {
            const T dps = d1_row(&PX[lz][lx + 4], 1);
            T *zp = A.zeta[2] + sh + o;
            const T zt = A.cb[2][gx] * (*zp) + A.ca[2][gx] * (d2x + dps);
            *zp = zt;
            rhs += dps + zt;
        }
        if (cpz) {
            const T dps = d1_row(&PZ[lz + 4][lx], TX);
            T *zp = A.zeta[0] + sh + o;
            const T zt = A.cb[0][gz] * (*zp) + A.ca[0][gz] * (d2z + dps);
            *zp = zt;
            rhs += dps + zt;
        }
        if (MODE == kModeAdjoint && A.cext) rhs += A.cext[sh + o];  // transposed CPML terms of u
        if (has_inj) rhs += A.src_scale * INJ[lz][lx];
        const T chv = A.ch[o];
        const T pp = pnx[o];
        T out, esum = T(0);
        if (spg) {
            esum = A.E[0][gz] + A.E[2][gx];
            const T a = chv * esum;
            out = (T(2) * p - (T(1) - a) * pp + chv * rhs) / (T(1) + a);
        } else {
            out = T(2) * p - pp + chv * rhs;
        }
        if (g.fs && gz == 0) out = T(0);
        pnx[o] = out;
        const long long ci = sh + o;  // imaging slots and G share the field layout
        if (MODE == kModeRecord) {
            qv[k] = esum * (out - pp) - rhs;
            if (A.q_fp16) tmax = fmaxf(tmax, fabsf((float)qv[k]));
            else static_cast<T *>(A.qslot)[ci] = qv[k];
        }
        if (MODE == kModeAdjoint) {
            T q;
            if (A.q_fp16) q = T(__half2float(static_cast<const __half *>(A.qslot)[ci]) * qs);
            else q = static_cast<const T *>(A.qslot)[ci];
            T *gp = A.G + ci;
            *gp += out * q;
        }
        const bool inside = gz >= g.oz && gz < g.oz + g.nz && gx >= g.ox && gx < g.ox + g.nx;
        if (MODE == kModeForward && max_next && inside) tmax = fmaxf(tmax, fabsf((float)out));
        if (snap_now && snaps && inside) {
            const long long si = sbase + (long long)(gz - g.oz) * g.nx + (gx - g.ox);
            if (fp16)
                static_cast<__half *>(snaps)[si] = __float2half_rn((float)p * sinv);
            else
                static_cast<T *>(snaps)[si] = p;
        }
    }

    // ---- FP16 imaging term: one power-of-two scale per tile and step
    if (MODE == kModeRecord && A.q_fp16) {
        const float m = block_max(tmax, red);
        const float s = pow2_scale(m), inv = 1.f / s;
        if (tid == 0) A.qscale[shot * ntiles + tile] = s;
#pragma unroll
        for (int k = 0; k < RZ; k++) {
            const int gz = z0 + ty + k * BY, gx = x0 + tx;
            if (gz >= g.NZ || gx >= g.NX) continue;
            static_cast<__half *>(A.qslot)[sh + cell_off(g, gz, 0, gx)] = __float2half_rn((float)qv[k] * inv);
        }
    }

    // ---- block max of p^{n+1} for the next snapshot's FP16 scale
    if (MODE == kModeForward && max_next && fp16 && snaps) {
        const float m = block_max(tmax, red);
        if (tid == 0) {
            const int k = (n1 - A.snap_begin) / A.snap_every;
            if (!(m <= FLT_MAX)) atomicOr(A.flags, kFlagUnstable);
            else atomicMax(&A.io->snap_max[shot * A.nsnap + k], __float_as_uint(m));
        }
    }
}

}  // namespace

template <typename T>
cudaError_t launch_step2d(const StepArgs<T> &a, int n, int nshots, int mode, cudaStream_t st) {
    dim3 grid(a.ntx, a.ntz, nshots), block(BX, BY);
    if (mode == kModeRecord)
        k_step2d<T, kModeRecord><<<grid, block, 0, st>>>(a, n);
    else if (mode == kModeAdjoint)
        k_step2d<T, kModeAdjoint><<<grid, block, 0, st>>>(a, n);
    else
        k_step2d<T, kModeForward><<<grid, block, 0, st>>>(a, n);
    return cudaGetLastError();
}

template cudaError_t launch_step2d<float>(const StepArgs<float> &, int, int, int, cudaStream_t);
template cudaError_t launch_step2d<double>(const StepArgs<double> &, int, int, int, cudaStream_t);

}  // namespace gsim
