// Resident FP32 2D forward solve: the whole time loop of one forward run in
// a single cooperative launch whose CTAs keep the wavefield on chip.
//
// The per-step kernel (fwd2d_f32.cu) pays, every step, a launch, a grid-wide
// dependency and a reload of p^n, p^{n-1} and c from L2. On a slice of a few
// hundred thousand to about a million cells the whole state fits in the SMs'
// shared memory and registers, so here each CTA owns one subdomain of 128
// columns and at most WZ = 16 RZ rows for the entire run. Subdomain heights
// vary (RTile descriptors from the host): subdomains with absorbing work get
// fewer rows, so every CTA takes about as long per step; warps take
// ceil(rows / 16) consecutive rows each.
//   - p^n with an 8-cell halo lives in shared memory in two buffers; the
//     other buffer's own cells still hold p^{n-1}, which each thread reads
//     and overwrites with p^{n+1} in place; c stays in registers;
//   - the CPML memory variables live in shared memory and are computed only
//     where they can be non-zero: psi on the absorbing strips (and the
//     4-cell band beyond the subdomain that a derivative of psi reaches,
//     recomputed redundantly as in the per-step kernel), zeta and the update
//     addend D1 psi + zeta on the strips widened by 4 cells. Outside the
//     strips both recursion coefficients are zero, so everything skipped is
//     exactly zero. x-strip work is spread over all threads (a strip is
//     narrower than a row of warps); z-strip work follows the rows of warps,
//     and zeta_z is fused into the update, which already holds D2z p;
//   - sponge subdomains precompute per cell the update weights 2/(1+a),
//     (1-a)/(1+a) and c/(1+a) (a = c eta dt / 2 is fixed in time), so the
//     step has no division;
//   - after each step a CTA publishes the 8 (4 without CPML) border rows and
//     columns of p^{n+1} to the global pressure buffer and raises its step
//     counter (release); a CTA starts step n once the counters of the
//     subdomains above, below and beside it (its descriptor lists them)
//     reach n (acquire), and copies their borders in as its halo. The
//     stencil is a cross, so corner neighbours are never needed.
// The launch is cooperative, so all CTAs are co-resident and the waits
// always end; each wait is still bounded (spin_limit polls), after which the
// kernel raises kFlagTimeout and every CTA returns.
//
// The scheme is the leapfrog update with the centred sponge term or the CPML
// memory terms (Sec. 2, App. E.3-E.4), free surface as an odd mirror with
// row 0 held at zero; the per-cell arithmetic is that of the per-step kernel
// up to the order of a few additions (rounding level). Forward mode with
// FP32 snapshots only: an FP16 snapshot's scale needs the grid-wide maximum
// of the previous step, which a schedule without a grid barrier lacks.
#include <algorithm>
#include <cfloat>

#include "f32_tile.cuh"
#include "sim_internal.h"

namespace gsim {
namespace {

using namespace f32;

constexpr int TX = kTileXF, HM = 8, SW = TX + 2 * HM;
constexpr int NWR = kResidentWarps, NTR = NWR * 32;

// Receivers of a subdomain whose entries are kept in shared memory (more
// are read from global memory every step).
constexpr int kRecCache = 128;

// Shared memory (floats): two p buffers, the injection weights, then either
// the CPML arrays (psi_x, psi_z, zeta_x, zeta_z, x addend) or the three
// sponge update weights, then the receiver cache (index, cell offset, 4
// weights per receiver).
template <int RZ>
constexpr size_t rsmem_x(int bc) {
    constexpr size_t WZ = (size_t)NWR * RZ;
    return bc == SIM_BC_CPML ? WZ * (TX + 8) + (WZ + 8) * TX + 3 * WZ * TX : bc == SIM_BC_SPONGE ? 3 * WZ * TX : 0;
}
template <int RZ>
constexpr size_t rsmem_floats(int bc) {
    constexpr size_t WZ = (size_t)NWR * RZ;
    const size_t coef = bc == SIM_BC_CPML ? 2 * (TX + 8) + 2 * (WZ + 8) : 0;  // CPML a, b slices
    return 2 * (WZ + 2 * HM) * SW + WZ * TX + rsmem_x<RZ>(bc) + coef + 6 * (size_t)kRecCache;
}

// Tile-local hull [lo, hi) of the parts of the absorbing strips [0, nb0) and
// [N - nb1, N) of one axis that fall in [clip0, clip1) (tile coordinates,
// origin o); lo >= hi when neither strip reaches the window.
__device__ __forceinline__ void strip_hull(int o, int N, int nb0, int nb1, int clip0, int clip1, int &lo, int &hi) {
    lo = 1 << 30;
    hi = -(1 << 30);
    if (nb0 > 0) {
        const int a = max(-o, clip0), b = min(nb0 - o, clip1);
        if (a < b) lo = min(lo, a), hi = max(hi, b);
    }
    if (nb1 > 0) {
        const int a = max(N - nb1 - o, clip0), b = min(N - o, clip1);
        if (a < b) lo = min(lo, a), hi = max(hi, b);
    }
}

template <int RZ>
__global__ void __launch_bounds__(NTR, 1) k_resident2d(const StepArgs<float> A, const ResidentArgs R) {
    constexpr int WZ = NWR * RZ;
    extern __shared__ float4 smem4[];
    __shared__ int s_abort;
    const bool cpml = A.bc == SIM_BC_CPML;
    float *const S0 = reinterpret_cast<float *>(smem4);
    float *const S1 = S0 + (WZ + 2 * HM) * SW;
    float *const INJ = S1 + (WZ + 2 * HM) * SW;    // WZ x TX: injection weight per cell
    float *const X0 = INJ + WZ * TX;
    // CPML
    float *const PX = X0;                          // WZ x (TX + 8): psi_x, cells [-4, TX + 4)
    float *const PZ = PX + WZ * (TX + 8);          // (WZ + 8) x TX: psi_z, rows [-4, WZ + 4)
    float *const ZX = PZ + (WZ + 8) * TX;          // WZ x TX: zeta_x
    float *const ZZ = ZX + WZ * TX;                // WZ x TX: zeta_z
    float *const AX = ZZ + WZ * TX;                // WZ x TX: D1x psi_x + zeta_x
    // sponge update weights
    float *const KA = X0, *const KB = X0 + WZ * TX, *const KC = X0 + 2 * WZ * TX;
    // CPML recursion coefficients of the subdomain: x in [-4, TX + 4), rows [-4, WZ + 4)
    float *const CAX = X0 + rsmem_x<RZ>(A.bc), *const CBX = CAX + TX + 8;
    float *const CAZ = CBX + TX + 8, *const CBZ = CAZ + WZ + 8;
    // receiver cache
    int *const RIDX = reinterpret_cast<int *>(X0 + rsmem_x<RZ>(A.bc) + (cpml ? 2 * (TX + 8) + 2 * (WZ + 8) : 0));
    int *const ROFF = RIDX + kRecCache;
    float *const RW = reinterpret_cast<float *>(ROFF + kRecCache);

    const Geom &g = A.g;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, tid = threadIdx.x;
    const int ntiles = R.ntiles;
    const int shot = blockIdx.x / ntiles, tile = blockIdx.x - shot * ntiles;
    const RTile *const D = R.tiles + tile;
    const int bx = D->bx, x0 = bx * TX, z0 = D->z0, rows = D->rows, rpw = D->rpw, P = g.P;
    const int my_nbr = lane < D->nnbr ? D->nbr[lane] : -1;  // the subdomain lane polls (warp 0)
    const long long sh = (long long)shot * g.fstride;
    const long long org = cell_off(g, z0, 0, x0);
    float *const gb0 = A.pbuf[0] + sh + org;
    float *const gb1 = A.pbuf[1] + sh + org;
    int *const done = R.done + shot * ntiles;

    const bool cpx = cpml && A.ca[2] &&
                     ((g.nbx0 > 0 && x0 - 4 < g.nbx0) || (g.nbx1 > 0 && x0 + TX + 4 > g.NX - g.nbx1));
    const bool cpz = cpml && A.ca[0] &&
                     ((g.nbz0 > 0 && z0 - 4 < g.nbz0) || (g.nbz1 > 0 && z0 + rows + 4 > g.NZ - g.nbz1));
    const bool spg = A.bc == SIM_BC_SPONGE &&
                     ((g.nbx0 > 0 && x0 < g.nbx0) || (g.nbx1 > 0 && x0 + TX > g.NX - g.nbx1) ||
                      (g.nbz0 > 0 && z0 < g.nbz0) || (g.nbz1 > 0 && z0 + rows > g.NZ - g.nbz1));
    const bool xedge = x0 + TX > g.NX;
    const bool top = g.fs && z0 == 0;
    const int H = cpml ? 8 : 4;                   // exchanged border depth
    const bool hasN = z0 > 0, hasS = z0 + rows < g.NZ, hasW = bx > 0, hasE = x0 + TX < g.NX;
    const int c0 = HM + 4 * lane, gx0 = x0 + 4 * lane, rb = HM + w * rpw;
    const int lo = w * rpw * P + 4 * lane;

    // CPML work ranges. x: psi on float4 chunks cx0 <= c < cx1 of PX (chunk c
    // holds cells [4c - 4, 4c)), zeta_x / addend on own chunks [ax0, ax1).
    // z: psi on rows [zp0, zp1) of [-4, rows + 4), zeta_z on rows [zz0, zz1).
    int cx0 = 0, cx1 = 0, ax0 = 0, ax1 = 0, zp0 = 0, zp1 = 0, zz0 = 0, zz1 = 0;
    if (cpx) {
        int plo, phi;
        strip_hull(x0, g.NX, g.nbx0, g.nbx1, -4, TX + 4, plo, phi);
        if (plo < phi) {
            cx0 = (plo + 4) >> 2;
            cx1 = (phi + 4 + 3) >> 2;
            ax0 = max(0, plo - 4) >> 2;
            ax1 = (min(TX, phi + 4) + 3) >> 2;
        }
    }
    if (cpz) {
        strip_hull(z0, g.NZ, g.nbz0, g.nbz1, -4, rows + 4, zp0, zp1);
        if (zp0 < zp1) {
            zz0 = max(0, zp0 - 4);
            zz1 = min(rows, zp1 + 4);
        } else {
            zp0 = zp1 = 0;
        }
    }
    const int ncx = cx1 - cx0, nax = ax1 - ax0;

    // Shared memory starts at zero: the halo of an absent neighbour, the rows
    // and columns beyond the grid and every CPML value outside the strips.
    {
        const int n4 = (int)(rsmem_floats<RZ>(A.bc) / 4);
        for (int i = tid; i < n4; i += NTR) smem4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (tid == 0) s_abort = 0;

    // run constants of the thread's own cells
    float4 ch4[RZ];
#pragma unroll
    for (int j = 0; j < RZ; j++) {
        const bool in = j < rpw && w * rpw + j < rows;
        ch4[j] = in ? __ldg(reinterpret_cast<const float4 *>(A.ch + org + lo + j * P)) : make_float4(0, 0, 0, 0);
    }
    if (cpml) {
        for (int i = tid; i < TX + 8; i += NTR) {
            CAX[i] = A.ca[2] ? A.ca[2][x0 - 4 + i] : 0.f;
            CBX[i] = A.cb[2] ? A.cb[2][x0 - 4 + i] : 0.f;
        }
        for (int i = tid; i < WZ + 8; i += NTR) {
            const int gz = z0 - 4 + i;
            const bool in = A.ca[0] && gz >= 0 && gz < g.NZ;
            CAZ[i] = in ? A.ca[0][gz] : 0.f;
            CBZ[i] = in ? A.cb[0][gz] : 0.f;
        }
    }
    __syncthreads();
    if (spg) {  // sponge: out = KA p - KB p^{n-1} + KC rhs, a = c (eta_z + eta_x)
        const float4 E4 = __ldg(reinterpret_cast<const float4 *>(A.E[2] + gx0));
#pragma unroll
        for (int j = 0; j < RZ; j++) {
            const int lz = w * rpw + j, gz = z0 + lz;
            if (j >= rpw || lz >= rows) continue;
            const float ez = A.E[0][gz];
            float ka[4], kb[4], kc[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float chv = lane_of(ch4[j], k), a = chv * (ez + lane_of(E4, k)), inv = 1.f / (1.f + a);
                ka[k] = 2.f * inv;
                kb[k] = (1.f - a) * inv;
                kc[k] = chv * inv;
            }
            st4(KA + lz * TX + 4 * lane, make_float4(ka[0], ka[1], ka[2], ka[3]));
            st4(KB + lz * TX + 4 * lane, make_float4(kb[0], kb[1], kb[2], kb[3]));
            st4(KC + lz * TX + 4 * lane, make_float4(kc[0], kc[1], kc[2], kc[3]));
        }
    }
    // Point sources: the injected value of a target cell at step n is its
    // weight (sum of its entries' weights) times w(n); the target cells are
    // fixed, so their weights are set once and the step only scales them.
    const int itile = A.inj_per_shot ? shot * ntiles + tile : tile;
    const int g0 = A.inj_start[itile], g1 = A.inj_start[itile + 1];
    const bool has_inj = g1 > g0;
    for (int gi = g0 + tid; gi < g1; gi += NTR) {
        const InjGroup G = A.inj_grp[gi];
        float wsum = 0.f;
        for (int e = G.e0; e < G.e1; e++) wsum += A.inj_ent[e].w;
        INJ[G.cell] = wsum;
    }
    const int r0 = A.sample ? A.rec_start[tile] : 0, r1 = A.sample ? A.rec_start[tile + 1] : 0;
    const bool rec_cached = r1 - r0 <= kRecCache;
    if (rec_cached)
        for (int e = r0 + tid; e < r1; e += NTR) {
            const RecEntryT<float> Rc = A.rec[e];
            RIDX[e - r0] = Rc.rec;
            ROFF[e - r0] = (HM + Rc.lz) * SW + HM + Rc.lx;
            for (int q = 0; q < 4; q++) RW[4 * (e - r0) + q] = Rc.w[q];
        }
    const SimIO *io = A.io;
    const float *const wav = static_cast<const float *>(io->wavelet);
    float *const gout = static_cast<float *>(io->gather);
    float *const snaps = static_cast<float *>(io->snaps);
    const int nrec = io->nrec;
    float wnext = (has_inj && A.nt > 0) ? wav[0] : 0.f;
    __syncthreads();

    for (int n = 0; n < A.nt; n++) {
        float *const cur = (n & 1) ? S1 : S0;
        float *const nxt = (n & 1) ? S0 : S1;
        const float *const gcur = (n & 1) ? gb1 : gb0;
        float *const gnxt = (n & 1) ? gb0 : gb1;

        // this step's wavelet sample (fetched one step ahead)
        const float wn = wnext;
        if (has_inj && n + 1 < A.nt) wnext = wav[n + 1];

        if (n > 0) {
            // the subdomains whose borders form the halo must have published p^n
            if (w == 0) {
                const int nb = my_nbr;
                bool need = nb >= 0, quit = false;
                long long spins = 0;
                for (;;) {
                    if (need && ld_acquire(done + nb) >= n) need = false;
                    if (!__any_sync(0xffffffffu, need)) break;
                    if (++spins > R.spin_limit) {
                        quit = true;
                        if (lane == 0) atomicOr(A.flags, kFlagTimeout);
                        break;
                    }
                    if ((spins & 1023) == 0) {
                        const unsigned f = lane == 0 ? *reinterpret_cast<volatile unsigned *>(A.flags) : 0u;
                        if (__shfl_sync(0xffffffffu, f, 0) & kFlagTimeout) {
                            quit = true;
                            break;
                        }
                    }
                }
                if (lane == 0) s_abort = quit;
            }
            __syncthreads();
            if (s_abort) return;
            // their borders become this step's halo
            if (hasN)
                for (int i = tid; i < H * 32; i += NTR) {
                    const int r = -H + (i >> 5), c = 4 * (i & 31);
                    cp_async16(cur + (HM + r) * SW + HM + c, gcur + r * P + c);
                }
            if (hasS)
                for (int i = tid; i < H * 32; i += NTR) {
                    const int r = rows + (i >> 5), c = 4 * (i & 31);
                    cp_async16(cur + (HM + r) * SW + HM + c, gcur + r * P + c);
                }
            const int hq = H / 4;
            if (hasW)
                for (int i = tid; i < rows * hq; i += NTR) {
                    const int r = i / hq, q = i - r * hq;
                    cp_async16(cur + (HM + r) * SW + HM - H + 4 * q, gcur + r * P - H + 4 * q);
                }
            if (hasE)
                for (int i = tid; i < rows * hq; i += NTR) {
                    const int r = i / hq, q = i - r * hq;
                    cp_async16(cur + (HM + r) * SW + HM + TX + 4 * q, gcur + r * P + TX + 4 * q);
                }
            cp_async_wait_all();
        }
        __syncthreads();
        if (top && n > 0) {  // odd mirror above the free surface: p(-k) = -p(k)
            const int nch = (TX + 2 * H) / 4;
            for (int k = 1 + w; k <= H; k += NWR) {
                float4 *d = reinterpret_cast<float4 *>(cur + (HM - k) * SW + (HM - H));
                const float4 *sr = reinterpret_cast<const float4 *>(cur + (HM + k) * SW + (HM - H));
                for (int c = lane; c < nch; c += 32) {
                    const float4 v = sr[c];
                    d[c] = make_float4(-v.x, -v.y, -v.z, -v.w);
                }
            }
            __syncthreads();
        }

        // CPML psi^n = b psi^{n-1} + a D1 p^n (scaled by h) on the strips
        if (ncx > 0) {
            for (int i = tid; i < rows * ncx; i += NTR) {
                const int lz = i / ncx, c = cx0 + (i - lz * ncx), gz = z0 + lz, gx = x0 + 4 * c - 4;
                const float *row = cur + (HM + lz) * SW + HM + 4 * c - 4;
                float v[12];
                unpack3(ld4(row - 4), ld4(row), ld4(row + 4), v);
                const float4 a4 = ld4(CAX + 4 * c), b4 = ld4(CBX + 4 * c);
                float *px = PX + lz * (TX + 8) + 4 * c;
                const float4 old = ld4(px);
                float o4[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const bool in = gz < g.NZ && gx + k >= 0 && gx + k < g.NX;
                    o4[k] = in ? lane_of(b4, k) * lane_of(old, k) + lane_of(a4, k) * d1w(v, k) : 0.f;
                }
                st4(px, make_float4(o4[0], o4[1], o4[2], o4[3]));
            }
        }
        if (zp1 > zp0) {
            for (int lzz = zp0 + w; lzz < zp1; lzz += NWR) {
                const int gz = z0 + lzz;
                const float *col = cur + (HM + lzz) * SW + c0;
                float4 q[9];
#pragma unroll
                for (int m = 0; m < 9; m++) q[m] = ld4(col + (m - 4) * SW);
                const bool zin = gz >= 0 && gz < g.NZ;
                const float az = CAZ[lzz + 4], bz = CBZ[lzz + 4];
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
                st4(pz, make_float4(o4[0], o4[1], o4[2], o4[3]));
            }
        }
        if (ncx > 0 || zp1 > zp0) __syncthreads();

        // zeta_x^n = b zeta_x^{n-1} + a (D2x p^n + D1x psi_x^n) and the addend
        // D1x psi_x^n + zeta_x^n on the widened x-strips
        if (nax > 0) {
            for (int i = tid; i < rows * nax; i += NTR) {
                const int lz = i / nax, c = ax0 + (i - lz * nax);
                float v[12], px[12];
                const float *row = cur + (HM + lz) * SW + HM + 4 * c;
                unpack3(ld4(row - 4), ld4(row), ld4(row + 4), v);
                const float *pr = PX + lz * (TX + 8) + 4 * c;
                unpack3(ld4(pr), ld4(pr + 4), ld4(pr + 8), px);
                const float4 a4 = ld4(CAX + 4 * c + 4), b4 = ld4(CBX + 4 * c + 4);
                float *zp = ZX + lz * TX + 4 * c;
                const float4 z4 = ld4(zp);
                float zo[4], ad[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float dps = d1w(px, k);
                    zo[k] = lane_of(b4, k) * lane_of(z4, k) + lane_of(a4, k) * (d2w(v, k) + dps);
                    ad[k] = dps + zo[k];
                }
                st4(zp, make_float4(zo[0], zo[1], zo[2], zo[3]));
                st4(AX + lz * TX + 4 * c, make_float4(ad[0], ad[1], ad[2], ad[3]));
            }
            __syncthreads();
        }

        // update: p^{n+1} into the other buffer, borders to the global buffer
        float4 zw[RZ + 8];
#pragma unroll
        for (int j = 0; j < RZ + 8; j++) zw[j] = ld4(cur + (rb - 4 + j) * SW + c0);
#pragma unroll
        for (int j = 0; j < RZ; j++) {
            const int lz = w * rpw + j;
            if (j >= rpw || lz >= rows) continue;
            float v[12];
            unpack3(ld4(cur + (rb + j) * SW + c0 - 4), zw[j + 4], ld4(cur + (rb + j) * SW + c0 + 4), v);
            const float4 pp4 = ld4(nxt + (rb + j) * SW + c0);  // p^{n-1}
            float4 ax4 = make_float4(0, 0, 0, 0), inj4 = make_float4(0, 0, 0, 0);
            if (cpx) ax4 = ld4(AX + lz * TX + 4 * lane);
            if (has_inj) inj4 = ld4(INJ + lz * TX + 4 * lane);
            // zeta_z^n = b zeta_z^{n-1} + a (D2z p^n + D1z psi_z^n) on the widened z-strips
            const bool zrow = lz >= zz0 && lz < zz1;
            float4 dz4 = make_float4(0, 0, 0, 0), zz4 = make_float4(0, 0, 0, 0);
            float az = 0.f, bzc = 0.f;
            if (zrow) {
                const float *pzc = PZ + (lz + 4) * TX + 4 * lane;
                float4 a = ld4(pzc + TX), b = ld4(pzc - TX);
                float d[4];
#pragma unroll
                for (int k = 0; k < 4; k++) d[k] = float(kD1) * (lane_of(a, k) - lane_of(b, k));
                a = ld4(pzc + 2 * TX), b = ld4(pzc - 2 * TX);
#pragma unroll
                for (int k = 0; k < 4; k++) d[k] += float(kD2) * (lane_of(a, k) - lane_of(b, k));
                a = ld4(pzc + 3 * TX), b = ld4(pzc - 3 * TX);
#pragma unroll
                for (int k = 0; k < 4; k++) d[k] += float(kD3) * (lane_of(a, k) - lane_of(b, k));
                a = ld4(pzc + 4 * TX), b = ld4(pzc - 4 * TX);
#pragma unroll
                for (int k = 0; k < 4; k++) d[k] += float(kD4) * (lane_of(a, k) - lane_of(b, k));
                dz4 = make_float4(d[0], d[1], d[2], d[3]);
                zz4 = ld4(ZZ + lz * TX + 4 * lane);
                az = CAZ[lz + 4];
                bzc = CBZ[lz + 4];
            }
            float4 ka4 = make_float4(0, 0, 0, 0), kb4 = ka4, kc4 = ka4;
            if (spg) {
                ka4 = ld4(KA + lz * TX + 4 * lane);
                kb4 = ld4(KB + lz * TX + 4 * lane);
                kc4 = ld4(KC + lz * TX + 4 * lane);
            }
            float res[4], zo[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float p = v[4 + k];
                const float d2x = d2w(v, k);
                const float d2z = d2c<float>(p, lane_of(zw[j + 3], k), lane_of(zw[j + 5], k), lane_of(zw[j + 2], k), lane_of(zw[j + 6], k),
                                         lane_of(zw[j + 1], k), lane_of(zw[j + 7], k), lane_of(zw[j], k), lane_of(zw[j + 8], k));
                float rhs = d2z + d2x;
                if (cpx) rhs += lane_of(ax4, k);
                zo[k] = 0.f;
                if (zrow) {
                    zo[k] = bzc * lane_of(zz4, k) + az * (d2z + lane_of(dz4, k));
                    rhs += lane_of(dz4, k) + zo[k];
                }
                if (has_inj) rhs += A.src_scale * (lane_of(inj4, k) * wn);
                const float pp = lane_of(pp4, k);
                res[k] = spg ? lane_of(ka4, k) * p - lane_of(kb4, k) * pp + lane_of(kc4, k) * rhs
                             : 2.f * p - pp + lane_of(ch4[j], k) * rhs;
            }
            if (zrow) st4(ZZ + lz * TX + 4 * lane, make_float4(zo[0], zo[1], zo[2], zo[3]));
            if (xedge) {
#pragma unroll
                for (int k = 0; k < 4; k++)
                    if (gx0 + k >= g.NX) res[k] = 0.f;
            }
            if (top && lz == 0) res[0] = res[1] = res[2] = res[3] = 0.f;
            const float4 r4 = make_float4(res[0], res[1], res[2], res[3]);
            st4(nxt + (rb + j) * SW + c0, r4);
            const bool border = (hasN && lz < H) || (hasS && lz >= rows - H) || (hasW && 4 * lane < H) ||
                                (hasE && 4 * lane >= TX - H);
            if (border) st4(gnxt + lo + j * P, r4);
        }

        // publish p^{n+1}: the release orders every thread's border stores
        // (ordered before it by the barrier) before the counter
        __syncthreads();
        if (tid == 0) st_release(done + tile, n + 1);

        // Off the critical path, while the neighbours proceed: receivers and
        // the snapshot sample p^n, still held in this buffer until the next
        // step's update overwrites it.
        if (r1 > r0 && gout) {
            const long long rowo = ((long long)shot * A.nt + n) * nrec;
            for (int e = tid; e < r1 - r0; e += NTR) {
                int ri, off;
                float w4[4];
                if (rec_cached) {
                    ri = RIDX[e];
                    off = ROFF[e];
                    for (int q = 0; q < 4; q++) w4[q] = RW[4 * e + q];
                } else {
                    const RecEntryT<float> Rc = A.rec[r0 + e];
                    ri = Rc.rec;
                    off = (HM + Rc.lz) * SW + HM + Rc.lx;
                    for (int q = 0; q < 4; q++) w4[q] = Rc.w[q];
                }
                const float *b = cur + off;
                const float val = w4[0] * b[0] + w4[1] * b[1] + w4[2] * b[SW] + w4[3] * b[SW + 1];
                gout[rowo + ri] = val;
                if (!isfinite(val)) atomicOr(A.flags, kFlagUnstable);
            }
        }
        if (snaps && A.nsnap > 0 && n >= A.snap_begin && n < A.snap_end && (n - A.snap_begin) % A.snap_every == 0) {
            const int snap_k = (n - A.snap_begin) / A.snap_every;
            const long long sbase = ((long long)shot * A.nsnap + snap_k) * g.nz * g.nx;
#pragma unroll
            for (int j = 0; j < RZ; j++) {
                const int gz = z0 + w * rpw + j;
                if (j >= rpw || w * rpw + j >= rows || gz < g.oz || gz >= g.oz + g.nz) continue;
                const float4 p4 = ld4(cur + (rb + j) * SW + c0);
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int gx = gx0 + k;
                    if (gx < g.ox || gx >= g.ox + g.nx) continue;
                    snaps[sbase + (long long)(gz - g.oz) * g.nx + (gx - g.ox)] = lane_of(p4, k);
                }
            }
        }
    }

    // final state: p^nt and p^{nt-1} into the global buffers of the per-step
    // layout (the buffer written last holds p^nt); own cells only, each
    // thread copying the cells it wrote
    if (A.nt > 0) {
        const float *fin = (A.nt & 1) ? S1 : S0, *prv = (A.nt & 1) ? S0 : S1;
        float *gl = (A.nt & 1) ? gb1 : gb0, *gp = (A.nt & 1) ? gb0 : gb1;
#pragma unroll
        for (int j = 0; j < RZ; j++) {
            if (j >= rpw || w * rpw + j >= rows) continue;
            st4(gl + lo + j * P, ld4(fin + (rb + j) * SW + c0));
            st4(gp + lo + j * P, ld4(prv + (rb + j) * SW + c0));
        }
    }
}

template <int RZ>
cudaError_t launch_rz(const StepArgs<float> &a, const ResidentArgs &r, int nshots, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(r.ntiles * nshots);
    cfg.blockDim = dim3(NTR);
    cfg.dynamicSmemBytes = rsmem_floats<RZ>(a.bc) * sizeof(float);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_resident2d<RZ>, a, r);
}

template <int RZ>
int blocks_per_sm(int bc) {
    const size_t bytes = rsmem_floats<RZ>(bc) * sizeof(float);
    if (bytes > kResidentMaxSmem) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_resident2d<RZ>, NTR, bytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

template <int RZ>
cudaError_t configure_rz() {
    size_t most = rsmem_floats<RZ>(SIM_BC_NONE);
    for (int bc : {SIM_BC_SPONGE, SIM_BC_CPML})
        if (rsmem_floats<RZ>(bc) * sizeof(float) <= kResidentMaxSmem) most = std::max(most, rsmem_floats<RZ>(bc));
    return cudaFuncSetAttribute(k_resident2d<RZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(most * sizeof(float)));
}

}  // namespace

cudaError_t configure_resident2d() {
    cudaError_t e = configure_rz<1>();
    if (e == cudaSuccess) e = configure_rz<2>();
    if (e == cudaSuccess) e = configure_rz<3>();
    if (e == cudaSuccess) e = configure_rz<4>();
    return e;
}

int resident2d_blocks_per_sm(int rz, int bc) {
    switch (rz) {
        case 1: return blocks_per_sm<1>(bc);
        case 2: return blocks_per_sm<2>(bc);
        case 3: return blocks_per_sm<3>(bc);
        case 4: return blocks_per_sm<4>(bc);
        default: return 0;
    }
}

cudaError_t launch_resident2d(const StepArgs<float> &a, const ResidentArgs &r, int rz, int nshots,
                              cudaStream_t st) {
    switch (rz) {
        case 1: return launch_rz<1>(a, r, nshots, st);
        case 2: return launch_rz<2>(a, r, nshots, st);
        case 3: return launch_rz<3>(a, r, nshots, st);
        case 4: return launch_rz<4>(a, r, nshots, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gsim
