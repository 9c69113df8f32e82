// Internal declarations of libsim: field layout, kernel argument blocks and
// the launch entry points each translation unit provides. Host code is C++17.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sim.h"

namespace gsim {

// ---------------------------------------------------------------- layout
//
// Every field (pressure ping-pong buffers, c = (v dt / h)^2, velocity, CPML
// memory) uses one padded layout per shot: the computational grid (interior +
// absorbing cells, NZ x NY x NX) surrounded by kGhost cells of zeros on every
// side, rows padded to a multiple of 32 elements. The ghost cells are never
// written, so a stencil that reads them sees p = 0 (Dirichlet) without a
// bounds check. Cell (z, y, x) of the computational grid sits at
//     org + (z * PY + y) * P + x
// where PY is the number of rows per z-plane (1 in 2D).
constexpr int kGhost = 8;      // >= the widest halo any kernel reads (CPML recompute)
constexpr int kTileX2 = 32;    // 2D tile (x) of the generic (any precision) stencil kernel
constexpr int kTileZ2 = 16;    // 2D tile (z) of the generic kernel
constexpr int kTileXF = 128;   // 2D tile (x) of the FP32 kernel; its z extent is tuned (8, 16, 32)
constexpr int kProfAlign = 128; // per-axis profile segments: aligned starts, room for a whole last tile
constexpr int kRoundX = 128;   // padded extents round up to these, so any tile
constexpr int kRoundZ = 32;    //   of the tuned set stays inside the allocation
constexpr int kRoundY = 32;
constexpr int kMinmaxBlocks = 512;  // partial (min, max, bad) triples written by launch_minmax

struct Geom {
    int ndim;
    int NZ, NY, NX;        // computational grid
    int nz, ny, nx;        // interior
    int oz, oy, ox;        // interior origin in the computational grid
    int nbz0, nbz1, nby0, nby1, nbx0, nbx1;
    int P;                 // row pitch (elements)
    int PY;                // rows per z-plane (1 in 2D)
    long long fstride;     // elements per field
    long long org;         // offset of cell (0,0,0)
    int fs;                // free surface on top
};

__host__ __device__ inline long long cell_off(const Geom &g, int z, int y, int x) {
    return g.org + ((long long)z * g.PY + y) * g.P + x;
}

// Receiver: base cell of its linear-interpolation stencil (local to the tile
// that samples it) and the 4 (2D) or 8 (3D) corner weights, corner order
// (dz, dy, dx) with dx fastest.
template <typename W>
struct RecEntryT {
    int rec;
    int lz, ly, lx;
    W w[8];
};

// Injection: one group per target cell of a tile, summing its entries in a
// fixed order (so the result is deterministic), value = weight * input[pt].
struct InjGroup {
    int cell;   // local linear index lz * TX + lx (2D) / (lz*TY + ly)*TX + lx (3D)
    int e0, e1; // entry range
    int pad;
};
template <typename W>
struct InjEntryT {
    int pt;     // index of the input value (shot for a source, receiver for a residual)
    W w;
};

// Per-call I/O block, resident on the device and refreshed before each run,
// so captured graphs stay valid across calls.
struct SimIO {
    const void *wavelet;     // [nt] (shared by the shots)
    void *gather;            // [nshots][nt][nrec]
    void *snaps;             // [nshots][nsnap][interior]
    float *snap_scale;       // [nshots][nsnap]
    unsigned *snap_max;      // [nshots][nsnap] float bits of max |p|
    const void *resid;       // [nshots][nt][nrec] adjoint residual
    int nrec;
    int nshots;
    int snap_fp16;
    int pad;
};

enum : unsigned { kFlagUnstable = 1u, kFlagTimeout = 2u };

template <typename T>
struct StepArgs {
    Geom g;
    T *pbuf[2];              // ping-pong bases (per shot: + shot * fstride)
    const T *ch;             // (v dt / h)^2, field layout, shared by the shots
    const T *E[3];           // sponge profile per axis: eta h^2 / (2 dt); NULL = none
    const T *ca[3], *cb[3];  // CPML recursion coefficients per axis; NULL = axis absent
    T *psi[3][2];            // CPML psi ping-pong (scaled by h), per shot stride fstride
    T *zeta[3];              // CPML zeta (scaled by h^2)
    int bc;
    T src_scale;             // h^(2-d)
    int ntx, nty, ntz;       // tiles per shot
    int nt;
    int nsnap, snap_every, snap_begin, snap_end;
    // receivers (tile-local lists, shared by the shots)
    const int *rec_start;
    const RecEntryT<T> *rec;
    // injection (sources: per shot and tile; residuals: per tile)
    const int *inj_start;
    const InjGroup *inj_grp;
    const InjEntryT<T> *inj_ent;
    int inj_per_shot;        // 1: inj lists are indexed by shot * ntiles + tile
    int inj_kind;            // 0: value = wavelet[n]; 1: value = resid[shot][n][pt]
    const SimIO *io;
    unsigned *flags;
    int sample;              // 1: receivers sample p^n into io->gather
    int inj_reverse;         // 1: injection row = nt - n (adjoint sweep), rows >= nt inject 0
    // adjoint-state imaging term Q'^n = E (p^{n+1} - p^{n-1}) - h^2 (L p^n + s^n), per cell
    void *qslot;             // this launch's slot, field layout per shot (T, or half when q_fp16)
    float *qscale;           // FP16 slots: power-of-two scale per [shot][tile]
    int q_fp16;
    T *G;                    // adjoint sweep: G += u^{n+1} Q'^n, field layout per shot
    const T *cext;           // adjoint sweep of a CPML problem: per-cell term added to the Laplacian
};

// Per-launch facts of one step, resolved on the host (so the kernel does no
// integer division on them): buffer parity / gather row, snapshot index to
// write (-1: none), snapshot index whose FP16 scale this step's output feeds
// (-1: none), injection row (-1: none), and the imaging-term slot.
struct StepTime {
    int n;
    int snap_k;
    int max_k;
    int inj_row;
    void *qslot;
    float *qscale;
};

// CPML terms of the adjoint sweep (cpml_adj.cu): the multipliers nu (of
// zeta) and mu (of psi) of each absorbing axis, nu ping-ponged by step
// parity; in 2D the term `ext` the step kernel adds to the Laplacian of u
// (A.cext), in 3D c times that term added to u^k after the update.
template <typename T>
struct CpmlAdjArgs {
    const T *u;   // u^{k+1}, field layout per shot
    T *nu[3][2];  // [axis][parity] (absent axes unused)
    T *mu[3];     // [axis]
    T *ext;       // 2D: the bracket, added to the Laplacian by the step kernel
    T *uo;        // 3D: u^k, receives c times the bracket (NULL in 2D)
    const T *q;   // 3D: the recorded imaging term of the step
    T *G;         // 3D: gradient accumulator
};
template <typename T>
cudaError_t launch_cpml_adjoint(const StepArgs<T> &a, const CpmlAdjArgs<T> &c, int parity, int nshots,
                                cudaStream_t st);

// Step kernel modes: plain forward; forward that records Q'^n; adjoint sweep
// that accumulates G from the recorded Q'.
enum StepMode { kModeForward = 0, kModeRecord = 1, kModeAdjoint = 2 };

// A point of the 3D path: field offsets of its 8 trilinear corners (-1 where
// the weight is zero or the corner is a held free-surface cell) and weights.
struct Pt3 {
    long long cell[8];
    float w[8];
};

// Batch (persistent) execution: see k_batch2d in fwd2d_f32.cu.
struct BatchMember {
    int slice;       // index into BatchArgs::slices
    int shot;
    int tile0;       // first of this member's tiles within one step of its group
    int done0;       // offset of this member's per-tile step counters
};
struct BatchGroup {
    long long base;  // first item of the group
    int T;           // tiles per step over the group's members
    int m0, m1;      // member range
};
struct BatchArgs {
    const StepArgs<float> *slices;
    const BatchGroup *groups;
    int ngroups;
    int nmembers;
    const BatchMember *members;
    int *done;                 // per (slice, shot, tile): steps completed
    unsigned long long *head;  // work counter
    long long total;           // items
    long long spin_limit;      // polls before a wait gives up
    unsigned *flags;           // kFlagTimeout on a wait that gave up
};
cudaError_t launch_batch2d(const BatchArgs &b, int tz, bool cpml, int grid, cudaStream_t st);
// Stepped batch (k_multi2d): step n of every member in one launch of
// nblocks = all members' tiles; members' tile0 is global (prefix over members).
cudaError_t launch_multi2d(const BatchArgs &b, int tz, bool cpml, int nblocks, int n, cudaStream_t st, bool pdl);
int batch_blocks_per_sm(int tz, bool cpml);

// Row march (march2d.cu): the 2D FP32 forward step as warps that each walk
// down the rows [z0, z1) of one 128-column strip (bx) of one member (slice,
// shot). The warps take the nitems segments in order from the step's
// counter ctr[n & 1] (ctr[0] zeroed before the first step; each step zeroes
// the next step's). tz is the tile height of the slices' receiver and
// injection lists.
constexpr int kMarchW = 128;
struct MarchSeg {
    int slice, shot, bx, z0, z1;
    int pad[3];
};
struct MarchArgs {
    const StepArgs<float> *slices;
    const MarchSeg *segs;
    unsigned *ctr;
    int nwarps;
    int nitems;
    int tz;
    int pad;
};
cudaError_t configure_march2d();
int march2d_warps_per_sm(bool cpml);
cudaError_t launch_march2d(const MarchArgs &m, bool cpml, const StepTime &t, cudaStream_t st, bool pdl);

// Temporal blocking of the row march (march2x.cu): two steps per pass for
// members without CPML. A member (slice, shot) has two more pressure fields
// (p3 and p3 + pstride: the four fields alternate as two pairs over the
// passes) and up to four source corners; items are MarchSeg over 120-column
// strips (slice = member index). Receivers are TBSample entries sampled
// after each pass.
constexpr int kTBW = 120;
struct TBMember {
    int slice, shot;
    float *p3;             // third and fourth pressure fields of the slice (per shot: + shot * fstride)
    long long pstride;     // from the third field to the fourth
    int nsrc, pad;
    int sz[4], sx[4];      // source corners: computational-grid row and column
    float sw[4];           // bilinear weights
};
struct TBSample {
    int member, rec;
    int z, x;              // base cell (computational grid) of the 2 x 2 corners
    float w[4];            // corner weights (z, x), (z, x+1), (z+1, x), (z+1, x+1)
};
struct TBArgs {
    const StepArgs<float> *slices;
    const TBMember *members;
    const MarchSeg *segs;
    const TBSample *samples;
    unsigned *ctr;         // two per-pass item counters
    int nitems;
    int pad;
    long long nsamples;
};
struct TBPass {
    int k;                 // pass index: even passes read fields 0, 1, odd passes fields 2, 3
    int n;                 // first step of the pass
    int two;               // 1: steps n and n + 1; 0: step n only
    int inj0, inj1;        // wavelet rows injected at the two steps (-1: none)
    int pad;
};
cudaError_t configure_march2x();
int march2x_warps_per_sm();
cudaError_t launch_march2x(const TBArgs &b, const TBPass &t, int nwarps, cudaStream_t st);

// 3D launchers (fwd3d.cu). Per step: snapshot, sample, CPML psi, z-march
// update, CPML zeta + addend, source injection.
// z-march variants: kZMarchAsync stages each plane by per-thread 16-byte
// cp.async copies; kZMarchTma by three bulk tensor copies (TMA) per plane
// issued by one thread, completion on mbarriers, and folds the x-strip CPML
// in where it can; kZMarchTmaPlain is the TMA march leaving the x strips to
// their own pass; the two ...Loop variants are the same without unrolling
// the plane loop (smaller code, the register queue shifted by moves);
// kZMarchTmaLoop3 unrolls it by 3 (the queue rotated by moves once per three
// planes). All take z chunks of `zchunk` planes per CTA.
enum { kZMarchAsync = 1, kZMarchTma = 2, kZMarchTmaPlain = 3, kZMarchTmaLoop = 4, kZMarchTmaFoldLoop = 5, kZMarchTmaLoop3 = 6 };
struct Tma3 {
    CUtensorMap ph;  // p (both parities, all shots): 136 x 16 x 1 boxes, the plane with its x / y halo
    CUtensorMap po;  // the same buffers: 128 x 8 x 1 boxes, a tile's own cells
    CUtensorMap c;   // c = (v dt / h)^2: 128 x 8 x 1 boxes
};
cudaError_t configure_step3d();
// The TMA march of the forward and record modes takes over the x-strip CPML
// pass when the widened strips lie inside the first / last x tile.
bool zmarch_folds_x(const StepArgs<float> &a, int variant, int mode);
cudaError_t launch_step3d(const StepArgs<float> &a, int n, int variant, int zchunk, int nshots, cudaStream_t st,
                          bool pdl, int mode = kModeForward, float *qs = nullptr, float *Gs = nullptr);
// 3D point injection grouped by target cell (the adjoint path): group =
// cell offset within a field, entry range, shot (-1: the same for every
// shot, the launch's y index).
struct Inj3 {
    long long cell;
    int e0, e1;
    int shot, pad;
};
struct InjE3 {
    int pt;
    float w;
};
cudaError_t launch_inj3d(const StepArgs<float> &a, int n, int row, const Inj3 *grp, int ngrp, const InjE3 *ent,
                         int kind, int nshots, int mode, float *qs, float *Gs, cudaStream_t st);
cudaError_t launch_cpml3d(const StepArgs<float> &a, int n, int ax, int phase, int nshots, cudaStream_t st,
                          float *qs = nullptr);
cudaError_t launch_sample3d(const StepArgs<float> &a, const StepTime &t, const void *rec, int nrec, int nshots,
                            cudaStream_t st);
cudaError_t launch_inject3d(const StepArgs<float> &a, const StepTime &t, const void *src, int nshots,
                            cudaStream_t st);
cudaError_t launch_snap3d(const StepArgs<float> &a, const StepTime &t, int fp16, int nshots, cudaStream_t st);

// Resident execution (resident2d.cu): one cooperative launch runs the whole
// forward time loop of a 2D FP32 problem whose state fits on chip; each CTA
// of kResidentWarps warps owns one subdomain: columns [128 bx, 128 bx + 128),
// rows [z0, z0 + rows) with rows <= 16 RZ, warps taking rpw rows each.
// nbr lists the subdomains whose borders form its halo (same shot). done[]
// holds one step counter per (shot, subdomain), zeroed before the launch.
constexpr int kResidentWarps = 16;
constexpr size_t kResidentMaxSmem = 227 * 1024;
constexpr int kResidentMaxNbr = 11;
struct RTile {
    int bx, z0, rows, rpw;
    int nnbr;
    int nbr[kResidentMaxNbr];
};
struct ResidentArgs {
    int *done;
    long long spin_limit;
    const RTile *tiles;  // device array, per shot
    int ntiles;
};
cudaError_t configure_resident2d();
int resident2d_blocks_per_sm(int rz, int bc);  // 0: does not fit
cudaError_t launch_resident2d(const StepArgs<float> &a, const ResidentArgs &r, int rz, int nshots,
                              cudaStream_t st);

// Message returned by sim_last_error(NULL) for failures of this thread.
void set_thread_error(const char *msg);

// Launchers (one translation unit each).
template <typename T>
cudaError_t launch_step2d(const StepArgs<T> &a, int n, int nshots, int mode, cudaStream_t st);

// FP32 kernel with a 128 x tz tile (tz in {8, 16, 32}).
// pdl: let step n+1 launch while step n drains (programmatic dependent launch);
// the kernel waits for its predecessor before reading any field.
cudaError_t launch_step2d_f32(const StepArgs<float> &a, const StepTime &t, int tz, int nshots, int mode,
                              cudaStream_t st, bool pdl);
cudaError_t configure_step2d_f32();

// Checkpoint of one state (computational grid of each shot): FP32/FP64 copy
// or FP16 with a power-of-two scale per 2D tile.
template <typename T>
cudaError_t launch_store_state(const Geom &g, const T *field, void *dst, float *scale, int fp16, int nshots,
                               long long shot_stride, int ntx, int ntz, cudaStream_t st);
template <typename T>
cudaError_t launch_load_state(const Geom &g, T *field, const void *src, const float *scale, int fp16, int nshots,
                              long long shot_stride, int ntx, int ntz, cudaStream_t st);
// Checkpoint of the CPML memory of one axis: only the boxes of its strips
// (the memory is zero elsewhere), compact [shot][rows][x] with, in FP16, a
// power-of-two scale per (shot, box row). row0 / elem0 are prefix sums over
// the boxes (row0[n] rows and elem0[n] elements per shot).
struct CkBox {
    int z0, z1, y0, y1, x0, x1;
};
constexpr int kMaxCkBoxes = 2;
struct CkBoxes {
    int n;
    CkBox b[kMaxCkBoxes];
    long long row0[kMaxCkBoxes + 1];
    long long elem0[kMaxCkBoxes + 1];
};
template <typename T>
cudaError_t launch_store_boxes(const Geom &g, const CkBoxes &b, const T *field, void *dst, float *scale, int fp16,
                               int nshots, cudaStream_t st);
template <typename T>
cudaError_t launch_load_boxes(const Geom &g, const CkBoxes &b, T *field, const void *src, const float *scale,
                              int fp16, int nshots, cudaStream_t st);
// res = g - d (all shots), per-block partial sums of res^2 / 2 into part.
template <typename T>
cudaError_t launch_residual(const T *g, const T *d, T *res, long long n, double *part, int nblocks, cudaStream_t st);
// acc[interior] += sum over shots and replicated padding cells of -2 G / (v h^2).
template <typename T>
cudaError_t launch_fold_gradient(const Geom &g, const T *G, long long gshot, int nshots, const T *vpad,
                                 double inv_h2, double *acc, cudaStream_t st);
template <typename T>
cudaError_t launch_add_gradient(const double *acc, T *grad, long long n, cudaStream_t st);

template <typename T>
cudaError_t launch_setup_model(const Geom &g, const T *vel, T *ch, T *vpad, double dt_over_h,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_minmax(const Geom &g, const T *vel, double *out2, cudaStream_t st);
template <typename T>
cudaError_t launch_check_finite(const Geom &g, const T *f, int nshots, unsigned *flags,
                                cudaStream_t st);

}  // namespace gsim
