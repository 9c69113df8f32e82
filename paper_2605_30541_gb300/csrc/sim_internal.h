// Internal declarations of libsim: field layout, kernel argument blocks and
// the launch entry points each translation unit provides. Host code is C++17.
#pragma once

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
constexpr int kTileX2 = 32;    // 2D tile (x) of the stencil kernels
constexpr int kTileZ2 = 16;    // 2D tile (z)
constexpr int kRoundX = 64;    // padded extents round up to these, so any tile
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
struct RecEntry {
    int rec;
    int lz, ly, lx;
    double w[8];
};

// Injection: one group per target cell of a tile, summing its entries in a
// fixed order (so the result is deterministic), value = weight * input[pt].
struct InjGroup {
    int cell;   // local linear index lz * TX + lx (2D) / (lz*TY + ly)*TX + lx (3D)
    int e0, e1; // entry range
    int pad;
};
struct InjEntry {
    int pt;     // index of the input value (shot for a source, receiver for a residual)
    int pad;
    double w;
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
    const RecEntry *rec;
    // injection (sources: per shot and tile; residuals: per tile)
    const int *inj_start;
    const InjGroup *inj_grp;
    const InjEntry *inj_ent;
    int inj_per_shot;        // 1: inj lists are indexed by shot * ntiles + tile
    int inj_kind;            // 0: value = wavelet[n]; 1: value = resid[shot][n][pt]
    const SimIO *io;
    unsigned *flags;
};

// Launchers (one translation unit each).
template <typename T>
cudaError_t launch_step2d(const StepArgs<T> &a, int n, int nshots, cudaStream_t st);

template <typename T>
cudaError_t launch_setup_model(const Geom &g, const T *vel, T *ch, T *vpad, double dt_over_h,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_minmax(const Geom &g, const T *vel, double *out2, cudaStream_t st);
template <typename T>
cudaError_t launch_check_finite(const Geom &g, const T *f, int nshots, unsigned *flags,
                                cudaStream_t st);

}  // namespace gsim
