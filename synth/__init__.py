"""Seeded synthetic inputs for the acoustic FDTD path.

This module produces DATA only — velocity models, source wavelets and
acquisition geometries — and holds none of the solver's arithmetic. Both the
CUDA library's tests/benchmark and the FP64 oracle consume its output; neither
side's code lives here.

The generators stand in for the paper's field-scale slices (App. E.1: 619 x 1000
cells at 10 m, velocities normalised to [1500, 5000] m/s; the dataset itself is
not used): seeded layered models with sinusoidal folding and planar normal
faults. Seeds follow ``seed = 1000 * config + slice`` with numpy's PCG64.

Positions are metres from the interior origin, ordered (x, z) in 2D and
(x, y, z) in 3D.
"""
import math

import numpy as np

VMIN, VMAX = 1500.0, 5000.0


def ricker(f0, t0, dt, nt, dtype=np.float32):
    """Ricker wavelet (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = t - t0,
    sampled at t = n dt (paper Sec. 2 and App. E.4 name it as the source)."""
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f0 * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(dtype)


def two_layer(nz, nx, h, z_if, v_top, v_bot, dtype=np.float32):
    """Flat interface: rows with depth z = row * h < z_if take v_top, others v_bot."""
    z = np.arange(nz) * h
    v = np.where(z[:, None] < z_if, v_top, v_bot) * np.ones((1, nx))
    return v.astype(dtype)


def _layer_table(rng, nl, depth):
    """Layer tops (jittered even spacing) and velocities increasing with depth."""
    k = np.arange(1, nl)
    tops = (k + rng.uniform(-0.3, 0.3, nl - 1)) * depth / nl
    tops = np.sort(tops)
    base = np.linspace(VMIN, 4700.0, nl) + rng.uniform(-300.0, 300.0, nl)
    vel = np.clip(np.sort(base), VMIN, VMAX)
    vel[0] = VMIN
    return tops, vel


def procedural_2d(nz, nx, h, seed, dtype=np.float32):
    """2D layered model: 12-20 layers with velocity increasing in depth
    (+-300 m/s jitter), one sinusoidal fold shared by all interfaces
    (amplitude 50-300 m, wavelength 2-8 km) and 2-5 planar normal faults
    (dip 50-70 deg, throw 20-200 m; hanging wall pulled down-dip, nearest
    sample). Clipped to [1500, 5000] m/s."""
    rng = np.random.default_rng(seed)
    nl = int(rng.integers(12, 21))
    depth = nz * h
    tops, lv = _layer_table(rng, nl, depth)
    amp = rng.uniform(50.0, 300.0)
    lam = rng.uniform(2000.0, 8000.0)
    phi = rng.uniform(0.0, 2.0 * math.pi)
    x = np.arange(nx) * h
    z = np.arange(nz) * h
    zz = z[:, None] - amp * np.sin(2.0 * math.pi * x / lam + phi)[None, :]
    v = lv[np.searchsorted(tops, zz, side="right")]
    nf = int(rng.integers(2, 6))
    for _ in range(nf):
        dip = math.radians(rng.uniform(50.0, 70.0))
        throw = rng.uniform(20.0, 200.0)
        x0 = rng.uniform(0.1, 0.9) * nx * h
        sgn = 1.0 if rng.uniform() < 0.5 else -1.0
        hang = (x[None, :] - x0) * sgn - z[:, None] / math.tan(dip) > 0
        dx = throw * math.cos(dip) * sgn
        dz = throw * math.sin(dip)
        iz = np.clip(np.rint((z[:, None] - dz) / h), 0, nz - 1).astype(np.int64)
        ix = np.clip(np.rint((x[None, :] - dx) / h), 0, nx - 1).astype(np.int64)
        iz, ix = np.broadcast_arrays(iz, ix)
        v = np.where(hang, v[iz, ix], v)
    return np.clip(v, VMIN, VMAX).astype(dtype)


def procedural_3d(nz, ny, nx, h, seed, dtype=np.float32):
    """3D layered model with a 2D fold A sin(kx x + px) sin(ky y + py) and three
    planar normal faults of random strike; built slab by slab in depth."""
    rng = np.random.default_rng(seed)
    nl = int(rng.integers(12, 21))
    depth = nz * h
    tops, lv = _layer_table(rng, nl, depth)
    amp = rng.uniform(50.0, 300.0)
    kx = 2.0 * math.pi / rng.uniform(2000.0, 8000.0)
    ky = 2.0 * math.pi / rng.uniform(2000.0, 8000.0)
    px, py = rng.uniform(0.0, 2.0 * math.pi, 2)
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    fold = amp * np.sin(kx * x[None, :] + px) * np.sin(ky * y[:, None] + py)  # (ny, nx)
    faults = []
    for _ in range(3):
        dip = math.radians(rng.uniform(50.0, 70.0))
        strike = rng.uniform(0.0, 2.0 * math.pi)
        throw = rng.uniform(20.0, 200.0)
        x0 = rng.uniform(0.2, 0.8) * nx * h
        y0 = rng.uniform(0.2, 0.8) * ny * h
        faults.append((dip, strike, throw, x0, y0))

    def layered(zv, yv, xv):
        """Unfaulted velocity at arbitrary (z, y, x) sample points (metres)."""
        iy = np.clip(np.rint(yv / h), 0, ny - 1).astype(np.int64)
        ix = np.clip(np.rint(xv / h), 0, nx - 1).astype(np.int64)
        return lv[np.searchsorted(tops, zv - fold[iy, ix], side="right")]

    v = np.empty((nz, ny, nx), dtype=dtype)
    Y, X = np.meshgrid(y, x, indexing="ij")

    def slab(z0):
        zv = np.full_like(X, z0 * h)
        yv, xv = Y.copy(), X.copy()
        hd, t = np.empty_like(X), np.empty_like(X)
        hang = np.empty(X.shape, dtype=bool)
        # faults are applied in order: each pulls its hanging wall down-dip
        # (in-place form of hd = (x - fx) cos s + (y - fy) sin s; hanging
        # where hd - z / tan(dip) > 0, moved by the throw along the dip)
        for dip, strike, throw, fx, fy in reversed(faults):
            np.subtract(xv, fx, out=hd)
            hd *= math.cos(strike)
            np.subtract(yv, fy, out=t)
            t *= math.sin(strike)
            hd += t
            np.divide(zv, math.tan(dip), out=t)
            hd -= t
            np.greater(hd, 0, out=hang)
            np.subtract(zv, throw * math.sin(dip), out=zv, where=hang)
            np.subtract(xv, throw * math.cos(dip) * math.cos(strike), out=xv, where=hang)
            np.subtract(yv, throw * math.cos(dip) * math.sin(strike), out=yv, where=hang)
        zs = np.clip(np.rint(zv / h), 0, nz - 1) * h
        v[z0] = layered(zs, yv, xv)

    # slabs are independent: large volumes build them on a thread pool (numpy
    # releases the interpreter lock in these array operations)
    if nz * ny * nx >= (1 << 24):
        import os
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max(1, min(32, os.cpu_count() or 1))) as ex:
            list(ex.map(slab, range(nz)))
    else:
        for z0 in range(nz):
            slab(z0)
    return np.clip(v, VMIN, VMAX, out=v)


def smooth(v, sigma_cells):
    """Separable Gaussian smoothing (truncated at 4 sigma, reflected edges);
    used to make a starting model from a true model."""
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(v.astype(np.float64), sigma=sigma_cells, mode="reflect",
                           truncate=4.0).astype(v.dtype)


def line(x0, x1, n, z):
    """n points from x0 to x1 (inclusive) at depth z, 2D order (x, z)."""
    xs = np.linspace(x0, x1, n)
    return np.stack([xs, np.full(n, float(z))], axis=1)


def grid_xy(x0, x1, nxr, y0, y1, nyr, z):
    """A regular (nyr x nxr) receiver grid at depth z, 3D order (x, y, z)."""
    xs = np.linspace(x0, x1, nxr)
    ys = np.linspace(y0, y1, nyr)
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(X.size, float(z))], axis=1)


def _problem(**kw):
    base = dict(ndim=2, ny=1, bc="cpml", nb=[0] * 6, free_surface=0, R=1e-3,
                f_ref=10.0, snap_every=0, snap_begin=0, snap_end=0)
    base.update(kw)
    return base


def config_c1(nt=1000, bc="cpml", nb=20):
    """Two-layer 201 x 201 model, h = 10 m, absorbing layer on all four sides,
    Ricker f0 = 10 Hz (t0 = 0.12 s) at (1000 m, 20 m), 201 receivers at 20 m."""
    p = _problem(name="c1", nz=201, nx=201, h=10.0, dt=1e-3, nt=nt, bc=bc,
                 nb=[nb, nb, 0, 0, nb, nb], free_surface=0, f_ref=10.0)
    p["vel"] = two_layer(201, 201, 10.0, 1000.0, 1500.0, 2500.0)
    p["wavelet"] = ricker(10.0, 0.12, 1e-3, nt)
    p["src"] = np.array([[1000.0, 20.0]])
    p["rec"] = line(0.0, 2000.0, 201, 20.0)
    return p


def config_c2(nt=8000, seed=2000, snaps=True):
    """Field-scale slice: 619 x 1000 cells at 10 m, 50-cell CPML on the left,
    right and bottom, free surface on top; Ricker 10 Hz (t0 = 1/f0) at the
    surface centre (5000 m, 10 m); 1000 receivers every 10 m at 10 m depth;
    dt = 1 ms; FP32 snapshots every 10 steps for the first 5 s."""
    p = _problem(name="c2", nz=619, nx=1000, h=10.0, dt=1e-3, nt=nt, bc="cpml",
                 nb=[0, 50, 0, 0, 50, 50], free_surface=1, f_ref=10.0)
    if snaps:
        p.update(snap_every=10, snap_begin=0, snap_end=min(5000, nt))
    p["vel"] = procedural_2d(619, 1000, 10.0, seed)
    p["wavelet"] = ricker(10.0, 0.1, 1e-3, nt)
    p["src"] = np.array([[5000.0, 10.0]])
    p["rec"] = line(0.0, 9990.0, 1000, 10.0)
    return p


def config_c3(nt=4000, nslices=16):
    """Batched forward: one C2-type slice with 64 shots every 150 m
    (x = 275 ... 9725 m) plus ``nslices`` seeded slices of uneven size
    (depth 300-619, width 400-1000 cells) with 8 shots each; receivers every
    10 m at 10 m depth; 50-cell CPML, free surface; 4 s records."""
    slices = []
    main = config_c2(nt=nt, seed=3000, snaps=False)
    main["name"] = "c3_main"
    main["src"] = np.stack([275.0 + 150.0 * np.arange(64), np.full(64, 10.0)], axis=1)
    slices.append(main)
    rng = np.random.default_rng(3000)
    for j in range(1, nslices + 1):
        nz = int(rng.integers(300, 620))
        nx = int(rng.integers(400, 1001))
        p = _problem(name="c3_%d" % j, nz=nz, nx=nx, h=10.0, dt=1e-3, nt=nt, bc="cpml",
                     nb=[0, 50, 0, 0, 50, 50], free_surface=1, f_ref=10.0)
        p["vel"] = procedural_2d(nz, nx, 10.0, 3000 + j)
        p["wavelet"] = ricker(10.0, 0.1, 1e-3, nt)
        xs = np.rint((np.arange(8) + 0.5) * nx / 8.0) * 10.0
        p["src"] = np.stack([xs, np.full(8, 10.0)], axis=1)
        p["rec"] = line(0.0, (nx - 1) * 10.0, nx, 10.0)
        slices.append(p)
    return slices


def config_c4(nt=4000, nshots=16, bc="cpml", nb=20):
    """FWI gradient on the config-1 slice geometry (201 x 201, 20-cell CPML on
    every side, no free surface) filled by the procedural model (seed 4000);
    starting model = true model smoothed with a 250 m (25-cell) Gaussian; 16
    shots equally spaced at 20 m depth; 201 receivers at 20 m depth; Ricker
    10 Hz."""
    p = _problem(name="c4", nz=201, nx=201, h=10.0, dt=1e-3, nt=nt, bc=bc,
                 nb=[nb, nb, 0, 0, nb, nb], free_surface=0, f_ref=10.0)
    p["vel_true"] = procedural_2d(201, 201, 10.0, 4000)
    p["vel"] = smooth(p["vel_true"], 25.0)
    p["wavelet"] = ricker(10.0, 0.12, 1e-3, nt)
    xs = np.rint((np.arange(nshots) + 0.5) * 201 / nshots) * 10.0
    p["src"] = np.stack([xs, np.full(nshots, 20.0)], axis=1)
    p["rec"] = line(0.0, 2000.0, 201, 20.0)
    return p


def config_c5(nt=2500, dt=8e-4, n=(619, 1000, 1000), nb=30, seed=5000, nrec_side=201):
    """3D field-scale volume: (nz, ny, nx) = (619, 1000, 1000) at 10 m, 30-cell
    CPML on x, y and bottom, free surface; Ricker 8 Hz at the surface centre;
    a 201 x 201 receiver grid spanning the interior (spacing 49.95 m) at 10 m.
    dt = 0.8 ms and nt = 2500 keep the 2 s record under the 3D CFL bound."""
    nz, ny, nx = n
    p = _problem(name="c5", ndim=3, nz=nz, ny=ny, nx=nx, h=10.0, dt=dt, nt=nt, bc="cpml",
                 nb=[0, nb, nb, nb, nb, nb], free_surface=1, f_ref=8.0)
    p["vel"] = procedural_3d(nz, ny, nx, 10.0, seed)
    p["wavelet"] = ricker(8.0, 1.0 / 8.0, dt, nt)
    p["src"] = np.array([[(nx // 2) * 10.0, (ny // 2) * 10.0, 10.0]])
    p["rec"] = grid_xy(0.0, (nx - 1) * 10.0, nrec_side, 0.0, (ny - 1) * 10.0, nrec_side, 10.0)
    return p


# the paper's five frequency bands: (f_lo, f_hi, f0) in Hz (Tab. bands, Sec. "Source Wavelet")
BANDS = [(3.0, 6.0, 4.50), (3.0, 8.5, 5.75), (3.0, 12.0, 7.50), (3.0, 17.5, 10.25), (3.0, 25.0, 14.00)]


def config_c6(kind="gather", band=0, nt=None, seed=6000, nshots=64):
    """The paper's production runs on one 619 x 1000 slice at 10 m with a
    60-cell sponge on the left, right and bottom and a free top, dt = 1 ms,
    band-passed Ricker source (parameters in ``band``: the wavelet itself is
    made by the library's band-pass kernel). kind="gather": 8 s (nt = 8001),
    ``nshots`` sources uniformly spaced over [1.1 km, x_max - 1.1 km] at 10 m
    depth, 1000 receivers uniformly spaced over the full width at 10 m (saved
    every 14 steps = the rows 0, 14, ... of the full gather). kind="wavefield":
    5 s (nt = 5001), one source at a seeded uniform position in the same
    interval, snapshots every 14 steps (358), no receivers."""
    nz, nx, h = 619, 1000, 10.0
    if nt is None:
        nt = 8001 if kind == "gather" else 5001
    p = _problem(name="c6" + kind[0], nz=nz, nx=nx, h=h, dt=1e-3, nt=nt, bc="sponge",
                 nb=[0, 60, 0, 0, 60, 60], free_surface=1, f_ref=10.0)
    p["vel"] = procedural_2d(nz, nx, h, seed)
    p["band"] = BANDS[band]
    xmax = (nx - 1) * h
    if kind == "gather":
        p["src"] = np.stack([np.linspace(1100.0, xmax - 1100.0, nshots), np.full(nshots, 10.0)], axis=1)
        p["rec"] = line(0.0, xmax, 1000, 10.0)
        p["save_every"] = 14
    else:
        rng = np.random.default_rng(seed)
        p["src"] = np.array([[float(rng.uniform(1100.0, xmax - 1100.0)), 10.0]])
        p["rec"] = np.zeros((0, 2))
        p.update(snap_every=14, snap_begin=0, snap_end=nt)
    return p
