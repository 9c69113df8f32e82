"""Velocity-model builder warps of the paper's model generator (App. "Model
builder modules"): the pull-sample steps of Squish (Alg. squish), Fault
(Alg. fault) and a simplified Deposit (Alg. deposit), written plainly in FP64
numpy on (nz, ny, nx) grids (ny = 1 for a 2D slice).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import this module; the library never does.

Random draws of the paper's modules (fractal-noise displacements, bed
thicknesses and velocities, noise-perturbed bed boundaries, texture fields)
are inputs here, as they are to the GPU kernels.

Readings where the paper is silent (listed with the others in the design
notes):
  M1 "sinc interpolation" = Lanczos-windowed sinc with 8 taps per axis
     (window sinc(x/4) on |x| < 4), weights normalised to sum 1; taps beyond
     the grid take the edge value. Integer positions reproduce the samples.
  M2 fill: a voxel whose pulled depth lies outside [0, nz) takes the fill
     velocity and fill label (Alg. fault states this; Squish uses the same
     rule); depths down to -1e-6 count as 0, so that rounding in the
     coordinate arithmetic does not fill the top row of an unmoved voxel.
     Labels are pulled by nearest neighbour (round half to even), indices
     clamped to the grid.
  M3 Fault frame, (z, y, x) with z down: dip-azimuth direction
     e_d = (0, cos a, sin a), strike direction e_s = (0, -sin a, cos a),
     e_z = (1, 0, 0); cylinder centre c~ = c - (R sin t) e_z - (R cos t) e_d;
     slip as rotation by s / R radians (= s / (2 pi R) x 360 degrees).
  M4 Deposit (simplified): the slab of thickness t is laid on top of the
     model (rows z < t; the model below is pushed down by t rows, labels
     likewise); bed index = number of bed boundaries H_i(y, x) below z (the
     searchsorted count); the texture is read at depth z - floor(S_l) + o_l
     (S_l the bed's start depth: the deepest boundary above z, 0 in the
     first bed; o_l its drawn offset), clamped to the field; a zero taper fraction means no taper on that side; the final
     conformance to an underlying topography is not applied.
"""
import numpy as np

TAPS = 8  # sinc taps per axis


def lanczos(x):
    """Lanczos-windowed sinc, window half-width 4 (reading M1)."""
    x = np.asarray(x, np.float64)
    return np.where(np.abs(x) < 4.0, np.sinc(x) * np.sinc(x / 4.0), 0.0)


def sinc_taps(s):
    """First tap index and normalised weights of the 8 taps around position s."""
    s = np.asarray(s, np.float64)
    i0 = np.floor(s).astype(np.int64) - 3
    j = i0[..., None] + np.arange(TAPS)
    w = lanczos(s[..., None] - j)
    return i0, w / w.sum(axis=-1, keepdims=True)


def sample(v, sz, sy, sx):
    """Separable sinc interpolation of v (nz, ny, nx) at fractional positions
    (sz, sy, sx) (arrays of one shape), edge values beyond the grid."""
    nz, ny, nx = v.shape
    out = np.zeros(np.shape(sz))
    iz, wz = sinc_taps(sz)
    iy, wy = sinc_taps(sy)
    ix, wx = sinc_taps(sx)
    for a in range(TAPS):
        za = np.clip(iz + a, 0, nz - 1)
        for b in range(TAPS):
            yb = np.clip(iy + b, 0, ny - 1)
            wab = wz[..., a] * wy[..., b]
            for c in range(TAPS):
                xc = np.clip(ix + c, 0, nx - 1)
                out += wab * wx[..., c] * v[za, yb, xc]
    return out


def nearest(lab, sz, sy, sx):
    nz, ny, nx = lab.shape
    iz = np.clip(np.rint(sz).astype(np.int64), 0, nz - 1)
    iy = np.clip(np.rint(sy).astype(np.int64), 0, ny - 1)
    ix = np.clip(np.rint(sx).astype(np.int64), 0, nx - 1)
    return lab[iz, iy, ix]


def _pull(v, lab, sz, sy, sx, fill, fill_label):
    """Pull-sample v (sinc) and lab (nearest) at the source positions; the
    fill rule of reading M2."""
    nz = v.shape[0]
    out_v = sample(v, sz, sy, sx)
    out_l = nearest(lab, sz, sy, sx)
    bad = (sz < -1e-6) | (sz >= nz)
    out_v[bad] = fill
    out_l[bad] = fill_label
    return out_v, out_l


def grid(shape):
    nz, ny, nx = shape
    return np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                       np.arange(nx, dtype=np.float64), indexing="ij")


def squish(v, lab, dz, fill, fill_label):
    """Alg. squish: pull-sample every column at z + dz(y, x) (dz in cells,
    a drawn fractal-noise field passed in)."""
    v = np.asarray(v, np.float64)
    z, y, x = grid(v.shape)
    return _pull(v, lab, z + np.asarray(dz, np.float64)[None], y, x, fill, fill_label)


def fault_source(shape, cz, cy, cx, azimuth, dip, radius, slip, direction, d_die, d_perp, theta_die):
    """Alg. fault, per voxel: the source position 2 p - p_fwd of the pull,
    with p_fwd the rotation of p about the cylinder axis by the tapered slip
    angle (frame of reading M3; angles in radians, lengths in cells)."""
    z, y, x = grid(shape)
    ed = np.array([0.0, np.cos(azimuth), np.sin(azimuth)])
    es = np.array([0.0, -np.sin(azimuth), np.cos(azimuth)])
    ez = np.array([1.0, 0.0, 0.0])
    dz_, daz = radius * np.sin(dip), radius * np.cos(dip)
    ct = np.array([cz, cy, cx]) - dz_ * ez - daz * ed
    th0 = np.arctan2(dz_, daz)
    shift = slip / radius
    wz, wy, wx = z - ct[0], y - ct[1], x - ct[2]
    u = wy * ed[1] + wx * ed[2]
    vz = wz
    a_s = wy * es[1] + wx * es[2]
    r = np.hypot(u, vz)
    th = np.arctan2(vz, u)
    rr = np.abs(r - radius) / d_die
    rt = np.abs(th - th0) / theta_die
    rs = np.abs(a_s) / d_perp
    inside = (rr < 1) & (rt < 1) & (rs < 1)
    taper = np.where(inside, np.cos(0.5 * np.pi * rr) * np.cos(0.5 * np.pi * rt) * np.cos(0.5 * np.pi * rs), 0.0)
    chi = np.where(r >= radius, 1.0, -1.0)
    thn = th - chi * direction * taper * shift
    fz = ct[0] + r * np.sin(thn)
    fy = ct[1] + r * np.cos(thn) * ed[1] + a_s * es[1]
    fx = ct[2] + r * np.cos(thn) * ed[2] + a_s * es[2]
    return 2 * z - fz, 2 * y - fy, 2 * x - fx


def fault(v, lab, params, fill, fill_label):
    """Alg. fault: pull-sample v (sinc) and lab (nearest) at the fault's
    source positions; params as fault_source's keyword arguments."""
    v = np.asarray(v, np.float64)
    sz, sy, sx = fault_source(v.shape, **params)
    return _pull(v, lab, sz, sy, sx, fill, fill_label)


def deposit(v, lab, t, bounds, vbed, beta, a_eta, f_top, f_base, eta, offsets, label0):
    """Alg. deposit (simplified, reading M4): lay a slab of t rows with beds
    on top of the model. bounds [nbeds - 1, ny, nx] bed boundary depths in
    the slab (cells, noise already applied), vbed [nbeds] bed velocities,
    beta depth gradient (m/s per cell), a_eta texture amplitude, f_top /
    f_base taper fractions, eta [nzt, ny, nx] texture field, offsets [nbeds]
    texture depth offsets, label0 the first bed's label."""
    v = np.asarray(v, np.float64)
    nz, ny, nx = v.shape
    bounds = np.asarray(bounds, np.float64).reshape(-1, ny, nx)
    vbed = np.asarray(vbed, np.float64)
    eta = np.asarray(eta, np.float64)
    nzt = eta.shape[0]
    vbar = vbed.mean()
    out_v = np.empty_like(v)
    out_l = np.empty_like(lab)
    for z in range(nz):
        if z >= t:
            out_v[z] = v[z - t]
            out_l[z] = lab[z - t]
            continue
        ell = np.sum(bounds < z, axis=0)  # bed of each column
        start = np.max(np.where(bounds < z, bounds, 0.0), axis=0) if len(bounds) else np.zeros((ny, nx))
        top = min(z / (f_top * t), 1.0) if f_top > 0 else 1.0
        base = min((t - z) / (f_base * t), 1.0) if f_base > 0 else 1.0
        tau = top * base
        zt = np.clip(z - np.floor(start).astype(np.int64) + np.asarray(offsets)[ell], 0, nzt - 1)
        tex = eta[zt, np.arange(ny)[:, None], np.arange(nx)[None, :]]
        out_v[z] = (vbar + beta * z) + tau * ((vbed[ell] - vbar) + a_eta * tex)
        out_l[z] = label0 + ell
    return out_v, out_l
