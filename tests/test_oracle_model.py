"""Pins of the model-builder oracle (oracle/model.py) against facts that do
not depend on its own code: the interpolator reproduces samples at integer
positions and constants everywhere, and band-limited signals at fractional
shifts; Squish with an integer displacement is an exact shift with the fill
rule beyond the grid; Fault with zero slip is the identity, leaves voxels
outside its die-off region unchanged, moves the fault centre by the chord
2 R sin(s / 2R) of the slip rotation, and moves the two walls in opposite
directions; Deposit reduces to closed forms without texture and taper and
pushes the model below down by the slab thickness."""
import numpy as np
import pytest

from oracle import model


def test_sinc_weights_sum_to_one_and_are_exact_at_integers():
    s = np.array([0.0, 3.0, 7.25, -2.5, 11.9])
    i0, w = model.sinc_taps(s)
    assert np.allclose(w.sum(axis=-1), 1.0, atol=1e-14)
    i0, w = model.sinc_taps(np.array([5.0]))
    k = 5 - i0[0]
    assert abs(w[0, k] - 1.0) < 1e-14 and np.abs(np.delete(w[0], k)).max() < 1e-14
    # symmetric kernel: position 2.5 weighs taps 2 and 3 alike
    i0, w = model.sinc_taps(np.array([2.5]))
    assert np.allclose(w[0], w[0][::-1], atol=1e-15)


def test_sample_reproduces_samples_constants_and_bandlimited_shifts():
    rng = np.random.default_rng(1)
    v = rng.standard_normal((20, 3, 17))
    z, y, x = model.grid(v.shape)
    assert np.allclose(model.sample(v, z, y, x), v, atol=1e-12)
    c = np.full((9, 1, 9), 1875.0)
    zz, yy, xx = np.meshgrid(np.linspace(-2, 10, 7), [0.3], np.linspace(-1, 9.5, 5), indexing="ij")
    assert np.allclose(model.sample(c, zz, yy, xx), 1875.0, atol=1e-9)
    # cosines of 10 and 40 cells per wavelength at fractional positions, away
    # from the edges: an 8-tap windowed sinc is good to a few 1e-3 there
    nz = 120
    zc = np.arange(nz, dtype=np.float64)
    for cells, tol in ((10, 4e-3), (40, 3e-3)):
        f = 1.0 / cells
        col = np.cos(2 * np.pi * f * zc)[:, None, None]
        for frac in (0.37, 0.5, 0.81):
            s = np.arange(20, 100) + frac
            got = model.sample(col, s[:, None, None], np.zeros((80, 1, 1)), np.zeros((80, 1, 1)))[:, 0, 0]
            assert np.abs(got - np.cos(2 * np.pi * f * s)).max() < tol, (cells, frac)


def test_squish_integer_shift_is_exact_with_fill():
    rng = np.random.default_rng(2)
    v = rng.uniform(1500, 4500, (30, 2, 11))
    lab = rng.integers(0, 9, v.shape)
    dz = np.zeros((2, 11))
    dz[:, :5] = 3.0
    dz[:, 5:] = -2.0
    out, ol = model.squish(v, lab, dz, 1234.0, -1)
    assert np.allclose(out[:27, :, :5], v[3:, :, :5], atol=1e-9)
    assert np.all(out[27:, :, :5] == 1234.0) and np.all(ol[27:, :, :5] == -1)
    assert np.allclose(out[2:, :, 5:], v[:-2, :, 5:], atol=1e-9)
    assert np.all(out[:2, :, 5:] == 1234.0)
    assert np.array_equal(ol[:27, :, :5], lab[3:, :, :5])
    same, sl = model.squish(v, lab, np.zeros((2, 11)), 0.0, 0)
    assert np.allclose(same, v, atol=1e-9) and np.array_equal(sl, lab)


FAULT = dict(cz=20.0, cy=0.0, cx=25.0, azimuth=np.pi / 2, dip=np.deg2rad(60.0), radius=400.0, slip=6.0,
             direction=1, d_die=15.0, d_perp=50.0, theta_die=np.deg2rad(20.0))


def test_fault_identity_cases():
    rng = np.random.default_rng(3)
    v = rng.uniform(1500, 4500, (48, 1, 56))
    lab = rng.integers(0, 9, v.shape)
    out, ol = model.fault(v, lab, dict(FAULT, slip=0.0), 0.0, -1)
    assert np.allclose(out, v, atol=1e-9) and np.array_equal(ol, lab)
    # along the radius through the centre (r = R +- k exactly), voxels k >=
    # d_die cells from the fault surface do not move, nearer ones do
    sz, sy, sx = model.fault_source(v.shape, **FAULT)
    th = FAULT["dip"]
    nz_, nx_ = np.sin(th), np.cos(th)  # radial direction at the centre, (z, x)
    for k, moves in ((16.0, False), (-16.0, False), (4.0, True), (-4.0, True)):
        zq, xq = FAULT["cz"] + k * nz_, FAULT["cx"] + k * nx_
        src = model.fault_source((1, 1, 1), **dict(FAULT, cz=FAULT["cz"] - zq, cx=FAULT["cx"] - xq))
        d = np.hypot(src[0][0, 0, 0], src[2][0, 0, 0])
        assert (d > 1e-6) == moves, (k, d)


def test_fault_centre_moves_by_the_chord_and_walls_move_oppositely():
    p = FAULT
    sz, sy, sx = model.fault_source((48, 1, 56), **p)
    iz, ix = int(p["cz"]), int(p["cx"])
    d = np.hypot(sz[iz, 0, ix] - iz, sx[iz, 0, ix] - ix)
    chord = 2 * p["radius"] * np.sin(p["slip"] / p["radius"] / 2)
    assert abs(d - chord) < 1e-9
    # along the fault plane near the centre the two walls move apart: the
    # footwall (r >= R) and hanging wall (r < R) displacements point oppositely
    n = np.array([np.sin(p["dip"]), np.cos(p["dip"])])  # (z, x) direction away from the axis at the centre

    def disp(k):  # displacement of the point k cells along n from the centre
        zq, xq = p["cz"] + k * n[0], p["cx"] + k * n[1]
        src = model.fault_source((1, 1, 1), **dict(p, cz=p["cz"] - zq, cx=p["cx"] - xq))
        return np.array([src[0][0, 0, 0], src[2][0, 0, 0]])

    da, db = disp(3.0), disp(-3.0)
    assert np.dot(da, db) < 0
    # each moves by the chord of its own radius at the taper cos(pi/2 * 3/d_die)
    w = np.cos(0.5 * np.pi * 3.0 / p["d_die"])
    half = 0.5 * w * p["slip"] / p["radius"]
    assert abs(np.linalg.norm(da) - 2 * (p["radius"] + 3.0) * np.sin(half)) < 1e-9
    assert abs(np.linalg.norm(db) - 2 * (p["radius"] - 3.0) * np.sin(half)) < 1e-9


def test_deposit_closed_forms():
    nz, ny, nx = 40, 2, 6
    rng = np.random.default_rng(4)
    v = rng.uniform(2000, 4000, (nz, ny, nx))
    lab = rng.integers(0, 5, v.shape)
    t = 12
    eta = rng.standard_normal((30, ny, nx))
    # one velocity for every bed, no texture: v0 + beta z in the slab
    bounds = np.array([np.full((ny, nx), 4.3), np.full((ny, nx), 8.1)])
    out, ol = model.deposit(v, lab, t, bounds, [1800.0] * 3, 7.5, 0.0, 0.2, 0.2, eta, [0, 3, 5], 10)
    z = np.arange(t)[:, None, None]
    assert np.allclose(out[:t], 1800.0 + 7.5 * z, atol=1e-9)
    assert np.allclose(out[t:], v[:nz - t], atol=0) and np.array_equal(ol[t:], lab[:nz - t])
    beds = np.where(z < 4.3, 0, np.where(z < 8.1, 1, 2)) + 0 * out[:t]
    assert np.array_equal(ol[:t], 10 + beds.astype(int))
    # bed velocities without taper: v_l + beta z, and the texture read at
    # z - floor(S_l) + o_l
    vb = [1700.0, 2100.0, 1950.0]
    out, _ = model.deposit(v, lab, t, bounds, vb, 5.0, 0.0, 0.0, 0.0, eta, [0, 3, 5], 0)
    expect = np.choose(beds.astype(int), [np.full_like(out[:t], q) for q in vb]) + 5.0 * z
    assert np.allclose(out[:t], expect, atol=1e-9)
    out, _ = model.deposit(v, lab, t, bounds, vb, 0.0, 2.0, 0.0, 0.0, eta, [0, 3, 5], 0)
    zz = np.arange(t)
    for k, zi in enumerate(zz):
        ell = 0 if zi < 4.3 else (1 if zi < 8.1 else 2)
        start = [0, 4, 8][ell]
        zt = min(max(zi - start + [0, 3, 5][ell], 0), 29)
        assert np.allclose(out[zi], vb[ell] + 2.0 * eta[zt], atol=1e-9)
