"""Pins of the FP64 oracle against what the mathematics and the paper fix.

Each test would fail under a plausible mistake in the oracle: a wrong stencil
weight or order (polynomial exactness, analytic Green's functions), a wrong
source normalisation (analytic amplitudes), a wrong time discretisation
(convergence order, energy), a wrong free-surface sign (image source), a wrong
interface rule (reflection coefficient), a non-symmetric operator
(reciprocity, transposes), a wrong absorbing layer (truncation test) or a wrong
adjoint (brute-force Jacobian, complex step, finite differences, dot tests).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import bruteforce as bf


def ricker_fn(f0, t0):
    return lambda t: (1 - 2 * (math.pi * f0 * (t - t0)) ** 2) * np.exp(-(math.pi * f0 * (t - t0)) ** 2)


def green2d(w, r, v, t):
    """p(r, t) = (1/2pi) int_0^{acosh(vt/r)} w(t - (r/v) cosh u) du: the 2D
    free-space Green's function of (1/v^2) p_tt - lap p = delta convolved with w."""
    out = np.zeros(len(t))
    for i, ti in enumerate(t):
        if v * ti <= r:
            continue
        u = np.linspace(0.0, np.arccosh(v * ti / r), 4001)
        out[i] = np.trapezoid(w(ti - (r / v) * np.cosh(u)), u) / (2 * math.pi)
    return out


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def prob(nz, nx, h=10.0, dt=1e-3, nt=100, bc="none", nb=(0, 0, 0, 0, 0, 0), fs=0, **kw):
    d = dict(ndim=2, nz=nz, ny=1, nx=nx, h=h, dt=dt, nt=nt, bc=bc, nb=list(nb), free_surface=fs)
    d.update(kw)
    return d


# ---------------------------------------------------------------- stencil


@pytest.mark.parametrize("axis", ["x", "z"])
def test_laplacian_exact_on_polynomials_up_to_degree_9(axis):
    # 8th-order central weights (App. E.3, M = 4) differentiate x^k exactly for k <= 9
    n = 41
    cfg = prob(n, n, h=1.0)
    s = np.arange(n) - 20.0
    for k in range(11):
        f1 = s ** k
        f = np.tile(f1, (n, 1)) if axis == "x" else np.tile(f1[:, None], (1, n))
        out = oracle.laplacian(cfg, f)
        exact1 = k * (k - 1) * s ** (k - 2) if k >= 2 else np.zeros(n)
        core = slice(5, n - 5)
        got = out[20, core] if axis == "x" else out[core, 20]
        want = exact1[core]
        err = np.max(np.abs(got - want)) / max(1.0, np.max(np.abs(want)))
        if k <= 9:
            assert err < 1e-9, (k, err)
        else:
            # degree 10 is the first one it misses: at s = 0 the exact value is 0
            # and the stencil returns 2 sum_m w_m m^10 = -1151.43...
            at0 = out[20, 20]
            assert abs(at0 - 2 * (8 / 5 - 1024 / 5 + 8 * 59049 / 315 - 1048576 / 560)) < 1e-6, at0


def test_fd_weights_symbol_and_cfl_limits():
    # the symbol of the 1D stencil peaks at theta = pi with 6.5016 (Courant limit 2/sqrt(d*6.5016))
    n = 64
    cfg = prob(20, n, h=1.0)
    f = np.tile(np.cos(np.pi * np.arange(n))[None, :], (20, 1))   # constant along z
    out = oracle.laplacian(cfg, f)
    sym = -out[10, 20] / f[10, 20]
    assert abs(sym - 6.501587301587302) < 1e-12
    assert abs(2 / math.sqrt(2 * sym) - 0.5546) < 1e-4
    assert abs(2 / math.sqrt(3 * sym) - 0.4529) < 1e-4


@pytest.mark.parametrize("fs", [0, 1])
def test_laplacian_transpose_and_dense_matrix(fs):
    rng = np.random.default_rng(3)
    nz, nx = 13, 11
    cfg = prob(nz, nx, h=7.0, fs=fs)
    x = rng.standard_normal((nz, nx))
    y = rng.standard_normal((nz, nx))
    Lx = oracle.laplacian(cfg, x)
    LTy = oracle.laplacian(cfg, y, transpose=True)
    assert abs(np.vdot(Lx, y) - np.vdot(x, LTy)) < 1e-12 * np.linalg.norm(Lx) * np.linalg.norm(y)
    L = bf.laplacian_matrix((nz, nx), 7.0, free_surface=bool(fs))
    assert np.allclose(L @ x.ravel(), Lx.ravel(), rtol=0, atol=1e-13 * np.abs(Lx).max())
    if fs:
        # on fields with the surface row held at zero the operator is symmetric
        x[0] = 0
        y[0] = 0
        a = np.vdot(oracle.laplacian(cfg, x)[1:], y[1:])
        b = np.vdot(x[1:], oracle.laplacian(cfg, y)[1:])
        assert abs(a - b) < 1e-12 * abs(a)


def test_laplacian_transpose_3d():
    rng = np.random.default_rng(4)
    cfg = dict(ndim=3, nz=7, ny=6, nx=5, h=5.0, dt=1e-3, nt=1, bc="none", nb=[0] * 6, free_surface=1)
    x = rng.standard_normal((7, 6, 5))
    y = rng.standard_normal((7, 6, 5))
    assert abs(np.vdot(oracle.laplacian(cfg, x), y) - np.vdot(x, oracle.laplacian(cfg, y, transpose=True))) < 1e-10
    L = bf.laplacian_matrix((7, 6, 5), 5.0, free_surface=True)
    assert np.allclose(L @ x.ravel(), oracle.laplacian(cfg, x).ravel(), atol=1e-12)


# ---------------------------------------------------------------- invariants


@pytest.mark.parametrize("fs", [0, 1])
def test_energy_conserved_without_absorption(fs):
    # E^{n+1/2} = sum m ((p^{n+1}-p^n)/dt)^2 - sum p^{n+1} (L p^n) is invariant
    rng = np.random.default_rng(5)
    nz, nx, h, dt = 60, 70, 10.0, 1e-3
    vel = rng.uniform(1500.0, 3000.0, (nz, nx))
    zz, xx = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    p0 = np.exp(-((zz - 25.0) ** 2 + (xx - 30.0) ** 2) / 20.0)
    if fs:
        p0[0] = 0
    m = 1.0 / vel ** 2

    def energy(cfg, pp, pc):
        return np.sum(m * ((pc - pp) / dt) ** 2) - np.sum(pc * oracle.laplacian(cfg, pp))

    c1 = prob(nz, nx, h, dt, nt=1, fs=fs)
    r1 = oracle.forward(c1, vel, init_prev=p0, init_cur=p0, final=True)
    e1 = energy(c1, r1["final_prev"], r1["final_cur"])
    cN = prob(nz, nx, h, dt, nt=3000, fs=fs)
    rN = oracle.forward(cN, vel, init_prev=p0, init_cur=p0, final=True)
    eN = energy(cN, rN["final_prev"], rN["final_cur"])
    assert np.max(np.abs(rN["final_cur"])) > 1e-3  # the field did not vanish
    assert abs(eN - e1) < 1e-11 * abs(e1), (e1, eN)


@pytest.mark.parametrize("ndim,stable,unstable", [(2, 0.55, 0.56), (3, 0.45, 0.46)])
def test_von_neumann_limit(ndim, stable, unstable):
    rng = np.random.default_rng(6)
    n = 40 if ndim == 2 else 20
    shape = (n, n) if ndim == 2 else (n, n, n)
    p0 = rng.standard_normal(shape)
    out = {}
    for cour in (stable, unstable):
        cfg = dict(ndim=ndim, nz=n, ny=n if ndim == 3 else 1, nx=n, h=10.0, dt=cour * 10.0 / 2000.0,
                   nt=800, bc="none", nb=[0] * 6)
        r = oracle.forward(cfg, np.full(shape, 2000.0), init_prev=p0, init_cur=p0, final=True)
        out[cour] = np.nanmax(np.abs(r["final_cur"]))
    assert out[stable] < 50 * np.abs(p0).max()
    assert not (out[unstable] < 1e6 * np.abs(p0).max())


# ---------------------------------------------------------------- closed forms


def test_green_2d_analytic_and_second_order_in_time():
    v, h, n = 2000.0, 10.0, 161
    W = ricker_fn(10.0, 0.1)
    rec = np.array([[900.0, 800.0], [1000.0, 800.0], [1100.0, 800.0]])
    errs = {}
    for dt in (1e-3, 5e-4):
        nt = int(round(0.4 / dt))
        cfg = prob(n, n, h, dt, nt)
        g = oracle.forward(cfg, np.full((n, n), v), synth.ricker(10.0, 0.1, dt, nt, np.float64),
                           src=(800.0, 800.0), rec=rec)["gather"]
        t = np.arange(nt) * dt
        errs[dt] = [rel(g[:, k], green2d(W, r, v, t)) for k, r in enumerate([100.0, 200.0, 300.0])]
    assert max(errs[1e-3]) < 5e-3, errs
    for a, b in zip(errs[1e-3], errs[5e-4]):
        assert 3.3 < a / b < 4.7, errs  # error ~ dt^2


def test_green_3d_analytic():
    v, h, n, dt, nt = 2000.0, 10.0, 81, 1e-3, 300
    cfg = dict(ndim=3, nz=n, ny=n, nx=n, h=h, dt=dt, nt=nt, bc="none", nb=[0] * 6)
    rec = np.array([[500.0, 400.0, 400.0], [550.0, 400.0, 400.0], [400.0, 600.0, 400.0]])
    g = oracle.forward(cfg, np.full((n, n, n), v), synth.ricker(10.0, 0.1, dt, nt, np.float64),
                       src=(400.0, 400.0, 400.0), rec=rec)["gather"]
    t = np.arange(nt) * dt
    W = ricker_fn(10.0, 0.1)
    for k, r in enumerate([100.0, 150.0, 200.0]):
        assert rel(g[:, k], W(t - r / v) / (4 * math.pi * r)) < 5e-3


def test_free_surface_equals_image_source():
    # p = G(x - xs) - G(x - xs*) for p = 0 on z = 0 (Eq. free_surface)
    v, h, dt, nt, nz, nx = 2000.0, 10.0, 5e-4, 800, 100, 161
    cfg = prob(nz, nx, h, dt, nt, fs=1)
    rec = np.array([[900.0, 30.0], [1000.0, 30.0], [1100.0, 30.0]])
    g = oracle.forward(cfg, np.full((nz, nx), v), synth.ricker(10.0, 0.1, dt, nt, np.float64),
                       src=(800.0, 50.0), rec=rec)["gather"]
    t = np.arange(nt) * dt
    W = ricker_fn(10.0, 0.1)
    for k, dx in enumerate([100.0, 200.0, 300.0]):
        want = green2d(W, math.hypot(dx, 20.0), v, t) - green2d(W, math.hypot(dx, 80.0), v, t)
        assert rel(g[:, k], want) < 3e-3


def test_flat_interface_reflection_coefficient():
    # pre-critical plane-wave R(theta) = (v2 cos t1 - v1 cos t2)/(v2 cos t1 + v1 cos t2);
    # the discrete interface (z < z_if -> v1, z >= z_if -> v2) sits on the cell face
    v1, v2, h, dt, nt, nz, nx = 1500.0, 2500.0, 10.0, 5e-4, 2200, 251, 301
    vel = synth.two_layer(nz, nx, h, 1500.0, v1, v2, np.float64)
    cfg = prob(nz, nx, h, dt, nt)
    offs = [0.0, 100.0, 200.0, 300.0]
    rec = np.array([[1500.0 + o, 1000.0] for o in offs])
    g = oracle.forward(cfg, vel, synth.ricker(10.0, 0.1, dt, nt, np.float64), src=(1500.0, 1000.0), rec=rec)["gather"]
    t = np.arange(nt) * dt
    W = ricker_fn(10.0, 0.1)
    win = (t > 0.55) & (t < 1.0)
    half = 1495.0 - 1000.0   # source to the cell face between rows 149 and 150
    for k, o in enumerate(offs):
        direct = green2d(W, o, v1, t) if o > 0 else np.zeros(nt)
        image = green2d(W, math.hypot(o, 2 * half), v1, t)
        th1 = math.atan2(o, 2 * half)
        s2 = v2 / v1 * math.sin(th1)
        c2 = math.sqrt(1 - s2 * s2)
        R = (v2 * math.cos(th1) - v1 * c2) / (v2 * math.cos(th1) + v1 * c2)
        refl = (g[:, k] - direct)[win]
        fit = np.dot(refl, image[win]) / np.dot(image[win], image[win])
        assert abs(fit / R - 1) < 0.03, (o, fit, R)
        assert abs(np.linalg.norm(refl) / np.linalg.norm(image[win]) / R - 1) < 0.05
    assert abs(0.25 - (v2 - v1) / (v2 + v1)) < 1e-15


def test_reciprocity_with_sponge_free_surface_and_off_grid_points():
    nz, nx = 50, 70
    vel = synth.procedural_2d(nz, nx, 10.0, 11).astype(np.float64)
    cfg = prob(nz, nx, 10.0, 1e-3, 500, bc="sponge", nb=(0, 10, 0, 0, 10, 10), fs=1)
    w = synth.ricker(12.0, 0.08, 1e-3, 500, np.float64)
    A = (155.3, 23.7)
    B = (512.0, 41.2)
    gab = oracle.forward(cfg, vel, w, src=A, rec=[B])["gather"][:, 0]
    gba = oracle.forward(cfg, vel, w, src=B, rec=[A])["gather"][:, 0]
    assert np.abs(gab).max() > 0
    assert rel(gab, gba) < 1e-12


def _truncation_case(bc, nb, v):
    h, dt, nt, n, E = 10.0, 1e-3, 700, 101, 80
    offs = [(0, -300), (300, 0), (-200, 200), (450, 450), (-450, -450)]
    w = synth.ricker(10.0, 0.1, dt, nt, np.float64)
    cfg = prob(n, n, h, dt, nt, bc=bc, nb=(nb, nb, 0, 0, nb, nb), f_ref=10.0)
    g = oracle.forward(cfg, np.full((n, n), v), w, src=(500.0, 500.0),
                       rec=[(500.0 + a, 500.0 + b) for a, b in offs])["gather"]
    N = n + 2 * E
    ref = oracle.forward(prob(N, N, h, dt, nt), np.full((N, N), v), w, src=(500.0 + E * h, 500.0 + E * h),
                         rec=[(500.0 + a + E * h, 500.0 + b + E * h) for a, b in offs])["gather"]
    return rel(g, ref)


def test_absorbing_layers_against_large_domain_reference():
    # the large domain is wide enough that no edge reflection returns within nt,
    # so the difference is the absorbing layer's own error
    for v in (1500.0, 2000.0):
        sp20 = _truncation_case("sponge", 20, v)
        sp60 = _truncation_case("sponge", 60, v)
        pml20 = _truncation_case("cpml", 20, v)
        assert sp60 < sp20 / 4
        assert pml20 < 2e-3
        assert pml20 < sp20 / 100
    assert _truncation_case("sponge", 60, 1500.0) < 1e-2


_OFFS3 = [(0, 0, 150), (0, 0, -150), (0, 150, 0), (0, -150, 0), (150, 0, 0), (-150, 0, 0),
          (140, 140, 140), (-140, 140, -140)]


def _truncation_3d(v, cases):
    """Per-receiver relative L2 error of 3D runs with absorbing layers on all
    six faces against a large-domain reference (Dirichlet, no absorption) whose
    edges are far enough that no reflection returns within nt. Receivers face
    each of the six faces and two corners (where the per-axis layers overlap)."""
    h, dt, nt, n, E, c = 10.0, 1e-3, 300, 41, 35, 200.0
    w = synth.ricker(15.0, 1 / 15.0, dt, nt, np.float64)
    rec = [(c + a, c + b, c + d) for a, b, d in _OFFS3]
    N = n + 2 * E
    big = dict(ndim=3, nz=N, ny=N, nx=N, h=h, dt=dt, nt=nt, bc="none", nb=[0] * 6)
    ref = oracle.forward(big, np.full((N, N, N), v), w, src=(c + E * h,) * 3,
                         rec=[(x + E * h, y + E * h, z + E * h) for x, y, z in rec])["gather"]
    out = {}
    for bc, nb in cases:
        cfg = dict(ndim=3, nz=n, ny=n, nx=n, h=h, dt=dt, nt=nt, bc=bc, nb=[nb] * 6, f_ref=15.0)
        g = oracle.forward(cfg, np.full((n, n, n), v), w, src=(c, c, c), rec=rec)["gather"]
        out[(bc, nb)] = np.array([rel(g[:, k], ref[:, k]) for k in range(len(rec))])
    return out


def test_absorbing_layers_3d_against_large_domain_reference():
    # the 3D layers on every face (z, y and x, edges and corners): the CPML must
    # leave a small error at every receiver and beat the sponge of equal width;
    # a wider layer must absorb better; the cube is symmetric, so the six face
    # receivers see the same error, whatever axis they face
    for v in (1500.0, 2500.0):
        e = _truncation_3d(v, [("sponge", 10), ("sponge", 20), ("cpml", 5), ("cpml", 10)])
        assert e[("cpml", 10)].max() < 1e-3
        assert np.all(e[("cpml", 10)] < e[("sponge", 10)] / 100)
        assert np.all(e[("cpml", 10)] < e[("cpml", 5)] / 3)
        assert np.all(e[("sponge", 20)] < e[("sponge", 10)] / 2.5)
        for k in e.values():
            assert np.ptp(k[:6]) <= 1e-6 * k[:6].max()
    assert _truncation_3d(1500.0, [("cpml", 10)])[("cpml", 10)].max() < 1e-5


@pytest.mark.parametrize("bc", ["cpml", "sponge"])
def test_3d_axis_permutation_with_unequal_layers(bc):
    # swapping two axes of the whole problem (model, positions and the widths
    # of the absorbing faces) permutes the solution: the y axis (profiles, face
    # widths, strides, corner sums) is treated exactly as x and z
    nz, ny, nx, nt = 22, 26, 30, 200
    vel = synth.procedural_3d(nz, ny, nx, 10.0, 31).astype(np.float64)
    nb = [5, 7, 6, 9, 8, 4]
    cfg = dict(ndim=3, nz=nz, ny=ny, nx=nx, h=10.0, dt=8e-4, nt=nt, bc=bc, nb=nb, f_ref=12.0)
    w = synth.ricker(12.0, 0.09, 8e-4, nt, np.float64)
    src = (123.4, 151.7, 88.2)
    rec = np.array([[10.0, 20.0, 30.0], [280.0, 240.0, 200.0], [5.0, 250.0, 111.0], [150.5, 3.3, 207.0]])
    g = oracle.forward(cfg, vel, w, src=src, rec=rec)["gather"]
    assert np.abs(g).max() > 0
    cxy = dict(cfg, ny=nx, nx=ny, nb=[nb[0], nb[1], nb[4], nb[5], nb[2], nb[3]])
    gxy = oracle.forward(cxy, vel.transpose(0, 2, 1).copy(), w, src=(src[1], src[0], src[2]),
                         rec=rec[:, [1, 0, 2]])["gather"]
    czy = dict(cfg, nz=ny, ny=nz, nb=[nb[2], nb[3], nb[0], nb[1], nb[4], nb[5]])
    gzy = oracle.forward(czy, vel.transpose(1, 0, 2).copy(), w, src=(src[0], src[2], src[1]),
                         rec=rec[:, [0, 2, 1]])["gather"]
    assert rel(gxy, g) < 1e-12
    assert rel(gzy, g) < 1e-12


def test_sponge_profile_constants():
    # Eq. cerjan_damp: eta = (c_damp/h)[rho - sin(2 pi rho)/(2 pi)], c_damp = 1.5 ln(1/R)/n_bl
    nb = 60
    cfg = prob(10, 200, 10.0, 1e-3, 1, bc="sponge", nb=(0, 0, 0, 0, nb, nb), R=1e-3)
    v = 2000.0
    co = oracle.coefficients(cfg, np.full((10, 200), v))
    assert co["a"].shape == (10, 200 + 2 * nb)
    eta = co["a"] / (v * v * 1e-3 / 2.0)
    cdamp = 1.5 * math.log(1000.0) / 60.0
    assert abs(cdamp - 0.17269388197455343) < 1e-15
    assert abs(eta[5, 0] - 1e-3 * cdamp / 10.0) < 1e-15           # rho = 1 at the outer cell
    assert abs(eta[5, 319] - 1e-3 * cdamp / 10.0) < 1e-15
    assert abs(eta[5, 30] - 1e-3 * cdamp / 10.0 * 0.5) < 1e-15     # rho = 1/2
    assert np.all(eta[:, nb:nb + 200] == 0)
    assert np.all(np.diff(eta[5, :nb]) < 0) and np.all(np.diff(eta[5, nb + 200:]) > 0)
    assert np.allclose(co["c"], v * v * 1e-6)


# ---------------------------------------------------------------- brute force


def _tiny(fs, bc="sponge"):
    rng = np.random.default_rng(7 + fs)
    nz, nx, nb = 8, 9, 3
    cfg = prob(nz, nx, 10.0, 1e-3, 30, bc=bc, nb=(0 if fs else nb, nb, 0, 0, nb, nb), fs=fs)
    vel = rng.uniform(1500.0, 3000.0, (nz, nx))
    w = rng.standard_normal(30)
    return cfg, vel, w


@pytest.mark.parametrize("fs", [0, 1])
def test_forward_matches_dense_brute_force(fs):
    cfg, vel, w = _tiny(fs)
    src = (30.0, 20.0)
    rec = np.array([[0.0, 10.0], [50.0, 70.0], [80.0, 40.0]])
    g = oracle.forward(cfg, vel, w, src=src, rec=rec)["gather"]
    nb = cfg["nb"]
    dims = (nb[0] + cfg["nz"] + nb[1], nb[4] + cfg["nx"] + nb[5])
    co = oracle.coefficients(cfg, vel)
    F = bf.replication_matrix((cfg["nz"], cfg["nx"]), nb, 2)
    vpad = F @ vel.ravel()
    eta = co["a"].ravel() / (vpad ** 2 * cfg["dt"] / 2)
    L = bf.laplacian_matrix(dims, 10.0, bool(fs))

    def cell(p):
        return (int(p[1] / 10) + nb[0]) * dims[1] + int(p[0] / 10) + nb[4]
    rows = list(range(dims[1])) if fs else []
    gb, J = bf.simulate(L, co["c"], eta, vpad, cfg["dt"], w, cell(src), 1.0 / 100.0,
                        [cell(p) for p in rec], rows, tangent=True)
    assert rel(g, gb) < 1e-12
    # gradient of J = 1/2 ||g - d||^2 by forward mode vs the oracle's reverse mode
    d = np.random.default_rng(9).standard_normal(g.shape) * np.abs(g).max()
    res = (gb - d).reshape(-1)
    grad_fwd = F.T @ (J.reshape(-1, J.shape[-1]).T @ res)
    out = oracle.gradient(cfg, vel, w, src, rec, d)
    assert rel(out["grad"].ravel(), grad_fwd) < 1e-10
    assert abs(out["misfit"] - 0.5 * np.sum(res ** 2)) < 1e-12 * out["misfit"]


# ---------------------------------------------------------------- adjoint checks


def _c4_small(bc="sponge", fs=0, nt=400):
    nz, nx = 40, 50
    vel_true = synth.procedural_2d(nz, nx, 10.0, 4001).astype(np.float64)
    vel0 = synth.smooth(vel_true, 5.0)
    cfg = prob(nz, nx, 10.0, 1e-3, nt, bc=bc, nb=(0 if fs else 10, 10, 0, 0, 10, 10), fs=fs)
    w = synth.ricker(15.0, 0.07, 1e-3, nt, np.float64)
    src = (245.0, 20.0)
    rec = synth.line(0.0, 490.0, 50, 20.0 if not fs else 10.0)
    d = oracle.forward(cfg, vel_true, w, src=src, rec=rec)["gather"]
    return cfg, vel0, w, src, rec, d


@pytest.mark.parametrize("fs", [0, 1])
def test_gradient_matches_complex_step(fs):
    cfg, vel, w, src, rec, d = _c4_small(fs=fs, nt=250)
    out = oracle.gradient(cfg, vel, w, src, rec, d)
    rng = np.random.default_rng(10)
    cells = [(0, 0), (cfg["nz"] - 1, cfg["nx"] - 1)] + [tuple(rng.integers(0, s) for s in vel.shape) for _ in range(3)]
    eps = 1e-30
    for (iz, ix) in cells:
        vc = vel.astype(np.complex128)
        vc[iz, ix] += 1j * eps * vel[iz, ix]
        J = oracle.gradient(cfg, vc, w, src, rec, d, complex_=True)["misfit"]
        cs = J.imag / (eps * vel[iz, ix])
        assert abs(cs - out["grad"][iz, ix]) <= 1e-9 * abs(out["grad"]).max(), (iz, ix, cs, out["grad"][iz, ix])


@pytest.mark.parametrize("fs", [0, 1])
def test_cpml_gradient_matches_complex_step(fs):
    # the exact adjoint of the CPML recursions (psi, zeta multipliers); the
    # CPML coefficients are constants of the map (cpml_vmax fixed)
    cfg, vel, w, src, rec, d = _c4_small(bc="cpml", fs=fs, nt=250)
    cfg["cpml_vmax"] = float(vel.max())
    out = oracle.gradient(cfg, vel, w, src, rec, d)
    rng = np.random.default_rng(11)
    cells = [(0, 0), (cfg["nz"] - 1, cfg["nx"] - 1), (cfg["nz"] - 1, 3), (2, cfg["nx"] - 2)] + \
        [tuple(rng.integers(0, s) for s in vel.shape) for _ in range(3)]
    eps = 1e-30
    for (iz, ix) in cells:
        vc = vel.astype(np.complex128)
        vc[iz, ix] += 1j * eps * vel[iz, ix]
        J = oracle.gradient(cfg, vc, w, src, rec, d, complex_=True)["misfit"]
        cs = J.imag / (eps * vel[iz, ix])
        assert abs(cs - out["grad"][iz, ix]) <= 1e-9 * abs(out["grad"]).max(), (iz, ix, cs, out["grad"][iz, ix])


@pytest.mark.parametrize("fs", [0, 1])
def test_cpml_dot_product_source_to_gather(fs):
    cfg, vel, _, src, rec, _ = _c4_small(bc="cpml", fs=fs, nt=200)
    rng = np.random.default_rng(13)
    x = rng.standard_normal(cfg["nt"])
    y = rng.standard_normal((cfg["nt"], len(rec)))
    Ax = oracle.forward(cfg, vel, x, src=src, rec=rec)["gather"]
    ATy = oracle.gradient(cfg, vel, np.zeros(cfg["nt"]), src, rec, -y)["grad_wavelet"]
    lhs, rhs = np.vdot(Ax, y), np.vdot(x, ATy)
    assert abs(lhs - rhs) / (np.linalg.norm(Ax) * np.linalg.norm(y)) < 1e-12


def test_gradient_matches_central_differences():
    cfg, vel, w, src, rec, d = _c4_small(nt=300)
    g = oracle.gradient(cfg, vel, w, src, rec, d)["grad"]
    rng = np.random.default_rng(4000)
    for _ in range(10):
        iz, ix = rng.integers(0, vel.shape[0]), rng.integers(0, vel.shape[1])
        e = 1e-4 * vel[iz, ix]
        vp, vm = vel.copy(), vel.copy()
        vp[iz, ix] += e
        vm[iz, ix] -= e
        Jp = oracle.gradient(cfg, vp, w, src, rec, d)["misfit"]
        Jm = oracle.gradient(cfg, vm, w, src, rec, d)["misfit"]
        fd = (Jp - Jm) / (2 * e)
        assert abs(fd - g[iz, ix]) <= 1e-6 * abs(g).max() + 1e-6 * abs(g[iz, ix])


@pytest.mark.parametrize("fs", [0, 1])
def test_dot_product_source_to_gather(fs):
    # A: w -> g is linear; A^T y is the wavelet gradient of 1/2||A w - d||^2 at w = 0, d = -y
    cfg, vel, _, src, rec, _ = _c4_small(fs=fs, nt=200)
    rng = np.random.default_rng(12)
    x = rng.standard_normal(cfg["nt"])
    y = rng.standard_normal((cfg["nt"], len(rec)))
    Ax = oracle.forward(cfg, vel, x, src=src, rec=rec)["gather"]
    ATy = oracle.gradient(cfg, vel, np.zeros(cfg["nt"]), src, rec, -y)["grad_wavelet"]
    lhs, rhs = np.vdot(Ax, y), np.vdot(x, ATy)
    assert abs(lhs - rhs) / (np.linalg.norm(Ax) * np.linalg.norm(y)) < 1e-12


def test_dot_product_born_jacobian():
    # J dv by complex step of the forward map; J^T dd by the adjoint-state gradient
    cfg, vel, w, src, rec, _ = _c4_small(nt=200)
    rng = np.random.default_rng(13)
    dv = rng.standard_normal(vel.shape)
    dd = rng.standard_normal((cfg["nt"], len(rec)))
    eps = 1e-20
    gc = oracle.forward(cfg, vel + 1j * eps * dv, w, src=src, rec=rec, complex_=True)["gather"]
    Jdv = gc.imag / eps
    g0 = gc.real
    JTdd = oracle.gradient(cfg, vel, w, src, rec, g0 - dd)["grad"]
    lhs, rhs = np.vdot(Jdv, dd), np.vdot(dv, JTdd)
    assert abs(lhs - rhs) / (np.linalg.norm(Jdv) * np.linalg.norm(dd)) < 1e-10


# ---------------------------------------------------------------- source wavelet (Sec. "Source Wavelet")

def test_wavelet_ricker_spectrum_is_the_closed_form():
    # |FT| of the Ricker pulse is proportional to f^2 exp(-f^2 / f0^2): peak at f0
    from oracle import wavelet as W
    dt, nt = 1e-3, 8192
    for f0 in (4.5, 10.25):
        r = W.ricker(f0, nt * dt / 2, dt, nt)
        spec = np.abs(np.fft.rfft(r))
        f = np.fft.rfftfreq(nt, dt)
        model = f ** 2 * np.exp(-(f / f0) ** 2)
        assert np.max(np.abs(spec / spec.max() - model / model.max())) < 1e-6
        assert abs(f[np.argmax(spec)] - f0) <= f[1]


def test_wavelet_norm_and_zero_phase():
    from oracle import wavelet as W
    dt, nt = 1e-3, 8001
    for lo, hi, f0 in W.BANDS:
        w = W.bandpass_ricker(f0, lo, hi, dt, nt)
        assert abs(np.linalg.norm(w) - np.sqrt((hi - lo) / 24.0)) < 1e-12
    # a pulse centred in the record comes out symmetric about its centre
    y = W.bandpass(W.ricker(7.5, 4.0, dt, nt), 3.0, 12.0, dt)
    c = 4000
    assert np.max(np.abs(y[c:c + 3000] - y[c:c - 3000:-1])) <= 1e-9 * np.abs(y).max()


def test_wavelet_filter_gain_is_the_squared_analog_butterworth():
    # forward-backward gain of a pure tone = |H_a(j W)|^2 of the analog band-pass
    # prototype of order N at the prewarped frequency W = 2 fs tan(pi f / fs)
    from oracle import wavelet as W
    dt, nt, N, lo, hi = 1e-3, 40000, 4, 3.0, 12.0
    fs = 1.0 / dt
    wl, wh = 2 * fs * np.tan(np.pi * lo / fs), 2 * fs * np.tan(np.pi * hi / fs)
    w0, bw = np.sqrt(wl * wh), wh - wl
    t = np.arange(nt) * dt
    mid = slice(nt // 4, 3 * nt // 4)
    for f in (1.5, 3.0, 5.0, 12.0, 20.0):
        y = W.bandpass(np.sin(2 * np.pi * f * t), lo, hi, dt, N)
        basis = np.stack([np.sin(2 * np.pi * f * t[mid]), np.cos(2 * np.pi * f * t[mid])], 1)
        ab, *_ = np.linalg.lstsq(basis, y[mid], rcond=None)
        gain = np.hypot(*ab)
        wf = 2 * fs * np.tan(np.pi * f / fs)
        expect = 1.0 / (1.0 + ((wf ** 2 - w0 ** 2) / (wf * bw)) ** (2 * N))
        assert abs(gain - expect) <= 1e-6 + 1e-6 * expect, (f, gain, expect)


def _small_3d(bc, fs, nt=60):
    nz, ny, nx, nb = 9, 8, 10, 3
    cfg = dict(ndim=3, nz=nz, ny=ny, nx=nx, h=10.0, dt=8e-4, nt=nt, bc=bc,
               nb=[0 if fs else nb, nb, nb, nb, nb, nb], free_surface=fs, R=1e-3, f_ref=15.0)
    vel = synth.procedural_3d(nz, ny, nx, 10.0, 23).astype(np.float64)
    if bc == "cpml":
        cfg["cpml_vmax"] = float(vel.max())  # the CPML coefficients are constants of the map
    src = (45.0, 35.0, 20.0)
    rec = np.array([[10.0 * i, 10.0 * j, 60.0] for i in range(1, 9, 3) for j in range(1, 7, 3)])
    return cfg, vel, src, rec


@pytest.mark.parametrize("bc", ["sponge", "cpml"])
@pytest.mark.parametrize("fs", [0, 1])
def test_gradient_3d_matches_complex_step(fs, bc):
    # the same adjoint-state gradient on a 3D grid (2 receiver planes off the
    # source); with CPML the transposed psi / zeta recursions of all three axes
    cfg, vel, src, rec = _small_3d(bc, fs)
    w = synth.ricker(25.0, 0.03, 8e-4, 60, np.float64)
    d = 0.5 * oracle.forward(cfg, vel * 1.03, w, src=src, rec=rec)["gather"]
    out = oracle.gradient(cfg, vel, w, src, rec, d)
    rng = np.random.default_rng(31)
    eps = 1e-30
    edge = [(0, 0, 0), tuple(n - 1 for n in vel.shape)]  # cells whose velocity fills absorbing cells
    for iz, iy, ix in edge + [tuple(int(rng.integers(0, s)) for s in vel.shape) for _ in range(4)]:
        vc = vel.astype(np.complex128)
        vc[iz, iy, ix] += 1j * eps * vel[iz, iy, ix]
        J = oracle.gradient(cfg, vc, w, src, rec, d, complex_=True)["misfit"]
        cs = J.imag / (eps * vel[iz, iy, ix])
        assert abs(cs - out["grad"][iz, iy, ix]) <= 1e-9 * abs(out["grad"]).max(), (iz, iy, ix)


@pytest.mark.parametrize("fs", [0, 1])
def test_cpml_dot_product_source_to_gather_3d(fs):
    # w -> g is linear; its transpose is the wavelet gradient at w = 0, d = -y
    cfg, vel, src, rec = _small_3d("cpml", fs, nt=80)
    rng = np.random.default_rng(14 + fs)
    x = rng.standard_normal(cfg["nt"])
    y = rng.standard_normal((cfg["nt"], len(rec)))
    Ax = oracle.forward(cfg, vel, x, src=src, rec=rec)["gather"]
    ATy = oracle.gradient(cfg, vel, np.zeros(cfg["nt"]), src, rec, -y)["grad_wavelet"]
    lhs, rhs = np.vdot(Ax, y), np.vdot(x, ATy)
    assert abs(lhs - rhs) / (np.linalg.norm(Ax) * np.linalg.norm(y)) < 1e-12
