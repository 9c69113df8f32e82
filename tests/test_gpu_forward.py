"""GPU forward parity: libsim's FP32 (and FP64) kernels against the FP64 oracle,
element by element on the same seeded inputs, through the C ABI.

Tolerance: relative L2 <= 1e-4 for FP32 gathers and snapshots (the target the
method's users set for this solver); FP64 handles agree to 1e-10. FP16
snapshots: |half*s - p| <= 2^-11 max|p| + FP32 error."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_30541_gb300 as p
    p.abi.load()
    return p


def rel(a, b):
    a = np.asarray(a, np.float64)
    nb = np.linalg.norm(b)
    if nb == 0:
        return 0.0 if not np.any(a) else float("inf")
    return float(np.linalg.norm(a - b) / nb)


def run_both(pkg, cfg, vel, wavelet, srcs, rec, snaps=False, precision=0, snap_fp16=False):
    sim = pkg.Simulator(cfg, vel, max_shots=len(srcs), max_rec=len(rec), precision=precision,
                        snap_fp16=snap_fp16)
    out = sim.forward(wavelet, srcs, rec, gather=True, snapshots=snaps)
    torch.cuda.synchronize()
    sim.sync()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    sim.close()
    v64 = np.asarray(vel, np.float64)
    w64 = np.asarray(wavelet, np.float64)
    refs = [oracle.forward(cfg, v64, w64, src=s, rec=rec, snaps=snaps) for s in srcs]
    return res, refs


def test_c1_full_cpml(pkg):
    c = synth.config_c1(nt=1000)
    res, refs = run_both(pkg, c, c["vel"], c["wavelet"], c["src"], c["rec"])
    assert rel(res["gather"][0], refs[0]["gather"]) <= 1e-4


@pytest.mark.parametrize("bc", ["sponge", "none"])
def test_c1_other_boundaries(pkg, bc):
    c = synth.config_c1(nt=600, bc=bc)
    res, refs = run_both(pkg, c, c["vel"], c["wavelet"], c["src"], c["rec"])
    assert rel(res["gather"][0], refs[0]["gather"]) <= 1e-4


@pytest.mark.parametrize("bc", ["sponge", "cpml"])
def test_ragged_free_surface_off_grid_multishot(pkg, bc):
    # extents that are not tile multiples, a free surface, off-grid points, 3 shots
    nz, nx = 45, 77
    cfg = dict(ndim=2, nz=nz, ny=1, nx=nx, h=10.0, dt=1e-3, nt=400, bc=bc, nb=[0, 13, 0, 0, 11, 9],
               free_surface=1, R=1e-3, f_ref=12.0, snap_every=7, snap_begin=3, snap_end=390)
    vel = synth.procedural_2d(nz, nx, 10.0, 77)
    w = synth.ricker(12.0, 0.08, 1e-3, 400)
    # the third source sits on the free surface, where p is held at zero: no wavefield at all
    srcs = np.array([[123.4, 5.0], [400.0, 17.3], [760.0, 0.0]])
    rec = np.stack([np.linspace(0.0, 760.0, 53), np.linspace(3.0, 440.0, 53)], axis=1)
    res, refs = run_both(pkg, cfg, vel, w, srcs, rec, snaps=True)
    for k in range(3):
        assert rel(res["gather"][k], refs[k]["gather"]) <= 1e-4, k
        assert rel(res["snaps"][k], refs[k]["snaps"]) <= 1e-4, k
    assert np.abs(refs[0]["gather"]).max() > 0 and not np.any(res["gather"][2])


def test_fp16_snapshots(pkg):
    nz, nx = 60, 90
    cfg = dict(ndim=2, nz=nz, ny=1, nx=nx, h=10.0, dt=1e-3, nt=300, bc="sponge", nb=[10, 10, 0, 0, 10, 10],
               free_surface=0, snap_every=10, snap_begin=0, snap_end=300)
    vel = synth.procedural_2d(nz, nx, 10.0, 5)
    w = synth.ricker(15.0, 0.06, 1e-3, 300)
    res, refs = run_both(pkg, cfg, vel, w, [[450.0, 200.0]], [[100.0, 100.0]], snaps=True, snap_fp16=True)
    q = res["snaps"][0].astype(np.float64)
    s = res["snap_scale"][0].astype(np.float64)
    ref = refs[0]["snaps"]
    for k in range(len(s)):
        assert np.log2(s[k]) == np.round(np.log2(s[k]))   # power of two
        m = np.abs(q[k]).max()
        if np.abs(ref[k]).max() == 0:
            assert s[k] == 1.0 and m == 0
            continue
        assert 2 ** 14 <= m < 2 ** 15 + 1
        err = np.abs(q[k] * s[k] - ref[k]).max()
        assert err <= 2.0 ** -11 * np.abs(ref[k]).max() * 1.01 + 1e-5 * np.abs(ref[k]).max()


def test_fp64_handle_matches_oracle_tightly(pkg):
    c = synth.config_c1(nt=300, bc="sponge")
    res, refs = run_both(pkg, c, c["vel"].astype(np.float64), c["wavelet"].astype(np.float64), c["src"],
                         c["rec"], precision=1)
    assert rel(res["gather"][0], refs[0]["gather"]) <= 1e-10


def test_c2_field_slice_shortened(pkg):
    # the field-scale slice (619 x 1000 + 50-cell CPML, free surface) over 1500 steps
    c = synth.config_c2(nt=1500)
    res, refs = run_both(pkg, c, c["vel"], c["wavelet"], c["src"], c["rec"], snaps=True)
    assert rel(res["gather"][0], refs[0]["gather"]) <= 1e-4
    assert rel(res["snaps"][0], refs[0]["snaps"]) <= 1e-4


def test_host_buffers_through_the_abi(pkg):
    # numpy (host) inputs and outputs: the library stages them itself
    c = synth.config_c1(nt=200)
    d = pkg.make_desc(c, max_shots=1, max_rec=len(c["rec"]))
    h = pkg.sim_create(d, np.ascontiguousarray(c["vel"], np.float32))
    g = np.zeros((1, 200, len(c["rec"])), np.float32)
    pkg.sim_forward(h, 1, np.ascontiguousarray(c["wavelet"]), np.ascontiguousarray(c["src"]), len(c["rec"]),
                    np.ascontiguousarray(c["rec"]), g)
    pkg.sim_destroy(h)
    ref = oracle.forward(c, c["vel"], c["wavelet"], src=c["src"][0], rec=c["rec"])["gather"]
    assert rel(g[0], ref) <= 1e-4


def test_argument_errors(pkg):
    c = synth.config_c1(nt=50)
    sim = pkg.Simulator(c, c["vel"], max_shots=1, max_rec=4)
    with pytest.raises(pkg.SimError) as e:
        sim.forward(c["wavelet"], [[5000.0, 20.0]], c["rec"][:4])   # source outside the interior
    assert e.value.code == pkg.abi.SIM_ERR_ARG
    with pytest.raises(pkg.SimError):
        sim.forward(c["wavelet"], c["src"], c["rec"][:5])           # more receivers than max_rec
    with pytest.raises(pkg.SimError):
        sim.forward(c["wavelet"], np.concatenate([c["src"], c["src"]]), c["rec"][:4])
    sim.close()
    bad = c["vel"].copy()
    bad[3, 3] = np.nan
    with pytest.raises(pkg.SimError):
        pkg.Simulator(c, bad, max_rec=4)
    fast = c["vel"] * 4.0   # 10000 m/s: Courant 1.0
    with pytest.raises(pkg.SimError) as e:
        pkg.Simulator(c, fast, max_rec=4)
    assert e.value.code == pkg.abi.SIM_ERR_CFL


def test_instability_is_reported(pkg):
    # past the CFL bound (checks skipped on purpose) the field blows up; the
    # library reports SIM_ERR_UNSTABLE instead of returning garbage
    c = synth.config_c1(nt=400, bc="none")
    vel = np.full_like(c["vel"], 5700.0)   # Courant 0.57 > 0.5546
    sim = pkg.Simulator(c, vel, max_rec=len(c["rec"]), skip_cfl_check=True)
    with pytest.raises(pkg.SimError) as e:
        sim.forward(c["wavelet"], c["src"], c["rec"])
        sim.sync()
    assert e.value.code == pkg.abi.SIM_ERR_UNSTABLE
    sim.close()
