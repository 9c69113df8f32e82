"""Resident 2D forward path (one cooperative launch for the whole time loop,
wavefield kept on chip): parity with the FP64 oracle (relative L2 <= 1e-4,
the FP32 tolerance of the other forward tests), agreement with the per-step
kernel path (the same per-cell arithmetic up to the order of a few additions
and, in sponge cells, multiplication by precomputed 1/(1+a) weights instead
of a division: <= 1e-5 relative), path selection, and a bounded
wait that runs out reporting SIM_ERR_TIMEOUT instead of hanging. With the
resident path off, 2D FP32 forwards take the per-step kernel or the row march
(path 4), whichever the autotuner timed faster; GSIM_MARCH=0 forces the
per-step kernel."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PATH_STEP, PATH_RESIDENT, PATH_MARCH = 1, 2, 4


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


class env:
    """Set environment variables for the duration of a with-block."""

    def __init__(self, **kv):
        self.kv = kv

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kv}
        os.environ.update({k: str(v) for k, v in self.kv.items()})

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def forward(pkg, cfg, vel, w, srcs, rec, snaps=False, resident=True, max_shots=None):
    with env(GSIM_RESIDENT=1 if resident else 0, GSIM_MARCH=0):
        sim = pkg.Simulator(cfg, vel, max_shots=max_shots or len(srcs), max_rec=len(rec))
        out = sim.forward(w, srcs, rec, gather=True, snapshots=snaps)
        sim.sync()
        info = pkg.sim_get_info(sim.handle)
        res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
        sim.close()
    return res, info


def check_case(pkg, cfg, vel, w, srcs, rec, snaps=False):
    res, info = forward(pkg, cfg, vel, w, srcs, rec, snaps)
    assert info.last_path == PATH_RESIDENT
    step, info1 = forward(pkg, cfg, vel, w, srcs, rec, snaps, resident=False)
    assert info1.last_path == PATH_STEP
    v64, w64 = np.asarray(vel, np.float64), np.asarray(w, np.float64)
    for k, s in enumerate(srcs):
        ref = oracle.forward(cfg, v64, w64, src=s, rec=rec, snaps=snaps)
        assert rel(res["gather"][k], ref["gather"]) <= 1e-4, k
        assert rel(res["gather"][k], step["gather"][k]) <= 1e-5, k
        if snaps:
            assert rel(res["snaps"][k], ref["snaps"]) <= 1e-4, k
            assert rel(res["snaps"][k], step["snaps"][k]) <= 1e-5, k
    return res, info


@pytest.mark.parametrize("bc", ["cpml", "sponge", "none"])
def test_c1_every_boundary(pkg, bc):
    c = synth.config_c1(nt=700, bc=bc)
    check_case(pkg, c, c["vel"], c["wavelet"], c["src"], c["rec"])


@pytest.mark.parametrize("bc", ["cpml", "sponge"])
def test_ragged_free_surface_snapshots_multishot(pkg, bc):
    # extents that are not subdomain multiples (last row of subdomains holds
    # fewer rows than the exchanged border), free surface, off-grid points,
    # FP32 snapshots, three shots resident at once
    nz, nx = 53, 301
    cfg = dict(ndim=2, nz=nz, ny=1, nx=nx, h=10.0, dt=1e-3, nt=450, bc=bc, nb=[0, 14, 0, 0, 11, 9],
               free_surface=1, R=1e-3, f_ref=12.0, snap_every=9, snap_begin=4, snap_end=440)
    vel = synth.procedural_2d(nz, nx, 10.0, 303)
    w = synth.ricker(12.0, 0.08, 1e-3, 450)
    srcs = np.array([[123.4, 5.0], [1600.0, 27.3], [2990.0, 60.0]])
    rec = np.stack([np.linspace(0.0, 3000.0, 97), np.linspace(3.0, 520.0, 97)], axis=1)
    check_case(pkg, cfg, vel, w, srcs, rec, snaps=True)


def test_c2_field_slice(pkg):
    # the 619 x 1000 slice with its 50-cell CPML and free surface; 1500 steps
    c = synth.config_c2(nt=1500)
    c.update(snap_every=50, snap_end=1500)
    res, info = check_case(pkg, c, c["vel"], c["wavelet"], c["src"], c["rec"], snaps=True)
    assert 8 <= info.last_rows <= 48


def test_repeat_calls_start_from_rest(pkg):
    c = synth.config_c1(nt=300)
    with env(GSIM_RESIDENT=1):
        sim = pkg.Simulator(c, c["vel"], max_rec=len(c["rec"]))
        a = sim.forward(c["wavelet"], c["src"], c["rec"])["gather"].clone()
        b = sim.forward(c["wavelet"], c["src"], c["rec"])["gather"]
        sim.sync()
        assert pkg.sim_get_info(sim.handle).last_path == PATH_RESIDENT
        sim.close()
    assert torch.equal(a, b)


def test_falls_back_when_it_does_not_fit(pkg):
    # FP16 snapshots need a grid-wide maximum per step: a per-step path (the row march)
    c = synth.config_c1(nt=200)
    c.update(snap_every=10, snap_end=200)
    sim = pkg.Simulator(c, c["vel"], max_rec=len(c["rec"]), snap_fp16=True)
    sim.forward(c["wavelet"], c["src"], c["rec"], snapshots=True)
    sim.sync()
    assert pkg.sim_get_info(sim.handle).last_path in (PATH_STEP, PATH_MARCH)
    sim.close()
    # 32 shots of the 619 x 1000 slice need more subdomains than the GPU holds
    c = synth.config_c2(nt=20, snaps=False)
    srcs = np.stack([500.0 + 280.0 * np.arange(32), np.full(32, 10.0)], axis=1)
    sim = pkg.Simulator(c, c["vel"], max_shots=32, max_rec=len(c["rec"]))
    sim.forward(c["wavelet"], srcs, c["rec"])
    sim.sync()
    assert pkg.sim_get_info(sim.handle).last_path in (PATH_STEP, PATH_MARCH)
    sim.close()


def test_timeout_is_reported(pkg):
    c = synth.config_c1(nt=200)
    with env(GSIM_RESIDENT=1, GSIM_SPIN_LIMIT=0):  # every wait on a neighbour gives up at once
        sim = pkg.Simulator(c, c["vel"], max_rec=len(c["rec"]))
        with pytest.raises(pkg.SimError) as e:
            sim.forward(c["wavelet"], c["src"], c["rec"])
            sim.sync()
        assert e.value.code == pkg.abi.SIM_ERR_TIMEOUT
        sim.close()
    # the context is still usable
    res, info = forward(pkg, c, c["vel"], c["wavelet"], c["src"], c["rec"])
    assert info.last_path == PATH_RESIDENT and np.isfinite(res["gather"]).all()


@pytest.mark.parametrize("nt", [1, 2, 3])
def test_shortest_runs(pkg, nt):
    # the first steps: p^0 = 0 everywhere, the source enters at n = 0
    c = synth.config_c1(nt=nt)
    c["wavelet"] = np.ones(nt, np.float32)
    res, info = forward(pkg, c, c["vel"], c["wavelet"], c["src"], c["rec"])
    assert info.last_path == PATH_RESIDENT
    ref = oracle.forward(c, c["vel"].astype(np.float64), c["wavelet"].astype(np.float64), src=c["src"][0],
                         rec=c["rec"])["gather"]
    step, _ = forward(pkg, c, c["vel"], c["wavelet"], c["src"], c["rec"], resident=False)
    assert np.allclose(res["gather"][0], ref, rtol=1e-5, atol=1e-7 * max(1.0, np.abs(ref).max()))
    assert np.allclose(res["gather"][0], step["gather"][0], rtol=1e-6, atol=0)
