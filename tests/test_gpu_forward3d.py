"""3D forward parity: the z-marching FP32 path against the FP64 oracle through
the C ABI (relative L2 <= 1e-4 for gathers and snapshots)."""
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
    return float(np.linalg.norm(a - b) / nb) if nb else float(np.linalg.norm(a))


def case3d(bc, fs, nb=6, n=(30, 26, 34), nt=160, snaps=False, top=None):
    nz, ny, nx = n
    top = (0 if fs else nb) if top is None else top
    cfg = dict(ndim=3, nz=nz, ny=ny, nx=nx, h=10.0, dt=8e-4, nt=nt, bc=bc,
               nb=[top, nb, nb, nb, nb, nb], free_surface=fs, R=1e-3, f_ref=15.0)
    if snaps:
        cfg.update(snap_every=9, snap_begin=2, snap_end=nt)
    vel = synth.procedural_3d(nz, ny, nx, 10.0, 17)
    w = synth.ricker(15.0, 0.06, 8e-4, nt)
    return cfg, vel, w


def run(pkg, cfg, vel, w, srcs, rec, snaps=False, snap_fp16=False):
    sim = pkg.Simulator(cfg, vel, max_shots=len(srcs), max_rec=len(rec), snap_fp16=snap_fp16)
    out = sim.forward(w, srcs, rec, gather=True, snapshots=snaps)
    sim.sync()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    sim.close()
    refs = [oracle.forward(cfg, np.asarray(vel, np.float64), np.asarray(w, np.float64), src=s, rec=rec,
                           snaps=snaps) for s in srcs]
    return res, refs


@pytest.mark.parametrize("bc,fs", [("cpml", 1), ("cpml", 0), ("sponge", 1), ("none", 0)])
def test_small_3d_parity(pkg, bc, fs):
    cfg, vel, w = case3d(bc, fs, snaps=True)
    srcs = np.array([[163.0, 124.0, 42.0], [97.5, 203.3, 15.0]])
    rng = np.random.default_rng(3)
    rec = np.stack([rng.uniform(0, 330, 40), rng.uniform(0, 250, 40), rng.uniform(0, 290, 40)], axis=1)
    rec[:5, 2] = 10.0
    res, refs = run(pkg, cfg, vel, w, srcs, rec, snaps=True)
    for k in range(2):
        assert rel(res["gather"][k], refs[k]["gather"]) <= 1e-4, k
        assert rel(res["snaps"][k], refs[k]["snaps"]) <= 1e-4, k


@pytest.mark.parametrize("n,fs", [((6, 5, 9), 0), ((3, 18, 20), 1)])
def test_3d_cpml_strip_layouts(pkg, n, fs):
    # z and y strips whose widened ranges meet (one range per marching
    # column), and a bottom z strip whose widened range reaches the free
    # surface (the mirrored z-derivative of the two-kernel path)
    cfg, vel, w = case3d("cpml", fs, n=n, nt=120)
    nz, ny, nx = n
    srcs = np.array([[0.55 * (nx - 1) * 10.0, 0.4 * (ny - 1) * 10.0, 0.5 * (nz - 1) * 10.0]])
    rng = np.random.default_rng(5)
    rec = np.stack([rng.uniform(0, (nx - 1) * 10.0, 20), rng.uniform(0, (ny - 1) * 10.0, 20),
                    rng.uniform(0, (nz - 1) * 10.0, 20)], axis=1)
    res, refs = run(pkg, cfg, vel, w, srcs, rec)
    assert rel(res["gather"][0], refs[0]["gather"]) <= 1e-4


def test_3d_fp16_snapshots(pkg):
    cfg, vel, w = case3d("sponge", 1, snaps=True)
    res, refs = run(pkg, cfg, vel, w, [[160.0, 120.0, 40.0]], [[20.0, 20.0, 20.0]], snaps=True, snap_fp16=True)
    q = res["snaps"][0].astype(np.float64)
    s = res["snap_scale"][0].astype(np.float64)
    ref = refs[0]["snaps"]
    for k in range(len(s)):
        m = np.abs(ref[k]).max()
        if m == 0:
            continue
        assert np.log2(s[k]) == np.round(np.log2(s[k]))
        assert np.abs(q[k] * s[k] - ref[k]).max() <= 2.0 ** -11 * m * 1.01 + 1e-5 * m


def test_c5_type_volume_reduced(pkg):
    # the 3D field-scale configuration (30-cell CPML on x, y and bottom, free
    # surface, 8 Hz source at the surface centre, receiver grid at 10 m) on a
    # reduced 62 x 100 x 100 volume and 300 steps of 0.8 ms
    c = synth.config_c5(nt=300, n=(62, 100, 100), nb=20, nrec_side=21)
    res, refs = run(pkg, c, c["vel"], c["wavelet"], c["src"], c["rec"])
    assert rel(res["gather"][0], refs[0]["gather"]) <= 1e-4
