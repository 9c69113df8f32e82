"""Row-march 2D forward path (each warp streams down the rows of a 128-column
strip; one launch per step): parity with the FP64 oracle (relative L2 <= 1e-4,
the FP32 tolerance of the other forward tests) and agreement with the tiled
per-step kernel (the same per-cell arithmetic up to the order of a few
additions: <= 1e-5 relative) on every boundary, ragged extents, free surface
and absorbing top, off-grid points, several shots, FP32 and FP16 snapshots and
the shortest runs. Both schedules are covered: dynamic (warps take items of a
fixed number of rows from a per-step counter; the default) and static (a
host plan of equal-cost segments). Items and segments are forced down to a
few rows, so they start inside CPML strips, just below the free surface and
in the middle of a list tile; the result must not depend on where they start:
bit for bit where every row takes the same loop (sponge), to FP32 rounding
of a zero addend where a row may take either the CPML loop or the plain one."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PATH_STEP, PATH_MARCH = 1, 4


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_30541_gb300 as p
    p.abi.load()
    return p


class env:
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


def rel(a, b):
    a = np.asarray(a, np.float64)
    nb = np.linalg.norm(b)
    if nb == 0:
        return 0.0 if not np.any(a) else float("inf")
    return float(np.linalg.norm(a - b) / nb)


def run(pkg, cfg, w, srcs, rec, snaps=False, march=True, min_rows=None, item=None, snap_fp16=False):
    kv = dict(GSIM_RESIDENT=0, GSIM_MARCH=1 if march else 0)
    if min_rows is not None:
        kv["GSIM_MARCH_MINROWS"] = min_rows
    if item is not None:
        kv["GSIM_MARCH_ITEM"] = item
    with env(**kv):
        sim = pkg.Simulator(cfg, cfg["vel"], max_shots=len(srcs), max_rec=len(rec), snap_fp16=snap_fp16)
        out = sim.forward(w, srcs, rec, gather=True, snapshots=snaps)
        sim.sync()
        info = pkg.sim_get_info(sim.handle)
        res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
        sim.close()
    assert info.last_path == (PATH_MARCH if march else PATH_STEP)
    return res


def check(pkg, cfg, srcs, rec, snaps=False, item=None):
    w = cfg["wavelet"]
    res = run(pkg, cfg, w, srcs, rec, snaps, item=item)
    step = run(pkg, cfg, w, srcs, rec, snaps, march=False)
    v64, w64 = cfg["vel"].astype(np.float64), np.asarray(w, np.float64)
    for k, s in enumerate(srcs):
        ref = oracle.forward(cfg, v64, w64, src=s, rec=rec, snaps=snaps)
        assert rel(res["gather"][k], ref["gather"]) <= 1e-4, k
        assert rel(res["gather"][k], step["gather"][k]) <= 1e-5, k
        if snaps:
            assert rel(res["snaps"][k], ref["snaps"]) <= 1e-4, k
            assert rel(res["snaps"][k], step["snaps"][k]) <= 1e-5, k
    return res


def ragged_cfg(bc, fs, nt=420):
    nz, nx = 57, 301
    nb = 13
    cfg = dict(ndim=2, nz=nz, ny=1, nx=nx, h=10.0, dt=1e-3, nt=nt, bc=bc,
               nb=[0 if fs else 11, nb, 0, 0, 9, nb], free_surface=fs, R=1e-3, f_ref=12.0,
               snap_every=11, snap_begin=3, snap_end=nt - 5)
    cfg["vel"] = synth.procedural_2d(nz, nx, 10.0, 404)
    cfg["wavelet"] = synth.ricker(12.0, 0.08, 1e-3, nt)
    return cfg


SRCS = np.array([[123.4, 5.0], [1600.0, 27.3], [2990.0, 60.0]])


def rec_line():
    return np.stack([np.linspace(0.0, 3000.0, 97), np.linspace(3.0, 560.0, 97)], axis=1)


@pytest.mark.parametrize("item", [None, 0])
@pytest.mark.parametrize("bc", ["cpml", "sponge", "none"])
def test_c1_every_boundary(pkg, bc, item):
    c = synth.config_c1(nt=700, bc=bc)
    check(pkg, c, c["src"], c["rec"], item=item)


@pytest.mark.parametrize("bc,fs", [("cpml", 1), ("cpml", 0), ("sponge", 1), ("sponge", 0), ("none", 1)])
def test_ragged_snapshots_multishot(pkg, bc, fs):
    cfg = ragged_cfg(bc, fs)
    check(pkg, cfg, SRCS, rec_line(), snaps=True)


@pytest.mark.parametrize("split", [dict(item=4), dict(item=8), dict(item=0, min_rows=1), dict(item=0, min_rows=7)])
@pytest.mark.parametrize("bc,fs", [("cpml", 1), ("cpml", 0), ("sponge", 1)])
def test_short_segments_change_nothing(pkg, bc, fs, split):
    # items / segments of a few rows start everywhere: inside z strips, right
    # below the free surface, mid list tile; every cell must come out the same
    cfg = ragged_cfg(bc, fs, nt=160)
    rec = rec_line()
    base = run(pkg, cfg, cfg["wavelet"], SRCS, rec, snaps=True)
    short = run(pkg, cfg, cfg["wavelet"], SRCS, rec, snaps=True, **split)
    if bc == "sponge":
        assert np.array_equal(base["gather"], short["gather"])
        assert np.array_equal(base["snaps"], short["snaps"])
    else:
        assert rel(short["gather"], base["gather"]) <= 1e-6
        assert rel(short["snaps"], base["snaps"]) <= 1e-6


def test_fp16_snapshots_match_the_step_kernel(pkg):
    cfg = ragged_cfg("cpml", 1, nt=300)
    rec = rec_line()
    a = run(pkg, cfg, cfg["wavelet"], SRCS, rec, snaps=True, snap_fp16=True)
    b = run(pkg, cfg, cfg["wavelet"], SRCS, rec, snaps=True, snap_fp16=True, march=False)
    # the same power-of-two scales, FP16 values within one rounding of each other
    assert np.array_equal(a["snap_scale"], b["snap_scale"])
    sa = a["snaps"].astype(np.float64) * a["snap_scale"][..., None, None]
    sb = b["snaps"].astype(np.float64) * b["snap_scale"][..., None, None]
    assert rel(sa, sb) <= 2e-3
    ref = oracle.forward(cfg, cfg["vel"].astype(np.float64), cfg["wavelet"].astype(np.float64), src=SRCS[1],
                         rec=rec, snaps=True)["snaps"]
    assert rel(sa[1], ref) <= 1e-2


def test_c2_field_slice(pkg):
    c = synth.config_c2(nt=1200)
    c.update(snap_every=100, snap_end=1200)
    check(pkg, c, c["src"], c["rec"], snaps=True)


@pytest.mark.parametrize("nt", [1, 2, 3])
def test_shortest_runs(pkg, nt):
    c = synth.config_c1(nt=nt)
    c["wavelet"] = np.ones(nt, np.float32)
    res = run(pkg, c, c["wavelet"], c["src"], c["rec"])
    ref = oracle.forward(c, c["vel"].astype(np.float64), c["wavelet"].astype(np.float64), src=c["src"][0],
                         rec=c["rec"])["gather"]
    step = run(pkg, c, c["wavelet"], c["src"], c["rec"], march=False)
    assert np.allclose(res["gather"][0], ref, rtol=1e-5, atol=1e-7 * max(1.0, np.abs(ref).max()))
    assert np.allclose(res["gather"][0], step["gather"][0], rtol=1e-6, atol=0)
