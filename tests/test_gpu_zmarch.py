"""The two staging variants of the 3D z-march (per-thread cp.async copies,
and bulk tensor copies by the tensor memory accelerator with mbarrier
completion; the latter also takes over the x-strip CPML pass), at several z
chunks per CTA: within a variant, every chunk gives the same bits; the two
variants give the same bits where no x strip is folded in (sponge) and agree
to FP32 rounding where it is (the same expressions, compiled into different
kernels, may contract their multiply-adds differently); all within 1e-4 of
the FP64 oracle; the 3D gradient likewise."""
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
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def case(bc, fs, nt=140):
    nz, ny, nx, nb = 37, 21, 150, 8
    cfg = dict(ndim=3, nz=nz, ny=ny, nx=nx, h=10.0, dt=8e-4, nt=nt, bc=bc,
               nb=[0 if fs else nb, nb, nb, nb, nb, nb], free_surface=fs, R=1e-3, f_ref=15.0,
               snap_every=47, snap_begin=3, snap_end=nt)
    vel = synth.procedural_3d(nz, ny, nx, 10.0, 61)
    w = synth.ricker(15.0, 0.06, 8e-4, nt)
    src = np.array([[733.0, 102.5, 40.0], [80.0, 30.0, 300.0]])
    rng = np.random.default_rng(8)
    rec = np.stack([rng.uniform(0, 1490, 50), rng.uniform(0, 200, 50), rng.uniform(0, 360, 50)], axis=1)
    return cfg, vel, w, src, rec


def run(pkg, monkeypatch, variant, chunk, cfg, vel, w, src, rec):
    monkeypatch.setenv("GSIM_ZMARCH", variant)
    monkeypatch.setenv("GSIM_ZCHUNK", str(chunk))
    sim = pkg.Simulator(cfg, vel, max_shots=len(src), max_rec=len(rec))
    out = sim.forward(w, src, rec, snapshots=True)
    sim.sync()
    res = out["gather"].cpu().numpy(), out["snaps"].cpu().numpy()
    sim.close()
    return res


@pytest.mark.parametrize("bc,fs", [("cpml", 1), ("sponge", 0)])
def test_variants_and_chunks_agree_with_oracle(pkg, monkeypatch, bc, fs):
    cfg, vel, w, src, rec = case(bc, fs)
    ref = [oracle.forward(cfg, vel.astype(np.float64), w.astype(np.float64), src=s, rec=rec, snaps=True)
           for s in src]
    first = {}
    for variant in ("async", "tma", "tma-plain", "tma-loop", "tma-loop-fold", "tma-loop3"):
        for chunk in (cfg["nz"] + 8, 13, 5):
            g, sn = run(pkg, monkeypatch, variant, chunk, cfg, vel, w, src, rec)
            for k in range(len(src)):
                assert rel(g[k], ref[k]["gather"]) <= 1e-4, (variant, chunk, k)
                assert rel(sn[k], ref[k]["snaps"]) <= 1e-4, (variant, chunk, k)
            if variant not in first:
                first[variant] = (g, sn)
            else:
                assert np.array_equal(g, first[variant][0]) and np.array_equal(sn, first[variant][1]), (variant, chunk)
    (ga, sa), (gt, st), (gp, sp) = first["async"], first["tma"], first["tma-plain"]
    assert np.array_equal(gp, ga) and np.array_equal(sp, sa)  # the same passes, the same bits
    assert np.array_equal(first["tma-loop"][0], ga) and np.array_equal(first["tma-loop"][1], sa)
    assert np.array_equal(first["tma-loop3"][0], ga) and np.array_equal(first["tma-loop3"][1], sa)
    assert rel(first["tma-loop-fold"][0], ga) <= 1e-6 and rel(first["tma-loop-fold"][1], sa) <= 1e-6
    if bc == "cpml":
        assert rel(gt, ga) <= 1e-6 and rel(st, sa) <= 1e-6
    else:
        assert np.array_equal(gt, ga) and np.array_equal(st, sa)


def test_variants_give_the_same_gradient(pkg, monkeypatch):
    cfg, vel, w, src, rec = case("cpml", 0, nt=90)
    cfg.update(snap_every=0, snap_end=0)
    v0 = np.asarray(0.95 * synth.smooth(vel, 3.0), np.float32)  # a misfit far above the FP32 rounding of g
    d = np.stack([oracle.forward(cfg, vel.astype(np.float64), w.astype(np.float64), src=s, rec=rec)["gather"]
                  for s in src])
    ref = np.zeros(v0.shape)
    for k, s in enumerate(src):
        ref += oracle.gradient(cfg, v0.astype(np.float64), w.astype(np.float64), s, rec, d[k])["grad"]
    out = []
    for variant in ("async", "tma", "tma-loop3", "tma-plain"):
        monkeypatch.setenv("GSIM_ZMARCH", variant)
        monkeypatch.setenv("GSIM_ZCHUNK", "11")
        sim = pkg.Simulator(cfg, v0, max_shots=len(src), max_rec=len(rec))
        grad = torch.zeros(v0.shape, device="cuda")
        pkg.sim_adjoint(sim.handle, len(src), torch.as_tensor(w, device="cuda"), np.ascontiguousarray(src), len(rec),
                        np.ascontiguousarray(rec), torch.as_tensor(d, dtype=torch.float32, device="cuda"), None, None,
                        0, grad)
        sim.sync()
        out.append(grad.cpu().numpy())
        sim.close()
    assert rel(out[1], out[0]) <= 1e-6  # CPML: the x strips are folded into the TMA march
    # unfolded TMA marches (record and adjoint modes, loop unrolled by 3 or 9): the cp.async march's bits
    assert np.array_equal(out[2], out[0]) and np.array_equal(out[3], out[0])
    assert rel(out[0], ref) <= 1e-4 and rel(out[1], ref) <= 1e-4
