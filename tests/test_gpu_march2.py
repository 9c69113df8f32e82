"""The two-step row march (temporal blocking: p^{n+1} and p^{n+2} in one pass
over HBM) for batches without CPML. Each cell's arithmetic is the one-step
march's, so its gathers must equal the one-step march's bit for bit, for odd
and even step counts (a last pass of one step), with and without the free
surface (the odd mirror of both steps' windows), with item heights below the
stencil radius, and agree with the FP64 oracle to FP32 tolerance."""
import os

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


@pytest.fixture(autouse=True)
def clean_env(monkeypatch):
    for k in ("GSIM_BATCH", "GSIM_TB_ROWS", "GSIM_TILE_Z"):
        monkeypatch.delenv(k, raising=False)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def slices_without_cpml(nt):
    # uneven grids: widths that are neither multiples of 4 nor of the
    # 120-column strips, heights that are not multiples of the item height;
    # sources on strip edges, next to the free surface and in the sponge
    out = []
    for j, (nz, nx, bc, fs, nb) in enumerate([(61, 243, "sponge", 1, 14), (47, 121, "sponge", 0, 10),
                                              (38, 357, "none", 1, 0), (29, 119, "none", 0, 0)]):
        cfg = dict(ndim=2, nz=nz, ny=1, nx=nx, h=10.0, dt=1e-3, nt=nt, bc=bc,
                   nb=[0 if fs else nb, nb, 0, 0, nb, nb], free_surface=fs, f_ref=12.0)
        cfg["vel"] = synth.procedural_2d(nz, nx, 10.0, 700 + j)
        cfg["wavelet"] = synth.ricker(12.0, 0.06, 1e-3, nt)
        xs = [1190.5, 1200.0, 15.0, (nx - 2) * 10.0]
        zs = [10.0, 3.0, 25.0, (nz - 2) * 10.0]
        src = np.array([[min(x, (nx - 1) * 10.0), z] for x, z in zip(xs, zs)], np.float64)
        cfg["src"] = src
        cfg["rec"] = np.concatenate([synth.line(0.0, (nx - 1) * 10.0, nx // 4, 5.0 if fs else 20.0),
                                     np.array([[1195.0 if nx > 121 else 600.0, (nz - 1) * 10.0 - 5.0]])])
        out.append(cfg)
    return out


def run(pkg, sims, slices, sched, rows=None):
    os.environ["GSIM_BATCH"] = sched
    if rows is not None:
        os.environ["GSIM_TB_ROWS"] = str(rows)
    try:
        outs = pkg.batch([dict(sim=s, wavelet=c["wavelet"], src=c["src"], rec=c["rec"]) for s, c in zip(sims, slices)])
        torch.cuda.synchronize()
        return [g.clone() for g in outs]
    finally:
        os.environ.pop("GSIM_BATCH", None)
        os.environ.pop("GSIM_TB_ROWS", None)


def open_sims(pkg, slices):
    return [pkg.Simulator(c, c["vel"], max_shots=len(c["src"]), max_rec=len(c["rec"])) for c in slices]


@pytest.mark.parametrize("nt", [160, 161])
def test_two_step_equals_one_step_and_oracle(pkg, nt):
    slices = slices_without_cpml(nt)
    sims = open_sims(pkg, slices)
    one = run(pkg, sims, slices, "march")
    two = run(pkg, sims, slices, "march2")
    for k, (a, b) in enumerate(zip(one, two)):
        d = float((a - b).abs().max())
        assert torch.equal(a, b), (k, d)
    for c, g in zip(slices, two):
        for shot in (0, 1):
            o = oracle.forward(c, c["vel"].astype(np.float64), c["wavelet"].astype(np.float64), src=c["src"][shot],
                               rec=c["rec"])["gather"]
            assert rel(g[shot].cpu().numpy(), o) <= 1e-4
    for s in sims:
        s.close()


@pytest.mark.parametrize("rows", [3, 5, 64])
def test_item_heights(pkg, rows):
    # items of 3 and 5 rows start below row 4 next to the free surface, so the
    # mirror of the p^{n+1} window is taken in an item that does not own row 0
    slices = slices_without_cpml(61)
    sims = open_sims(pkg, slices)
    ref = run(pkg, sims, slices, "march")
    got = run(pkg, sims, slices, "march2", rows=rows)
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    for s in sims:
        s.close()


def test_repeated_runs_and_single_step(pkg):
    # the graph is replayed with its counters reset; one step is one pass of one step
    slices = slices_without_cpml(1)
    sims = open_sims(pkg, slices)
    a = run(pkg, sims, slices, "march")
    b = run(pkg, sims, slices, "march2")
    assert all(torch.equal(x, y) for x, y in zip(a, b))
    for s in sims:
        s.close()
    slices = slices_without_cpml(41)
    sims = open_sims(pkg, slices)
    first = run(pkg, sims, slices, "march2")
    again = run(pkg, sims, slices, "march2")
    assert all(torch.equal(x, y) for x, y in zip(first, again))
    for s in sims:
        s.close()


def test_cpml_item_is_refused(pkg):
    c = slices_without_cpml(20)[1]
    c = dict(c, bc="cpml")
    s = pkg.Simulator(c, c["vel"], max_shots=len(c["src"]), max_rec=len(c["rec"]))
    with pytest.raises(pkg.SimError) as e:
        run(pkg, [s], [c], "march2")
    assert e.value.code == pkg.abi.SIM_ERR_UNSUPPORTED
    s.close()


def test_autotuner_candidates_without_cpml(pkg, monkeypatch):
    # without CPML the tuner also times the two-step march; its pick gives
    # the bits of one of the schedules forced
    monkeypatch.setenv("GSIM_TUNE_LOG", "1")
    slices = slices_without_cpml(120)
    sims = open_sims(pkg, slices)
    entries = [dict(sim=s, wavelet=c["wavelet"], src=c["src"], rec=c["rec"]) for s, c in zip(sims, slices)]
    tuned = [g.clone() for g in pkg.batch(entries)]
    torch.cuda.synchronize()
    forced = [run(pkg, sims, slices, "march"), run(pkg, sims, slices, "march2")]
    for tz in ("8", "16", "32"):
        monkeypatch.setenv("GSIM_TILE_Z", tz)
        forced.append(run(pkg, sims, slices, "stepped"))
        monkeypatch.delenv("GSIM_TILE_Z")
    assert any(all(torch.equal(a, b) for a, b in zip(tuned, f)) for f in forced)
    for s in sims:
        s.close()


def test_production_gathers_full_length(pkg):
    # the production run itself (64 shots, 8001 steps, 60-cell sponge, free
    # surface, 1000 receivers, band-passed wavelet): the two-step march gives
    # the one-step march's bits on every gather sample (whichever of the two
    # the batch autotuner picks is compared with the FP64 oracle at full
    # length in test_gpu_fullsize)
    c6 = synth.config_c6("gather")
    lo, hi, f0 = c6["band"]
    wav = pkg.bandpass_ricker(c6["nt"], c6["dt"], f0, lo, hi).cpu().numpy()
    sim = pkg.Simulator(c6, c6["vel"], max_shots=len(c6["src"]), max_rec=len(c6["rec"]))
    one = run(pkg, [sim], [dict(c6, wavelet=wav)], "march")[0]
    two = run(pkg, [sim], [dict(c6, wavelet=wav)], "march2")[0]
    assert torch.isfinite(two).all()
    assert torch.equal(one, two)
    sim.close()
