"""Parity of the measured configurations at their full sizes and lengths.

- The 619 x 1000 slice (50-cell CPML, free top) over all 8000 steps with its
  500 FP32 snapshots, on the resident path: gathers and snapshots against the
  FP64 oracle, with the relative L2 error reported every 1000 steps (FP32
  drift over the whole record).
- One shot of the paper's 64-shot production gather run (60-cell sponge,
  band-passed source, nt = 8001) on the batch autotuner's schedule (the
  one-step or the two-step row march), and the 5 s production
  wavefield (358 snapshots, nt = 5001) on the resident path.
- The 3D volume at its full size (619 x 1000 x 1000 + 30-cell CPML on x, y
  and bottom, free top: 729 M padded cells, 2.9 GB per field) for the first
  24 steps. A value spreads at most 4 cells per step (8 inside a CPML layer,
  whose memory terms chain two first derivatives), so after 24 steps the
  field is exactly zero beyond that reach; the oracle runs on a crop that
  holds the whole reach (with the real CPML faces where the crop meets
  them), and everything outside the crop must be exactly zero on the GPU.
  Two shots: the surface centre, and a corner next to the -x, -y and bottom
  CPML faces (edges and the corner of the layers).

Bar: relative L2 <= 1e-4 against the oracle (the FP32 tolerance)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import wavelet as W

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
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_c2_full_length_gathers_and_snapshots(pkg):
    c = synth.config_c2()
    assert c["nt"] == 8000
    sim = pkg.Simulator(c, c["vel"], max_shots=1, max_rec=len(c["rec"]))
    out = sim.forward(c["wavelet"], c["src"], c["rec"], snapshots=True)
    sim.sync()
    assert pkg.sim_get_info(sim.handle).last_path == 2  # resident, as benched
    g = out["gather"][0].cpu().numpy()
    sn = out["snaps"][0].cpu().numpy()
    sim.close()
    assert sn.shape == (500, 619, 1000)
    ref = oracle.forward(c, c["vel"].astype(np.float64), c["wavelet"].astype(np.float64), src=c["src"][0],
                         rec=c["rec"], snaps=True)
    # snapshots whose reference is all zero (before the wave leaves the
    # source cell's neighbourhood: p^0 = 0) must be exactly zero
    zero = [j for j in range(500) if not np.any(ref["snaps"][j])]
    for j in zero:
        assert not np.any(sn[j]), j
    curve = []
    for n in range(1000, 8001, 1000):
        k = min(500, n // 10)
        js = [j for j in range(max(0, k - 100), k) if j not in zero]
        es = max(rel(sn[j], ref["snaps"][j]) for j in js) if n <= 5000 else None
        curve.append((n, rel(g[:n], ref["gather"][:n]), es))
    print("C2 relative L2 vs steps (gather rows < n, worst snapshot of the last 100 before n):", curve)
    for n, eg, es in curve:
        assert eg <= 1e-4, (n, eg)
        assert es is None or es <= 1e-4, (n, es)
    assert rel(sn, ref["snaps"]) <= 1e-4


def test_production_gather_shot_full_length(pkg):
    c = synth.config_c6("gather")
    assert c["nt"] == 8001 and len(c["src"]) == 64
    lo, hi, f0 = c["band"]
    w = pkg.bandpass_ricker(c["nt"], c["dt"], f0, lo, hi)
    sim = pkg.Simulator(c, c["vel"], max_shots=64, max_rec=len(c["rec"]))
    (g,) = pkg.batch([dict(sim=sim, wavelet=w, src=c["src"], rec=c["rec"])])
    torch.cuda.synchronize()
    k = 37
    got = g[k].cpu().numpy()
    sim.close()
    w64 = W.bandpass_ricker(f0, lo, hi, c["dt"], c["nt"])
    ref = oracle.forward(c, c["vel"].astype(np.float64), w64, src=c["src"][k], rec=c["rec"])["gather"]
    assert rel(got, ref) <= 1e-4
    assert rel(got[::c["save_every"]], ref[::c["save_every"]]) <= 1e-4


def test_production_wavefield_full_length(pkg):
    c = synth.config_c6("wavefield")
    assert c["nt"] == 5001
    lo, hi, f0 = c["band"]
    w = pkg.bandpass_ricker(c["nt"], c["dt"], f0, lo, hi)
    sim = pkg.Simulator(c, c["vel"], max_rec=0)
    out = sim.forward(w, c["src"], None, snapshots=True)
    sim.sync()
    assert pkg.sim_get_info(sim.handle).last_path == 2
    snaps = out["snaps"][0].cpu().numpy()
    sim.close()
    assert snaps.shape == (358, 619, 1000)
    w64 = W.bandpass_ricker(f0, lo, hi, c["dt"], c["nt"])
    ref = oracle.forward(c, c["vel"].astype(np.float64), w64, src=c["src"][0], snaps=True)["snaps"]
    assert rel(snaps, ref) <= 1e-4


def _crop_case(c, vel, lo, hi, nb, fs, vmax):
    """Oracle problem on the interior box [lo, hi] (cells, (z, y, x) order,
    inclusive) of the full volume: absorbing faces where the box meets the
    full volume's CPML faces, open (unreached) faces elsewhere."""
    dims = [hi[k] - lo[k] + 1 for k in range(3)]
    crop = dict(ndim=3, nz=dims[0], ny=dims[1], nx=dims[2], h=c["h"], dt=c["dt"], nt=c["nt"], bc="cpml",
                nb=nb, free_surface=fs, R=c["R"], f_ref=c["f_ref"], cpml_vmax=vmax,
                snap_every=c["snap_every"], snap_begin=c["snap_begin"], snap_end=c["snap_end"])
    v = np.ascontiguousarray(vel[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1], np.float64)
    return crop, v


def test_c5_full_size_first_steps(pkg):
    nt = 24
    c = synth.config_c5(nt=nt)
    nz, ny, nx = c["nz"], c["ny"], c["nx"]
    assert (nz, ny, nx) == (619, 1000, 1000) and c["nb"] == [0, 30, 30, 30, 30, 30]
    c.update(snap_every=nt, snap_begin=nt - 1, snap_end=nt)  # one snapshot: p at step nt - 1
    h = c["h"]
    w = synth.ricker(30.0, 0.01, c["dt"], nt)  # peaks within the 24 steps
    vel = c["vel"]
    vmax = float(vel.max())
    srcs = np.array([[500 * h, 500 * h, 1 * h],        # surface centre
                     [2.3 * h, 3.6 * h, 616.5 * h]])   # next to the -x, -y and bottom CPML faces
    rng = np.random.default_rng(5024)
    corner = np.stack([rng.uniform(0, 40 * h, 64), rng.uniform(0, 40 * h, 64), rng.uniform(580 * h, 616.9 * h, 64)], 1)
    rec = np.concatenate([c["rec"], corner])
    sim = pkg.Simulator(c, vel, max_shots=2, max_rec=len(rec))
    out = sim.forward(w, srcs, rec, snapshots=True)
    sim.sync()
    g = out["gather"].cpu().numpy()            # (2, nt, nrec)
    sn = out["snaps"][:, 0].cpu().numpy()      # (2, nz, ny, nx)
    sim.close()
    reach_open, reach_cpml = 4 * nt + 8, 8 * nt + 8
    cases = [
        # centre: the CPML is out of reach; the crop's faces are all open but the free top
        dict(lo=(0, 500 - reach_open, 500 - reach_open), hi=(reach_open, 500 + reach_open, 500 + reach_open),
             nb=[0, 0, 0, 0, 0, 0], fs=1),
        # corner: the crop keeps the -x, -y and bottom CPML faces of the volume
        dict(lo=(nz - 1 - reach_cpml, 0, 0), hi=(nz - 1, reach_cpml, reach_cpml),
             nb=[0, 30, 30, 0, 30, 0], fs=0),
    ]
    for k, cs in enumerate(cases):
        lo, hi = cs["lo"], cs["hi"]
        crop, v = _crop_case(c, vel, lo, hi, cs["nb"], cs["fs"], vmax)
        off = np.array([lo[2], lo[1], lo[0]], np.float64) * h  # (x, y, z) metres
        cell = rec / h
        inside = np.all((cell[:, [2, 1, 0]] >= np.array(lo)) & (cell[:, [2, 1, 0]] <= np.array(hi) - 1), axis=1)
        assert inside.sum() >= 16, k
        ref = oracle.forward(crop, v, w.astype(np.float64), src=srcs[k] - off, rec=rec[inside] - off, snaps=True)
        # everything beyond the reach is exactly zero; inside, the oracle's values
        assert np.all(g[k][:, ~inside] == 0), k
        assert rel(g[k][:, inside], ref["gather"]) <= 1e-4, k
        box = sn[k][lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1]
        assert np.count_nonzero(sn[k]) == np.count_nonzero(box), k
        assert rel(box, ref["snaps"][0]) <= 1e-4, k
