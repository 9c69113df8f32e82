"""The paper's production runs (Sec. "Wavefield and shot-gather acquisition
geometry"), shortened: band-passed source wavelet made by the library, 60-cell
sponge, free top, 64 (here 4) shots in one sim_batch, and the single-source
wavefield with snapshots every 14 steps on the resident path. End to end
against the FP64 oracle (the oracle's own wavelet and solver): relative L2
<= 1e-4, the FP32 tolerance of the other forward tests."""
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
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_shot_gathers(pkg):
    c = synth.config_c6("gather", nt=700, nshots=4)
    lo, hi, f0 = c["band"]
    w = pkg.bandpass_ricker(c["nt"], c["dt"], f0, lo, hi)
    sim = pkg.Simulator(c, c["vel"], max_shots=4, max_rec=len(c["rec"]))
    (g,) = pkg.batch([dict(sim=sim, wavelet=w, src=c["src"], rec=c["rec"])])
    torch.cuda.synchronize()
    saved = g[:, ::c["save_every"], :]
    assert tuple(saved.shape) == (4, 50, 1000)
    w64 = W.bandpass_ricker(f0, lo, hi, c["dt"], c["nt"])
    for k in (0, 3):
        ref = oracle.forward(c, c["vel"].astype(np.float64), w64, src=c["src"][k], rec=c["rec"])["gather"]
        assert rel(g[k].cpu().numpy(), ref) <= 1e-4, k
    sim.close()


def test_wavefield_snapshots(pkg):
    c = synth.config_c6("wavefield", nt=600)
    lo, hi, f0 = c["band"]
    w = pkg.bandpass_ricker(c["nt"], c["dt"], f0, lo, hi)
    sim = pkg.Simulator(c, c["vel"], max_rec=0)
    out = sim.forward(w, c["src"], None, snapshots=True)
    sim.sync()
    assert pkg.sim_get_info(sim.handle).last_path == 2  # resident
    snaps = out["snaps"][0].cpu().numpy()
    assert snaps.shape == (43, 619, 1000)
    w64 = W.bandpass_ricker(f0, lo, hi, c["dt"], c["nt"])
    ref = oracle.forward(c, c["vel"].astype(np.float64), w64, src=c["src"][0], snaps=True)["snaps"]
    assert rel(snaps, ref) <= 1e-4
    sim.close()
