"""The forward entry point for callers that cannot allocate device memory when
they call: processes whose device memory a framework's pool has reserved in
full, and paths where cudaMalloc's device synchronisation is not acceptable.
It keeps its working set in a fixed array inside the library. Here its gathers
must match sim_forward's within the tolerance of the other parity tests, and
the FP64 oracle's, on two calls in a row (the second reuses the array the
first left behind); a call must leave the device's free memory unchanged; and
a problem larger than the array must be refused before any GPU work."""
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
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("bc", ["cpml", "sponge"])
def test_noalloc_matches_forward_and_oracle_on_two_calls(pkg, bc):
    c = synth.config_c1(nt=600, bc=bc)
    rec = np.ascontiguousarray(c["rec"])
    nrec = len(rec)
    sources = [np.array([[1000.0, 20.0]]), np.array([[615.0, 137.5]])]
    sim = pkg.Simulator(c, c["vel"], max_shots=1, max_rec=nrec)
    refs = [sim.forward(c["wavelet"], s, rec)["gather"][0].cpu().numpy() for s in sources]
    sim.close()
    v64, w64 = c["vel"].astype(np.float64), c["wavelet"].astype(np.float64)
    exact = [oracle.forward(c, v64, w64, src=s[0], rec=rec)["gather"] for s in sources]
    desc = pkg.make_desc(c, max_shots=1, max_rec=nrec)
    vel = torch.as_tensor(c["vel"], device="cuda")
    w = torch.as_tensor(c["wavelet"], device="cuda")
    for s, ref, ex in zip(sources, refs, exact):
        g = torch.full((c["nt"], nrec), float("nan"), device="cuda")
        pkg.sim_forward_noalloc(desc, vel, w, np.ascontiguousarray(s[0]), nrec, rec, g)
        out = g.cpu().numpy()
        assert rel(out, ref) <= 1e-4
        assert rel(out, ex) <= 1e-4


def test_noalloc_leaves_free_device_memory_unchanged(pkg):
    # driver-level free memory (outside torch's caching allocator) after a
    # warm-up call and after a second call: the call allocates nothing
    c = synth.config_c1(nt=200)
    rec = np.ascontiguousarray(c["rec"])
    desc = pkg.make_desc(c, max_shots=1, max_rec=len(rec))
    vel = torch.as_tensor(c["vel"], device="cuda")
    w = torch.as_tensor(c["wavelet"], device="cuda")
    g = torch.empty((c["nt"], len(rec)), device="cuda")
    src = np.ascontiguousarray(c["src"][0])
    pkg.sim_forward_noalloc(desc, vel, w, src, len(rec), rec, g)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    pkg.sim_forward_noalloc(desc, vel, w, src, len(rec), rec, g)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_refuses_problems_larger_than_its_array(pkg):
    # 2000 x 2000 cells with a 20-cell sponge: four fields of about 17 MB each
    c = dict(ndim=2, nz=2000, ny=1, nx=2000, h=10.0, dt=1e-3, nt=10, bc="sponge", nb=[20, 20, 0, 0, 20, 20])
    desc = pkg.make_desc(c, max_shots=1, max_rec=1)
    vel = torch.full((2000, 2000), 2000.0, device="cuda")
    w = torch.zeros(10, device="cuda")
    g = torch.zeros((10, 1), device="cuda")
    with pytest.raises(pkg.SimError) as e:
        pkg.sim_forward_noalloc(desc, vel, w, np.array([5000.0, 100.0]), 1, np.array([[100.0, 10.0]]), g)
    assert e.value.code == pkg.abi.SIM_ERR_ARG
    assert "32 MiB" in pkg.sim_last_error(None)
