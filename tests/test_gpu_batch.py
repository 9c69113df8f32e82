"""sim_batch: many shots on uneven grids, as one row-march launch per step over
all members, one tiled-kernel launch per step ("stepped") or one dataflow
launch ("persistent"); by default the batch autotuner picks between the first
two by timing. Results must equal per-handle sim_forward bit
for bit (the row march on both sides; each cell's arithmetic does not depend on
how the work is split), the two tiled schedules must equal each other bit for
bit, the march must agree with them to FP32 rounding, and everything must
match the FP64 oracle; a bounded wait of the persistent schedule that runs out
reports SIM_ERR_TIMEOUT, not a hang."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(autouse=True)
def march_forward():
    # the bit-for-bit comparisons below are against per-handle forwards on the
    # row march, the kernel of the default batch schedule
    keys = ("GSIM_RESIDENT", "GSIM_MARCH", "GSIM_BATCH")
    old = {k: os.environ.get(k) for k in keys}
    os.environ["GSIM_RESIDENT"] = "0"
    os.environ["GSIM_MARCH"] = "1"
    os.environ["GSIM_BATCH"] = "march"
    yield
    for k, v in old.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_30541_gb300 as p
    p.abi.load()
    return p


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def uneven_slices(nt=300):
    out = []
    for j, (nz, nx, bc, fs, ns) in enumerate([(60, 150, "cpml", 1, 3), (41, 97, "sponge", 1, 2),
                                              (75, 260, "cpml", 0, 4)]):
        nb = 12
        cfg = dict(ndim=2, nz=nz, ny=1, nx=nx, h=10.0, dt=1e-3, nt=nt, bc=bc,
                   nb=[0 if fs else nb, nb, 0, 0, nb, nb], free_surface=fs, f_ref=12.0)
        cfg["vel"] = synth.procedural_2d(nz, nx, 10.0, 900 + j)
        cfg["wavelet"] = synth.ricker(12.0, 0.08, 1e-3, nt)
        cfg["src"] = np.stack([np.linspace(50.0, (nx - 5) * 10.0, ns), np.full(ns, 10.0 + 5 * j)], axis=1)
        cfg["rec"] = synth.line(0.0, (nx - 1) * 10.0, nx // 3, 20.0)
        out.append(cfg)
    return out


def sims_for(pkg, slices):
    return [pkg.Simulator(c, c["vel"], max_shots=len(c["src"]), max_rec=len(c["rec"])) for c in slices]


def test_batch_equals_forward_and_oracle(pkg):
    slices = uneven_slices()
    sims = sims_for(pkg, slices)
    gb = pkg.batch([dict(sim=s, wavelet=c["wavelet"], src=c["src"], rec=c["rec"]) for s, c in zip(sims, slices)])
    torch.cuda.synchronize()
    for s, c, g in zip(sims, slices, gb):
        ref = s.forward(c["wavelet"], c["src"], c["rec"])["gather"]
        assert torch.equal(g, ref)
        o = oracle.forward(c, c["vel"].astype(np.float64), c["wavelet"].astype(np.float64), src=c["src"][-1],
                           rec=c["rec"])["gather"]
        assert rel(g[-1].cpu().numpy(), o) <= 1e-4
    for s in sims:
        s.close()


def batch_with(pkg, entries, schedule):
    if schedule is None:
        return [g.clone() for g in pkg.batch(entries)]
    os.environ["GSIM_BATCH"] = schedule
    try:
        return [g.clone() for g in pkg.batch(entries)]
    finally:
        del os.environ["GSIM_BATCH"]


def test_schedules_agree(pkg):
    slices = uneven_slices(nt=200)
    sims = sims_for(pkg, slices)
    entries = [dict(sim=s, wavelet=c["wavelet"], src=c["src"], rec=c["rec"]) for s, c in zip(sims, slices)]
    march = batch_with(pkg, entries, None)
    stepped = batch_with(pkg, entries, "stepped")
    persistent = batch_with(pkg, entries, "persistent")
    for a, b, c in zip(march, stepped, persistent):
        assert torch.equal(b, c)
        assert rel(a.cpu().numpy(), b.cpu().numpy().astype(np.float64)) <= 1e-5
    for s in sims:
        s.close()


def test_batch_timeout_is_reported_and_recoverable(pkg):
    slices = uneven_slices(nt=40)
    sims = sims_for(pkg, slices)
    entries = [dict(sim=s, wavelet=c["wavelet"], src=c["src"], rec=c["rec"]) for s, c in zip(sims, slices)]
    os.environ["GSIM_SPIN_LIMIT"] = "0"   # every wait on a neighbour gives up at once
    os.environ["GSIM_BATCH"] = "persistent"  # the schedule whose tiles wait on one another
    try:
        with pytest.raises(pkg.SimError) as e:
            pkg.batch(entries)
        assert e.value.code == pkg.abi.SIM_ERR_TIMEOUT
    finally:
        del os.environ["GSIM_SPIN_LIMIT"]
        del os.environ["GSIM_BATCH"]
    gb = pkg.batch(entries)   # the GPU and the handles stay usable
    ref = sims[0].forward(slices[0]["wavelet"], slices[0]["src"], slices[0]["rec"])["gather"]
    assert torch.equal(gb[0], ref)
    for s in sims:
        s.close()


def test_c3_batched_workload_sampled(pkg):
    # 64 shots on the field-scale slice + 16 uneven slices with 8 shots each, one launch
    nt = 4000
    slices = synth.config_c3(nt=nt)
    sims = sims_for(pkg, slices)
    gb = pkg.batch([dict(sim=s, wavelet=c["wavelet"], src=c["src"], rec=c["rec"]) for s, c in zip(sims, slices)])
    torch.cuda.synchronize()
    # bitwise against per-handle forwards on three slices
    for k in (0, 5, 16):
        ref = sims[k].forward(slices[k]["wavelet"], slices[k]["src"], slices[k]["rec"])["gather"]
        assert torch.equal(gb[k], ref), k
    # FP64 oracle on sampled shots over the first 600 steps
    for k, shot in ((0, 31), (9, 7)):
        c = dict(slices[k], nt=600)
        o = oracle.forward(c, c["vel"].astype(np.float64), c["wavelet"][:600].astype(np.float64),
                           src=c["src"][shot], rec=c["rec"])["gather"]
        assert rel(gb[k][shot, :600].cpu().numpy(), o) <= 1e-4
    for s in sims:
        s.close()


def test_autotuned_batch_matches_its_schedule_and_oracle(pkg, monkeypatch):
    # the schedule the batch autotuner picks (march or stepped, with a tile
    # height) gives the same bits as that schedule forced, and the oracle's
    # gathers to FP32 tolerance
    monkeypatch.delenv("GSIM_BATCH", raising=False)
    monkeypatch.setenv("GSIM_TUNE_LOG", "1")
    slices = uneven_slices()
    sims = sims_for(pkg, slices)
    entries = [dict(sim=s, wavelet=c["wavelet"], src=c["src"], rec=c["rec"]) for s, c in zip(sims, slices)]
    tuned = [g.clone() for g in pkg.batch(entries)]
    torch.cuda.synchronize()
    forced = []
    for sched, tz in (("march", "16"), ("stepped", "8"), ("stepped", "16"), ("stepped", "32")):
        monkeypatch.setenv("GSIM_BATCH", sched)
        monkeypatch.setenv("GSIM_TILE_Z", tz)
        forced.append([g.clone() for g in pkg.batch(entries)])
        torch.cuda.synchronize()
    assert any(all(torch.equal(a, b) for a, b in zip(tuned, f)) for f in forced)
    for c, g in zip(slices, tuned):
        o = oracle.forward(c, c["vel"].astype(np.float64), c["wavelet"].astype(np.float64), src=c["src"][0],
                           rec=c["rec"])["gather"]
        assert rel(g[0].cpu().numpy(), o) <= 1e-4
    for s in sims:
        s.close()


def test_cpml_batch_in_one_or_two_kernels(pkg, monkeypatch):
    # a batch with CPML runs its CPML and plain row-march items as two kernels
    # per step (on two streams); one kernel for all items gives the same bits
    slices = uneven_slices(nt=120)
    sims = sims_for(pkg, slices)
    entries = [dict(sim=s, wavelet=c["wavelet"], src=c["src"], rec=c["rec"]) for s, c in zip(sims, slices)]
    two = [g.clone() for g in pkg.batch(entries)]
    monkeypatch.setenv("GSIM_MARCH_SPLIT", "0")
    one = [g.clone() for g in pkg.batch(entries)]
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(one, two))
    for s in sims:
        s.close()
