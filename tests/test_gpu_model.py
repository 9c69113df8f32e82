"""GPU model-builder warps (sim_model_squish / _fault / _deposit) against the
FP64 oracle (oracle/model.py) on the same seeded inputs: velocities within
FP32 rounding of the interpolation sums (relative 2e-6 of the velocity
range, interior and fill voxels alike), labels bit for bit. 2D slices and 3D
volumes, curved and planar faults in both walls' directions, sorted and
crossing bed boundaries with texture and tapers, displacements reaching
beyond the grid (fill). Then a model built on the device by a chain of the
warps feeds Simulator and sim_batch without a host copy: the batch gathers
equal per-handle forwards on the same device models bit for bit, and the
device model equals the oracle's chain."""
import numpy as np
import pytest

import synth
from oracle import model as om

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_30541_gb300 as p
    p.abi.load()
    return p


def check(vg, lg, vo, lo):
    vg = vg.cpu().numpy().astype(np.float64)
    span = max(1.0, float(np.ptp(vo)))
    assert np.abs(vg - vo).max() <= 2e-6 * max(span, float(np.abs(vo).max())), np.abs(vg - vo).max()
    if lo is not None:
        assert np.array_equal(lg.cpu().numpy(), lo)


def field(shape, seed, lo=1500.0, hi=4500.0):
    rng = np.random.default_rng(seed)
    v = synth.smooth(rng.uniform(lo, hi, shape).astype(np.float32), 1.5).astype(np.float32)
    lab = rng.integers(0, 12, shape).astype(np.int32)
    return v, lab


@pytest.mark.parametrize("shape", [(57, 1, 83), (20, 9, 13)])
def test_squish_matches_oracle(pkg, shape):
    from paper_2605_30541_gb300 import model
    v, lab = field(shape, 11)
    nz, ny, nx = shape
    rng = np.random.default_rng(12)
    dz = (synth.smooth(rng.uniform(-7, 7, (ny, nx)).astype(np.float32), 2.0) * 2.5).astype(np.float32)
    dz.flat[0] = 3.0       # an integer shift
    dz.flat[-1] = -0.5     # a half-cell tie for the labels
    vg, lg = model.squish(torch.as_tensor(v, device="cuda"), torch.as_tensor(lab, device="cuda"), dz, 1234.0, -1)
    vo, lo = om.squish(v, lab, dz.astype(np.float64), 1234.0, -1)
    check(vg, lg, vo, lo)
    assert (lo == -1).any()  # some columns pulled from beyond the grid


FAULTS = [
    dict(cz=25.0, cy=0.0, cx=40.0, azimuth=np.pi / 2, dip=np.deg2rad(60.0), radius=600.0, slip=7.3, direction=1,
         d_die=18.0, d_perp=1e9, theta_die=np.deg2rad(25.0)),
    dict(cz=15.0, cy=0.0, cx=50.0, azimuth=-np.pi / 2, dip=np.deg2rad(55.0), radius=45.0, slip=5.0, direction=-1,
         d_die=12.0, d_perp=1e9, theta_die=np.deg2rad(70.0)),
]


@pytest.mark.parametrize("k", [0, 1])
def test_fault_2d_matches_oracle(pkg, k):
    from paper_2605_30541_gb300 import model
    v, lab = field((60, 1, 90), 21 + k)
    p = FAULTS[k]
    vg, lg = model.fault(torch.as_tensor(v[:, 0], device="cuda"), torch.as_tensor(lab[:, 0], device="cuda"),
                         fill=999.0, fill_label=-2, **p)
    vo, lo = om.fault(v, lab, p, 999.0, -2)
    check(vg.unsqueeze(1), lg.unsqueeze(1), vo, lo)
    assert np.abs(vo - v).max() > 100.0  # the fault moved something


def test_fault_3d_matches_oracle(pkg):
    from paper_2605_30541_gb300 import model
    v, lab = field((24, 18, 22), 31)
    p = dict(cz=10.0, cy=8.0, cx=11.0, azimuth=0.7, dip=np.deg2rad(62.0), radius=80.0, slip=3.5, direction=1,
             d_die=9.0, d_perp=7.0, theta_die=np.deg2rad(40.0))
    vg, lg = model.fault(torch.as_tensor(v, device="cuda"), torch.as_tensor(lab, device="cuda"), fill=0.0,
                         fill_label=-1, **p)
    vo, lo = om.fault(v, lab, p, 0.0, -1)
    check(vg, lg, vo, lo)


@pytest.mark.parametrize("shape", [(70, 1, 64), (30, 7, 11)])
def test_deposit_matches_oracle(pkg, shape):
    from paper_2605_30541_gb300 import model
    v, lab = field(shape, 41)
    nz, ny, nx = shape
    t, nb = 23, 5
    rng = np.random.default_rng(42)
    base = np.sort(rng.uniform(2, t - 2, nb - 1))
    bounds = (base[:, None, None] + 1.5 * rng.standard_normal((nb - 1, ny, nx))).astype(np.float32)
    bounds = np.clip(bounds, 0, t - 1)  # neighbouring boundaries may cross
    vbed = rng.normal(2200.0, 150.0, nb).astype(np.float32)
    eta = rng.standard_normal((40, ny, nx)).astype(np.float32)
    off = rng.integers(0, 12, nb)
    args = dict(beta=6.0, a_eta=35.0, f_top=0.15, f_base=0.2)
    vg, lg = model.deposit(torch.as_tensor(v, device="cuda"), torch.as_tensor(lab, device="cuda"), t, bounds, vbed,
                           eta=eta, offsets=off, label0=20, **args)
    vo, lo = om.deposit(v, lab, t, bounds.astype(np.float64), vbed.astype(np.float64), args["beta"], args["a_eta"],
                        args["f_top"], args["f_base"], eta.astype(np.float64), off, 20)
    check(vg, lg, vo, lo)


def test_argument_errors(pkg):
    from paper_2605_30541_gb300 import model
    v = torch.full((10, 12), 2000.0, device="cuda")
    with pytest.raises(pkg.SimError) as e:
        pkg.sim_model_squish(10, 1, 12, v, None, torch.zeros(12, device="cuda"), 0.0, 0, v, None)
    assert e.value.code == pkg.abi.SIM_ERR_ARG
    with pytest.raises(pkg.SimError):
        model.fault(v, None, 5.0, 6.0, 1.0, 0.0, 1.0)  # radius 0
    with pytest.raises(pkg.SimError):
        model.deposit(v, None, 0, None, [2000.0])       # t = 0


def chain_inputs(nz, nx, seed):
    rng = np.random.default_rng(seed)
    base = np.full((nz, 1, nx), 3600.0, np.float32)
    lab = np.zeros((nz, 1, nx), np.int32)
    layers = []
    for k in range(3):
        t = 18
        nb = 3
        b = np.sort(rng.uniform(3, t - 3, nb - 1))[:, None, None] + rng.standard_normal((nb - 1, 1, nx)) * 0.8
        layers.append(dict(t=t, bounds=np.clip(b, 0, t - 1).astype(np.float32),
                           vbed=rng.normal(2000.0 + 400.0 * (2 - k), 120.0, nb).astype(np.float32),
                           eta=rng.standard_normal((30, 1, nx)).astype(np.float32), off=rng.integers(0, 8, nb),
                           label0=10 * (k + 1)))
    dz = (synth.smooth(rng.uniform(-1, 1, (1, nx)).astype(np.float32), 6.0) * 40.0).astype(np.float32)
    flt = dict(cz=30.0, cy=0.0, cx=nx * 0.55, azimuth=np.pi / 2, dip=np.deg2rad(60.0), radius=900.0, slip=6.0,
               direction=1, d_die=25.0, d_perp=1e9, theta_die=np.deg2rad(30.0))
    return base, lab, layers, dz, flt


def test_device_models_feed_the_batch(pkg):
    from paper_2605_30541_gb300 import model
    nz, nx = 80, 150
    slices, models = [], []
    for seed in (51, 52):
        base, lab, layers, dz, flt = chain_inputs(nz, nx, seed)
        vg, lg = torch.as_tensor(base, device="cuda"), torch.as_tensor(lab, device="cuda")
        vo, lo = base.astype(np.float64), lab.copy()
        for L in layers:
            vg, lg = model.deposit(vg, lg, L["t"], L["bounds"], L["vbed"], beta=4.0, a_eta=25.0, f_top=0.1,
                                   f_base=0.1, eta=L["eta"], offsets=L["off"], label0=L["label0"])
            vo, lo = om.deposit(vo, lo, L["t"], L["bounds"].astype(np.float64), L["vbed"].astype(np.float64), 4.0,
                                25.0, 0.1, 0.1, L["eta"].astype(np.float64), L["off"], L["label0"])
        vg, lg = model.squish(vg, lg, dz, 1500.0, 0)
        vo, lo = om.squish(vo.astype(np.float32).astype(np.float64), lo, dz.astype(np.float64), 1500.0, 0)
        vg, lg = model.fault(vg, lg, fill=1500.0, fill_label=0, **flt)
        vo, lo = om.fault(vo.astype(np.float32).astype(np.float64), lo, flt, 1500.0, 0)
        # each step starts from the GPU's FP32 result rounded the same way; the
        # chain as a whole stays within a few FP32 roundings per step
        assert np.abs(vg.cpu().numpy().astype(np.float64) - vo).max() < 5e-3
        models.append(vg[:, 0].contiguous())
        cfg = dict(ndim=2, nz=nz, ny=1, nx=nx, h=10.0, dt=1e-3, nt=300, bc="sponge", nb=[0, 20, 0, 0, 20, 20],
                   free_surface=1, R=1e-3, f_ref=12.0, snap_every=0, snap_begin=0, snap_end=0)
        slices.append(cfg)
    w = synth.ricker(12.0, 0.08, 1e-3, 300)
    src = np.array([[300.0, 10.0], [900.0, 10.0]])
    rec = synth.line(0.0, (nx - 1) * 10.0, 50, 10.0)
    sims = [pkg.Simulator(c, m, max_shots=2, max_rec=len(rec)) for c, m in zip(slices, models)]
    import os
    os.environ["GSIM_BATCH"] = "march"  # the bit-for-bit reference below is the row march
    try:
        gb = pkg.batch([dict(sim=s, wavelet=w, src=src, rec=rec) for s in sims])
        torch.cuda.synchronize()
    finally:
        del os.environ["GSIM_BATCH"]
    os.environ["GSIM_MARCH"] = "1"
    os.environ["GSIM_RESIDENT"] = "0"
    try:
        for s, g in zip(sims, gb):
            ref = s.forward(w, src, rec)["gather"]
            assert torch.equal(g, ref)
            assert torch.isfinite(g).all() and g.abs().max() > 0
    finally:
        del os.environ["GSIM_MARCH"], os.environ["GSIM_RESIDENT"]
    for s in sims:
        s.close()
