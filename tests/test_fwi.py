"""Multi-iteration FWI (host drivers over the adjoint-state gradient).

CPU: both drivers on the FP64 oracle's misfit and gradient for a small
two-anomaly model: the accepted misfits never increase, they fall by at
least half within a few iterations, the model moves towards the true one
and stays inside the bounds. A quadratic with a known minimiser pins the
drivers themselves.

GPU: L-BFGS on the C4 gradient problem (201 x 201 procedural model, start =
the 250 m smoothed model, 16 shots, 4 s) with FP16 checkpoints and every
shot in one sim_adjoint per evaluation: the misfit falls below 60% of its
start in 6 iterations and the model error falls."""
import numpy as np
import pytest

import oracle
import synth
from paper_2605_30541_gb300 import fwi


def quadratic(target, weights):
    def fun(v):
        r = v - target
        return 0.5 * float(np.sum(weights * r * r)), weights * r
    return fun


@pytest.mark.parametrize("driver", ["lbfgs", "gd"])
def test_drivers_on_a_quadratic(driver):
    rng = np.random.default_rng(3)
    target = 2000.0 + 300.0 * rng.standard_normal((12, 9))
    weights = rng.uniform(0.5, 2.0, target.shape) * 1e-6
    v0 = np.full(target.shape, 2000.0)
    fun = quadratic(target, weights)
    if driver == "lbfgs":
        out = fwi.lbfgs(fun, v0, 1000.0, 3000.0, iters=40)
        assert np.allclose(out["vel"], np.clip(target, 1000.0, 3000.0), atol=1.0)
    else:
        out = fwi.gradient_descent(fun, v0, 1000.0, 3000.0, iters=60, first_step=0.2)
        assert out["misfit"][-1] < 0.05 * out["misfit"][0]
    assert all(b <= a + 1e-12 for a, b in zip(out["misfit"][1:], out["misfit"][2:]))


def small_problem():
    nz, nx, nt = 40, 48, 420
    cfg = dict(ndim=2, nz=nz, ny=1, nx=nx, h=10.0, dt=1e-3, nt=nt, bc="sponge", nb=[8, 8, 0, 0, 8, 8],
               free_surface=0, R=1e-3, f_ref=15.0, snap_every=0, snap_begin=0, snap_end=0)
    z, x = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    v_true = 2000.0 + 250.0 * np.exp(-((z - 22) ** 2 + (x - 16) ** 2) / 30.0) \
        - 200.0 * np.exp(-((z - 18) ** 2 + (x - 34) ** 2) / 25.0)
    v0 = np.full((nz, nx), 2000.0)
    w = synth.ricker(15.0, 0.07, 1e-3, nt).astype(np.float64)
    src = np.array([[60.0, 20.0], [240.0, 20.0], [420.0, 20.0]])
    rec = synth.line(0.0, 470.0, 48, 20.0)
    d = [oracle.forward(cfg, v_true, w, src=s, rec=rec)["gather"] for s in src]
    return cfg, v_true, v0, w, src, rec, d


def oracle_objective(cfg, w, src, rec, d):
    def fun(v):
        J, g = 0.0, np.zeros(v.shape)
        for s, dk in zip(src, d):
            o = oracle.gradient(cfg, v, w, s, rec, dk)
            J += float(o["misfit"])
            g += o["grad"]
        return J, g
    return fun


@pytest.mark.parametrize("driver", ["lbfgs", "gd"])
def test_drivers_on_the_oracle_gradient(driver):
    cfg, v_true, v0, w, src, rec, d = small_problem()
    fun = oracle_objective(cfg, w, src, rec, d)
    if driver == "lbfgs":
        out = fwi.lbfgs(fun, v0, 1700.0, 2400.0, iters=5)
    else:
        out = fwi.gradient_descent(fun, v0, 1700.0, 2400.0, iters=5)
    J = out["misfit"]
    assert J[-1] <= 0.5 * J[0], J
    if driver == "gd":
        assert all(b <= a for a, b in zip(J, J[1:])), J
    v = out["vel"]
    assert v.min() >= 1700.0 and v.max() <= 2400.0
    assert np.linalg.norm(v - v_true) < np.linalg.norm(v0 - v_true)


@pytest.mark.gpu
def test_lbfgs_on_c4_with_fp16_checkpoints():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2605_30541_gb300 as pkg
    c = synth.config_c4()
    ns, nrec = len(c["src"]), len(c["rec"])
    true = pkg.Simulator(c, c["vel_true"], max_shots=ns, max_rec=nrec)
    d = true.forward(c["wavelet"], c["src"], c["rec"])["gather"].clone()
    true.close()
    sim = pkg.Simulator(c, c["vel"], max_shots=ns, max_rec=nrec)
    fun = fwi.sim_objective(sim, c["wavelet"], c["src"], c["rec"], d, ckpt_fp16=True)
    v0 = c["vel"].astype(np.float64)
    out = fwi.lbfgs(fun, v0, 1500.0, 5000.0, iters=6)
    sim.close()
    J = out["misfit"]
    assert J[-1] < 0.6 * J[0], J
    vt = c["vel_true"].astype(np.float64)
    assert np.linalg.norm(out["vel"] - vt) < np.linalg.norm(v0 - vt)
