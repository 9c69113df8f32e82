"""Checkpoint schedules, the vector-Jacobian product and the batched gradient,
through the C ABI.

- A device-memory budget (sim_desc.adj_budget) too small for sqrt(nt)
  checkpoints makes sim_adjoint choose two checkpoint levels (three forward
  sweeps). With FP32 storage every restored state is exact, so the gradient
  must equal the one-level gradient bit for bit (2D and 3D, sponge and CPML
  with its memory checkpointed on the strips only); with FP16 storage it must
  stay within 1e-2 of the FP64 oracle.
- sim_adjoint_vjp with a cotangent 1e-6 times the size of the gathers against
  the oracle's gradient of <cot, g> (FP32 tolerance 1e-4).
- The gradient mode of the batch (sim_batch_ex mode 1) on uneven slices with
  several shots each: per-slice FP64 sums against the oracle (FP32 storage
  1e-4, FP16 1e-2) and the per-slice misfits."""
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


def case2d(bc, fs, nt=500, nshots=2):
    nz, nx = 48, 70
    vt = synth.procedural_2d(nz, nx, 10.0, 4001)
    v0 = synth.smooth(vt, 5.0)
    cfg = dict(ndim=2, nz=nz, ny=1, nx=nx, h=10.0, dt=1e-3, nt=nt, bc=bc, nb=[0 if fs else 12, 12, 0, 0, 12, 12],
               free_surface=fs)
    w = synth.ricker(15.0, 0.07, 1e-3, nt)
    src = np.stack([np.linspace(105.0, 585.0, nshots), np.full(nshots, 20.0)], axis=1)
    rec = synth.line(0.0, 690.0, 70, 10.0 if fs else 20.0)
    d = np.stack([oracle.forward(cfg, vt.astype(np.float64), w.astype(np.float64), src=s, rec=rec)["gather"]
                  for s in src])
    return cfg, v0, w, src, rec, d


def case3d(bc, fs, nt=150):
    nz, ny, nx, nb = 20, 18, 40, 6
    cfg = dict(ndim=3, nz=nz, ny=ny, nx=nx, h=10.0, dt=8e-4, nt=nt, bc=bc,
               nb=[0 if fs else nb, nb, nb, nb, nb, nb], free_surface=fs, R=1e-3, f_ref=15.0)
    vt = synth.procedural_3d(nz, ny, nx, 10.0, 41)
    v0 = np.asarray(synth.smooth(vt, 20.0), np.float32)
    w = synth.ricker(15.0, 0.06, 8e-4, nt)
    src = np.array([[55.0, 45.0, 20.0], [160.0, 120.0, 20.0]])
    rec = np.array([[10.0 * i + 3.0, 10.0 * j + 1.0, 10.0 if fs else 30.0] for i in range(0, nx - 1, 4)
                    for j in range(0, 17, 4)])
    d = np.stack([oracle.forward(cfg, vt.astype(np.float64), w.astype(np.float64), src=s, rec=rec)["gather"]
                  for s in src])
    return cfg, v0, w, src, rec, d


def oracle_grad(cfg, v0, w, src, rec, d):
    tot, J = np.zeros(v0.shape), 0.0
    for k in range(len(src)):
        o = oracle.gradient(cfg, v0.astype(np.float64), w.astype(np.float64), src[k], rec, d[k])
        tot += o["grad"]
        J += o["misfit"]
    return tot, J


def run_grad(pkg, cfg, v0, w, src, rec, d, fp16, budget=0):
    sim = pkg.Simulator(cfg, v0, max_shots=len(src), max_rec=len(rec), adj_budget=budget)
    grad = torch.zeros(v0.shape, device="cuda")
    mis = np.zeros(1)
    pkg.sim_adjoint(sim.handle, len(src), torch.as_tensor(w, device="cuda"), np.ascontiguousarray(src), len(rec),
                    np.ascontiguousarray(rec), torch.as_tensor(np.ascontiguousarray(d), dtype=torch.float32,
                                                               device="cuda"), None, mis, fp16, grad)
    sim.sync()
    info = pkg.sim_get_info(sim.handle)
    out = grad.cpu().numpy()
    sim.close()
    return out, float(mis[0]), info


def two_level(pkg, args, fp16):
    """The gradient under the largest budget (a fraction of the one-level
    plan's bytes) that makes the plan take two levels."""
    g1, J1, i1 = run_grad(pkg, *args, fp16)
    assert i1.adj_levels == 1
    for frac in (0.8, 0.7, 0.6, 0.5, 0.4, 0.3):
        try:
            g2, J2, i2 = run_grad(pkg, *args, fp16, budget=int(frac * i1.adj_bytes))
        except pkg.SimError as e:
            assert e.code == pkg.abi.SIM_ERR_OOM
            continue
        if i2.adj_levels == 2:
            assert i2.adj_bytes <= frac * i1.adj_bytes
            assert i2.adj_top * i2.adj_inner * i2.adj_slots >= args[0]["nt"]
            return (g1, J1, i1), (g2, J2, i2)
    raise AssertionError("no budget gave a two-level plan")


@pytest.mark.parametrize("bc,fs", [("sponge", 1), ("cpml", 0), ("cpml", 1)])
def test_two_level_checkpoints_2d(pkg, bc, fs):
    args = case2d(bc, fs)
    (g1, J1, _), (g2, J2, i2) = two_level(pkg, args, 0)
    assert np.array_equal(g1, g2)
    assert J1 == J2
    ref, Jref = oracle_grad(*args)
    assert rel(g2, ref) <= 1e-4
    (h1, _, _), (h2, _, _) = two_level(pkg, args, 1)
    assert rel(h2, ref) <= 1e-2
    assert rel(h1, ref) <= 1e-2


@pytest.mark.parametrize("bc,fs", [("sponge", 1), ("cpml", 0)])
def test_two_level_checkpoints_3d(pkg, bc, fs):
    args = case3d(bc, fs)
    (g1, J1, _), (g2, J2, _) = two_level(pkg, args, 0)
    assert np.array_equal(g1, g2)
    assert J1 == J2
    ref, _ = oracle_grad(*args)
    assert rel(g2, ref) <= 1e-4
    (_, _, _), (h2, _, _) = two_level(pkg, args, 1)
    assert rel(h2, ref) <= 1e-2


def test_fp32_storage_after_fp16_replans(pkg):
    # buffers sized for FP16 storage are re-planned when FP32 storage is asked
    # for; the FP32 result equals a fresh handle's
    cfg, v0, w, src, rec, d = case2d("cpml", 1, nt=300)
    sim = pkg.Simulator(cfg, v0, max_shots=len(src), max_rec=len(rec))
    args = (len(src), torch.as_tensor(w, device="cuda"), np.ascontiguousarray(src), len(rec), np.ascontiguousarray(rec),
            torch.as_tensor(np.ascontiguousarray(d), dtype=torch.float32, device="cuda"), None, None)
    g16 = torch.zeros(v0.shape, device="cuda")
    pkg.sim_adjoint(sim.handle, *args, 1, g16)
    b16 = pkg.sim_get_info(sim.handle).adj_bytes
    g32 = torch.zeros(v0.shape, device="cuda")
    pkg.sim_adjoint(sim.handle, *args, 0, g32)
    b32 = pkg.sim_get_info(sim.handle).adj_bytes
    sim.close()
    assert b32 > b16
    fresh, _, _ = run_grad(pkg, cfg, v0, w, src, rec, d, 0)
    assert np.array_equal(g32.cpu().numpy(), fresh)


@pytest.mark.parametrize("ndim", [2, 3])
def test_vjp_with_a_small_cotangent(pkg, ndim):
    cfg, v0, w, src, rec, _ = case2d("cpml", 1, nt=400) if ndim == 2 else case3d("cpml", 0, nt=120)
    g = np.stack([oracle.forward(cfg, v0.astype(np.float64), w.astype(np.float64), src=s, rec=rec)["gather"]
                  for s in src])
    cot = np.random.default_rng(77).standard_normal(g.shape) * np.abs(g).max() * 1e-6
    ref, _ = oracle_grad(cfg, v0, w, src, rec, g - cot)   # J = 1/2 |g - (g - cot)|^2: gradient J^T cot
    sim = pkg.Simulator(cfg, v0, max_shots=len(src), max_rec=len(rec))
    grad = torch.zeros(v0.shape, device="cuda")
    pkg.sim_adjoint_vjp(sim.handle, len(src), torch.as_tensor(w, device="cuda"), np.ascontiguousarray(src), len(rec),
                        np.ascontiguousarray(rec), torch.as_tensor(cot, dtype=torch.float32, device="cuda"), None, 0,
                        grad)
    sim.sync()
    sim.close()
    assert rel(grad.cpu().numpy(), ref) <= 1e-4


def test_autograd_backward_with_a_small_cotangent(pkg):
    from paper_2605_30541_gb300.autograd import gathers
    cfg, v0, w, src, rec, _ = case2d("sponge", 1, nt=300)
    sim = pkg.Simulator(cfg, v0, max_shots=len(src), max_rec=len(rec))
    v = torch.as_tensor(v0, device="cuda").requires_grad_(True)
    out = gathers(v, sim, torch.as_tensor(w), src, rec)
    g64 = np.stack([oracle.forward(cfg, v0.astype(np.float64), w.astype(np.float64), src=s, rec=rec)["gather"]
                    for s in src])
    cot = np.random.default_rng(78).standard_normal(g64.shape) * np.abs(g64).max() * 1e-6
    (out * torch.as_tensor(cot, dtype=torch.float32, device="cuda")).sum().backward()
    ref, _ = oracle_grad(cfg, v0, w, src, rec, g64 - cot)
    sim.close()
    assert rel(v.grad.cpu().numpy(), ref) <= 1e-4


def uneven_slices(nt=400):
    """Three slices of uneven size with 3, 2 and 4 shots (CPML, free top)."""
    out = []
    for j, (nz, nx, ns) in enumerate([(40, 64, 3), (52, 90, 2), (34, 76, 4)]):
        vt = synth.procedural_2d(nz, nx, 10.0, 3100 + j)
        # a start model far enough from the truth that g - d is far above the
        # FP32 rounding of g (else the residual itself carries that rounding)
        v0 = (0.95 * synth.smooth(vt, 4.0)).astype(np.float32)
        cfg = dict(ndim=2, nz=nz, ny=1, nx=nx, h=10.0, dt=1e-3, nt=nt, bc="cpml", nb=[0, 10, 0, 0, 10, 10],
                   free_surface=1, f_ref=15.0)
        w = synth.ricker(15.0, 0.07, 1e-3, nt)
        src = np.stack([np.linspace(40.0, (nx - 5) * 10.0, ns), np.full(ns, 10.0)], axis=1)
        rec = synth.line(0.0, (nx - 1) * 10.0, nx // 2, 10.0)
        d = np.stack([oracle.forward(cfg, vt.astype(np.float64), w.astype(np.float64), src=s, rec=rec)["gather"]
                      for s in src])
        out.append((cfg, v0, w, src, rec, d))
    return out


def test_batch_gradient_on_uneven_slices(pkg):
    sl = uneven_slices()
    refs = [oracle_grad(*c) for c in sl]
    for fp16, tol in ((0, 1e-4), (1, 1e-2)):
        sims = [pkg.Simulator(c[0], c[1], max_shots=len(c[3]), max_rec=len(c[4])) for c in sl]
        entries = [dict(sim=s, wavelet=c[2], src=c[3], rec=c[4], d_obs=c[5]) for s, c in zip(sims, sl)]
        grads, mis = pkg.batch_gradient(entries, ckpt_fp16=fp16)
        torch.cuda.synchronize()
        for (ref, Jref), g, J in zip(refs, grads, mis):
            assert g.dtype == torch.float64
            assert rel(g.cpu().numpy(), ref) <= tol
            assert abs(J - Jref) <= 1e-4 * Jref
        # accumulation: a second call adds the same gradient again
        g1 = [g.clone() for g in grads]
        pkg.batch_gradient([dict(e, grad=g) for e, g in zip(entries, grads)], ckpt_fp16=fp16)
        torch.cuda.synchronize()
        for a, b in zip(g1, grads):
            assert torch.allclose(b, 2 * a, rtol=1e-12, atol=0)
        for s in sims:
            s.close()
