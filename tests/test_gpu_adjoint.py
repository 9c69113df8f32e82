"""GPU adjoint-state gradient against the FP64 oracle, finite differences and
the FP64 dot-product test, all through the C ABI.

Tolerances (relative L2 over the interior): FP32 storage <= 1e-4, FP16-scaled
checkpoints and imaging terms <= 1e-2; FP64 dot test <= 1e-6 (sponge and
CPML)."""
import multiprocessing as mp
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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def small_case(fs=0, nt=500, nshots=2, bc="sponge"):
    nz, nx = 48, 70
    vel_true = synth.procedural_2d(nz, nx, 10.0, 4001)
    vel0 = synth.smooth(vel_true, 5.0)
    cfg = dict(ndim=2, nz=nz, ny=1, nx=nx, h=10.0, dt=1e-3, nt=nt, bc=bc, nb=[0 if fs else 12, 12, 0, 0, 12, 12],
               free_surface=fs)
    w = synth.ricker(15.0, 0.07, 1e-3, nt)
    src = np.stack([np.linspace(105.0, 585.0, nshots), np.full(nshots, 20.0)], axis=1)
    rec = synth.line(0.0, 690.0, 70, 20.0 if not fs else 10.0)
    return cfg, vel_true, vel0, w, src, rec


def oracle_grad(cfg, vel0, w, src, rec, d):
    tot = np.zeros(vel0.shape)
    J = 0.0
    for k in range(len(src)):
        o = oracle.gradient(cfg, vel0.astype(np.float64), w.astype(np.float64), src[k], rec, d[k])
        tot += o["grad"]
        J += o["misfit"]
    return tot, J


def gpu_grad(pkg, cfg, vel0, w, src, rec, d, fp16=0, precision=0):
    sim = pkg.Simulator(cfg, vel0, max_shots=len(src), max_rec=len(rec), precision=precision)
    dt = torch.float64 if precision else torch.float32
    grad = torch.zeros(vel0.shape, dtype=dt, device="cuda")
    mis = np.zeros(1)
    dd = torch.as_tensor(np.ascontiguousarray(d), dtype=dt, device="cuda")
    ww = torch.as_tensor(w, dtype=dt, device="cuda")
    pkg.sim_adjoint(sim.handle, len(src), ww, np.ascontiguousarray(src), len(rec), np.ascontiguousarray(rec), dd,
                    None, mis, fp16, grad)
    sim.sync()
    out = grad.cpu().numpy().astype(np.float64)
    sim.close()
    return out, float(mis[0])


def observed(cfg, vel_true, w, src, rec):
    return np.stack([oracle.forward(cfg, vel_true.astype(np.float64), w.astype(np.float64), src=s, rec=rec)["gather"]
                     for s in src])


@pytest.mark.parametrize("fs", [0, 1])
def test_gradient_fp32_matches_oracle(pkg, fs):
    cfg, vt, v0, w, src, rec = small_case(fs=fs)
    d = observed(cfg, vt, w, src, rec)
    ref, Jref = oracle_grad(cfg, v0, w, src, rec, d)
    g, J = gpu_grad(pkg, cfg, v0, w, src, rec, d)
    # J sums squared differences of nearly equal gathers, so the FP32 rounding of
    # g is amplified by |g| / |g - d|: 1e-4 bounds it; the gradient keeps 1e-4
    assert abs(J - Jref) <= 1e-4 * Jref
    assert rel(g, ref) <= 1e-4


def test_gradient_fp16_checkpoints_within_1e2(pkg):
    cfg, vt, v0, w, src, rec = small_case(nt=700)
    d = observed(cfg, vt, w, src, rec)
    ref, _ = oracle_grad(cfg, v0, w, src, rec, d)
    g16, _ = gpu_grad(pkg, cfg, v0, w, src, rec, d, fp16=1)
    g32, _ = gpu_grad(pkg, cfg, v0, w, src, rec, d, fp16=0)
    e16, e32 = rel(g16, ref), rel(g32, ref)
    assert e32 <= 1e-4
    assert e16 <= 1e-2
    assert e16 > e32   # the FP16 path really stores half-precision states


def test_gradient_fp64_matches_oracle_and_finite_differences(pkg):
    cfg, vt, v0, w, src, rec = small_case(nt=300, nshots=1)
    d = observed(cfg, vt, w, src, rec)
    ref, _ = oracle_grad(cfg, v0, w, src, rec, d)
    g, J = gpu_grad(pkg, cfg, v0.astype(np.float64), w, src, rec, d, precision=1)
    assert rel(g, ref) <= 1e-10
    sim = pkg.Simulator(cfg, v0.astype(np.float64), max_shots=1, max_rec=len(rec), precision=1)
    rng = np.random.default_rng(4000)

    def misfit(v):
        sim.set_model(v)
        out = sim.forward(w.astype(np.float64), src, rec)["gather"].cpu().numpy()
        return 0.5 * np.sum((out - d) ** 2)
    for _ in range(10):
        iz, ix = rng.integers(0, v0.shape[0]), rng.integers(0, v0.shape[1])
        e = 1e-4 * v0[iz, ix]
        vp = v0.astype(np.float64).copy()
        vm = vp.copy()
        vp[iz, ix] += e
        vm[iz, ix] -= e
        fd = (misfit(vp) - misfit(vm)) / (2 * e)
        assert abs(fd - g[iz, ix]) <= 1e-6 * np.abs(g).max() + 1e-6 * abs(g[iz, ix])
    sim.close()


def test_dot_product_fp64_born(pkg):
    # <J dv, dd> = <dv, J^T dd>: J dv by central differences of the FP64 forward
    # (error O(eps^2) ~ 1e-10), J^T dd by sim_adjoint with residual dd
    cfg, vt, v0, w, src, rec = small_case(nt=300, nshots=1, fs=1)
    v0 = v0.astype(np.float64)
    rng = np.random.default_rng(31)
    dv = rng.standard_normal(v0.shape)
    sim = pkg.Simulator(cfg, v0, max_shots=1, max_rec=len(rec), precision=1)
    eps = 1e-5 * np.abs(v0).mean() / np.abs(dv).max()

    def fwd(v):
        sim.set_model(v)
        return sim.forward(w.astype(np.float64), src, rec)["gather"].cpu().numpy()[0]
    g0 = fwd(v0)
    Jdv = (fwd(v0 + eps * dv) - fwd(v0 - eps * dv)) / (2 * eps)
    dd = rng.standard_normal(g0.shape) * np.abs(g0).max()
    grad = torch.zeros(v0.shape, dtype=torch.float64, device="cuda")
    sim.set_model(v0)
    pkg.sim_adjoint(sim.handle, 1, torch.as_tensor(w, dtype=torch.float64, device="cuda"), np.ascontiguousarray(src),
                    len(rec), np.ascontiguousarray(rec),
                    torch.as_tensor((g0 - dd)[None], device="cuda"), None, None, 0, grad)
    JTdd = grad.cpu().numpy()
    lhs, rhs = np.vdot(Jdv, dd), np.vdot(dv, JTdd)
    assert abs(lhs - rhs) / (np.linalg.norm(Jdv) * np.linalg.norm(dd)) <= 1e-6
    sim.close()


def test_autograd_function_matches_oracle_and_vjp(pkg):
    # the backward pass is sim_adjoint_vjp driven by the cotangent g - d of
    # the loss 1/2 |g - d|^2: the oracle's gradient within the FP32 bar, and
    # the entry point called directly with the same cotangent, bit for bit
    from paper_2605_30541_gb300.autograd import gathers
    cfg, vt, v0, w, src, rec = small_case(nt=300)
    d = observed(cfg, vt, w, src, rec)
    sim = pkg.Simulator(cfg, v0, max_shots=len(src), max_rec=len(rec))
    v = torch.as_tensor(v0, device="cuda").requires_grad_(True)
    g = gathers(v, sim, torch.as_tensor(w), src, rec)
    loss = 0.5 * ((g.double() - torch.as_tensor(d, device="cuda")) ** 2).sum()
    loss.backward()
    ref, Jref = oracle_grad(cfg, v0, w, src, rec, d)
    assert rel(v.grad.cpu().numpy(), ref) <= 1e-4
    assert abs(loss.item() - Jref) <= 1e-4 * Jref
    cot = (g.detach().double() - torch.as_tensor(d, device="cuda")).float().contiguous()
    direct = torch.zeros(v0.shape, device="cuda")
    pkg.sim_adjoint_vjp(sim.handle, len(src), torch.as_tensor(w, device="cuda"), np.ascontiguousarray(src), len(rec),
                        np.ascontiguousarray(rec), cot, None, 0, direct)
    sim.sync()
    assert torch.equal(direct, v.grad)
    sim.close()


def test_gradient_accumulates(pkg):
    cfg, vt, v0, w, src, rec = small_case(nt=200, nshots=1)
    d = observed(cfg, vt, w, src, rec)
    sim = pkg.Simulator(cfg, v0, max_shots=1, max_rec=len(rec))
    grad = torch.zeros(v0.shape, dtype=torch.float32, device="cuda")
    args = (1, torch.as_tensor(w, device="cuda"), np.ascontiguousarray(src), len(rec), np.ascontiguousarray(rec),
            torch.as_tensor(d, dtype=torch.float32, device="cuda"), None, None, 0, grad)
    pkg.sim_adjoint(sim.handle, *args)
    once = grad.clone()
    pkg.sim_adjoint(sim.handle, *args)
    assert torch.allclose(grad, 2 * once, rtol=1e-6, atol=0)
    sim.close()


@pytest.mark.parametrize("fs", [0, 1])
def test_cpml_gradient_fp32_matches_oracle(pkg, fs):
    # the exact transpose of the CPML recursions, FP32 storage
    cfg, vt, v0, w, src, rec = small_case(fs=fs, bc="cpml")
    d = observed(cfg, vt, w, src, rec)
    ref, Jref = oracle_grad(cfg, v0, w, src, rec, d)
    g, J = gpu_grad(pkg, cfg, v0, w, src, rec, d)
    assert abs(J - Jref) <= 1e-4 * Jref
    assert rel(g, ref) <= 1e-4


def test_cpml_gradient_fp16_checkpoints_within_1e2(pkg):
    cfg, vt, v0, w, src, rec = small_case(nt=700, bc="cpml")
    d = observed(cfg, vt, w, src, rec)
    ref, _ = oracle_grad(cfg, v0, w, src, rec, d)
    g16, _ = gpu_grad(pkg, cfg, v0, w, src, rec, d, fp16=1)
    assert rel(g16, ref) <= 1e-2


def test_cpml_gradient_fp64_matches_oracle_and_finite_differences(pkg):
    # the transposed CPML recursions in FP64: the oracle's gradient to 1e-10
    # and central differences of the FP64 misfit on 10 cells
    cfg, vt, v0, w, src, rec = small_case(nt=300, nshots=1, bc="cpml")
    d = observed(cfg, vt, w, src, rec)
    ref, _ = oracle_grad(cfg, v0, w, src, rec, d)
    g, _ = gpu_grad(pkg, cfg, v0.astype(np.float64), w, src, rec, d, precision=1)
    assert rel(g, ref) <= 1e-10
    sim = pkg.Simulator(cfg, v0.astype(np.float64), max_shots=1, max_rec=len(rec), precision=1)
    rng = np.random.default_rng(4100)
    vmax = float(v0.max())

    def misfit(v):
        sim.set_model(v)
        out = sim.forward(w.astype(np.float64), src, rec)["gather"].cpu().numpy()
        return 0.5 * np.sum((out - d) ** 2)
    done = 0
    while done < 10:
        # the CPML coefficients follow the model's maximum velocity at set-up
        # and are constants of the differentiated map: keep the maximum
        iz, ix = rng.integers(0, v0.shape[0]), rng.integers(0, v0.shape[1])
        e = 1e-4 * v0[iz, ix]
        if v0[iz, ix] + 2 * e >= vmax:
            continue
        done += 1
        vp = v0.astype(np.float64).copy()
        vm = vp.copy()
        vp[iz, ix] += e
        vm[iz, ix] -= e
        fd = (misfit(vp) - misfit(vm)) / (2 * e)
        assert abs(fd - g[iz, ix]) <= 1e-6 * np.abs(g).max() + 1e-6 * abs(g[iz, ix])
    sim.close()


@pytest.mark.parametrize("fs", [0, 1])
def test_dot_product_fp64_born_cpml(pkg, fs):
    # <J dv, dd> = <dv, J^T dd> with CPML (the CPML coefficients held fixed,
    # as in the forward map): J dv by central differences of the FP64 forward
    cfg, vt, v0, w, src, rec = small_case(nt=300, nshots=1, fs=fs, bc="cpml")
    v0 = v0.astype(np.float64)
    rng = np.random.default_rng(32 + fs)
    dv = rng.standard_normal(v0.shape)
    dv[v0 >= v0.max() - 1.0] = 0.0  # the model maximum (which sets the CPML coefficients) stays put
    sim = pkg.Simulator(cfg, v0, max_shots=1, max_rec=len(rec), precision=1)
    eps = 1e-5 * np.abs(v0).mean() / np.abs(dv).max()

    def fwd(v):
        sim.set_model(v)
        return sim.forward(w.astype(np.float64), src, rec)["gather"].cpu().numpy()[0]
    g0 = fwd(v0)
    Jdv = (fwd(v0 + eps * dv) - fwd(v0 - eps * dv)) / (2 * eps)
    dd = rng.standard_normal(g0.shape) * np.abs(g0).max()
    grad = torch.zeros(v0.shape, dtype=torch.float64, device="cuda")
    sim.set_model(v0)
    pkg.sim_adjoint(sim.handle, 1, torch.as_tensor(w, dtype=torch.float64, device="cuda"), np.ascontiguousarray(src),
                    len(rec), np.ascontiguousarray(rec),
                    torch.as_tensor((g0 - dd)[None], device="cuda"), None, None, 0, grad)
    JTdd = grad.cpu().numpy()
    lhs, rhs = np.vdot(Jdv, dd), np.vdot(dv, JTdd)
    assert abs(lhs - rhs) / (np.linalg.norm(Jdv) * np.linalg.norm(dd)) <= 1e-6
    sim.close()


def _oracle_shot(args):
    cfg, v0, w, s, rec, d = args
    o = oracle.gradient(cfg, v0, w, s, rec, d)
    return o["grad"], o["misfit"]


def test_c4_full_gradient_16_shots(pkg):
    # the FWI-gradient workload: 201 x 201 procedural model, 16 shots, 4 s records
    c = synth.config_c4()
    w64 = c["wavelet"].astype(np.float64)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, mp.cpu_count()), initializer=_one_thread) as pool:
        d = np.stack(pool.map(_fwd_shot, [(c, c["vel_true"].astype(np.float64), w64, s, c["rec"]) for s in c["src"]]))
        outs = pool.map(_oracle_shot, [(c, c["vel"].astype(np.float64), w64, s, c["rec"], d[k])
                                       for k, s in enumerate(c["src"])])
    ref = sum(o[0] for o in outs)
    Jref = sum(o[1] for o in outs)
    g32, J = gpu_grad(pkg, c, c["vel"], c["wavelet"], c["src"], c["rec"], d, fp16=0)
    g16, _ = gpu_grad(pkg, c, c["vel"], c["wavelet"], c["src"], c["rec"], d, fp16=1)
    assert abs(J - Jref) <= 1e-4 * Jref
    assert rel(g32, ref) <= 1e-4
    assert rel(g16, ref) <= 1e-2


def _one_thread():
    os.environ["OMP_NUM_THREADS"] = "1"


def _fwd_shot(args):
    cfg, v, w, s, rec = args
    return oracle.forward(cfg, v, w, src=s, rec=rec)["gather"]
