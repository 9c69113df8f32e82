"""3D adjoint-state gradient (sim_adjoint on a 3D handle: z-march in record /
adjoint modes, cell-grouped point injection, sqrt(nt) checkpoints; sponge and
CPML, whose transposed recursions run after each update of the sweep) against
the FP64 oracle gradient, summed over shots: relative L2 <= 1e-4 with FP32
checkpoints (the FP32 tolerance of the 2D gradient tests), <= 1e-2 with FP16
checkpoints; misfit to 1e-4."""
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


def case(fs, nt=150, bc="sponge", nx=22):
    nz, ny, nb = 20, 18, 6
    cfg = dict(ndim=3, nz=nz, ny=ny, nx=nx, h=10.0, dt=8e-4, nt=nt, bc=bc,
               nb=[0 if fs else nb, nb, nb, nb, nb, nb], free_surface=fs, R=1e-3, f_ref=15.0)
    vel_true = synth.procedural_3d(nz, ny, nx, 10.0, 41)
    vel0 = np.asarray(synth.smooth(vel_true, 20.0), np.float32)
    w = synth.ricker(15.0, 0.06, 8e-4, nt)
    srcs = np.array([[55.0, 45.0, 20.0], [160.0, 120.0, 20.0]])
    rec = np.array([[10.0 * i + 3.0, 10.0 * j + 1.0, 10.0 if fs else 30.0] for i in range(0, nx - 1, 4)
                    for j in range(0, 17, 4)])
    d = np.stack([oracle.forward(cfg, vel_true.astype(np.float64), w.astype(np.float64), src=s, rec=rec)["gather"]
                  for s in srcs])
    return cfg, vel0, w, srcs, rec, d


def gpu_grad(pkg, cfg, vel0, w, srcs, rec, d, fp16):
    sim = pkg.Simulator(cfg, vel0, max_shots=len(srcs), max_rec=len(rec))
    grad = torch.zeros(vel0.shape, device="cuda")
    mis = np.zeros(1)
    pkg.sim_adjoint(sim.handle, len(srcs), torch.as_tensor(w, device="cuda"), np.ascontiguousarray(srcs), len(rec),
                    np.ascontiguousarray(rec), torch.as_tensor(np.ascontiguousarray(d), dtype=torch.float32,
                                                               device="cuda"), None, mis, fp16, grad)
    sim.sync()
    out = grad.cpu().numpy().astype(np.float64)
    sim.close()
    return out, float(mis[0])


@pytest.mark.parametrize("fs", [0, 1])
def test_gradient_matches_oracle(pkg, fs):
    cfg, vel0, w, srcs, rec, d = case(fs)
    ref = np.zeros(vel0.shape)
    Jref = 0.0
    for k, s in enumerate(srcs):
        o = oracle.gradient(cfg, vel0.astype(np.float64), w.astype(np.float64), s, rec, d[k])
        ref += o["grad"]
        Jref += o["misfit"]
    g32, J = gpu_grad(pkg, cfg, vel0, w, srcs, rec, d, 0)
    assert abs(J - Jref) <= 1e-4 * Jref
    assert rel(g32, ref) <= 1e-4
    g16, _ = gpu_grad(pkg, cfg, vel0, w, srcs, rec, d, 1)
    assert rel(g16, ref) <= 1e-2


@pytest.mark.parametrize("fs,nx", [(0, 22), (1, 40)])
def test_cpml_gradient_matches_oracle(pkg, fs, nx):
    # the transposed CPML recursions of all three axes after each update of
    # the sweep, the addend in the recorded imaging term, psi / zeta in every
    # checkpoint; nx = 22 takes the two-kernel x-strip path of the forward
    # passes (strip ends close together), nx = 40 the half-warp pass
    cfg, vel0, w, srcs, rec, d = case(fs, bc="cpml", nx=nx)
    ref = np.zeros(vel0.shape)
    Jref = 0.0
    for k, s in enumerate(srcs):
        o = oracle.gradient(cfg, vel0.astype(np.float64), w.astype(np.float64), s, rec, d[k])
        ref += o["grad"]
        Jref += o["misfit"]
    g32, J = gpu_grad(pkg, cfg, vel0, w, srcs, rec, d, 0)
    assert abs(J - Jref) <= 1e-4 * Jref
    assert rel(g32, ref) <= 1e-4
    g16, _ = gpu_grad(pkg, cfg, vel0, w, srcs, rec, d, 1)
    assert rel(g16, ref) <= 1e-2
