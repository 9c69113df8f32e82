"""Full-waveform inversion as a host loop over the adjoint-state gradient.

Each evaluation sets a velocity model on a handle and calls sim_adjoint,
which returns the L2 data misfit J = 1/2 sum_shots ||g - d||^2 and its
gradient with respect to the interior velocity (the outer iteration of the
paper's FWI use of the data; all per-step work stays in the library's
kernels). Two drivers work on any objective `fun(v) -> (J, dJ/dv)` of numpy
arrays:

  lbfgs            limited-memory BFGS within velocity bounds (scipy's
                   L-BFGS-B), on the model scaled by its mean so the
                   quasi-Newton metric starts near unit scale;
  gradient_descent projected steepest descent, each step chosen by Armijo
                   backtracking (halving from a first step that moves the
                   fastest cell by `first_step` of the mean velocity).

`sim_objective` binds the objective to a Simulator (FP32 or FP64 handle,
optional FP16 checkpoints). Velocities outside [vmin, vmax] are never
evaluated: both drivers project onto the bounds, which the caller picks
inside the handle's stability range (sim_plan).
"""
import numpy as np

from . import sim_adjoint


def sim_objective(sim, wavelet, src, rec, d_obs, ckpt_fp16=False):
    """Objective v -> (J, dJ/dv) on `sim`'s device: d_obs [nshots, nt, nrec]."""
    import torch
    d = sim.desc
    src = np.ascontiguousarray(np.asarray(src, np.float64).reshape(-1, d.ndim))
    rec = np.ascontiguousarray(np.asarray(rec, np.float64).reshape(-1, d.ndim))
    w = sim._tensor(wavelet)
    dd = sim._tensor(d_obs)
    shape = sim.interior_shape

    def fun(v):
        vt = sim._tensor(np.asarray(v).reshape(shape))
        sim.set_model(vt)
        grad = torch.zeros_like(vt)
        mis = np.zeros(1)
        sim_adjoint(sim.handle, src.shape[0], w, src, rec.shape[0], rec, dd, None, mis, int(ckpt_fp16), grad)
        sim.sync()
        return float(mis[0]), grad.cpu().numpy().astype(np.float64)

    return fun


def lbfgs(fun, v0, vmin, vmax, iters=10, history=8, callback=None):
    """L-BFGS-B on the velocity, bounded by [vmin, vmax]. Returns a dict with
    the final model, the misfit per iteration (the first entry is J(v0)) and
    the number of objective evaluations."""
    from scipy.optimize import minimize
    v0 = np.asarray(v0, np.float64)
    scale = float(np.mean(v0))
    shape = v0.shape
    hist = []
    count = [0]

    def f(x):
        J, g = fun(x.reshape(shape) * scale)
        count[0] += 1
        return J, np.asarray(g, np.float64).ravel() * scale

    J0, _ = f(v0.ravel() / scale)
    hist.append(J0)

    def cb(xk):
        v = xk.reshape(shape) * scale
        if callback:
            callback(v)

    res = minimize(f, v0.ravel() / scale, jac=True, method="L-BFGS-B",
                   bounds=[(vmin / scale, vmax / scale)] * v0.size, callback=cb,
                   options={"maxiter": iters, "maxcor": history})
    v = res.x.reshape(shape) * scale
    hist.append(float(res.fun))
    return {"vel": v, "misfit": hist, "evaluations": count[0], "iterations": int(res.nit)}


def gradient_descent(fun, v0, vmin, vmax, iters=10, first_step=0.02, armijo=1e-4, max_halvings=12,
                     callback=None):
    """Projected steepest descent with Armijo backtracking. Returns the final
    model, the accepted misfits (first entry J(v0)) and the evaluation count."""
    v = np.clip(np.asarray(v0, np.float64), vmin, vmax)
    J, g = fun(v)
    hist, count = [J], 1
    vmean = float(np.mean(v))
    for _ in range(iters):
        gmax = float(np.max(np.abs(g)))
        if gmax == 0.0:
            break
        alpha = first_step * vmean / gmax
        accepted = False
        for _ in range(max_halvings):
            vn = np.clip(v - alpha * g, vmin, vmax)
            Jn, gn = fun(vn)
            count += 1
            # sufficient decrease along the projected step
            if Jn <= J - armijo * float(np.sum(g * (v - vn))):
                accepted = True
                break
            alpha *= 0.5
        if not accepted:
            break
        v, J, g = vn, Jn, gn
        hist.append(J)
        if callback:
            callback(v)
    return {"vel": v, "misfit": hist, "evaluations": count, "iterations": len(hist) - 1}
