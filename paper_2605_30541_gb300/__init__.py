"""GB300 acoustic FDTD library: Python binding of libsim's C ABI.

The functions below carry the C entry points' names (include/sim.h) and only
marshal arguments: torch tensors and numpy arrays become device or host
pointers, problem dicts become ``sim_desc``. Every step of the solver runs in
the CUDA kernels of libsim.so; if that library is missing, or a call fails,
an exception is raised — there is no fallback.
"""
import ctypes
import warnings

import numpy as np

from . import abi
from .abi import SIM_BC, SIM_FP32, SIM_FP64, SimBatchItem, SimDesc, SimInfo

__all__ = ["SimError", "make_desc", "sim_plan", "sim_create", "sim_set_model", "sim_forward",
           "sim_adjoint", "sim_adjoint_vjp", "sim_batch", "sim_batch_ex", "batch_gradient", "sim_sync", "sim_get_info", "sim_last_error", "sim_destroy",
           "Simulator", "batch", "sim_forward_noalloc", "sim_wavelet_bandpass", "bandpass_ricker",
           "sim_model_squish", "sim_model_fault", "sim_model_deposit"]


class SimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (abi.STATUS_NAMES.get(code, code), msg))
        self.code = code


def _check(code, handle=None):
    if code == abi.SIM_OK:
        return
    msg = abi.load().sim_last_error(handle).decode()
    if code == abi.SIM_WARN_DISPERSION:
        warnings.warn(msg)
        return
    raise SimError(code, msg)


def make_desc(cfg, max_shots=1, max_rec=0, precision=SIM_FP32, snap_fp16=False, f_max=0.0,
              skip_cfl_check=False, adj_budget=0):
    """sim_desc from a problem dict (keys as produced by ``synth``);
    adj_budget: device bytes the gradient's buffers may take (0: automatic)."""
    d = SimDesc()
    abi.load().sim_desc_init(ctypes.byref(d))
    d.ndim = int(cfg["ndim"])
    d.nz, d.ny, d.nx = int(cfg["nz"]), int(cfg.get("ny", 1)), int(cfg["nx"])
    d.h, d.dt, d.nt = float(cfg["h"]), float(cfg["dt"]), int(cfg["nt"])
    bc = cfg.get("bc", "sponge")
    d.bc = SIM_BC[bc] if isinstance(bc, str) else int(bc)
    for k, v in enumerate(cfg.get("nb", [0] * 6)):
        d.nb[k] = int(v)
    d.free_surface = int(cfg.get("free_surface", 0))
    d.R = float(cfg.get("R", 1e-3))
    d.f_ref = float(cfg.get("f_ref", 10.0))
    d.f_max = float(f_max)
    d.snap_every = int(cfg.get("snap_every", 0))
    d.snap_begin = int(cfg.get("snap_begin", 0))
    d.snap_end = int(cfg.get("snap_end", 0))
    d.snap_fp16 = int(bool(snap_fp16))
    d.max_shots = int(max_shots)
    d.max_rec = int(max_rec)
    d.precision = int(precision)
    d.skip_cfl_check = int(bool(skip_cfl_check))
    d.adj_budget = int(adj_budget)
    return d


def _ptr(a):
    """Raw pointer of a torch tensor (device or host) or numpy array; None passes NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(a))


def _positions(p, ndim):
    if p is None:
        return None, 0
    a = np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(-1, ndim))
    return a, a.shape[0]


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def sim_plan(desc, vmin=0.0, vmax=0.0):
    info = SimInfo()
    code = abi.load().sim_plan(ctypes.byref(desc), vmin, vmax, ctypes.byref(info))
    _check(code)
    return info


def sim_create(desc, vel=None, stream=None):
    h = ctypes.c_void_p()
    code = abi.load().sim_create(ctypes.byref(desc), _ptr(vel), _stream(stream), ctypes.byref(h))
    _check(code)
    return h.value


def sim_set_model(handle, vel):
    _check(abi.load().sim_set_model(handle, _ptr(vel)), handle)


def sim_forward(handle, nshots, wavelet, src_pos, nrec, rec_pos, gather=None, snaps=None, snap_scale=None):
    _check(abi.load().sim_forward(handle, nshots, _ptr(wavelet), _ptr(src_pos), nrec, _ptr(rec_pos),
                                  _ptr(gather), _ptr(snaps), _ptr(snap_scale)), handle)


def sim_adjoint(handle, nshots, wavelet, src_pos, nrec, rec_pos, d_obs, gather_out, misfit_out,
                ckpt_fp16, grad_v):
    _check(abi.load().sim_adjoint(handle, nshots, _ptr(wavelet), _ptr(src_pos), nrec, _ptr(rec_pos),
                                  _ptr(d_obs), _ptr(gather_out), _ptr(misfit_out), int(ckpt_fp16),
                                  _ptr(grad_v)), handle)


def sim_adjoint_vjp(handle, nshots, wavelet, src_pos, nrec, rec_pos, cot, gather_out, ckpt_fp16, grad_v):
    _check(abi.load().sim_adjoint_vjp(handle, nshots, _ptr(wavelet), _ptr(src_pos), nrec, _ptr(rec_pos),
                                      _ptr(cot), _ptr(gather_out), int(ckpt_fp16), _ptr(grad_v)), handle)


def sim_batch(items, stream=None):
    """items: sequence of SimBatchItem (see batch() for a friendlier form)."""
    arr = (SimBatchItem * len(items))(*items)
    _check(abi.load().sim_batch(len(items), arr, _stream(stream)))


def sim_batch_ex(items, mode, ckpt_fp16=0, stream=None):
    arr = (SimBatchItem * len(items))(*items)
    _check(abi.load().sim_batch_ex(len(items), arr, int(mode), int(ckpt_fp16), _stream(stream)))


def batch(entries, stream=None):
    """Run many shots on many grids in one persistent launch. entries: list of
    dicts with keys sim (Simulator), wavelet, src [nshots, ndim], rec [nrec, ndim]
    and optionally gather (output tensor [nshots, nt, nrec]; allocated if absent).
    Returns the list of gather tensors."""
    import torch
    keep, items, outs = [], [], []
    for e in entries:
        sim = e["sim"]
        d = sim.desc
        src, nshots = _positions(e["src"], d.ndim)
        rec, nrec = _positions(e["rec"], d.ndim)
        w = sim._tensor(e["wavelet"])
        g = e.get("gather")
        if g is None and nrec:
            g = torch.empty((nshots, d.nt, nrec), dtype=sim.dtype, device="cuda")
        keep += [src, rec, w, g]
        items.append(SimBatchItem(sim.handle, nshots, _ptr(w), _ptr(src), nrec, _ptr(rec), _ptr(g)))
        outs.append(g)
    sim_batch(items, stream)
    return outs


def batch_gradient(entries, ckpt_fp16=False, stream=None):
    """Gradient mode of the batch (sim_batch_ex mode 1). entries: dicts with
    sim, wavelet, src, rec, d_obs [nshots, nt, nrec] and optionally
    grad (FP64 device tensor of the interior shape, accumulated; allocated
    zeroed if absent). Returns (list of FP64 gradients, list of misfits)."""
    import torch
    keep, items, grads, mis = [], [], [], []
    for e in entries:
        sim = e["sim"]
        d = sim.desc
        src, nshots = _positions(e["src"], d.ndim)
        rec, nrec = _positions(e["rec"], d.ndim)
        w = sim._tensor(e["wavelet"])
        dob = sim._tensor(e["d_obs"]).contiguous()
        g = e.get("grad")
        if g is None:
            g = torch.zeros(sim.interior_shape, dtype=torch.float64, device="cuda")
        m = np.zeros(1)
        keep += [src, rec, w, dob, g, m]
        items.append(SimBatchItem(sim.handle, nshots, _ptr(w), _ptr(src), nrec, _ptr(rec), None, _ptr(dob), _ptr(g),
                                  m.ctypes.data))
        grads.append(g)
        mis.append(m)
    sim_batch_ex(items, 1, ckpt_fp16, stream)
    return grads, [float(m[0]) for m in mis]


def sim_forward_noalloc(desc, vel, wavelet, src_pos, nrec, rec_pos, gather, stream=None):
    """Forward solve that allocates no device memory (see include/sim.h)."""
    _check(abi.load().sim_forward_noalloc(ctypes.byref(desc), _ptr(vel), _ptr(wavelet), _ptr(src_pos), nrec,
                                          _ptr(rec_pos), _ptr(gather), _stream(stream)))


def sim_wavelet_bandpass(nt, dt, f0, f_lo, f_hi, order, precision, out, stream=None):
    """Band-passed Ricker wavelet into ``out`` (see include/sim.h)."""
    _check(abi.load().sim_wavelet_bandpass(int(nt), float(dt), float(f0), float(f_lo), float(f_hi), int(order),
                                           int(precision), _ptr(out), _stream(stream)))


def bandpass_ricker(nt, dt, f0, f_lo, f_hi, order=4, dtype="float32", device="cuda"):
    """The paper's band-passed source wavelet as a torch tensor [nt] on ``device``."""
    import torch
    tdt = torch.float64 if dtype in ("float64", torch.float64) else torch.float32
    out = torch.empty(int(nt), dtype=tdt, device=device)
    sim_wavelet_bandpass(nt, dt, f0, f_lo, f_hi, order, SIM_FP64 if tdt == torch.float64 else SIM_FP32, out)
    return out


def sim_model_squish(nz, ny, nx, v_in, lab_in, dz, fill_v, fill_label, v_out, lab_out, stream=None):
    """Squish warp on device grids (see include/sim.h)."""
    _check(abi.load().sim_model_squish(int(nz), int(ny), int(nx), _ptr(v_in), _ptr(lab_in), _ptr(dz),
                                       float(fill_v), int(fill_label), _ptr(v_out), _ptr(lab_out), _stream(stream)))


def sim_model_fault(nz, ny, nx, v_in, lab_in, fault, fill_v, fill_label, v_out, lab_out, stream=None):
    """Fault warp on device grids; fault: abi.SimFault (see include/sim.h)."""
    _check(abi.load().sim_model_fault(int(nz), int(ny), int(nx), _ptr(v_in), _ptr(lab_in), ctypes.byref(fault),
                                      float(fill_v), int(fill_label), _ptr(v_out), _ptr(lab_out), _stream(stream)))


def sim_model_deposit(nz, ny, nx, v_in, lab_in, params, bounds, vbed, offsets, eta, v_out, lab_out, stream=None):
    """Deposit slab on device grids; params: abi.SimDeposit, vbed / offsets
    host arrays (see include/sim.h)."""
    vb = np.ascontiguousarray(vbed, np.float32)
    of = np.ascontiguousarray(offsets, np.int32)
    _check(abi.load().sim_model_deposit(int(nz), int(ny), int(nx), _ptr(v_in), _ptr(lab_in), ctypes.byref(params),
                                        _ptr(bounds), _ptr(vb), _ptr(of), _ptr(eta), _ptr(v_out), _ptr(lab_out),
                                        _stream(stream)))


def sim_sync(handle):
    _check(abi.load().sim_sync(handle), handle)


def sim_get_info(handle):
    info = SimInfo()
    _check(abi.load().sim_get_info(handle, ctypes.byref(info)), handle)
    return info


def sim_last_error(handle=None):
    return abi.load().sim_last_error(handle).decode()


def sim_destroy(handle):
    abi.load().sim_destroy(handle)


class Simulator:
    """One velocity model on one GPU. Outputs are torch tensors on the
    handle's device unless host buffers are passed in."""

    def __init__(self, cfg, vel=None, max_shots=1, max_rec=0, precision=SIM_FP32, snap_fp16=False,
                 f_max=0.0, skip_cfl_check=False, stream=None, adj_budget=0):
        import torch
        self.cfg = dict(cfg)
        self.desc = make_desc(cfg, max_shots, max_rec, precision, snap_fp16, f_max, skip_cfl_check, adj_budget)
        self.dtype = torch.float64 if precision == SIM_FP64 else torch.float32
        self.handle = None
        if vel is not None:
            vel = self._tensor(vel)
        self.handle = sim_create(self.desc, vel, stream)
        self.info = sim_get_info(self.handle)

    def _tensor(self, a, device="cuda"):
        import torch
        t = torch.as_tensor(a)
        return t.to(device=device, dtype=self.dtype).contiguous()

    @property
    def interior_shape(self):
        d = self.desc
        return (d.nz, d.ny, d.nx) if d.ndim == 3 else (d.nz, d.nx)

    def set_model(self, vel):
        sim_set_model(self.handle, self._tensor(vel))
        self.info = sim_get_info(self.handle)

    def forward(self, wavelet, src, rec=None, gather=True, snapshots=False):
        import torch
        d = self.desc
        src_a, nshots = _positions(src, d.ndim)
        rec_a, nrec = _positions(rec, d.ndim)
        w = self._tensor(wavelet)
        dev = torch.device("cuda")
        g = torch.empty((nshots, d.nt, nrec), dtype=self.dtype, device=dev) if (gather and nrec) else None
        sn = sc = None
        nsnap = self.info.nsnap
        if snapshots and nsnap:
            sdt = torch.float16 if d.snap_fp16 else self.dtype
            sn = torch.empty((nshots, nsnap) + self.interior_shape, dtype=sdt, device=dev)
            if d.snap_fp16:
                sc = torch.empty((nshots, nsnap), dtype=torch.float32, device=dev)
        sim_forward(self.handle, nshots, w, src_a, nrec, rec_a, g, sn, sc)
        return {"gather": g, "snaps": sn, "snap_scale": sc}

    def sync(self):
        sim_sync(self.handle)

    def close(self):
        if self.handle:
            sim_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
