"""FP64 CPU oracle of the acoustic FDTD path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. It shares no
code with the CUDA library in ``paper_2605_30541_gb300/`` and never imports it.

The arithmetic lives in ``fdtd_oracle.c`` (plain loops in FP64, one pass per
term of the scheme of the paper's App. E.2-E.3; readings of the gaps are listed
at its top). This module only compiles it with gcc and marshals numpy arrays.
``bruteforce.py`` is the second, independent oracle for tiny grids (dense
matrices assembled from the same equations).

Parity status: every function here is pinned by tests/test_oracle_pins.py
(closed forms, invariants, brute force, complex step); none is "parity unpinned".
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "fdtd_oracle.c")
_LOCK = threading.Lock()
_LIBS = {}

BC = {"sponge": 0, "cpml": 1, "none": 2}


def _lib_path(complex_):
    return os.path.join(_BUILD, "liboracle_cs.so" if complex_ else "liboracle.so")


def build(force=False):
    """Compile the real and the complex-step oracle libraries (gcc, -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "oracle.h")
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(hdr))
    procs = []
    for cs in (False, True):
        out = _lib_path(cs)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
            continue
        tmp = out + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
               "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"]
        if cs:
            cmd.insert(1, "-DORACLE_COMPLEX")
        procs.append((subprocess.Popen(cmd, stderr=subprocess.PIPE), tmp, out))
    for p, tmp, out in procs:
        _, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + err.decode())
        os.replace(tmp, out)


def _lib(complex_=False):
    with _LOCK:
        if complex_ not in _LIBS:
            if not os.path.exists(_lib_path(complex_)) or \
                    os.path.getmtime(_lib_path(complex_)) < os.path.getmtime(_SRC):
                build()
            lib = ctypes.CDLL(_lib_path(complex_))
            lib.oracle_num_threads.restype = ctypes.c_int
            _LIBS[complex_] = lib
        return _LIBS[complex_]


class Params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("nz", ctypes.c_int), ("ny", ctypes.c_int), ("nx", ctypes.c_int),
        ("h", ctypes.c_double), ("dt", ctypes.c_double), ("nt", ctypes.c_int),
        ("bc", ctypes.c_int), ("nb", ctypes.c_int * 6), ("free_surface", ctypes.c_int),
        ("R", ctypes.c_double), ("f_ref", ctypes.c_double), ("cpml_vmax", ctypes.c_double),
        ("snap_every", ctypes.c_int), ("snap_begin", ctypes.c_int), ("snap_end", ctypes.c_int),
    ]


def params(cfg):
    """Build the oracle parameter block from a problem dict (the keys that
    ``synth`` configurations carry: ndim, nz, ny, nx, h, dt, nt, bc, nb,
    free_surface, R, f_ref, snap_every, snap_begin, snap_end)."""
    p = Params()
    p.ndim = int(cfg["ndim"])
    p.nz, p.ny, p.nx = int(cfg["nz"]), int(cfg.get("ny", 1)), int(cfg["nx"])
    p.h, p.dt, p.nt = float(cfg["h"]), float(cfg["dt"]), int(cfg["nt"])
    bc = cfg.get("bc", "sponge")
    p.bc = BC[bc] if isinstance(bc, str) else int(bc)
    nb = list(cfg.get("nb", [0] * 6))
    for k in range(6):
        p.nb[k] = int(nb[k])
    p.free_surface = int(cfg.get("free_surface", 0))
    p.R = float(cfg.get("R", 1e-3))
    p.f_ref = float(cfg.get("f_ref", 10.0))
    p.cpml_vmax = float(cfg.get("cpml_vmax", 0.0))
    p.snap_every = int(cfg.get("snap_every", 0))
    p.snap_begin = int(cfg.get("snap_begin", 0))
    p.snap_end = int(cfg.get("snap_end", 0))
    return p


def num_threads():
    return _lib().oracle_num_threads()


def padded_dims(cfg):
    p = params(cfg)
    dims = (ctypes.c_int * 3)()
    if _lib().oracle_padded_dims(ctypes.byref(p), dims) != 0:
        raise ValueError("bad oracle parameters")
    return tuple(dims)


def nsnap(cfg):
    every = int(cfg.get("snap_every", 0))
    if every <= 0:
        return 0
    end = min(int(cfg.get("snap_end", 0)), int(cfg["nt"]))
    begin = int(cfg.get("snap_begin", 0))
    return max(0, -(-(end - begin) // every)) if end > begin >= 0 else 0


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _real(a, complex_):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.complex128 if complex_ else np.float64)


def _points(a, ndim):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1, ndim))
    return a


def forward(cfg, vel, wavelet=None, src=None, rec=None, snaps=False,
            init_prev=None, init_cur=None, final=False, complex_=False):
    """One shot of the forward scheme. ``vel``: interior (nz, [ny,] nx) m/s;
    ``wavelet``: (nt,); ``src``: position (x, z) / (x, y, z) in metres;
    ``rec``: (nrec, ndim) positions. Returns a dict with ``gather`` (nt, nrec),
    ``snaps`` (nsnap, nz, [ny,] nx) and optionally the final padded states."""
    lib = _lib(complex_)
    p = params(cfg)
    dims = padded_dims(cfg)
    ndim = p.ndim
    rdt = np.complex128 if complex_ else np.float64
    vel = _real(vel, complex_)
    if vel.size != p.nz * p.ny * p.nx:
        raise ValueError("velocity size mismatch")
    w = None if wavelet is None else np.ascontiguousarray(wavelet, dtype=np.float64)
    s = None if src is None else np.ascontiguousarray(np.asarray(src, dtype=np.float64).reshape(ndim))
    if rec is None:
        nrec, r = 0, None
    else:
        r = _points(rec, ndim)
        nrec = r.shape[0]
    g = np.zeros((p.nt, nrec), dtype=rdt) if nrec else None
    interior = (p.nz, p.ny, p.nx) if ndim == 3 else (p.nz, p.nx)
    ns = nsnap(cfg)
    sn = np.zeros((ns,) + interior, dtype=rdt) if (snaps and ns) else None
    ip = _real(init_prev, complex_)
    ic = _real(init_cur, complex_)
    padded = (dims[0], dims[1], dims[2]) if ndim == 3 else (dims[0], dims[2])
    fp = np.zeros(padded, dtype=rdt) if final else None
    fc = np.zeros(padded, dtype=rdt) if final else None
    rc = lib.oracle_forward(ctypes.byref(p), _ptr(vel), _ptr(w), _ptr(s), ctypes.c_int(nrec),
                            _ptr(r), _ptr(g), _ptr(sn), _ptr(ip), _ptr(ic), _ptr(fp), _ptr(fc))
    if rc != 0:
        raise ValueError("oracle_forward failed (%d)" % rc)
    return {"gather": g, "snaps": sn, "final_prev": fp, "final_cur": fc}


def gradient(cfg, vel, wavelet, src, rec, d_obs, complex_=False):
    """Misfit J = 1/2 ||g - d_obs||^2 of one shot, its gradient with respect to
    the interior velocity, the wavelet gradient and the modelled gather."""
    lib = _lib(complex_)
    p = params(cfg)
    ndim = p.ndim
    rdt = np.complex128 if complex_ else np.float64
    vel = _real(vel, complex_)
    w = np.ascontiguousarray(wavelet, dtype=np.float64)
    s = np.ascontiguousarray(np.asarray(src, dtype=np.float64).reshape(ndim))
    r = _points(rec, ndim)
    nrec = r.shape[0]
    d = np.ascontiguousarray(d_obs, dtype=np.float64).reshape(p.nt, nrec)
    J = np.zeros(1, dtype=rdt)
    grad = np.zeros(vel.shape, dtype=rdt)
    gw = np.zeros(p.nt, dtype=rdt)
    g = np.zeros((p.nt, nrec), dtype=rdt)
    rc = lib.oracle_gradient(ctypes.byref(p), _ptr(vel), _ptr(w), _ptr(s), ctypes.c_int(nrec), _ptr(r),
                             _ptr(d), _ptr(J), _ptr(grad), _ptr(gw), _ptr(g))
    if rc != 0:
        raise ValueError("oracle_gradient failed (%d)" % rc)
    return {"misfit": J[0], "grad": grad, "grad_wavelet": gw, "gather": g}


def laplacian(cfg, f, transpose=False):
    """L f (gather form) or L^T f (explicit scatter transpose) on the padded grid."""
    lib = _lib(False)
    p = params(cfg)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros_like(f)
    fn = lib.oracle_apply_laplacian_T if transpose else lib.oracle_apply_laplacian
    if fn(ctypes.byref(p), _ptr(f), _ptr(out)) != 0:
        raise ValueError("bad parameters")
    return out


def coefficients(cfg, vel):
    """Padded c = v^2 dt^2, a = eta v^2 dt / 2, and per-axis CPML (a, b) lists
    (axis order z, y, x)."""
    lib = _lib(False)
    p = params(cfg)
    dims = padded_dims(cfg)
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    shape = dims if p.ndim == 3 else (dims[0], dims[2])
    c = np.zeros(shape)
    a = np.zeros(shape)
    ntot = dims[0] + dims[1] + dims[2]
    ca = np.zeros(ntot)
    cb = np.zeros(ntot)
    if lib.oracle_coefficients(ctypes.byref(p), _ptr(vel), _ptr(c), _ptr(a), _ptr(ca), _ptr(cb)) != 0:
        raise ValueError("bad parameters")
    o = np.cumsum([0, dims[0], dims[1], dims[2]])
    return {"c": c, "a": a,
            "cpml_a": [ca[o[k]:o[k + 1]] for k in range(3)],
            "cpml_b": [cb[o[k]:o[k + 1]] for k in range(3)]}
