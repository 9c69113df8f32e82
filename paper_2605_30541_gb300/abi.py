"""ctypes mirror of include/sim.h. Argument marshalling only: every step of the
solver runs inside libsim.so; nothing here computes."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsim.so")

SIM_OK = 0
SIM_ERR_ARG = 1
SIM_ERR_CFL = 2
SIM_WARN_DISPERSION = 3
SIM_ERR_OOM = 4
SIM_ERR_CUDA = 5
SIM_ERR_TIMEOUT = 6
SIM_ERR_UNSTABLE = 7
SIM_ERR_STATE = 8
SIM_ERR_UNSUPPORTED = 9
STATUS_NAMES = {0: "SIM_OK", 1: "SIM_ERR_ARG", 2: "SIM_ERR_CFL", 3: "SIM_WARN_DISPERSION",
                4: "SIM_ERR_OOM", 5: "SIM_ERR_CUDA", 6: "SIM_ERR_TIMEOUT", 7: "SIM_ERR_UNSTABLE",
                8: "SIM_ERR_STATE", 9: "SIM_ERR_UNSUPPORTED"}

SIM_BC = {"sponge": 0, "cpml": 1, "none": 2}
SIM_FP32, SIM_FP64 = 0, 1


class SimDesc(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("nz", ctypes.c_int), ("ny", ctypes.c_int), ("nx", ctypes.c_int),
        ("h", ctypes.c_double), ("dt", ctypes.c_double), ("nt", ctypes.c_int),
        ("space_order", ctypes.c_int), ("bc", ctypes.c_int), ("nb", ctypes.c_int * 6),
        ("free_surface", ctypes.c_int), ("R", ctypes.c_double), ("f_ref", ctypes.c_double),
        ("f_max", ctypes.c_double), ("snap_every", ctypes.c_int), ("snap_begin", ctypes.c_int),
        ("snap_end", ctypes.c_int), ("snap_fp16", ctypes.c_int), ("max_shots", ctypes.c_int),
        ("max_rec", ctypes.c_int), ("precision", ctypes.c_int), ("skip_cfl_check", ctypes.c_int),
        ("pad0", ctypes.c_int), ("adj_budget", ctypes.c_longlong),
    ]


class SimInfo(ctypes.Structure):
    _fields_ = [
        ("NZ", ctypes.c_int), ("NY", ctypes.c_int), ("NX", ctypes.c_int), ("nsnap", ctypes.c_int),
        ("courant", ctypes.c_double), ("courant_limit", ctypes.c_double),
        ("courant_exact", ctypes.c_double), ("vmin", ctypes.c_double), ("vmax", ctypes.c_double),
        ("c_damp", ctypes.c_double * 6), ("cells_per_shot", ctypes.c_longlong),
        ("device_bytes", ctypes.c_size_t), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
        ("tile_z", ctypes.c_int), ("last_path", ctypes.c_int), ("last_rows", ctypes.c_int),
        ("adj_levels", ctypes.c_int), ("adj_slots", ctypes.c_int), ("adj_inner", ctypes.c_int),
        ("adj_top", ctypes.c_int), ("adj_sub", ctypes.c_int), ("pad1", ctypes.c_int),
        ("adj_bytes", ctypes.c_size_t), ("z_variant", ctypes.c_int), ("z_chunk", ctypes.c_int),
        ("batch_sched", ctypes.c_int), ("batch_tile", ctypes.c_int),
    ]


class SimBatchItem(ctypes.Structure):
    _fields_ = [
        ("sim", ctypes.c_void_p), ("nshots", ctypes.c_int), ("wavelet", ctypes.c_void_p),
        ("src_pos", ctypes.c_void_p), ("nrec", ctypes.c_int), ("rec_pos", ctypes.c_void_p),
        ("gather", ctypes.c_void_p), ("d_obs", ctypes.c_void_p), ("grad_sum_fp64", ctypes.c_void_p),
        ("misfit", ctypes.c_void_p),
    ]


class SimFault(ctypes.Structure):
    _fields_ = [
        ("cz", ctypes.c_double), ("cy", ctypes.c_double), ("cx", ctypes.c_double),
        ("azimuth", ctypes.c_double), ("dip", ctypes.c_double), ("radius", ctypes.c_double),
        ("slip", ctypes.c_double), ("direction", ctypes.c_int), ("pad", ctypes.c_int),
        ("d_die", ctypes.c_double), ("d_perp", ctypes.c_double), ("theta_die", ctypes.c_double),
    ]


class SimDeposit(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_int), ("nbeds", ctypes.c_int), ("nzt", ctypes.c_int), ("label0", ctypes.c_int),
        ("beta", ctypes.c_float), ("a_eta", ctypes.c_float), ("f_top", ctypes.c_float), ("f_base", ctypes.c_float),
    ]


_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_F = ctypes.c_float
_PROTOS = {
    "sim_desc_init": (None, [ctypes.POINTER(SimDesc)]),
    "sim_plan": (_I, [ctypes.POINTER(SimDesc), _D, _D, ctypes.POINTER(SimInfo)]),
    "sim_create": (_I, [ctypes.POINTER(SimDesc), _VP, _VP, ctypes.POINTER(_VP)]),
    "sim_set_model": (_I, [_VP, _VP]),
    "sim_forward": (_I, [_VP, _I, _VP, _VP, _I, _VP, _VP, _VP, _VP]),
    "sim_adjoint": (_I, [_VP, _I, _VP, _VP, _I, _VP, _VP, _VP, _VP, _I, _VP]),
    "sim_adjoint_vjp": (_I, [_VP, _I, _VP, _VP, _I, _VP, _VP, _VP, _I, _VP]),
    "sim_batch": (_I, [_I, ctypes.POINTER(SimBatchItem), _VP]),
    "sim_batch_ex": (_I, [_I, ctypes.POINTER(SimBatchItem), _I, _I, _VP]),
    "sim_forward_noalloc": (_I, [ctypes.POINTER(SimDesc), _VP, _VP, _VP, _I, _VP, _VP, _VP]),
    "sim_wavelet_bandpass": (_I, [_I, _D, _D, _D, _D, _I, _I, _VP, _VP]),
    "sim_model_squish": (_I, [_I, _I, _I, _VP, _VP, _VP, _F, _I, _VP, _VP, _VP]),
    "sim_model_fault": (_I, [_I, _I, _I, _VP, _VP, ctypes.POINTER(SimFault), _F, _I, _VP, _VP, _VP]),
    "sim_model_deposit": (_I, [_I, _I, _I, _VP, _VP, ctypes.POINTER(SimDeposit), _VP, _VP, _VP, _VP, _VP, _VP,
                               _VP]),
    "sim_sync": (_I, [_VP]),
    "sim_get_info": (_I, [_VP, ctypes.POINTER(SimInfo)]),
    "sim_last_error": (ctypes.c_char_p, [_VP]),
    "sim_destroy": (None, [_VP]),
}

_lib = None


def load():
    """Load libsim.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libsim.so is not built (run __graft_entry__.build())")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
