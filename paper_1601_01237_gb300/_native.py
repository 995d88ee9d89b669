"""ctypes loader of libmclbm.so, the CUDA library behind include/lbm.h.

Loading fails loudly when the library has not been built: there is no CPU or
Python fallback for any part of the step.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY may point at another build of the same C ABI (e.g. a kernel
# variant under evaluation); by default the in-tree build is loaded.
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(HERE, "libmclbm.so")

# lbm_status codes
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENOTSUP, LBM_ENUMERIC = range(6)
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA",
                4: "LBM_ENOTSUP", 5: "LBM_ENUMERIC"}
# lbm_storage, lbm_collision, lbm_wall_model
STORAGE = {"f64": 0, "f32": 1, "f16_dev": 2, "bf16_dev": 3, "f16_rel": 4, "bf16_rel": 5}
COLLISION = {"bgk": 0, "regularized": 1, "regularized3": 2}
WALL_MODEL = {"potential": 0, "mirror": 1}
FORCING = {"edm": 0, "guo": 1}


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("tau", ctypes.c_double * 2),
        ("G", (ctypes.c_double * 2) * 2),
        ("g_ext", ctypes.c_double * 3),
        ("rho_s", ctypes.c_double * 2),
        ("rho0_dev", ctypes.c_double),
        ("storage", ctypes.c_int),
        ("collision", ctypes.c_int),
        ("wall_model", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("forcing", ctypes.c_int),
    ]


# (name, restype, argtypes) of every entry point declared in include/lbm.h
_VP, _DP, _I, _L, _SZ = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_long, ctypes.c_size_t
SIGNATURES = [
    ("lbm_lattice_dirs", _I, [ctypes.POINTER(ctypes.c_int), _DP]),
    ("lbm_create", _I, [ctypes.POINTER(lbm_params), ctypes.POINTER(_VP)]),
    ("lbm_init_fields", _I, [_VP, _VP, _VP, _VP, _I]),
    ("lbm_step", _I, [_VP, _L]),
    ("lbm_step_timed", _I, [_VP, _L, _DP, ctypes.POINTER(_L), ctypes.POINTER(ctypes.c_char_p),
                            ctypes.POINTER(_I)]),
    ("lbm_moments", _I, [_VP, _I, _VP, _VP, _VP, _I]),
    ("lbm_reduce", _I, [_VP, _DP]),
    ("lbm_pressure_jump", _I, [_VP, _DP, ctypes.c_double, ctypes.c_double, _DP]),
    ("lbm_droplet_stats", _I, [_VP, ctypes.c_double, _DP, _DP]),
    ("lbm_set_solid", _I, [_VP, _VP, _I]),
    ("lbm_get_populations", _I, [_VP, _VP, _I]),
    ("lbm_set_populations", _I, [_VP, _VP, _I]),
    ("lbm_state_bytes", _I, [_VP, ctypes.POINTER(_SZ)]),
    ("lbm_get_state", _I, [_VP, _VP, _SZ]),
    ("lbm_set_state", _I, [_VP, _VP, _SZ]),
    ("lbm_step_count", _I, [_VP, ctypes.POINTER(_L)]),
    ("lbm_sync", _I, [_VP]),
    ("lbm_record", _I, [_VP, _L, _I]),
    ("lbm_adjoint", _I, [_VP, _VP, _VP, _I, _VP, _VP, _DP]),
    ("lbm_step_noalloc", _I, [ctypes.POINTER(lbm_params), _VP, _VP]),
    ("lbm_destroy", None, [_VP]),
    ("lbm_last_error", ctypes.c_char_p, [_VP]),
]

_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libmclbm.so is not built (expected at %s); run "
                "`python -m paper_1601_01237_gb300.build` (needs nvcc)" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def check(status, handle=None):
    if status != LBM_OK:
        msg = lib().lbm_last_error(handle)
        raise LBMError(status, msg.decode() if msg else "")
    return status
