"""ctypes binding of libsem.so: the C ABI of include/sem.h with the same names.

Argument marshalling only.  Loading fails loudly when the library has not been
built: there is no fallback implementation.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsem.so")

SEM_OK = 0
SEM_ERR_ARG = -1
SEM_ERR_ALIAS = -2
SEM_ERR_OOM = -3
SEM_ERR_NONFINITE = -4
SEM_ERR_STATE = -5
SEM_ERR_CUDA = -6

SEM_RK4, SEM_SSPRK3, SEM_EULER, SEM_CN, SEM_BS3 = 0, 1, 2, 3, 4
SEM_PREC_FP64, SEM_PREC_FP32_BULK, SEM_PREC_FP64_DF = 0, 1, 2
SEM_CONTRACT_CUDA_CORE, SEM_CONTRACT_TENSOR = 0, 1
SEM_CKPT_AUTO, SEM_CKPT_STAGES, SEM_CKPT_STATES, SEM_CKPT_BINOMIAL, SEM_CKPT_TWO_LEVEL = 0, 1, 2, 3, 4


class sem_opts(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("E", ctypes.c_int), ("N", ctypes.c_int),
                ("nu", ctypes.c_double), ("L", ctypes.c_double), ("precision", ctypes.c_int),
                ("ckpt_mode", ctypes.c_int), ("ckpt_slots", ctypes.c_int),
                ("ckpt_budget_bytes", ctypes.c_size_t)]


class SemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libsem error %d: %s" % (code, msg))
        self.code = code


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_H = ctypes.c_void_p            # sem_t
_SIGS = {
    "sem_create": (_I, [_I, _I, _I, _D, ctypes.POINTER(_H)]),
    "sem_create_ex": (_I, [ctypes.POINTER(sem_opts), ctypes.POINTER(_H)]),
    "sem_destroy": (None, [_H]),
    "sem_ndof": (ctypes.c_size_t, [_H]),
    "sem_coords": (_I, [_H, _P]),
    "sem_rhs": (_I, [_H, _P, _P, _P]),
    "sem_jac_apply": (_I, [_H, _P, _P, _P, _P]),
    "sem_jacT_apply": (_I, [_H, _P, _P, _P, _P]),
    "sem_rk_forward": (_I, [_H, _I, _D, _I, _P, _P, _P]),
    "sem_rk_adjoint": (_I, [_H, _P, _P, _P]),
    "sem_objective": (_I, [_H, _P, _P, ctypes.POINTER(_D), _P, _P]),
    "sem_objective_grad": (_I, [_H, _I, _D, _I, _P, _P, ctypes.POINTER(_D), _P, _P]),
    "sem_ckpt_plan": (_I, [_I, _I, ctypes.POINTER(ctypes.c_longlong)]),
    "sem_sweep_stats": (_I, [_H, ctypes.POINTER(ctypes.c_longlong)]),
    "sem_set_solver": (_I, [_H, _D, _D, _I, _I]),
    "sem_set_advection": (_I, [_H, _P, _P]),
    "sem_set_host_tier": (_I, [_H, ctypes.c_size_t]),
    "sem_set_adaptive": (_I, [_H, _D, _D]),
    "sem_launch_count": (_I, [_H, ctypes.POINTER(ctypes.c_longlong)]),
    "sem_set_dependent_launch": (_I, [_I]),
    "sem_set_contraction": (_I, [_H, _I]),
    "sem_adaptive_steps": (_I, [_H, ctypes.POINTER(_I), ctypes.POINTER(_I), _P, _I]),
    "sem_trajectory_info": (_I, [_H, ctypes.POINTER(ctypes.c_longlong)]),
    "sem_solver_stats": (_I, [_H, ctypes.POINTER(ctypes.c_longlong)]),
    "sem_profile": (_I, [_H, _I]),
    "sem_profile_read": (_I, [_H, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D), _I]),
    "sem_rhs_noalloc": (_I, [_H, _P, _P, _P]),
    "sem_set_graph": (_I, [_H, _I]),
    "sem_graph_replays": (ctypes.c_longlong, [_H]),
    "sem_batch_create": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D),
                              ctypes.POINTER(sem_opts), ctypes.POINTER(_H)]),
    "sem_batch_count": (_I, [_H]),
    "sem_batch_layout": (_I, [_H, _I, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "sem_batch_coords": (_I, [_H, _I, _P]),
    "sem_batch_autotune": (_I, [_H, ctypes.POINTER(_D), ctypes.POINTER(_I), _P]),
    "sem_batch_objective_grad": (_I, [_H, _I, _D, _I, _P, _P, ctypes.POINTER(_D), _P, _P]),
    "sem_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded libsem.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libsem.so is not built (%s); run `python -m paper_1806_01422_gb300.build` "
                              "or `__graft_entry__.build()`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code):
    if code != SEM_OK:
        raise SemError(code, lib().sem_last_error().decode())
    return code


def __getattr__(name):
    # sem_* functions are forwarded to the loaded library under their C names
    if name.startswith("sem_"):
        return getattr(lib(), name)
    raise AttributeError(name)
