"""ctypes binding of libsupergpu.so: the same names and arguments as include/sg.h.

Argument marshalling only.  Every step of the evolution runs in the library's
CUDA kernels; there is no Python or CPU fallback, and importing a function of this
module when the library has not been built raises.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsupergpu.so")

SG_OK = 0
SG_E_INVALID, SG_E_NOMEM, SG_E_STATE, SG_E_CUDA, SG_E_TIMEOUT = -1, -2, -3, -4, -5
SG_SOLVER_RK4, SG_SOLVER_Q1, SG_SOLVER_Q2, SG_SOLVER_Q4, SG_SOLVER_Q4J = 0, 1, 2, 4, 5
SG_COMP_NONE, SG_COMP_VZ = 0, 1
SG_BASIS_PRODUCT, SG_BASIS_DRESSED = 0, 1
SG_E_PENDING, SG_E_NOMEM_RETRY, SG_E_CANCELLED, SG_E_NOTFOUND, SG_E_UNSUPPORTED = -6, -7, -8, -9, -10
SG_OP_N, SG_OP_PHI = 0, 1
SG_ENV_GAUSSIAN, SG_ENV_PWC, SG_ENV_COSINE = 0, 1, 2
SG_FP64, SG_MIXED = 0, 1
SG_FRAME_INTERACTION, SG_FRAME_LAB = 0, 1
SG_FID_AVG, SG_FID_STATE = 0, 1


class sg_pulse(C.Structure):
    _fields_ = [("kind", C.c_int), ("nseg", C.c_int), ("amps", C.POINTER(C.c_double)),
                ("amp", C.c_double), ("sigma", C.c_double), ("t0", C.c_double),
                ("length", C.c_double), ("omega_d", C.c_double), ("omega_mode", C.c_int),
                ("phase", C.c_double)]


class sg_evolve_opts(C.Structure):
    _fields_ = [("T", C.c_double), ("dt", C.c_double), ("precision", C.c_int),
                ("frame", C.c_int), ("ncols", C.c_int),
                ("col_index", C.POINTER(C.c_longlong)), ("solver", C.c_int), ("compensation", C.c_int),
                ("basis", C.c_int)]


class sg_request(C.Structure):
    _fields_ = [("sys", C.c_void_p), ("opts", sg_evolve_opts),
                ("target_re_im", C.POINTER(C.c_double)), ("kind", C.c_int),
                ("want_grad", C.c_int)]


class sg_result(C.Structure):
    _fields_ = [("status", C.c_int), ("F", C.c_double * 2),
                ("grad_pulse", C.POINTER(C.c_double)), ("grad_ham", C.POINTER(C.c_double)),
                ("n_pulse", C.c_int), ("n_ham", C.c_int), ("submit_s", C.c_double),
                ("start_s", C.c_double), ("done_s", C.c_double), ("error", C.c_char * 192)]


class sg_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64),
                ("cancelled", C.c_uint64), ("rejected", C.c_uint64),
                ("solves_per_s", C.c_double), ("p50_s", C.c_double), ("p99_s", C.c_double),
                ("gpu_busy_frac", C.c_double), ("mem_in_use", C.c_size_t),
                ("mem_budget", C.c_size_t), ("active_slots", C.c_int), ("max_slots", C.c_int),
                ("batches", C.c_longlong), ("batched_requests", C.c_longlong),
                ("batched_launches", C.c_longlong), ("batched_launch_members", C.c_longlong)]


_P = C.c_void_p
_I = C.c_int
# int (*sg_allreduce_fn)(double* buf, int n, void* user)
SG_ALLREDUCE_FN = C.CFUNCTYPE(C.c_int, C.POINTER(C.c_double), C.c_int, C.c_void_p)
_D = C.c_double
_PD = C.POINTER(C.c_double)
_PI = C.POINTER(C.c_int)

# name -> (restype, argtypes); mirrors include/sg.h
SIGNATURES = {
    "sg_ctx_create": (_I, [C.POINTER(_P), _I, _P]),
    "sg_ctx_destroy": (_I, [_P]),
    "sg_last_error": (C.c_char_p, [_P]),
    "sg_version": (C.c_char_p, []),
    "sg_system_create": (_I, [_P, C.POINTER(_P)]),
    "sg_system_destroy": (_I, [_P]),
    "sg_add_transmon": (_I, [_P, _D, _D, _D, _I, _I, _PI]),
    "sg_add_fluxonium": (_I, [_P, _D, _D, _D, _D, _I, _I, _PI]),
    "sg_add_coupling": (_I, [_P, _I, _I, _I, _I, _D, _PI]),
    "sg_set_coupler": (_I, [_P, _I, _I]),
    "sg_add_local_op": (_I, [_P, _I, _PD, _PI]),
    "sg_add_drive": (_I, [_P, _I, _I, C.POINTER(sg_pulse), _PI]),
    "sg_param_counts": (_I, [_P, _PI, _PI]),
    "sg_get_params": (_I, [_P, _PD, _PD]),
    "sg_set_params": (_I, [_P, _PD, _PD]),
    "sg_prepare": (_I, [_P]),
    "sg_get_spectrum": (_I, [_P, _I, _PD, _PD, _PD]),
    "sg_dims": (_I, [_P, C.POINTER(C.c_longlong), _PI]),
    "sg_evolve": (_I, [_P, C.POINTER(sg_evolve_opts), _P]),
    "sg_evolve_noalloc": (_I, [_P, C.POINTER(sg_evolve_opts), _P]),
    "sg_evolve_batch": (_I, [C.POINTER(_P), _I, C.POINTER(sg_evolve_opts), _P]),
    "sg_add_collapse": (_I, [_P, _I, _PD, _D, _PI]),
    "sg_evolve_open": (_I, [_P, C.POINTER(sg_evolve_opts), _PD, _PD]),
    "sg_gate_fidelity_open": (_I, [_P, C.POINTER(sg_evolve_opts), _PD, _PD]),
    "sg_gate_fidelity_open_grad": (_I, [_P, C.POINTER(sg_evolve_opts), _PD, _I, _PD, _PD, _PD, _I]),
    "sg_fidelity": (_I, [_P, C.POINTER(sg_evolve_opts), _PD, _PD, _PD]),
    "sg_fidelity_grad": (_I, [_P, C.POINTER(sg_evolve_opts), _PD, _I, _PD, _PD, _PD, _I]),
    "sg_fidelity_grad_sharded": (_I, [_P, C.POINTER(sg_evolve_opts), _PD, _I, _PD, _PD, _PD, _I,
                                      SG_ALLREDUCE_FN, _P]),
    "sg_last_stats": (_I, [_P, _PD]),
    "sg_kernel_times": (_I, [_P, _PD, _I]),
    "sg_server_create": (_I, [_P, C.c_size_t, _I, C.POINTER(_P)]),
    "sg_server_destroy": (_I, [_P]),
    "sg_server_submit": (_I, [_P, C.POINTER(sg_request), C.POINTER(C.c_uint64)]),
    "sg_server_poll": (_I, [_P, C.c_uint64, C.POINTER(sg_result)]),
    "sg_server_wait": (_I, [_P, C.c_uint64, C.POINTER(sg_result)]),
    "sg_server_cancel": (_I, [_P, C.c_uint64]),
    "sg_server_stats": (_I, [_P, C.POINTER(sg_stats)]),
    "sg_server_set_batch": (_I, [_P, _I]),
}

_lib = None


def lib():
    """The loaded library.  Raises when it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2406_18155_gb300.build` "
                "(the CUDA library is required; there is no CPU path)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class SGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def check(rc, ctx=None):
    if rc != SG_OK:
        m = lib().sg_last_error(ctx)
        raise SGError(rc, m.decode() if m else "error")
    return rc


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)
