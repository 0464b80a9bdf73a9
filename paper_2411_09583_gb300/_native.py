"""ctypes declarations of the C ABI in include/nuht.h (argument marshalling only).

The shared library is built in-tree by ``build_native.build()``.  Loading
fails loudly if it is missing: there is no fallback implementation.
"""
import ctypes
import os
import threading

from . import build_native

_lock = threading.Lock()
_lib = None

NUHT_OK = 0
NUHT_ERR_INVALID_ARG = 1
NUHT_ERR_DOMAIN = 2
NUHT_ERR_NOMEM = 3
NUHT_ERR_CUDA = 4
NUHT_ERR_TIMEOUT = 5
NUHT_ERR_UNSUPPORTED = 6
NUHT_ERR_SCRATCH = 7
NUHT_ERR_BAD_BLOCKS = 8
NOALLOC_MAX_MOMENTS = 32768

PREC_FP64 = 0
PREC_MIXED = 1
BLOCK_LOCAL, BLOCK_ASY, BLOCK_DIRECT = 0, 1, 2

# every symbol include/nuht.h declares
EXPORTED = ["nuht_default_opts", "nuht_choose_params", "nuht_plan", "nuht_execute",
            "nuht_adjoint", "nuht_transform_host", "nuht_info", "nuht_get_blocks",
            "nuht_get_permutations", "nuht_destroy", "nuht_strerror",
            "nuht_last_cuda_error", "nuht_stage_times", "nuht_stage_name",
            "nuht_kernel_launch_count", "nuht_local_apply_noalloc", "nuht_plan_many",
            "nuht_probe_alu", "nuht_check_blocks", "nuht_plan_deriv", "nuht_grad_r",
            "nuht_grad_omega", "nuht_status"]
NUM_STAGES = 8


class NuhtOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("min_size", ctypes.c_int),
                ("n_split_cand", ctypes.c_int), ("m_terms", ctypes.c_int),
                ("class_mask", ctypes.c_int), ("timing", ctypes.c_int),
                ("spread_tile", ctypes.c_int), ("deterministic", ctypes.c_int),
                ("persistent", ctypes.c_int), ("interp_tile", ctypes.c_int),
                ("vec_group", ctypes.c_int), ("reserved", ctypes.c_int)]


class NuhtPlanInfo(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_int), ("M", ctypes.c_int), ("L", ctypes.c_int),
                ("nufft_width", ctypes.c_int), ("nufft_degree", ctypes.c_int), ("asy_members", ctypes.c_int),
                ("z", ctypes.c_double), ("eps", ctypes.c_double),
                ("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("n_local", ctypes.c_int64), ("n_asy", ctypes.c_int64),
                ("n_direct", ctypes.c_int64), ("direct_entries", ctypes.c_int64),
                ("local_rows_cols", ctypes.c_int64), ("asy_rows_cols", ctypes.c_int64),
                ("fft_points", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("plan_ms", ctypes.c_double * 4)]


class NuhtError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = lib().nuht_strerror(code).decode()
        if code == NUHT_ERR_CUDA:
            msg += " (" + lib().nuht_last_cuda_error().decode() + ")"
        super().__init__("%s: %s [code %d]" % (what, msg, code) if what else msg)


def check(code, what=""):
    if code != NUHT_OK:
        raise NuhtError(code, what)


def lib_path():
    return build_native.LIB


def lib():
    """Load libnuht.so (built by build_native.build()); raises if it is absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("libnuht.so is not built (%s); run build_native.build() "
                               "or __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        i, i64, d, p = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        L.nuht_default_opts.argtypes = [ctypes.POINTER(NuhtOpts)]
        L.nuht_default_opts.restype = None
        L.nuht_choose_params.argtypes = [i, d, i, ctypes.POINTER(i), ctypes.POINTER(d),
                                         ctypes.POINTER(i)]
        L.nuht_choose_params.restype = i
        L.nuht_plan.argtypes = [ctypes.POINTER(p), i, p, i64, p, i64, d,
                                ctypes.POINTER(NuhtOpts), p]
        L.nuht_plan.restype = i
        L.nuht_execute.argtypes = [p, p, p, i, i, p]
        L.nuht_execute.restype = i
        L.nuht_adjoint.argtypes = [p, p, p, i, i, p]
        L.nuht_adjoint.restype = i
        L.nuht_transform_host.argtypes = [i, p, i64, p, i64, d, p, p, i,
                                          ctypes.POINTER(NuhtOpts), p]
        L.nuht_transform_host.restype = i
        L.nuht_info.argtypes = [p, ctypes.POINTER(NuhtPlanInfo)]
        L.nuht_info.restype = i
        L.nuht_get_blocks.argtypes = [p, i, p, i64, ctypes.POINTER(i64)]
        L.nuht_get_blocks.restype = i
        L.nuht_get_permutations.argtypes = [p, p, p]
        L.nuht_get_permutations.restype = i
        L.nuht_destroy.argtypes = [p]
        L.nuht_destroy.restype = None
        L.nuht_strerror.argtypes = [i]
        L.nuht_strerror.restype = ctypes.c_char_p
        L.nuht_last_cuda_error.argtypes = []
        L.nuht_last_cuda_error.restype = ctypes.c_char_p
        L.nuht_stage_times.argtypes = [p, p, i]
        L.nuht_stage_times.restype = i
        L.nuht_stage_name.argtypes = [i]
        L.nuht_stage_name.restype = ctypes.c_char_p
        L.nuht_kernel_launch_count.argtypes = []
        L.nuht_kernel_launch_count.restype = i64
        L.nuht_local_apply_noalloc.argtypes = [i, d, p, i64, d, p, i64, d, p, p, i, p]
        L.nuht_local_apply_noalloc.restype = i
        L.nuht_plan_many.argtypes = [ctypes.POINTER(p), i, p, p, p, p, p, d,
                                     ctypes.POINTER(NuhtOpts), p]
        L.nuht_plan_many.restype = i
        L.nuht_probe_alu.argtypes = [i, i64, ctypes.POINTER(d), ctypes.POINTER(d), p]
        L.nuht_probe_alu.restype = i
        L.nuht_check_blocks.argtypes = [i, d, i, p, i64, p, i64, i, p, p, i64]
        L.nuht_check_blocks.restype = i
        L.nuht_plan_deriv.argtypes = [ctypes.POINTER(p), p, p]
        L.nuht_plan_deriv.restype = i
        L.nuht_grad_r.argtypes = [p, p, p, p, i, p]
        L.nuht_grad_r.restype = i
        L.nuht_grad_omega.argtypes = [p, p, p, p, i, p]
        L.nuht_grad_omega.restype = i
        L.nuht_status.argtypes = [p, p]
        L.nuht_status.restype = i
        _lib = L
        return _lib
