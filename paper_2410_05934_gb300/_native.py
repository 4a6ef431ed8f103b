"""ctypes loader of libntt_gb300.so (the C ABI in include/ntt_gb300.h).

Argument marshalling only: every step of the transform runs in the library's
CUDA kernels.  There is no fallback: if the library is missing this module
raises, and callers must build it first (``__graft_entry__.build()`` or
``python -m paper_2410_05934_gb300.build``).
"""
import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libntt_gb300.so")

u32, u64, i32, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
U64P = ctypes.POINTER(ctypes.c_uint64)
U32P = ctypes.POINTER(ctypes.c_uint32)

class NttRequest(ctypes.Structure):
    """ntt_request_t of the C ABI."""
    _fields_ = [("log2n", ctypes.c_uint32), ("n_moduli", ctypes.c_uint32), ("n_polys", ctypes.c_uint32),
                ("moduli_offset", ctypes.c_uint32), ("inverse", ctypes.c_uint32), ("schedule", ctypes.c_uint32),
                ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p)]


REQP = ctypes.POINTER(NttRequest)


class NttPlanRequest(ctypes.Structure):
    """ntt_plan_request_t of the C ABI (allocation-free batch execution)."""
    _fields_ = [("plan", ctypes.c_void_p), ("n_polys", ctypes.c_uint32), ("inverse", ctypes.c_uint32),
                ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p)]


PREQP = ctypes.POINTER(NttPlanRequest)

# (name, restype, argtypes) for every symbol the header declares
SIGNATURES = [
    ("ntt_plan", i32, [ctypes.POINTER(vp), u32, U64P, u32, u32, u32]),
    ("ntt_plan_destroy", i32, [vp]),
    ("ntt_plan_root", i32, [vp, u32, U64P]),
    ("ntt_plan_shape", i32, [vp, U32P, U32P, U32P, U64P]),
    ("ntt_forward", i32, [vp, vp, vp, vp]),
    ("ntt_inverse", i32, [vp, vp, vp, vp]),
    ("ntt_forward_inverse", i32, [vp, vp, vp, vp, vp, vp, vp]),
    ("ntt_forward_rows", i32, [vp, vp, vp, u64, u64, vp]),
    ("ntt_inverse_rows", i32, [vp, vp, vp, u64, u64, vp]),
    ("poly_mul_pointwise", i32, [vp, vp, vp, vp, u32, vp]),
    ("ntt_hmul_tensor", i32, [vp, vp, vp, vp, vp]),
    ("ntt_rescale", i32, [vp, vp, vp, vp, u32, vp]),
    ("ntt_inverse_mul", i32, [vp, vp, U32P, u32, vp, U32P, u32, vp, vp]),
    ("ntt_schedule_count", i32, [u32]),
    ("ntt_schedule_name", i32, [u32, u32, ctypes.c_char_p, ctypes.c_size_t]),
    ("ntt_plan_set_schedule", i32, [vp, u32]),
    ("ntt_default_schedule", i32, [u32, u64]),
    ("ntt_schedule_params", i32, [u32, u32, ctypes.POINTER(ctypes.c_int32), u32]),
    ("ntt_plan_get_schedule", i32, [vp, U32P]),
    ("ntt_status", i32, [vp, vp]),
    ("ntt_plan_last_launches", i32, [vp, U32P]),
    ("ntt_bench_butterflies", i32, [u64, u32, u32, u32, u32, vp, vp]),
    ("ntt_debug_bounded_wait", i32, [vp, u32, u32, vp, vp]),
    ("ntt_batch_plan", i32, [ctypes.POINTER(vp), REQP, u32, U64P, u32, u32]),
    ("ntt_batch_update", i32, [vp, REQP, u32, vp]),
    ("ntt_batch_execute", i32, [vp, vp]),
    ("ntt_batch_execute_plain", i32, [vp, U32P, vp]),
    ("ntt_batch_destroy", i32, [vp]),
    ("ntt_batch_status", i32, [vp, vp]),
    ("ntt_batch_info", i32, [vp, U64P, U32P, U64P]),
    ("ntt_batch_execute_static", i32, [PREQP, u32, vp]),
    ("ntt_mlp_forward", i32, [vp, vp, u32, vp, vp]),
    ("ntt_mlp_backward", i32, [vp, vp, vp, vp, vp, u32, ctypes.c_float, vp, vp, vp, vp]),
    ("ntt_mlp_adam", i32, [vp, vp, vp, vp, u32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                           ctypes.c_float, u32, vp]),
    ("tfhe_key_prepare", i32, [vp, vp, u32, vp, vp]),
    ("tfhe_external_product", i32, [vp, vp, vp, u32, u32, vp, u64, vp]),
    ("tfhe_cmux_rotate", i32, [vp, vp, vp, vp, u32, u32, vp, u64, vp]),
    ("ntt_bconv_plan", i32, [ctypes.POINTER(vp), U64P, u32, U64P, u32]),
    ("ntt_bconv", i32, [vp, vp, vp, u32, u64, vp]),
    ("ntt_bconv_destroy", i32, [vp]),
    ("ntt_strerror", ctypes.c_char_p, [i32]),
    ("ntt_version", ctypes.c_char_p, []),
]

_lib = None


def load():
    """Loads the library once; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libntt_gb300.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class NttError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = load().ntt_strerror(code).decode()
        super().__init__("%s failed: %s (%d)" % (what, msg, code) if what else "%s (%d)" % (msg, code))


def check(code, what=""):
    if code != 0:
        raise NttError(code, what)
    return code
