"""ctypes declarations for ``libhps_gb300.so`` (the C ABI in include/hps.h).

Argument marshalling only: every step of the solver runs in the native library.  Loading
fails loudly when the library has not been built -- there is no fallback path.
"""
import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhps_gb300.so")

HPS_OK = 0
HPS_FP64 = 0
HPS_MIXED = 1
HPS_NODES_CHEB_LEAF = 0
HPS_NODES_GAUSS_BOUNDARY = 1
HPS_NODES_GAUSS_ALL = 2
HPS_BC_DIRICHLET = 0
HPS_BC_PERIODIC = 1
HPS_BC_NEUMANN = 2
HPS_GEMM_TENSOR = 0
HPS_GEMM_SIMT = 1

STATUS_NAMES = {
    0: "OK", 1: "INVALID_ARG", 2: "NOT_ELLIPTIC", 3: "SINGULAR", 4: "OOM", 5: "CUDA",
    6: "TIMEOUT", 7: "NO_CONVERGENCE", 8: "STATE",
}

# Every symbol include/hps.h declares, with (restype, argtypes).
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class hps_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class hps_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("q", C.c_int), ("store_leaf_ops", C.c_int),
                ("ir_tol", C.c_double), ("ir_max_iter", C.c_int), ("fp64_top_levels", C.c_int),
                ("use_graphs", C.c_int), ("autotune", C.c_int), ("autotune_cache", C.c_char_p),
                ("shared_leaf", C.c_int), ("bc_we", C.c_int), ("bc_sn", C.c_int),
                ("fp64_gemm", C.c_int), ("fp32_gemm", C.c_int)]


P = C.c_void_p
SIGNATURES = {
    "hps_opts_default": (None, [C.POINTER(hps_opts)]),
    "hps_tree_uniform": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.POINTER(P)]),
    "hps_tree_destroy": (C.c_int, [P]),
    "hps_tree_mask": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, P, C.POINTER(P)]),
    "hps_tree_refine": (C.c_int, [P, P, C.c_int, C.c_int, C.POINTER(P)]),
    "hps_tree_info": (C.c_int, [P, C.c_int] + [C.POINTER(C.c_int)] * 5),
    "hps_nodes": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P, C.POINTER(C.c_int64)]),
    "hps_plan_check": (C.c_int, [P, C.c_int, C.POINTER(hps_opts)]),
    "hps_apply": (C.c_int, [P, P, P, C.c_int, C.c_double, C.c_double, P, P]),
    "hps_build": (C.c_int, [P, P, C.c_int, C.POINTER(hps_opts), C.POINTER(hps_allocator), P, C.POINTER(P)]),
    "hps_solve": (C.c_int, [P, P, P, C.c_int, P, P]),
    "hps_solve_noalloc": (C.c_int, [P, P, P, C.c_int, P, P]),
    "hps_solve_ext": (C.c_int, [P, P, P, P, C.c_int, P, P, C.POINTER(C.c_int), P]),
    "hps_adjoint": (C.c_int, [P, P, C.c_int, P, P, P, P, P]),
    "hps_handle_info": (C.c_int, [P] + [C.POINTER(C.c_int)] * 5 + [C.POINTER(C.c_int64)]),
    "hps_sync_status": (C.c_int, [P, P]),
    "hps_destroy": (C.c_int, [P]),
    "hps_last_error": (C.c_char_p, []),
    "hps_selftest_wait_timeout": (C.c_int, [C.c_int, P]),
    "hps_timing_enable": (C.c_int, [C.c_int]),
    "hps_timing_reset": (C.c_int, []),
    "hps_timing_count": (C.c_int, [C.POINTER(C.c_int)]),
    "hps_timing_get": (C.c_int, [C.c_int, C.c_char_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double)]),
}

_lib = None


class HPSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hps error %d (%s): %s" % (code, STATUS_NAMES.get(code, "?"), msg))
        self.code = code


def load():
    """Load the native library (build it first with paper_1612_02736_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libhps_gb300.so is not built (run `python -m paper_1612_02736_gb300.build`); "
                          "the solver has no non-native fallback")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code):
    if code != HPS_OK:
        raise HPSError(code, load().hps_last_error().decode(errors="replace"))


def timing_table():
    """Per-category launch timing recorded while hps_timing_enable(1) was on:
    list of dicts (name, launches, ms, flops, bytes)."""
    lib = load()
    n = C.c_int()
    check(lib.hps_timing_count(C.byref(n)))
    out = []
    buf = C.create_string_buffer(128)
    for i in range(n.value):
        la, ms, fl, by = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
        check(lib.hps_timing_get(i, buf, 128, C.byref(la), C.byref(ms), C.byref(fl), C.byref(by)))
        out.append({"name": buf.value.decode(), "launches": la.value, "ms": ms.value, "flops": fl.value,
                    "bytes": by.value})
    return out
