"""ctypes loader for libadjwt.so with the prototypes of include/adjwt.h.

The library is built in-tree by build_ext.py.  There is no fallback: if the
shared object is missing or fails to load, every call raises.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# ADJWT_LIBRARY selects another build of the same library (e.g. the checked
# build made by build_ext.build(checked=True)); the default is the in-tree one.
LIB_PATH = os.environ.get("ADJWT_LIBRARY") or os.path.join(HERE, "libadjwt.so")

I64 = C.c_int64
VP = C.c_void_p
SZ = C.c_size_t
DP = C.POINTER(C.c_double)


class FistaProblem(C.Structure):
    _fields_ = [("wt", VP), ("blur", VP), ("b", VP), ("lam", C.c_double), ("lipschitz", C.c_double),
                ("gradient", C.c_int)]


class FistaState(C.Structure):
    _fields_ = [("x", VP), ("y", VP), ("t", C.c_double), ("k", I64)]


# name -> (restype, argtypes)
PROTOTYPES = {
    "adjwt_last_error": (C.c_char_p, []),
    "adjwt_version": (C.c_int, []),
    "adjwt_device_status": (C.c_int, [C.POINTER(C.c_int), C.c_int]),
    "adjwt_wait_selftest": (C.c_int, [C.c_int, VP]),
    "adjwt_wt_plan_create": (C.c_int, [C.POINTER(VP), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "adjwt_wt_plan_destroy": (None, [VP]),
    "adjwt_wt_layout": (C.c_int, [VP, C.POINTER(I64), C.POINTER(I64), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "adjwt_wt_workspace_size": (SZ, [VP]),
    "adjwt_wt_filters": (C.c_int, [VP, DP, DP, DP, DP, C.POINTER(C.c_int)]),
    "wt_synth": (C.c_int, [VP, VP, VP, VP, SZ, VP]),
    "wt_synth_adjoint": (C.c_int, [VP, VP, VP, VP, SZ, VP]),
    "wt_analysis": (C.c_int, [VP, VP, VP, VP, SZ, VP]),
    "adjwt_blur_plan_create": (C.c_int, [C.POINTER(VP), C.c_int, C.c_int, DP, C.c_int, DP, C.c_int, C.c_int]),
    "adjwt_blur_plan_destroy": (None, [VP]),
    "adjwt_blur_image_pitch": (C.c_int, [VP]),
    "adjwt_blur_workspace_size": (SZ, [VP]),
    "blur": (C.c_int, [VP, VP, VP, VP]),
    "blur_adjoint": (C.c_int, [VP, VP, VP, VP]),
    "blur_normal": (C.c_int, [VP, VP, VP, VP, VP, VP, SZ, VP]),
    "adjwt_conv_adjoint_workspace_size": (SZ, [C.c_int, I64, C.c_int]),
    "conv_adjoint": (C.c_int, [C.c_int, I64, C.c_int, VP, VP, VP, VP, VP, VP, SZ, VP]),
    "conv_residual": (C.c_int, [C.c_int, I64, C.c_int, VP, VP, VP, VP, VP]),
    "conv_adjoint_noalloc": (C.c_int, [C.c_int, I64, C.c_int, VP, VP, VP, VP, VP, VP]),
    "adjwt_conv_gradient_workspace_size": (SZ, [C.c_int, I64, C.c_int]),
    "conv_gradient": (C.c_int, [C.c_int, I64, C.c_int, VP, VP, VP, VP, VP, VP, VP, SZ, VP]),
    "adjwt_fista_workspace_size": (SZ, [C.POINTER(FistaProblem)]),
    "fista_step": (C.c_int, [C.POINTER(FistaProblem), C.POINTER(FistaState), VP, SZ, DP, VP]),
    "adjwt_bce_gradient_workspace_size": (SZ, [C.c_int, I64, C.c_int]),
    "bce_gradient": (C.c_int, [C.c_int, I64, C.c_int, VP, VP, VP, C.c_double, C.c_double, VP, VP, VP, SZ, VP]),
    "fista_step_device": (C.c_int, [C.POINTER(FistaProblem), VP, VP, VP, SZ, VP, VP]),
    "adjwt_fista_device_reset": (C.c_int, [C.POINTER(FistaProblem), VP, SZ, VP]),
    "adjwt_fista_batch_workspace_size": (SZ, [C.c_int, C.POINTER(FistaProblem)]),
    "adjwt_fista_batch_create": (C.c_int, [C.POINTER(VP), C.c_int, C.POINTER(FistaProblem), C.POINTER(VP),
                                           C.POINTER(VP), VP, SZ]),
    "adjwt_fista_batch_destroy": (None, [VP]),
    "adjwt_fista_batch_reset": (C.c_int, [VP, VP]),
    "adjwt_fista_batch_set_iteration": (C.c_int, [VP, I64, VP]),
    "adjwt_fista_batch_run": (C.c_int, [VP, C.c_int, VP]),
    "adjwt_fista_batch_objective": (C.c_int, [VP, VP, VP]),
    "adjwt_fista_batch_wait_selftest": (C.c_int, [VP, VP]),
    "adjwt_fista_batch_info": (C.c_int, [VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "adjwt_wt_plan_set_tma": (C.c_int, [VP, C.c_int, C.c_int, C.c_int]),
    "adjwt_wt_plan_uses_tma": (C.c_int, [VP, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "adjwt_wt_plan_set_tma_ctas": (C.c_int, [VP, C.c_int, C.c_int, C.c_int]),
    "adjwt_wt_plan_tma_ctas": (C.c_int, [VP, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "adjwt_wt_plan_set_level_chain": (C.c_int, [VP, C.c_int]),
    "adjwt_wt_plan_chain_start": (C.c_int, [VP, C.c_int, C.POINTER(C.c_int)]),
    "adjwt_wt_plan_autotune": (C.c_int, [VP, C.c_int, C.POINTER(C.c_int), VP]),
    "adjwt_gaussian_taps": (C.c_int, [C.c_int, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "adjwt_fista_momentum": (C.c_int, [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_float)]),
    "adjwt_reduce_workspace_size": (SZ, []),
    "adjwt_axpby": (C.c_int, [I64, C.c_float, VP, C.c_float, VP, VP, VP]),
    "adjwt_soft_threshold": (C.c_int, [C.c_int64, VP, C.c_double, VP, VP]),
    "adjwt_dot": (C.c_int, [C.c_int, I64, I64, VP, VP, VP, VP, SZ, VP]),
    "fista_prox_vjp": (C.c_int, [I64, VP, VP, VP, VP, VP, SZ, VP]),
    "adjwt_fista_vjp_workspace_size": (SZ, [C.POINTER(FistaProblem)]),
    "adjwt_cnn_param_count": (SZ, []),
    "adjwt_cnn_packed_bytes": (SZ, []),
    "adjwt_cnn_activation_bytes": (SZ, [C.c_int, C.c_int, C.c_int]),
    "adjwt_cnn_workspace_size": (SZ, [C.c_int, C.c_int, C.c_int]),
    "adjwt_cnn_wgrad_workspace_size": (SZ, []),
    "cnn_pack": (C.c_int, [VP, VP, VP]),
    "cnn_forward": (C.c_int, [C.c_int, C.c_int, C.c_int, VP, I64, VP, VP, VP, VP, VP]),
    "cnn_backward": (C.c_int, [C.c_int, C.c_int, C.c_int, VP, VP, VP, I64, VP, VP, VP, VP, VP, VP, SZ, VP]),
    "cnn_adam": (C.c_int, [I64, VP, VP, VP, VP, I64, C.c_double, C.c_double, C.c_double, C.c_double, VP]),
    "cnn_conv32": (C.c_int, [C.c_int, C.c_int, C.c_int, VP, VP, VP, C.c_int, VP, VP, VP]),
    "cnn_conv32_wgrad": (C.c_int, [C.c_int, C.c_int, C.c_int, VP, VP, VP, VP, VP, SZ, VP]),
    "fista_vjp_step": (C.c_int, [C.POINTER(FistaProblem), VP, VP, VP, VP, C.c_double, VP, VP, VP, VP, VP, VP, SZ,
                                 VP]),
    "adjwt_fista_objective": (C.c_int, [C.POINTER(FistaProblem), VP, VP, SZ, DP, VP]),
    "adjwt_fista_lipschitz": (C.c_int, [C.POINTER(FistaProblem), VP, C.c_int, VP, SZ, DP, VP]),
    "adjwt_trace_enable": (C.c_int, [C.c_int]),
    "adjwt_trace_reset": (C.c_int, []),
    "adjwt_trace_count": (C.c_int, []),
    "adjwt_trace_get": (C.c_int, [C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "adjwt_trace_span": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_float)]),
    "adjwt_trace_set_level": (C.c_int, [C.c_int]),
    "adjwt_fp32_fma_peak": (C.c_int, [C.POINTER(C.c_double), VP]),
}

_lib = None


class AdjwtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"adjwt error {code}: {msg}")
        self.code = code


def load(path=LIB_PATH):
    """Load libadjwt.so and attach the prototypes (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1707_02018_gb300.build_ext.build() "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc):
    if rc != 0:
        raise AdjwtError(rc, load().adjwt_last_error().decode())
    return rc
