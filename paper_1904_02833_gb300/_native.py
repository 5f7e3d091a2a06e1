"""ctypes binding of libsnakesim.so (the C-ABI declared in include/snakesim.h and
include/femlink.h).

Argument marshalling only: every step of the simulation runs in the library's CUDA
kernels.  Loading fails loudly when the library has not been built; there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsnakesim.so")

SIM_OK, SIM_NOT_CONVERGED, SIM_EINVAL, SIM_ECUDA, SIM_ENOMEM, SIM_ENAN = 0, 1, -1, -2, -3, -4
WARM_COLD, WARM_PREVIOUS, WARM_LEARNED = 0, 1, 2


class SimConfig(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("n_sub", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("tol", ctypes.c_float), ("omega", ctypes.c_float),
                ("gravity", ctypes.c_float * 3), ("contact", ctypes.c_int32),
                ("warm", ctypes.c_int32), ("beta", ctypes.c_float),
                ("latency", ctypes.c_int32), ("k_inflate", ctypes.c_float),
                ("k_deflate", ctypes.c_float), ("t_p", ctypes.c_float),
                ("p_source", ctypes.c_float), ("law_dt", ctypes.c_float),
                ("solver", ctypes.c_int32), ("pcr_iters", ctypes.c_int32),
                ("net_rows", ctypes.c_int32), ("net_every", ctypes.c_int32), ("beta_net", ctypes.c_float)]


SNAKE_FLOAT_FIELDS = ("L0", "mass", "alpha_s", "alpha_b", "gain", "tau_inf", "tau_def", "mu",
                      "damping", "radius", "gait_amp", "gait_freq", "gait_lag", "gait_offset",
                      "gait_scale", "gait_alternate", "x0", "y0", "z0", "yaw0")


class SnakeParams(ctypes.Structure):
    _fields_ = ([("n_links", ctypes.c_int32), ("seg_per_link", ctypes.c_int32),
                 ("n_fixed", ctypes.c_int32), ("mu_side", ctypes.c_float)]
                + [(f, ctypes.c_float) for f in SNAKE_FLOAT_FIELDS])


assert ctypes.sizeof(SnakeParams) == 96
assert ctypes.sizeof(SimConfig) == 96


# tetrahedral soft link (include/femlink.h)
class FemConfig(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("n_sub", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("tol", ctypes.c_float), ("pcr_iters", ctypes.c_int32), ("gravity", ctypes.c_float * 3)]


FEM_FLOAT_FIELDS = ("youngs", "poisson", "density", "damping", "alpha_inext", "alpha_perim", "alpha_act",
                    "press_amp", "press_freq", "press_phase", "press_offset")


class FemLinkParams(ctypes.Structure):
    _fields_ = [(f, ctypes.c_float) for f in FEM_FLOAT_FIELDS]


class FemMesh(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int32), ("n_tets", ctypes.c_int32), ("n_rows", ctypes.c_int32),
                ("rest", ctypes.c_void_p), ("tets", ctypes.c_void_p), ("rows", ctypes.c_void_p),
                ("kinds", ctypes.c_void_p), ("fixed", ctypes.c_void_p)]

_lib = None
P = ctypes.c_void_p
H = ctypes.c_void_p
I64P = ctypes.POINTER(ctypes.c_int64)
I32P = ctypes.POINTER(ctypes.c_int32)

SIGNATURES = {
    "sim_create": ([ctypes.POINTER(SimConfig), ctypes.c_int, ctypes.POINTER(SnakeParams), P,
                    ctypes.POINTER(H)]),
    "sim_set_config": [H, ctypes.POINTER(SimConfig)],
    "sim_set_pressure": [H, P, ctypes.c_int],
    "sim_step": [H, ctypes.c_int],
    "sim_step_graph": [H, ctypes.c_int],
    "sim_get_state": [H, P, P, P, P, P, ctypes.c_int],
    "sim_set_state": [H, P, P, P, P, ctypes.c_int],
    "sim_get_lambda": [H, P, ctypes.c_int],
    "sim_get_info": [H, I64P, I64P, I32P, I64P],
    "sim_set_step_index": [H, ctypes.c_int64],
    "sim_device_state": [H, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                         ctypes.POINTER(P)],
    "sim_get_status": [H, P],
    "sim_autotune": [H, ctypes.c_int],
    "sim_get_layout": [H, ctypes.c_int, I32P, I32P],
    "sim_set_layout": [H, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "sim_launch_count": [H, I64P],
    "sim_kernel_timing": [H, ctypes.c_int],
    "sim_feature_offsets": [H, P],
    "sim_kernel_times": [H, P, P],
    "sim_destroy": [H],
    "sim_fp32_fma_probe": [P, ctypes.c_int, ctypes.c_int, P],
    "sim_set_mlp": [H, H],
    "sim_snapshot_save": [H],
    "sim_calib_forward": [H, P, ctypes.c_int, ctypes.c_int, P],
    "sim_calib_backward": [H, P, P],
    "sim_snapshot_restore": [H],
    "sim_split_begin": [H],
    "sim_split_finish": [H],
    "sim_features": [H, ctypes.POINTER(P), I64P],
    "sim_training_rows": [H, P, P, ctypes.c_float, P, P, ctypes.c_int64, I64P],
    "sim_partition": [ctypes.c_int, ctypes.POINTER(SnakeParams), ctypes.c_int, P],
    "mlp_create": [P, ctypes.POINTER(H)],
    "mlp_set_params": [H, P, ctypes.c_int],
    "mlp_get_params": [H, P, ctypes.c_int],
    "mlp_forward": [H, P, ctypes.c_int64, P],
    "mlp_grad": [H, P, P, ctypes.c_int64, ctypes.c_float, P, P],
    "mlp_train_step": [H, P, P, ctypes.c_int64, ctypes.c_float, P],
    "mlp_check": [H],
    "mlp_wait_selftest": [ctypes.c_uint32, P, ctypes.POINTER(ctypes.c_int32)],
    "mlp_destroy": [H],
    "mlp_forward_noalloc": [P, ctypes.c_int32, P, ctypes.c_int64, P, P],
    "fem_create": [ctypes.POINTER(FemConfig), ctypes.POINTER(FemMesh), ctypes.c_int,
                   ctypes.POINTER(FemLinkParams), P, ctypes.POINTER(H)],
    "fem_set_config": [H, ctypes.POINTER(FemConfig)],
    "fem_step": [H, ctypes.c_int],
    "fem_get_state": [H, P, P, P, P, ctypes.c_int],
    "fem_set_state": [H, P, P, ctypes.c_int],
    "fem_set_frame": [H, ctypes.c_int64],
    "fem_launch_count": [H, I64P],
    "fem_destroy": [H],
}
MLP_NUM_PARAMS = 19841


class SimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("snakesim status %d: %s" % (status, msg))
        self.status = status


def load():
    """Loads libsnakesim.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libsnakesim.so is not built (%s); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.sim_last_error.argtypes = []
        L.sim_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def check(status, ok=(SIM_OK,)):
    if status in ok:
        return status
    msg = load().sim_last_error().decode(errors="replace")
    raise SimError(status, msg)
