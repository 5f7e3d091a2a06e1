"""FP64 CPU oracle of the soft-snake constraint solve (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use
this package.  It is independent of the CUDA path: it shares no kernels, headers or
helpers with it and never imports it.  The arithmetic lives in ``snake_oracle.cpp`` (plain
loops, FP64, templated on a dual-number type for parameter derivatives) and
``mlp_oracle.py`` (the warm-start network in FP64); the tetrahedral soft link in
``fem_oracle.cpp`` (wrapped by ``fem.py``).

Parity unpinned: the full locomotion runs (one 4-link snake, batched snakes) have no
closed form and no published trajectory data; only their invariances (momentum, rotation
about the vertical) are pinned, and the GPU path is checked against this oracle.
Everything the oracle computes on the way is pinned by the tests listed in
``snake_oracle.cpp`` and ``fem_oracle.cpp``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("snake_oracle.cpp", "fem_oracle.cpp")]
_LIB = os.path.join(_HERE, "liboracle.so")

PRM_FIELDS = ("L0", "mass", "alpha_s", "alpha_b", "gain", "tau_inf", "tau_def", "mu",
              "damping", "radius", "gait_amp", "gait_freq", "gait_lag", "gait_offset",
              "gait_scale", "gait_alternate", "x0", "y0", "z0", "yaw0", "mu_side")
NK = 6  # multiplier slots per node: stretch, yaw, pitch, contact, friction x, friction y
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with the host compiler."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(map(os.path.getmtime, _SRCS)):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared"] + _SRCS + ["-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.oracle_init.argtypes = [ctypes.c_int, P, P, P, P, P, P, P]
        L.oracle_step.argtypes = [ctypes.c_int, P, P, P, P, P, ctypes.c_longlong, ctypes.c_int,
                                  P, P, P, P, P, P, P, P, P, ctypes.c_int]
        L.oracle_rows.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P, P]
        L.oracle_residual.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P]
        L.oracle_residual.restype = ctypes.c_double
        L.oracle_calib_grad.argtypes = [ctypes.c_int, P, P, P, P, P, ctypes.c_longlong,
                                        ctypes.c_int, P, P, P, P, P, P, P, ctypes.c_int]
        L.oracle_features.argtypes = [ctypes.c_int, P, P, P, P, P, ctypes.c_longlong, P, P, P, P,
                                      P, P]
        L.oracle_mlp_forward.argtypes = [P, ctypes.c_longlong, P, P]
        L.fem_oracle_polar.argtypes = [P, P, P]
        L.fem_oracle_tet.argtypes = [P, P, P, P, P, P]
        L.fem_oracle_step.argtypes = [ctypes.c_int] * 4 + [P] * 7 + [ctypes.c_longlong, ctypes.c_int,
                                                                     P, P, P, P, ctypes.c_int, ctypes.c_int]
        assert L.oracle_nprm() == len(PRM_FIELDS)
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def pack_params(w: dict) -> np.ndarray:
    return np.ascontiguousarray(np.stack([np.asarray(w[f], np.float64) for f in PRM_FIELDS], 1))


def pack_cfg(s: dict) -> np.ndarray:
    g = s["gravity"]
    return np.array([s["dt"], s["n_sub"], s["iters"], s["tol"], s["omega"], g[0], g[1], g[2],
                     1.0 if s["contact"] else 0.0, s["warm"], s.get("beta", 1.0),
                     s.get("latency", 0), s.get("k_inflate", 0.23), s.get("k_deflate", 0.23),
                     s.get("t_p", 0.085), s.get("p_source", 1.0), s.get("law_dt", 0.0083),
                     s.get("solver", 0), s.get("pcr_iters", 20), s.get("net_rows", 0),
                     s.get("net_every", 1), s.get("beta_net", -1.0)], np.float64)


class OracleSim:
    """Batch of snakes advanced by the FP64 oracle; state kept as numpy arrays."""

    def __init__(self, w: dict, settings: dict, n_threads: int | None = None):
        self.w = w
        self.s = dict(settings)
        self.n = len(w["n_links"])
        self.nl = np.ascontiguousarray(w["n_links"], np.int32)
        self.seg = np.ascontiguousarray(w["seg_per_link"], np.int32)
        self.nfix = np.ascontiguousarray(w["n_fixed"], np.int32)
        self.prm = pack_params(w)
        self.cfg = pack_cfg(self.s)
        assert len(self.cfg) == lib().oracle_ncfg()
        if self.s.get("solver", 0) == 1 and self.s["contact"]:
            raise ValueError("the Newton + PCR solver covers contact-free substeps only")
        nn = self.nl.astype(np.int64) * self.seg + 1
        self.node_off = np.concatenate([[0], np.cumsum(nn)])
        self.link_off = np.concatenate([[0], np.cumsum(self.nl)])
        self.n_nodes = int(self.node_off[-1])
        self.n_links = int(self.link_off[-1])
        self.x = np.zeros((self.n_nodes, 3))
        self.v = np.zeros((self.n_nodes, 3))
        self.press = np.zeros((self.n_links, 2))
        self.lam = np.zeros((self.n_nodes, NK))
        self.resid = np.zeros(self.n)
        self.iters = np.zeros(self.n, np.int32)
        self.step_index = 0
        self.n_threads = n_threads or os.cpu_count() or 1
        lib().oracle_init(self.n, _p(self.nl), _p(self.seg), _p(self.prm), _p(self.x),
                          _p(self.v), _p(self.press), _p(self.lam))

    def set_cfg(self, **kw):
        self.s.update(kw)
        self.cfg = pack_cfg(self.s)

    def step(self, n_steps: int = 1, ucmd=None, tip=False, mlp=None):
        """mlp: network parameters (used when the settings' warm = 2)."""
        u = None if ucmd is None else np.ascontiguousarray(ucmd, np.float64)
        tips = np.zeros((n_steps, self.n, 3)) if tip else None
        l0 = None if mlp is None else np.ascontiguousarray(mlp, np.float64)
        lib().oracle_step(self.n, _p(self.nl), _p(self.seg), _p(self.nfix), _p(self.prm),
                          _p(self.cfg), self.step_index, n_steps, _p(self.x), _p(self.v),
                          _p(self.press), _p(self.lam), _p(u), _p(self.resid), _p(self.iters),
                          _p(tips), _p(l0), self.n_threads)
        self.step_index += n_steps
        return tips

    def features(self, ucmd=None):
        """Features [nodes * 6, 24] of substep 0 of the next env-step (state unchanged)."""
        u = None if ucmd is None else np.ascontiguousarray(ucmd, np.float64)
        F = np.zeros((self.n_nodes * NK, 24))
        lib().oracle_features(self.n, _p(self.nl), _p(self.seg), _p(self.nfix), _p(self.prm),
                              _p(self.cfg), self.step_index, _p(self.x), _p(self.v), _p(self.press),
                              _p(self.lam), _p(u), _p(F))
        return F

    def snake_nodes(self, s: int) -> slice:
        return slice(int(self.node_off[s]), int(self.node_off[s + 1]))

    def snake_links(self, s: int) -> slice:
        return slice(int(self.link_off[s]), int(self.link_off[s + 1]))

    def calib_grad(self, n_steps: int, target: np.ndarray):
        """Loss and d loss / d(alpha_b, damping, tau_inf, tau_def, gain) per snake for the
        mean squared tip error against target [n_steps][n][3], from the current state."""
        loss = np.zeros(self.n)
        grad = np.zeros((self.n, 5))
        tg = np.ascontiguousarray(target, np.float64)
        lib().oracle_calib_grad(self.n, _p(self.nl), _p(self.seg), _p(self.nfix), _p(self.prm),
                                _p(self.cfg), self.step_index, n_steps, _p(self.x), _p(self.v),
                                _p(self.press), _p(self.lam), _p(tg), _p(loss), _p(grad),
                                self.n_threads)
        return loss, grad


def mlp_forward(params, feat):
    """Network outputs for features [rows, 24] (bfloat16 operands, FP64 arithmetic)."""
    p = np.ascontiguousarray(params, np.float64)
    f = np.ascontiguousarray(feat, np.float64)
    y = np.zeros(len(f))
    lib().oracle_mlp_forward(_p(p), len(f), _p(f), _p(y))
    return y


def rows(w1: dict, settings: dict, x, xs, press):
    """Row values, existence flags and node gradients of one snake (index 0 of w1)."""
    prm = pack_params(w1)[:1]
    cfg = pack_cfg(settings)
    N = int(w1["n_links"][0] * w1["seg_per_link"][0] + 1)
    c = np.zeros((N, NK))
    g = np.zeros((N, NK, 3, 3))
    on = np.zeros((N, NK), np.int32)
    x = np.ascontiguousarray(x, np.float64)
    xs = np.ascontiguousarray(xs, np.float64)
    press = np.ascontiguousarray(press, np.float64)
    lib().oracle_rows(int(w1["n_links"][0]), int(w1["seg_per_link"][0]), _p(prm), _p(cfg),
                      _p(x), _p(xs), _p(press), _p(c), _p(g), _p(on))
    return c, g, on.astype(bool)


def residual(w1: dict, settings: dict, x, xs, press, lam) -> float:
    """The normalised residual the solver loops stop on, for one snake (index 0 of w1)
    at positions x, substep-start positions xs, pressures press and multipliers lam."""
    prm = pack_params(w1)[:1]
    cfg = pack_cfg(settings)
    arr = [np.ascontiguousarray(a, np.float64) for a in (x, xs, press, lam)]
    return float(lib().oracle_residual(int(w1["n_links"][0]), int(w1["seg_per_link"][0]),
                                       int(w1["n_fixed"][0]), _p(prm), _p(cfg), *map(_p, arr)))
