"""FP64 oracle of the tetrahedral soft link (test infrastructure; see fem_oracle.cpp).

Only the tests, ``__graft_entry__.smoke()`` and the CPU leg of ``bench.py`` use it.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import lib

FEM_PRM_FIELDS = ("youngs", "poisson", "density", "damping", "alpha_inext", "alpha_perim",
                  "alpha_act", "press_amp", "press_freq", "press_phase", "press_offset")


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def pack_params(w: dict) -> np.ndarray:
    return np.ascontiguousarray(np.stack([np.asarray(w[f], np.float64) for f in FEM_PRM_FIELDS], 1))


def pack_cfg(s: dict) -> np.ndarray:
    g = s["gravity"]
    return np.array([s["dt"], s["n_sub"], s["iters"], s["tol"], s["pcr_iters"], g[0], g[1], g[2]],
                    np.float64)


def polar(F):
    """Polar decomposition F = R S of one 3x3 matrix."""
    F = np.ascontiguousarray(F, np.float64)
    R, S = np.zeros((3, 3)), np.zeros((3, 3))
    lib().fem_oracle_polar(_p(F), _p(R), _p(S))
    return R, S


def tet(Xr, x):
    """Strain rows of one element: rest vertices Xr [4, 3], current x [4, 3] -> strains c [6]
    (Voigt xx yy zz yz xz xy, tensor shears), gradients G [6, 4, 3] (R fixed), R, volume."""
    Xr = np.ascontiguousarray(Xr, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    c, G, R, vol = np.zeros(6), np.zeros((6, 4, 3)), np.zeros((3, 3)), np.zeros(1)
    lib().fem_oracle_tet(_p(Xr), _p(x), _p(c), _p(G), _p(R), _p(vol))
    return c, G, R, float(vol[0])


class OracleFem:
    """Batch of links on one mesh advanced by the oracle; state [n, P, 3] numpy arrays."""

    def __init__(self, mesh: dict, w: dict, settings: dict, n_threads: int | None = None):
        L = lib()
        assert L.fem_oracle_nprm() == len(FEM_PRM_FIELDS) and L.fem_oracle_ncfg() == 8
        self.mesh = {k: np.ascontiguousarray(v) for k, v in mesh.items()}
        self.Xr = np.ascontiguousarray(mesh["X"], np.float64)
        self.tets = np.ascontiguousarray(mesh["tets"], np.int32)
        self.rows = np.ascontiguousarray(mesh["rows"], np.int32)
        self.kinds = np.ascontiguousarray(mesh["kinds"], np.int32)
        self.fixed = np.ascontiguousarray(mesh["fixed"], np.int32)
        self.P, self.NT, self.ND = len(self.Xr), len(self.tets), len(self.rows)
        self.w = w
        self.s = dict(settings)
        self.prm = pack_params(w)
        self.n = len(self.prm)
        self.x = np.ascontiguousarray(np.broadcast_to(self.Xr, (self.n, self.P, 3)), np.float64).copy()
        self.v = np.zeros((self.n, self.P, 3))
        self.resid = np.zeros(self.n)
        self.mv = np.zeros(self.n, np.int32)
        self.frame = 0
        self.n_threads = n_threads or os.cpu_count() or 1

    def step(self, n_frames: int = 1, fp32: bool = False):
        cfg = pack_cfg(self.s)
        lib().fem_oracle_step(self.n, self.P, self.NT, self.ND, _p(self.Xr), _p(self.tets), _p(self.rows),
                              _p(self.kinds), _p(self.fixed), _p(self.prm), _p(cfg), self.frame, n_frames,
                              _p(self.x), _p(self.v), _p(self.resid), _p(self.mv), self.n_threads,
                              1 if fp32 else 0)
        self.frame += n_frames
