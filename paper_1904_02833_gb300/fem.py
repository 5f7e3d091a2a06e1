"""Batches of tetrahedral soft links on the GPU (binding of include/femlink.h).

Argument marshalling only: the prediction, the Newton + PCR solve of the element, centre
layer, perimeter and actuation rows and the velocity update all run in the library's
CUDA kernels (fem.cu).  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N


def make_fem_config(s: dict) -> N.FemConfig:
    c = N.FemConfig()
    c.dt = s["dt"]
    c.n_sub = s["n_sub"]
    c.iters = s["iters"]
    c.tol = s["tol"]
    c.pcr_iters = s["pcr_iters"]
    for k in range(3):
        c.gravity[k] = s["gravity"][k]
    return c


def make_fem_params(w: dict):
    n = len(w["youngs"])
    arr = (N.FemLinkParams * n)()
    for i in range(n):
        for f in N.FEM_FLOAT_FIELDS:
            setattr(arr[i], f, float(w[f][i]))
    return arr


class FemSim:
    """n links on one mesh; state lives on the device, work goes to torch's current stream."""

    def __init__(self, mesh: dict, w: dict, settings: dict, device: str = "cuda"):
        self.lib = N.load()
        self.device = torch.device(device)
        self.stream = torch.cuda.current_stream(self.device)
        self._arrays = dict(
            rest=np.ascontiguousarray(mesh["X"], np.float64),
            tets=np.ascontiguousarray(mesh["tets"], np.int32),
            rows=np.ascontiguousarray(mesh["rows"], np.int32).reshape(-1, 2),
            kinds=np.ascontiguousarray(mesh["kinds"], np.int32),
            fixed=np.ascontiguousarray(mesh["fixed"], np.int32))
        a = self._arrays
        m = N.FemMesh()
        m.n_particles, m.n_tets, m.n_rows = len(a["rest"]), len(a["tets"]), len(a["rows"])
        for k in ("rest", "tets", "rows", "kinds", "fixed"):
            setattr(m, k, a[k].ctypes.data_as(ctypes.c_void_p))
        self.P, self.NT, self.ND = m.n_particles, m.n_tets, m.n_rows
        self.n = len(w["youngs"])
        self.cfg = make_fem_config(settings)
        self.prm = make_fem_params(w)
        self.h = ctypes.c_void_p()
        N.check(self.lib.fem_create(ctypes.byref(self.cfg), ctypes.byref(m), self.n, self.prm,
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.h)))

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.fem_destroy(h)
            self.h = ctypes.c_void_p()

    def set_config(self, settings: dict):
        self.cfg = make_fem_config(settings)
        N.check(self.lib.fem_set_config(self.h, ctypes.byref(self.cfg)))

    def step(self, n_frames: int = 1):
        N.check(self.lib.fem_step(self.h, int(n_frames)))

    def set_frame(self, frame: int):
        N.check(self.lib.fem_set_frame(self.h, int(frame)))

    def launch_count(self) -> int:
        n = ctypes.c_int64()
        N.check(self.lib.fem_launch_count(self.h, ctypes.byref(n)))
        return n.value

    def state(self):
        """Positions, velocities [n, P, 3], last-frame residuals [n] and products [n] (numpy)."""
        x = np.zeros((self.n, self.P, 3), np.float32)
        v = np.zeros_like(x)
        r = np.zeros(self.n, np.float32)
        mv = np.zeros(self.n, np.int32)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        N.check(self.lib.fem_get_state(self.h, p(x), p(v), p(r), p(mv), 0))
        return x, v, r, mv

    def state_device(self):
        """The same as torch tensors on the device (copied on the stream)."""
        x = torch.empty((self.n, self.P, 3), dtype=torch.float32, device=self.device)
        v = torch.empty_like(x)
        r = torch.empty(self.n, dtype=torch.float32, device=self.device)
        mv = torch.empty(self.n, dtype=torch.int32, device=self.device)
        N.check(self.lib.fem_get_state(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                       ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(mv.data_ptr()), 1))
        return x, v, r, mv

    def set_state(self, x=None, v=None):
        """Host arrays [n, P, 3] (either may be None)."""
        xs = None if x is None else np.ascontiguousarray(x, np.float32)
        vs = None if v is None else np.ascontiguousarray(v, np.float32)
        p = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
        N.check(self.lib.fem_set_state(self.h, p(xs), p(vs), 0))


def _main():
    """Times a batch of soft links on the synthetic 13-cross-section mesh (one launch per
    frame, CUDA events on the stream):  python -m paper_1904_02833_gb300.fem --links N
    --frames F."""
    import argparse
    import json
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--links", type=int, default=1216)
    ap.add_argument("--frames", type=int, default=3)
    a = ap.parse_args()
    M = W.fem_link_mesh()
    sim = FemSim(M, W.fem_links(a.links, seed=6), W.fem_settings())
    st = torch.cuda.current_stream()
    ms = []
    for _ in range(a.frames):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        sim.step(1)
        e1.record(st)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    x, v, r, mv = sim.state()
    print(json.dumps({"links": a.links, "frames": a.frames, "ms_per_frame": ms, "residual_max": float(r.max()),
                      "products_last_frame": int(mv.max()), "finite": bool(np.isfinite(x).all())}))


if __name__ == "__main__":
    _main()
