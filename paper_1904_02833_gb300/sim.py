"""Python face of the simulator: a thin wrapper over the C-ABI (include/snakesim.h).

Device memory and streams come from PyTorch; every computation runs in the library's
CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _view_bf16(ptr, n, device):
    """A torch tensor over n bf16 values of library-owned device memory."""
    class _Arr:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<i2", "data": (ptr, False),
                                    "version": 3, "strides": None}
    return torch.as_tensor(_Arr(), device=device).view(torch.bfloat16)


def make_params(w: dict):
    n = len(w["n_links"])
    arr = (N.SnakeParams * n)()
    for i in range(n):
        p = arr[i]
        p.n_links = int(w["n_links"][i])
        p.seg_per_link = int(w["seg_per_link"][i])
        p.n_fixed = int(w["n_fixed"][i])
        p.mu_side = float(w["mu_side"][i]) if "mu_side" in w else 0.0
        for f in N.SNAKE_FLOAT_FIELDS:
            setattr(p, f, float(w[f][i]))
    return arr


def make_config(s: dict) -> N.SimConfig:
    c = N.SimConfig()
    c.dt = float(s["dt"])
    c.n_sub = int(s["n_sub"])
    c.iters = int(s["iters"])
    c.tol = float(s["tol"])
    c.omega = float(s["omega"])
    for k in range(3):
        c.gravity[k] = float(s["gravity"][k])
    c.contact = 1 if s["contact"] else 0
    c.warm = int(s["warm"])
    c.beta = float(s.get("beta", 1.0))
    c.latency = int(s.get("latency", 0))
    c.k_inflate = float(s.get("k_inflate", 0.23))
    c.k_deflate = float(s.get("k_deflate", 0.23))
    c.t_p = float(s.get("t_p", 0.085))
    c.p_source = float(s.get("p_source", 1.0))
    c.law_dt = float(s.get("law_dt", 0.0083))
    c.solver = int(s.get("solver", 0))
    c.pcr_iters = int(s.get("pcr_iters", 20))
    c.net_rows = int(s.get("net_rows", 0))
    c.net_every = int(s.get("net_every", 1))
    c.beta_net = float(s.get("beta_net", -1.0))
    return c


def partition(w: dict, parts: int) -> np.ndarray:
    """Contiguous snake ranges of a batch for `parts` GPUs, balanced by node count
    (sim_partition): part p owns snakes [first[p], first[p + 1])."""
    first = np.zeros(parts + 1, np.int32)
    params = make_params(w)
    N.check(N.load().sim_partition(len(w["n_links"]), params, int(parts), first.ctypes.data_as(ctypes.c_void_p)))
    return first


class SnakeSim:
    """A batch of snakes stepped on the GPU by libsnakesim."""

    def __init__(self, w: dict, settings: dict, device: int | None = None, stream=None):
        self.lib = N.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.settings = dict(settings)
        self._cfg = make_config(self.settings)
        self._params = make_params(w)
        self.n = len(w["n_links"])
        h = ctypes.c_void_p()
        N.check(self.lib.sim_create(ctypes.byref(self._cfg), self.n, self._params,
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        nn, nl, ns, si = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        N.check(self.lib.sim_get_info(h, ctypes.byref(nn), ctypes.byref(nl), ctypes.byref(ns),
                                      ctypes.byref(si)))
        self.n_nodes, self.n_links = nn.value, nl.value
        nodes = np.asarray(w["n_links"], np.int64) * np.asarray(w["seg_per_link"]) + 1
        self.node_off = np.concatenate([[0], np.cumsum(nodes)])
        self.link_off = np.concatenate([[0], np.cumsum(w["n_links"])])

    # ------------------------------------------------------------------ stepping
    def step(self, n_steps: int = 1, graph: bool = False):
        f = self.lib.sim_step_graph if graph else self.lib.sim_step
        N.check(f(self.h, int(n_steps)))

    def set_config(self, **kw):
        self.settings.update(kw)
        self._cfg = make_config(self.settings)
        N.check(self.lib.sim_set_config(self.h, ctypes.byref(self._cfg)))

    def set_pressure(self, u):
        """u: tensor [n_links] on the device (or None to return to the gait)."""
        if u is None:
            N.check(self.lib.sim_set_pressure(self.h, None, 1))
            return
        u = u.to(device=self.device, dtype=torch.float32).contiguous()
        N.check(self.lib.sim_set_pressure(self.h, _ptr(u), 1))
        self._ucmd_keep = u

    def kernel_timing(self, enable: bool = True):
        """Record CUDA events around every solver kernel launch of sim_step / split calls."""
        N.check(self.lib.sim_kernel_timing(self.h, 1 if enable else 0))

    def kernel_times(self) -> dict:
        """{(lanes, nodes per lane): (summed ms, launches)} since the last call."""
        ms = np.zeros(12, np.float32)
        n = np.zeros(12, np.int64)
        N.check(self.lib.sim_kernel_times(self.h, ms.ctypes.data_as(ctypes.c_void_p),
                                          n.ctypes.data_as(ctypes.c_void_p)))
        return {(8 << (l // 4), l % 4 + 1): (float(ms[l]), int(n[l])) for l in range(12) if n[l]}

    def autotune(self, n_steps: int = 1):
        N.check(self.lib.sim_autotune(self.h, int(n_steps)))

    def layout(self, nodes: int):
        a, b = ctypes.c_int32(), ctypes.c_int32()
        N.check(self.lib.sim_get_layout(self.h, int(nodes), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_layout(self, nodes: int, lanes: int, npl: int):
        N.check(self.lib.sim_set_layout(self.h, int(nodes), int(lanes), int(npl)))

    @property
    def step_index(self) -> int:
        si = ctypes.c_int64()
        N.check(self.lib.sim_get_info(self.h, None, None, None, ctypes.byref(si)))
        return si.value

    @step_index.setter
    def step_index(self, v: int):
        N.check(self.lib.sim_set_step_index(self.h, int(v)))

    def launches(self) -> int:
        c = ctypes.c_int64()
        N.check(self.lib.sim_launch_count(self.h, ctypes.byref(c)))
        return c.value

    # ------------------------------------------------------------------ state
    def state(self) -> dict:
        """Device copies: pos/vel [nodes, 3], press [links, 2], resid [snakes], iters [snakes]."""
        f32 = dict(device=self.device, dtype=torch.float32)
        out = dict(pos=torch.empty(self.n_nodes, 3, **f32), vel=torch.empty(self.n_nodes, 3, **f32),
                   press=torch.empty(self.n_links, 2, **f32), resid=torch.empty(self.n, **f32),
                   iters=torch.empty(self.n, device=self.device, dtype=torch.int32))
        N.check(self.lib.sim_get_state(self.h, _ptr(out["pos"]), _ptr(out["vel"]), _ptr(out["press"]),
                                       _ptr(out["resid"]), _ptr(out["iters"]), 1))
        return out

    def state_host(self) -> dict:
        """Host numpy copies (synchronises the stream)."""
        out = dict(pos=np.empty((self.n_nodes, 3), np.float32), vel=np.empty((self.n_nodes, 3), np.float32),
                   press=np.empty((self.n_links, 2), np.float32), resid=np.empty(self.n, np.float32),
                   iters=np.empty(self.n, np.int32))
        p = {k: v.ctypes.data_as(ctypes.c_void_p) for k, v in out.items()}
        N.check(self.lib.sim_get_state(self.h, p["pos"], p["vel"], p["press"], p["resid"], p["iters"], 0))
        return out

    def lam(self) -> torch.Tensor:
        out = torch.empty(self.n_nodes, 6, device=self.device, dtype=torch.float32)
        N.check(self.lib.sim_get_lambda(self.h, _ptr(out), 1))
        return out

    def set_state_host(self, pos, vel, press, lam):
        """State from host buffers (numpy arrays or pinned CPU tensors, float32, contiguous)
        through the C-ABI's host path (is_device = 0)."""
        p = [ctypes.c_void_p(a.data_ptr()) if isinstance(a, torch.Tensor) else a.ctypes.data_as(ctypes.c_void_p)
             for a in (pos, vel, press, lam)]
        N.check(self.lib.sim_set_state(self.h, p[0], p[1], p[2], p[3], 0))

    def get_state_host(self, pos, vel, press, lam, resid=None, iters=None):
        """State into host buffers (pinned CPU tensors, float32 / int32 for iters) through
        the C-ABI's host path (is_device = 0); synchronises the stream."""
        N.check(self.lib.sim_get_state(self.h, _ptr(pos), _ptr(vel), _ptr(press), _ptr(resid), _ptr(iters), 0))
        N.check(self.lib.sim_get_lambda(self.h, _ptr(lam), 0))

    def set_state(self, pos=None, vel=None, press=None, lam=None):
        conv = lambda t: None if t is None else torch.as_tensor(t).to(self.device, torch.float32).contiguous()
        pos, vel, press, lam = conv(pos), conv(vel), conv(press), conv(lam)
        N.check(self.lib.sim_set_state(self.h, _ptr(pos), _ptr(vel), _ptr(press), _ptr(lam), 1))

    # ------------------------------------------------------------------ learned warm start
    def set_mlp(self, mlp):
        """Attaches a WarmStartMLP (None detaches); used when warm = 2."""
        N.check(self.lib.sim_set_mlp(self.h, None if mlp is None else mlp.h))
        self._mlp_keep = mlp

    def snapshot_save(self):
        N.check(self.lib.sim_snapshot_save(self.h))

    def snapshot_restore(self):
        N.check(self.lib.sim_snapshot_restore(self.h))

    def split_begin(self):
        N.check(self.lib.sim_split_begin(self.h))

    def split_finish(self):
        N.check(self.lib.sim_split_finish(self.h))

    def features(self, raw: bool = False) -> torch.Tensor:
        """The features [6 * nodes, 32] bf16 in node order (row 6 i + k: node i, row kind k),
        gathered from the library's buffer; raw=True: the buffer itself (zero copy, snakes
        grouped by lane layout, see sim_feature_offsets)."""
        p, r = ctypes.c_void_p(), ctypes.c_int64()
        N.check(self.lib.sim_features(self.h, ctypes.byref(p), ctypes.byref(r)))
        buf = _view_bf16(p.value, r.value * 32, self.device).view(r.value, 32)
        if raw:
            return buf
        first = np.zeros(self.n, np.int32)
        N.check(self.lib.sim_feature_offsets(self.h, first.ctypes.data_as(ctypes.c_void_p)))
        rows = np.diff(self.node_off) * 6
        idx = np.repeat(first.astype(np.int64) - 6 * self.node_off[:-1], rows) + np.arange(6 * self.n_nodes)
        return buf[torch.as_tensor(idx, device=self.device)]

    def training_rows(self, lam_star: torch.Tensor, lam_prev: torch.Tensor, beta: float):
        """Features [rows, 32] bf16 and targets [rows] float of the existing rows of the
        substep in progress (sim_training_rows), on the device."""
        n = ctypes.c_int64()
        N.check(self.lib.sim_training_rows(self.h, None, None, 0.0, None, None, 0, ctypes.byref(n)))
        feat = torch.empty(n.value, 32, dtype=torch.bfloat16, device=self.device)
        target = torch.empty(n.value, dtype=torch.float32, device=self.device)
        a, b = lam_star.contiguous(), lam_prev.contiguous()
        assert a.dtype == b.dtype == torch.float32 and a.numel() == b.numel() == 6 * self.n_nodes
        N.check(self.lib.sim_training_rows(self.h, _ptr(a), _ptr(b), float(beta), _ptr(feat), _ptr(target),
                                           n.value, ctypes.byref(n)))
        self._train_keep = (a, b)
        return feat, target

    def status(self):
        st = np.zeros(self.n, np.int32)
        worst = self.lib.sim_get_status(self.h, st.ctypes.data_as(ctypes.c_void_p))
        return worst, st

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.sim_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
