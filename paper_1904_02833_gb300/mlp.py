"""Warm-start network: thin wrapper over the mlp_* entry points of include/snakesim.h, and
the data logging / training loop that uses only those entry points and the simulator's
substep-by-substep stepping."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N

N_PARAMS = N.MLP_NUM_PARAMS


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation: W1 [128][24], b1, W2 [128][128], b2, w3 [128], b3."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2.0 / 24), 128 * 24), np.zeros(128),
             rng.normal(0, np.sqrt(2.0 / 128), 128 * 128), np.zeros(128),
             rng.normal(0, np.sqrt(1.0 / 128), 128), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class WarmStartMLP:
    """24 -> 128 -> 128 -> 1 SiLU network on the tensor cores (BF16, FP32 accumulate)."""

    def __init__(self, params=None, device=None, stream=None):
        self.lib = N.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        N.check(self.lib.mlp_create(ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        self.set_params(init_params() if params is None else params)
        self._loss = torch.zeros(1, device=self.device)

    def set_params(self, p):
        t = torch.as_tensor(np.asarray(p, np.float32)).to(self.device).contiguous()
        assert t.numel() == N_PARAMS
        N.check(self.lib.mlp_set_params(self.h, _p(t), 1))
        torch.cuda.current_stream(self.device).synchronize()

    def params(self) -> np.ndarray:
        t = torch.empty(N_PARAMS, device=self.device)
        N.check(self.lib.mlp_get_params(self.h, _p(t), 1))
        return t.cpu().numpy()

    def forward(self, feat: torch.Tensor) -> torch.Tensor:
        """feat: [rows, 32] bf16 on the device -> [rows] float32."""
        assert feat.dtype == torch.bfloat16 and feat.shape[1] == 32 and feat.is_contiguous()
        out = torch.empty(feat.shape[0], device=self.device)
        N.check(self.lib.mlp_forward(self.h, _p(feat), feat.shape[0], _p(out)))
        return out

    def grad(self, feat, target, scale):
        g = torch.empty(N_PARAMS, device=self.device)
        loss = torch.empty(1, device=self.device)
        N.check(self.lib.mlp_grad(self.h, _p(feat), _p(target), feat.shape[0], float(scale), _p(g),
                                  _p(loss)))
        return float(loss.item()), g

    def train_step(self, feat, target, lr):
        N.check(self.lib.mlp_train_step(self.h, _p(feat), _p(target), feat.shape[0], float(lr),
                                        _p(self._loss)))
        return self._loss

    def check(self):
        N.check(self.lib.mlp_check(self.h))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.mlp_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pad_features(f24: torch.Tensor) -> torch.Tensor:
    """[rows, 24] float -> [rows, 32] bf16 (zero padded), the layout the kernels read."""
    out = torch.zeros(f24.shape[0], 32, dtype=torch.bfloat16, device=f24.device)
    out[:, :24] = f24.to(torch.bfloat16)
    return out


def collect(sim, n_steps: int, substeps=None, every: int = 1, target_tol: float = 1e-6,
            target_iters: int = 20000, skip: float | None = None, target_warm: int = 0):
    """Logs training pairs along the simulator's own trajectory (its current settings:
    tolerance, warm start and, in the learned mode, its network), so the features carry
    the previous multipliers the deployed solver produces.  At each logged substep the
    substep is also solved from the same start to `target_tol` on a snapshot (from zero
    multipliers, target_warm = 0, or from beta times the previous ones, target_warm = 1);
    sim_training_rows then writes the features and target (the multiplier reached there
    minus beta times the previous multiplier, over m g h^2: the network predicts the
    correction to the beta-weighted previous multiplier) of every existing row whose
    features the simulator writes (all kinds; in the learned warm start, the kinds the
    network predicts).  Returns bf16 features [n, 32] and float targets [n], on the
    device."""
    w = dict(sim.settings)
    n_sub = w["n_sub"]
    beta = float(w.get("beta", 1.0)) if skip is None else float(skip)
    target_cfg = dict(w, tol=float(target_tol), iters=int(target_iters), warm=int(target_warm), beta=beta)
    feats, targets = [], []
    substeps = list(range(n_sub)) if substeps is None else list(substeps)
    for k in range(n_steps):
        log = (k % every) == 0
        sim.split_begin()
        for s in range(n_sub):
            if log and s in substeps:
                lam_prev = sim.lam().clone()
                sim.snapshot_save()
                sim.set_config(**target_cfg)
                sim.split_finish()
                lam_star = sim.lam().clone()
                sim.snapshot_restore()
                sim.set_config(**w)
                f, t = sim.training_rows(lam_star, lam_prev, beta)
                feats.append(f)
                targets.append(t)
            sim.split_finish()
    return torch.cat(feats), torch.cat(targets)


def train(mlp: WarmStartMLP, feat, target, epochs: int = 10, batch: int = 16384, lr: float = 1e-3,
          seed: int = 0, lr_final: float = 1e-4):
    """Adam on the mean squared error over shuffled mini-batches; returns the loss trace."""
    g = torch.Generator(device=feat.device)
    g.manual_seed(seed)
    n = feat.shape[0]
    steps = epochs * max(1, n // batch)
    losses = []
    it = 0
    for e in range(epochs):
        perm = torch.randperm(n, device=feat.device, generator=g)
        for b in range(max(1, n // batch)):
            idx = perm[b * batch:(b + 1) * batch]
            frac = it / max(1, steps - 1)
            cur = lr * (lr_final / lr) ** frac
            loss = mlp.train_step(feat[idx].contiguous(), target[idx].contiguous(), cur)
            if b == 0:
                losses.append(float(loss.item()))
            it += 1
    mlp.check()
    return losses


def train_warm_start(n_snakes: int = 1024, seeds=None, rounds: int = 2, settle: int = 6,
                     steps: int = 10, tol: float = 1e-4, epochs0: int = 20, epochs: int = 10,
                     batch: int = 16384, log=None, make_batch=None, skip: float = 0.5,
                     target_warm: int = 1, deploy: dict | None = None):
    """Trains the warm-start network on data the plain solver generates.

    Round 0 follows cold-start trajectories; every later round follows trajectories of
    the learned warm start itself (on new seeds), so the network sees the previous
    multipliers it will meet when deployed.  Targets: at a logged substep, the
    multipliers the plain solver reaches at `tol` from the same start (cold, or from
    `skip` times the previous multipliers with target_warm = 1), minus `skip` times the
    previous multipliers (the learned warm start adds the network's output to the
    previous multipliers weighted by beta = skip).  `deploy` (net_rows, net_every and
    beta, the weight of the previous multipliers at the substeps without the network)
    sets the row kinds and period the learned trajectories use the network on, and the
    logged substeps are then network substeps, so that the previous multipliers in the
    data come from the schedule the network will be deployed with.  All simulation and
    all training run in the library's kernels.  Returns the network and a record of the
    rounds."""
    import workloads as W  # seeded parameter generator (no simulation arithmetic)
    from .sim import SnakeSim

    make_batch = make_batch or (lambda n, seed: W.batched(n=n, seed=seed))
    seeds = list(seeds) if seeds is not None else W.training_seeds(rounds + 2)
    net = WarmStartMLP()
    feats, targets, record = [], [], []
    deploy = dict(deploy or {})
    every = int(deploy.get("net_every", 1))

    def gather(seed, learned):
        sim = SnakeSim(make_batch(n_snakes, seed), W.solver_settings(iters=5000, tol=tol, warm=0))
        sim.step(settle)
        if learned:
            sim.set_mlp(net)
            cfg = dict(warm=2, beta=skip)
            cfg.update(deploy)
            sim.set_config(beta_net=skip, **cfg)
            sim.step(2)
        logged = (0, 7, 14)
        if learned:  # the network substeps nearest to those
            last = (sim.settings["n_sub"] - 1) // every * every
            logged = tuple(sorted({min(round(s / every) * every, last) for s in logged}))
        f, t = collect(sim, steps, substeps=logged, every=2, target_tol=tol, skip=skip,
                       target_warm=target_warm)
        sim.close()
        return f, t

    for r in range(rounds + 1):
        use = seeds[:2] if r == 0 else [seeds[1 + r]]
        for seed in use:
            f, t = gather(seed, learned=r > 0)
            feats.append(f)
            targets.append(t)
        F, T = torch.cat(feats), torch.cat(targets)
        losses = train(net, F, T, epochs=epochs0 if r == 0 else epochs, batch=batch,
                       lr=2e-3 if r == 0 else 1e-3)
        record.append({"round": r, "rows": int(F.shape[0]), "loss_first": losses[0],
                       "loss_last": losses[-1]})
        if log:
            log(record[-1])
    return net, record
