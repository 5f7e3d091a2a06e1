"""The tensor-core warm-start network and the learned warm start, through the C-ABI,
against the oracle.

Tolerances: the kernels read bfloat16 operands (as the oracle emulates) and evaluate
SiLU with the hardware tanh approximation (relative error ~2^-11 of tanh, i.e. an absolute
error ~2.5e-4 |z| of silu(z)); the inference kernel evaluates the first layer's SiLU in
bfloat16 pairs (its result is rounded to bfloat16 for the second GEMM in any case: one
to two bfloat16 units of the last place instead of half of one); accumulation is FP32
against the oracle's FP64.  Outputs: 5e-3 of the output scale; gradients: 2e-2 of each
block's largest entry against the bfloat16-emulating oracle, 6e-2 against the plain FP64
gradient (the bfloat16 bound).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp_oracle as M
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_02833_gb300.build import build
    build()
    torch.cuda.set_device(0)


def mlp(params=None):
    from paper_1904_02833_gb300.mlp import WarmStartMLP
    return WarmStartMLP(params)


def feats(rows, seed):
    rng = np.random.default_rng(seed)
    f = rng.normal(scale=1.0, size=(rows, 24))
    f[:, :6] = 0
    f[np.arange(rows), rng.integers(0, 6, rows)] = 1.0
    return f


def to_dev(f):
    from paper_1904_02833_gb300.mlp import pad_features
    return pad_features(torch.tensor(f, dtype=torch.float32, device="cuda"))


@pytest.mark.parametrize("rows", [1, 127, 1000, 40000])
def test_forward_matches_oracle(rows):
    p = M.init_params(5)
    p[M.N_PARAMS - 1] = 0.3
    f = feats(rows, rows)
    net = mlp(p)
    y = net.forward(to_dev(f)).cpu().numpy()
    ref = oracle.mlp_forward(p, M.bf16(f))
    scale = np.abs(ref).mean() + 1e-3
    assert np.abs(y - ref).max() <= 5e-3 * max(scale, np.abs(ref).max())


def test_gradient_matches_oracle():
    rows = 3000
    p = M.init_params(6)
    f = feats(rows, 9)
    rng = np.random.default_rng(2)
    t = rng.normal(size=rows)
    net = mlp(p)
    L, g = net.grad(to_dev(f), torch.tensor(t, dtype=torch.float32, device="cuda"), 1.0 / rows)
    g = g.cpu().numpy()
    L_ref, g_ref = M.loss_and_grad(p, M.bf16(f), t, 1.0 / rows, bf16_ops=True)
    _, g_fp64 = M.loss_and_grad(p, M.bf16(f), t, 1.0 / rows, bf16_ops=False)
    assert L == pytest.approx(L_ref, rel=5e-3)
    o = 0
    for name, shape in M.SIZES:
        n = int(np.prod(shape))
        a, b, c = g[o:o + n], g_ref[o:o + n], g_fp64[o:o + n]
        assert np.abs(a - b).max() <= 2e-2 * np.abs(b).max() + 1e-7, name
        assert np.abs(a - c).max() <= 6e-2 * np.abs(c).max() + 1e-7, name
        o += n


def test_training_reduces_loss_on_a_smooth_target():
    rows = 65536
    f = feats(rows, 11)
    t = np.tanh(f[:, 6] - 0.5 * f[:, 7]) + 0.3 * f[:, 13] * f[:, 0]
    from paper_1904_02833_gb300.mlp import train
    net = mlp(M.init_params(7))
    fd = to_dev(f)
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    losses = train(net, fd, td, epochs=20, batch=4096, lr=2e-3)
    assert losses[-1] < 0.1 * losses[0]
    # the trained parameters reproduce their own loss on the oracle
    p = net.params().astype(np.float64)
    y = oracle.mlp_forward(p, M.bf16(f[:2000]))
    assert np.mean((y - t[:2000]) ** 2) < 0.15 * losses[0]


def test_features_match_oracle():
    from paper_1904_02833_gb300.sim import SnakeSim
    w = W.batched(n=24, seed=31, links=(1, 8))
    s = W.solver_settings(iters=10)
    g, o = SnakeSim(w, s), oracle.OracleSim(w, s)
    g.step(3)
    o.step(3)
    g.split_begin()
    fg = g.features().float().cpu().numpy()[:, :24]
    fo = o.features()
    assert not fg[:, 24:].any() if fg.shape[1] > 24 else True
    err = np.abs(fg - fo)
    # geometry and kinematics: bf16 rounding of the FP32 values
    assert (err[:, :23] <= 1e-2 * np.abs(fo[:, :23]) + 2e-3).all(), err[:, :23].max()
    # previous multipliers of an unconverged (10-update) solve: FP32 vs FP64 differences
    # reach ~5e-3 of the largest multiplier
    assert (err[:, 23] <= 5e-3 * np.abs(fo[:, 23]).max() + 1e-2 * np.abs(fo[:, 23])).all()
    # finishing the substeps splits the env-step without changing it
    for _ in range(s["n_sub"]):
        g.split_finish()
    o.step(1)
    st = g.state_host()
    assert np.abs(st["pos"] - o.x).max() <= 1e-5 * np.abs(o.x).max()


def test_split_stepping_matches_fused_stepping():
    """The same arithmetic in two kernels: equal update counts, states equal to FP32
    rounding (the compiler may contract multiply-adds differently in the two)."""
    from paper_1904_02833_gb300.sim import SnakeSim
    w = W.batched(n=40, seed=32, links=(1, 8))
    for warm in (0, 1):
        s = W.solver_settings(iters=10, warm=warm)
        a, b = SnakeSim(w, s), SnakeSim(w, s)
        a.step(2)
        for _ in range(2):
            b.split_begin()
            for _ in range(s["n_sub"]):
                b.split_finish()
        sa, sb = a.state_host(), b.state_host()
        assert np.array_equal(sa["iters"], sb["iters"])
        assert np.array_equal(sa["press"], sb["press"])
        tol_x = 1e-6 * np.abs(sa["pos"]).max()
        assert np.abs(sa["pos"] - sb["pos"]).max() <= tol_x
        # velocities are the last substep's displacement over h: the same bound over h
        h = s["dt"] / s["n_sub"]
        assert np.abs(sa["vel"] - sb["vel"]).max() <= tol_x / h


@pytest.mark.parametrize("net_rows,net_every,beta", [(0, 1, 0.5), (1, 1, 0.5), (0, 4, 0.5), (1, 7, 0.5),
                                                     (0, 20, 0.5), (2, 1, 0.5), (2, 3, 0.5), (1, 3, 0.75)])
def test_learned_mode_matches_oracle(net_rows, net_every, beta):
    """Same network parameters on both sides; fixed iteration count; the network on all
    row kinds or the bilateral ones, at every substep or every net_every-th (the launches
    then finish several substeps each), its prediction on 0.5 lambda_prev and the other
    rows and substeps from beta lambda_prev."""
    from paper_1904_02833_gb300.sim import SnakeSim
    w = W.batched(n=16, seed=33, links=(1, 8))
    p = M.init_params(8) * 0.5
    s = W.solver_settings(iters=10, warm=1, beta=0.5)
    g, o = SnakeSim(w, s), oracle.OracleSim(w, s)
    g.step(2)
    o.step(2)
    net = mlp(p)
    g.set_mlp(net)
    g.set_config(warm=2, net_rows=net_rows, net_every=net_every, beta=beta, beta_net=0.5)
    o.set_cfg(warm=2, net_rows=net_rows, net_every=net_every, beta=beta, beta_net=0.5)
    g.step(1)
    o.step(1, mlp=p)
    # the parity bounds of tests/test_gpu_parity.py, with the floor of a solve started by
    # the bfloat16 network
    from test_gpu_parity import compare
    compare(g, o, vel_floor=5e-3)


def test_trained_warm_start_needs_fewer_updates_than_cold_start():
    """Trained by the library's own kernels on seeds disjoint from the evaluation seed,
    the learned warm start reaches residual 1e-4 with fewer Jacobi updates than the plain
    cold start on the same trajectory start."""
    from paper_1904_02833_gb300.mlp import train_warm_start
    from paper_1904_02833_gb300.sim import SnakeSim
    net, rec = train_warm_start(n_snakes=384, rounds=1, steps=8, epochs0=15, epochs=8)
    assert rec[0]["loss_last"] < 0.5 * rec[0]["loss_first"]
    w = W.batched(n=256, seed=4)
    res = {}
    for mode, warm, beta in (("cold", 0, 1.0), ("learned", 2, 0.5)):
        sim = SnakeSim(w, W.solver_settings(iters=5000, tol=1e-4, warm=0))
        sim.step(6)
        sim.set_mlp(net)
        sim.set_config(warm=warm, beta=beta)
        its = []
        for _ in range(4):
            sim.step(1)
            st = sim.state_host()
            assert (st["resid"] <= 1e-4).all()
            its.append(st["iters"].mean())
        res[mode] = float(np.mean(its))
    assert res["learned"] < 0.8 * res["cold"], res


def _mid_step(w, s, subs=2):
    from paper_1904_02833_gb300.sim import SnakeSim
    g = SnakeSim(w, s)
    g.step(3)
    g.split_begin()
    for _ in range(subs):
        g.split_finish()
    return g


@pytest.mark.parametrize("contact", [True, False])
def test_training_rows_match_oracle(contact):
    """sim_training_rows against the oracle's definition of the training rows on the same
    features and multipliers: the same rows in the same order, features bit for bit,
    targets (lambda* - beta lambda_prev) / (m g h^2) to FP32 rounding; snakes with held
    nodes and uneven masses included."""
    w = W.batched(n=21, seed=34, links=(1, 8))
    w["n_fixed"][:5] = [0, 1, 2, 3, 0]
    w["mass"][::3] = 0.02
    beta = 0.5
    s = W.solver_settings(iters=5000, tol=1e-4, warm=1, beta=beta, contact=contact)
    g = _mid_step(w, s)
    lam_prev = g.lam().clone()
    fnode = g.features().float().cpu().numpy()
    g.snapshot_save()
    g.set_config(tol=1e-6, iters=20000, warm=0)
    g.split_finish()
    lam_star = g.lam().clone()
    g.snapshot_restore()
    g.set_config(**s)
    F, T = g.training_rows(lam_star, lam_prev, beta)
    F, T = F.float().cpu().numpy(), T.cpu().numpy()
    h = s["dt"] / s["n_sub"]
    Fo, To = M.training_rows(g.node_off, w["mass"], fnode, lam_star.cpu().numpy().astype(np.float64),
                             lam_prev.cpu().numpy().astype(np.float64), beta, h)
    assert F.shape == Fo.shape and len(T) == len(To) > 0
    assert np.array_equal(F, Fo)
    scale = (np.abs(lam_star.cpu().numpy()).max() + np.abs(lam_prev.cpu().numpy()).max()) / (w["mass"].min() * 9.81 * h * h)
    assert np.abs(T - To).max() <= 1e-6 * scale
    # the restored features are the begun substep's, not those the branch wrote
    assert np.array_equal(g.features().float().cpu().numpy(), fnode)


@pytest.mark.parametrize("net_rows,kinds", [(1, 3), (2, 1)])
def test_learned_mode_writes_the_predicted_kinds_only(net_rows, kinds):
    """In the learned warm start the feature writer fills only the row kinds the network
    predicts (bilateral: stretch, yaw, pitch; stretch alone): those rows equal the
    oracle's features, the other kinds' rows keep what was there (zero in a new handle),
    and sim_training_rows emits the predicted kinds' existing rows only, in the oracle's
    order with the oracle's targets."""
    from paper_1904_02833_gb300.mlp import WarmStartMLP
    from paper_1904_02833_gb300.sim import SnakeSim
    w = W.batched(n=21, seed=36, links=(1, 8))
    w["n_fixed"][:3] = [0, 1, 2]
    beta = 0.5
    s = W.solver_settings(iters=10)
    g, o = SnakeSim(w, s), oracle.OracleSim(w, s)
    g.step(3)
    o.step(3)
    net = WarmStartMLP(M.init_params(11) * 0.5)
    g.set_mlp(net)
    learned = dict(s, warm=2, beta=beta, net_rows=net_rows)
    g.set_config(**learned)
    g.split_begin()
    fg = g.features().float().cpu().numpy()
    fo = o.features()
    kind = np.arange(len(fg)) % 6
    assert not fg[kind >= kinds].any()
    sel = kind < kinds
    err = np.abs(fg[sel, :24] - fo[sel, :24])
    assert (err[:, :23] <= 1e-2 * np.abs(fo[sel, :23]) + 2e-3).all(), err[:, :23].max()
    assert (err[:, 23] <= 5e-3 * np.abs(fo[sel, 23]).max() + 1e-2 * np.abs(fo[sel, 23])).all()
    # training rows of the substep in progress, targets from a tight solve on a snapshot
    lam_prev = g.lam().clone()
    g.snapshot_save()
    g.set_config(tol=1e-6, iters=20000, warm=0)
    g.split_finish()
    lam_star = g.lam().clone()
    g.snapshot_restore()
    g.set_config(**learned)
    F, T = g.training_rows(lam_star, lam_prev, beta)
    F, T = F.float().cpu().numpy(), T.cpu().numpy()
    fnode = g.features().float().cpu().numpy()
    assert np.array_equal(fnode, fg)
    nn = W.n_nodes(w).astype(np.int64)
    expect = (nn - 1) + (2 * (nn - 2) if kinds >= 3 else 0)
    h = s["dt"] / s["n_sub"]
    Fo, To = M.training_rows(g.node_off, w["mass"], fnode, lam_star.cpu().numpy().astype(np.float64),
                             lam_prev.cpu().numpy().astype(np.float64), beta, h)
    assert len(T) == len(To) == int(expect.sum())
    assert np.array_equal(F, Fo)
    assert np.all(np.argmax(F[:, :6], 1) < kinds)
    scale = (np.abs(lam_star.cpu().numpy()).max() + np.abs(lam_prev.cpu().numpy()).max()) / (w["mass"].min() * 9.81 * h * h)
    assert np.abs(T - To).max() <= 1e-6 * scale
    g.close()
    net.close()


def test_snapshot_branch_inside_a_split_step_is_invisible():
    """Saving inside a split env-step, finishing the substep with another configuration,
    restoring and finishing it in the learned mode gives, bit for bit, what a run that
    never branched gives (state, multipliers, residuals and update counts)."""
    w = W.batched(n=30, seed=35, links=(1, 8))
    p = M.init_params(8) * 0.5
    s = W.solver_settings(iters=5000, tol=1e-4, warm=2, beta=0.5)
    net = mlp(p)
    runs = []
    for branch in (False, True):
        from paper_1904_02833_gb300.sim import SnakeSim
        g = SnakeSim(w, dict(s, warm=0))
        g.step(2)
        g.set_mlp(net)
        g.set_config(**s)
        g.split_begin()
        for sub in range(s["n_sub"]):
            if branch and sub in (1, 7):
                g.snapshot_save()
                g.set_config(tol=1e-6, iters=20000, warm=0)
                g.split_finish()
                g.snapshot_restore()
                g.set_config(**s)
            g.split_finish()
        st = g.state_host()
        st["lam"] = g.lam().cpu().numpy()
        runs.append(st)
        g.close()
    for k in runs[0]:
        assert np.array_equal(runs[0][k], runs[1][k]), k


def test_training_rows_and_learned_options_reject_bad_arguments():
    """sim_training_rows refuses a call outside a begun substep, an output smaller than the
    row count and a misaligned feature buffer, and reports the count when asked; the
    configuration refuses unknown row kinds and a negative network period."""
    import ctypes
    from paper_1904_02833_gb300 import _native as N
    from paper_1904_02833_gb300.sim import SnakeSim
    lib = N.load()
    w = W.batched(n=6, seed=36, links=(1, 3))
    s = W.solver_settings(iters=10)
    g = SnakeSim(w, s)
    lam = g.lam().clone()
    n = ctypes.c_int64(-1)
    P = ctypes.c_void_p
    assert lib.sim_training_rows(g.h, None, None, 0.5, None, None, 0, ctypes.byref(n)) == N.SIM_EINVAL
    g.split_begin()
    # the autotuner would time whole env-steps: refused while one is split
    assert lib.sim_autotune(g.h, 1) == N.SIM_EINVAL
    assert lib.sim_training_rows(g.h, None, None, 0.5, None, None, 0, ctypes.byref(n)) == N.SIM_OK
    rows = n.value
    nodes = W.n_nodes(w)
    assert rows == int(sum(N_ - 1 + 2 * (N_ - 2) + 3 * N_ for N_ in nodes))
    feat = torch.empty(rows + 1, 32, dtype=torch.bfloat16, device="cuda")
    tgt = torch.empty(rows, device="cuda")
    lp = P(lam.data_ptr())
    assert lib.sim_training_rows(g.h, lp, lp, 0.5, P(feat.data_ptr()), P(tgt.data_ptr()), rows - 1,
                                 ctypes.byref(n)) == N.SIM_EINVAL
    assert lib.sim_training_rows(g.h, lp, lp, 0.5, P(feat.data_ptr() + 8), P(tgt.data_ptr()), rows,
                                 ctypes.byref(n)) == N.SIM_EINVAL
    assert b"aligned" in lib.sim_last_error()
    assert lib.sim_training_rows(g.h, lp, lp, 1.5, P(feat.data_ptr()), P(tgt.data_ptr()), rows,
                                 ctypes.byref(n)) == N.SIM_EINVAL
    assert lib.sim_training_rows(g.h, lp, lp, 0.5, P(feat.data_ptr()), P(tgt.data_ptr()), rows,
                                 ctypes.byref(n)) == N.SIM_OK
    torch.cuda.synchronize()
    g.split_finish()
    for bad in (dict(net_rows=3), dict(net_rows=-1), dict(net_every=-2)):
        with pytest.raises(N.SimError):
            g.set_config(**dict(s, **bad))
    g.close()


def test_bounded_tensor_core_wait_times_out_and_leaves_the_device_usable():
    """A tensor-core completion that never arrives: the bounded wait runs out, the block
    records it and frees its tensor memory; the status reaches the host, and the network
    kernels (which allocate all of an SM's tensor memory between two blocks) run and agree
    with the oracle afterwards."""
    import ctypes
    from paper_1904_02833_gb300 import _native as N
    lib = N.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(3):
        out = ctypes.c_int32(-1)
        assert lib.mlp_wait_selftest(4096, st, ctypes.byref(out)) == N.SIM_OK
        assert out.value == 1
    assert lib.mlp_wait_selftest(0, st, ctypes.byref(ctypes.c_int32())) == N.SIM_EINVAL
    p = M.init_params(9)
    f = feats(4000, 3)
    y = mlp(p).forward(to_dev(f)).cpu().numpy()
    ref = oracle.mlp_forward(p, M.bf16(f))
    assert np.abs(y - ref).max() <= 5e-3 * max(np.abs(ref).mean() + 1e-3, np.abs(ref).max())
