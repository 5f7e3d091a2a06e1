"""Pins of the oracle's warm-start network and row features (CPU)."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp_oracle as M
import workloads as W


def test_backward_matches_central_differences():
    """The FP64 backward pass of the network against central differences of its forward."""
    rng = np.random.default_rng(0)
    p = M.init_params(1) + rng.normal(scale=0.05, size=M.N_PARAMS)
    x = rng.normal(size=(7, M.N_IN))
    t = rng.normal(size=7)
    L, g = M.loss_and_grad(p, x, t, 0.3, bf16_ops=False)
    idx = np.concatenate([rng.choice(M.N_PARAMS, 60, replace=False), [M.N_PARAMS - 1]])
    for i in idx:
        e = np.zeros(M.N_PARAMS)
        e[i] = 1e-6
        Lp = M.loss_and_grad(p + e, x, t, 0.3, bf16_ops=False)[0]
        Lm = M.loss_and_grad(p - e, x, t, 0.3, bf16_ops=False)[0]
        assert g[i] == pytest.approx((Lp - Lm) / 2e-6, rel=1e-5, abs=1e-9), i


def test_bf16_rounding_matches_library():
    """Round-to-nearest-even bfloat16 against torch's conversion, including ties."""
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(scale=10, size=5000), [1 + 2 ** -8, 1 + 3 * 2 ** -8, -0.0, 65504.0,
                                                          1e-30, 3.0e38]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).float().double().numpy()
    assert np.array_equal(M.bf16(x), ref)


def test_cpp_network_matches_numpy_network():
    rng = np.random.default_rng(4)
    p = M.init_params(2)
    x = rng.normal(size=(50, M.N_IN))
    y_np = M.forward(p, x, bf16_ops=True)[0]
    y_c = oracle.mlp_forward(p, x)
    assert np.allclose(y_c, y_np, rtol=1e-12, atol=1e-12)


def test_features_of_a_straight_snake_at_rest():
    """Hand values: a straight 2-link snake on the ground, heading 0.7 rad, at rest.  In
    every row frame the next node sits at (1, 0, 0) L0 and the one after at (2, 0, 0) L0;
    gravity's prediction puts every node g h^2 below its contact height; velocities are
    -g h along z; multipliers and rest angles are zero; non-existent rows are empty."""
    w = W.subset(W.single_snake(), [0])
    w["n_links"][:] = 2
    w["yaw0"][:] = 0.7
    w["gait_amp"][:] = 0.0
    s = W.solver_settings()
    o = oracle.OracleSim(w, s)
    F = o.features().reshape(21, 6, 24)
    h = s["dt"] / s["n_sub"]
    L0, g = 0.02, 9.81
    for i in range(21):
        for k in range(6):
            f = F[i, k]
            exists = (k == 0 and i <= 19) or (k in (1, 2) and 1 <= i <= 19) or k >= 3
            if not exists:
                assert not f.any()
                continue
            assert f[k] == 1.0 and f[:6].sum() == 1.0
            assert f[6] == pytest.approx(-g * h * h / L0, rel=1e-9)
            if k == 0:
                assert np.allclose(f[7:10], [1, 0, 0], atol=1e-12)
            if k in (1, 2):
                assert np.allclose(f[7:10], [1, 0, 0], atol=1e-12)
                assert np.allclose(f[10:13], [2, 0, 0], atol=1e-12)
            nodes = 2 if k == 0 else 3 if k in (1, 2) else 1
            for u in range(3):
                vz = -g * h * h / L0 if u < nodes else 0.0
                assert np.allclose(f[13 + 3 * u:16 + 3 * u], [0, 0, vz], atol=1e-15)
            assert f[22] == 0.0 and f[23] == 0.0


def test_friction_row_frame_is_world_aligned():
    """A node sliding along +y reads its velocity as (0, v) in the friction-x frame and
    (v, 0) in the friction-y frame; a yaw row of a pressurised link reads its rest angle."""
    w = W.subset(W.single_snake(), [0])
    w["n_links"][:] = 1
    s = W.solver_settings()
    o = oracle.OracleSim(w, s)
    o.v[:, 1] = 0.3
    o.press[0] = [0.5, 0.0]
    F = o.features(ucmd=np.array([0.5])).reshape(11, 6, 24)
    h, L0 = s["dt"] / s["n_sub"], 0.02
    assert F[4, 4, 13:15] == pytest.approx([0.0, 0.3 * h / L0])
    assert F[4, 5, 13:15] == pytest.approx([0.3 * h / L0, 0.0])
    assert F[4, 1, 22] == pytest.approx(20.0 * 0.5 * L0)


@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0])
def test_training_target_inverts_the_learned_warm_start(beta):
    """The training target of a row is the network output that would make the oracle's
    learned warm start land on the given multipliers.  A network whose output is the
    constant c (all weights zero, output bias c) starts a substep from
    beta lambda_prev + m g h^2 c; with no update applied (iteration cap 0) that start is
    the substep's result, and the targets computed from it must be c on every existing
    row, whatever the snake's mass, the substep length and beta."""
    w = W.batched(n=5, seed=12, links=(1, 4))
    w["mass"][:] = [0.01, 0.02, 0.005, 0.013, 0.01]
    s = W.solver_settings(iters=10, n_sub=3)
    o = oracle.OracleSim(w, s)
    o.step(2)
    c = 0.8125
    p = np.zeros(M.N_PARAMS)
    p[-1] = c
    o.set_cfg(n_sub=1, iters=0, warm=2, beta=beta)
    feat = o.features()
    lam_prev = o.lam.copy()
    o.step(1, mlp=p)
    h = s["dt"] / 1
    F, T = M.training_rows(o.node_off, w["mass"], feat, o.lam, lam_prev, beta, h)
    n = len(W.n_nodes(w))
    nodes = W.n_nodes(w)
    # stretch (N - 1), yaw and pitch (2 (N - 2)), contact and friction (3 N) per snake
    assert len(T) == int(sum(N - 1 + 2 * (N - 2) + 3 * N for N in nodes)) and n == 5
    assert np.allclose(T, c, rtol=1e-12, atol=1e-12)
    assert np.array_equal(F[:, :6].sum(1), np.ones(len(F)))


@pytest.mark.parametrize("net_rows,net_every,beta_net",
                         [(0, 1, None), (0, 2, None), (1, 2, None), (1, 1, None), (2, 1, None), (2, 3, None),
                          (1, 3, 0.25), (0, 2, 0.75), (2, 1, 0.0)])
def test_learned_warm_start_schedule_closed_form(net_rows, net_every, beta_net):
    """Which substeps and row kinds take the network's prediction.  With no updates
    applied (cap 0) a substep ends on its warm start, so with a network of constant output
    c a row's multiplier after three substeps is m_2 m_1 m_0 l_init plus c m g h^2 times
    m_2 m_1 (substep 0), m_2 (substep 1) and 1 (substep 2) for each network substep
    (s % net_every == 0), where m_s = beta_net at a network substep on the predicted kinds
    (all six; stretch, yaw, pitch; or stretch) and beta otherwise (beta_net unset: beta)."""
    w = W.batched(n=3, seed=13, links=(1, 3))
    s = W.solver_settings(iters=10, n_sub=3)
    o = oracle.OracleSim(w, s)
    o.step(2)
    c, b = 0.375, 0.5
    bn = b if beta_net is None else beta_net
    p = np.zeros(M.N_PARAMS)
    p[-1] = c
    o.set_cfg(iters=0, warm=2, beta=b, net_rows=net_rows, net_every=net_every,
              beta_net=-1.0 if beta_net is None else beta_net)
    lam0 = o.lam.copy()
    o.step(1, mlp=p)
    h = s["dt"] / 3
    sc = np.repeat(w["mass"] * 9.81 * h * h, W.n_nodes(w))[:, None]
    pred = {0: np.ones((1, 6)), 1: np.array([[1, 1, 1, 0, 0, 0]]), 2: np.array([[1, 0, 0, 0, 0, 0]])}[net_rows]
    net = [k % net_every == 0 for k in range(3)]
    m = [bn if net[k] else b for k in range(3)]  # factor of a predicted row at substep k
    lin = m[0] * m[1] * m[2]
    add = sum(np.prod(m[k + 1:]) for k in range(3) if net[k])
    expect = np.where(pred > 0, lin * lam0 + c * add * sc, b ** 3 * lam0)
    # rows that do not exist stay zero (the chain's ends)
    F = o.features()
    exists = np.abs(F[:, :6]).sum(1).reshape(-1, 6) > 0
    assert np.allclose(o.lam[exists], expect[exists], rtol=1e-12, atol=1e-15)
    assert (o.lam[~exists] == 0).all()
