"""The calibration adjoint (reverse mode through the executed solver map) through the
C-ABI and torch.autograd, against the oracle's forward-mode dual-number gradient and
central finite differences.

Tolerance: the adjoint runs in FP32 through 20 substeps x 10 Jacobi updates per env-step;
the oracle's gradient is exact in FP64.  Relative agreement is bounded by the FP32
forward's own sensitivity (~1e-6 relative per substep amplified through the iterations):
2e-2 of each parameter's largest gradient magnitude over the snakes.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_02833_gb300.build import build
    build()
    torch.cuda.set_device(0)


def setup_case(n, contact, steps, settle=2, seed=5):
    from paper_1904_02833_gb300.calib import theta_of
    truth, guess = W.calibration(n=n, seed=seed)
    s = W.solver_settings(iters=10, contact=contact)
    ot = oracle.OracleSim(truth, s)
    ot.step(settle)
    target = ot.step(steps, tip=True)
    return truth, guess, s, target, theta_of(guess)


def gpu_grad(guess, s, target, theta, steps, ckpt, settle=2):
    from paper_1904_02833_gb300.calib import rollout
    from paper_1904_02833_gb300.sim import SnakeSim
    sim = SnakeSim(guess, s)
    sim.step(settle)
    th = theta.clone().cuda().requires_grad_(True)
    tips = rollout(sim, th, steps, ckpt)
    tg = torch.tensor(target, dtype=torch.float32, device="cuda")
    loss = ((tips - tg) ** 2).sum(-1).mean(0)
    loss.sum().backward()
    return loss.detach().cpu().numpy(), th.grad.cpu().numpy(), tips.detach().cpu().numpy()


@pytest.mark.parametrize("contact", [False, True])
def test_adjoint_matches_oracle_dual_gradient(contact):
    steps = 6
    truth, guess, s, target, theta = setup_case(6, contact, steps)
    loss, g, tips = gpu_grad(guess, s, target, theta, steps, ckpt=2)
    og = oracle.OracleSim(guess, s)
    og.step(2)
    loss_o, g_o = og.calib_grad(steps, target)
    tips_o = og.step(steps, tip=True)
    # FP32 trajectories of 10-update substeps drift ~1e-5 m from FP64 over the window;
    # the loss measures centimetre-scale tip errors, so it agrees to ~1e-2 relative
    assert np.abs(tips - tips_o).max() < 1e-4
    assert np.allclose(loss, loss_o, rtol=1e-2)
    for k in range(5):
        scale = np.abs(g_o[:, k]).max()
        assert np.abs(g[:, k] - g_o[:, k]).max() <= 2e-2 * scale, (k, g[:, k], g_o[:, k])


def test_checkpoint_spacing_does_not_change_the_gradient():
    steps = 6
    _, guess, s, target, theta = setup_case(4, True, steps)
    _, g1, t1 = gpu_grad(guess, s, target, theta, steps, ckpt=1)
    _, g6, t6 = gpu_grad(guess, s, target, theta, steps, ckpt=6)
    assert np.array_equal(t1, t6)
    # the same arithmetic; only the grouping of the per-segment parameter sums differs
    assert np.allclose(g1, g6, rtol=1e-5, atol=1e-6 * np.abs(g6).max())


def test_adjoint_matches_central_differences_without_contact():
    """Central differences (step 1e-3 relative) of the same loss evaluated in FP64 by the
    oracle (differences of the FP32 loss itself are dominated by its rounding)."""
    steps = 4
    _, guess, s, target, theta = setup_case(3, False, steps)
    _, g, _ = gpu_grad(guess, s, target, theta, steps, ckpt=2)
    names = ["alpha_b", "damping", "tau_inf", "tau_def", "gain"]

    def loss_of(wd):
        # the window starts from the unperturbed settled state; only the window's
        # parameters move (as in the differentiated rollout)
        o = oracle.OracleSim(guess, s)
        o.step(2)
        o.prm = oracle.pack_params(wd)
        tips = o.step(steps, tip=True)
        return np.mean(np.sum((tips - target) ** 2, -1), 0)

    for k, nm in enumerate(names):
        hstep = 1e-3 * guess[nm]
        wp = {a: b.copy() for a, b in guess.items()}
        wm = {a: b.copy() for a, b in guess.items()}
        wp[nm] += hstep
        wm[nm] -= hstep
        fd = (loss_of(wp) - loss_of(wm)) / (2 * hstep)
        scale = np.abs(fd).max()
        assert np.abs(g[:, k] - fd).max() <= 3e-2 * scale + 1e-12, (k, g[:, k], fd)


def test_calibration_batch_runs_and_matches_oracle_on_samples():
    """1024 4-link snakes, 20 env-steps with checkpoints every 5 (the calibration batch
    over a shortened horizon); 3 sampled snakes against the oracle alone."""
    steps = 20
    truth, guess = W.calibration(n=1024, seed=5)
    s = W.solver_settings(iters=10)
    ot = oracle.OracleSim(W.subset(truth, [0, 511, 1023]), s)
    ot.step(1)
    tgt3 = ot.step(steps, tip=True)
    from paper_1904_02833_gb300.calib import rollout, theta_of
    from paper_1904_02833_gb300.sim import SnakeSim
    gt = SnakeSim(truth, s)
    gt.step(1)
    with torch.no_grad():
        target = rollout(gt, theta_of(truth).cuda(), steps, 5)
    sim = SnakeSim(guess, s)
    sim.step(1)
    th = theta_of(guess).cuda().requires_grad_(True)
    tips = rollout(sim, th, steps, 5)
    loss = ((tips - target) ** 2).sum(-1).mean(0)
    loss.sum().backward()
    g = th.grad.cpu().numpy()
    assert np.isfinite(g).all()
    sel = [0, 511, 1023]
    og = oracle.OracleSim(W.subset(guess, sel), s)
    og.step(1)
    _, g_o = og.calib_grad(steps, target[:, sel].double().cpu().numpy())
    for k in range(5):
        scale = np.abs(g_o[:, k]).max()
        assert np.abs(g[sel, k] - g_o[:, k]).max() <= 2e-2 * scale, (k, g[sel, k], g_o[:, k])
