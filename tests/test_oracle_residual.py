"""Pins of the oracle's normalised residual: the quantity the metric's stop test
"residual <= 1e-4" compares.

Each case is a hand-built state of a three-node snake (one link of two segments) in which
every row but the one under test is exactly satisfied, so that the residual the oracle
reports must equal a value fixed by the definitions alone:

  * bilateral rows satisfy c + E lambda = 0 at a solution (Sec. IV, equations of motion;
    E = alpha / h^2 for the compliant rows), so a stretch or bend row reports
    |c + alpha~ lambda| over its length scale L0, with c known by construction (a length
    error, a 90-degree turn against a pressure-set rest angle, a 30-degree rise);
  * contact is complementarity 0 <= c_n perp lambda_n >= 0 (Eq. 7), measured with the
    Fischer-Burmeister function the paper uses for it (Sec. IV-D),
    phi(a, b) = a + b - sqrt(a^2 + b^2) on (c_n, w lambda_n): 0 at rest on the ground with
    any lambda_n >= 0 and on a lifted node with lambda_n = 0; 2 |c_n| for a penetrating
    node without force; 2 k for (3 k, 4 k), a Pythagorean pair;
  * friction obeys the Coulomb cone (Sec. IV, last lines of the equations of motion):
    a sticking pair has no slip, so a slip u inside the cone reports |u|; a pair on the
    cone's rim opposite to the slip is a valid sliding state and reports 0; a pair on the
    rim along the slip reports |u| (lambda_t could still decrease); the same along and
    across the body with anisotropic friction (the ellipse of coefficients mu, mu_side);
  * rows that touch only fixed nodes carry no multiplier and are not measured.

A wrong normaliser on any term (a missing / L0, the inverse mass applied twice, the cone
radius without mu) changes at least one of these values.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

H = 1.0 / 1200.0  # substep of the default settings: dt 1/60 s over 20 substeps


def snake(**kw):
    w = W.subset(W.single_snake(), [0])
    w["n_links"][:] = 1
    w["seg_per_link"][:] = 2
    w["n_fixed"][:] = 0
    w["gait_alternate"][:] = 0.0
    for k, v in kw.items():
        w[k][:] = v
    return w


S = W.solver_settings(iters=10)


def straight(w):
    L0, r = float(w["L0"][0]), float(w["radius"][0])
    return np.array([[i * L0, 0.0, r] for i in range(3)])


def resid(w, x, xs=None, press=None, lam=None):
    xs = x if xs is None else xs
    press = np.zeros((1, 2)) if press is None else press
    lam = np.zeros((3, 6)) if lam is None else lam
    return oracle.residual(w, S, x, xs, press, lam)


def test_straight_snake_at_rest_on_the_ground_is_a_solution():
    w = snake()
    x = straight(w)
    assert resid(w, x) == pytest.approx(0.0, abs=1e-13)
    # resting contact carries any non-negative normal multiplier (here m g h^2)
    lam = np.zeros((3, 6))
    lam[:, 3] = 0.01 * 9.81 * H * H
    assert resid(w, x, lam=lam) == pytest.approx(0.0, abs=1e-13)


def test_contact_fischer_burmeister_special_values():
    w = snake()
    L0, m = 0.02, 0.01
    x = straight(w)
    # every node 1e-4 m below its contact height, no normal force: phi(-d, 0) = -2 d
    d = 1e-4
    xp = x.copy()
    xp[:, 2] -= d
    assert resid(w, xp) == pytest.approx(2 * d / L0, rel=1e-12)
    # lifted by d with no force: complementarity holds
    xl = x.copy()
    xl[:, 2] += d
    assert resid(w, xl) == pytest.approx(0.0, abs=1e-13)
    # lifted by 3 k with w lambda_n = 4 k: phi = 3k + 4k - 5k = 2k
    k = 2e-5
    xk = x.copy()
    xk[:, 2] += 3 * k
    lam = np.zeros((3, 6))
    lam[:, 3] = 4 * k * m  # w lambda_n = lambda_n / m
    assert resid(w, xk, lam=lam) == pytest.approx(2 * k / L0, rel=1e-10)


def test_friction_sticking_and_sliding():
    mu, m, L0 = 0.5, 0.01, 0.02
    w = snake(mu=mu)
    xs = straight(w)
    ln = 0.01 * 9.81 * H * H  # resting normal multiplier
    rho = mu * ln / m         # cone radius in displacement units, w mu lambda_n
    u = np.array([0.3, -0.4]) * rho  # slip of the substep, |u| = rho / 2
    x = xs.copy()
    x[:, :2] += u  # rigid horizontal shift: only the friction rows see it
    lam = np.zeros((3, 6))
    lam[:, 3] = ln
    # sticking with zero tangential force: the slip itself is the residual
    assert resid(w, x, xs, lam=lam) == pytest.approx(np.linalg.norm(u) / L0, rel=1e-10)
    # a tangential force strictly inside the cone still sticks: residual |u|
    lam2 = lam.copy()
    lam2[:, 4:6] = m * np.array([-0.1, 0.2]) * rho
    assert resid(w, x, xs, lam=lam2) == pytest.approx(np.linalg.norm(u) / L0, rel=1e-10)
    # on the cone's rim opposite to the slip: a valid sliding state
    uhat = u / np.linalg.norm(u)
    lam3 = lam.copy()
    lam3[:, 4:6] = -m * rho * uhat
    assert resid(w, x, xs, lam=lam3) == pytest.approx(0.0, abs=1e-12)
    # on the rim along the slip: not a solution, residual |u|
    lam4 = lam.copy()
    lam4[:, 4:6] = m * rho * uhat
    assert resid(w, x, xs, lam=lam4) == pytest.approx(np.linalg.norm(u) / L0, rel=1e-10)
    # no normal force: any tangential force is wrong; with no slip the residual is |w lambda_t|
    lam5 = np.zeros((3, 6))
    lam5[:, 4] = m * 1e-5
    assert resid(w, xs, xs, lam=lam5) == pytest.approx(1e-5 / L0, rel=1e-10)


def test_anisotropic_friction_rim_along_and_across_the_body():
    mu, mu_side, m, L0 = 0.3, 0.9, 0.01, 0.02
    w = snake(mu=mu, mu_side=mu_side, yaw0=0.0)
    xs = straight(w)  # body along world x
    ln = 0.01 * 9.81 * H * H
    lam = np.zeros((3, 6))
    lam[:, 3] = ln
    for axis, coef in ((0, mu), (1, mu_side)):
        rho = coef * ln / m
        u = np.zeros(2)
        u[axis] = 0.5 * rho
        x = xs.copy()
        x[:, :2] += u
        slide = lam.copy()
        slide[:, 4 + axis] = -m * rho  # on the ellipse's rim, opposite to the slip
        assert resid(w, x, xs, lam=slide) == pytest.approx(0.0, abs=1e-12), axis
        # sticking on the rim's inside: residual |u|; the disc of radius mu lambda_n would
        # cut the sideways pair back and report another value
        stick = lam.copy()
        stick[:, 4 + axis] = -m * 0.5 * rho
        assert resid(w, x, xs, lam=stick) == pytest.approx(0.5 * rho / L0, rel=1e-10), axis


def test_stretch_row_reports_c_plus_compliance_times_lambda():
    w = snake()
    L0, alpha_s = 0.02, 1e-8
    xs = straight(w)
    x = xs.copy()
    eps = 3e-6
    x[2, 0] += eps  # stretch row (1, 2) longer by eps; the chain stays straight
    lam = np.zeros((3, 6))
    ls = -2e-4  # pulls against the stretch; alpha~ lambda = -2.88e-6 m
    lam[1, 0] = ls
    expect = abs(eps + alpha_s / H ** 2 * ls) / L0
    # the friction rows of node 2 see its displacement eps too, unless anchored there
    assert resid(w, x, x, lam=lam) == pytest.approx(expect, rel=1e-8)
    lam[1, 0] = 0.0
    assert resid(w, x, x, lam=lam) == pytest.approx(eps / L0, rel=1e-8)


def test_yaw_row_against_pressure_set_rest_angle():
    """A 90-degree turn at node 1 against the rest angle G (p_R - p_L) L0 of Eq. 3-4."""
    G, alpha_b, L0, r = 20.0, 1e-4, 0.02, 0.01
    w = snake(gain=G)
    x = np.array([[0.0, 0.0, r], [L0, 0.0, r], [L0, L0, r]])
    press = np.array([[0.7, 0.2]])
    theta = G * 0.5 * L0
    assert resid(w, x, press=press) == pytest.approx(math.pi / 2 - theta, rel=1e-12)
    lam = np.zeros((3, 6))
    lb = 3e-7
    lam[1, 1] = lb
    expect = abs(L0 * (math.pi / 2 - theta) + alpha_b / H ** 2 * lb) / L0
    assert resid(w, x, press=press, lam=lam) == pytest.approx(expect, rel=1e-12)
    # a turn the other way against a left-chamber rest angle
    xm = x.copy()
    xm[2, 1] = -L0
    pm = np.array([[0.0, 0.4]])
    assert resid(w, xm, press=pm) == pytest.approx(abs(-math.pi / 2 + G * 0.4 * L0), rel=1e-12)


def test_pitch_row_thirty_degree_rise():
    L0, r = 0.02, 0.01
    w = snake()
    a = math.radians(30.0)
    x = np.array([[0.0, 0.0, r], [L0, 0.0, r], [L0 + L0 * math.cos(a), 0.0, r + L0 * math.sin(a)]])
    # node 2 lifted, no normal force: contact satisfied; the pitch row reports 30 degrees
    assert resid(w, x) == pytest.approx(a, rel=1e-12)


def test_max_over_terms_and_fixed_rows():
    L0 = 0.02
    w = snake()
    x = straight(w)
    x[:, 2] -= 1e-5  # contact term 2e-5 / L0 = 1e-3
    x[2, 0] += 4e-5  # stretch term 4e-5 / L0 = 2e-3 (and friction of node 2 if anchored)
    assert resid(w, x, x) == pytest.approx(2e-3, rel=1e-8)
    # all nodes fixed: no row touches a free node, nothing is measured
    wf = snake(n_fixed=3)
    assert resid(wf, x, x) == 0.0
    # nodes 0 and 1 fixed: stretch (0, 1) touches no free node and is not measured
    w2 = snake()
    w2["n_fixed"][:] = 2
    x2 = straight(w2)
    x2[1, 0] += 5e-5   # stretch (0, 1) violated, only fixed nodes
    x2[2, 0] += 5e-5   # node 2 moves with node 1: stretch (1, 2) exact
    # the bend rows centred on node 1 see node 2 and are still exact (straight chain)
    assert resid(w2, x2, x2) == pytest.approx(0.0, abs=1e-12)


@pytest.mark.parametrize("mu_side", [0.0, 0.3])
def test_residual_is_invariant_under_rotations_about_z_and_horizontal_shifts(mu_side):
    """Random states of a 7-node snake (positions near the ground, substep-start
    positions, pressures, multipliers of every kind): rotating the whole state about the
    vertical (positions, start positions and the friction pair in world x / y) and
    shifting it horizontally leaves the residual unchanged, since every term is a
    length measured in the row's own frame or along z."""
    rng = np.random.default_rng(7)
    w = snake(mu_side=mu_side)
    w["seg_per_link"][:] = 6
    L0, r = float(w["L0"][0]), float(w["radius"][0])
    for _ in range(20):
        x = np.array([[i * L0, 0.0, r] for i in range(7)]) + rng.normal(0, 0.3 * L0, (7, 3))
        xs = x + rng.normal(0, 0.05 * L0, (7, 3))
        press = rng.uniform(0, 1, (1, 2))
        lam = rng.normal(0, 1e-6, (7, 6))
        lam[:, 3] = np.abs(lam[:, 3])
        ref = resid(w, x, xs, press, lam)
        th = rng.uniform(0, 2 * math.pi)
        c, s_ = math.cos(th), math.sin(th)
        R = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]])
        off = np.array([rng.uniform(-3, 3), rng.uniform(-3, 3), 0.0])
        lr = lam.copy()
        lr[:, 4] = c * lam[:, 4] - s_ * lam[:, 5]
        lr[:, 5] = s_ * lam[:, 4] + c * lam[:, 5]
        got = resid(w, x @ R.T + off, xs @ R.T + off, press, lr)
        assert ref > 0 and got == pytest.approx(ref, rel=1e-9)
