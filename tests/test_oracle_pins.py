"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed forms, textbook special cases, invariants and brute force.

Each test names the part of the method it pins.  A plausible mistake (wrong sign of a
gradient, a dropped compliance term, a transposed index, a wrong rest angle at the
connectors, the wrong filter branch) breaks at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

G = 9.81
HERE = os.path.dirname(os.path.abspath(__file__))


def one(w, **kw):
    w = W.subset(w, [0])
    for k, v in kw.items():
        w[k][:] = v
    return w


# ------------------------------------------------------------------ latency filter
def test_filter_step_response_closed_form():
    """First-order latency: a command step 0 -> 1 gives p(n h) = 1 - exp(-n h / tau_inf)
    exactly (the update is the exact exponential discretisation); releasing gives
    p = p0 exp(-n h / tau_def).  The opposite chamber stays empty (Sec. III)."""
    w = one(W.single_snake(), n_links=1, gait_alternate=0.0)
    s = W.solver_settings(iters=2, gravity=(0, 0, 0), contact=False)
    o = oracle.OracleSim(w, s)
    h = s["dt"] / s["n_sub"]
    o.step(3, ucmd=np.array([1.0]))
    n = 3 * s["n_sub"]
    assert o.press[0, 0] == pytest.approx(1 - math.exp(-n * h / 0.15), rel=1e-13)
    assert o.press[0, 1] == 0.0
    p0 = o.press[0, 0]
    o.step(2, ucmd=np.array([0.0]))
    assert o.press[0, 0] == pytest.approx(p0 * math.exp(-2 * s["n_sub"] * h / 0.25), rel=1e-13)
    # a negative command inflates the left chamber with tau_inflate, deflates the right
    pR = o.press[0, 0]
    o.step(1, ucmd=np.array([-0.7]))
    m = s["n_sub"]
    assert o.press[0, 1] == pytest.approx(0.7 * (1 - math.exp(-m * h / 0.15)), rel=1e-13)
    assert o.press[0, 0] == pytest.approx(pR * math.exp(-m * h / 0.25), rel=1e-13)


def test_gait_hand_values():
    """Eq. 9 at t = 0.25 s against values worked by hand (tests/golden/gait_hand_values.txt)."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "gait_hand_values.txt"))
            if l.strip() and not l.startswith("#")]
    for form, A, phi, t, k, pR, pL in rows:
        A, phi, t, k, pR, pL = float(A), float(phi), float(t), int(k), float(pR), float(pL)
        w = one(W.single_snake(), n_links=4, gait_amp=A, gait_offset=phi, gait_freq=1.0,
                gait_lag=math.pi / 2, tau_inf=1e-12, tau_def=1e-12)
        w["gait_scale"][:] = 0.5 if form == "alternating" else 1.0
        w["gait_alternate"][:] = 1.0 if form == "alternating" else 0.0
        s = W.solver_settings(iters=1, gravity=(0, 0, 0), contact=False)
        o = oracle.OracleSim(w, s)
        # the last substep of step n samples the gait at (n + 1) dt
        o.step_index = int(round(t / s["dt"])) - 1
        o.step(1)
        assert o.press[k, 0] == pytest.approx(pR, abs=1e-12), (form, k)
        assert o.press[k, 1] == pytest.approx(pL, abs=1e-12), (form, k)


def test_chamber_law_hand_values():
    """The discrete chamber law of Sec. V-A against sequences worked by hand
    (tests/golden/chamber_law_hand_values.txt): inflation by the square of the remaining
    difference, deflation linear up to the threshold T_p and proportional below it,
    the valve stopping at the target, antagonistic chambers, the law's period."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "chamber_law_hand_values.txt"))
            if l.strip() and not l.startswith("#")]
    for case, ki, kd, tp, ps, every, u, pr0, pl0, n, pr, pl in rows:
        w = one(W.single_snake(), n_links=1, gait_alternate=0.0)
        dt = 1.0 / 60.0
        s = W.solver_settings(dt=dt, n_sub=1, iters=1, gravity=(0, 0, 0), contact=False, latency=1,
                              k_inflate=float(ki), k_deflate=float(kd), t_p=float(tp),
                              p_source=float(ps), law_dt=int(every) * dt)
        o = oracle.OracleSim(w, s)
        o.press[0] = [float(pr0), float(pl0)]
        o.step(int(n), ucmd=np.array([float(u)]))
        assert o.press[0, 0] == pytest.approx(float(pr), abs=1e-15), (case, n)
        assert o.press[0, 1] == pytest.approx(float(pl), abs=1e-15), (case, n)


def test_chamber_law_closed_forms():
    """Closed forms of the law: below the threshold (p k_d < T_p) deflation is geometric,
    p_n = p_0 (1 - k_d)^n; above it, linear, p_n = p_0 - n T_p; inflation satisfies the
    discrete Riccati identity 1/d' = 1/d + k_i/p_s + k_i^2 d / (p_s^2 (1 - k_i d / p_s))
    for the remaining difference d = p^ - p; within a law period the chambers hold."""
    w = one(W.single_snake(), n_links=1, gait_alternate=0.0)
    dt = 1.0 / 60.0
    base = dict(dt=dt, n_sub=1, iters=1, gravity=(0, 0, 0), contact=False, latency=1)
    o = oracle.OracleSim(w, W.solver_settings(**base, k_deflate=0.3, t_p=0.5, law_dt=dt))
    o.press[0] = [0.9, 0.0]
    for n in range(1, 30):
        o.step(1, ucmd=np.array([0.0]))
        assert o.press[0, 0] == pytest.approx(0.9 * 0.7 ** n, rel=1e-12)
    o = oracle.OracleSim(w, W.solver_settings(**base, k_deflate=0.9, t_p=0.05, law_dt=dt))
    o.press[0] = [1.0, 0.0]
    for n in range(1, 15):  # p k_d >= T_p while p >= 0.0556
        o.step(1, ucmd=np.array([0.0]))
        assert o.press[0, 0] == pytest.approx(1.0 - 0.05 * n, abs=1e-12)
    ki, ps, tgt = 0.37, 1.3, 0.8
    o = oracle.OracleSim(w, W.solver_settings(**base, k_inflate=ki, p_source=ps, law_dt=dt))
    d = tgt
    for n in range(40):
        o.step(1, ucmd=np.array([tgt]))
        d_new = tgt - o.press[0, 0]
        expect = 1.0 / d + ki / ps + ki * ki * d / (ps * ps * (1.0 - ki * d / ps))
        assert 1.0 / d_new == pytest.approx(expect, rel=1e-9)
        d = d_new
    # period of 5 substeps inside a 20-substep env-step: four moves per env-step
    s = W.solver_settings(**dict(base, n_sub=20), k_inflate=0.5, law_dt=5 * dt / 20)
    o = oracle.OracleSim(w, s)
    o.step(1, ucmd=np.array([1.0]))
    p, d = 0.0, 1.0
    for _ in range(4):
        p += 0.5 * d * d
        d = 1.0 - p
    assert o.press[0, 0] == pytest.approx(p, rel=1e-14)


# ------------------------------------------------------------------ geometry of the rows
def _settle(o, steps, ucmd=None):
    for _ in range(steps):
        o.step(1, ucmd=ucmd)


@pytest.mark.parametrize("n_links,p", [(1, 1.0 / 3.0), (2, 0.8), (1, 1.0)])
def test_uniform_pressure_settles_to_discrete_arc(n_links, p):
    """Eq. 3-4 reduced to a rest curvature: a cantilever (nodes 0, 1 clamped along x) under
    uniform pressure p, without gravity, settles to the exact discrete polyline whose
    segment headings advance by theta = G p L0 at every node inside a link and by 0 at a
    rigid connector; the tip lies on a circle of radius L0 / (2 sin(theta / 2))."""
    w = one(W.static_sweep(), n_links=n_links, alpha_b=3e-5, damping=20.0)
    s = W.solver_settings(tol=1e-11, iters=20000, gravity=(0, 0, 0), contact=False)
    o = oracle.OracleSim(w, s)
    o.press[:, 0] = p
    _settle(o, 150, ucmd=np.full(n_links, p))
    L0, theta = 0.02, 20.0 * p * 0.02
    N = 10 * n_links + 1
    head = 0.0
    ref = [o.x[0].copy(), o.x[0] + np.array([L0, 0, 0])]
    for i in range(1, N - 1):
        head += 0.0 if i % 10 == 0 else theta
        ref.append(ref[-1] + L0 * np.array([math.cos(head), math.sin(head), 0.0]))
    ref = np.array(ref)
    assert np.abs(o.x - ref).max() < 1e-9
    if n_links == 1:
        # a regular polyline is inscribed in a circle: its first chord (node 0 -> 1) lies
        # along x, so the centre sits on that chord's perpendicular bisector
        R = L0 / (2 * math.sin(theta / 2))
        cx = o.x[0, 0] + L0 / 2
        cy = o.x[0, 1] + (L0 / 2) / math.tan(theta / 2)
        d = np.hypot(o.x[:, 0] - cx, o.x[:, 1] - cy)
        assert np.allclose(d, R, rtol=1e-9)


def test_cantilever_sag_small_deflection():
    """A clamped actuator under gravity (p = 0) sags like a discrete Euler-Bernoulli
    cantilever: every pitch hinge k turns by phi_k = alpha_b M_k / L0^2 (rotational
    stiffness L0^2 / alpha_b of a length-unit bend row) with M_k the moment of the node
    weights beyond it; the tip drops by sum_k phi_k (x_tip - x_k).  The continuum
    w L^4 / (8 EI), EI = L0^3 / alpha_b, agrees only to O(1/N) (about 40 % with 9
    hinges, where the hinge sum is a one-sided Riemann sum of the beam integral)."""
    alpha_b, m, L0 = 1e-5, 0.01, 0.02
    w = one(W.static_sweep(), n_links=1, alpha_b=alpha_b, gait_offset=0.0, damping=30.0)
    s = W.solver_settings(tol=1e-12, iters=50000, contact=False)
    o = oracle.OracleSim(w, s)
    _settle(o, 200)
    assert np.abs(o.v).max() < 1e-9
    N = 11
    sag = 0.0
    for k in range(1, N - 1):
        Mk = m * G * sum((j - k) * L0 for j in range(k + 1, N))
        sag += alpha_b * Mk / L0 ** 2 * (N - 1 - k) * L0
    drop = o.x[0, 2] - o.x[-1, 2]
    assert drop == pytest.approx(sag, rel=2e-3)
    Lc = (N - 2) * L0
    eb = (m * G / L0) * Lc ** 4 / (8 * L0 ** 3 / alpha_b)
    assert eb < drop < 1.5 * eb
    # no sideways motion, clamped nodes untouched
    assert np.abs(o.x[:, 1]).max() < 1e-12
    assert np.allclose(o.x[1], [L0, 0, 1.0], atol=1e-15)


def test_pendulum_period():
    """A stiff two-node pendulum of length l has period 2 pi sqrt(l / g) (1 + theta0^2/16)
    at small amplitude theta0; implicit Euler shifts it by O((omega h)^2)."""
    l, th0 = 0.1, 0.05
    w = W.pendulum(l)
    s = W.solver_settings(dt=1.0 / 1200.0, n_sub=1, tol=1e-12, iters=5000, contact=False)
    o = oracle.OracleSim(w, s)
    o.x[1] = [l * math.sin(th0), 0.0, 1.0 - l * math.cos(th0)]
    steps = 1900
    tips = o.step(steps, tip=True)[:, 0, 0]
    t = (np.arange(steps) + 1) * s["dt"]
    zc = [t[i] - tips[i] * (t[i + 1] - t[i]) / (tips[i + 1] - tips[i])
          for i in range(steps - 1) if tips[i] > 0 >= tips[i + 1] or tips[i] < 0 <= tips[i + 1]]
    period = 2 * np.mean(np.diff(zc))
    ref = 2 * math.pi * math.sqrt(l / G) * (1 + th0 ** 2 / 16)
    assert len(zc) >= 5
    assert period == pytest.approx(ref, rel=1e-3)


def test_momentum_conserved_without_external_forces():
    """No gravity, contact, clamps or damping: every internal row's gradients sum to zero,
    so sum m v is constant to rounding.  The rows are invariant under rotations about z,
    so the only change of the z angular momentum is the first-order integrator's own
    dissipation: halving h halves the drift."""
    m = 0.01
    drift = []
    for n_sub in (20, 40):
        w = one(W.single_snake(), n_links=2, damping=0.0, gait_alternate=0.0, gait_offset=0.0,
                gait_scale=1.0, gait_amp=1.0, gait_freq=2.0, z0=0.5)
        s = W.solver_settings(iters=20000, tol=1e-11, n_sub=n_sub, gravity=(0, 0, 0),
                              contact=False)
        o = oracle.OracleSim(w, s)
        rng = np.random.default_rng(0)
        o.v[:] = rng.normal(scale=0.01, size=o.v.shape) + np.array([0.2, -0.1, 0.05])
        o.v[:, 1] += 0.5 * (o.x[:, 0] - o.x[:, 0].mean())
        P0 = m * o.v.sum(0)
        L0 = m * np.sum(o.x[:, 0] * o.v[:, 1] - o.x[:, 1] * o.v[:, 0])
        o.step(30)
        assert np.allclose(m * o.v.sum(0), P0, rtol=0, atol=1e-10)
        L1 = m * np.sum(o.x[:, 0] * o.v[:, 1] - o.x[:, 1] * o.v[:, 0])
        drift.append((L1 - L0) / abs(L0))
    assert abs(drift[0]) < 0.03
    assert 1.5 < drift[0] / drift[1] < 2.5


def _rows_value(w1, s, x, xs, press):
    c, g, on = oracle.rows(w1, s, x, xs, press)
    return c, g, on


def test_row_gradients_match_central_differences():
    """Analytic gradients of every row (stretch, yaw, pitch, contact, friction) against
    central finite differences of the row values, on a randomly bent 3D chain."""
    w = one(W.single_snake(), n_links=2)
    s = W.solver_settings()
    N = 21
    rng = np.random.default_rng(1)
    x = np.zeros((N, 3))
    head, pitch = 0.3, 0.0
    for i in range(1, N):
        head += rng.uniform(-0.4, 0.4)
        pitch = rng.uniform(-0.3, 0.3)
        x[i] = x[i - 1] + 0.02 * np.array([math.cos(head) * math.cos(pitch),
                                           math.sin(head) * math.cos(pitch), math.sin(pitch)])
    xs = x + rng.normal(scale=1e-3, size=x.shape)
    press = rng.uniform(0, 1, size=(2, 2))
    c, g, on = _rows_value(w, s, x, xs, press)
    eps = 1e-7
    local = {0: 2, 1: 3, 2: 3, 3: 1, 4: 1, 5: 1}
    worst = 0.0
    for i in range(N):
        for k in range(6):
            if not on[i, k]:
                continue
            for l in range(local[k]):
                node = i + l if k == 0 else (i - 1 + l if k in (1, 2) else i)
                for d in range(3):
                    xp, xm = x.copy(), x.copy()
                    xp[node, d] += eps
                    xm[node, d] -= eps
                    fd = (_rows_value(w, s, xp, xs, press)[0][i, k]
                          - _rows_value(w, s, xm, xs, press)[0][i, k]) / (2 * eps)
                    worst = max(worst, abs(fd - g[i, k, l, d]))
    assert worst < 1e-7


def test_row_values_known_geometry():
    """Row values on a hand-built chain: a 90-degree left turn in the plane reads yaw =
    +L0 pi/2 (counter-clockwise about the ground normal), a 30-degree climb reads pitch =
    L0 pi/6, stretching one segment by 1 mm reads 1 mm, a node 3 mm above its contact
    height reads 3 mm."""
    w = one(W.single_snake(), n_links=1, seg_per_link=3, radius=0.01)
    s = W.solver_settings()
    L0 = 0.02
    x = np.array([[0, 0, 0.013], [L0, 0, 0.01], [L0, L0, 0.01],
                  [L0, L0 + 0.021 * math.cos(math.pi / 6), 0.01 + 0.021 * math.sin(math.pi / 6)]])
    c, g, on = _rows_value(w, s, x, x, np.zeros((1, 2)))
    assert c[1, 1] == pytest.approx(L0 * math.pi / 2, rel=1e-12)
    assert c[2, 2] == pytest.approx(L0 * math.pi / 6, rel=1e-12)
    assert c[2, 0] == pytest.approx(0.001, rel=1e-9)
    assert c[0, 3] == pytest.approx(0.003, rel=1e-9)
    # a pressurised link shifts the yaw reading by - G p L0 * L0 on interior nodes
    c2, _, _ = _rows_value(w, s, x, x, np.array([[0.5, 0.0]]))
    assert c2[1, 1] == pytest.approx(L0 * (math.pi / 2 - 20 * 0.5 * L0), rel=1e-12)


# ------------------------------------------------------------------ the solver
def _c_fd(x, L0, at_rows):
    """Row values of a 3-node chain written from the definitions (for the Newton check)."""
    e1, e2 = x[1] - x[0], x[2] - x[1]
    cs = [np.linalg.norm(e1) - L0, np.linalg.norm(e2) - L0]
    yaw = math.atan2(e1[0] * e2[1] - e1[1] * e2[0], e1[0] * e2[0] + e1[1] * e2[1])
    pit = math.asin(e2[2] / np.linalg.norm(e2)) - math.asin(e1[2] / np.linalg.norm(e1))
    return np.array(cs + [L0 * (yaw - at_rows[0]), L0 * pit])


@pytest.mark.parametrize("solver", [0, 1])
def test_three_node_substep_matches_newton_solution(solver):
    """Brute force: on a 3-node chain (2 stretch + yaw + pitch rows) one implicit substep
    is solved by Newton's method on  M (x - x~) = J(x)^T lambda,  c(x) + alpha~ lambda = 0
    (finite-difference Jacobians).  The Jacobi iterates (solver 0) and the Newton + PCR
    steps (solver 1) drive the residual to 1e-12 and land on that solution up to the
    second-order term both drop (x moves by M^-1 J^T dlambda with J of the current iterate)."""
    w = one(W.single_snake(), n_links=1, seg_per_link=2, alpha_b=2e-4, alpha_s=1e-6,
            tau_inf=1e-12, tau_def=1e-12, damping=0.0)
    dt = 1.0 / 1200.0
    s = W.solver_settings(dt=dt, n_sub=1, tol=1e-12, iters=200000, contact=False, solver=solver)
    o = oracle.OracleSim(w, s)
    rng = np.random.default_rng(7)
    o.x += rng.normal(scale=1e-4, size=o.x.shape)
    o.v[:] = rng.normal(scale=0.02, size=o.v.shape)
    p = 0.01
    o.press[0] = [p, 0.0]
    x0, v0 = o.x.copy(), o.v.copy()
    o.step(1, ucmd=np.array([p]))
    assert o.resid[0] < 1e-12
    # Newton on the full system
    m, L0 = 0.01, 0.02
    theta = 20.0 * p * L0
    at = np.array([1e-6, 1e-6, 2e-4, 2e-4]) / dt ** 2
    xt = x0 + dt * (v0 + dt * np.array([0, 0, -G]))

    def F(z):
        x = z[:9].reshape(3, 3)
        lam = z[9:]
        c = _c_fd(x, L0, [theta])
        J = np.zeros((4, 9))
        for d in range(9):
            xp, xm = x.copy().ravel(), x.copy().ravel()
            xp[d] += 1e-7
            xm[d] -= 1e-7
            J[:, d] = (_c_fd(xp.reshape(3, 3), L0, [theta]) - _c_fd(xm.reshape(3, 3), L0, [theta])) / 2e-7
        return np.concatenate([m * (x.ravel() - xt.ravel()) - J.T @ lam, c + at * lam])

    z = np.concatenate([xt.ravel(), np.zeros(4)])
    for _ in range(30):
        f = F(z)
        Jf = np.zeros((13, 13))
        for d in range(13):
            zp, zm = z.copy(), z.copy()
            hd = 1e-9 if d < 9 else 1e-12
            zp[d] += hd
            zm[d] -= hd
            Jf[:, d] = (F(zp) - F(zm)) / (2 * hd)
        z = z - np.linalg.solve(Jf, f)
    xn = z[:9].reshape(3, 3)
    disp = np.abs(xn - xt).max()
    assert disp > 1e-6  # the substep does move the nodes
    assert np.abs(o.x - xn).max() < 2e-3 * disp


def test_sliding_node_pair_stops_at_coulomb_distance():
    """Coulomb friction (Sec. IV, cone |lambda_f| <= mu lambda_n): a node pair sliding along
    its axis at v0 loses mu g h of speed per substep while it slides and sticks once a
    substep's predicted slip is below mu g h^2; the stop distance follows that recursion,
    which tends to v0^2 / (2 mu g)."""
    mu, v0 = 0.5, 0.4
    w = one(W.pendulum(0.02), n_fixed=0, z0=0.01, mu=mu)
    s = W.solver_settings(tol=1e-12, iters=20000)
    o = oracle.OracleSim(w, s)
    o.v[:, 0] = v0
    h = s["dt"] / s["n_sub"]
    o.step(12)
    dist, v = 0.0, v0
    while h * v > mu * G * h * h:
        dist += h * v - mu * G * h * h
        v -= mu * G * h
    assert np.allclose(o.x[:, 0] - [0.0, 0.02], dist, rtol=1e-7, atol=1e-12)
    assert np.abs(o.v).max() < 1e-10
    assert dist == pytest.approx(v0 ** 2 / (2 * mu * G), rel=0.02)
    # resting on the ground: lambda_n carries the weight impulse m g h^2
    assert np.allclose(o.lam[:, 3], 0.01 * G * h * h, rtol=1e-9)


# ------------------------------------------------------------------ Newton + PCR (Sec. IV-D)
def _pcr_case():
    w = one(W.single_snake(), n_links=2, seg_per_link=4, damping=0.0, tau_inf=1e-12, tau_def=1e-12)
    rng = np.random.default_rng(5)
    return w, rng


def test_pcr_newton_step_solves_the_schur_system():
    """One Newton step with enough PCR iterations (finite termination of the conjugate
    residual method on a symmetric positive definite system) equals the dense solution of
    (J M^-1 J^T + alpha~) dlambda = -c at the predicted positions, with J assembled here
    from the oracle's row gradients, and moves the nodes by M^-1 J^T dlambda."""
    w, rng = _pcr_case()
    dt, m_it = 1.0 / 1200.0, 40
    s = W.solver_settings(dt=dt, n_sub=1, tol=0.0, iters=1 + m_it, contact=False, solver=1, pcr_iters=m_it)
    o = oracle.OracleSim(w, s)
    o.x += rng.normal(scale=2e-4, size=o.x.shape)
    o.v[:] = rng.normal(scale=0.05, size=o.v.shape)
    x0, v0 = o.x.copy(), o.v.copy()
    o.step(1, ucmd=np.array([0.0, 0.0]))
    assert o.iters[0] == 1 + m_it
    xt = x0 + dt * (v0 + dt * np.array([0.0, 0.0, -G]))
    c, g, on = oracle.rows(w, s, xt, x0, np.zeros((2, 2)))
    N = xt.shape[0]
    rows = [(i, k) for i in range(N) for k in range(3) if on[i, k]]
    nodes = {0: (0, 1), 1: (-1, 0, 1), 2: (-1, 0, 1)}
    J = np.zeros((len(rows), 3 * N))
    for r, (i, k) in enumerate(rows):
        for l, off in enumerate(nodes[k]):
            J[r, 3 * (i + off):3 * (i + off) + 3] = g[i, k, l]
    at = np.array([(1e-8 if k == 0 else 1e-4) / dt ** 2 for i, k in rows])
    A = J @ J.T / 0.01 + np.diag(at)
    dl = np.linalg.solve(A, -np.array([c[i, k] for i, k in rows]))
    got = np.array([o.lam[i, k] for i, k in rows])
    assert np.allclose(got, dl, rtol=1e-8, atol=1e-14 * np.abs(dl).max())
    assert np.allclose(o.x, xt + (J.T @ dl / 0.01).reshape(N, 3), atol=1e-13)


def test_pcr_and_jacobi_reach_the_same_substep_solution():
    """Newton + PCR and the Jacobi relaxation solve the same substep system of a 9-node
    chain to residual 1e-11.  Both move x by M^-1 J^T dlambda with J of the current
    iterate, so where they end depends on the path by a second-order term (here up to
    ~0.4 % of the substep's displacement; the 3-node brute force above bounds it against
    the exact implicit solution); the Newton solve needs far fewer matrix-vector products
    than Jacobi needs passes."""
    w, rng = _pcr_case()
    dx = rng.normal(scale=2e-4, size=(9, 3))
    v = rng.normal(scale=0.05, size=(9, 3))
    out = {}
    dt = 1.0 / 1200.0
    for solver in (0, 1):
        s = W.solver_settings(dt=dt, n_sub=1, tol=1e-11, iters=200000, contact=False,
                              solver=solver, pcr_iters=20)
        o = oracle.OracleSim(w, s)
        o.x += dx
        x0 = o.x.copy()
        o.v[:] = v
        o.step(1, ucmd=np.array([0.3, -0.2]))
        assert o.resid[0] <= 1e-11
        out[solver] = (o.x.copy(), o.lam.copy(), int(o.iters[0]))
    xt = x0 + dt * (v + dt * np.array([0.0, 0.0, -G]))
    disp = np.abs(out[0][0] - xt).max()
    assert disp > 1e-6
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-2 * disp
    l0, l1 = out[0][1][:, :3], out[1][1][:, :3]
    assert np.abs(l0 - l1).max() < 5e-2 * np.abs(l0).max()
    assert out[1][2] < 0.2 * out[0][2], (out[0][2], out[1][2])


def _slide(mu, mu_side, v0, axis):
    w = one(W.pendulum(0.02), n_fixed=0, z0=0.01, mu=mu, mu_side=mu_side)
    s = W.solver_settings(tol=1e-12, iters=20000)
    o = oracle.OracleSim(w, s)
    o.v[:, axis] = v0
    o.step(20)  # 0.33 s: past the stop time v0 / (mu g) of every case below
    return o, s["dt"] / s["n_sub"]


def _coulomb_stop(mu, v0, h):
    dist, v = 0.0, v0
    while h * v > mu * G * h * h:
        dist += h * v - mu * G * h * h
        v -= mu * G * h
    return dist


def test_anisotropic_friction_along_and_across_the_body():
    """Anisotropic friction (wheels / scales, Sec. V): the node pair of the sliding test
    lies along x; sliding along its axis it stops after the Coulomb distance of mu, sliding
    across it after that of mu_side; with mu_side = mu the trajectory is the isotropic one."""
    mu, mu_side, v0 = 0.2, 0.7, 0.4
    o, h = _slide(mu, mu_side, v0, 0)
    assert np.allclose(o.x[:, 0] - [0.0, 0.02], _coulomb_stop(mu, v0, h), rtol=1e-7, atol=1e-12)
    assert np.abs(o.x[:, 1]).max() < 1e-12
    o, h = _slide(mu, mu_side, v0, 1)
    assert np.allclose(o.x[:, 1], _coulomb_stop(mu_side, v0, h), rtol=1e-7, atol=1e-12)
    assert np.allclose(o.x[:, 0], [0.0, 0.02], atol=1e-12)
    w = W.batched(n=4, seed=8)
    s = W.solver_settings(iters=40)
    a = oracle.OracleSim(w, s)
    w2 = {k: v.copy() for k, v in w.items()}
    w2["mu_side"] = w2["mu"].copy()
    b = oracle.OracleSim(w2, s)
    a.step(4)
    b.step(4)
    assert np.abs(a.x - b.x).max() <= 1e-12 * np.abs(a.x).max()


def test_calibration_gradient_matches_central_differences():
    """Forward-mode dual numbers through the oracle against central differences (step 1e-3
    relative) of the same loss, in a contact-free window with a fixed iteration count."""
    w = W.subset(W.calibration(n=2, seed=11)[0], [0, 1])
    s = W.solver_settings(iters=10, contact=False)
    truth = oracle.OracleSim(w, s)
    target = truth.step(8, tip=True)
    w2 = {k: v.copy() for k, v in w.items()}
    w2["alpha_b"] *= 1.3
    w2["damping"] *= 0.7
    w2["tau_inf"] *= 1.2
    w2["tau_def"] *= 0.8
    w2["gain"] *= 1.1
    o = oracle.OracleSim(w2, s)
    loss, grad = o.calib_grad(8, target)
    names = ["alpha_b", "damping", "tau_inf", "tau_def", "gain"]
    for j, nm in enumerate(names):
        for sgn_snake in range(2):
            hstep = 1e-3 * w2[nm][sgn_snake]
            lp = []
            for sg in (1, -1):
                wp = {k: v.copy() for k, v in w2.items()}
                wp[nm][sgn_snake] += sg * hstep
                op = oracle.OracleSim(wp, s)
                tp = op.step(8, tip=True)
                lp.append(np.mean(np.sum((tp[:, sgn_snake] - target[:, sgn_snake]) ** 2, -1)))
            fd = (lp[0] - lp[1]) / (2 * hstep)
            assert grad[sgn_snake, j] == pytest.approx(fd, rel=2e-3, abs=1e-9 * abs(loss[sgn_snake]) / hstep), (nm, sgn_snake)


@pytest.mark.parametrize("mu_side", [0.0, 0.9])
def test_env_steps_are_equivariant_under_rotations_about_the_vertical(mu_side):
    """Every row is invariant under rotations about z (stretch, heading difference,
    elevation, contact height) and the friction pair is limited by a disc, or an ellipse
    in the body frame, so two snakes that differ only by their initial heading evolve
    into each other rotated, through unconverged fixed-count Jacobi passes as well."""
    w = W.batched(n=2, seed=21, links=(3, 3))
    for k in W.FLOAT_FIELDS:
        w[k][1] = w[k][0]
    theta = 1.1
    w["yaw0"][:] = [0.4, 0.4 + theta]
    w["x0"][:] = 0.0
    w["y0"][:] = 0.0
    w["mu_side"][:] = mu_side
    o = oracle.OracleSim(w, W.solver_settings(iters=10))
    o.step(3)
    c, s_ = math.cos(theta), math.sin(theta)
    Rz = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]])
    a, b = o.x[o.snake_nodes(0)], o.x[o.snake_nodes(1)]
    assert np.abs(b - a @ Rz.T).max() < 1e-12
    va, vb = o.v[o.snake_nodes(0)], o.v[o.snake_nodes(1)]
    assert np.abs(vb - va @ Rz.T).max() < 1e-9 * np.abs(va).max()
    assert np.abs(va).max() > 1e-3  # the snakes are moving


@pytest.mark.parametrize("mu_side,tol", [(0.0, 0.0), (0.9, 0.0), (0.0, 1e-4)])
def test_env_steps_are_equivariant_under_horizontal_translations(mu_side, tol):
    """The ground plane, gravity and every row depend on position differences and on
    heights only, and the friction pair is anchored at the substep start, so two snakes
    that differ only by a horizontal offset of their start evolve into each other
    shifted (fixed-count passes, and to a tolerance with the same update counts); a term
    that used an absolute horizontal position would break it."""
    w = W.batched(n=2, seed=22, links=(3, 3))
    for k in W.FLOAT_FIELDS:
        w[k][1] = w[k][0]
    off = np.array([3.75, -2.5, 0.0])
    w["x0"][:] = [0.1, 0.1 + off[0]]
    w["y0"][:] = [-0.2, -0.2 + off[1]]
    w["mu_side"][:] = mu_side
    o = oracle.OracleSim(w, W.solver_settings(iters=5000 if tol > 0 else 10, tol=tol))
    o.step(3)
    a, b = o.x[o.snake_nodes(0)], o.x[o.snake_nodes(1)]
    assert np.abs(b - (a + off)).max() < 1e-9
    va, vb = o.v[o.snake_nodes(0)], o.v[o.snake_nodes(1)]
    assert np.abs(vb - va).max() < 1e-6 * max(1.0, np.abs(va).max())
    assert np.abs(va).max() > 1e-3  # the snakes are moving
    if tol > 0:
        assert o.iters[0] == o.iters[1]
