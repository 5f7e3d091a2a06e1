"""Pins of the tetrahedral soft-link oracle (Sec. III-A, III-B, IV-A, IV-D) against the
mathematics: scipy's polar decomposition, strains of known deformations, central
differences, the textbook linear FEM stiffness assembled here from shape functions,
momentum conservation and the actuation rest length of Eq. 2."""
import numpy as np
import pytest

import workloads as W
from oracle import fem as F


def _rot(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    return q if np.linalg.det(q) > 0 else -q


def _rest_tet():
    return np.array([[0.0, 0.0, 0.0], [0.011, 0.001, -0.002], [0.002, 0.009, 0.001], [-0.001, 0.002, 0.012]])


def test_polar_matches_scipy():
    sl = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(1)
    for k in range(20):
        A = rng.normal(size=(3, 3)) * (0.1 if k % 2 else 1.0) + np.eye(3)
        if np.linalg.det(A) <= 0:
            continue
        R, S = F.polar(A)
        u, p = sl.polar(A)
        assert np.abs(R - u).max() < 1e-12 and np.abs(S - p).max() < 1e-12
        assert abs(np.linalg.det(R) - 1.0) < 1e-12


def test_polar_rejects_inverted():
    R, S = F.polar(np.diag([1.0, 1.0, -1.0]))
    assert np.isnan(R).all() and np.isnan(S).all()


def test_strain_of_rigid_motion_is_zero():
    rng = np.random.default_rng(2)
    X = _rest_tet()
    for _ in range(10):
        Q = _rot(rng)
        x = X @ Q.T + rng.normal(size=3)
        c, G, R, vol = F.tet(X, x)
        assert np.abs(c).max() < 1e-12
        assert np.abs(R - Q).max() < 1e-12
        assert vol == pytest.approx(np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], 1)) / 6)


def test_strain_of_rotated_symmetric_stretch():
    """x = Q U X with U = I + E symmetric positive definite: the polar factors are Q and U,
    so the strains are E in Voigt order xx yy zz yz xz xy (tensor shears)."""
    rng = np.random.default_rng(3)
    X = _rest_tet()
    for _ in range(10):
        E = rng.normal(size=(3, 3)) * 0.05
        E = 0.5 * (E + E.T)
        Q = _rot(rng)
        x = X @ (Q @ (np.eye(3) + E)).T
        c, _, R, _ = F.tet(X, x)
        want = [E[0, 0], E[1, 1], E[2, 2], E[1, 2], E[0, 2], E[0, 1]]
        assert np.abs(c - want).max() < 1e-12
        assert np.abs(R - Q).max() < 1e-11


def test_gradient_matches_central_differences_at_scaled_rotated_rest():
    """At x = s Q X the stretch is isotropic, where holding R fixed is exact: the rows'
    gradients equal the central differences of the strains."""
    rng = np.random.default_rng(4)
    X = _rest_tet()
    for s in (1.0, 1.07, 0.93):
        x = s * X @ _rot(rng).T
        _, G, _, _ = F.tet(X, x)
        h = 1e-7
        for a in range(4):
            for d in range(3):
                xp, xm = x.copy(), x.copy()
                xp[a, d] += h
                xm[a, d] -= h
                fd = (F.tet(X, xp)[0] - F.tet(X, xm)[0]) / (2 * h)
                assert np.abs(fd - G[:, a, d]).max() < 1e-6 * np.abs(G).max()
        assert np.abs(G.sum(1)).max() < 1e-9 * np.abs(G).max()  # rows are translation invariant


def _small_mesh(rows=True):
    M = W.fem_link_mesh(m=4, n_sec=3, length=0.04, radius=0.0125)
    if not rows:
        M = dict(M, rows=np.zeros((0, 2), np.int32), kinds=np.zeros(0, np.int32))
    return M


def _lumped_masses(M, rho):
    m = np.zeros(len(M["X"]))
    for t in M["tets"]:
        V = abs(np.linalg.det(M["X"][t[1:]] - M["X"][t[0]])) / 6
        m[t] += rho * V / 4
    return m


def _linear_fem_stiffness(M, Y, nu):
    """K = sum_e V_e Y B_e^T C^-1 B_e with B_e from the linear shape functions of each
    element (coefficients of [1 x y z] solved at its four vertices); strains in Voigt
    order xx yy zz yz xz xy with tensor shears, C the element compliance pattern."""
    X, T = M["X"], M["tets"]
    n = len(X)
    K = np.zeros((3 * n, 3 * n))
    C = np.zeros((6, 6))
    C[:3, :3] = -nu
    np.fill_diagonal(C[:3, :3], 1.0)
    C[3:, 3:] = np.eye(3) * (1.0 + nu)
    D = np.linalg.inv(C) * Y
    for t in T:
        A = np.hstack([np.ones((4, 1)), X[t]])
        coef = np.linalg.inv(A)  # column a: shape function N_a = coef[:, a] . [1 x y z]
        dN = coef[1:, :].T       # [4, 3]
        B = np.zeros((6, 12))
        for a in range(4):
            gx, gy, gz = dN[a]
            B[0, 3 * a] = gx
            B[1, 3 * a + 1] = gy
            B[2, 3 * a + 2] = gz
            B[3, 3 * a + 1], B[3, 3 * a + 2] = 0.5 * gz, 0.5 * gy
            B[4, 3 * a], B[4, 3 * a + 2] = 0.5 * gz, 0.5 * gx
            B[5, 3 * a], B[5, 3 * a + 1] = 0.5 * gy, 0.5 * gx
        V = abs(np.linalg.det(A)) / 6
        idx = np.array([[3 * v, 3 * v + 1, 3 * v + 2] for v in t]).ravel()
        K[np.ix_(idx, idx)] += V * B.T @ D @ B
    return K


@pytest.mark.parametrize("nu", [0.3, 0.45])
def test_static_sag_matches_linear_fem(nu):
    """A clamped link under a tiny gravity load settles (damped, every substep solved to
    1e-13) at the solution of the linear FEM system K u = m g of its free particles."""
    M = _small_mesh(rows=False)
    g = (0.0, -2e-3, -1e-3)
    w = W.fem_const_pressure(1, [0.0], poisson=nu, damping=40.0)
    s = W.fem_settings(dt=1.0 / 60.0, n_sub=1, iters=20000, tol=1e-13, pcr_iters=400, gravity=g)
    o = F.OracleFem(M, w, s, n_threads=1)
    for _ in range(40):
        o.step(1)
    assert np.abs(o.v).max() < 1e-12
    free = np.flatnonzero(M["fixed"] == 0)
    K = _linear_fem_stiffness(M, w["youngs"][0], nu)
    m = _lumped_masses(M, w["density"][0])
    dof = np.array([[3 * v, 3 * v + 1, 3 * v + 2] for v in free]).ravel()
    f = (m[free][:, None] * np.asarray(g)[None, :]).ravel()
    u = np.linalg.solve(K[np.ix_(dof, dof)], f).reshape(-1, 3)
    got = o.x[0, free] - M["X"][free]
    assert np.abs(got - u).max() < 2e-4 * np.abs(u).max()


def test_static_sag_with_compliant_distance_rows():
    """The same settling with the centre-layer and perimeter rows made compliant (alpha):
    each adds the spring stiffness (1 / alpha) n n^T between its two particles to K."""
    M = _small_mesh(rows=True)
    g = (0.0, -2e-3, -1e-3)
    a_in, a_pe = 2e-3, 5e-3
    w = W.fem_const_pressure(1, [0.0], poisson=0.3, damping=40.0, alpha_inext=a_in, alpha_perim=a_pe)
    s = W.fem_settings(dt=1.0 / 60.0, n_sub=1, iters=20000, tol=1e-13, pcr_iters=400, gravity=g)
    o = F.OracleFem(M, w, s, n_threads=1)
    for _ in range(40):
        o.step(1)
    X = M["X"]
    K = _linear_fem_stiffness(M, w["youngs"][0], 0.3)
    for (i, j), kind in zip(M["rows"], M["kinds"]):
        if kind not in (W.FEM_INEXT, W.FEM_PERIM):
            continue  # actuation rows do not exist at zero pressure
        n = (X[j] - X[i]) / np.linalg.norm(X[j] - X[i])
        k = np.outer(n, n) / (a_in if kind == W.FEM_INEXT else a_pe)
        for a, b, sg in ((i, i, 1), (j, j, 1), (i, j, -1), (j, i, -1)):
            K[3 * a:3 * a + 3, 3 * b:3 * b + 3] += sg * k
    free = np.flatnonzero(M["fixed"] == 0)
    m = _lumped_masses(M, w["density"][0])
    dof = np.array([[3 * v, 3 * v + 1, 3 * v + 2] for v in free]).ravel()
    f = (m[free][:, None] * np.asarray(g)[None, :]).ravel()
    u = np.linalg.solve(K[np.ix_(dof, dof)], f).reshape(-1, 3)
    got = o.x[0, free] - X[free]
    assert np.abs(got - u).max() < 2e-4 * np.abs(u).max()
    # the rows are stiff enough to matter: without them the sag differs
    u0 = np.linalg.solve(_linear_fem_stiffness(M, w["youngs"][0], 0.3)[np.ix_(dof, dof)], f).reshape(-1, 3)
    assert np.abs(u0 - u).max() > 0.05 * np.abs(u).max()


def test_curvature_is_linear_in_small_pressures():
    """Sec. VI-A: the link's curvature grows linearly with pressure in the small-strain
    range; the settled tip deflection at 2 p is twice that at p to 1 %."""
    M = W.fem_link_mesh(m=4, n_sec=5, length=0.05)
    w = W.fem_const_pressure(2, [200.0, 400.0], poisson=0.3, damping=40.0)
    s = W.fem_settings(n_sub=1, iters=20000, tol=1e-12, pcr_iters=300)
    o = F.OracleFem(M, w, s)
    for _ in range(40):
        o.step(1)
    tip = (o.x[:, -9:] - M["X"][None, -9:]).mean(1)[:, 1]
    assert tip[0] > 0 and tip[1] / tip[0] == pytest.approx(2.0, rel=1e-2)


def test_newton_step_equals_dense_schur_solve():
    """Sec. IV-D: one Newton step whose PCR iterations run to convergence moves the
    particles by M^-1 J^T dlambda with (J M^-1 J^T + E / h^2) dlambda = -c, assembled here
    densely from the element rows (the paper's compliance block per element) and the
    centre-layer, perimeter and driven-chamber distance rows at the predicted positions."""
    M = _small_mesh(rows=True)
    X, T, fixed = M["X"], M["tets"], M["fixed"]
    p, dt, g = 3000.0, 1.0 / 60.0, np.array([0.0, -1.0, -9.81])
    w = W.fem_const_pressure(1, [p], poisson=0.45, alpha_inext=1e-5, alpha_perim=2e-5)
    K = 3000
    s = W.fem_settings(dt=dt, n_sub=1, iters=1 + K, tol=0.0, pcr_iters=K, gravity=g)
    o = F.OracleFem(M, w, s, n_threads=1)
    o.step(1)
    assert o.mv[0] == 1 + K
    P, h = len(X), dt
    Y, nu = w["youngs"][0], w["poisson"][0]
    m = _lumped_masses(M, w["density"][0])
    Wm = np.where(fixed == 1, 0.0, 1.0 / m)
    xt = X + np.where(fixed[:, None] == 1, 0.0, h * h * g[None, :])
    C = np.zeros((6, 6))
    C[:3, :3] = -nu
    np.fill_diagonal(C[:3, :3], 1.0)
    C[3:, 3:] = np.eye(3) * (1.0 + nu)
    J, c, comp = [], [], []
    for t in T:
        ct, G, _, vol = F.tet(X[t], xt[t])
        for k in range(6):
            row = np.zeros(3 * P)
            for a in range(4):
                row[3 * t[a]:3 * t[a] + 3] = G[k, a]
            J.append(row)
            c.append(ct[k])
        comp.append(C / (vol * Y * h * h))
    eps = 1.0 + abs(p) / Y
    for (i, j), kind in zip(M["rows"], M["kinds"]):
        if kind == W.FEM_ACT_LEFT or Wm[i] + Wm[j] == 0.0:
            continue  # the left chamber is not driven; rows between held particles do not exist
        r0 = np.linalg.norm(X[j] - X[i])
        e = xt[j] - xt[i]
        n = e / np.linalg.norm(e)
        row = np.zeros(3 * P)
        row[3 * j:3 * j + 3], row[3 * i:3 * i + 3] = n, -n
        J.append(row)
        c.append(np.linalg.norm(e) - (r0 * eps if kind == W.FEM_ACT_RIGHT else r0))
        alpha = {W.FEM_INEXT: w["alpha_inext"][0], W.FEM_PERIM: w["alpha_perim"][0]}.get(kind, w["alpha_act"][0])
        comp.append(np.array([[alpha / (h * h)]]))
    J, c = np.array(J), np.array(c)
    E = np.zeros((len(c), len(c)))
    o_ = 0
    for B in comp:
        E[o_:o_ + len(B), o_:o_ + len(B)] = B
        o_ += len(B)
    Wv = np.repeat(Wm, 3)
    dl = np.linalg.solve((J * Wv) @ J.T + E, -c)
    want = xt + (Wv * (J.T @ dl)).reshape(-1, 3)
    assert np.abs(o.x[0] - want).max() < 1e-9 * np.abs(want - xt).max()


@pytest.mark.parametrize("p", [4000.0, 0.0])
def test_residual_is_the_largest_normalised_row_value(p):
    """With no solve (a cap of 0 products) the reported residual is the largest row value
    at the predicted positions with zero multipliers: strains as they are, distance rows
    |length - rest| over their unactuated rest length, the driven chamber's rows at rest
    length r (1 + |p| / Y), the other chamber's rows and rows between held particles absent."""
    M = _small_mesh(rows=True)
    X, fixed = M["X"], M["fixed"]
    rng = np.random.default_rng(6)
    w = W.fem_const_pressure(1, [p])
    o = F.OracleFem(M, w, W.fem_settings(n_sub=1, iters=0), n_threads=1)
    x0 = X + np.where(fixed[:, None] == 1, 0.0, rng.normal(size=X.shape) * 2e-4)
    o.x[0] = x0
    o.step(1)
    assert o.mv[0] == 0 and np.array_equal(o.x[0], x0)
    want = max(np.abs(F.tet(X[t], x0[t])[0]).max() for t in M["tets"])
    eps = 1.0 + p / w["youngs"][0]
    for (i, j), kind in zip(M["rows"], M["kinds"]):
        if kind == W.FEM_ACT_LEFT or (kind == W.FEM_ACT_RIGHT and p == 0) or (fixed[i] and fixed[j]):
            continue
        r0 = np.linalg.norm(X[j] - X[i])
        rest = r0 * eps if kind == W.FEM_ACT_RIGHT else r0
        want = max(want, abs(np.linalg.norm(x0[j] - x0[i]) - rest) / r0)
    assert o.resid[0] == pytest.approx(want, rel=1e-12)


def test_whole_step_is_rotation_equivariant():
    """Every row is invariant under rotations (corotational strains, distances), so a
    frame started from Q x with gravity Q g ends at Q times the frame started from x with
    gravity g, through the unconverged fixed-budget Newton + PCR solve as well."""
    M = _small_mesh(rows=True)
    X, fixed = M["X"], M["fixed"]
    rng = np.random.default_rng(7)
    Q = _rot(rng)
    g = np.array([0.3, -0.5, -9.81])
    x0 = X + np.where(fixed[:, None] == 1, 0.0, rng.normal(size=X.shape) * 1e-4)
    v0 = np.where(fixed[:, None] == 1, 0.0, rng.normal(size=X.shape) * 1e-2)
    w = W.fem_const_pressure(1, [3000.0], poisson=0.45, alpha_inext=1e-5)
    out = []
    for R, gg in ((np.eye(3), g), (Q, Q @ g)):
        o = F.OracleFem(M, w, W.fem_settings(gravity=tuple(gg)), n_threads=1)
        o.x[0] = x0 @ R.T
        o.v[0] = v0 @ R.T
        o.step(2)
        out.append((o.x[0].copy(), o.v[0].copy(), o.resid[0]))
    (x1, v1, r1), (x2, v2, r2) = out
    assert np.abs(x2 - x1 @ Q.T).max() < 1e-12
    assert np.abs(v2 - v1 @ Q.T).max() < 1e-7 * np.abs(v1).max()  # (x rounding / h)
    assert r2 == pytest.approx(r1, rel=1e-8)


def test_actuation_row_rest_length_follows_eq2():
    """One element, three vertices held, a hard actuation row from a held vertex to the
    free one: after a solved substep their distance is r (1 + |p| / Y) when that row's
    chamber is the driven one, and r otherwise."""
    X = _rest_tet()
    base = dict(X=X, tets=np.array([[0, 1, 2, 3]], np.int32), rows=np.array([[0, 3]], np.int32),
                fixed=np.array([1, 1, 1, 0], np.int32))
    r = np.linalg.norm(X[3] - X[0])
    Y = 66243.0
    for kind in (W.FEM_ACT_LEFT, W.FEM_ACT_RIGHT):
        for p in (20000.0, -20000.0):
            M = dict(base, kinds=np.array([kind], np.int32))
            w = W.fem_const_pressure(1, [p], alpha_act=0.0, damping=0.0)
            s = W.fem_settings(n_sub=1, iters=4000, tol=1e-13, pcr_iters=50)
            o = F.OracleFem(M, w, s, n_threads=1)
            o.step(1)
            d = np.linalg.norm(o.x[0, 3] - o.x[0, 0])
            driven = (kind == W.FEM_ACT_RIGHT) == (p > 0)
            want = r * (1 + abs(p) / Y) if driven else r
            assert d == pytest.approx(want, rel=1e-9), (kind, p)


def test_linear_momentum_is_conserved():
    """No held particles, no gravity, no damping: internal rows (elements, distance rows,
    the driven chamber) change no total momentum, sum_i m_i v_i."""
    M = dict(W.fem_link_mesh(m=4, n_sec=4, length=0.05))
    M["fixed"] = np.zeros_like(M["fixed"])
    w = W.fem_const_pressure(1, [5000.0], damping=0.0)
    s = W.fem_settings(n_sub=2, iters=25, pcr_iters=12)
    o = F.OracleFem(M, w, s, n_threads=1)
    rng = np.random.default_rng(5)
    o.v[:] = rng.normal(size=o.v.shape) * 0.01
    m = _lumped_masses(M, w["density"][0])
    p0 = (m[:, None] * o.v[0]).sum(0)
    o.step(3)
    p1 = (m[:, None] * o.v[0]).sum(0)
    assert np.abs(p1 - p0).max() < 1e-12 * np.abs(m[:, None] * o.v[0]).sum()


def test_rest_state_stays_at_rest():
    M = W.fem_link_mesh()
    w = W.fem_const_pressure(2, [0.0, 0.0])
    o = F.OracleFem(M, w, W.fem_settings())
    o.step(3)
    assert np.abs(o.x - M["X"][None]).max() < 1e-15 and np.abs(o.v).max() < 1e-13
    assert o.resid.max() < 1e-12


def test_driven_chamber_bends_the_link_away_from_it():
    """Inflating the right chamber (y < 0) lengthens that side against the inextensible
    centre layer, so the free end swings to +y; the left chamber swings it to -y."""
    M = W.fem_link_mesh()
    w = W.fem_const_pressure(2, [6894.76, -6894.76])
    o = F.OracleFem(M, w, W.fem_settings())
    o.step(10)
    tip = o.x[:, -17:, 1].mean(1)
    assert tip[0] > 1e-3 and tip[1] < -1e-3
    assert abs(tip[0] + tip[1]) < 0.1 * abs(tip[0])
