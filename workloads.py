"""Seeded synthetic snake workloads shared by the CUDA path's tests/bench and the oracle.

This module only draws parameters.  It holds none of the simulation's arithmetic
(no constraint, filter or integrator maths), so the oracle and the CUDA path can both
consume its arrays without sharing any method code.

A workload is a dict of numpy arrays, one entry per snake:

  ints    : n_links, seg_per_link, n_fixed
  floats  : L0, mass, alpha_s, alpha_b, gain, tau_inf, tau_def, mu, damping, radius,
            gait_amp, gait_freq, gait_lag, gait_offset, gait_scale, gait_alternate,
            x0, y0, z0, yaw0, mu_side (sideways friction coefficient; 0 = isotropic mu)

and a dict of global solver settings (dt, n_sub, iters, tol, omega, gravity, contact,
warm start, chamber model).

The shapes follow the paper's snake (four soft links joined by rigid connectors, Sec. III
and Sec. V) and its open-loop gait (Eq. 9, Sec. V-A): links are discretised into
segments of equal rest length, pressure is normalised to [0, 1] per chamber, and the
gait drives one chamber of each link at a time.
"""
from __future__ import annotations

import math

import numpy as np

INT_FIELDS = ("n_links", "seg_per_link", "n_fixed")
FLOAT_FIELDS = (
    "L0", "mass", "alpha_s", "alpha_b", "gain", "tau_inf", "tau_def", "mu",
    "damping", "radius", "gait_amp", "gait_freq", "gait_lag", "gait_offset",
    "gait_scale", "gait_alternate", "x0", "y0", "z0", "yaw0", "mu_side",
)

# Physical defaults of the 1D-actuator snake (segment length, node mass, compliances,
# curvature gain, latency constants, friction, contact radius).
DEFAULTS = dict(
    L0=0.02, mass=0.01, alpha_s=1e-8, alpha_b=1e-4, gain=20.0, tau_inf=0.15,
    tau_def=0.25, mu=0.5, damping=0.05, radius=0.01, gait_amp=1.0, gait_freq=1.0,
    gait_lag=math.pi / 2, gait_offset=0.0, gait_scale=1.0, gait_alternate=0.0,
    x0=0.0, y0=0.0, z0=0.01, yaw0=0.0, mu_side=0.0,
)


def solver_settings(dt=1.0 / 60.0, n_sub=20, iters=10, tol=0.0, omega=1.0 / 3.0,
                    gravity=(0.0, 0.0, -9.81), contact=True, warm=0, beta=1.0, latency=0,
                    k_inflate=0.23, k_deflate=0.23, t_p=0.68 / 8.0, p_source=1.0, law_dt=0.0083,
                    solver=0, pcr_iters=20, net_rows=0, net_every=1, beta_net=-1.0):
    """Global settings: env-step dt, substeps, iteration cap, residual tolerance
    (0 = run exactly `iters` updates), Jacobi relaxation, gravity, ground contact on/off,
    warm start (0 = cold, 1 = beta x previous substep's multipliers, 2 = that plus the
    learned correction), chamber model (0 = first-order latency with tau_inf / tau_def,
    1 = the discrete law of Sec. V-A with gains k_inflate, k_deflate, deflation threshold
    t_p and source pressure p_source in units of the maximum pressure, applied every
    law_dt seconds; defaults: the paper's gains 0.23 / 0.23, T_p = 0.68 psi of an 8 psi
    maximum, source = maximum pressure, its 0.0083 s time step), and the solver (0 = the
    Jacobi relaxation, `iters` capping its passes; 1 = Newton steps each with `pcr_iters`
    preconditioned conjugate residual iterations, Sec. IV-D, `iters` capping the
    matrix-vector products; contact-free only); for the learned warm start, the row kinds
    the network predicts (net_rows 0 = all six, 1 = stretch, yaw and pitch only, 2 = stretch
    only), every how many substeps it runs (net_every; the substeps in between start from
    beta x the previous multipliers) and the weight of the previous multipliers under its
    prediction (beta_net; negative: beta)."""
    return dict(dt=float(dt), n_sub=int(n_sub), iters=int(iters), tol=float(tol),
                omega=float(omega), gravity=tuple(float(g) for g in gravity),
                contact=bool(contact), warm=int(warm), beta=float(beta), latency=int(latency),
                k_inflate=float(k_inflate), k_deflate=float(k_deflate), t_p=float(t_p),
                p_source=float(p_source), law_dt=float(law_dt), solver=int(solver),
                pcr_iters=int(pcr_iters), net_rows=int(net_rows), net_every=int(net_every),
                beta_net=float(beta_net))


def _base(n: int) -> dict:
    w = {k: np.full(n, DEFAULTS[k], dtype=np.float64) for k in FLOAT_FIELDS}
    w["n_links"] = np.full(n, 4, dtype=np.int32)
    w["seg_per_link"] = np.full(n, 10, dtype=np.int32)
    w["n_fixed"] = np.zeros(n, dtype=np.int32)
    return w


def n_nodes(w: dict) -> np.ndarray:
    return (w["n_links"].astype(np.int64) * w["seg_per_link"] + 1)


def subset(w: dict, idx) -> dict:
    idx = np.asarray(idx)
    return {k: np.ascontiguousarray(v[idx]) for k, v in w.items()}


def single_snake() -> dict:
    """One 4-link snake (41 nodes).  Link i is driven with 0.5 + 0.5 sin(2 pi t + i pi/2)
    on alternating sides (sign (-1)^i), mu = 0.5."""
    w = _base(1)
    w["gait_offset"][:] = 0.5
    w["gait_scale"][:] = 0.5
    w["gait_amp"][:] = 1.0
    w["gait_freq"][:] = 1.0
    w["gait_lag"][:] = math.pi / 2
    w["gait_alternate"][:] = 1.0
    w["mu"][:] = 0.5
    return w


def static_sweep(seed: int = 2, n_press: int = 16, n_comp: int = 16) -> dict:
    """Cantilevered single actuators (10 segments, nodes 0 and 1 clamped) held in the air,
    constant chamber pressure on 16 uniformly spaced levels in [0, 1] crossed with 16
    bend compliances drawn log-uniform in [1e-5, 1e-3]."""
    rng = np.random.default_rng(seed)
    n = n_press * n_comp
    w = _base(n)
    press = np.linspace(0.0, 1.0, n_press)
    comp = 10.0 ** rng.uniform(-5.0, -3.0, size=n_comp)
    P, C = np.meshgrid(press, comp, indexing="ij")
    w["n_links"][:] = 1
    w["n_fixed"][:] = 2
    w["alpha_b"][:] = C.ravel()
    # constant command u = p on the "right" chamber: offset p, no oscillation
    w["gait_offset"][:] = P.ravel()
    w["gait_scale"][:] = 0.0
    w["gait_amp"][:] = 1.0
    w["gait_freq"][:] = 0.0
    w["z0"][:] = 1.0
    return w


def batched(n: int = 4096, seed: int = 3, links=(2, 8)) -> dict:
    """Uneven batch: link counts uniform in {2..8}, gait amplitude U[0.3, 1], frequency
    U[0.5, 2] Hz, phase lag U[pi/4, pi], mu U[0.3, 0.8], initial yaw U[0, 2 pi),
    zero offset (the paper's gait, Eq. 9, with phi = 0)."""
    rng = np.random.default_rng(seed)
    w = _base(n)
    w["n_links"][:] = rng.integers(links[0], links[1] + 1, size=n)
    w["gait_amp"][:] = rng.uniform(0.3, 1.0, size=n)
    w["gait_freq"][:] = rng.uniform(0.5, 2.0, size=n)
    w["gait_lag"][:] = rng.uniform(math.pi / 4, math.pi, size=n)
    w["mu"][:] = rng.uniform(0.3, 0.8, size=n)
    w["yaw0"][:] = rng.uniform(0.0, 2 * math.pi, size=n)
    w["gait_offset"][:] = 0.0
    w["gait_scale"][:] = 1.0
    return w


def learned(n: int = 16384, seed: int = 4) -> dict:
    """Evaluation batch for the learned warm start (drawn like `batched`)."""
    return batched(n=n, seed=seed)


def training_seeds(k: int = 4, base: int = 1000) -> list[int]:
    """Seeds for the logged training data; disjoint from every evaluation seed (< 1000)."""
    return [base + i for i in range(k)]


def calibration(n: int = 1024, seed: int = 5) -> tuple[dict, dict]:
    """Calibration batch: 4-link snakes.  Returns (ground truth, initial guess); both draw
    bend compliance log-U[1e-5, 1e-3], damping U[0.01, 0.2], tau_inflate / tau_deflate
    U[0.05, 0.4] s and curvature gain U[10, 30] rad/m; the gait is the paper's Eq. 9."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(2):
        w = _base(n)
        w["alpha_b"][:] = 10.0 ** rng.uniform(-5.0, -3.0, size=n)
        w["damping"][:] = rng.uniform(0.01, 0.2, size=n)
        w["tau_inf"][:] = rng.uniform(0.05, 0.4, size=n)
        w["tau_def"][:] = rng.uniform(0.05, 0.4, size=n)
        w["gain"][:] = rng.uniform(10.0, 30.0, size=n)
        out.append(w)
    shared = rng.uniform(size=(n, 3))
    for w in out:
        w["gait_amp"][:] = 0.5 + 0.5 * shared[:, 0]
        w["gait_freq"][:] = 0.5 + 1.5 * shared[:, 1]
        w["gait_lag"][:] = math.pi / 4 + (3 * math.pi / 4) * shared[:, 2]
    return out[0], out[1]


def pendulum(length: float = 0.1) -> dict:
    """Two nodes: node 0 clamped, node 1 hanging at `length` (one stretch row)."""
    w = _base(1)
    w["n_links"][:] = 1
    w["seg_per_link"][:] = 1
    w["n_fixed"][:] = 1
    w["L0"][:] = length
    w["z0"][:] = 1.0
    w["damping"][:] = 0.0
    w["gait_amp"][:] = 0.0
    return w


# ---------------------------------------------------------------- tetrahedral soft link
# A soft link as the paper models it (Sec. III-A, III-B, IV): a solid silicone body meshed
# with tetrahedra, an inextensible layer along its centre plane, a perimeter held by the
# fibre reinforcement and actuation distance rows along the chambers.  The paper meshes
# its link with TetGen; this generator stands in for that mesh with a radially symmetric
# one of the same kind: `n_sec` cross-sections along the axis (the paper uses 13), each a
# centre particle and two rings of `m` particles (radius R/2 and R), every cross-section
# triangle swept to the next section as a prism split into three tetrahedra.  Geometry and
# connectivity only; no mechanics.

FEM_FLOAT_FIELDS = ("youngs", "poisson", "density", "damping", "alpha_inext", "alpha_perim",
                    "alpha_act", "press_amp", "press_freq", "press_phase", "press_offset")

# Ecoflex 00-30 (Sec. V: Y = 66.243 kPa, nu = 0.4999; specific gravity 1.07), hard
# inextensible and perimeter rows, compliant actuation rows, a 2 psi, 1 Hz pressure wave.
FEM_DEFAULTS = dict(youngs=66243.0, poisson=0.4999, density=1070.0, damping=1.0,
                    alpha_inext=0.0, alpha_perim=0.0, alpha_act=1e-3, press_amp=13790.0,
                    press_freq=1.0, press_phase=0.0, press_offset=0.0)

# distance-row kinds of the link mesh
FEM_INEXT, FEM_PERIM, FEM_ACT_LEFT, FEM_ACT_RIGHT = 0, 1, 2, 3


def fem_link_mesh(m: int = 8, n_sec: int = 13, length: float = 0.1, radius: float = 0.0125) -> dict:
    """Rest particles [P, 3] (axis along x, cross-section point (y, z) = rho (cos phi, sin phi)
    with phi = 2 pi k / m), positively oriented tetrahedra [T, 4], distance rows [D, 2] with
    their kinds [D] and the fixed flags [P] (the first cross-section, held by its rigid
    cap).  The centre plane y = 0 carries the inextensible layer; the left chamber is y > 0,
    the right one y < 0.  m must be a multiple of 4 (particles on the centre plane)."""
    assert m % 4 == 0 and m >= 4 and n_sec >= 2
    per = 1 + 2 * m

    def pid(s, ring, k):
        return s * per + (0 if ring == 0 else 1 + (ring - 1) * m + (k % m))

    phi = 2.0 * math.pi * np.arange(m) / m
    cphi = np.round(np.cos(phi), 12)
    X = np.zeros((n_sec * per, 3))
    for s in range(n_sec):
        xs = length * s / (n_sec - 1)
        X[pid(s, 0, 0)] = (xs, 0.0, 0.0)
        for ring, rho in ((1, 0.5 * radius), (2, radius)):
            for k in range(m):
                X[pid(s, ring, k)] = (xs, rho * math.cos(phi[k]), rho * math.sin(phi[k]))
    tris = []
    for k in range(m):
        tris.append((pid(0, 0, 0), pid(0, 1, k), pid(0, 1, k + 1)))
        tris.append((pid(0, 1, k), pid(0, 2, k), pid(0, 2, k + 1)))
        tris.append((pid(0, 1, k), pid(0, 2, k + 1), pid(0, 1, k + 1)))
    tets = []
    for s in range(n_sec - 1):
        for tri in tris:
            a, b, c = sorted(v + s * per for v in tri)
            A, B, C = a + per, b + per, c + per
            # sorted-vertex split: the diagonal of every side face depends only on the
            # order of its two bottom vertices, so neighbouring prisms agree
            for t in ((a, b, c, A), (b, c, A, B), (c, A, B, C)):
                e1, e2, e3 = X[t[1]] - X[t[0]], X[t[2]] - X[t[0]], X[t[3]] - X[t[0]]
                tets.append(t if np.dot(np.cross(e1, e2), e3) > 0 else (t[0], t[2], t[1], t[3]))
    rows, kinds = [], []
    for s in range(n_sec - 1):
        plane = [pid(s, 0, 0)] + [pid(s, r, k) for r in (1, 2) for k in range(m) if cphi[k] == 0.0]
        for p in plane:
            rows.append((p, p + per)); kinds.append(FEM_INEXT)
    for s in range(n_sec):
        for k in range(m):
            rows.append((pid(s, 2, k), pid(s, 2, k + 1))); kinds.append(FEM_PERIM)
    for s in range(n_sec - 1):
        for side, kind in ((1.0, FEM_ACT_LEFT), (-1.0, FEM_ACT_RIGHT)):
            for r in (1, 2):
                for k in range(m):
                    if cphi[k] * side > 0.0:
                        rows.append((pid(s, r, k), pid(s + 1, r, k))); kinds.append(kind)
    fixed = np.zeros(n_sec * per, np.int32)
    fixed[:per] = 1
    return dict(X=X, tets=np.asarray(tets, np.int32), rows=np.asarray(rows, np.int32),
                kinds=np.asarray(kinds, np.int32), fixed=fixed)


def fem_settings(dt=1.0 / 60.0, n_sub=2, iters=21, tol=0.0, pcr_iters=20, gravity=(0.0, 0.0, 0.0)):
    """Global settings of the link solve: frame dt, substeps (the paper's benchmark runs 2
    per frame with 20 solver iterations each), the cap on matrix-vector products per
    substep, the residual tolerance that ends the Newton loop (0 = run to the cap), PCR
    iterations per Newton step and gravity (off: the link rests on its wheels)."""
    return dict(dt=float(dt), n_sub=int(n_sub), iters=int(iters), tol=float(tol),
                pcr_iters=int(pcr_iters), gravity=tuple(float(g) for g in gravity))


def fem_links(n: int = 1216, seed: int = 6) -> dict:
    """Batch of soft links on the same mesh: Young's modulus U[0.8, 1.2] x 66.243 kPa,
    the paper's Poisson ratio, pressure amplitude U[1, 3] psi, frequency U[0.5, 2] Hz,
    phase U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    w = {k: np.full(n, FEM_DEFAULTS[k], dtype=np.float64) for k in FEM_FLOAT_FIELDS}
    w["youngs"][:] = FEM_DEFAULTS["youngs"] * rng.uniform(0.8, 1.2, size=n)
    w["press_amp"][:] = 6894.76 * rng.uniform(1.0, 3.0, size=n)
    w["press_freq"][:] = rng.uniform(0.5, 2.0, size=n)
    w["press_phase"][:] = rng.uniform(0.0, 2 * math.pi, size=n)
    return w


def fem_const_pressure(n: int, press, **kw) -> dict:
    """Links held at constant pressures `press` (Pa, signed: > 0 inflates the right
    chamber, < 0 the left one)."""
    w = {k: np.full(n, FEM_DEFAULTS[k], dtype=np.float64) for k in FEM_FLOAT_FIELDS}
    w["press_amp"][:] = np.abs(np.broadcast_to(np.asarray(press, np.float64), (n,)))
    w["press_freq"][:] = 0.0
    w["press_phase"][:] = np.where(np.broadcast_to(np.asarray(press), (n,)) < 0, -math.pi / 2, math.pi / 2)
    for k, v in kw.items():
        w[k][:] = v
    return w
