"""Host-side marshalling of the soft-link binding: configs and per-link parameters reach
the C structs field by field (no GPU needed)."""
import numpy as np
import pytest

import workloads as W


def test_config_and_params_marshalling():
    from paper_1904_02833_gb300 import _native as N
    from paper_1904_02833_gb300.fem import make_fem_config, make_fem_params
    s = W.fem_settings(dt=0.02, n_sub=3, iters=17, tol=2e-3, pcr_iters=9, gravity=(0.5, -1.0, -9.81))
    c = make_fem_config(s)
    assert (c.dt, c.n_sub, c.iters, c.pcr_iters) == (0.02, 3, 17, 9)
    assert c.tol == pytest.approx(2e-3) and list(c.gravity) == pytest.approx([0.5, -1.0, -9.81])
    w = W.fem_links(5, seed=9)
    p = make_fem_params(w)
    assert len(p) == 5
    for f in N.FEM_FLOAT_FIELDS:
        got = np.array([getattr(p[i], f) for i in range(5)])
        assert np.allclose(got, w[f].astype(np.float32), rtol=0, atol=0), f


def test_constant_pressure_recipe_drives_the_named_chamber():
    """fem_const_pressure: the command of Eq. 9 evaluates to +-1 at every time (frequency 0,
    phase +-pi/2), so the signed amplitude is the pressure at every substep."""
    w = W.fem_const_pressure(3, [5000.0, -2000.0, 0.0])
    for t in (0.0, 0.37, 12.5):
        u = np.clip(np.sin(2 * np.pi * w["press_freq"] * t + w["press_phase"]) + w["press_offset"], -1, 1)
        assert np.allclose(w["press_amp"] * u, [5000.0, -2000.0, 0.0])
