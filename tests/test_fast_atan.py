"""The solver's own arctangent (an odd polynomial fitted for the library, with the
pi/2 - atan(1/t) reduction) against the error bound it is used under: the bend angles
feed rows whose tolerance is 1e-4 x L0, so 2e-7 rad is far inside it.  The polynomial
is evaluated exactly as the kernel does (FP32 fused multiply-adds in Horner order),
with the coefficients read from the kernel source."""
import math
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1904_02833_gb300", "csrc", "solver.cuh")


def coeffs():
    body = open(SRC).read()
    fn = body[body.index("float atan_unit(float t)"):body.index("float atan_any(float t)")]
    return [np.float32(float(c)) for c in re.findall(r"(-?\d\.\d+e[-+]\d+)f", fn)]


def fmaf(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def atan_unit(t, c):
    t = np.float32(t)
    s = np.float32(t * t)
    p = c[0]
    for ci in c[1:]:
        p = fmaf(p, s, ci)
    return np.float32(t * p)


def atan_any(t, c):
    a = abs(np.float32(t))
    if a <= 1:
        return atan_unit(t, c)
    r = atan_unit(np.float32(1.0) / a, c)
    return math.copysign(float(np.float32(np.float32(1.57079632679489662) - r)), float(t))


def test_coefficients_present():
    assert len(coeffs()) == 9


def test_error_bound_on_unit_interval_and_beyond():
    c = coeffs()
    worst = 0.0
    for t in np.concatenate([np.linspace(-1, 1, 20001), np.geomspace(1e-8, 1, 2001),
                             -np.geomspace(1e-8, 1, 2001)]):
        worst = max(worst, abs(float(atan_unit(t, c)) - math.atan(float(np.float32(t)))))
    assert worst < 2e-7
    for t in np.concatenate([np.geomspace(1.0001, 1e6, 3001), -np.geomspace(1.0001, 1e6, 3001)]):
        assert abs(atan_any(t, c) - math.atan(float(np.float32(t)))) < 3e-7


def test_relative_accuracy_for_small_angles():
    c = coeffs()
    for t in np.geomspace(1e-7, 1e-2, 500):
        assert abs(float(atan_unit(t, c)) / math.atan(float(np.float32(t))) - 1) < 3e-7


def test_coefficients_are_the_fit_script_output():
    """tests/fit_atan.py regenerates the kernel's coefficients (float32, Horner order);
    allow two float32 units of the last place for LAPACK rounding differences."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("fit_atan", os.path.join(os.path.dirname(__file__), "fit_atan.py"))
    fa = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(fa)
    mine = fa.horner_order(fa.fit())
    for a, b in zip(mine, coeffs()):
        assert abs(float(a) - float(b)) <= 2 * abs(float(np.spacing(np.float32(b)))), (a, b)
