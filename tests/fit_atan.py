"""Fits the solver's arctangent polynomial (the coefficients of atan_unit in
paper_1904_02833_gb300/csrc/solver.cuh) and prints them as the kernel source writes them.

atan(t) on [-1, 1] is approximated by the odd polynomial t P(t^2), P of degree 8, close to
minimax in absolute error: Lawson's algorithm (iteratively reweighted least squares,
C. L. Lawson 1961) on Chebyshev nodes of [0, 1], where each weight is multiplied by the
current absolute error at its node, which drives the weighted least-squares solution
towards the minimax one.  The coefficients are then rounded to float32.

    python tests/fit_atan.py
"""
import numpy as np

DEGREE = 8        # P(s) = sum_j c_j s^j, j = 0..8: t P(t^2) has degree 17
NODES = 4000
ITERATIONS = 400


def fit(degree=DEGREE, nodes=NODES, iterations=ITERATIONS):
    """Coefficients c_0..c_degree of P (c_0 first), float64."""
    k = np.arange(nodes)
    t = 0.5 * (1.0 + np.cos(np.pi * (k + 0.5) / nodes))  # Chebyshev nodes of [0, 1]
    A = np.stack([t ** (2 * j + 1) for j in range(degree + 1)], 1)
    f = np.arctan(t)
    w = np.full(nodes, 1.0 / nodes)
    c = None
    for _ in range(iterations):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], f * sw, rcond=None)
        e = np.abs(A @ c - f)
        w = w * e
        w /= w.sum()
    return c


def horner_order(c):
    """The coefficients in the kernel's Horner order (highest power of s first), float32."""
    return [np.float32(x) for x in c[::-1]]


def main():
    for x in horner_order(fit()):
        print("%.9ef" % float(x))


if __name__ == "__main__":
    main()
