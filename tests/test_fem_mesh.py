"""The synthetic soft-link mesh (`workloads.fem_link_mesh`, standing in for the paper's
TetGen mesh of Sec. V): conforming, positively oriented, filling the polygonal cylinder,
with the distance rows where the link's structure puts them."""
from collections import Counter
import math

import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("m,n_sec", [(8, 13), (4, 3), (12, 5)])
def test_mesh_is_conforming_and_fills_the_prism(m, n_sec):
    L, R = 0.1, 0.0125
    M = W.fem_link_mesh(m=m, n_sec=n_sec, length=L, radius=R)
    X, T = M["X"], M["tets"]
    assert len(X) == n_sec * (1 + 2 * m) and len(T) == (n_sec - 1) * 9 * m
    vol = np.array([np.linalg.det(X[t[1:]] - X[t[0]]) / 6 for t in T])
    assert (vol > 0).all()
    # the cross-section is the regular m-gon of circumradius R
    assert vol.sum() == pytest.approx(0.5 * m * R * R * math.sin(2 * math.pi / m) * L, rel=1e-12)
    faces = Counter(tuple(sorted(np.delete(t, a))) for t in T for a in range(4))
    # interior faces are shared by two elements; boundary faces: two caps of 3m triangles
    # and 2m triangles on each of the n_sec - 1 side bands
    assert set(faces.values()) == {1, 2}
    assert sum(1 for c in faces.values() if c == 1) == 2 * 3 * m + (n_sec - 1) * 2 * m


def test_distance_rows_follow_the_link_structure():
    m, n_sec = 8, 13
    M = W.fem_link_mesh(m=m, n_sec=n_sec)
    X, rows, kinds = M["X"], M["rows"], M["kinds"]
    d = X[rows[:, 1]] - X[rows[:, 0]]
    cnt = Counter(kinds.tolist())
    # centre plane y = 0: the centre and two particles per ring
    assert cnt[W.FEM_INEXT] == (n_sec - 1) * 5
    assert cnt[W.FEM_PERIM] == n_sec * m
    assert cnt[W.FEM_ACT_LEFT] == cnt[W.FEM_ACT_RIGHT] == (n_sec - 1) * 2 * (m // 2 - 1)
    axial = np.isin(kinds, [W.FEM_INEXT, W.FEM_ACT_LEFT, W.FEM_ACT_RIGHT])
    assert np.allclose(d[axial][:, 1:], 0) and (d[axial][:, 0] > 0).all()
    assert np.allclose(X[rows[kinds == W.FEM_INEXT]][..., 1], 0)
    assert (X[rows[kinds == W.FEM_ACT_LEFT]][..., 1] > 0).all()
    assert (X[rows[kinds == W.FEM_ACT_RIGHT]][..., 1] < 0).all()
    ring = np.linalg.norm(X[rows[kinds == W.FEM_PERIM]][..., 1:], axis=-1)
    assert np.allclose(ring, 0.0125) and np.allclose(d[kinds == W.FEM_PERIM][:, 0], 0)
    assert M["fixed"].sum() == 1 + 2 * m and (X[M["fixed"] == 1][:, 0] == 0).all()
