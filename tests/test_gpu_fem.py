"""Parity of the tetrahedral soft link on the GPU (fem.cu, through the C-ABI) with the
FP64 oracle, element by element.

Tolerances.  A fixed budget of PCR iterations leaves the solve unconverged (the paper's
budget: 2 substeps of 20 iterations per frame), so FP32 rounding propagates through the
Krylov iterates.  Each case measures that propagation on the oracle itself, running the
same steps in float arithmetic, and allows the GPU 20 times the float-vs-double deviation
of the case, with floors of 2e-6 m on positions and 2e-4 m/s on velocities."""
import numpy as np
import pytest

import workloads as W
from oracle import fem as OF

pytestmark = pytest.mark.gpu


def _gpu(mesh, w, s, frames=1):
    from paper_1904_02833_gb300.fem import FemSim
    sim = FemSim(mesh, w, s)
    sim.step(frames)
    return sim, sim.state()


def _oracle(mesh, w, s, frames=1, fp32=False):
    o = OF.OracleFem(mesh, w, s)
    o.step(frames, fp32=fp32)
    return o


def _check(mesh, w, s, frames=1, idx=None):
    sim, (x, v, r, mv) = _gpu(mesh, w, s, frames)
    ws = w if idx is None else {k: a[idx] for k, a in w.items()}
    o64 = _oracle(mesh, ws, s, frames)
    o32 = _oracle(mesh, ws, s, frames, fp32=True)
    if idx is not None:
        x, v, r, mv = x[idx], v[idx], r[idx], mv[idx]
    tx = max(2e-6, 20 * np.abs(o32.x - o64.x).max())
    tv = max(2e-4, 20 * np.abs(o32.v - o64.v).max())
    tr = max(1e-5, 20 * np.abs(o32.resid - o64.resid).max())
    assert np.abs(x - o64.x).max() <= tx, (np.abs(x - o64.x).max(), tx)
    assert np.abs(v - o64.v).max() <= tv, (np.abs(v - o64.v).max(), tv)
    assert np.abs(r - o64.resid).max() <= tr, (np.abs(r - o64.resid).max(), tr)
    assert np.array_equal(mv, o64.mv)
    return sim, x, o64


def test_one_frame_at_the_papers_budget():
    M = W.fem_link_mesh()
    w = W.fem_links(8, seed=11)
    sim, x, o = _check(M, w, W.fem_settings())
    assert sim.launch_count() == 1
    assert np.abs(x - M["X"][None]).max() > 1e-4  # the links moved


def test_three_frames_nu_045_and_gravity():
    M = W.fem_link_mesh()
    w = W.fem_links(6, seed=12)
    w["poisson"][:] = 0.45
    _check(M, w, W.fem_settings(gravity=(0.0, 0.0, -9.81)), frames=3)


def test_small_mesh_more_substeps_and_iterations():
    """m = 4, two cross-sections (36 elements, 18 particles, one warp): ragged element
    slots, 4 substeps, 60 products per substep in Newton steps of 15 PCR iterations."""
    M = W.fem_link_mesh(m=4, n_sec=2, length=0.02)
    w = W.fem_links(5, seed=13)
    s = W.fem_settings(n_sub=4, iters=60, pcr_iters=15)
    _check(M, w, s, frames=2)


def test_compliant_rows_and_clamped_command():
    """Compliant centre-layer and perimeter rows, offsets that saturate the command
    (clamp at +-1) and a link whose command is exactly zero, over three frames."""
    M = W.fem_link_mesh()
    w = W.fem_links(6, seed=15)
    w["alpha_inext"][:] = 1e-4
    w["alpha_perim"][:] = 3e-4
    w["press_offset"][:] = [1.5, -1.5, 0.4, -0.4, 0.0, 0.0]
    w["press_amp"][5] = 0.0
    _check(M, w, W.fem_settings(), frames=3)


def test_largest_block_and_a_mesh_without_distance_rows():
    """15 cross-sections (1008 elements, 512 threads per block, 205 KB of shared memory,
    the largest launch shape) and the 13-section mesh with no distance rows at all,
    sagging under gravity."""
    M = W.fem_link_mesh(m=8, n_sec=15)
    _check(M, W.fem_links(4, seed=16), W.fem_settings())
    M0 = dict(W.fem_link_mesh(), rows=np.zeros((0, 2), np.int32), kinds=np.zeros(0, np.int32))
    _check(M0, W.fem_links(3, seed=17), W.fem_settings(gravity=(0.0, 0.0, -9.81)), frames=2)


def test_tolerance_stops_the_newton_loop():
    M = W.fem_link_mesh(m=4, n_sec=4, length=0.04)
    w = W.fem_const_pressure(4, [3000.0, -3000.0, 6000.0, 0.0], poisson=0.3)
    s = W.fem_settings(n_sub=1, iters=5000, tol=2e-3, pcr_iters=40)
    sim, (x, v, r, mv) = _gpu(M, w, s)
    o = _oracle(M, w, s)
    assert (r <= 2e-3).all() and (mv < 5000).all()
    assert (o.resid <= 2e-3).all()
    assert mv[3] == 0 and o.mv[3] == 0  # a link at rest needs no product
    assert np.abs(x - o.x).max() < 5e-5


def test_rest_and_direction():
    M = W.fem_link_mesh()
    w = W.fem_const_pressure(3, [0.0, 6894.76, -6894.76])
    sim, (x, v, r, mv) = _gpu(M, w, W.fem_settings(), frames=10)
    assert np.abs(x[0] - M["X"]).max() < 1e-6 and np.abs(v[0]).max() < 1e-4
    tip = x[:, -17:, 1].mean(1)
    assert tip[1] > 1e-3 and tip[2] < -1e-3


def test_full_batch_sampled_links_and_reproducibility():
    """The benchmark's batch (1216 links) in one launch; 12 sampled links against the
    oracle; a second run gives identical bits."""
    M = W.fem_link_mesh()
    w = W.fem_links(1216, seed=6)
    idx = np.sort(np.random.default_rng(0).choice(1216, 12, replace=False))
    sim, x, _ = _check(M, w, W.fem_settings(), idx=idx)
    from paper_1904_02833_gb300.fem import FemSim
    sim2 = FemSim(M, w, W.fem_settings())
    sim2.step(1)
    assert np.array_equal(sim2.state()[0], sim.state()[0])


def test_state_round_trip_and_frame_index():
    M = W.fem_link_mesh(m=4, n_sec=3)
    w = W.fem_links(3, seed=14)
    s = W.fem_settings()
    from paper_1904_02833_gb300.fem import FemSim
    a = FemSim(M, w, s)
    a.step(2)
    xa, va, _, _ = a.state()
    b = FemSim(M, w, s)
    b.set_state(xa, va)
    b.set_frame(2)
    a.step(1)
    b.step(1)
    assert np.array_equal(a.state()[0], b.state()[0])
    xd, vd, rd, mvd = a.state_device()
    assert np.array_equal(xd.cpu().numpy(), a.state()[0])
