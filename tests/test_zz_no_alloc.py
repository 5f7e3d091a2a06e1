"""The allocation-free forward pass of the warm-start network.

Callers that cannot allocate device memory (a control loop with a hard real-time budget,
or a host application whose device memory belongs to its own allocator) use
mlp_forward_noalloc with a parameter vector they own; its working memory is a fixed
device array inside the library.  This checks it, through the C-ABI, against the
handle-based mlp_forward on two calls in a row with different networks, and that it
refuses a parameter vector its array cannot hold.  Kept in a file that runs last.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_02833_gb300.build import build
    build()
    torch.cuda.set_device(0)


def test_noalloc_forward_matches_handle_forward_twice():
    from paper_1904_02833_gb300 import _native as N
    from paper_1904_02833_gb300.mlp import WarmStartMLP, init_params, pad_features

    lib = N.load()
    rng = np.random.default_rng(12)
    rows = 3001
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((21, 22)):
        params = init_params(seed)
        params[-1] = 0.1 * (call + 1)
        f = rng.normal(size=(rows, 24))
        f[:, :6] = 0
        f[np.arange(rows), rng.integers(0, 6, rows)] = 1.0
        feat = pad_features(torch.tensor(f, dtype=torch.float32, device="cuda"))
        ref = WarmStartMLP(params).forward(feat).cpu().numpy()
        p_dev = torch.tensor(params, dtype=torch.float32, device="cuda")
        out = torch.full((rows,), float("nan"), device="cuda")
        st = lib.mlp_forward_noalloc(ctypes.c_void_p(p_dev.data_ptr()), N.MLP_NUM_PARAMS,
                                     ctypes.c_void_p(feat.data_ptr()), rows,
                                     ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
        assert st == N.SIM_OK, lib.sim_last_error()
        y = out.cpu().numpy()
        scale = max(np.abs(ref).mean() + 1e-3, np.abs(ref).max())
        assert np.isfinite(y).all()
        assert np.abs(y - ref).max() <= 5e-3 * scale, call


def test_noalloc_rejects_a_parameter_vector_it_cannot_hold():
    from paper_1904_02833_gb300 import _native as N

    lib = N.load()
    p = torch.zeros(N.MLP_NUM_PARAMS + 128, device="cuda")
    f = torch.zeros(128, 32, dtype=torch.bfloat16, device="cuda")
    out = torch.zeros(128, device="cuda")
    st = lib.mlp_forward_noalloc(ctypes.c_void_p(p.data_ptr()), N.MLP_NUM_PARAMS + 128,
                                 ctypes.c_void_p(f.data_ptr()), 128, ctypes.c_void_p(out.data_ptr()),
                                 None)
    assert st == N.SIM_EINVAL
    assert b"exactly one" in lib.sim_last_error()


def test_noalloc_and_handle_forward_reject_misaligned_features():
    """The kernels read a feature row as four 16-byte vectors: a feature pointer off a
    16-byte boundary is refused before anything is enqueued, by both entry points."""
    from paper_1904_02833_gb300 import _native as N
    from paper_1904_02833_gb300.mlp import WarmStartMLP, init_params

    lib = N.load()
    params = init_params(3)
    p = torch.tensor(params, dtype=torch.float32, device="cuda")
    f = torch.zeros(129 * 32 + 8, dtype=torch.bfloat16, device="cuda")
    out = torch.zeros(128, device="cuda")
    bad = ctypes.c_void_p(f.data_ptr() + 2 * 4)  # 8 bytes past an aligned base
    st = lib.mlp_forward_noalloc(ctypes.c_void_p(p.data_ptr()), N.MLP_NUM_PARAMS, bad, 128,
                                 ctypes.c_void_p(out.data_ptr()), None)
    assert st == N.SIM_EINVAL and b"aligned" in lib.sim_last_error()
    net = WarmStartMLP(params)
    st = lib.mlp_forward(net.h, bad, 128, ctypes.c_void_p(out.data_ptr()))
    assert st == N.SIM_EINVAL and b"aligned" in lib.sim_last_error()
    net.close()
