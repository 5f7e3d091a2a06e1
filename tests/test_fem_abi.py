"""C-ABI of the tetrahedral soft link (include/femlink.h): every declared entry point is
exported and bound, the struct layouts agree with the binding's, and argument validation
answers before any CUDA call (so it runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "femlink.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1904_02833_gb300.build import build
    build()
    from paper_1904_02833_gb300 import _native
    return _native.load()


def test_every_declared_fem_symbol_is_exported_and_bound(lib):
    from paper_1904_02833_gb300 import _native
    names = sorted(set(re.findall(r"^SimStatus\s+(fem_\w+)\s*\(", open(HEADER).read(), re.M)))
    assert len(names) == 8
    for n in names:
        assert hasattr(lib, n), n
        assert n in _native.SIGNATURES, n


def test_fem_struct_layout_matches_header(tmp_path):
    from paper_1904_02833_gb300 import _native as N
    c = tmp_path / "sz.c"
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "femlink.h"\nint main(void){'
                 'printf("%zu %zu %zu\\n", sizeof(FemConfig), sizeof(FemLinkParams), sizeof(FemMesh));'
                 'printf("%zu %zu %zu\\n", offsetof(FemConfig, tol), offsetof(FemConfig, pcr_iters), offsetof(FemConfig, gravity));'
                 'printf("%zu %zu\\n", offsetof(FemLinkParams, alpha_act), offsetof(FemLinkParams, press_offset));'
                 'printf("%zu %zu\\n", offsetof(FemMesh, rest), offsetof(FemMesh, fixed));'
                 'printf("%d %d %d %d\\n", FEM_ROW_INEXT, FEM_ROW_PERIM, FEM_ROW_ACT_LEFT, FEM_ROW_ACT_RIGHT);'
                 'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[:3] == [ctypes.sizeof(N.FemConfig), ctypes.sizeof(N.FemLinkParams), ctypes.sizeof(N.FemMesh)]
    assert out[3:6] == [N.FemConfig.tol.offset, N.FemConfig.pcr_iters.offset, N.FemConfig.gravity.offset]
    assert out[6:8] == [N.FemLinkParams.alpha_act.offset, N.FemLinkParams.press_offset.offset]
    assert out[8:10] == [N.FemMesh.rest.offset, N.FemMesh.fixed.offset]
    assert out[10:] == [W.FEM_INEXT, W.FEM_PERIM, W.FEM_ACT_LEFT, W.FEM_ACT_RIGHT]


def _mesh_struct(N, M):
    keep = dict(rest=np.ascontiguousarray(M["X"], np.float64), tets=np.ascontiguousarray(M["tets"], np.int32),
                rows=np.ascontiguousarray(M["rows"], np.int32), kinds=np.ascontiguousarray(M["kinds"], np.int32),
                fixed=np.ascontiguousarray(M["fixed"], np.int32))
    m = N.FemMesh()
    m.n_particles, m.n_tets, m.n_rows = len(keep["rest"]), len(keep["tets"]), len(keep["rows"])
    for k, a in keep.items():
        setattr(m, k, a.ctypes.data_as(ctypes.c_void_p))
    return m, keep


def test_fem_argument_validation_without_gpu(lib):
    from paper_1904_02833_gb300 import _native as N
    from paper_1904_02833_gb300.fem import make_fem_config, make_fem_params
    M = W.fem_link_mesh(m=4, n_sec=3)
    cfg = make_fem_config(W.fem_settings())
    prm = make_fem_params(W.fem_links(2))
    h = ctypes.c_void_p()

    def create(cfg=cfg, mesh=M, n=2, prm=prm):
        m, keep = _mesh_struct(N, mesh)
        st = lib.fem_create(ctypes.byref(cfg), ctypes.byref(m), n, prm, None, ctypes.byref(h))
        return st, lib.sim_last_error().decode()

    assert create(n=0) == (N.SIM_EINVAL, "n_links < 1 or null params")
    st, msg = create(cfg=make_fem_config(W.fem_settings(n_sub=0)))
    assert st == N.SIM_EINVAL and "n_sub" in msg
    st, msg = create(cfg=make_fem_config(W.fem_settings(pcr_iters=0)))
    assert st == N.SIM_EINVAL and "pcr_iters" in msg
    bad = dict(M, tets=M["tets"].copy())
    bad["tets"][3, 1] = len(M["X"])
    st, msg = create(mesh=bad)
    assert st == N.SIM_EINVAL and "element 3" in msg
    inv = dict(M, tets=M["tets"].copy())
    inv["tets"][5, [1, 2]] = inv["tets"][5, [2, 1]]
    st, msg = create(mesh=inv)
    assert st == N.SIM_EINVAL and "non-positive rest volume" in msg
    lone = dict(M, X=np.vstack([M["X"], [[1.0, 1.0, 1.0]]]), fixed=np.append(M["fixed"], 0).astype(np.int32))
    st, msg = create(mesh=lone)
    assert st == N.SIM_EINVAL and "belongs to no element" in msg
    badrow = dict(M, kinds=M["kinds"].copy())
    badrow["kinds"][0] = 7
    st, msg = create(mesh=badrow)
    assert st == N.SIM_EINVAL and "distance row 0" in msg
    p2 = make_fem_params(W.fem_links(2))
    p2[1].poisson = 0.5
    st, msg = create(prm=p2)
    assert st == N.SIM_EINVAL and "link 1" in msg
    big = W.fem_link_mesh(m=12, n_sec=13)  # 1296 elements > 1024
    st, msg = create(mesh=big)
    assert st == N.SIM_EINVAL and "limits" in msg
    assert h.value is None
    for f in ("fem_step", "fem_destroy"):
        assert getattr(lib, f)(None, *([1] if f == "fem_step" else [])) == N.SIM_EINVAL
