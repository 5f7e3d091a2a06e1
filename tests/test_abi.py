"""The C-ABI library: it loads, exports every entry point include/*.h declares, its
struct layouts agree with the binding's, and argument validation answers without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "snakesim.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1904_02833_gb300.build import build
    build()
    from paper_1904_02833_gb300 import _native
    return _native.load()


def declared():
    """Every function declared in include/*.h (snakesim.h, femlink.h)."""
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^(?:SimStatus|const char\*)\s+(\w+)\s*\(", src, re.M))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 45
    assert {"sim_create", "mlp_forward_noalloc", "fem_step", "sim_fp32_fma_probe"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    from paper_1904_02833_gb300 import _native
    assert set(names) - {"sim_last_error"} == set(_native.SIGNATURES)


def test_struct_layout_matches_header(tmp_path):
    from paper_1904_02833_gb300 import _native as N
    c = tmp_path / "sz.c"
    fields = ["n_links", "n_fixed", "mu_side", "L0", "alpha_b", "gait_amp", "yaw0"]
    body = "\n".join('printf("%%zu\\n", offsetof(SnakeParams, %s));' % f for f in fields)
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "snakesim.h"\nint main(void){'
                 'printf("%zu\\n%zu\\n", sizeof(SimConfig), sizeof(SnakeParams));'
                 'printf("%zu\\n%zu\\n", offsetof(SimConfig, tol), offsetof(SimConfig, warm));'
                 'printf("%zu\\n", offsetof(SimConfig, law_dt));'
                 + body + "return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(N.SimConfig)
    assert out[1] == ctypes.sizeof(N.SnakeParams)
    assert out[2] == N.SimConfig.tol.offset and out[3] == N.SimConfig.warm.offset
    assert out[4] == N.SimConfig.law_dt.offset
    for f, off in zip(fields, out[5:]):
        assert getattr(N.SnakeParams, f).offset == off, f


def test_argument_validation_without_gpu(lib):
    """Invalid arguments are rejected before any CUDA call, with a message."""
    from paper_1904_02833_gb300 import _native as N
    from paper_1904_02833_gb300.sim import make_config, make_params
    import workloads as W

    cfg = make_config(W.solver_settings())
    prm = make_params(W.single_snake())
    h = ctypes.c_void_p()
    assert lib.sim_create(ctypes.byref(cfg), 0, prm, None, ctypes.byref(h)) == N.SIM_EINVAL
    assert h.value is None
    assert b"n_snakes" in lib.sim_last_error()
    bad = make_params(W.single_snake())
    bad[0].mass = 0.0
    assert lib.sim_create(ctypes.byref(cfg), 1, bad, None, ctypes.byref(h)) == N.SIM_EINVAL
    aniso = make_params(W.single_snake())
    aniso[0].mu_side = 1.0
    aniso[0].mu = 0.0  # anisotropic friction needs a positive coefficient along the body
    assert lib.sim_create(ctypes.byref(cfg), 1, aniso, None, ctypes.byref(h)) == N.SIM_EINVAL
    long = make_params(W.single_snake())
    long[0].n_links = 20  # 201 nodes > 128
    assert lib.sim_create(ctypes.byref(cfg), 1, long, None, ctypes.byref(h)) == N.SIM_EINVAL
    cfg2 = make_config(W.solver_settings(n_sub=0))
    assert lib.sim_create(ctypes.byref(cfg2), 1, prm, None, ctypes.byref(h)) == N.SIM_EINVAL
    for bad_law in (dict(latency=2), dict(latency=1, k_inflate=0.0), dict(latency=1, k_deflate=1.5),
                    dict(latency=1, t_p=0.0), dict(latency=1, p_source=-1.0), dict(latency=1, law_dt=-1.0)):
        cfg3 = make_config(W.solver_settings(**bad_law))
        assert lib.sim_create(ctypes.byref(cfg3), 1, prm, None, ctypes.byref(h)) == N.SIM_EINVAL, bad_law
    assert b"law" in lib.sim_last_error() or b"latency" in lib.sim_last_error()
    for bad_net in (dict(net_rows=3), dict(net_rows=-1), dict(net_every=-1), dict(beta_net=1.5),
                    dict(beta=1.2), dict(warm=3)):
        cfg4 = make_config(W.solver_settings(**bad_net))
        assert lib.sim_create(ctypes.byref(cfg4), 1, prm, None, ctypes.byref(h)) == N.SIM_EINVAL, bad_net
        assert h.value is None
    assert lib.sim_create(ctypes.byref(cfg), 1, prm, None, None) == N.SIM_EINVAL
    # calls on a null handle
    assert lib.sim_step(None, 1) == N.SIM_EINVAL
    assert lib.sim_set_config(None, ctypes.byref(cfg)) == N.SIM_EINVAL
    assert lib.sim_get_state(None, None, None, None, None, None, 0) == N.SIM_EINVAL
    assert lib.sim_autotune(None, 1) == N.SIM_EINVAL
    assert lib.sim_destroy(None) == N.SIM_OK


def test_product_path_has_no_oracle_dependency():
    """The package never imports or loads the oracle (it is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_1904_02833_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.lower(), os.path.join(dirpath, f)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the built library every entry point of the binding raises."""
    from paper_1904_02833_gb300 import _native
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "libsnakesim.so"))
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(ImportError, match="not built"):
        _native.load()
    import workloads as W
    from paper_1904_02833_gb300.fem import FemSim
    from paper_1904_02833_gb300.sim import SnakeSim
    with pytest.raises(ImportError):
        FemSim(W.fem_link_mesh(m=4, n_sec=2), W.fem_links(1), W.fem_settings(), device="cpu")
    with pytest.raises(ImportError):
        SnakeSim(W.single_snake(), W.solver_settings())
