"""C-ABI checks that need no GPU: the library builds and loads, it exports
every function include/gkba.h declares, and invalid arguments are rejected
by host-side validation before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import gkba_inputs as gi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_01180_gb300 import build as b
    b.build()
    from paper_1905_01180_gb300 import gkba
    return gkba.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gkba.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gkba_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "gkba_init" in names and "gkba_collision" in names and "gkba_step" in names
    for n in names:
        assert hasattr(lib, n), n
    from paper_1905_01180_gb300 import gkba
    assert sorted(gkba.EXPORTED) == names


def test_config_struct_matches_header():
    # the binding's ctypes struct lists gkba_config's members in the header's order
    from paper_1905_01180_gb300 import gkba
    src = open(os.path.join(ROOT, "include", "gkba.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} gkba_config;", src, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    members = re.findall(r"\b([A-Za-z_0-9]+)\s*;", body)
    assert members == [f[0] for f in gkba.Config._fields_]


def _init(lib, N=4, dt=0.05, prec=0, h=None, v=None, d=None, rho=None, interaction=0,
          history=0):
    from paper_1905_01180_gb300 import gkba
    s = gi.system(4, 4, seed=0)
    h = s["h"] if h is None else h
    v = s["v"] if v is None else v
    d = s["d"] if d is None else d
    rho = s["rho0"] if rho is None else rho
    cfg = gkba.Config(N=N, dt=dt, max_steps=1, precision=prec, cuda_stream=None,
                      workspace_bytes=0, device=-1, timing=0, acc_window=0,
                      interaction=interaction, history=history)
    out = ctypes.c_void_p()
    arrs = [np.ascontiguousarray(x) for x in (h, v, d, rho)]
    st = lib.gkba_init(ctypes.byref(out), ctypes.byref(cfg), *[a.ctypes.data for a in arrs], 0)
    return st, out, lib.gkba_last_error(None).decode()


def test_init_rejects_bad_sizes_and_inputs(lib):
    from paper_1905_01180_gb300 import gkba
    st, out, msg = _init(lib, N=0)
    assert st == gkba.EINVAL and out.value is None and "N=0" in msg
    st, _, _ = _init(lib, N=129)
    assert st == gkba.EINVAL
    st, _, msg = _init(lib, dt=-1.0)
    assert st == gkba.EINVAL and "dt" in msg
    st, _, _ = _init(lib, prec=7)
    assert st == gkba.EINVAL
    s = gi.system(4, 4, seed=0)
    h = s["h"].copy()
    h[0, 1] += 0.3
    st, _, msg = _init(lib, h=h)
    assert st == gkba.EINVAL and "Hermitian" in msg
    v = s["v"].copy()
    v[0, 1, 2, 3] += 1.0
    st, _, msg = _init(lib, v=v)
    assert st == gkba.EINVAL and "symmetry" in msg
    rho = s["rho0"].copy()
    rho[1, 1] = np.nan
    st, _, msg = _init(lib, rho=rho)
    assert st == gkba.EINVAL and "non-finite" in msg


def test_init_rejects_bad_structured_interactions(lib):
    # Sec. III A/B interactions: an unknown kind, a split-TF32 precision (these
    # paths run in FP64) and a non-symmetric V are refused before device work
    from paper_1905_01180_gb300 import gkba
    c = gi.chain(4, "symmetric")
    st, _, msg = _init(lib, interaction=3, v=c["v"])
    assert st == gkba.EINVAL and "interaction" in msg
    st, _, msg = _init(lib, interaction=gkba.V_SYMMETRIC, prec=gkba.SPLIT_TF32, v=c["v"])
    assert st == gkba.EINVAL and "FP64" in msg
    V = c["v"].copy()
    V[0, 2] += 0.1
    st, _, msg = _init(lib, interaction=gkba.V_SYMMETRIC, v=V)
    assert st == gkba.EINVAL and "not symmetric" in msg
    U = np.array([1.0, np.inf, 1.0, 1.0])
    st, _, msg = _init(lib, interaction=gkba.V_DIAGONAL, v=U)
    assert st == gkba.EINVAL and "non-finite" in msg


def test_init_rejects_bad_history_modes(lib):
    # the time-linear history needs a general v; a structured interaction and
    # unknown modes are refused before device work
    from paper_1905_01180_gb300 import gkba
    st, _, msg = _init(lib, history=2)
    assert st == gkba.EINVAL and "history" in msg
    c = gi.chain(4, "symmetric")
    st, _, msg = _init(lib, history=gkba.HISTORY_TIME_LINEAR, interaction=gkba.V_SYMMETRIC,
                       v=c["v"])
    assert st == gkba.EUNSUPPORTED and "time-linear" in msg


def test_batch_create_rejects_bad_arguments(lib):
    # host-side validation of gkba_batch_create, before any device work
    from paper_1905_01180_gb300 import gkba
    out = ctypes.c_void_p()
    assert lib.gkba_batch_create(ctypes.byref(out), None, 0, 0) == gkba.EINVAL
    arr = (ctypes.c_void_p * 2)(None, None)
    st = lib.gkba_batch_create(ctypes.byref(out), ctypes.cast(arr, ctypes.c_void_p), 2, 0)
    assert st == gkba.EINVAL and out.value is None
    assert b"NULL" in lib.gkba_batch_last_error(None)
    assert lib.gkba_batch_step(None, None, None, None, None) == gkba.EINVAL
    assert lib.gkba_batch_set_options(None, 1) == gkba.EINVAL
    assert lib.gkba_batch_autotune(None, None, None, None, None, None, None) == gkba.EINVAL
    lib.gkba_batch_destroy(None)
    assert lib.gkba_selftest_timeout(None, 10.0, None) == gkba.EINVAL
    # gradients and the trilinear form: NULL context or arrays are refused on the host
    assert lib.gkba_sigma3(None, 1, None, None, None, None, 0) == gkba.EINVAL
    assert lib.gkba_collision_vjp(None, 1, None, None, None, None, None, None, None, 0) == gkba.EINVAL
    assert lib.gkba_adjoint(None, None, None, None, None) == gkba.EINVAL


def test_null_context_calls_fail_cleanly(lib):
    from paper_1905_01180_gb300 import gkba
    assert lib.gkba_collision(None, 1, None, None, None, None, 0) == gkba.EINVAL
    assert lib.gkba_step(None, 0.0, 0.0, None, None, None) == gkba.EINVAL
    assert lib.gkba_sigma(None, 1, None, None, None, 0) == gkba.EINVAL
    lib.gkba_destroy(None)


def test_product_path_does_not_import_oracle():
    import subprocess
    import sys
    code = ("import sys; import paper_1905_01180_gb300 as p; p.load(); "
            "assert 'oracle' not in sys.modules, 'oracle imported'")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
