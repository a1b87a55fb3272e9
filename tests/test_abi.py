"""The C-ABI library builds, loads and exports every entry point include/mstar.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2001_03180_gb300 import build as B
from paper_2001_03180_gb300 import mstar as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mstar.h")).read()
    return sorted(set(re.findall(r"MSTAR_API\s+[\w\s\*]+?\b(mstar_\w+)\s*\(", src)))


def test_header_declares_the_binding_names():
    assert declared_functions() == sorted(M.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_only_entry_points_without_gpu():
    B.build()
    p = M.mstar_default_params()
    assert p.k_fix == 8 and p.n_d == 2 and p.eta_gbs == 1e-12 and p.a_gbs == 0.9
    assert M.mstar_strerror(M.MSTAR_ERR_NO_CONVERGENCE).startswith("GBS step")
    assert M.mstar_workspace_bytes(10002, p) > 0
    assert M.mstar_workspace_bytes(1, p) == 0
    assert M.mstar_workspace_bytes(M.MSTAR_MAX_N + 1, p) == 0
    bad = M.mstar_default_params(k_fix=1)
    assert M.mstar_workspace_bytes(100, bad) == 0
    bad = M.mstar_default_params(n_d=3)
    assert M.mstar_workspace_bytes(100, bad) == 0
    with pytest.raises(TypeError):
        M.mstar_default_params(eta=1e-10)       # the field is eta_gbs; a typo must not be ignored


def test_batch_layout_rules_without_gpu():
    """The host checks of a batch's CSR offsets (a system has 2 .. MSTAR_BATCH_MAX_N bodies, at
    least one system, offsets from 0): a batch the library would reject has no workspace."""
    B.build()
    p = M.mstar_default_params()
    ok = M.mstar_batch_workspace_bytes(3, [0, 2, 5, 5 + M.MSTAR_BATCH_MAX_N], p)
    assert ok > 0
    assert M.mstar_batch_workspace_bytes(4, [0, 2, 5, 7, 107], p) > M.mstar_batch_workspace_bytes(3, [0, 2, 5, 7], p)
    for nsys, off in [(0, [0]),                                   # empty batch
                      (2, [0, 1, 4]),                             # a one-body system
                      (2, [0, 3, 3]),                             # an empty system
                      (2, [1, 3, 6]),                             # offsets not from 0
                      (2, [0, 4, 2]),                             # decreasing offsets
                      (1, [0, M.MSTAR_BATCH_MAX_N + 1])]:         # above the batch limit
        assert M.mstar_batch_workspace_bytes(nsys, off, p) == 0, (nsys, off)
    bad = M.mstar_default_params(k_fix=1)
    assert M.mstar_batch_workspace_bytes(1, [0, 3], bad) == 0
    with pytest.raises(M.MstarError) as e:
        M.Batch([])
    assert e.value.code == M.MSTAR_ERR_INVALID_ARG


def test_binding_checks_array_shapes_before_any_device_work():
    """The library reads n masses and 3n coordinates through each pointer: the binding refuses
    arrays of any other shape instead of letting the copy read past them."""
    m, r, v = np.ones(5), np.zeros((5, 3)), np.zeros((5, 3))
    for bad in [(m, r[:4], v), (m, r, v[:, :2]), (m.reshape(5, 1), r, v), (m, r.T, v), (m, r, np.zeros(14))]:
        with pytest.raises(ValueError):
            M.Integrator(*bad)
        with pytest.raises(ValueError):
            M.Batch([(m, r, v), bad])
    mm, rr, vv = M._system(m, r.ravel(), v)          # flat 3n coordinates in body order are accepted
    assert rr.shape == (5, 3) and vv.shape == (5, 3) and mm.shape == (5,)


def test_no_cpu_fallback_in_product_path():
    """The package never imports the oracle: product sources mention no oracle module."""
    pkg = os.path.join(ROOT, "paper_2001_03180_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "mstar_oracle" not in text, f


def test_missing_library_fails_loudly(monkeypatch):
    """Without the built library every entry point raises: there is no fallback path."""
    monkeypatch.setattr(M, "_lib", None)
    monkeypatch.setattr(M, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libmstar.so"))
    with pytest.raises(ImportError):
        M.load()
    with pytest.raises(ImportError):
        M.mstar_default_params()


def test_no_gpu_means_no_integrator():
    """On a machine without a CUDA GPU the integrator refuses to start instead of running
    anything on the host."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m = [1.0, 1.0]
    r = [[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]]
    v = [[0.0, 0.0, 0.0], [0.0, 1.0, 0.0]]
    for make in (lambda: M.Integrator(m, r, v), lambda: M.Batch([(m, r, v)])):
        with pytest.raises(RuntimeError):
            make()


def test_c_entry_points_without_gpu_return_errors():
    """Called directly without a GPU, mstar_init and mstar_batch_init return an error code and
    no context: nothing is computed on the host."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes as C

    B.build()
    L = M.load()
    m = np.ones(4)
    r = np.random.default_rng(0).random((4, 3))
    v = np.zeros((4, 3))
    p = M.mstar_default_params()
    ctx = C.c_void_p()
    rc = L.mstar_init(C.byref(ctx), 4, m.ctypes.data, r.ctypes.data, v.ctypes.data, C.byref(p), None, 0, None)
    assert rc in (M.MSTAR_ERR_CUDA, M.MSTAR_ERR_NOMEM) and not ctx.value
    offs = np.array([0, 4], np.int32)
    b = C.c_void_p()
    rc = L.mstar_batch_init(C.byref(b), 1, offs.ctypes.data, m.ctypes.data, r.ctypes.data, v.ctypes.data,
                            C.byref(p), None, 0, None)
    assert rc in (M.MSTAR_ERR_CUDA, M.MSTAR_ERR_NOMEM) and not b.value
