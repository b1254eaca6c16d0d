"""CPU tests of the C-ABI library: it builds, loads, exports every function
that include/xg.h, xg_batch.h, xg_closure.h, xg_dynamics.h and xg_imex.h declare, and rejects invalid
arguments on the host before any GPU work (no compute calls here)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("xg.h", "xg_batch.h", "xg_closure.h",
                                                    "xg_dynamics.h", "xg_imex.h")]


@pytest.fixture(scope="module")
def lib():
    from paper_2504_08157_gb300 import build, xg
    build.build()
    return xg.library()


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(xg_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("xg_mesh_create", "xg_set_state", "xg_set_forcing", "xg_rhs", "xg_step",
                     "xg_destroy", "xg_batch_create", "xg_batch_step", "xg_batch_autotune",
                     "xg_batch_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_function(lib):
    """The Python binding gives every declared function its ctypes signature
    (restype and argtypes) and a wrapper of the same name."""
    from paper_2504_08157_gb300 import xg
    for name in declared_functions():
        f = getattr(lib, name)
        assert f.argtypes is not None, name
        assert hasattr(xg, name), name


def test_status_strings(lib):
    from paper_2504_08157_gb300 import xg
    for s in range(7):
        assert xg.xg_status_str(s).startswith("XG_")
    assert xg.xg_status_str(99) == "XG_UNKNOWN"


def _desc(**kw):
    from paper_2504_08157_gb300 import xg
    geo = dict(nel=(2, 2, 2), order=4, lo=(0, 0, 0), hi=(1e3, 1e3, 1e3), periodic=(0, 0, 0))
    extra = {k: v for k, v in kw.items() if k not in geo}
    geo.update({k: v for k, v in kw.items() if k in geo})
    return xg.mesh_desc(geo["nel"], geo["order"], geo["lo"], geo["hi"], geo["periodic"], **extra)


@pytest.mark.parametrize("bad", [
    dict(nel=(0, 2, 2)), dict(order=0), dict(order=9), dict(hi=(1e3, 0.0, 1e3)),
    dict(cp=-1.0), dict(cv=1004.5), dict(g=float("nan")),
])
def test_mesh_create_rejects_bad_arguments(lib, bad):
    from paper_2504_08157_gb300 import xg
    with pytest.raises(xg.XgError) as e:
        xg.xg_mesh_create(_desc(**bad))
    assert e.value.status == xg.XG_ERR_ARG


def test_unsupported_precision(lib):
    from paper_2504_08157_gb300 import xg
    with pytest.raises(xg.XgError) as e:
        xg.xg_mesh_create(_desc(precision=7))
    assert e.value.status == xg.XG_ERR_UNSUPPORTED


def test_null_arguments(lib):
    from paper_2504_08157_gb300 import xg
    P = ctypes.c_void_p
    assert lib.xg_mesh_create(None, None) == xg.XG_ERR_ARG
    out = P()
    assert lib.xg_mesh_create(None, ctypes.byref(out)) == xg.XG_ERR_ARG and not out.value
    assert lib.xg_set_state(None, None, None, None, 0, None) == xg.XG_ERR_ARG
    assert lib.xg_set_forcing(None, None, 0, None) == xg.XG_ERR_ARG
    assert lib.xg_rhs(None, None, 0, None) == xg.XG_ERR_ARG
    assert lib.xg_step(None, 0.1, 1, None) == xg.XG_ERR_ARG
    assert lib.xg_get_state(None, None, 0, None) == xg.XG_ERR_ARG
    n = ctypes.c_longlong()
    assert lib.xg_mesh_np(None, ctypes.byref(n)) == xg.XG_ERR_ARG
    assert lib.xg_set_fused(None, 1) == xg.XG_ERR_ARG
    assert lib.xg_step_stream(None, 0, None, None, 0.1, 1, None) == xg.XG_ERR_ARG
    assert lib.xg_set_contraction(None, 0) == xg.XG_ERR_ARG
    assert lib.xg_correction_set(None, None, None) == xg.XG_ERR_ARG
    lib.xg_destroy(None)  # no-op


def test_noalloc_rejects_an_output_that_overlaps_its_input(lib):
    """xg_rhs_noalloc compares the addresses of q, S_theta and dqdt on the host
    and rejects overlapping ranges before any device work (the addresses
    below are never dereferenced)."""
    from paper_2504_08157_gb300 import xg
    d = _desc()
    nx, ny, nz = [4 * d.nel[k] + (0 if d.periodic[k] else 1) for k in range(3)]
    vec = 8 * nx * ny * nz
    q, r0, t0 = 1 << 32, 1 << 33, (1 << 33) + 4096
    for out, S in ((q, None), (q + 8, None), (q - 4 * vec, None), (q + 5 * vec, q + 5 * vec)):
        assert lib.xg_rhs_noalloc(ctypes.byref(d), q, r0, t0, S, out, None) == xg.XG_ERR_ARG
    assert lib.xg_rhs_noalloc(ctypes.byref(d), q, None, t0, None, q + 5 * vec, None) == xg.XG_ERR_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2504_08157_gb300 import xg
    monkeypatch.setattr(xg, "_lib", None)
    monkeypatch.setattr(xg, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError):
        xg.library()


# ------------------------------------------------------------------ batched form (host checks)

@pytest.mark.parametrize("kw,status", [
    (dict(precision=0), "XG_ERR_UNSUPPORTED"),     # FP64 instances are not batched
    (dict(precision=2), "XG_ERR_UNSUPPORTED"),
    (dict(precision=1, order=2), "XG_ERR_UNSUPPORTED"),
    (dict(precision=1, order=7), "XG_ERR_UNSUPPORTED"),
    (dict(precision=1, order=9), "XG_ERR_ARG"),
])
def test_batch_create_rejects_on_the_host(lib, kw, status):
    from paper_2504_08157_gb300 import xg
    descs = [_desc(precision=1), _desc(**kw)]
    with pytest.raises(xg.XgError) as e:
        xg.xg_batch_create(descs)
    assert e.value.status == getattr(xg, status)


def test_batch_null_arguments(lib):
    from paper_2504_08157_gb300 import xg
    P = ctypes.c_void_p
    out = P()
    assert lib.xg_batch_create(None, 1, ctypes.byref(out)) == xg.XG_ERR_ARG and not out.value
    d = (xg.xg_mesh_desc * 1)(_desc(precision=1))
    assert lib.xg_batch_create(d, 0, ctypes.byref(out)) == xg.XG_ERR_ARG
    assert lib.xg_batch_create(d, 5000, ctypes.byref(out)) == xg.XG_ERR_ARG
    assert lib.xg_batch_create(d, 1, None) == xg.XG_ERR_ARG
    assert lib.xg_batch_instance(None, 0) is None
    assert lib.xg_batch_step(None, None, 1, None) == xg.XG_ERR_ARG
    assert lib.xg_batch_rhs(None, None, 0, None) == xg.XG_ERR_ARG
    assert lib.xg_batch_autotune(None, None, 1, None, None) == xg.XG_ERR_ARG
    assert lib.xg_batch_set_tuning(None, None) == xg.XG_ERR_ARG
    assert lib.xg_batch_get_tuning(None, None) == xg.XG_ERR_ARG
    assert lib.xg_batch_barrier_selftest(None, 10, None) == xg.XG_ERR_ARG
    n = ctypes.c_int()
    assert lib.xg_batch_count(None, ctypes.byref(n)) == xg.XG_ERR_ARG
    lib.xg_batch_destroy(None)
