"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every entry point declared in include/lbm.h; argument validation
returns the documented status codes before any device work; the product path
has no oracle or CPU fallback."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1601_01237_gb300 import build, _native
    build.build()
    return _native.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = header_functions()
    assert "lbm_step" in names and "lbm_create" in names and len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    from paper_1601_01237_gb300._native import SIGNATURES
    assert sorted(n for n, _, _ in SIGNATURES) == names


def test_lattice_dirs(L):
    from paper_1601_01237_gb300 import lbm_lattice_dirs
    c, w = lbm_lattice_dirs()
    assert len({tuple(v) for v in c}) == 19
    assert abs(w.sum() - 1) < 1e-15
    for i in range(1, 19):   # opposite pairs side by side
        j = i + 1 if i % 2 else i - 1
        assert (c[j] == -c[i]).all()


def _status(L, **kw):
    from paper_1601_01237_gb300 import make_params
    p = make_params(**kw)
    h = ctypes.c_void_p()
    st = L.lbm_create(ctypes.byref(p), ctypes.byref(h))
    assert not h.value
    return st, L.lbm_last_error(None).decode()


@pytest.mark.parametrize("kw,code", [
    (dict(shape=(0, 4, 4)), 1),
    (dict(shape=(4, 4, 4), tau=(0.5, 1.0)), 1),
    (dict(shape=(4, 4, 4), tau=(1.0, float("nan"))), 1),
    (dict(shape=(4, 4, 4), storage="f64", rho0_dev=0.5), 1),
    (dict(shape=(4, 4, 4), G12=float("inf")), 1),
    (dict(shape=(4, 4, 4), periodic=(0, 1, 1)), 4),
    (dict(shape=(4, 4, 4), periodic=(1, 0, 1)), 4),
    (dict(shape=(4, 4, 4), storage="f16_rel", rho0_dev=0.5), 1),
    (dict(shape=(4, 4, 4), forcing="guo", storage="f32", rho0_dev=0.1), 1),
])
def test_validation_codes(L, kw, code):
    st, msg = _status(L, **kw)
    assert st == code, msg
    assert msg.startswith("lbm_create")


def test_self_interaction_not_supported(L):
    from paper_1601_01237_gb300 import make_params
    p = make_params((4, 4, 4))
    p.G[0][0] = -1.0
    h = ctypes.c_void_p()
    assert L.lbm_create(ctypes.byref(p), ctypes.byref(h)) == 4


def test_null_arguments(L):
    assert L.lbm_create(None, None) == 1
    assert L.lbm_step(None, 1) == 1
    assert L.lbm_reduce(None, None) == 1
    L.lbm_destroy(None)   # NULL-safe


def test_missing_library_fails_loudly(monkeypatch):
    from paper_1601_01237_gb300 import _native
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native, "LIB_PATH", "/nonexistent/libmclbm.so")
    with pytest.raises(RuntimeError, match="not built"):
        _native.lib()


def test_product_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1601_01237_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", src, flags=re.M), f
                assert "lbm_oracle" not in src, f


def test_unknown_forcing_and_storage_rejected(L):
    from paper_1601_01237_gb300 import make_params
    for field, val in (("forcing", 2), ("storage", 6)):
        p = make_params((4, 4, 4))
        setattr(p, field, val)
        h = ctypes.c_void_p()
        assert L.lbm_create(ctypes.byref(p), ctypes.byref(h)) == 1
        assert field in L.lbm_last_error(None).decode()


def test_noalloc_rejects_overlapping_states(L):
    """The allocation-free step refuses f_out overlapping f_in (any part of
    the state, not only the same address) before it touches either buffer:
    the pointers here are never dereferenced."""
    from paper_1601_01237_gb300 import make_params
    for storage, shift in (("f32", 8), ("f32", 16 * 16 * 16 * 152 - 4), ("bf16_rel", 16 * 16 * 16 * 84 - 8)):
        p = make_params((16, 16, 16), storage=storage)
        base = 1 << 40
        st = L.lbm_step_noalloc(ctypes.byref(p), ctypes.c_void_p(base), ctypes.c_void_p(base + shift))
        assert st == 1
        assert "overlap" in L.lbm_last_error(None).decode()
