"""The allocation-free step, lbm_step_noalloc.

Some callers own all device memory themselves and may not call cudaMalloc
while stepping (for example an application whose memory-pool policy forbids
allocation, or a real-time loop that must not take the allocator's locks).
For them the library offers lbm_step_noalloc: one step from a caller buffer
to another, with the density scratch held in a static device array inside the
library instead of an allocation.  These tests check that it computes what
the ordinary handle-based lbm_step computes, on two calls in a row (the second
call reuses the static scratch the first call left behind), and that it
refuses lattices larger than its fixed scratch.

This file is collected last on purpose: a run that stops at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1601_01237_gb300 import workloads as wl
from _helpers import G_STRONG


def test_noalloc_rejects_oversized_lattice():
    """Sizes beyond LBM_NOALLOC_MAX_CELLS fail with LBM_EINVAL before any
    device work (runs without a GPU too)."""
    from paper_1601_01237_gb300 import NOALLOC_MAX_CELLS, build, make_params, _native
    build.build()
    L = _native.lib()
    p = make_params((129, 128, 128), storage="f32")
    assert 129 * 128 * 128 > NOALLOC_MAX_CELLS
    buf_a = ctypes.c_void_p(256)   # never dereferenced: the size check comes first
    buf_b = ctypes.c_void_p(512)
    st = L.lbm_step_noalloc(ctypes.byref(p), buf_a, buf_b)
    assert st == _native.LBM_EINVAL
    assert "LBM_NOALLOC_MAX_CELLS" in L.lbm_last_error(None).decode()
    hdr = open(__file__.rsplit("/tests/", 1)[0] + "/include/lbm.h").read()
    assert "#define LBM_NOALLOC_MAX_CELLS %dL" % NOALLOC_MAX_CELLS in hdr


@pytest.mark.gpu
@pytest.mark.parametrize("storage,kw,tol", [
    ("f32", dict(tau=(0.8, 1.1), G12=G_STRONG), 1e-6),
    ("f64", dict(tau=(0.7, 0.9), G12=-1.3, periodic=(1, 1, 0), collision="regularized",
                 g_ext=(1e-5, 0.0, -2e-5)), 1e-13),
])
def test_noalloc_step_matches_lbm_step(gpu_lib, storage, kw, tol):
    """Two consecutive lbm_step_noalloc calls (A -> B -> C) against two steps of
    the handle-based lbm_step, compared on the raw state within the
    tolerance the other parity tests use for this storage."""
    import torch
    from paper_1601_01237_gb300 import Lattice, lbm_step_noalloc
    shape = (20, 24, 28)
    r1, r2 = wl.droplet(shape, 6)
    lat = Lattice(shape, storage=storage, **kw)
    lat.init_fields(r1, r2)
    nbytes = lat.state_bytes()
    dt = torch.float32 if storage == "f32" else torch.float64
    elems = nbytes // (4 if storage == "f32" else 8)
    A = torch.empty(elems, dtype=dt, device="cuda")
    B = torch.full((elems,), float("nan"), dtype=dt, device="cuda")
    C = torch.full((elems,), float("nan"), dtype=dt, device="cuda")
    lat.get_state(A)
    torch.cuda.synchronize()
    params = lat.params          # same lbm_params, stream = torch's current stream
    lbm_step_noalloc(params, A, B)
    lbm_step_noalloc(params, B, C)
    ref = []
    for _ in range(2):
        lat.step(1)
        R = torch.empty(elems, dtype=dt, device="cuda")
        lat.get_state(R)
        ref.append(R)
    torch.cuda.synchronize()
    lat.close()
    for got, want in ((B, ref[0]), (C, ref[1])):
        g = got.cpu().numpy()
        w = want.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.max(np.abs(g - w)) <= tol * np.max(np.abs(w))
