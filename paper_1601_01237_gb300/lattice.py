"""Python binding of the C ABI in include/lbm.h.

Argument marshalling only: every step of the update runs in the CUDA library
(libmclbm.so).  The module-level functions carry the C names one to one; the
``Lattice`` class wraps a handle for convenience.  Host arrays are numpy
arrays; device arrays are torch CUDA tensors (torch provides device memory and
streams, nothing else).
"""
import ctypes

import numpy as np

from . import _native as nat
from ._native import check, lib

Q = 19
CUDA_STREAM_LEGACY = 0x1   # cudaStreamLegacy


def _ptr(x):
    """(address, on_device) of a numpy array or a torch tensor."""
    if x is None:
        return None, 0
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
        return x.ctypes.data, 0
    # torch tensor
    assert x.is_contiguous(), "tensors must be contiguous"
    return x.data_ptr(), 1 if x.is_cuda else 0


# --------------------------------------------------------------------------
# C-named functions

def lbm_lattice_dirs():
    c = (ctypes.c_int * (Q * 3))()
    w = (ctypes.c_double * Q)()
    check(lib().lbm_lattice_dirs(c, w))
    return np.array(c, dtype=np.int64).reshape(Q, 3), np.array(w)


def lbm_create(params):
    h = ctypes.c_void_p()
    check(lib().lbm_create(ctypes.byref(params), ctypes.byref(h)))
    return h


def lbm_init_fields(h, rho1, rho2, u=None):
    p1, d1 = _ptr(rho1)
    p2, d2 = _ptr(rho2)
    pu, du = _ptr(u)
    on_dev = d1
    assert d2 == on_dev and (u is None or du == on_dev), "mixed host/device inputs"
    check(lib().lbm_init_fields(h, p1, p2, pu, on_dev), h)


def lbm_step(h, n_steps):
    check(lib().lbm_step(h, int(n_steps)), h)


def lbm_step_timed(h, n_steps):
    """Advance n_steps with per-kernel CUDA events; returns
    {kernel name: (total ms, launches)}."""
    ms = (ctypes.c_double * 4)()
    nl = (ctypes.c_long * 4)()
    names = (ctypes.c_char_p * 4)()
    nk = ctypes.c_int()
    check(lib().lbm_step_timed(h, int(n_steps), ms, nl, names, ctypes.byref(nk)), h)
    return {names[k].decode(): (ms[k], nl[k]) for k in range(nk.value)}


def lbm_moments(h, rho1=None, rho2=None, uF=None, out_f64=True):
    ptrs = [_ptr(x) for x in (rho1, rho2, uF)]
    devs = {d for (p, d), x in zip(ptrs, (rho1, rho2, uF)) if x is not None}
    assert len(devs) <= 1, "mixed host/device outputs"
    on_dev = devs.pop() if devs else 0
    check(lib().lbm_moments(h, int(bool(out_f64)), ptrs[0][0], ptrs[1][0], ptrs[2][0], on_dev), h)


def lbm_reduce(h):
    out = (ctypes.c_double * 6)()
    check(lib().lbm_reduce(h, out), h)
    return list(out)


def lbm_pressure_jump(h, center, r_in, r_out):
    """(p_in, p_out, dp) with p = T0 rho - G12 T0 rho1 rho2; center = (x, y, z)."""
    c = (ctypes.c_double * 3)(*[float(v) for v in center])
    out = (ctypes.c_double * 3)()
    check(lib().lbm_pressure_jump(h, c, float(r_in), float(r_out), out), h)
    return tuple(out)


def lbm_droplet_stats(h, threshold, origin=(0.0, 0.0, 0.0)):
    o = (ctypes.c_double * 3)(*[float(v) for v in origin])
    out = (ctypes.c_double * 7)()
    check(lib().lbm_droplet_stats(h, float(threshold), o, out), h)
    return {"volume": out[0], "com": (out[1], out[2], out[3]), "mass": out[4], "film_rho": out[5],
            "film_cells": out[6]}


def lbm_set_solid(h, solid):
    """solid: N = nx ny nz flags (numpy array on the host, or a contiguous
    torch uint8/bool tensor), non-zero = solid site; None removes the mask.
    The library copies N bytes: the caller guarantees the size
    (Lattice.set_solid checks it)."""
    if solid is None:
        check(lib().lbm_set_solid(h, None, 0), h)
        return
    if isinstance(solid, np.ndarray):
        solid = np.ascontiguousarray(solid != 0, dtype=np.uint8)
    p, d = _ptr(solid)
    check(lib().lbm_set_solid(h, p, d), h)


def lbm_get_populations(h, out):
    p, d = _ptr(out)
    check(lib().lbm_get_populations(h, p, d), h)


def lbm_set_populations(h, src):
    p, d = _ptr(src)
    check(lib().lbm_set_populations(h, p, d), h)


def lbm_state_bytes(h):
    n = ctypes.c_size_t()
    check(lib().lbm_state_bytes(h, ctypes.byref(n)), h)
    return n.value


def lbm_get_state(h, dev_buf):
    p, d = _ptr(dev_buf)
    assert d == 1, "state buffers live on the device"
    check(lib().lbm_get_state(h, p, dev_buf.numel() * dev_buf.element_size()), h)


def lbm_set_state(h, dev_buf):
    p, d = _ptr(dev_buf)
    assert d == 1, "state buffers live on the device"
    check(lib().lbm_set_state(h, p, dev_buf.numel() * dev_buf.element_size()), h)


def lbm_step_count(h):
    n = ctypes.c_long()
    check(lib().lbm_step_count(h, ctypes.byref(n)), h)
    return n.value


def lbm_sync(h):
    check(lib().lbm_sync(h), h)


def lbm_record(h, n_steps, ckpt_every):
    check(lib().lbm_record(h, int(n_steps), int(ckpt_every)), h)


def lbm_adjoint(h, dL_drho1=None, dL_drho2=None, out_rho1_0=None, out_rho2_0=None):
    """Reverse pass over the last lbm_record.  Inputs and outputs are all host
    (numpy float64) or all device (torch float64) arrays; returns
    [dL/dG12, dL/dG21, dL/dtau1, dL/dtau2]."""
    arrs = [x for x in (dL_drho1, dL_drho2, out_rho1_0, out_rho2_0) if x is not None]
    devs = {_ptr(x)[1] for x in arrs}
    assert len(devs) <= 1, "mixed host/device arrays"
    on_dev = devs.pop() if devs else 0
    par = (ctypes.c_double * 4)()
    check(lib().lbm_adjoint(h, _ptr(dL_drho1)[0], _ptr(dL_drho2)[0], on_dev, _ptr(out_rho1_0)[0],
                            _ptr(out_rho2_0)[0], par), h)
    return list(par)


NOALLOC_MAX_CELLS = 2097152   # LBM_NOALLOC_MAX_CELLS of include/lbm.h


def lbm_step_noalloc(params, f_in, f_out):
    """One step from f_in to f_out (raw-state device buffers owned by the
    caller) without any device allocation; see include/lbm.h."""
    pi, di = _ptr(f_in)
    po, do = _ptr(f_out)
    assert di == 1 and do == 1, "state buffers live on the device"
    check(lib().lbm_step_noalloc(ctypes.byref(params), pi, po))


def lbm_destroy(h):
    lib().lbm_destroy(h)


# --------------------------------------------------------------------------

def make_params(shape, tau=(1.0, 1.0), G12=0.0, G21=None, g_ext=(0.0, 0.0, 0.0), periodic=(1, 1, 1),
                rho_s=(0.0, 0.0), rho0_dev=0.0, storage="f32", collision="bgk", wall_model="mirror",
                stream=None, forcing="edm"):
    """lbm_params for a lattice of shape (nz, ny, nx).  G12, G21 are the signed
    G^{12}, G^{21} of Eq. 7 (G21 defaults to G12).  forcing: "edm" (exact
    difference of equilibria) or "guo" (Guo, Zheng & Shi 2002)."""
    nz, ny, nx = shape
    p = nat.lbm_params()
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    for d in range(3):
        p.periodic[d] = int(periodic[d])
        p.g_ext[d] = float(g_ext[d])
    p.tau[0], p.tau[1] = float(tau[0]), float(tau[1])
    p.G[0][0] = 0.0
    p.G[1][1] = 0.0
    p.G[0][1] = float(G12)
    p.G[1][0] = float(G12 if G21 is None else G21)
    p.rho_s[0], p.rho_s[1] = float(rho_s[0]), float(rho_s[1])
    p.rho0_dev = float(rho0_dev)
    p.storage = nat.STORAGE[storage]
    p.collision = nat.COLLISION[collision]
    p.wall_model = nat.WALL_MODEL[wall_model]
    p.forcing = nat.FORCING[forcing]
    # A handle of 0 is the legacy default stream (torch's default stream);
    # the C ABI reserves NULL for "library-owned stream", so pass the
    # runtime's explicit legacy-stream handle instead.
    p.stream = CUDA_STREAM_LEGACY if stream == 0 else stream
    return p


class Lattice:
    """A two-component D3Q19 lattice living on the current CUDA device."""

    def __init__(self, shape, **kw):
        if kw.get("stream", None) is None and kw.pop("torch_stream", True):
            import torch
            kw["stream"] = torch.cuda.current_stream().cuda_stream
        self.shape = tuple(int(s) for s in shape)
        self.N = int(np.prod(self.shape))
        self.params = make_params(self.shape, **kw)
        self.storage = kw.get("storage", "f32")
        self.h = lbm_create(self.params)

    def close(self):
        if self.h is not None:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init_fields(self, rho1, rho2, u=None):
        if isinstance(rho1, np.ndarray):
            rho1 = np.ascontiguousarray(rho1, dtype=np.float64)
            rho2 = np.ascontiguousarray(rho2, dtype=np.float64)
            u = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        lbm_init_fields(self.h, rho1, rho2, u)

    def step(self, n=1):
        lbm_step(self.h, n)

    def record(self, n, ckpt_every):
        lbm_record(self.h, n, ckpt_every)

    def adjoint(self, dL_drho1=None, dL_drho2=None, out_rho1_0=None, out_rho2_0=None):
        return lbm_adjoint(self.h, dL_drho1, dL_drho2, out_rho1_0, out_rho2_0)

    def step_timed(self, n):
        return lbm_step_timed(self.h, n)

    def moments(self, out_f64=True):
        """Host copies (rho1, rho2, uF) shaped (nz,ny,nx), (nz,ny,nx), (nz,ny,nx,3)."""
        dt = np.float64 if out_f64 else np.float32
        r1 = np.empty(self.shape, dt)
        r2 = np.empty(self.shape, dt)
        uF = np.empty(self.shape + (3,), dt)
        lbm_moments(self.h, r1, r2, uF, out_f64)
        return r1, r2, uF

    def moments_device(self, rho1=None, rho2=None, uF=None, out_f64=False):
        lbm_moments(self.h, rho1, rho2, uF, out_f64)

    def reduce(self):
        v = lbm_reduce(self.h)
        return {"mass1": v[0], "mass2": v[1], "momentum": v[2:5], "max_uF": v[5]}

    def pressure_jump(self, center, r_in, r_out):
        return lbm_pressure_jump(self.h, center, r_in, r_out)

    def droplet_stats(self, threshold, origin=(0.0, 0.0, 0.0)):
        return lbm_droplet_stats(self.h, threshold, origin)

    def set_solid(self, solid):
        """Staircase walls: solid (nz, ny, nx) flags, non-zero = solid site (a
        numpy array, or a torch uint8/bool tensor of that shape); None removes
        the mask."""
        if solid is not None:
            if isinstance(solid, np.ndarray):
                if solid.shape != self.shape:
                    raise ValueError("mask shape %s != lattice shape %s" % (solid.shape, self.shape))
            else:
                import torch
                if tuple(solid.shape) != self.shape or solid.dtype not in (torch.uint8, torch.bool):
                    raise ValueError("mask must be a uint8 or bool tensor of shape %s" % (self.shape,))
        lbm_set_solid(self.h, solid)

    def get_populations(self):
        """Host copy of f_i^a(x, t), shape (2, 19, nz, ny, nx), library direction order."""
        out = np.empty((2, Q) + self.shape)
        lbm_get_populations(self.h, out)
        return out

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64) if isinstance(f, np.ndarray) else f
        lbm_set_populations(self.h, f)

    def state_bytes(self):
        return lbm_state_bytes(self.h)

    def get_state(self, buf):
        lbm_get_state(self.h, buf)

    def set_state(self, buf):
        lbm_set_state(self.h, buf)

    def step_count(self):
        return lbm_step_count(self.h)

    def sync(self):
        lbm_sync(self.h)
