"""FP64 CPU oracle of the two-component D3Q19 Shan-Chen LBM step.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.  It shares no code with the
CUDA path.  The arithmetic lives in ``lbm_oracle.c`` (plain loops in the order
of Sec. 2 of Otomo et al., arXiv:1601.01237); this module only marshals numpy
arrays into it.

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py`` (closed forms, invariants, brute force).
"""
import ctypes
import numpy as np

from .build import build as _build

Q = 19


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("tau", ctypes.c_double * 2),
        ("G", (ctypes.c_double * 2) * 2),
        ("g_ext", ctypes.c_double * 3),
        ("rho_s", ctypes.c_double * 2),
        ("collision", ctypes.c_int),
        ("wall_model", ctypes.c_int),
        ("solid", ctypes.c_void_p),
        ("forcing", ctypes.c_int),
    ]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(OracleParams)
        _lib.oracle_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), dp]
        _lib.oracle_feq.argtypes = [ctypes.c_double, dp, dp]
        _lib.oracle_init.argtypes = [pp, dp, dp, dp, dp]
        _lib.oracle_step.argtypes = [pp, dp, dp, ctypes.c_long]
        _lib.oracle_moments.argtypes = [pp, dp, dp, dp, dp]
        _lib.oracle_moments_raw.argtypes = [pp, dp, dp, dp, dp]
        _lib.oracle_interaction_sums.argtypes = [pp, dp, ctypes.c_double, dp, dp]
        _lib.oracle_accelerations.argtypes = [pp, dp, dp, dp, dp]
        _lib.oracle_collide_cell.argtypes = [pp, ctypes.c_int, dp, ctypes.c_double, dp, dp, dp]
        _lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib.oracle_set_threads.restype = ctypes.c_int
    return _lib


def set_threads(n):
    """Threads of the oracle's cell loops (1 = serial); returns the count in
    use (1 without OpenMP).  The results do not depend on it."""
    return int(_L().oracle_set_threads(int(n)))


def _dp(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(shape, tau=(1.0, 1.0), G12=0.0, G21=None, g_ext=(0.0, 0.0, 0.0),
                periodic=(1, 1, 1), rho_s=(0.0, 0.0), collision="bgk", wall_model="mirror", solid=None,
                forcing="edm"):
    """shape = (nz, ny, nx).  G12/G21 are the signed G^{12}, G^{21} of Eq. 7.
    solid: optional (nz, ny, nx) array, non-zero at solid sites.  forcing:
    "edm" (exact difference of equilibria) or "guo" (Guo, Zheng & Shi 2002
    with the common equilibrium velocity u + g/2)."""
    nz, ny, nx = shape
    p = OracleParams()
    p.nx, p.ny, p.nz = nx, ny, nz
    for d in range(3):
        p.periodic[d] = int(periodic[d])
        p.g_ext[d] = float(g_ext[d])
    p.tau[0], p.tau[1] = float(tau[0]), float(tau[1])
    p.G[0][0] = 0.0
    p.G[1][1] = 0.0
    p.G[0][1] = float(G12)
    p.G[1][0] = float(G12 if G21 is None else G21)
    p.rho_s[0], p.rho_s[1] = float(rho_s[0]), float(rho_s[1])
    p.collision = {"bgk": 0, "regularized": 1, "regularized3": 2}[collision]
    p.wall_model = {"potential": 0, "mirror": 1}[wall_model]
    p.forcing = {"edm": 0, "guo": 1}[forcing]
    if solid is not None:
        m = np.ascontiguousarray(np.asarray(solid).reshape(shape) != 0, dtype=np.uint8)
        p._solid = m            # keeps the flags alive as long as the params
        p.solid = m.ctypes.data
    else:
        p.solid = None
    return p


def lattice():
    """(c[19,3] int, w[19]) in the oracle's own direction order."""
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    _L().oracle_lattice(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w))
    return c.astype(np.int64), w


def feq(rho, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(Q)
    _L().oracle_feq(float(rho), _dp(u), _dp(out))
    return out


def init(p, rho1, rho2, u=None):
    """Populations f[2,19,nz,ny,nx] = f^eq(rho^a_0, u_0) (Eq. 3)."""
    shape = (p.nz, p.ny, p.nx)
    rho1 = np.ascontiguousarray(rho1, dtype=np.float64).reshape(shape)
    rho2 = np.ascontiguousarray(rho2, dtype=np.float64).reshape(shape)
    f = np.zeros((2, Q) + shape)
    up = None
    if u is not None:
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(shape + (3,))
        up = _dp(u)
    _L().oracle_init(ctypes.byref(p), _dp(rho1), _dp(rho2), up, _dp(f))
    return f


def step(p, f, nsteps=1):
    """Advance f (modified in place and returned) by nsteps full updates."""
    assert f.shape == (2, Q, p.nz, p.ny, p.nx)
    work = np.empty_like(f)
    _L().oracle_step(ctypes.byref(p), _dp(f), _dp(work), int(nsteps))
    return f


def moments(p, f):
    """(rho1, rho2, uF[...,3]) with u_F = u + g/2 (Eqs. 8-9)."""
    shape = (p.nz, p.ny, p.nx)
    r1 = np.zeros(shape); r2 = np.zeros(shape); uF = np.zeros(shape + (3,))
    _L().oracle_moments(ctypes.byref(p), _dp(f), _dp(r1), _dp(r2), _dp(uF))
    return r1, r2, uF


def moments_raw(p, f):
    """(rho1, rho2, u[...,3]) of Eqs. 4-6 (u without the force shift)."""
    shape = (p.nz, p.ny, p.nx)
    r1 = np.zeros(shape); r2 = np.zeros(shape); u = np.zeros(shape + (3,))
    _L().oracle_moments_raw(ctypes.byref(p), _dp(f), _dp(r1), _dp(r2), _dp(u))
    return r1, r2, u


def interaction_sums(p, rho_b, rho_s_b=0.0):
    """(S_fluid, S_wall)[...,3] of Eqs. 7 and 13 for one density field."""
    shape = (p.nz, p.ny, p.nx)
    rho_b = np.ascontiguousarray(rho_b, dtype=np.float64).reshape(shape)
    sf = np.zeros(shape + (3,)); sw = np.zeros(shape + (3,))
    _L().oracle_interaction_sums(ctypes.byref(p), _dp(rho_b), float(rho_s_b), _dp(sf), _dp(sw))
    return sf, sw


def accelerations(p, rho1, rho2):
    shape = (p.nz, p.ny, p.nx)
    rho1 = np.ascontiguousarray(rho1, dtype=np.float64).reshape(shape)
    rho2 = np.ascontiguousarray(rho2, dtype=np.float64).reshape(shape)
    g1 = np.zeros(shape + (3,)); g2 = np.zeros(shape + (3,))
    _L().oracle_accelerations(ctypes.byref(p), _dp(rho1), _dp(rho2), _dp(g1), _dp(g2))
    return g1, g2


def collide_cell(p, a, fin, rho_a, u, g_a):
    fin = np.ascontiguousarray(fin, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    g_a = np.ascontiguousarray(g_a, dtype=np.float64)
    out = np.zeros(Q)
    _L().oracle_collide_cell(ctypes.byref(p), int(a), _dp(fin), float(rho_a), _dp(u), _dp(g_a), _dp(out))
    return out
