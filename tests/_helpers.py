"""Shared test helpers: run the CUDA library and the oracle on the same seeded
inputs and compare.  The oracle is imported here only, for tests."""
import numpy as np

import oracle

Q = 19


# A strongly separating G of Eq. 7 (flat-interface coexistence 1.056 / 0.0045
# at tau = 1) for the droplet tests; parity and the pins need no particular G.
G_STRONG = -2.7


def direction_map():
    """perm such that oracle direction perm[i] has the library's c_i."""
    from paper_1601_01237_gb300 import lbm_lattice_dirs
    c_lib, w_lib = lbm_lattice_dirs()
    c_or, w_or = oracle.lattice()
    perm = np.array([int(np.where((c_or == c_lib[i]).all(1))[0][0]) for i in range(Q)])
    assert np.allclose(w_or[perm], w_lib)
    return perm


def oracle_run(shape, rho1, rho2, u, nsteps, tau=(1.0, 1.0), G12=0.0, G21=None, g_ext=(0, 0, 0),
               periodic=(1, 1, 1), rho_s=(0.0, 0.0), collision="bgk", wall_model="mirror", rho0_dev=None,
               solid=None, forcing="edm"):
    p = oracle.make_params(shape, tau=tau, G12=G12, G21=G21, g_ext=g_ext, periodic=periodic, rho_s=rho_s,
                           collision=collision, wall_model=wall_model, solid=solid, forcing=forcing)
    f = oracle.init(p, rho1, rho2, u)
    if nsteps:
        oracle.step(p, f, nsteps)
    return p, f


def gpu_run(shape, rho1, rho2, u, nsteps, storage="f64", solid=None, **kw):
    from paper_1601_01237_gb300 import Lattice
    lat = Lattice(shape, storage=storage, **kw)
    if solid is not None:
        lat.set_solid(solid)
    lat.init_fields(rho1, rho2, u)
    if nsteps:
        lat.step(nsteps)
    return lat


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
