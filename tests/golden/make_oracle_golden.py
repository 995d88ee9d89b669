"""Write the oracle's expected values for the long GPU comparisons that are
too slow to recompute inside a test.  Calls only the FP64 CPU oracle
(``oracle/``) and host-side numpy measurements; nothing here runs the CUDA
library.

    python tests/golden/make_oracle_golden.py c2   # spinodal statistics, 64^3
    python tests/golden/make_oracle_golden.py c1   # Laplace fit of 3D droplets, 64^3
    python tests/golden/make_oracle_golden.py guo  # surface tension against tau, Guo forcing

c2: the spinodal mixture of the c2 case (Sec. 2 update with the regularized
filter of Eqs. 10-11; tau = 0.7, G^{12} = G^{21} = -1.2 of Eq. 7;
rho^a = 0.5 (1 +- 1 %) SplitMix64 noise with seeds 20160105 + a) on a 64^3
periodic lattice: per-component mass, <|rho^1 - rho^2|>, the first moment
k* of the spherically averaged structure factor and the interface area
(links across which rho^1 - rho^2 changes sign), every few hundred steps up
to 5000.

c1: static 3D droplets (Sec. 3; tanh spheres 1.0 / 0.03, W = 2, R0 = 10, 12,
14, 16, centred) on a 64^3 periodic lattice, BGK, tau = 1, G = -1.8, 3000
steps: the pressure jump of Eq. 12 with p = T0 rho - G T0 rho^1 rho^2 (mean
over r < R0/2 minus mean over r > R0 + 8), the equivalent radius of the
cells with rho^1 > 0.515 and the fit dp = 2 sigma / R + c.

guo: quasi-2D static droplets (Sec. 3; tanh discs 1.0 / 0.03, W = 2,
R0 = 8 and 12 on periodic squares of side 5 R0) with the regularized filter
and Guo's forcing (the second reading of the Sec. 2 forcing term),
G = -3.6, 20000 steps, for (tau_1 inside, tau_2 outside) = (0.55, 0.55),
(1, 1), (3, 3) and (0.525, 3) (viscosity ratio 100): the pressure jump of
Eq. 12 and the excess-mass radius of component 1 (diagnostics.mass_radius),
and the 2D fit dp = sigma / R + c per tau pair.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1601_01237_gb300 import diagnostics as dg  # noqa: E402
from paper_1601_01237_gb300 import workloads as wl  # noqa: E402

T0 = 1.0 / 3.0
C2 = dict(n=64, tau=(0.7, 0.7), G=-1.2, collision="regularized",
          checkpoints=(200, 500, 1000, 1500, 2000, 2500, 3000, 3500, 4000, 4500, 5000))
C1 = dict(n=64, tau=(1.0, 1.0), G=-1.8, collision="bgk", radii=(10, 12, 14, 16), steps=3000, thr=0.515)
GUO = dict(G=-3.6, collision="regularized", forcing="guo", radii=(8, 12), steps=20000,
           taus=((0.55, 0.55), (1.0, 1.0), (3.0, 3.0), (0.525, 3.0)))


def oracle_source_sha():
    with open(os.path.join(ROOT, "oracle", "lbm_oracle.c"), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def pressure_jump(a, b, G, center_xyz, r_in, r_out):
    nz, ny, nx = a.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def mi(d, n):
        return (d + n / 2.0) % n - n / 2.0
    r = np.sqrt(mi(x - center_xyz[0], nx) ** 2 + mi(y - center_xyz[1], ny) ** 2 + mi(z - center_xyz[2], nz) ** 2)
    p = T0 * (a + b) - G * T0 * a * b
    return float(p[r < r_in].mean() - p[r > r_out].mean())


def make_c2():
    n = C2["n"]
    shape = (n, n, n)
    r1, r2 = wl.spinodal(shape)
    p = oracle.make_params(shape, tau=C2["tau"], G12=C2["G"], collision=C2["collision"])
    f = oracle.init(p, r1, r2)
    rows, done, t0 = [], 0, time.time()
    for cp in C2["checkpoints"]:
        oracle.step(p, f, cp - done)
        done = cp
        a, b, _ = oracle.moments(p, f)
        st = dg.spinodal_stats(a, b)
        st["step"] = cp
        rows.append(st)
        print(json.dumps(st), "%.0f s" % (time.time() - t0), flush=True)
    out = {"case": "c2 spinodal mixture on a 64^3 periodic lattice (the c2 recipe: workloads.spinodal, "
                   "regularized, tau = 0.7, G = -1.2), FP64 oracle",
           "params": {k: v for k, v in C2.items() if k != "checkpoints"},
           "oracle_source_sha": oracle_source_sha(), "stats": rows}
    with open(os.path.join(HERE, "c2_spinodal64_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)


def make_c1():
    n = C1["n"]
    shape = (n, n, n)
    ctr = ((n - 1) / 2.0,) * 3
    rows = []
    for R0 in C1["radii"]:
        r1, r2 = wl.droplet(shape, R0)
        p = oracle.make_params(shape, tau=C1["tau"], G12=C1["G"], collision=C1["collision"])
        f = oracle.init(p, r1, r2)
        t0 = time.time()
        oracle.step(p, f, C1["steps"])
        a, b, _ = oracle.moments(p, f)
        dp = pressure_jump(a, b, C1["G"], ctr, R0 / 2.0, R0 + 8.0)
        vol = int((a > C1["thr"]).sum())
        rows.append({"R0": R0, "dp": dp, "volume": vol, "R_eq": dg.equivalent_radius(vol, False)})
        print(json.dumps(rows[-1]), "%.0f s" % (time.time() - t0), flush=True)
    sigma, icpt, res = dg.laplace_fit([r["R_eq"] for r in rows], [r["dp"] for r in rows], dims=3)
    out = {"case": "c1 3D static droplets on a 64^3 periodic lattice (BGK, tau = 1, G = -1.8, 3000 steps), "
                   "FP64 oracle",
           "params": {k: v for k, v in C1.items()}, "oracle_source_sha": oracle_source_sha(),
           "droplets": rows, "sigma": sigma, "intercept": icpt, "max_residual": res}
    with open(os.path.join(HERE, "c1_laplace64_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)


def _guo_droplet(job):
    tau, R0 = job
    oracle.set_threads(1)
    n = 5 * R0
    shape = (1, n, n)
    r1, r2 = wl.droplet(shape, R0)
    p = oracle.make_params(shape, tau=tau, G12=GUO["G"], collision=GUO["collision"], forcing=GUO["forcing"])
    f = oracle.init(p, r1, r2)
    oracle.step(p, f, GUO["steps"])
    a, b, _ = oracle.moments(p, f)
    c = ((n - 1) / 2.0, (n - 1) / 2.0, 0.0)
    dp = pressure_jump(a, b, GUO["G"], c, R0 / 2.0, R0 + 8.0)
    R, rin, rout = dg.mass_radius(a, c, R0 / 2.0, R0 + 8.0)
    return {"tau": list(tau), "R0": R0, "dp": dp, "R_mass": R, "rho_in": rin, "rho_out": rout}


def make_guo():
    import multiprocessing as mp
    jobs = [(tau, R0) for tau in GUO["taus"] for R0 in GUO["radii"]]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        rows = pool.map(_guo_droplet, jobs)
    fits = []
    for tau in GUO["taus"]:
        rs = [r for r in rows if tuple(r["tau"]) == tuple(tau)]
        sigma, icpt, res = dg.laplace_fit([r["R_mass"] for r in rs], [r["dp"] for r in rs])
        fits.append({"tau": list(tau), "sigma": sigma, "intercept": icpt})
        print(json.dumps(fits[-1]), flush=True)
    out = {"case": "quasi-2D static droplets, regularized filter with Guo forcing, G = -3.6, 20000 steps, FP64 oracle",
           "params": {k: (list(v) if isinstance(v, tuple) else v) for k, v in GUO.items()},
           "oracle_source_sha": oracle_source_sha(), "droplets": rows, "fits": fits}
    with open(os.path.join(HERE, "guo_sigma_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    which = sys.argv[1:] or ["c2", "c1", "guo"]
    if "c2" in which:
        make_c2()
    if "c1" in which:
        make_c1()
    if "guo" in which:
        make_guo()
