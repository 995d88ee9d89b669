"""Run one of the five synthetic cases on the GPU and print its measurements
as one JSON line.

    python -m paper_1601_01237_gb300.run_config c0 [--steps N] [--stride K]

c0  quasi-2D droplet 64x64x1, FP64: Delta p, spurious current max|u_F|, mass drift
c1  3D droplets 128^3, FP32: Delta p vs 1/R fit (surface tension) per tau
c2  spinodal mixture 256^3: FP32 / FP16-dev / BF16-dev, MLUPS, mass drift,
    interface measure <|rho1 - rho2|>
c3  differentiation 96^3: loss, gradients (tied G, tau_1), adjoint/forward time
c4  wall-bounded 512x512x384, regularized, mirror wetting, tilted gravity:
    MLUPS, droplet drift velocity, thin-film density, volume ratio

Everything runs through the C ABI of include/lbm.h; torch provides device
buffers and the stream only.
"""
import argparse
import json
import time

import numpy as np

from . import diagnostics as dg
from . import workloads as wl
from .lattice import Lattice


def _timed_steps(lat, n, chunk=500):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = 0
    while done < n:
        k = min(chunk, n - done)
        lat.step(k)
        done += k
    lat.sync()
    return time.perf_counter() - t0


def run_c0(steps=None):
    c = wl.CONFIGS["c0_droplet2d_f64"]
    steps = steps or c["steps"]
    shape = c["shape"]
    lat = Lattice(shape, storage=c["storage"], tau=c["tau"], G12=c["G"])
    r1, r2 = wl.droplet(shape, c["R"])
    lat.init_fields(r1, r2)
    m0 = lat.reduce()
    dt = _timed_steps(lat, steps)
    m1 = lat.reduce()
    ctr = ((shape[2] - 1) / 2.0, (shape[1] - 1) / 2.0, 0.0)
    pin, pout, dp = lat.pressure_jump(ctr, c["R"] / 2.0, c["R"] + 8.0)
    st = lat.droplet_stats(0.5 * (1.0 + 0.03), origin=ctr)
    lat.close()
    R = dg.equivalent_radius(st["volume"], True)
    return {"case": "c0", "steps": steps, "delta_p": dp, "p_in": pin, "p_out": pout, "R_equiv": R,
            "sigma_estimate": dp * R, "spurious_max_uF": m1["max_uF"],
            "mass_drift": [abs(m1["mass1"] - m0["mass1"]) / m0["mass1"], abs(m1["mass2"] - m0["mass2"]) / m0["mass2"]],
            "MLUPS": np.prod(shape) * steps / dt / 1e6}


def run_c1(steps=None, radii=None, taus=None, shape=None, storage=None):
    c = wl.CONFIGS["c1_droplet3d_f32"]
    steps = steps or c["steps"]
    shape = tuple(shape or c["shape"])
    storage = storage or c["storage"]
    radii = radii or c["radii"]
    taus = taus or c["taus"]
    out = {"case": "c1", "steps": steps, "shape": shape, "storage": storage, "fits": {}}
    for tau in taus:
        # the tau = 0.55 BGK runs diverge for every tested G (see the design notes);
        # they are run with the regularized operator at G = -1.2
        if tau < 0.6:
            G, col = -1.2, "regularized"
        else:
            G, col = c["G"], "bgk"
        Rs, dps, spur = [], [], []
        for R0 in radii:
            lat = Lattice(shape, storage=storage, tau=(tau, tau), G12=G, collision=col)
            r1, r2 = wl.droplet(shape, R0)
            lat.init_fields(r1, r2)
            lat.step(steps)
            ctr = ((shape[2] - 1) / 2.0, (shape[1] - 1) / 2.0, (shape[0] - 1) / 2.0)
            _, _, dp = lat.pressure_jump(ctr, R0 / 2.0, R0 + 8.0)
            st = lat.droplet_stats(0.5 * (1.0 + 0.03), origin=ctr)
            spur.append(lat.reduce()["max_uF"])
            lat.close()
            Rs.append(dg.equivalent_radius(st["volume"], False))
            dps.append(dp)
        sigma, icpt, res = dg.laplace_fit(Rs, dps, dims=3)
        out["fits"][str(tau)] = {"collision": col, "G_eq7": G, "R": Rs, "delta_p": dps, "sigma": sigma,
                                 "intercept": icpt, "max_residual": res, "spurious_max_uF": spur}
    return out


def run_c2(steps=None, storages=("f32", "f16_dev", "bf16_dev")):
    c = wl.CONFIGS["c2_spinodal256"]
    steps = steps or c["steps"]
    shape = c["shape"]
    r1, r2 = wl.spinodal(shape)
    out = {"case": "c2", "steps": steps, "runs": {}}
    for st in storages:
        kw = {"rho0_dev": 0.5} if st.endswith("_dev") else {}
        lat = Lattice(shape, storage=st, tau=c["tau"], G12=c["G"], **kw)
        lat.init_fields(r1, r2)
        m0 = lat.reduce()
        dt = _timed_steps(lat, steps)
        a, b, _ = lat.moments(out_f64=False)
        m1 = lat.reduce()
        lat.close()
        out["runs"][st] = {"MLUPS": np.prod(shape) * steps / dt / 1e6,
                           "mass_drift": abs(m1["mass1"] - m0["mass1"]) / m0["mass1"],
                           "mean_abs_rho1_minus_rho2": float(np.mean(np.abs(a - b))),
                           "rho1_range": [float(a.min()), float(a.max())]}
    return out


def run_c3(steps=None):
    import torch
    c = wl.CONFIGS["c3_adjoint96"]
    steps = steps or c["steps"]
    shape = c["shape"]
    r1, r2 = wl.droplet(shape, c["R"])
    tgt, _ = wl.ellipsoid(shape, c["target_axes"])
    lat = Lattice(shape, storage=c["storage"], tau=c["tau"], G12=c["G"])
    lat.init_fields(r1, r2)
    t_f = _timed_steps(lat, steps)
    lat.init_fields(r1, r2)
    lat.record(steps, c["ckpt_every"])
    a = torch.empty(shape, dtype=torch.float64, device="cuda")
    lat.moments_device(rho1=a, out_f64=True)
    t = torch.from_numpy(tgt).cuda()
    loss = float(((a - t) ** 2).sum())
    g0 = torch.empty(shape, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    par = lat.adjoint(2.0 * (a - t), None, g0, None)
    t_a = time.perf_counter() - t0
    lat.close()
    return {"case": "c3", "steps": steps, "loss": loss, "dL_dG_tied": par[0] + par[1], "dL_dtau1": par[2],
            "grad_rho1_0_norm": float(torch.linalg.norm(g0)), "forward_s": t_f, "adjoint_s": t_a,
            "adjoint_forward_ratio": t_a / t_f}


def run_c4(steps=None, stride=None, shape=None):
    c = wl.CONFIGS["c4_wall512"]
    steps = steps or c["steps"]
    shape = tuple(shape or c["shape"])
    g = wl.tilted_gravity(c["g_mag"], c["tilt_deg"])
    lat = Lattice(shape, storage=c["storage"], tau=c["tau"], G12=c["G"], collision=c["collision"],
                  periodic=c["periodic"], g_ext=g, wall_model="mirror")
    r1, r2 = wl.hemisphere(shape, c["R"])
    lat.init_fields(r1, r2)
    nz, ny, nx = shape
    origin = ((nx - 1) / 2.0, (ny - 1) / 2.0, -0.5)
    thr = 0.5 * (1.0 + 0.03)
    # drift over the last quarter of the run (the paper measures between
    # 8.0e4 and 8.5e4 steps of a longer run)
    t_a = steps - max(steps // 4, 1)
    dt = _timed_steps(lat, t_a)
    s_a = lat.droplet_stats(thr, origin)
    dt += _timed_steps(lat, steps - t_a)
    s_b = lat.droplet_stats(thr, origin)
    red = lat.reduce()
    lat.close()
    v = dg.drift_velocity(s_a["com"], s_b["com"], steps - t_a)
    return {"case": "c4", "steps": steps, "shape": shape, "MLUPS": np.prod(shape) * steps / dt / 1e6,
            "drift_velocity": v.tolist(), "film_rho1": s_b["film_rho"], "volume_ratio": s_b["volume"] / np.prod(shape),
            "droplet_volume": s_b["volume"], "max_uF": red["max_uF"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["c0", "c1", "c2", "c3", "c4"])
    ap.add_argument("--steps", type=int, default=None)
    args = ap.parse_args()
    fn = {"c0": run_c0, "c1": run_c1, "c2": run_c2, "c3": run_c3, "c4": run_c4}[args.case]
    print(json.dumps(fn(args.steps), default=float))


if __name__ == "__main__":
    main()
