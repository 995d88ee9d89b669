"""Staircase walls (a mask of solid sites, the inclined walls of Sec. 4.2) on
the GPU against the FP64 oracle: every population after a few steps, fields
after many, the inclined channel of the wall study in FP32, conservation, and
the refusals of calls that take no mask."""
import numpy as np
import pytest

import oracle
from paper_1601_01237_gb300 import workloads as wl
from _helpers import direction_map, gpu_run, oracle_run, rel_err

pytestmark = pytest.mark.gpu


def _blocks(shape, seed):
    """A staircase along the bottom, a pillar and scattered solid sites on a
    periodic lattice (ragged in every direction)."""
    nz, ny, nx = shape
    m = np.zeros(shape, np.uint8)
    for x in range(nx):
        m[: 1 + (2 * x) // nx, :, x] = 1
    m[nz // 2:, : ny // 2 + 1, nx // 3] = 1
    rng = np.random.default_rng(seed)
    for _ in range(max(3, m.size // 60)):
        m[rng.integers(0, nz), rng.integers(0, ny), rng.integers(0, nx)] = 1
    return m


MASK_CASES = [
    ("bgk_mirror", (7, 5, 9), dict(tau=(0.8, 1.1), G12=-1.4, g_ext=(1e-4, -5e-5, 2e-4))),
    ("reg_mirror_rhos", (6, 7, 5), dict(tau=(0.7, 1.2), G12=-1.3, rho_s=(0.05, 0.1), collision="regularized")),
    ("reg3_mirror", (5, 6, 8), dict(tau=(0.6, 0.9), G12=-1.2, rho_s=(0.0, 0.08), collision="regularized3")),
    ("bgk_potential", (6, 4, 7), dict(tau=(1.0, 0.8), G12=-1.1, rho_s=(0.0, 0.2), wall_model="potential")),
    ("quasi2d", (9, 1, 11), dict(tau=(0.9, 0.9), G12=-1.6, rho_s=(0.0, 0.1))),
]


@pytest.mark.parametrize("name,shape,kw", MASK_CASES, ids=[c[0] for c in MASK_CASES])
def test_mask_populations_f64(gpu_lib, name, shape, kw):
    """Every population (solid sites included, which hold zeros) after 0, 1
    and 3 steps from a random state, FP64."""
    perm = direction_map()
    solid = _blocks(shape, seed=3)
    r1, r2, u = wl.random_state(shape, seed=12, u_max=0.04)
    for nsteps in (0, 1, 3):
        _, f_or = oracle_run(shape, r1, r2, u, nsteps, solid=solid, **kw)
        lat = gpu_run(shape, r1, r2, u, nsteps, storage="f64", solid=solid, **kw)
        f_gpu = lat.get_populations()
        lat.close()
        assert rel_err(f_gpu, f_or[:, perm]) < 1e-13, (name, nsteps)
        assert np.all(f_gpu[:, :, solid == 1] == 0)


@pytest.mark.parametrize("name,shape,kw", MASK_CASES[:3], ids=[c[0] for c in MASK_CASES[:3]])
def test_mask_fields_200_steps_f64(gpu_lib, name, shape, kw):
    """rho^1, rho^2, u_F after 200 steps, FP64; masses as the oracle's."""
    solid = _blocks(shape, seed=4)
    r1, r2, u = wl.random_state(shape, seed=6, u_max=0.02)
    p, f_or = oracle_run(shape, r1, r2, u, 200, solid=solid, **kw)
    a, b, uF = oracle.moments(p, f_or)
    lat = gpu_run(shape, r1, r2, u, 200, storage="f64", solid=solid, **kw)
    ga, gb, guF = lat.moments(out_f64=True)
    red = lat.reduce()
    lat.close()
    assert rel_err(ga, a) < 1e-11 and rel_err(gb, b) < 1e-11
    assert np.max(np.abs(guF - uF)) < 1e-11 * max(np.abs(uF).max(), 1e-3)
    assert np.all(ga[solid == 1] == 0) and np.all(guF[solid == 1] == 0)
    assert abs(red["mass1"] - a.sum()) < 1e-12 * a.sum() and abs(red["mass2"] - b.sum()) < 1e-12 * b.sum()


@pytest.mark.parametrize("theta", [30, 70])
@pytest.mark.parametrize("wall_model", ["mirror", "potential"])
def test_inclined_channel_f32(gpu_lib, theta, wall_model):
    """The inclined-wall geometry (channel height 16, staircase walls) with a
    droplet of component 2 on the lower wall, FP32 storage, 300 steps,
    against the FP64 oracle: densities within 1e-5 of the largest density
    (the FP32 bar) and velocities within 1e-6."""
    shape, solid, info = wl.inclined_channel(theta)
    r1, r2 = wl.channel_droplet(shape, info, 7.0)
    kw = dict(tau=(1.0, 1.0), G12=wl.G_DROPLET, rho_s=(0.0, 0.4), wall_model=wall_model, collision="regularized")
    p, f_or = oracle_run(shape, r1, r2, None, 300, solid=solid, **kw)
    a, b, uF = oracle.moments(p, f_or)
    lat = gpu_run(shape, r1, r2, None, 300, storage="f32", solid=solid, **kw)
    ga, gb, guF = lat.moments()
    lat.close()
    fl = solid == 0
    ea = np.max(np.abs(ga - a)[fl]) / a.max()
    eb = np.max(np.abs(gb - b)[fl]) / b.max()
    print("inclined %d deg %s: |drho|/max rho %.3g %.3g, per cell %.3g, |du| %.3g" % (
        theta, wall_model, ea, eb, np.max(np.abs(gb - b)[fl] / b[fl]), np.max(np.abs(guF - uF))))
    assert ea < 1e-5 and eb < 1e-5
    assert np.max(np.abs(guF - uF)) < 1e-6
    assert np.all(ga[~fl] == 0)


def test_mask_mass_conserved_long_run(gpu_lib):
    """Bounce-back conserves each component's mass: 5000 FP64 steps of the
    30-degree channel with a wetting droplet, mass drift below 1e-12."""
    shape, solid, info = wl.inclined_channel(30)
    r1, r2 = wl.channel_droplet(shape, info, 7.0)
    from paper_1601_01237_gb300 import Lattice
    lat = Lattice(shape, storage="f64", tau=(1.0, 1.0), G12=wl.G_DROPLET, rho_s=(0.0, 0.4))
    lat.set_solid(solid)
    lat.init_fields(r1, r2)
    m0 = lat.reduce()
    lat.step(5000)
    m1 = lat.reduce()
    lat.close()
    fl = solid == 0
    assert abs(m0["mass1"] - r1[fl].sum()) < 1e-12 * m0["mass1"]
    assert abs(m1["mass1"] - m0["mass1"]) < 1e-12 * m0["mass1"]
    assert abs(m1["mass2"] - m0["mass2"]) < 1e-12 * m0["mass2"]


def test_empty_mask_matches_no_mask(gpu_lib, monkeypatch):
    """A mask with no solid site steps exactly like the two-kernel step
    without a mask (FP32, bitwise)."""
    monkeypatch.setenv("LBM_FUSED", "0")
    shape = (10, 6, 12)
    r1, r2, u = wl.random_state(shape, seed=2, u_max=0.03)
    kw = dict(tau=(0.8, 1.0), G12=-1.3, collision="regularized")
    a = gpu_run(shape, r1, r2, u, 20, storage="f32", **kw)
    b = gpu_run(shape, r1, r2, u, 20, storage="f32", solid=np.zeros(shape, np.uint8), **kw)
    fa, fb = a.get_populations(), b.get_populations()
    a.close()
    b.close()
    assert np.array_equal(fa, fb)


# The fused single-pass step under a mask, on lattices of several tiles with
# ragged edges (solid halo cells, solid sites at chunk boundaries): both wall
# models, the three collision operators, and Guo's forcing.
FUSED_MASK_CASES = [
    ("bgk_mirror", (37, 19, 45), dict(tau=(0.6, 1.3), G12=-1.3, g_ext=(1e-5, -2e-5, 1e-5), rho_s=(0.05, 0.1))),
    ("reg_potential", (20, 11, 70), dict(tau=(0.7, 0.9), G12=-1.2, rho_s=(0.0, 0.2), wall_model="potential",
                                         collision="regularized")),
    ("reg3_mirror", (19, 9, 33), dict(tau=(0.8, 1.1), G12=-1.3, collision="regularized3")),
    ("guo_reg_mirror", (24, 10, 40), dict(tau=(0.55, 0.9), G12=-1.2, rho_s=(0.0, 0.1), collision="regularized",
                                          forcing="guo")),
]


def _path(lat):
    return sorted(lat.step_timed(1))


@pytest.mark.parametrize("name,shape,kw", FUSED_MASK_CASES, ids=[c[0] for c in FUSED_MASK_CASES])
def test_mask_fused_f32_against_oracle(gpu_lib, monkeypatch, name, shape, kw):
    """FP32 fused step with a mask against the FP64 oracle after 21 steps:
    densities within 2e-6 per fluid cell, velocities within 2e-7; solid sites
    hold zero."""
    monkeypatch.setenv("LBM_FUSED", "1")
    solid = _blocks(shape, seed=5)
    r1, r2, u = wl.random_state(shape, seed=4, u_max=0.03)
    p, f_or = oracle_run(shape, r1, r2, u, 21, solid=solid, **kw)
    a, b, uF = oracle.moments(p, f_or)
    lat = gpu_run(shape, r1, r2, u, 20, storage="f32", solid=solid, **kw)
    assert _path(lat) == ["k_step_fused"]   # the 21st step, timed
    ga, gb, guF = lat.moments()
    lat.close()
    fl = solid == 0
    ea = np.max(np.abs(ga - a)[fl] / a[fl])
    eb = np.max(np.abs(gb - b)[fl] / b[fl])
    print("%s: max |drho|/rho %.3g %.3g, |du| %.3g" % (name, ea, eb, np.max(np.abs(guF - uF))))
    assert ea < 2e-6 and eb < 2e-6
    assert np.max(np.abs(guF - uF)) < 2e-7
    assert np.all(ga[~fl] == 0) and np.all(gb[~fl] == 0)


@pytest.mark.parametrize("storage", ["f32", "bf16_dev", "f16_rel", "bf16_rel"])
@pytest.mark.parametrize("name,shape,kw", FUSED_MASK_CASES[:2], ids=[c[0] for c in FUSED_MASK_CASES[:2]])
def test_mask_fused_matches_split(gpu_lib, monkeypatch, storage, name, shape, kw):
    """Fused and two-kernel steps under the same mask agree to rounding in
    every storage format after 8 steps (the two paths sum a wall site's fluid
    neighbours' densities in different orders; the 16-bit formats may round a
    population either way where those differ)."""
    solid = _blocks(shape, seed=6)
    r1, r2, u = wl.random_state(shape, seed=8, u_max=0.03)
    extra = {"rho0_dev": 0.5} if storage.endswith("_dev") else {}
    out = {}
    for fused in ("1", "0"):
        monkeypatch.setenv("LBM_FUSED", fused)
        lat = gpu_run(shape, r1, r2, u, 7, storage=storage, solid=solid, **kw, **extra)
        assert _path(lat) == (["k_step_fused"] if fused == "1" else ["k_collide", "k_density"])
        out[fused] = lat.get_populations()
        lat.close()
    diff = np.max(np.abs(out["1"] - out["0"]))
    print("%s %s: fused vs two-kernel, max |df| %.3g" % (name, storage, diff))
    if storage == "f32":
        assert rel_err(out["1"], out["0"]) < 1e-6
    elif storage.endswith("_rel"):
        # one flipped 16-bit rounding of a relative deviation (as without a mask)
        assert diff <= 2.0 ** -5 * np.abs(out["0"]).max()
    else:
        # a few BF16 ulps of the largest deviation from w_i rho0 over the fluid cells
        from paper_1601_01237_gb300 import lbm_lattice_dirs
        _, w = lbm_lattice_dirs()
        dev = np.abs(out["0"] - 0.5 * w[None, :, None, None, None])[:, :, solid == 0]
        assert diff <= 2.0 ** -5 * dev.max()
    assert np.all(out["1"][:, :, solid == 1] == 0)


def test_mask_refusals(gpu_lib):
    from paper_1601_01237_gb300 import LBMError, Lattice
    shape = (6, 4, 5)
    solid = _blocks(shape, seed=1)
    lat = Lattice(shape, storage="f32", periodic=(1, 1, 0))
    with pytest.raises(LBMError, match="ENOTSUP"):
        lat.set_solid(solid)
    lat.close()
    lat = Lattice(shape, storage="f32", G12=-1.2)
    lat.set_solid(solid)
    lat.init_fields(np.full(shape, 0.5), np.full(shape, 0.5))
    lat.record(2, 1)          # the reverse pass takes the mask
    with pytest.raises(ValueError):
        lat.set_solid(solid[:, :, :-1])
    lat.set_solid(None)       # dropping the mask drops the recording
    with pytest.raises(LBMError, match="EINVAL"):
        lat.adjoint(np.zeros(shape), None)
    lat.close()


def test_mask_droplet_stats_and_pressure(gpu_lib):
    """Droplet statistics and the pressure jump on a masked lattice (inclined
    channel, droplet on the wall, FP64, 200 steps) against the same sums over
    the oracle's fields: solid sites left out, and the thin-film layer is the
    fluid cells next to a solid site."""
    shape, solid, info = wl.inclined_channel(30)
    r1, r2 = wl.channel_droplet(shape, info, 7.0)
    # component 1 as the droplet: swap the roles
    r1, r2 = r2, r1
    kw = dict(tau=(1.0, 1.0), G12=wl.G_DROPLET, rho_s=(0.3, 0.0))
    p, f_or = oracle_run(shape, r1, r2, None, 200, solid=solid, **kw)
    a, b, _ = oracle.moments(p, f_or)
    lat = gpu_run(shape, r1, r2, None, 200, storage="f64", solid=solid, **kw)
    nz, _, nx = shape
    thr = 0.5
    origin = ((nx - 1) / 2.0, 0.0, (nz - 1) / 2.0)
    st = lat.droplet_stats(thr, origin=origin)
    pin, pout, dp = lat.pressure_jump(origin, 3.0, 12.0)
    lat.close()
    fl = solid == 0
    z, y, x = np.meshgrid(np.arange(nz), np.arange(1), np.arange(nx), indexing="ij")
    drop = fl & (a > thr)
    mi = lambda d, n: d - n * np.round(d / n)
    assert st["volume"] == drop.sum()
    assert abs(st["mass"] - a[drop].sum()) < 1e-10 * a[drop].sum()
    assert abs(st["com"][0] - mi(x - origin[0], nx)[drop].mean()) < 1e-9
    assert abs(st["com"][2] - mi(z - origin[2], nz)[drop].mean()) < 1e-9
    near = np.zeros_like(fl)
    for dz in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dz or dx:
                near |= np.roll(np.roll(solid == 1, -dz, axis=0), -dx, axis=2)
    # quasi-2D: links along y land on the cell's own column
    film = fl & ~drop & near
    assert film.sum() > 0 and abs(st["film_rho"] - a[film].mean()) < 1e-10
    pr = (a + b) / 3.0 - wl.G_DROPLET / 3.0 * a * b
    r = np.sqrt(mi(x - origin[0], nx) ** 2 + mi(z - origin[2], nz) ** 2)
    assert abs(pin - pr[fl & (r < 3.0)].mean()) < 1e-12 and abs(pout - pr[fl & (r > 12.0)].mean()) < 1e-12
