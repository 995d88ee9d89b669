"""Gradients of the hand-written reverse pass (lbm_record / lbm_adjoint)
against central finite differences of the FP64 oracle.

Case (the differentiation configuration): a 96^3 droplet (R = 20) and a
target from an ellipsoidal initialisation with semi-axes (24, 20, 16); the
check runs on an 8^3 periodic crop of both at the interface, centred at
(x, y, z) = (68, 48, 48), for 20 steps with checkpoints every 5.
Loss L = sum_x (rho^1_N - rho^1_target)^2; gradients with respect to every
initial rho^1 cell, the tied G^{12} = G^{21} and tau_1; central differences
with h = 1e-3.  Bar: relative error <= 1e-4.
"""
import numpy as np
import pytest

import oracle
from paper_1601_01237_gb300 import workloads as wl
from _helpers import G_STRONG

pytestmark = pytest.mark.gpu

H = 1e-3
STEPS = 20
CKPT = 5


def crop_case():
    full1, full2 = wl.droplet((96, 96, 96), 20)
    tgt, _ = wl.ellipsoid((96, 96, 96), (24, 20, 16))
    sl = (slice(44, 52), slice(44, 52), slice(64, 72))
    return full1[sl].copy(), full2[sl].copy(), tgt[sl].copy()


def oracle_loss(r1, r2, tgt, G, tau1, tau2, steps, **kw):
    p = oracle.make_params(r1.shape, tau=(tau1, tau2), G12=G, G21=G, **kw)
    f = oracle.init(p, r1, r2)
    oracle.step(p, f, steps)
    a, _, _ = oracle.moments(p, f)
    return float(((a - tgt) ** 2).sum())


def fd_grads(r1, r2, tgt, G, tau1, tau2, steps, cells=None, h=H, **kw):
    L = lambda **o: oracle_loss(o.get("r1", r1), r2, tgt, o.get("G", G), o.get("tau1", tau1), tau2, steps, **kw)
    gG = (L(G=G + h) - L(G=G - h)) / (2 * h)
    gT = (L(tau1=tau1 + h) - L(tau1=tau1 - h)) / (2 * h)
    gr = np.zeros(r1.shape)
    idx = list(np.ndindex(r1.shape)) if cells is None else cells
    for c in idx:
        rp = r1.copy(); rp[c] += h
        rm = r1.copy(); rm[c] -= h
        gr[c] = (L(r1=rp) - L(r1=rm)) / (2 * h)
    return gG, gT, gr


def gpu_grads(r1, r2, tgt, G, tau1, tau2, steps, storage, **kw):
    from paper_1601_01237_gb300 import Lattice
    lat = Lattice(r1.shape, storage=storage, tau=(tau1, tau2), G12=G, G21=G, **kw)
    lat.init_fields(r1, r2)
    lat.record(steps, CKPT)
    a, _, _ = lat.moments()
    d1 = np.empty(r1.shape)
    par = lat.adjoint(2 * (a - tgt), None, d1, None)
    lat.close()
    return par[0] + par[1], par[2], d1


@pytest.fixture(scope="module")
def fd_reference():
    r1, r2, tgt = crop_case()
    G = G_STRONG
    return (r1, r2, tgt, G) + fd_grads(r1, r2, tgt, G, 1.0, 1.0, STEPS)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_adjoint_matches_finite_differences(gpu_lib, fd_reference, storage):
    r1, r2, tgt, G, fG, fT, fr = fd_reference
    gG, gT, gr = gpu_grads(r1, r2, tgt, G, 1.0, 1.0, STEPS, storage)
    eG = abs(gG - fG) / abs(fG)
    eT = abs(gT - fT) / abs(fT)
    er = np.linalg.norm(gr - fr) / np.linalg.norm(fr)
    print("%s adjoint vs FD: dG %.3g (%.6g vs %.6g), dtau1 %.3g, drho1_0 %.3g" % (storage, eG, gG, fG, eT, er))
    assert eG <= 1e-4 and eT <= 1e-4 and er <= 1e-4
    big = np.abs(fr) > 1e-3 * np.abs(fr).max()
    assert np.max(np.abs(gr - fr)[big] / np.abs(fr)[big]) <= 1e-3


@pytest.mark.parametrize("storage", ["f16_dev", "bf16_dev", "f16_rel", "bf16_rel"])
def test_adjoint_16bit_storage_tracks_fp32(gpu_lib, storage):
    """The reverse pass on 16-bit storage (states decoded to FP32, the
    rounding of the stored values taken as identity) against the FP32 reverse
    pass on the differentiation crop: the gradients differ by the 16-bit
    trajectory's own deviation from the FP32 one."""
    r1, r2, tgt = crop_case()
    G = G_STRONG
    ref = gpu_grads(r1, r2, tgt, G, 1.0, 1.0, STEPS, "f32")
    extra = {"rho0_dev": 0.5} if storage.endswith("_dev") else {}
    got = gpu_grads(r1, r2, tgt, G, 1.0, 1.0, STEPS, storage, **extra)
    eG = abs(got[0] - ref[0]) / abs(ref[0])
    eT = abs(got[1] - ref[1]) / abs(ref[1])
    er = np.linalg.norm(got[2] - ref[2]) / np.linalg.norm(ref[2])
    print("%s vs FP32 adjoint: dG %.3g, dtau1 %.3g, drho1_0 %.3g" % (storage, eG, eT, er))
    # measured: FP16-dev <= 5.5e-4, FP16-rel <= 4.3e-4, BF16-rel <= 1.9e-3,
    # BF16-dev <= 5.1e-3 (the tau_1 derivative is the most sensitive)
    bound = 2e-3 if storage.startswith("f16") else 2e-2
    assert eG <= bound and eT <= bound and er <= bound


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("collision", ["bgk", "regularized", "regularized3"])
def test_adjoint_walls_and_forcing(gpu_lib, collision, storage):
    """Reverse pass through mirror wetting walls, bounce-back, g_ext, unequal
    tau and the regularized operator, on sampled cells (FP64: 1e-5 of the
    oracle's central differences; FP32, whose force-adjoint stencil runs in
    the tiled kernel: 1e-4)."""
    shape = (6, 5, 7)
    r1, r2, _ = wl.random_state(shape, seed=17, u_max=0.0)
    tgt = np.roll(r1, 2, axis=2)
    kw = dict(periodic=(1, 1, 0), g_ext=(2e-4, -1e-4, 3e-4), collision=collision, rho_s=(0.03, 0.0))
    G, t1, t2, steps = -1.3, 0.8, 1.2, 6
    rng = np.random.default_rng(3)
    cells = [tuple(int(v) for v in (rng.integers(0, 6), rng.integers(0, 5), rng.integers(0, 7))) for _ in range(10)]
    cells += [(0, 2, 3), (5, 1, 1)]   # both wall layers
    fG, fT, fr = fd_grads(r1, r2, tgt, G, t1, t2, steps, cells=cells, **kw)
    from paper_1601_01237_gb300 import Lattice
    lat = Lattice(shape, storage=storage, tau=(t1, t2), G12=G, G21=G, **kw)
    lat.init_fields(r1, r2)
    lat.record(steps, 4)
    a, _, _ = lat.moments()
    d1 = np.empty(shape)
    par = lat.adjoint(2 * (a - tgt), None, d1, None)
    lat.close()
    tol = 1e-5 if storage == "f64" else 1e-4
    print("%s %s walls: dG %.6g vs %.6g, dtau1 %.6g vs %.6g" % (storage, collision, par[0] + par[1], fG, par[2], fT))
    assert abs(par[0] + par[1] - fG) <= tol * abs(fG)
    assert abs(par[2] - fT) <= tol * abs(fT)
    scale = np.abs([fr[q] for q in cells]).max()
    for c in cells:
        assert abs(d1[c] - fr[c]) <= tol * scale, (c, d1[c], fr[c])


def _staircase(shape, seed):
    """A staircase along the bottom, a pillar and a few scattered solid
    sites on a periodic lattice."""
    nz, ny, nx = shape
    m = np.zeros(shape, np.uint8)
    for x in range(nx):
        m[: 1 + (2 * x) // nx, :, x] = 1
    m[nz // 2:, : ny // 2, nx // 2] = 1
    rng = np.random.default_rng(seed)
    for _ in range(3):
        m[rng.integers(0, nz), rng.integers(0, ny), rng.integers(0, nx)] = 1
    return m


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("wall_model,collision", [("mirror", "bgk"), ("mirror", "regularized"),
                                                  ("potential", "bgk")])
def test_adjoint_solid_mask(gpu_lib, wall_model, collision, storage):
    """Reverse pass through a mask of solid sites (Sec. 4.2 staircase walls):
    bounce-back links and, for the mirror model, the wall densities' dependence
    on the fluid densities (Eq. 13), on sampled fluid cells, many of them next
    to a solid site, against the oracle's central differences (FP64 1e-5,
    FP32 1e-4); solid sites get a zero initial-density gradient.  The step is
    h = 1e-4: this case's dL/dG is small (-0.0192), and at h = 1e-3 the
    central difference is 2.3e-5 away from its limit (the oracle's
    differences at h = 1e-2 .. 1e-4 converge to -0.01920134)."""
    shape = (7, 5, 6)
    solid = _staircase(shape, seed=2)
    r1, r2, _ = wl.random_state(shape, seed=21, u_max=0.0)
    tgt = np.roll(r1, 1, axis=2)
    kw = dict(g_ext=(2e-4, -1e-4, 3e-4), collision=collision, rho_s=(0.03, 0.1), wall_model=wall_model)
    G, t1, t2, steps = -1.3, 0.8, 1.2, 6
    fluid = [tuple(int(v) for v in c) for c in np.argwhere(solid == 0)]
    rng = np.random.default_rng(5)
    cells = [fluid[k] for k in rng.choice(len(fluid), 14, replace=False)]
    fG, fT, fr = fd_grads(r1, r2, tgt, G, t1, t2, steps, cells=cells, h=1e-4, solid=solid, **kw)
    from paper_1601_01237_gb300 import Lattice
    lat = Lattice(shape, storage=storage, tau=(t1, t2), G12=G, G21=G, **kw)
    lat.set_solid(solid)
    lat.init_fields(r1, r2)
    lat.record(steps, 4)
    a, _, _ = lat.moments()
    d1 = np.empty(shape)
    par = lat.adjoint(2 * (a - tgt), None, d1, None)
    lat.close()
    tol = 1e-5 if storage == "f64" else 1e-4
    print("%s %s %s mask: dG %.6g vs %.6g, dtau1 %.6g vs %.6g" % (storage, wall_model, collision,
                                                                   par[0] + par[1], fG, par[2], fT))
    assert abs(par[0] + par[1] - fG) <= tol * abs(fG)
    assert abs(par[2] - fT) <= tol * abs(fT)
    scale = np.abs([fr[q] for q in cells]).max()
    for c in cells:
        assert abs(d1[c] - fr[c]) <= tol * scale, (c, d1[c], fr[c])
    assert np.all(d1[solid == 1] == 0)


GUO_CASES = [
    ("bgk_walls", dict(periodic=(1, 1, 0), collision="bgk", rho_s=(0.03, 0.0)), None),
    ("reg_walls", dict(periodic=(1, 1, 0), collision="regularized", rho_s=(0.03, 0.0)), None),
    ("reg3_walls", dict(periodic=(1, 1, 0), collision="regularized3", rho_s=(0.03, 0.0)), None),
    ("reg_mask_mirror", dict(collision="regularized", rho_s=(0.03, 0.1)), "mask"),
]


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("name,kw,geom", GUO_CASES, ids=[c[0] for c in GUO_CASES])
def test_adjoint_guo_forcing(gpu_lib, name, kw, geom, storage):
    """Reverse pass under Guo's forcing (the second reading of the Sec. 2
    forcing term: f^eq at the common u* = u + (F^1 + F^2)/(2 rho), forcing
    term with F^a = rho^a g^a) through z walls or a mask, g_ext and unequal
    tau, against the oracle's central differences (FP64 1e-5, FP32 1e-4).
    The step is h = 1e-4: at h = 1e-3 the oracle's difference in tau_1 is
    1.1e-4 (relative) from its limit in the BGK case."""
    shape = (6, 5, 7)
    r1, r2, _ = wl.random_state(shape, seed=17, u_max=0.0)
    tgt = np.roll(r1, 2, axis=2)
    kw = dict(kw, g_ext=(2e-4, -1e-4, 3e-4), forcing="guo")
    solid = _staircase(shape, seed=4) if geom == "mask" else None
    G, t1, t2, steps = -1.3, 0.8, 1.2, 6
    rng = np.random.default_rng(3)
    pool = [tuple(int(v) for v in c) for c in np.argwhere(solid == 0)] if solid is not None else \
        [tuple(int(v) for v in c) for c in np.ndindex(shape)]
    cells = [pool[k] for k in rng.choice(len(pool), 12, replace=False)]
    extra = {"solid": solid} if solid is not None else {}
    fG, fT, fr = fd_grads(r1, r2, tgt, G, t1, t2, steps, cells=cells, h=1e-4, **kw, **extra)
    from paper_1601_01237_gb300 import Lattice
    lat = Lattice(shape, storage=storage, tau=(t1, t2), G12=G, G21=G, **kw)
    if solid is not None:
        lat.set_solid(solid)
    lat.init_fields(r1, r2)
    lat.record(steps, 4)
    a, _, _ = lat.moments()
    d1 = np.empty(shape)
    par = lat.adjoint(2 * (a - tgt), None, d1, None)
    lat.close()
    tol = 1e-5 if storage == "f64" else 1e-4
    print("%s %s Guo: dG %.8g vs %.8g, dtau1 %.8g vs %.8g" % (storage, name, par[0] + par[1], fG, par[2], fT))
    assert abs(par[0] + par[1] - fG) <= tol * abs(fG)
    assert abs(par[2] - fT) <= tol * abs(fT)
    scale = np.abs([fr[q] for q in cells]).max()
    for c in cells:
        assert abs(d1[c] - fr[c]) <= tol * scale, (c, d1[c], fr[c])


def test_autograd_rollout_matches_adjoint(gpu_lib):
    """torch.autograd through LBMRollout equals the direct lbm_adjoint call."""
    import torch
    from paper_1601_01237_gb300.adjoint import LBMRollout
    r1, r2, tgt = crop_case()
    G = G_STRONG
    gG, gT, gr = gpu_grads(r1, r2, tgt, G, 1.0, 1.0, STEPS, "f64")
    x1 = torch.tensor(r1, device="cuda", requires_grad=True)
    x2 = torch.tensor(r2, device="cuda", requires_grad=True)
    Gt = torch.tensor(G, dtype=torch.float64, requires_grad=True)
    Tt = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    y1, _ = LBMRollout.apply(x1, x2, Gt, Tt, r1.shape, STEPS, CKPT, {"storage": "f64"})
    loss = ((y1 - torch.tensor(tgt, device="cuda")) ** 2).sum()
    loss.backward()
    assert np.allclose(x1.grad.cpu().numpy(), gr, rtol=1e-12, atol=1e-14)
    assert abs(Gt.grad.item() - gG) <= 1e-12 * abs(gG)
    assert abs(Tt.grad.item() - gT) <= 1e-12 * abs(gT)


def test_adjoint_errors(gpu_lib):
    from paper_1601_01237_gb300 import LBMError, Lattice
    lat = Lattice((4, 4, 4), storage="f32")
    lat.init_fields(np.full((4, 4, 4), 0.5), np.full((4, 4, 4), 0.5))
    with pytest.raises(LBMError, match="EINVAL"):
        lat.adjoint(np.zeros((4, 4, 4)))
    lat.step(2)
    lat.record(3, 1)
    with pytest.raises(LBMError, match="ENOTSUP"):
        lat.adjoint(np.zeros((4, 4, 4)), None, np.empty((4, 4, 4)))
    par = lat.adjoint(np.zeros((4, 4, 4)))
    assert par == [0.0, 0.0, 0.0, 0.0]
    lat.close()


def test_adjoint_repeated_calls_agree(gpu_lib):
    """lbm_record reserves the reverse pass's working memory once; repeated
    lbm_adjoint calls over the same recording reuse it and return the same
    gradients bit for bit."""
    from paper_1601_01237_gb300 import Lattice
    shape = (8, 6, 10)
    r1, r2, _ = wl.random_state(shape, seed=5, u_max=0.0)
    lat = Lattice(shape, storage="f32", tau=(0.9, 1.1), G12=G_STRONG)
    lat.init_fields(r1, r2)
    lat.record(7, 3)
    a, _, _ = lat.moments()
    outs = []
    for _ in range(2):
        d1 = np.empty(shape)
        par = lat.adjoint(2 * (a - r1), None, d1, None)
        outs.append((d1, par))
    lat.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert list(outs[0][1]) == list(outs[1][1])


def test_adjoint_graph_replay_is_bitwise(gpu_lib, monkeypatch):
    """Full checkpoint segments of the reverse pass replay captured CUDA
    graphs; the gradients equal plain launches bit for bit (odd segment
    length, so both ping-pong parities are used, and a ragged segment)."""
    from paper_1601_01237_gb300 import Lattice
    shape = (8, 6, 10)
    r1, r2, _ = wl.random_state(shape, seed=8, u_max=0.0)
    out = {}
    for graphs in ("1", "0"):
        monkeypatch.setenv("LBM_GRAPHS", graphs)
        lat = Lattice(shape, storage="f32", tau=(0.9, 1.1), G12=G_STRONG)
        lat.init_fields(r1, r2)
        lat.record(17, 5)
        a, _, _ = lat.moments()
        d1 = np.empty(shape)
        par = lat.adjoint(2 * (a - r1), None, d1, None)
        lat.close()
        out[graphs] = (d1, list(par))
    assert np.array_equal(out["1"][0], out["0"][0])
    assert out["1"][1] == out["0"][1]


# ---- the differentiation case at full size ---------------------------------
# 96^3, 500 steps, checkpoints every 25: the configuration and launch shapes
# the benchmark times.  The oracle is too slow for finite differences at this
# size, so the check is a property that holds at any size: the reverse pass's
# gradient projected on a direction equals the central difference of the loss
# along it, the loss evaluated by FP64 forward runs of this library (whose
# step the oracle pins on smaller lattices).  Central differences at h = 1e-4
# differ from those at h = 1e-3 by 5.7e-7 (relative, for G), so their
# truncation error is about 6e-9; bars 1e-6 for the FP64 reverse pass and the
# gradient bar 1e-4 for FP32.

def _c3_full():
    c = wl.CONFIGS["c3_adjoint96"]
    r1, r2 = wl.droplet(c["shape"], c["R"])
    tgt, _ = wl.ellipsoid(c["shape"], c["target_axes"])
    delta = wl.uniform_pm1(20260401, int(np.prod(c["shape"]))).reshape(c["shape"])
    return c, r1, r2, tgt, delta


@pytest.fixture(scope="module")
def c3_full_fd():
    from paper_1601_01237_gb300 import Lattice
    c, r1, r2, tgt, delta = _c3_full()
    G, (t1, t2) = c["G"], c["tau"]

    def loss(dr=0.0, dG=0.0, dT=0.0):
        lat = Lattice(c["shape"], storage="f64", tau=(t1 + dT, t2), G12=G + dG, G21=G + dG)
        lat.init_fields(r1 + dr * delta, r2)
        lat.step(c["steps"])
        a, _, _ = lat.moments()
        lat.close()
        return float(((a - tgt) ** 2).sum())

    h = 1e-4
    return ((loss(dG=h) - loss(dG=-h)) / (2 * h), (loss(dT=h) - loss(dT=-h)) / (2 * h),
            (loss(dr=h) - loss(dr=-h)) / (2 * h))


@pytest.mark.parametrize("storage,bar", [("f64", 1e-6), ("f32", 1e-4)])
def test_adjoint_full_size_directional_derivatives(gpu_lib, c3_full_fd, storage, bar):
    from paper_1601_01237_gb300 import Lattice
    c, r1, r2, tgt, delta = _c3_full()
    lat = Lattice(c["shape"], storage=storage, tau=c["tau"], G12=c["G"], G21=c["G"])
    lat.init_fields(r1, r2)
    lat.record(c["steps"], c["ckpt_every"])
    a, _, _ = lat.moments()
    g0 = np.empty(c["shape"])
    par = lat.adjoint(2 * (a - tgt), None, g0, None)
    lat.close()
    got = (par[0] + par[1], par[2], float((g0 * delta).sum()))
    err = [abs(x - y) / abs(y) for x, y in zip(got, c3_full_fd)]
    print("c3 96^3 %s: dL/dG %.3g, dL/dtau1 %.3g, dL/drho1_0 . delta %.3g" % (storage, *err))
    assert max(err) <= bar, (got, c3_full_fd)
