"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
of the equilibrium (Eq. 3) and of the Shan-Chen sum (Eq. 7), lattice isotropy,
conservation laws, exact special cases (uniform states, the quasi-2D
reduction, Poiseuille flow between half-way bounce-back walls), symmetry,
the spinodal threshold and Laplace's law (Eq. 12), and a brute-force
restatement of the interaction sum on a tiny grid.
"""
import numpy as np
import pytest

import oracle
from paper_1601_01237_gb300 import workloads as wl
from _helpers import G_STRONG

T0 = 1.0 / 3.0
RNG = np.random.default_rng(1601)


def test_lattice_isotropy():
    """D3Q19 (Sec. 2): sum w = 1, sum w c = 0, sum w c_a c_b = T0 delta,
    odd third moments vanish, fourth moment T0^2 (dd + dd + dd)."""
    c, w = oracle.lattice()
    assert c.shape == (19, 3)
    assert len({tuple(v) for v in c}) == 19
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2, T0 * np.eye(3), atol=1e-15)
    M3 = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.allclose(M3, 0.0, atol=1e-16)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = T0 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                     + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(M4, iso, atol=1e-15)
    # weights by speed class: 1/3 rest, 1/18 axis, 1/36 diagonal
    m = (c ** 2).sum(1)
    assert np.allclose(w[m == 0], 1 / 3) and np.allclose(w[m == 1], 1 / 18) and np.allclose(w[m == 2], 1 / 36)
    assert (m == 1).sum() == 6 and (m == 2).sum() == 12


def test_quasi2d_weights_reduce_to_d2q9():
    """Summing D3Q19 over c_z gives the D2Q9 weights 4/9, 1/9, 1/36."""
    c, w = oracle.lattice()
    d2 = {}
    for ci, wi in zip(c, w):
        d2[(ci[0], ci[1])] = d2.get((ci[0], ci[1]), 0.0) + wi
    assert len(d2) == 9
    for (x, y), v in d2.items():
        ref = 4 / 9 if x == y == 0 else (1 / 9 if x * x + y * y == 1 else 1 / 36)
        assert abs(v - ref) < 1e-15


@pytest.mark.parametrize("trial", range(5))
def test_feq_moments_closed_form(trial):
    """Eq. 3 on D3Q19: sum f^eq = rho, sum c f^eq = rho u (the third-order
    terms cancel by fourth-order isotropy), sum c c f^eq = rho (T0 I + u u)."""
    c, w = oracle.lattice()
    rho = RNG.uniform(0.05, 2.0)
    u = RNG.uniform(-0.15, 0.15, 3)
    f = oracle.feq(rho, u)
    assert abs(f.sum() - rho) < 1e-14 * rho
    assert np.allclose(c.T @ f, rho * u, atol=1e-15)
    P = np.einsum("ia,ib,i->ab", c, c, f)
    assert np.allclose(P, rho * (T0 * np.eye(3) + np.outer(u, u)), atol=1e-14)
    # direct evaluation of the printed polynomial for one direction
    i = trial + 7
    cu = c[i] @ u
    uu = u @ u
    ref = rho * w[i] * (1 + cu / T0 + cu ** 2 / (2 * T0 ** 2) - uu / (2 * T0) + cu ** 3 / (6 * T0 ** 3)
                        - cu * uu / (2 * T0 ** 2))
    assert abs(f[i] - ref) < 1e-15


def test_feq_rest_state():
    c, w = oracle.lattice()
    assert np.allclose(oracle.feq(0.7, np.zeros(3)), 0.7 * w, rtol=0, atol=1e-16)


@pytest.mark.parametrize("collision", ["bgk", "regularized"])
def test_collision_moments(collision):
    """Post-collision moments of one component (Eqs. 1-2 / 10-11 with the
    exact-difference forcing): mass kept; momentum
      BGK:         j* = j - (j - rho u)/tau + rho g
      regularized: j* = rho (u + g)
    and for the regularized operator the second moment
      P* = rho (T0 I + v v) + (1 - 1/tau) Pi_neq,  v = u + g,
    since the Hermite projection reproduces Pi_neq exactly."""
    c, w = oracle.lattice()
    tau = 0.8
    p = oracle.make_params((1, 1, 1), tau=(tau, tau), collision=collision)
    for _ in range(4):
        rho = RNG.uniform(0.2, 1.5)
        u = RNG.uniform(-0.08, 0.08, 3)
        g = RNG.uniform(-0.01, 0.01, 3)
        fin = oracle.feq(rho, RNG.uniform(-0.08, 0.08, 3)) * (1 + 0.05 * RNG.uniform(-1, 1, 19))
        rho_in = fin.sum()
        j = c.T @ fin
        fp = oracle.collide_cell(p, 0, fin, rho_in, u, g)
        assert abs(fp.sum() - rho_in) < 1e-14
        jp = c.T @ fp
        if collision == "bgk":
            assert np.allclose(jp, j - (j - rho_in * u) / tau + rho_in * g, atol=1e-15)
        else:
            assert np.allclose(jp, rho_in * (u + g), atol=1e-15)
            feq = oracle.feq(rho_in, u)
            Pneq = np.einsum("ia,ib,i->ab", c, c, fin - feq)
            v = u + g
            Pp = np.einsum("ia,ib,i->ab", c, c, fp)
            ref = rho_in * (T0 * np.eye(3) + np.outer(v, v)) + (1 - 1 / tau) * Pneq
            assert np.allclose(Pp, ref, atol=1e-14)


def _hermite_basis(c, w, order):
    """Values on the lattice of the Hermite polynomials of one order (all
    index tuples a <= b <= ...), as rows."""
    import itertools
    d = np.eye(3)
    rows = []
    for idx in itertools.combinations_with_replacement(range(3), order):
        if order == 0:
            rows.append(np.ones(len(w)))
        elif order == 1:
            rows.append(c[:, idx[0]].astype(float))
        elif order == 2:
            a, b = idx
            rows.append(c[:, a] * c[:, b] - T0 * d[a, b])
        else:
            a, b, e = idx
            rows.append(c[:, a] * c[:, b] * c[:, e] - T0 * (c[:, a] * d[b, e] + c[:, b] * d[a, e] + c[:, e] * d[a, b]))
    return np.array(rows, dtype=float)


def test_regularized3_keeps_moments_to_third_order_and_drops_the_rest():
    """Sec. 2: the filter keeps the non-equilibrium moments up to the chosen
    order (second: momentum flux; third: energy flux) and removes the rest.
    On D3Q19 the 19 populations split, in the w-weighted inner product, into
    orders 0 (1), 1 (3), 2 (6), 3 (6: H_xxx, H_yyy, H_zzz and H_xyz vanish on
    the lattice) and a 3-dimensional remainder.  So d = f* - f^eq(u + g) is
    fixed by: no mass or momentum; second and third Hermite moments equal to
    (1 - 1/tau) times those of f - f^eq(u); nothing in the remainder (computed
    here as the w-orthogonal complement of orders 0-3 with an SVD)."""
    c, w = oracle.lattice()
    c = c.astype(float)
    H = [_hermite_basis(c, w, k) for k in range(4)]
    low = np.vstack(H)                                   # 1 + 3 + 6 + 10 rows (4 vanish)
    # complement: h with sum_i w_i h_i H_k(c_i) = 0 for every k
    _, sv, vt = np.linalg.svd(low * w[None, :])
    rank = int((sv > 1e-12).sum())
    assert rank == 16
    comp = vt[rank:]
    assert comp.shape[0] == 3
    tau = 0.73
    p = oracle.make_params((1, 1, 1), tau=(tau, tau), collision="regularized3")
    for _ in range(4):
        u = RNG.uniform(-0.08, 0.08, 3)
        g = RNG.uniform(-0.01, 0.01, 3)
        fin = oracle.feq(RNG.uniform(0.2, 1.5), RNG.uniform(-0.08, 0.08, 3)) * (1 + 0.05 * RNG.uniform(-1, 1, 19))
        rho = fin.sum()
        fp = oracle.collide_cell(p, 0, fin, rho, u, g)
        d = fp - oracle.feq(rho, u + g)
        neq = fin - oracle.feq(rho, u)
        assert abs(d.sum()) < 1e-15
        assert np.allclose(c.T @ d, 0.0, atol=1e-15)
        assert np.allclose(H[2] @ d, (1 - 1 / tau) * (H[2] @ neq), atol=1e-15)
        assert np.allclose(H[3] @ d, (1 - 1 / tau) * (H[3] @ neq), atol=1e-15)
        assert np.allclose(comp @ d, 0.0, atol=1e-15)
        # the remainder of the input is not zero: the test has something to drop
        assert np.abs(comp @ neq).max() > 1e-5
        # and the third-order part is really kept: the second-order filter differs
        p2 = oracle.make_params((1, 1, 1), tau=(tau, tau), collision="regularized")
        d2 = oracle.collide_cell(p2, 0, fin, rho, u, g) - oracle.feq(rho, u + g)
        assert np.allclose(H[3] @ d2, 0.0, atol=1e-15)
        assert np.abs(H[3] @ neq).max() > 1e-5


def test_regularized_equals_bgk_at_tau_one_and_for_hermite_states():
    """At tau = 1 both operators return f^eq(u + g); for a population whose
    non-equilibrium part is a pure second-order Hermite term they agree at any tau."""
    c, w = oracle.lattice()
    rho, u, g = 0.9, np.array([0.02, -0.03, 0.01]), np.array([1e-3, 2e-3, -1e-3])
    fin = oracle.feq(rho, u) * (1 + 0.03 * RNG.uniform(-1, 1, 19))
    rho = fin.sum()
    pb = oracle.make_params((1, 1, 1), tau=(1.0, 1.0), collision="bgk")
    pr = oracle.make_params((1, 1, 1), tau=(1.0, 1.0), collision="regularized")
    a = oracle.collide_cell(pb, 0, fin, rho, u, g)
    b = oracle.collide_cell(pr, 0, fin, rho, u, g)
    assert np.allclose(a, oracle.feq(rho, u + g), atol=1e-16)
    assert np.allclose(b, a, atol=1e-16)
    Pi = np.array([[1e-3, 2e-4, 0], [2e-4, -5e-4, 1e-4], [0, 1e-4, 3e-4]])
    Qi = np.einsum("ia,ib->iab", c, c) - T0 * np.eye(3)
    fneq = w / (2 * T0 ** 2) * np.einsum("iab,ab->i", Qi, Pi)
    fin = oracle.feq(rho, u) + fneq
    pb = oracle.make_params((1, 1, 1), tau=(0.7, 0.7), collision="bgk")
    pr = oracle.make_params((1, 1, 1), tau=(0.7, 0.7), collision="regularized")
    assert np.allclose(oracle.collide_cell(pb, 0, fin, rho, u, g), oracle.collide_cell(pr, 0, fin, rho, u, g),
                       atol=1e-15)
    # third order: tau = 1 gives f^eq(u + g); a non-equilibrium part made of
    # second- and third-order Hermite terms passes the filter unchanged
    p3 = oracle.make_params((1, 1, 1), tau=(1.0, 1.0), collision="regularized3")
    assert np.allclose(oracle.collide_cell(p3, 0, fin, rho, u, g), oracle.feq(rho, u + g), atol=1e-16)
    H3 = _hermite_basis(c.astype(float), w, 3)
    fin3 = fin + w * (np.array([2e-3, -1e-3, 5e-4, 1e-3, 0, -2e-3, 7e-4, 3e-4, -6e-4, 1e-3]) @ H3)
    p3 = oracle.make_params((1, 1, 1), tau=(0.7, 0.7), collision="regularized3")
    assert np.allclose(oracle.collide_cell(pb, 0, fin3, rho, u, g), oracle.collide_cell(p3, 0, fin3, rho, u, g),
                       atol=1e-15)
    assert not np.allclose(oracle.collide_cell(pr, 0, fin3, rho, u, g), oracle.collide_cell(p3, 0, fin3, rho, u, g),
                           atol=1e-6)


def test_sc_sum_sinusoid_closed_form():
    """Eq. 7 sum for rho = A + B sin(k x + phi), periodic:
    S_x = (B/3) sin(k) cos(k x + phi), S_y = S_z = 0 (the six c_x = +1 links
    weigh 1/18 + 4/36 = 1/6 in total)."""
    nx, ny, nz = 24, 5, 4
    A, B, phi = 0.8, 0.15, 0.3
    k = 2 * np.pi * 3 / nx
    x = np.arange(nx)
    rho = np.broadcast_to(A + B * np.sin(k * x + phi), (nz, ny, nx)).copy()
    p = oracle.make_params((nz, ny, nx))
    sf, sw = oracle.interaction_sums(p, rho)
    ref = (B / 3) * np.sin(k) * np.cos(k * x + phi)
    assert np.allclose(sf[..., 0], ref[None, None, :], atol=1e-15)
    assert np.allclose(sf[..., 1:], 0.0, atol=1e-15)
    assert np.all(sw == 0.0)
    # the same along z and y (operands transposed)
    rz = np.broadcast_to((A + B * np.sin(k * np.arange(24) + phi))[:, None, None], (24, 5, 4)).copy()
    pz = oracle.make_params((24, 5, 4))
    sfz, _ = oracle.interaction_sums(pz, rz)
    assert np.allclose(sfz[..., 2], ((B / 3) * np.sin(k) * np.cos(k * np.arange(24) + phi))[:, None, None],
                       atol=1e-15)
    assert np.allclose(sfz[..., :2], 0.0, atol=1e-15)


def test_sc_sum_brute_force_tiny():
    """Brute-force restatement of the Eq. 7 sum on a random 4x3x5 periodic
    field: explicit neighbour loops in Python over the 18 moving links."""
    shape = (4, 3, 5)
    rho = RNG.uniform(0.1, 1.0, shape)
    p = oracle.make_params(shape)
    sf, _ = oracle.interaction_sums(p, rho)
    nz, ny, nx = shape
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                s = np.zeros(3)
                for dz in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            m = dx * dx + dy * dy + dz * dz
                            if m == 0 or m == 3:
                                continue
                            wgt = 1 / 18 if m == 1 else 1 / 36
                            s += wgt * np.array([dx, dy, dz]) * rho[(z + dz) % nz, (y + dy) % ny, (x + dx) % nx]
                assert np.allclose(sf[z, y, x], s, atol=1e-15)


def test_wall_density_mirror_and_potential():
    """Eq. 13: with walls along z, a solid neighbour presents the mirrored
    density plus rho_s (modified model) or rho_s alone (wall potential).
    A field that is uniform along z then gives zero normal force with the
    mirror model and rho_s = 0 (zero normal derivative)."""
    shape = (4, 3, 5)
    rho = np.broadcast_to(RNG.uniform(0.2, 1.0, (1, 3, 5)), shape).copy()
    pm = oracle.make_params(shape, periodic=(1, 1, 0), wall_model="mirror")
    sf, sw = oracle.interaction_sums(pm, rho, 0.0)
    tot = sf + sw
    assert np.allclose(tot[..., 2], 0.0, atol=1e-15)
    pp = oracle.make_params(shape, periodic=(1, 1, 1))
    sfp, _ = oracle.interaction_sums(pp, rho)
    assert np.allclose(tot, sfp, atol=1e-15)
    # point-wise potential rho_s at the solid sites: bottom layer feels
    # -sum_{c_z=-1} w = -1/6 times rho_s below, top layer +1/6 rho_s above
    rs = 0.3
    pw = oracle.make_params(shape, periodic=(1, 1, 0), wall_model="potential")
    _, sw = oracle.interaction_sums(pw, rho, rs)
    assert np.allclose(sw[0, ..., 2], -rs / 6, atol=1e-15)
    assert np.allclose(sw[-1, ..., 2], rs / 6, atol=1e-15)
    assert np.allclose(sw[1:-1], 0.0)


def _run(shape, r1, r2, nsteps, u=None, **kw):
    p = oracle.make_params(shape, **kw)
    f = oracle.init(p, r1, r2, u)
    oracle.step(p, f, nsteps)
    return p, f


def test_uniform_state_is_fixed_point():
    shape = (3, 4, 5)
    r1 = np.full(shape, 0.7)
    r2 = np.full(shape, 0.2)
    p, f = _run(shape, r1, r2, 10, G12=-2.7)
    a, b, uF = oracle.moments(p, f)
    assert np.allclose(a, 0.7, rtol=1e-15, atol=0) and np.allclose(b, 0.2, rtol=1e-15, atol=0)
    assert np.abs(uF).max() < 1e-16


def test_uniform_flow_is_galilean():
    """Uniform densities moving with uniform u stay exactly uniform (every cell
    identical) and keep u."""
    shape = (2, 3, 4)
    u0 = np.array([0.05, -0.02, 0.03])
    u = np.broadcast_to(u0, shape + (3,)).copy()
    p, f = _run(shape, np.full(shape, 0.6), np.full(shape, 0.4), 20, u=u, G12=-2.7, tau=(0.8, 0.8))
    a, b, uF = oracle.moments(p, f)
    assert np.allclose(uF, u0, atol=1e-15)
    assert np.allclose(a, 0.6, atol=1e-14) and np.allclose(b, 0.4, atol=1e-14)


@pytest.mark.parametrize("collision,tau", [("bgk", (0.8, 0.8)), ("regularized", (0.6, 1.3)),
                                           ("regularized3", (0.6, 1.3))])
def test_mass_and_momentum_conservation(collision, tau):
    """Periodic lattice, symmetric G: each component's mass is conserved and so
    is the total momentum sum_x sum_a j^a, since the pairwise Shan-Chen forces
    cancel (sum over x of rho^1 S^2 + rho^2 S^1 = 0) and the collision keeps
    momentum (equal tau for BGK; any tau for the regularized operator)."""
    shape = (6, 5, 7)
    r1, r2, u = wl.random_state(shape, seed=3, u_max=0.03)
    p = oracle.make_params(shape, tau=tau, G12=-1.5, collision=collision)
    f = oracle.init(p, r1, r2, u)
    a0, b0, uu0 = oracle.moments_raw(p, f)
    J0 = ((a0 + b0)[..., None] * uu0).sum(axis=(0, 1, 2))
    oracle.step(p, f, 200)
    a, b, uu = oracle.moments_raw(p, f)
    J = ((a + b)[..., None] * uu).sum(axis=(0, 1, 2))
    assert abs(a.sum() - a0.sum()) < 1e-13 * a0.sum()
    assert abs(b.sum() - b0.sum()) < 1e-13 * b0.sum()
    assert np.allclose(J, J0, atol=1e-13 * (a0.sum() + b0.sum()))


def test_quasi2d_nz1_equals_nz2():
    """A field uniform along z evolves identically on nz = 1 and nz = 2."""
    r1, r2 = wl.droplet((1, 24, 24), 6)
    pa, fa = _run((1, 24, 24), r1, r2, 60, G12=-2.7)
    r1b = np.concatenate([r1, r1]); r2b = np.concatenate([r2, r2])
    pb, fb = _run((2, 24, 24), r1b, r2b, 60, G12=-2.7)
    a1, a2, au = oracle.moments(pa, fa)
    b1, b2, bu = oracle.moments(pb, fb)
    assert np.allclose(b1[0], a1[0], atol=1e-14) and np.allclose(b1[1], a1[0], atol=1e-14)
    assert np.allclose(bu[0], au[0], atol=1e-14)
    assert np.abs(bu[..., 2]).max() < 1e-15


def test_droplet_symmetry():
    """A centred droplet keeps the lattice symmetries x <-> y and x -> n-1-x."""
    shape = (1, 20, 20)
    r1, r2 = wl.droplet(shape, 5)
    p, f = _run(shape, r1, r2, 100, G12=-2.7, tau=(0.7, 1.2))
    a, b, uF = oracle.moments(p, f)
    assert np.allclose(a[0], a[0].T, atol=1e-12)
    assert np.allclose(a[0], a[0][:, ::-1], atol=1e-12)
    assert np.allclose(uF[0, :, :, 0], -uF[0, :, ::-1, 0], atol=1e-12)


@pytest.mark.parametrize("tau", [0.7, 2.0])
def test_spinodal_threshold(tau):
    """Linear stability of the uniform mixture rho^1 = rho^2 = rho0 under the
    Eq. 7 force with the exact-difference forcing and BGK: to first order in
    the gradients the flux of component a relative to the mixture is
    tau F^a - (tau - 1/2) T0 grad rho^a, with F^1 = -G T0 rho0 grad(delta)
    for delta = rho^1 - rho0 = rho0 - rho^2.  The long-wave mode therefore
    grows iff |G| rho0 > 1 - 1/(2 tau) (the continuum criterion |G| rho0 > 1
    is recovered as tau -> infinity).  Checked 10 % either side."""
    n, m, eps, rho0 = 48, 1, 1e-4, 0.5
    x = np.arange(n)
    k = 2 * np.pi * m / n
    r1 = (rho0 * (1 + eps * np.cos(k * x)))[None, None, :]
    r2 = (rho0 * (1 - eps * np.cos(k * x)))[None, None, :]
    thr = (1 - 1 / (2 * tau)) / rho0
    amp = {}
    for fac in (0.9, 1.1):
        p, f = _run(r1.shape, r1, r2, 600, G12=-fac * thr, tau=(tau, tau))
        a, b, _ = oracle.moments(p, f)
        amp[fac] = np.abs(np.fft.rfft((a - b)[0, 0]))[m] / (n / 2) / (2 * rho0 * eps)
    assert amp[0.9] < 0.97
    assert amp[1.1] > 1.03


def test_poiseuille_half_way_bounce_back():
    """Single fluid (G = 0, both components alike) driven by g_ext along x
    between half-way bounce-back walls at z = -1/2 and H - 1/2.  The velocity
    u_F (Eq. 8) is the parabola g/(2 nu) z'(H - z'), z' = z + 1/2,
    nu = T0 (tau - 1/2), up to a uniform slip that vanishes for BGK at
    tau = 1/2 + sqrt(3/16) (the known bounce-back result); at any tau the
    second difference is the exact curvature -g/nu (momentum balance)."""
    H, g = 8, 1e-5
    for tau in (0.5 + np.sqrt(3 / 16), 1.4):
        shape = (H, 1, 2)
        r = np.full(shape, 0.5)
        p, f = _run(shape, r, r, 6000, G12=0.0, tau=(tau, tau), g_ext=(g, 0, 0), periodic=(1, 1, 0))
        _, _, uF = oracle.moments(p, f)
        ux = uF[:, 0, 0, 0]
        nu = T0 * (tau - 0.5)
        zp = np.arange(H) + 0.5
        exact = g / (2 * nu) * zp * (H - zp)
        d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
        assert np.allclose(d2, -g / nu, rtol=1e-8, atol=0)
        assert np.abs(uF[..., 1:]).max() < 1e-14
        if tau < 1:
            assert np.max(np.abs(ux - exact)) < 1e-9 * exact.max()
        else:
            slip = ux - exact
            assert np.ptp(slip) < 1e-9 * exact.max() and abs(slip[0]) > 1e-3 * exact.max()


@pytest.mark.slow
def test_laplace_law_2d():
    """Young-Laplace (Eq. 12): a static 2D droplet's pressure jump is linear
    in 1/R through the origin.  p = T0 rho - G T0 rho^1 rho^2 is the bulk
    pressure of the Eq. 7 force (sum_a F^{ab} -> G T0 grad(rho^1 rho^2)); R is
    the measured equivalent-area radius of the relaxed droplet."""
    G = G_STRONG
    n = 48
    Rs, dps = [], []
    for R0 in (6, 8, 10, 12):
        shape = (1, n, n)
        r1, r2 = wl.droplet(shape, R0)
        p, f = _run(shape, r1, r2, 2000, G12=G)
        a, b, _ = oracle.moments(p, f)
        pr = T0 * (a + b) - G * T0 * a * b
        c = (n - 1) / 2
        yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        r = np.hypot(xx - c, yy - c)
        dps.append(pr[0][r < R0 / 2].mean() - pr[0][r > R0 + 8].mean())
        Rs.append(np.sqrt((a > 0.5 * (a.max() + a.min())).sum() / np.pi))
    R = np.array(Rs)
    dp = np.array(dps)
    sig = dp * R
    assert np.ptp(sig) < 0.05 * sig.mean()
    A = np.vstack([1 / R, np.ones_like(R)]).T
    (sigma, icpt), *_ = np.linalg.lstsq(A, dp, rcond=None)
    assert sigma > 0
    assert abs(icpt) < 0.05 * dp.min()


# ---------------------------------------------------------------------------
# Staircase walls (a mask of solid sites; the inclined walls of Sec. 4.2)

def _layered_state(nz_fluid, ny, nx, seed):
    """Densities and velocities that vary along z only."""
    rng = np.random.default_rng(seed)
    r1 = np.broadcast_to(rng.uniform(0.2, 1.0, nz_fluid)[:, None, None], (nz_fluid, ny, nx)).copy()
    r2 = np.broadcast_to(rng.uniform(0.2, 1.0, nz_fluid)[:, None, None], (nz_fluid, ny, nx)).copy()
    u = np.zeros((nz_fluid, ny, nx, 3))
    u[..., 0] = rng.uniform(-0.03, 0.03, nz_fluid)[:, None, None]
    u[..., 2] = rng.uniform(-0.02, 0.02, nz_fluid)[:, None, None]
    u[0, ..., 2] = 0.0
    u[-1, ..., 2] = 0.0
    return r1, r2, u


@pytest.mark.parametrize("wall_model,rho_s", [("mirror", (0.0, 0.0)), ("mirror", (0.04, 0.1)),
                                              ("potential", (0.0, 0.15))])
def test_mask_planes_equal_flat_walls_for_layered_states(wall_model, rho_s):
    """Two solid planes of the mask around nz fluid layers (periodic lattice of
    nz + 2 layers) against the flat half-way walls of the non-periodic
    lattice: the same bounce-back links, and for fields that vary along the
    wall normal only the w-weighted mean over a solid site's fluid neighbours
    equals the mirrored density, so every fluid population agrees over 40
    steps (forces, walls, wetting potential)."""
    nz, ny, nx = 5, 3, 4
    r1, r2, u = _layered_state(nz, ny, nx, seed=7)
    kw = dict(tau=(0.8, 1.1), G12=-1.4, rho_s=rho_s, wall_model=wall_model, g_ext=(2e-4, 0.0, -1e-4))
    pf = oracle.make_params((nz, ny, nx), periodic=(1, 1, 0), **kw)
    ff = oracle.init(pf, r1, r2, u)
    oracle.step(pf, ff, 40)
    solid = np.zeros((nz + 2, ny, nx), np.uint8)
    solid[0] = solid[-1] = 1
    pad = lambda a, v: np.concatenate([np.full((1,) + a.shape[1:], v), a, np.full((1,) + a.shape[1:], v)])
    pm = oracle.make_params((nz + 2, ny, nx), periodic=(1, 1, 1), solid=solid, **kw)
    fm = oracle.init(pm, pad(r1, 1.0), pad(r2, 1.0), pad(u, 0.0))
    assert np.all(fm[:, :, 0] == 0) and np.all(fm[:, :, -1] == 0)
    oracle.step(pm, fm, 40)
    assert np.all(fm[:, :, 0] == 0) and np.all(fm[:, :, -1] == 0)
    assert np.max(np.abs(fm[:, :, 1:-1] - ff)) < 1e-13
    # and the same walls across x instead of z (transposed lattice)
    pfx = oracle.make_params((ny, nx, nz), periodic=(0, 1, 1), **dict(kw, g_ext=(-1e-4, 0.0, 2e-4)))
    tr = lambda a: np.ascontiguousarray(np.moveaxis(a, 0, 2))
    ux = np.ascontiguousarray(tr(u)[..., ::-1])
    ffx = oracle.init(pfx, tr(r1), tr(r2), ux)
    oracle.step(pfx, ffx, 40)
    a_f, b_f, _ = oracle.moments_raw(pf, ff)
    a_x, b_x, _ = oracle.moments_raw(pfx, ffx)
    assert np.max(np.abs(tr(a_f) - a_x)) < 1e-13 and np.max(np.abs(tr(b_f) - b_x)) < 1e-13


def _staircase(shape, seed):
    """A blob-and-step mask: a staircase wall along the bottom and a few
    solid sites scattered inside."""
    nz, ny, nx = shape
    m = np.zeros(shape, np.uint8)
    for x in range(nx):
        m[: 1 + (x * 3) // nx, :, x] = 1
    rng = np.random.default_rng(seed)
    for _ in range(3):
        m[rng.integers(2, nz), rng.integers(0, ny), rng.integers(0, nx)] = 1
    return m


@pytest.mark.parametrize("collision", ["bgk", "regularized"])
def test_mask_conserves_mass(collision):
    """Half-way bounce-back returns every population that meets a solid site
    to its cell: each component's mass is conserved, and solid sites stay
    empty."""
    shape = (7, 4, 9)
    solid = _staircase(shape, seed=2)
    r1, r2, u = wl.random_state(shape, seed=8, u_max=0.03)
    p = oracle.make_params(shape, tau=(0.7, 1.2), G12=-1.3, collision=collision, solid=solid, rho_s=(0.0, 0.05))
    f = oracle.init(p, r1, r2, u)
    a0, b0, _ = oracle.moments_raw(p, f)
    oracle.step(p, f, 150)
    a, b, uu = oracle.moments_raw(p, f)
    assert abs(a.sum() - a0.sum()) < 1e-12 * a0.sum() and abs(b.sum() - b0.sum()) < 1e-12 * b0.sum()
    assert np.all(a[solid == 1] == 0) and np.all(f[:, :, solid == 1] == 0)
    assert np.all(np.isfinite(uu))


def test_mask_uniform_rest_state_is_fixed_point():
    """Modified model, rho_s = 0: next to walls of any shape a uniform fluid at
    rest feels no wall force (each solid site presents the fluid's own
    density, so the interaction sums cancel) and bounce-back returns the rest
    equilibrium: the state does not change."""
    shape = (6, 3, 8)
    solid = _staircase(shape, seed=5)
    r1 = np.full(shape, 0.7)
    r2 = np.full(shape, 0.3)
    p = oracle.make_params(shape, tau=(0.9, 0.9), G12=-1.5, solid=solid, periodic=(1, 1, 0))
    f = oracle.init(p, r1, r2)
    f0 = f.copy()
    oracle.step(p, f, 30)
    assert np.max(np.abs(f - f0)) < 1e-15


def test_mask_mirror_symmetry():
    """A mask and state symmetric under x -> nx - 1 - x stay symmetric (with
    mirrored x velocities): checks the direction bookkeeping of bounce-back
    and of the solid-site densities on a staircase."""
    nz, ny, nx = 8, 1, 10
    m = np.zeros((nz, ny, nx), np.uint8)
    for x in range(nx // 2):
        m[: 1 + x // 2, :, x] = 1
        m[: 1 + x // 2, :, nx - 1 - x] = 1
    r1, r2 = wl.droplet((nz, ny, nx), 3.0, center=(4.0, 0.0, (nx - 1) / 2.0))
    p = oracle.make_params((nz, ny, nx), tau=(0.8, 0.8), G12=G_STRONG, solid=m, periodic=(1, 1, 0),
                           rho_s=(0.0, 0.08))
    f = oracle.init(p, r1, r2)
    oracle.step(p, f, 60)
    a, b, uu = oracle.moments_raw(p, f)
    assert np.max(np.abs(a - a[..., ::-1])) < 1e-13
    assert np.max(np.abs(uu[..., 0] + uu[..., ::-1, 0])) < 1e-13
    assert np.max(np.abs(uu[..., 2] - uu[..., ::-1, 2])) < 1e-13
    assert np.abs(uu).max() > 1e-5


def test_isolated_solid_site_presents_the_linear_field():
    """A solid site with only fluid neighbours, in a density field linear in
    x, y, z: the w-weighted mean over all 18 neighbours is the field's value
    at the site (the weights are symmetric), so next to it the interaction
    sum is that of the unbroken linear field, T0 grad(rho), and the wall part
    is w_i c_i rho(site).  A neighbour dropped from the mean or a wrong
    direction breaks both."""
    c, w = oracle.lattice()
    n = 9
    shape = (n, n, n)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    grad = np.array([0.01, -0.02, 0.03])
    rho = 0.5 + grad[0] * x + grad[1] * y + grad[2] * z
    solid = np.zeros(shape, np.uint8)
    s = (4, 4, 4)                      # (z, y, x)
    solid[s] = 1
    p = oracle.make_params(shape, solid=solid)
    Sf, Sw = oracle.interaction_sums(p, rho)
    for i in range(19):
        if not c[i].any():
            continue
        xz = (s[0] - c[i][2], s[1] - c[i][1], s[2] - c[i][0])    # the fluid cell that sees s along c_i
        tot = Sf[xz] + Sw[xz]
        assert np.allclose(tot, T0 * grad, atol=1e-15)
        assert np.allclose(Sw[xz], w[i] * c[i] * rho[s], atol=1e-15)


# ---------------------------------------------------------------------------
# The second forcing reading: Guo, Zheng & Shi (2002), one common equilibrium
# velocity u* = u + g/2 (Eqs. 8-9).

def _guo_term(c, w, u, F):
    """w_i [(c_i - u)/T0 + (c_i.u) c_i / T0^2] . F, written out per direction."""
    out = np.zeros(19)
    for i in range(19):
        cu = c[i] @ u
        out[i] = w[i] * sum(((c[i, k] - u[k]) / T0 + cu * c[i, k] / T0 ** 2) * F[k] for k in range(3))
    return out


@pytest.mark.parametrize("collision", ["bgk", "regularized", "regularized3"])
def test_guo_collision_moments(collision):
    """Post-collision moments of one component with Guo's forcing (F = rho g):
      mass kept;
      BGK:          j* = j - (j - rho u*)/tau + (1 - 1/(2 tau)) F,
      regularized:  j* = rho u* + F/2 (the first-order non-equilibrium part is
                    filtered out, as without forcing);
    and the forcing term's own moments 0, F, u* F + F u* (its second moment),
    so that the regularized second moment is
      rho (T0 I + u* u*) + (1 - 1/tau) (Pi_neq + (u* F + F u*)/2) + (u* F + F u*)/2,
    Pi_neq = sum c c (f - f^eq(u*)).  At tau = 1 both operators give
    f^eq(u*) + F_i/2."""
    c, w = oracle.lattice()
    for tau in (0.55, 0.8, 1.0, 2.5):
        p = oracle.make_params((1, 1, 1), tau=(tau, tau), collision=collision, forcing="guo")
        for _ in range(3):
            rho = RNG.uniform(0.05, 1.5)
            u = RNG.uniform(-0.08, 0.08, 3)
            g = RNG.uniform(-0.05, 0.05, 3)
            fin = oracle.feq(rho, RNG.uniform(-0.08, 0.08, 3)) * (1 + 0.05 * RNG.uniform(-1, 1, 19))
            r = fin.sum()
            j = c.T @ fin
            F = r * g
            Fi = _guo_term(c, w, u, F)
            assert abs(Fi.sum()) < 1e-15
            assert np.allclose(c.T @ Fi, F, atol=1e-15)
            assert np.allclose(np.einsum("ia,ib,i->ab", c, c, Fi), np.outer(u, F) + np.outer(F, u), atol=1e-15)
            fp = oracle.collide_cell(p, 0, fin, r, u, g)
            assert abs(fp.sum() - r) < 1e-14
            jp = c.T @ fp
            if collision == "bgk":
                assert np.allclose(jp, j - (j - r * u) / tau + (1 - 1 / (2 * tau)) * F, atol=1e-15)
            else:
                assert np.allclose(jp, r * u + F / 2, atol=1e-15)
                feq = oracle.feq(r, u)
                Pneq = np.einsum("ia,ib,i->ab", c, c, fin - feq)
                S = np.outer(u, F) + np.outer(F, u)
                ref = r * (T0 * np.eye(3) + np.outer(u, u)) + (1 - 1 / tau) * (Pneq + S / 2) + S / 2
                assert np.allclose(np.einsum("ia,ib,i->ab", c, c, fp), ref, atol=1e-14)
            if tau == 1.0:
                assert np.allclose(fp, oracle.feq(r, u) + Fi / 2, atol=1e-15)


@pytest.mark.parametrize("collision,tau", [("bgk", 0.7), ("bgk", 2.0), ("regularized", 0.6)])
def test_guo_spinodal_threshold_is_tau_independent(collision, tau):
    """With Guo's forcing the force and the density gradient enter the flux
    of a component relative to the mixture with the same factor (tau - 1/2),
    so the long-wave mode of the uniform mixture rho^1 = rho^2 = rho0 grows
    iff |G| rho0 > 1, the continuum criterion, at every tau (the
    exact-difference forcing gives 1 - 1/(2 tau) instead).  Checked 10 %
    either side of |G| = 1/rho0."""
    n, m, eps, rho0 = 48, 1, 1e-4, 0.5
    x = np.arange(n)
    k = 2 * np.pi * m / n
    r1 = (rho0 * (1 + eps * np.cos(k * x)))[None, None, :]
    r2 = (rho0 * (1 - eps * np.cos(k * x)))[None, None, :]
    amp = {}
    for fac in (0.9, 1.1):
        p, f = _run(r1.shape, r1, r2, 600, G12=-fac / rho0, tau=(tau, tau), collision=collision, forcing="guo")
        a, b, _ = oracle.moments(p, f)
        amp[fac] = np.abs(np.fft.rfft((a - b)[0, 0]))[m] / (n / 2) / (2 * rho0 * eps)
    assert amp[0.9] < 0.97
    assert amp[1.1] > 1.03


@pytest.mark.parametrize("collision", ["bgk", "regularized"])
def test_guo_conservation_and_fixed_point(collision):
    """Guo's forcing keeps each component's mass and, under periodic walls
    with symmetric G and equal tau (BGK) or any tau (regularized), the total
    momentum (the pairwise Eq. 7 forces sum to zero); a uniform state at rest
    stays bitwise fixed."""
    shape = (5, 6, 7)
    r1, r2, u = wl.random_state(shape, seed=8, u_max=0.03)
    tau = (0.8, 0.8) if collision == "bgk" else (0.6, 1.3)
    p, f = _run(shape, r1, r2, 0, u=u, G12=-1.3, tau=tau, collision=collision, forcing="guo")
    a0, b0, uF0 = oracle.moments(p, f)
    mom0 = (((a0 + b0)[..., None]) * uF0).sum((0, 1, 2))
    oracle.step(p, f, 300)
    a, b, uF = oracle.moments(p, f)
    assert abs(a.sum() - a0.sum()) < 1e-13 * a0.sum() and abs(b.sum() - b0.sum()) < 1e-13 * b0.sum()
    mom = (((a + b)[..., None]) * uF).sum((0, 1, 2))
    assert np.max(np.abs(mom - mom0)) < 1e-12 * (a0 + b0).sum()
    r = np.full(shape, 0.4)
    p, f = _run(shape, r, r, 0, G12=-1.3, collision=collision, forcing="guo")
    f0 = f.copy()
    oracle.step(p, f, 3)
    assert np.array_equal(f, f0)


def test_guo_poiseuille_curvature():
    """Single fluid driven by g_ext between half-way walls with Guo's
    forcing: the second difference of u_F is the exact curvature -g/nu,
    nu = T0 (tau - 1/2), at any tau (BGK and regularized)."""
    H, g = 8, 1e-5
    for collision in ("bgk", "regularized"):
        for tau in (0.6, 1.4):
            shape = (H, 1, 2)
            r = np.full(shape, 0.5)
            p, f = _run(shape, r, r, 6000, G12=0.0, tau=(tau, tau), g_ext=(g, 0, 0), periodic=(1, 1, 0),
                        collision=collision, forcing="guo")
            _, _, uF = oracle.moments(p, f)
            ux = uF[:, 0, 0, 0]
            nu = T0 * (tau - 0.5)
            d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
            assert np.allclose(d2, -g / nu, rtol=1e-8, atol=0), (collision, tau, d2 / (-g / nu))
            assert np.abs(uF[..., 1:]).max() < 1e-14
