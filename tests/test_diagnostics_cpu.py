"""Host-side measurement helpers against fields whose answer is known by
construction: circular caps and slug menisci of a given contact angle, drawn
as tanh profiles around exact circles (the contact-angle measurement of
Sec. 4.2 fits a circle to the interface)."""
import math

import numpy as np
import pytest

from paper_1601_01237_gb300 import diagnostics as dg
from paper_1601_01237_gb300 import workloads as wl

W = 2.0
HI, LO = 1.0, 0.03
THR = 0.5 * (HI + LO)


def _profile(d):
    """Density rising from LO to HI across d = 0 (tanh, width W)."""
    return LO + 0.5 * (HI - LO) * (1.0 + np.tanh(d / W))


def _cap(theta_deg, Rc, shape=(64, 1, 160)):
    """Droplet whose boundary is the circle of radius Rc meeting the wall
    z = -1/2 at theta (inside the droplet): centre height -1/2 - Rc cos theta."""
    nz, _, nx = shape
    zc = -0.5 - Rc * math.cos(math.radians(theta_deg))
    z, x = np.meshgrid(np.arange(nz, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    r = np.hypot(x - (nx - 1) / 2.0, z - zc)
    return _profile(Rc - r)[:, None, :]


def _slug(theta_deg, nz=32, nx=160, x_mid=50.0):
    """Slug centred in x spanning the channel between the walls z = -1/2 and
    nz - 1/2; each meniscus is a circular arc meeting both walls at theta
    (inside the slug).  The profile runs across the arc along x."""
    zc = (nz - 1) / 2.0
    a = nz / 2.0
    z = np.arange(nz, dtype=float)[:, None]
    x = np.arange(nx, dtype=float)[None, :]
    c = math.cos(math.radians(theta_deg))
    if abs(c) < 1e-12:
        xa = np.full_like(z, x_mid)
    else:
        R = a / abs(c)
        # wetting slug: centre on the other component's side
        xa = x_mid - math.copysign(1.0, c) * (R - np.sqrt(R * R - (z - zc) ** 2))
    # left half: slug to the right of the arc; right half mirrored
    d = np.where(x < nx / 2.0, x - xa, (nx - 1 - x) - xa)
    return _profile(d)[:, None, :]


@pytest.mark.parametrize("theta", [35.0, 60.0, 90.0, 115.0, 140.0])
@pytest.mark.parametrize("Rc", [18.3, 24.0, 29.7])
def test_cap_contact_angle_on_exact_caps(theta, Rc):
    got, h, b = dg.cap_contact_angle(_cap(theta, Rc), THR)
    zc = -0.5 - Rc * math.cos(math.radians(theta))
    assert abs(h - (zc + Rc + 0.5)) < 0.05
    assert abs(b - math.sqrt(Rc * Rc - zc * zc)) < 0.05
    assert abs(got - theta) < 0.5


@pytest.mark.parametrize("theta", [20.0, 40.0, 65.0, 90.0, 110.0, 140.0, 160.0])
def test_slug_contact_angle_on_exact_menisci(theta):
    got, each = dg.slug_contact_angle(_slug(theta), THR)
    assert len(each) == 4
    assert abs(got - theta) < 0.5
    assert max(each) - min(each) < 0.5


def test_slug_angle_is_the_supplement_for_the_other_component():
    rho2 = _slug(40.0)
    rho1 = HI + LO - rho2
    # component 1 occupies the ends: roll it so that it sits in the middle
    rho1 = np.roll(rho1, rho1.shape[2] // 2, axis=2)
    t2, _ = dg.slug_contact_angle(rho2, THR)
    t1, _ = dg.slug_contact_angle(rho1, THR)
    assert abs(t1 + t2 - 180.0) < 1.0


def test_fit_circle_recovers_centre_and_radius():
    t = np.linspace(0.3, 1.4, 40)
    x = 3.0 + 17.0 * np.cos(t)
    z = -2.0 + 17.0 * np.sin(t)
    xc, zc, R = dg.fit_circle(x, z)
    assert abs(xc - 3.0) < 1e-9 and abs(zc + 2.0) < 1e-9 and abs(R - 17.0) < 1e-9


def test_wall_layer_density():
    r = np.zeros((8, 1, 20))
    r[0, 0, :] = 0.1
    r[-1, 0, :] = 0.3
    r[0, 0, 5:10] = 9.0
    assert abs(dg.wall_layer_density(r, 10, 20) - 0.2) < 1e-15


@pytest.mark.parametrize("angle", [10, 30, 50, 70])
def test_channel_droplet_centre_tracks_displacement(angle):
    """Droplets drawn at known distances along an inclined channel (staircase
    walls, periodic copies): the centre found by channel_droplet_stats moves
    by the drawn displacement, across the periodic end of the channel too,
    and the droplet keeps its size."""
    from paper_1601_01237_gb300 import workloads as wl
    shape, solid, info = wl.inclined_channel(angle)
    L = info["L"]
    res = {}
    for s0 in (0.0, 17.0, L / 2 - 3.0, -L / 2 + 3.0):
        _, r2 = wl.channel_droplet(shape, info, 8.0, s0=s0)
        res[s0] = dg.channel_droplet_stats(r2, solid, info, 0.818)
    v0, c0, nfl = res[0.0]
    assert nfl == int((solid == 0).sum())
    assert abs((res[17.0][1] - c0) - 17.0) < 0.25
    d = res[-L / 2 + 3.0][1] - res[L / 2 - 3.0][1]
    d -= L * np.round(d / L)
    assert abs(d - 6.0) < 0.5          # 6 cells forward through the periodic end
    assert all(abs(r[0] - v0) <= 0.15 * v0 for r in res.values())


def test_sphere_array_cell_geometry():
    """The simple-cubic cell of touching spheres: porosity within 1 % of
    1 - pi/6, neighbouring spheres meet at the face centres, and the solid is
    symmetric under the cube's reflections."""
    from paper_1601_01237_gb300 import workloads as wl
    shape, solid, phi = wl.sphere_array_cell(34)
    assert shape == (34, 34, 34)
    assert abs(phi - (1 - np.pi / 6)) < 0.01 * (1 - np.pi / 6)
    assert solid[0, 16, 16] and solid[16, 0, 16] and solid[16, 16, 0] and not solid[0, 0, 0]
    for ax in range(3):
        assert np.array_equal(solid, np.flip(solid, axis=ax))
    assert np.array_equal(solid, solid.transpose(1, 0, 2)) and np.array_equal(solid, solid.transpose(2, 1, 0))


@pytest.mark.parametrize("angle", [10, 30, 50, 70])
def test_inclined_channel_geometry(angle):
    """The inclined channel: its angle within 0.3 degrees, length >= 96, the
    fluid band H = 16 wide across the channel (fluid fraction H / P of the
    lattice), at least 4 solid layers between periodic copies, and a single
    connected channel through the periodic ends."""
    from paper_1601_01237_gb300 import workloads as wl
    shape, solid, info = wl.inclined_channel(angle)
    nz, _, nx = shape
    assert abs(info["theta_deg"] - angle) <= 0.3 and info["L"] >= 96 and info["P"] >= 20
    fl = solid[:, 0, :] == 0
    assert abs(fl.mean() - 16.0 / info["P"]) < 0.03
    # cells on a line across the channel: fluid run of about H cells
    en = info["across"]
    c = np.array([(nx - 1) / 2.0, (nz - 1) / 2.0])
    run = [fl[int(round(c[1] + t * en[1])) % nz, int(round(c[0] + t * en[0])) % nx]
           for t in np.arange(-info["P"] / 2 + 0.25, info["P"] / 2, 0.5)]
    assert abs(0.5 * sum(run) - 16.0) <= 1.5
    # one channel: the fluid cells form a single region on the periodic
    # lattice (flood fill through the D2Q9 links, wrapping at the ends)
    seen = np.zeros_like(fl)
    start = tuple(np.argwhere(fl)[0])
    stack = [start]
    seen[start] = True
    while stack:
        z, x = stack.pop()
        for dz in (-1, 0, 1):
            for dx in (-1, 0, 1):
                q = ((z + dz) % nz, (x + dx) % nx)
                if fl[q] and not seen[q]:
                    seen[q] = True
                    stack.append(q)
    assert seen.sum() == fl.sum()


def test_spinodal_stats_closed_forms():
    """Statistics of the c2 comparison on fields with known answers: a single
    Fourier mode of wavenumber k0 (in units of 2 pi / L) puts all of S(k) on
    shell k0, so k* = k_peak = k0, and its phi = 0 surface is 2 k0 planes of
    L^2 faces; a slab has 2 L^2 faces; <|phi|> of a mode of amplitude A is
    2A/pi; the masses are the sums."""
    L = 32
    x = np.arange(L)
    for k0 in (1, 3, 5):
        phi = 0.3 * np.cos(2 * np.pi * k0 * (x + 0.25) / L)
        a = 0.5 + 0.5 * np.broadcast_to(phi, (L, L, L))
        b = 0.5 - 0.5 * np.broadcast_to(phi, (L, L, L))
        st = dg.spinodal_stats(a, b)
        assert abs(st["k_star"] - k0) < 1e-9 and st["k_peak"] == k0
        assert st["interface_area"] == 2 * k0 * L * L
        assert abs(st["mean_abs_phi"] - 2 * 0.3 / np.pi) < 1e-3
        assert abs(st["mass1"] - a.sum()) < 1e-9 and abs(st["mass2"] - b.sum()) < 1e-9
    # the mode along y and along z gives the same statistics (isotropy of the shells)
    phi_z = 0.3 * np.cos(2 * np.pi * 3 * (np.arange(L) + 0.25) / L)[:, None, None] * np.ones((1, L, L))
    st = dg.spinodal_stats(0.5 + 0.5 * phi_z, 0.5 - 0.5 * phi_z)
    assert abs(st["k_star"] - 3) < 1e-9 and st["interface_area"] == 6 * L * L
    slab = np.where(np.arange(L) < L // 2, 0.8, 0.2)[None, None, :] * np.ones((L, L, 1))
    st = dg.spinodal_stats(slab, 1.0 - slab)
    assert st["interface_area"] == 2 * L * L
    # a diagonal mode (k = (2, 2, 1), |k| = 3) sits on shell 3
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    phi = 0.2 * np.cos(2 * np.pi * (2 * xx + 2 * y + z + 0.1) / L)
    st = dg.spinodal_stats(0.5 + 0.5 * phi, 0.5 - 0.5 * phi)
    assert abs(st["k_star"] - 3) < 1e-9


def test_mass_radius_of_exact_discs_and_spheres():
    """The excess-mass radius equals the radius of a hard-edged disc or
    sphere of known area or volume (the count of its cells), and for a tanh
    profile of width W it moves continuously with R (no jumps of whole
    rings)."""
    n = 48
    z, y, x = np.meshgrid(np.arange(1), np.arange(n), np.arange(n), indexing="ij")
    c = ((n - 1) / 2.0, (n - 1) / 2.0, 0.0)
    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2)
    for R0 in (6.0, 9.3, 12.0):
        disc = np.where(r < R0, 1.1, 0.02)
        R, rin, rout = dg.mass_radius(disc, c, R0 / 2, R0 + 4)
        assert abs(R - np.sqrt((r < R0).sum() / np.pi)) < 1e-12
        assert abs(rin - 1.1) < 1e-14 and abs(rout - 0.02) < 1e-14
    m = 32
    z, y, x = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    c3 = ((m - 1) / 2.0,) * 3
    r3 = np.sqrt((x - c3[0]) ** 2 + (y - c3[1]) ** 2 + (z - c3[2]) ** 2)
    ball = np.where(r3 < 7.5, 1.0, 0.1)
    R, _, _ = dg.mass_radius(ball, c3, 3.0, 11.0, dims=3)
    assert abs(R - (3 * (r3 < 7.5).sum() / (4 * np.pi)) ** (1 / 3)) < 1e-12
    Rs = [dg.mass_radius(wl.droplet((1, n, n), R0)[0], c, R0 / 2, R0 + 8)[0] for R0 in np.linspace(8, 9, 11)]
    assert np.all(np.diff(Rs) > 0) and np.max(np.diff(Rs)) < 0.2
