"""Seeded synthetic inputs shaped like the paper's test cases.

This module holds input recipes only (density fields, noise, lattice sizes and
parameters); none of the method's arithmetic.  Both the CUDA path and the
oracle consume what it produces.

Recipes (Otomo et al., arXiv:1601.01237):
  * droplet / sphere: tanh profile rho^1(r) = rho_out + (rho_in - rho_out)/2 *
    (1 - tanh((r - R)/W)), component 2 mirrored so rho^1 + rho^2 is uniform
    (the static-droplet tests of Sec. 3);
  * ellipsoid: the same profile with r measured in units of the semi-axes;
  * spinodal mixture: rho^a = rho0 (1 + amp * U(-1, 1)), U from SplitMix64 over
    the linear cell index with seed + a;
  * hemisphere on a wall: a sphere centred on the wall plane z = -1/2 (the
    wall-attached droplet of Sec. 4.2);
  * slug: component 2 filling a channel section between two flat interfaces
    (the slug between plates of Sec. 4.2);
  * inclined channel: staircase solid sites around a channel of height H at
    an angle to the lattice, periodic along its length, with a droplet of
    component 2 on its lower wall (the inclined-wall case of Sec. 4.2).

Interaction strength: Eq. 7 takes a signed G (repulsion: G < 0).  The
droplet cases quote 1.0 inside / 0.03 outside; G = -1.8 is the value whose
flat-interface coexistence densities are those (1.026 / 0.029, measured on
the oracle at tau = 1), so the droplets start at equilibrium densities.  The
mixture cases use G = -1.2, which separates a 0.5 / 0.5 mixture into
0.897 / 0.148 with the regularized operator at every tau from 0.6 to 1.
"""
import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(seed, n):
    """First n outputs of SplitMix64 (Steele, Lea & Flood 2014) seeded with seed,
    as uint64; output k is the generator advanced k+1 times."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed, n):
    """n doubles uniform in [-1, 1) from the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return 2.0 * u - 1.0


def _radius(shape, center, scale=(1.0, 1.0, 1.0)):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    cz, cy, cx = center
    sz, sy, sx = scale
    return np.sqrt(((x - cx) / sx) ** 2 + ((y - cy) / sy) ** 2 + ((z - cz) / sz) ** 2)


def tanh_profile(r, R, rho_in, rho_out, width):
    rho1 = rho_out + 0.5 * (rho_in - rho_out) * (1.0 - np.tanh((r - R) / width))
    rho2 = rho_in + rho_out - rho1
    return rho1, rho2


def droplet(shape, R, rho_in=1.0, rho_out=0.03, width=2.0, center=None):
    """Circular (nz = 1) or spherical droplet of component 1 centred on the
    lattice: returns (rho1, rho2) of shape (nz, ny, nx)."""
    nz, ny, nx = shape
    if center is None:
        center = ((nz - 1) / 2.0, (ny - 1) / 2.0, (nx - 1) / 2.0)
    r = _radius(shape, center)
    if nz == 1:
        r = _radius(shape, (0.0, center[1], center[2]))
    return tanh_profile(r, R, rho_in, rho_out, width)


def ellipsoid(shape, semi_axes, rho_in=1.0, rho_out=0.03, width=2.0):
    """Ellipsoidal droplet with semi-axes (a_x, a_y, a_z), centred."""
    nz, ny, nx = shape
    ax, ay, az = semi_axes
    center = ((nz - 1) / 2.0, (ny - 1) / 2.0, (nx - 1) / 2.0)
    # distance along the ray scaled back to lattice units with the mean axis
    s = _radius(shape, center, scale=(az, ay, ax))
    R = (ax * ay * az) ** (1.0 / 3.0)
    return tanh_profile(s * R, R, rho_in, rho_out, width)


def hemisphere(shape, R, rho_in=1.0, rho_out=0.03, width=2.0):
    """Droplet of component 1 sitting on the wall z = -1/2, centred in x, y."""
    nz, ny, nx = shape
    r = _radius(shape, (-0.5, (ny - 1) / 2.0, (nx - 1) / 2.0))
    return tanh_profile(r, R, rho_in, rho_out, width)


def slug(shape, x_left, x_right, rho_in=1.0, rho_out=0.03, width=2.0):
    """Slug of component 2 filling the channel between x_left and x_right
    (flat interfaces; the static slug between plates of Sec. 4.2); returns
    (rho1, rho2)."""
    nz, ny, nx = shape
    x = np.broadcast_to(np.arange(nx, dtype=np.float64), shape)
    d = np.minimum(x - x_left, x_right - x)
    rho2, rho1 = tanh_profile(-d, 0.0, rho_in, rho_out, width)
    return rho1, rho2


def inclined_channel(theta_deg, H=16, min_len=96, min_gap=4, max_side=400):
    """Quasi-2D channel of perpendicular height H whose walls are inclined by
    theta_deg to the x axis, as staircase solid sites on a lattice periodic
    in x and z (the inclined-wall case of Sec. 4.2): the channel's centre
    line runs along (nx, nz) through the lattice centre and closes on itself
    after its length L = |(nx, nz)|; its periodic copies lie P = nx nz / L
    apart, and the cells farther than H/2 from the nearest copy are solid.
    (nx, nz) is the smallest lattice whose angle atan(nz/nx) is within 0.3
    degrees of theta_deg with L >= min_len and P >= H + min_gap.
    Returns (shape (nz, 1, nx), solid (nz, 1, nx) uint8, info dict with the
    angle, L, P and the unit vectors along and across the channel)."""
    t = math.radians(theta_deg)
    best = None
    for nx in range(1, max_side + 1):
        nz = int(round(nx * math.tan(t)))
        for cz in (nz, nz + 1):
            if cz < 1 or cz > max_side:
                continue
            L = math.hypot(nx, cz)
            P = nx * cz / L
            ang = math.degrees(math.atan2(cz, nx))
            if abs(ang - theta_deg) <= 0.3 and L >= min_len and P >= H + min_gap:
                if best is None or nx * cz < best[0] * best[1]:
                    best = (nx, cz)
    if best is None:
        raise ValueError("no lattice up to %d for %g degrees" % (max_side, theta_deg))
    nx, nz = best
    L = math.hypot(nx, nz)
    P = nx * nz / L
    es = np.array([nx, nz], dtype=np.float64) / L          # along the channel (x, z)
    en = np.array([-nz, nx], dtype=np.float64) / L         # across, towards the upper wall
    z, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    d = (x - (nx - 1) / 2.0) * en[0] + (z - (nz - 1) / 2.0) * en[1]
    d = d - P * np.round(d / P)                             # distance to the nearest copy
    solid = (np.abs(d) >= H / 2.0).astype(np.uint8)[:, None, :]
    info = {"theta_deg": math.degrees(math.atan2(nz, nx)), "L": L, "P": P, "H": H, "along": es, "across": en}
    return (nz, 1, nx), solid, info


def inclined_slab(shape, theta_deg=30.0, thickness=8):
    """Staircase wall for a 3D lattice periodic in every direction: the solid
    sites are the cells with (z - x tan(theta)) mod nz < thickness, a slab
    inclined by theta to the x axis along x and uniform along y (the inclined
    walls of Sec. 4.2 extruded across the lattice).  Returns the (nz, ny, nx)
    uint8 mask."""
    nz, ny, nx = shape
    z, x = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    h = np.mod(z - np.floor(x * math.tan(math.radians(theta_deg))), nz)
    return np.repeat((h < thickness).astype(np.uint8)[:, None, :], ny, axis=1)


def channel_droplet(shape, info, R, s0=0.0, rho_in=1.0, rho_out=0.03, width=2.0):
    """Droplet of component 2 in an inclined_channel: a disc of radius R
    centred on the lower wall, s0 along the centre line from the lattice
    centre (distances by minimum image on the periodic lattice; the part of
    the disc inside the wall is solid).  Returns (rho1, rho2)."""
    nz, _, nx = shape
    c = (np.array([(nx - 1) / 2.0, (nz - 1) / 2.0]) + s0 * info["along"] - (info["H"] / 2.0) * info["across"])
    z, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    dx = x - c[0]
    dz = z - c[1]
    dx = dx - nx * np.round(dx / nx)
    dz = dz - nz * np.round(dz / nz)
    r = np.sqrt(dx * dx + dz * dz)
    rho2, rho1 = tanh_profile(r, R, rho_in, rho_out, width)
    return rho1[:, None, :], rho2[:, None, :]


def sphere_array_cell(L=34, chi=1.0):
    """One cell of the simple-cubic array of spheres (Sec. 4.2): an L^3
    periodic lattice with a sphere of radius chi L / 2 centred in it (chi = 1:
    neighbouring spheres touch); solid sites are the cells whose centres lie
    inside.  Returns (shape, solid uint8, porosity)."""
    shape = (L, L, L)
    r = _radius(shape, ((L - 1) / 2.0,) * 3)
    solid = (r < chi * L / 2.0).astype(np.uint8)
    return shape, solid, float((solid == 0).mean())


def spinodal(shape, rho0=0.5, amp=0.01, seed=20160105):
    """Uniform mixture with +-amp relative seeded noise per component."""
    n = int(np.prod(shape))
    r1 = rho0 * (1.0 + amp * uniform_pm1(seed + 0, n))
    r2 = rho0 * (1.0 + amp * uniform_pm1(seed + 1, n))
    return r1.reshape(shape), r2.reshape(shape)


def random_state(shape, seed, rho_lo=0.2, rho_hi=1.0, u_max=0.05):
    """Random densities in [rho_lo, rho_hi] and velocities with |u_d| <= u_max,
    for parity tests of the raw update."""
    n = int(np.prod(shape))
    r1 = rho_lo + (rho_hi - rho_lo) * 0.5 * (1.0 + uniform_pm1(seed * 4 + 1, n))
    r2 = rho_lo + (rho_hi - rho_lo) * 0.5 * (1.0 + uniform_pm1(seed * 4 + 2, n))
    u = u_max * uniform_pm1(seed * 4 + 3, 3 * n)
    return r1.reshape(shape), r2.reshape(shape), u.reshape(shape + (3,))


# ---------------------------------------------------------------------------
# The five cases and the 512^3 throughput case.  "G" is the signed Eq. 7 value.
# Signed G^{12} = G^{21} of Eq. 7 per case.  The droplet cases start from
# 1.0 inside / 0.03 outside; G = -1.8 is where those are the flat-interface
# coexistence densities (1.026 / 0.029 on the oracle at tau = 1).  G = -1.2
# separates a 0.5 / 0.5 mixture into 0.897 / 0.148 with the regularized
# operator at any tau (BGK at tau < 1 separates further and diverges).
G_DROPLET = -1.8
G_MIXTURE = -1.2
# With Guo's forcing (the second reading of the forcing term) the force and
# the density gradient enter a component's flux with the same factor, so the
# coexistence of the regularized operator is that of the continuum criterion
# at G itself, where the exact-difference forcing acts like 2 G: the Guo
# values below give the same coexisting densities (1.047 / 0.019 and
# 0.918 / 0.141 on flat interfaces of the oracle) at every tau from 0.525 to 3.
G_DROPLET_GUO = -3.6
G_MIXTURE_GUO = -2.4


def g_droplet(forcing="edm"):
    """Signed Eq. 7 G of the droplet cases for a forcing reading."""
    return G_DROPLET_GUO if forcing == "guo" else G_DROPLET

CONFIGS = {
    "c0_droplet2d_f64": dict(shape=(1, 64, 64), storage="f64", tau=(1.0, 1.0), G=G_DROPLET,
                             R=16, steps=2000, init="droplet"),
    # tau = 1: BGK and regularized coincide; tau = 0.8: regularized (BGK
    # diverges); tau = 0.55 diverges with both operators at this G
    "c1_droplet3d_f32": dict(shape=(128, 128, 128), storage="f32", tau=(1.0, 1.0), G=G_DROPLET,
                             R=16, steps=10000, init="droplet", radii=(12, 16, 20, 24, 32),
                             taus=(0.55, 0.8, 1.0), collision_for_tau={0.55: "regularized", 0.8: "regularized",
                                                                       1.0: "bgk"}),
    "c2_spinodal256": dict(shape=(256, 256, 256), storage="f32", tau=(0.7, 0.7), G=G_MIXTURE,
                           collision="regularized", steps=5000, init="spinodal"),
    "c3_adjoint96": dict(shape=(96, 96, 96), storage="f32", tau=(1.0, 1.0), G=G_DROPLET,
                         R=20, steps=500, init="droplet", ckpt_every=25, target_axes=(24, 20, 16)),
    # tau = 0.55 holds no droplet at G_DROPLET: G_MIXTURE with the hemisphere at
    # that G's coexistence densities; no body force (g_mag = 0), the tilted
    # gravity of magnitude g_mag_tilted is a separate run
    "c4_wall512": dict(shape=(384, 512, 512), storage="f32", tau=(0.55, 0.55), G=G_MIXTURE,
                       R=48, steps=20000, init="hemisphere", rho_in=0.897, rho_out=0.148,
                       collision="regularized", periodic=(1, 1, 0), g_mag=0.0, g_mag_tilted=1e-5,
                       tilt_deg=30.0),
    "perf512_spinodal_f32": dict(shape=(512, 512, 512), storage="f32", tau=(1.0, 1.0), G=G_MIXTURE,
                                 init="spinodal"),
}


def tilted_gravity(g_mag, tilt_deg):
    """Body acceleration of magnitude g_mag tilted by tilt_deg from -z toward +x."""
    t = math.radians(tilt_deg)
    return (g_mag * math.sin(t), 0.0, -g_mag * math.cos(t))


def fields_for(name, shape=None, **over):
    """(rho1, rho2) for a named case, optionally on another shape."""
    c = dict(CONFIGS[name], **over)
    shape = tuple(shape or c["shape"])
    kind = c["init"]
    if kind == "droplet":
        return droplet(shape, c["R"])
    if kind == "spinodal":
        return spinodal(shape)
    if kind == "hemisphere":
        return hemisphere(shape, c["R"], rho_in=c.get("rho_in", 1.0), rho_out=c.get("rho_out", 0.03))
    raise KeyError(kind)
