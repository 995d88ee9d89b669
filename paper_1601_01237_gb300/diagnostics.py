"""Host-side helpers for the paper's measurements (Sec. 3-4): Young-Laplace fit
(Eq. 12), equivalent radius of a droplet from its volume, drift velocity,
contact angles of a sessile droplet and of a slug between plates, and the
position and size of a droplet in an inclined channel (Sec. 4.2).
The field reductions themselves run on the GPU (lbm_pressure_jump,
lbm_droplet_stats, lbm_reduce)."""
import math

import numpy as np


def equivalent_radius(volume, quasi_2d, hemisphere=False):
    """Radius of the disc (quasi-2D) or sphere (3D) or hemisphere of this volume."""
    if quasi_2d:
        return math.sqrt(volume / math.pi)
    if hemisphere:
        return (3.0 * volume / (2.0 * math.pi)) ** (1.0 / 3.0)
    return (3.0 * volume / (4.0 * math.pi)) ** (1.0 / 3.0)


def laplace_fit(radii, dps, dims=2):
    """Least-squares fit dp = s / R + c.  Eq. 12 is the 2D form dp = sigma / R;
    in 3D dp = 2 sigma / R.  Returns (sigma, intercept, max residual)."""
    R = np.asarray(radii, dtype=float)
    dp = np.asarray(dps, dtype=float)
    A = np.vstack([1.0 / R, np.ones_like(R)]).T
    (s, c), *_ = np.linalg.lstsq(A, dp, rcond=None)
    resid = float(np.max(np.abs(A @ np.array([s, c]) - dp)))
    return (s if dims == 2 else s / 2.0), float(c), resid


def drift_velocity(com_a, com_b, steps):
    """Centre-of-mass displacement per step between two measurements."""
    d = np.asarray(com_b, dtype=float) - np.asarray(com_a, dtype=float)
    return d / float(steps)


def _crossing(v, thr, k):
    """Position where the profile v crosses thr between cells k and k + 1
    (linear interpolation)."""
    return k + (thr - v[k]) / (v[k + 1] - v[k])


def cap_contact_angle(rho, thr):
    """Contact angle of a quasi-2D droplet (fields (nz, 1, nx)) on the wall
    z = -1/2, measured inside the droplet, for a circular cap: from its height
    h at the centre column and its half-width b on the first fluid layer (both
    where rho crosses thr, interpolated linearly), the circle through the top
    and the chord on z = 0.  Returns (theta in degrees, h, b); theta is None
    when no cell of the first layer exceeds thr."""
    col = np.asarray(rho)[:, 0, :]
    nz, nx = col.shape
    xs = np.nonzero(col[0] > thr)[0]
    if xs.size == 0:
        return None, 0.0, 0.0
    xc = int(round(xs.mean()))
    zc = col[:, xc]
    k = int(np.nonzero(zc > thr)[0].max())
    h = (_crossing(zc, thr, k) + 0.5) if k + 1 < nz else float(nz)
    row = col[0]
    lo, hi = int(xs.min()), int(xs.max())
    left = _crossing(row, thr, lo - 1) if lo > 0 else float(lo)
    right = _crossing(row, thr, hi) if hi + 1 < nx else float(hi)
    b = 0.5 * (right - left)
    # circle through the top (z = h - 1/2) and the chord 2 b on z = 0; the
    # angle between it and the wall z = -1/2 inside the droplet
    zt = h - 0.5
    Rc = (b * b + zt * zt) / (2.0 * zt)
    zcen = zt - Rc
    theta = np.degrees(np.arccos(np.clip(-(zcen + 0.5) / Rc, -1.0, 1.0)))
    return float(theta), float(h), float(b)


def fit_circle(x, z):
    """Algebraic least-squares circle x^2 + z^2 + D x + E z + F = 0 through
    the points (Kasa's fit).  Returns (xc, zc, R)."""
    x = np.asarray(x, dtype=float)
    z = np.asarray(z, dtype=float)
    A = np.vstack([x, z, np.ones_like(x)]).T
    (D, E, F), *_ = np.linalg.lstsq(A, -(x * x + z * z), rcond=None)
    xc, zc = -0.5 * D, -0.5 * E
    return xc, zc, math.sqrt(max(xc * xc + zc * zc - F, 0.0))


def slug_contact_angle(rho, thr, skip=2):
    """Contact angle of a quasi-2D slug (fields (nz, 1, nx)) spanning the
    channel between the walls z = -1/2 and z = nz - 1/2, measured inside the
    slug (the component whose density rho is given, rho > thr inside, centred
    in x).  Each meniscus is the set of per-row crossings of thr (rows skip ..
    nz - 1 - skip); a circle fitted to them meets both walls at the angle
    returned (the mean over the two menisci and two walls, degrees), with the
    per-meniscus angles."""
    col = np.asarray(rho)[:, 0, :]
    nz, nx = col.shape
    mid = nx // 2
    out = []
    for side in (-1, 1):
        xs, zs = [], []
        for z in range(skip, nz - skip):
            row = col[z]
            if side < 0:
                ks = np.nonzero((row[:mid] <= thr) & (row[1:mid + 1] > thr))[0]
                if ks.size:
                    xs.append(_crossing(row, thr, int(ks.max())))
                    zs.append(z)
            else:
                ks = np.nonzero((row[mid:-1] > thr) & (row[mid + 1:] <= thr))[0]
                if ks.size:
                    xs.append(_crossing(row, thr, int(ks.min()) + mid))
                    zs.append(z)
        if len(xs) < 3:
            return None, []
        if np.ptp(xs) < 1e-9:   # a straight meniscus
            out += [90.0, 90.0]
            continue
        xc, zc, R = fit_circle(xs, zs)
        # the slug wets (angle < 90) when the centre lies on the other
        # component's side of the meniscus
        s = 1.0 if (xc - np.mean(xs)) * side > 0 else -1.0
        # distance of the centre from each wall over R is the cosine
        for h in (zc + 0.5, nz - 0.5 - zc):
            out.append(float(np.degrees(np.arccos(np.clip(s * h / R, -1.0, 1.0)))))
    return float(np.mean(out)), out


def wall_layer_density(rho, x_lo, x_hi):
    """Mean density on the first fluid layers next to the walls (z = 0 and
    z = nz - 1) over x_lo <= x < x_hi, y = 0 (the thin-film measure)."""
    r = np.asarray(rho)
    return float(0.5 * (r[0, 0, x_lo:x_hi].mean() + r[-1, 0, x_lo:x_hi].mean()))


def channel_droplet_stats(b, solid, info, thr):
    """Droplet of component 2 in an inclined channel: number of fluid cells
    with rho^2 > thr, their rho^2-weighted centre along the channel (circular
    mean over the channel length L, each cell taken in the periodic copy of
    the channel that holds the lattice centre), and the fluid cell count."""
    nz, _, nx = b.shape
    es, en, P, L = info["along"], info["across"], info["P"], info["L"]
    z, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    X = x - (nx - 1) / 2.0
    Z = z - (nz - 1) / 2.0
    s = X * es[0] + Z * es[1]
    n = X * en[0] + Z * en[1]
    k = np.round(n / P)
    s = s + k * nx * es[0]            # translate by k (nx, 0): n -> n - k P
    rho = b[:, 0, :]
    fl = solid[:, 0, :] == 0
    drop = fl & (rho > thr)
    m = rho[drop]
    ph = 2.0 * np.pi * s[drop] / L
    com = L / (2.0 * np.pi) * np.arctan2((m * np.sin(ph)).sum(), (m * np.cos(ph)).sum()) if m.size else float("nan")
    return int(drop.sum()), float(com), int(fl.sum())


def structure_factor(phi):
    """Spherically averaged structure factor of a periodic order-parameter
    field phi (nz, ny, nx): S(k) = <|FFT(phi - <phi>)|^2> over the shells
    k - 1/2 <= |k| < k + 1/2, with |k| in units of 2 pi / L (a cube of side L).
    Returns (k, S) for the shells k = 1 .. L/2."""
    phi = np.asarray(phi, dtype=float)
    n = phi.shape[0]
    assert phi.shape == (n, n, n), "a cubic lattice"
    P = np.abs(np.fft.fftn(phi - phi.mean())) ** 2
    f = np.fft.fftfreq(n) * n
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    shell = np.rint(np.sqrt(kx * kx + ky * ky + kz * kz)).astype(int)
    kmax = n // 2
    S = np.bincount(shell.ravel(), weights=P.ravel(), minlength=kmax + 1)[:kmax + 1]
    cnt = np.bincount(shell.ravel(), minlength=kmax + 1)[:kmax + 1]
    k = np.arange(1, kmax + 1)
    return k, S[1:] / np.maximum(cnt[1:], 1)


def spinodal_stats(rho1, rho2):
    """Statistics of a two-component spinodal mixture on a periodic cube
    (order parameter phi = rho^1 - rho^2):
      mass1, mass2      sum of each density;
      mean_abs_phi      <|rho^1 - rho^2|> over the cells;
      k_star            first moment sum k S(k) / sum S(k) of the spherically
                        averaged structure factor (units of 2 pi / L), the
                        characteristic wavenumber of the domains;
      k_peak            the shell where S(k) is largest;
      interface_area    the number of lattice links (x, y and z neighbours,
                        periodic) across which phi changes sign: the area of
                        the phi = 0 surface in units of a cell face."""
    a = np.asarray(rho1, dtype=float)
    b = np.asarray(rho2, dtype=float)
    phi = a - b
    k, S = structure_factor(phi)
    pos = phi > 0
    area = sum(int(np.count_nonzero(pos != np.roll(pos, 1, axis=ax))) for ax in range(3))
    return {"mass1": float(a.sum()), "mass2": float(b.sum()), "mean_abs_phi": float(np.abs(phi).mean()),
            "k_star": float((k * S).sum() / S.sum()), "k_peak": int(k[int(np.argmax(S))]),
            "interface_area": area}


def mass_radius(rho, center, r_in, r_out, dims=2):
    """Radius of a droplet of the component with density field rho from its
    excess mass, a continuous measure (the count of cells above a threshold
    jumps by whole rings of cells): with rho_in, rho_out the mean densities
    over r < r_in and r > r_out around center = (x, y, z) (minimum image),
    the droplet holds (sum rho - rho_out N) / (rho_in - rho_out) cells of
    interior density, a disc (dims = 2, nz = 1) or sphere of that area or
    volume.  Returns (R, rho_in, rho_out)."""
    a = np.asarray(rho, dtype=float)
    nz, ny, nx = a.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def mi(d, n):
        return (d + n / 2.0) % n - n / 2.0
    dz = mi(z - center[2], nz) if dims == 3 else 0.0
    r = np.sqrt(mi(x - center[0], nx) ** 2 + mi(y - center[1], ny) ** 2 + dz ** 2)
    rin, rout = float(a[r < r_in].mean()), float(a[r > r_out].mean())
    vol = (a.sum() - rout * a.size) / (rin - rout)
    R = math.sqrt(vol / math.pi) if dims == 2 else (3.0 * vol / (4.0 * math.pi)) ** (1.0 / 3.0)
    return R, rin, rout
