"""Seeded synthetic particle sets shaped like the paper's workloads.

This module only draws inputs: positions, velocities, masses, internal
energies, starting smoothing lengths and active flags, as float32 NumPy
arrays in the periodic unit box. It computes no SPH sum. The CUDA path, the
oracle, the tests and the benchmark all take their inputs from here.

The paper measures the 3-D Gresho-Chan vortex on a uniform particle lattice
with roughly 64 particles per cell (Sec. 3.1); its initial-condition files are
not available, so the sets below stand in for it:

* ``lattice``   - jittered cubic lattice, equal masses, v = 0, u = 1.
* ``sedov``     - jittered 64^3 lattice, u = 1e-5, total energy 1 deposited
                  into the 32 particles nearest the centre.
* ``plummer``   - 64 Plummer spheres plus a 10 % uniform background
                  (cell occupancy from 1 to thousands), 10 % active particles.
* ``kh``        - Kelvin-Helmholtz slab: density 2 in |y-0.5| < 0.25 via a
                  finer lattice, vx = +-0.5, pressure 2.5.
* ``zeldovich`` - lattice displaced by a Gaussian random field with
                  P(k) ~ k^-2 (density contrast ~100), v proportional to the
                  displacement.
* ``gresho``    - the Gresho-Chan vortex itself (Sec. 3.1, Eqs. 27-28) on a
                  cubic lattice: rho = 1, gamma = 5/3, azimuthal velocity and
                  pressure from the analytic steady state.

Random streams: NumPy PCG64 seeded with ``SEED_BASE + config index``; the
active flags use splitmix64(seed ^ i) mod 10 == 0.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2505145380
ETA = 1.2348          # resolution parameter: about 48 weighted neighbours
GAMMA_EOS = 5.0 / 3.0


def _rng(index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index))


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea and Flood 2014) on uint64 arrays."""
    z = (np.asarray(x, np.uint64) + np.uint64(0x9E3779B97F4A7C15))
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def active_hash(n: int, seed: int, modulus: int = 10) -> np.ndarray:
    """uint8 flags: particle i is active when splitmix64(seed ^ i) % modulus == 0."""
    i = np.arange(n, dtype=np.uint64)
    return (splitmix64(np.uint64(seed) ^ i) % np.uint64(modulus) == 0).astype(np.uint8)


def _wrap(x: np.ndarray) -> np.ndarray:
    x = np.mod(x, 1.0)
    x[x >= 1.0] = 0.0
    return x


def _finish(name, pos, vel, m, u, h, active=None, **meta):
    pos = _wrap(np.asarray(pos, np.float64)).astype(np.float32)
    # float32 rounding can land exactly on 1.0
    pos[pos >= np.float32(1.0)] = np.float32(0.0)
    d = dict(name=name, pos=pos, vel=np.asarray(vel, np.float32), m=np.asarray(m, np.float32),
             u=np.asarray(u, np.float32), h=np.asarray(h, np.float32),
             active=None if active is None else np.asarray(active, np.uint8), box=(1.0, 1.0, 1.0))
    d.update(meta)
    return d


def lattice(n_side: int = 16, jitter: float = 0.1, index: int = 1, u: float = 1.0):
    """n_side^3 cubic lattice (spacing 1/n_side), each axis jittered by U(-jitter, jitter) spacing."""
    rng = _rng(index)
    dx = 1.0 / n_side
    g = (np.arange(n_side) + 0.5) * dx
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    pos = pos + rng.uniform(-jitter * dx, jitter * dx, size=pos.shape)
    n = len(pos)
    return _finish(f"lattice{n_side}", pos, np.zeros((n, 3)), np.full(n, 1.0 / n), np.full(n, u),
                   np.full(n, ETA * dx), spacing=dx)


def sedov(n_side: int = 64, jitter: float = 0.1, index: int = 2, energy: float = 1.0, n_hot: int = 32):
    """Sedov blast: jittered lattice, u = 1e-5, `energy` put into the n_hot particles nearest the centre.

    Deposition weight of hot particle i: s(r_i / R) with s the cubic-spline
    shape and R the distance to the (n_hot+1)-th nearest particle; ties in
    distance are broken by index.
    """
    d = lattice(n_side, jitter, index, u=1e-5)
    pos = d["pos"].astype(np.float64)
    n = len(pos)
    r = np.linalg.norm(pos - 0.5, axis=1)
    order = np.lexsort((np.arange(n), r))
    hot = order[:n_hot]
    R = r[order[n_hot]]
    q = r[hot] / R
    s = np.where(q < 0.5, 1 - 6 * q ** 2 + 6 * q ** 3, 2 * (1 - q) ** 3)
    m = 1.0 / n
    u = d["u"].astype(np.float64)
    u[hot] += energy * s / (m * s.sum())
    d["u"] = u.astype(np.float32)
    d["name"] = f"sedov{n_side}"
    d["hot"] = hot
    return d


def plummer(n_total: int = 2 ** 21, n_spheres: int = 64, bg_frac: float = 0.1, index: int = 3,
            a_min: float = 0.005, a_max: float = 0.05, active_mod: int = 10, h_grid: int = 32):
    """Mixture of Plummer spheres plus a uniform background; 1/active_mod of particles active.

    Radii follow the Plummer inverse CDF r = a (X^(-2/3) - 1)^(-1/2) truncated at
    10 a by rejection. Velocities N(0, 0.1^2) per axis, u = 1. Starting h is
    eta times the mean spacing of the particle's cell on an h_grid^3 grid.
    """
    rng = _rng(index)
    n_bg = int(n_total * bg_frac)
    n_sph = n_total - n_bg
    per = np.full(n_spheres, n_sph // n_spheres)
    per[: n_sph - per.sum()] += 1
    centres = rng.uniform(0, 1, size=(n_spheres, 3))
    radii = np.exp(rng.uniform(np.log(a_min), np.log(a_max), size=n_spheres))
    parts = [rng.uniform(0, 1, size=(n_bg, 3))]
    for s in range(n_spheres):
        k = per[s]
        rr = np.empty(0)
        while len(rr) < k:
            X = rng.uniform(0, 1, size=2 * k)
            X = X[X > 0]
            r = radii[s] / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
            rr = np.concatenate([rr, r[r < 10 * radii[s]]])
        rr = rr[:k]
        dirs = rng.normal(size=(k, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        parts.append(centres[s] + rr[:, None] * dirs)
    pos = _wrap(np.concatenate(parts, 0))
    n = len(pos)
    vel = rng.normal(0, 0.1, size=(n, 3))
    cid = np.minimum((pos * h_grid).astype(np.int64), h_grid - 1)
    lin = cid[:, 0] + h_grid * (cid[:, 1] + h_grid * cid[:, 2])
    counts = np.bincount(lin, minlength=h_grid ** 3)
    h0 = ETA * (1.0 / h_grid) / np.cbrt(counts[lin])
    act = active_hash(n, SEED_BASE + index, active_mod)
    return _finish(f"plummer{n}", pos, vel, np.full(n, 1.0 / n), np.ones(n), h0, act,
                   centres=centres, radii=radii)


def kh(nx: int = 32, ny_dense: int = 21, ny_light: int = 11, jitter: float = 0.01, index: int = 4,
       pressure: float = 2.5, shear: float = 0.5):
    """Kelvin-Helmholtz slab in the periodic unit box.

    Both layers use nx x nx columns in x, z; the slab |y-0.5| < 0.25 holds
    ny_dense layers and the outside ny_light layers, so the number-density
    ratio is ny_dense/ny_light (21/11 = 1.91 at the default 32^3 particles).
    Masses are equal and set so the outer density is 1; u = P/((gamma-1) rho)
    with the nominal layer density; vx = +shear inside the slab, -shear outside.
    """
    rng = _rng(index)
    dxz = 1.0 / nx
    gx = (np.arange(nx) + 0.5) * dxz
    yd = 0.25 + (np.arange(ny_dense) + 0.5) * (0.5 / ny_dense)
    yl = np.concatenate([(np.arange(ny_light) + 0.5) * (0.5 / ny_light) + 0.75, ])
    yl = np.mod(yl, 1.0)
    def layer(ys):
        X, Y, Z = np.meshgrid(gx, ys, gx, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    pd, pl = layer(yd), layer(yl)
    sp_d = np.array([dxz, 0.5 / ny_dense, dxz])
    sp_l = np.array([dxz, 0.5 / ny_light, dxz])
    pd = pd + rng.uniform(-1, 1, size=pd.shape) * jitter * sp_d
    pl = pl + rng.uniform(-1, 1, size=pl.shape) * jitter * sp_l
    pos = np.concatenate([pd, pl], 0)
    n = len(pos)
    n_light_density = len(pl) / 0.5
    m = 1.0 / n_light_density
    rho_d, rho_l = len(pd) / 0.5 * m, 1.0
    inside = np.concatenate([np.ones(len(pd), bool), np.zeros(len(pl), bool)])
    u = np.where(inside, pressure / ((GAMMA_EOS - 1) * rho_d), pressure / ((GAMMA_EOS - 1) * rho_l))
    vel = np.zeros((n, 3))
    vel[:, 0] = np.where(inside, shear, -shear)
    h = np.where(inside, ETA * np.cbrt(sp_d.prod()), ETA * np.cbrt(sp_l.prod()))
    return _finish(f"kh{n}", pos, vel, np.full(n, m), u, h, inside=inside)


def zeldovich(n_side: int = 256, index: int = 5, max_contrast: float = 100.0, spectral_index: float = -2.0):
    """Lattice displaced by a Zel'dovich field from a Gaussian random field with P(k) ~ k^n.

    psi_k = i k delta_k / k^2 (so div psi = -delta); the amplitude is set by
    bisection so that max over the grid of 1/det(I + grad psi) equals
    max_contrast. Velocities equal the displacement, u = 1, h = eta / n_side.
    """
    rng = _rng(index)
    n = n_side
    noise = rng.normal(size=(n, n, n))
    dk = np.fft.rfftn(noise)
    k1 = np.fft.fftfreq(n, 1.0 / n) * 2 * np.pi
    kz = np.fft.rfftfreq(n, 1.0 / n) * 2 * np.pi
    KX, KY, KZ = np.meshgrid(k1, k1, kz, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k2[0, 0, 0] = 1.0
    amp = np.sqrt(k2 ** (spectral_index / 2.0))
    amp[0, 0, 0] = 0.0
    dk = dk * amp
    ks = (KX, KY, KZ)
    psi = [np.fft.irfftn(1j * kk * dk / k2, s=(n, n, n), axes=(0, 1, 2)) for kk in ks]
    grad = [[np.fft.irfftn(-ks[a] * ks[b] * dk / k2, s=(n, n, n), axes=(0, 1, 2)).ravel() for b in range(3)] for a in range(3)]
    # det(I + A J) = 1 + A tr J + A^2 (sum of the principal 2x2 minors) + A^3 det J, per grid point
    J = grad  # J[a][b] = d psi_a / d q_b
    tr = J[0][0] + J[1][1] + J[2][2]
    m2 = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) + (J[0][0] * J[2][2] - J[0][2] * J[2][0]) + \
         (J[1][1] * J[2][2] - J[1][2] * J[2][1])
    dt = (J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
          + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]))
    del grad, J

    def min_det(A):
        return (1.0 + A * (tr + A * (m2 + A * dt))).min()

    target = 1.0 / max_contrast
    lo, hi = 0.0, 1.0
    while min_det(hi) > target:
        hi *= 2.0
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        if min_det(mid) > target:
            lo = mid
        else:
            hi = mid
    A = lo
    g = (np.arange(n) + 0.5) / n
    Q = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    disp = A * np.stack([p.ravel() for p in psi], 1)
    pos = Q + disp
    N = len(pos)
    return _finish(f"zeldovich{n}", pos, disp, np.full(N, 1.0 / N), np.ones(N), np.full(N, ETA / n),
                   amplitude=A)


def gresho_profile(r):
    """Analytic Gresho-Chan vortex (Eqs. 27-28): azimuthal speed v_phi(r) and pressure p(r)."""
    r = np.asarray(r, np.float64)
    v = np.where(r < 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))
    rs = np.maximum(r, 1e-300)
    p_mid = 9.0 - 4.0 * np.log(0.2) + 12.5 * r * r - 20.0 * r + 4.0 * np.log(rs)
    p = np.where(r < 0.2, 5.0 + 12.5 * r * r, np.where(r < 0.4, p_mid, 3.0 + 4.0 * np.log(2.0)))
    return v, p


def gresho(n_side: int = 64, jitter: float = 0.0, index: int = 6, rho0: float = 1.0):
    """Gresho-Chan vortex on an n_side^3 cubic lattice (Sec. 3.1).

    Axis along z through (0.5, 0.5); v = v_phi(r) (-(y - 0.5), x - 0.5, 0) / r
    with r the distance from the axis in the x-y plane; rho = rho0 (m = rho0 /
    N), u = p(r) / ((gamma - 1) rho0), h = eta / n_side.
    """
    rng = _rng(index)
    dx = 1.0 / n_side
    g = (np.arange(n_side) + 0.5) * dx
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    if jitter > 0:
        pos = pos + rng.uniform(-jitter * dx, jitter * dx, size=pos.shape)
    pos = _wrap(pos)
    rx, ry = pos[:, 0] - 0.5, pos[:, 1] - 0.5
    r = np.sqrt(rx * rx + ry * ry)
    vphi, p = gresho_profile(r)
    rs = np.where(r > 0, r, 1.0)
    vel = np.stack([-vphi * ry / rs, vphi * rx / rs, np.zeros_like(r)], 1)
    n = len(pos)
    u = p / ((GAMMA_EOS - 1.0) * rho0)
    return _finish(f"gresho{n_side}", pos, vel, np.full(n, rho0 / n), u, np.full(n, ETA * dx), spacing=dx)


CONFIGS = {
    "lattice16": lambda: lattice(16),
    "sedov64": lambda: sedov(64),
    "plummer2M": lambda: plummer(),
    "kh32": lambda: kh(),
    "zeldovich256": lambda: zeldovich(256),
    "gresho64": lambda: gresho(64),
    "gresho128": lambda: gresho(128),
}
