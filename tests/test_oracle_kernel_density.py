"""Pins of the oracle's kernel, neighbour search and density loop (CPU only).

Each test checks the oracle against something it does not compute itself:
quadrature of the kernel, a library neighbour search, a lattice sum written
out over integer offsets, finite differences, and symmetry identities.
"""
import numpy as np
import pytest
from scipy import integrate
from scipy.spatial import cKDTree

from paper_2505_14538_b300 import ics

KG = float(np.float32(1.825742))


def perfect_lattice(n_side, periodic=True):
    dx = 1.0 / n_side
    g = (np.arange(n_side) + 0.5) * dx
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1), dx


def test_kernel_normalisation_and_second_moment(O):
    """Integral of W over R^3 is 1; h = 2 sigma fixes H/h (cubic spline, Sec. 2.1.3 H = gamma_k h)."""
    h = 0.37
    W = lambda r: O.kernel(np.array([r]), h)[0][0]
    H = KG * h
    norm = integrate.quad(lambda r: 4 * np.pi * r * r * W(r), 0, H, points=[0.5 * H], epsabs=1e-13)[0]
    assert abs(norm - 1.0) < 1e-10
    m2 = integrate.quad(lambda r: 4 * np.pi * r ** 4 * W(r), 0, H, points=[0.5 * H], epsabs=1e-13)[0]
    sigma = np.sqrt(m2 / 3.0)
    assert abs(H / (2 * sigma) - 1.8257418583505538) < 1e-12 * 0 + 2e-7  # float32 gamma_k
    assert abs((2 * sigma) / h - 1.0) < 1e-6


def test_kernel_derivative_and_support(O):
    h = 0.05
    H = KG * h
    r = np.linspace(1e-4, 1.2 * H, 2001)
    eps = 1e-7
    Wp, _ = O.kernel(r + eps, h)
    Wm, _ = O.kernel(r - eps, h)
    _, dW = O.kernel(r, h)
    fd = (Wp - Wm) / (2 * eps)
    scale = np.abs(dW).max()
    assert np.max(np.abs(fd - dW)) < 1e-6 * scale
    W, dW = O.kernel(np.array([H, 1.5 * H, 0.5 * H * (1 - 1e-12), 0.5 * H * (1 + 1e-12)]), h)
    assert W[0] == 0 and W[1] == 0 and dW[0] == 0
    assert abs(W[2] - W[3]) < 1e-9 * W[2]           # continuous at q = 1/2
    assert abs(dW[2] - dW[3]) < 1e-9 * abs(dW[2])   # C1 at q = 1/2


def test_cell_ids_definition(O):
    nc = 7
    L = 1.0
    edges = np.arange(nc) / nc
    x = np.stack([edges, np.nextafter(edges, -1.0), edges], 1)
    ids = O.cell_ids(x, (L, L, L), nc)
    cx = ids % nc
    cy = (ids // nc) % nc
    k = np.arange(nc)
    # floor(x nc / L) on exact cell boundaries can round either way in FP64; check against the definition
    assert np.array_equal(cx, np.floor(edges * nc / L).astype(int).clip(0, nc - 1))
    assert np.array_equal(cy[1:], (k[1:] - 1))          # just below a boundary -> previous cell
    assert cy[0] == nc - 1                              # just below 0 wraps to the last cell
    # periodic wrap: x and x - L land in the same cell
    y = np.random.default_rng(0).uniform(0, 1, (1000, 3))
    assert np.array_equal(O.cell_ids(y, (L, L, L), nc), O.cell_ids(y - 1.0, (L, L, L), nc))


@pytest.mark.parametrize("periodic", [True, False])
def test_neighbour_counts_against_kdtree(O, periodic):
    """Integer neighbour counts (r < H_i, j != i) equal a library range search."""
    rng = np.random.default_rng(3)
    n = 1500
    x = rng.uniform(0, 1, (n, 3))
    h = rng.uniform(0.04, 0.09, n)
    p = O.Params(periodic=periodic, use_cells=False)
    d = O.density(p, x, np.zeros((n, 3)), np.full(n, 1.0 / n), h)
    tree = cKDTree(x, boxsize=1.0 if periodic else None)
    ref = np.array([len(tree.query_ball_point(x[i], KG * h[i] * (1 - 1e-12))) - 1 for i in range(n)])
    assert np.array_equal(d["ngb"], ref)


def test_cell_list_equals_brute_force(O):
    d0 = ics.lattice(12, jitter=0.3)
    n = len(d0["pos"])
    rng = np.random.default_rng(5)
    v = rng.normal(size=(n, 3))
    h = d0["h"] * rng.uniform(0.8, 1.2, n)
    a = O.density(O.Params(use_cells=False), d0["pos"], v, d0["m"], h)
    b = O.density(O.Params(use_cells=True), d0["pos"], v, d0["m"], h)
    assert np.array_equal(a["ngb"], b["ngb"])
    for k in ("n", "dn_dh", "rho", "drho_dh", "div", "curl"):
        assert np.allclose(a[k], b[k], rtol=1e-12, atol=1e-12 * np.abs(a[k]).max())


def test_lattice_density_closed_form(O):
    """Perfect lattice, h = eta*spacing: n * spacing^3 equals the lattice sum over integer offsets."""
    x, dx = perfect_lattice(12)
    n = len(x)
    h = np.full(n, ics.ETA * dx)
    d = O.density(O.Params(), x, np.zeros((n, 3)), np.full(n, 1.0 / n), h)
    H = KG * ics.ETA  # in units of the spacing
    k = np.arange(-4, 5)
    K = np.array(np.meshgrid(k, k, k, indexing="ij")).reshape(3, -1).T
    q = np.sqrt((K ** 2).sum(1)) / H
    w = np.where(q < 0.5, 1 - 6 * q ** 2 + 6 * q ** 3, np.where(q < 1, 2 * (1 - q) ** 3, 0.0))
    ref = 8 / np.pi / H ** 3 * w.sum()
    assert abs(ref - 1.0039808) < 1e-7
    assert np.allclose(d["n"] * dx ** 3, ref, rtol=1e-12)
    assert np.all(d["ngb"] == 56)
    assert np.allclose(d["rho"], d["n"] / n, rtol=1e-12)


def test_partition_of_unity_on_lattice(O):
    """Eq. 1 with Q = 1 on a perfect lattice with uniform h returns exactly 1."""
    x, dx = perfect_lattice(10)
    n = len(x)
    h = np.full(n, 1.1 * dx)
    m = np.full(n, 1.0 / n)
    d = O.density(O.Params(), x, np.zeros((n, 3)), m, h)
    one = O.interpolate(O.Params(), x, m, h, d["rho"], np.ones(n))
    assert np.allclose(one, 1.0, rtol=0, atol=1e-13)
    # jittered lattice: close to 1, and the error shrinks with the jitter (loosely bounded)
    errs = []
    for jit in (0.1, 0.03, 0.01):
        dj = ics.lattice(10, jitter=jit)
        dd = O.density(O.Params(), dj["pos"], np.zeros((n, 3)), m, dj["h"])
        one_j = O.interpolate(O.Params(), dj["pos"], m, dj["h"], dd["rho"], np.ones(n))
        errs.append(np.abs(one_j - 1).max())
    assert errs[0] < 6e-2 and errs[2] < errs[1] < errs[0]


def test_dn_dh_and_drho_dh_match_finite_differences(O):
    """Eq. 6 (and its mass-weighted twin) against central differences of Eq. 5 / Eq. 2 in h."""
    d0 = ics.lattice(10, jitter=0.2)
    n = len(d0["pos"])
    h = d0["h"].astype(np.float64)
    p = O.Params()
    d = O.density(p, d0["pos"], np.zeros((n, 3)), d0["m"], h)
    eps = 1e-7 * h
    dp = O.density(p, d0["pos"], np.zeros((n, 3)), d0["m"], h + eps)
    dm = O.density(p, d0["pos"], np.zeros((n, 3)), d0["m"], h - eps)
    same = (dp["ngb"] == d["ngb"]) & (dm["ngb"] == d["ngb"])
    assert same.mean() > 0.9
    fd_n = (dp["n"] - dm["n"]) / (2 * eps)
    fd_r = (dp["rho"] - dm["rho"]) / (2 * eps)
    assert np.allclose(d["dn_dh"][same], fd_n[same], rtol=2e-6, atol=1e-6 * np.abs(d["dn_dh"]).max())
    assert np.allclose(d["drho_dh"][same], fd_r[same], rtol=2e-6, atol=1e-6 * np.abs(d["drho_dh"]).max())


def test_nh3_is_monotone_in_h(O):
    """n(h) h^3 never decreases with h, so F(h) has one root (uniqueness of the h solution)."""
    d0 = ics.lattice(8, jitter=0.3)
    n = len(d0["pos"])
    p = O.Params()
    prev = None
    for s in np.linspace(0.6, 1.6, 21):
        h = d0["h"] * s
        d = O.density(p, d0["pos"], np.zeros((n, 3)), d0["m"], h)
        cur = d["n"] * h.astype(np.float64) ** 3
        if prev is not None:
            assert np.all(cur >= prev * (1 - 1e-13))
        prev = cur


def _interior_lattice(n_side=14):
    x, dx = perfect_lattice(n_side)
    c = np.array([0.5, 0.5, 0.5])
    return x, dx, c


def test_div_curl_rotation_and_expansion(O):
    """Differenced Eq. 3/4 on a perfect lattice: v = s(x-c) and v = Omega x (x-c) share one lattice factor.

    Interior particles of a non-periodic lattice see a cubic-symmetric
    neighbourhood, so curl v = 2 Omega K and div v = 3 s K with the same K;
    the sign of the curl is that of the continuum curl.
    """
    x, dx, c = _interior_lattice()
    n = len(x)
    h = np.full(n, ics.ETA * dx)
    m = np.full(n, 1.0 / n)
    p = O.Params(periodic=False, use_cells=False)
    inner = np.all(np.abs(x - c) < 0.5 - 2.5 * dx, axis=1)
    s = 0.7
    de = O.density(p, x, s * (x - c), m, h)
    Om = np.array([0.3, -0.5, 0.8])
    dr = O.density(p, x, np.cross(Om, x - c), m, h)
    K_div = de["div"][inner] / (3 * s)
    K_curl = dr["curl"][inner] / (2 * Om)
    assert np.allclose(K_div, K_div[0], rtol=1e-12)
    assert np.allclose(K_curl, K_div[0], rtol=1e-10)
    assert abs(K_div[0] - 1) < 2e-2
    assert np.allclose(de["curl"][inner], 0, atol=1e-12)
    assert np.allclose(dr["div"][inner], 0, atol=1e-12)
    # Galilean invariance of the differenced form
    dg = O.density(p, x, np.cross(Om, x - c) + np.array([3.0, -1.0, 2.0]), m, h)
    assert np.allclose(dg["curl"], dr["curl"], rtol=1e-12, atol=1e-12)
    assert np.allclose(dg["div"], dr["div"], atol=1e-11)
