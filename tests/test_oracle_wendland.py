"""Pins of the oracle's Wendland C2 and C4 kernels (Sec. 2.1.1 names them beside
the cubic spline), CPU only.

Each check rests on something the oracle does not compute itself: quadrature
of the kernel (normalisation, and H/h from the second-moment definition
h = 2 sigma), finite differences of W in r and of n in h, the order of the
kernel's contact with zero at the support edge, lattice sums converging to
the continuum integral as the resolution grows, the h iteration reaching its
target, and the conservation laws of the pairwise force loop.
"""
import numpy as np
import pytest
from scipy import integrate

from paper_2505_14538_b300 import ics

WENDLAND = {1: (np.sqrt(15.0) / 2.0, 4), 2: (np.sqrt(78.0) / 4.0, 6)}  # kind: (exact H/h, (1-q)^k at the edge)


def perfect_lattice(n_side):
    dx = 1.0 / n_side
    g = (np.arange(n_side) + 0.5) * dx
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1), dx


@pytest.mark.parametrize("kind", [1, 2])
def test_normalisation_and_second_moment(O, kind):
    kg = O.KERNEL_GAMMAS[kind]
    h = 0.41
    H = kg * h
    W = lambda r: O.kernel(np.array([r]), h, kg, kind)[0][0]
    norm = integrate.quad(lambda r: 4 * np.pi * r * r * W(r), 0, H, epsabs=1e-14)[0]
    assert abs(norm - 1.0) < 1e-10
    m2 = integrate.quad(lambda r: 4 * np.pi * r ** 4 * W(r), 0, H, epsabs=1e-14)[0]
    sigma = np.sqrt(m2 / 3.0)
    assert abs(H / (2 * sigma) - WENDLAND[kind][0]) < 2e-7  # the float32 H/h
    assert abs(2 * sigma / h - 1.0) < 2e-7


@pytest.mark.parametrize("kind", [1, 2])
def test_derivative_and_contact_at_the_edge(O, kind):
    kg = O.KERNEL_GAMMAS[kind]
    h = 0.05
    H = kg * h
    r = np.linspace(1e-4, 1.2 * H, 2001)
    eps = 1e-7
    Wp, _ = O.kernel(r + eps, h, kg, kind)
    Wm, _ = O.kernel(r - eps, h, kg, kind)
    W, dW = O.kernel(r, h, kg, kind)
    assert np.max(np.abs((Wp - Wm) / (2 * eps) - dW)) < 1e-6 * np.abs(dW).max()
    assert np.all(W >= 0) and np.all(np.diff(W) <= 0) and np.all(W[r >= H] == 0)
    # W ~ (1 - q)^k at the edge: halving the distance to it divides W by 2^k
    e = 1e-3
    Wa, _ = O.kernel(np.array([H * (1 - e), H * (1 - 2 * e)]), h, kg, kind)
    assert Wa[1] / Wa[0] == pytest.approx(2.0 ** WENDLAND[kind][1], rel=2e-2)


@pytest.mark.parametrize("kind", [1, 2])
def test_lattice_sum_tends_to_the_integral(O, kind):
    """n dx^3 on a perfect lattice approaches the continuum value 1 as h / dx grows."""
    x, dx = perfect_lattice(12)
    n = len(x)
    p = O.Params(kernel=kind, kernel_gamma=O.KERNEL_GAMMAS[kind])
    errs = []
    for eta in (1.2348, 1.5, 2.0):
        d = O.density(p, x, np.zeros((n, 3)), np.full(n, 1.0 / n), np.full(n, eta * dx))
        errs.append(abs(d["n"].mean() * dx ** 3 - 1.0))
        assert np.allclose(d["n"], d["n"][0], rtol=1e-12)
    assert errs[2] < errs[1] < errs[0] < 0.02 and errs[2] < 1e-3


@pytest.mark.parametrize("kind", [1, 2])
def test_dn_dh_finite_difference_and_h_solution(O, kind):
    d0 = ics.lattice(9, jitter=0.25)
    n = len(d0["pos"])
    p = O.Params(kernel=kind, kernel_gamma=O.KERNEL_GAMMAS[kind], h_tol=1e-12, h_max=0.3)
    h = d0["h"].astype(np.float64)
    d = O.density(p, d0["pos"], np.zeros((n, 3)), d0["m"], h)
    eps = 1e-7 * h
    dp = O.density(p, d0["pos"], np.zeros((n, 3)), d0["m"], h + eps)
    dm = O.density(p, d0["pos"], np.zeros((n, 3)), d0["m"], h - eps)
    fd = (dp["n"] - dm["n"]) / (2 * eps)
    assert np.allclose(d["dn_dh"], fd, rtol=2e-6, atol=1e-6 * np.abs(d["dn_dh"]).max())
    s = O.solve_h(p, d0["pos"], np.zeros((n, 3)), d0["m"], h)
    assert s["converged"].all()
    assert np.abs(s["n"] * s["h"] ** 3 / p.eta ** 3 - 1).max() < 1e-12


@pytest.mark.parametrize("kind", [1, 2])
def test_conservation_with_wendland(O, kind):
    rng = np.random.default_rng(3 + kind)
    d0 = ics.lattice(9, jitter=0.2)
    n = len(d0["pos"])
    m = d0["m"].astype(np.float64)
    v = rng.normal(0, 0.3, (n, 3))
    u = rng.uniform(0.5, 1.5, n)
    p = O.Params(kernel=kind, kernel_gamma=O.KERNEL_GAMMAS[kind], h_tol=1e-12, h_max=0.3)
    s = O.step(p, d0["pos"], v, m, u, d0["h"])
    ma = m[:, None] * s["accel"]
    assert np.abs(ma.sum(0)).max() < 1e-13 * np.abs(ma).sum()
    e = (m * ((v * s["accel"]).sum(1) + s["dudt"])).sum()
    assert abs(e) < 1e-13 * (m * (np.abs((v * s["accel"]).sum(1)) + np.abs(s["dudt"]))).sum()
    # and a static perfect lattice feels no force
    x, dx = perfect_lattice(10)
    nn = len(x)
    st = O.step(p, x, np.zeros((nn, 3)), np.full(nn, 1.0 / nn), np.ones(nn), np.full(nn, ics.ETA * dx))
    assert np.abs(st["accel"]).max() < 1e-12 * st["s_a"].max() and np.abs(st["dudt"]).max() == 0
