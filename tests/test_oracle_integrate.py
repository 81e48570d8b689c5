"""Pins of the FP64 integration oracle (oracle/integrate.py) against what the
mathematics fixes, independent of the formulas the oracle is written from:
exact motion under constant acceleration, second-order convergence and time
reversibility of the leapfrog on a harmonic oscillator, the closed-form decay
and rise of the switches, the first-order convergence of the Euler step of
Eq. 21 to its exponential solution, and conservation over whole SPH steps.
"""
import numpy as np
import pytest

from oracle import integrate as I

KG = I.O.KERNEL_GAMMA
BOX = (1000.0, 1000.0, 1000.0)  # no wrap in the oscillator runs


def leapfrog(tp, x, v, accel, dt, steps):
    """Drive kick_drift / kick_finish with a position-dependent acceleration."""
    n = len(x)
    u = np.ones(n)
    z = np.zeros(n)
    h = np.ones(n)
    a = accel(x)
    for _ in range(steps):
        kd = I.kick_drift(tp, BOX, dt, x, v, u, a, z, h, z)
        x = kd["x"]
        a = accel(x)
        kf = I.kick_finish(tp, KG, dt, h, kd["v"], kd["u"], a, z, z, z, z, None)
        v = kf["v"]
    return x, v


def test_constant_acceleration_is_exact():
    tp = I.TimeParams()
    rng = np.random.default_rng(0)
    x0 = 500.0 + rng.normal(size=(5, 3))
    v0 = rng.normal(size=(5, 3))
    g = rng.normal(size=(5, 3))
    dt = 0.37
    z, one = np.zeros(5), np.ones(5)
    kd = I.kick_drift(tp, BOX, dt, x0, v0, one, g, z, one, z)
    assert np.allclose(kd["x"], x0 + v0 * dt + 0.5 * g * dt * dt, rtol=0, atol=1e-12)
    assert np.allclose(kd["v_pred"], v0 + g * dt, rtol=0, atol=1e-13)
    kf = I.kick_finish(tp, KG, dt, one, kd["v"], kd["u"], g, z, z, z, z, None)
    assert np.allclose(kf["v"], v0 + g * dt, rtol=0, atol=1e-13)


def test_oscillator_second_order_reversible_bounded_energy():
    tp = I.TimeParams()
    w = 2.0 * np.pi
    c = 500.0
    x0 = np.array([[c + 0.1, c, c], [c, c - 0.2, c], [c + 0.05, c + 0.05, c - 0.3]])
    v0 = np.array([[0.0, 0.3, 0.0], [0.1, 0.0, 0.0], [0.0, 0.0, 0.2]])
    acc = lambda x: -w * w * (x - c)
    exact = lambda t: (c + (x0 - c) * np.cos(w * t) + v0 / w * np.sin(w * t))
    errs = []
    for dt in (0.01, 0.005):
        x, _ = leapfrog(tp, x0, v0, acc, dt, int(round(1.0 / dt)))
        errs.append(np.abs(x - exact(1.0)).max())
    assert 3.6 < errs[0] / errs[1] < 4.4  # second order
    # time reversal: 200 steps forward, flip v, 200 steps back
    x, v = leapfrog(tp, x0, v0, acc, 0.01, 200)
    xb, vb = leapfrog(tp, x, -v, acc, 0.01, 200)
    assert np.abs(xb - x0).max() < 1e-10 and np.abs(vb + v0).max() < 1e-10
    # energy error O((w dt)^2) and bounded: its envelope over the last ten
    # periods of fifty is the one over the first ten (no secular drift)
    E = lambda x, v: 0.5 * (v * v).sum() + 0.5 * w * w * ((x - c) ** 2).sum()
    E0 = E(x0, v0)
    x, v, dev = x0, v0, []
    for k in range(5000):
        x, v = leapfrog(tp, x, v, acc, 0.01, 1)
        dev.append(abs(E(x, v) / E0 - 1))
    assert max(dev) < (w * 0.01) ** 2
    assert max(dev[4000:]) < 1.1 * max(dev[:1000])


def test_drift_wraps_and_h_follows_exponential():
    tp = I.TimeParams()
    x = np.array([[0.995, 0.5, 0.002]])
    v = np.array([[1.0, 0.0, -1.0]])
    z1 = np.zeros(1)
    k = 3.0
    h = np.array([0.02])
    kd = I.kick_drift(tp, (1.0, 1.0, 1.0), 0.01, x, v, np.ones(1), np.zeros((1, 3)), z1, h, k * h)
    assert np.allclose(kd["x"], [[0.005, 0.5, 0.992]], atol=1e-15)
    # dh/dt = k h has the solution h e^{k t}; the drift is exact for it
    assert np.isclose(kd["h"][0], 0.02 * np.exp(k * 0.01), rtol=1e-15)


def test_half_kick_never_more_than_halves_u():
    tp = I.TimeParams()
    u = np.array([2.0, 2.0])
    dudt = np.array([-1e6, 10.0])
    kd = I.kick_drift(tp, (1.0, 1.0, 1.0), 0.1, np.full((2, 3), 0.5), np.zeros((2, 3)), u, np.zeros((2, 3)),
                      dudt, np.full(2, 0.01), np.zeros(2))
    assert np.allclose(kd["u"], [1.0, 2.5]) and np.allclose(kd["u_pred"], [0.5, 3.0])


def _visc(tp, dt, h, u, div, div_prev, vsig, alpha):
    return I.viscosity_switch(tp, 5.0 / 3.0, KG, dt, h, u, div, div_prev, vsig, alpha)


def test_viscosity_switch_closed_forms():
    tp = I.TimeParams()
    h, u, vs = np.array([0.01]), np.array([1.5]), np.array([3.0])
    H = KG * h
    c = np.sqrt(5.0 / 3.0 * (2.0 / 3.0) * u)
    # no compression: alpha decays as alpha0 exp(-l c t / H) however t is split into steps
    T = 0.002
    a1, _ = _visc(tp, T, h, u, np.zeros(1), np.zeros(1), vs, np.array([1.2]))
    a7 = np.array([1.2])
    for _ in range(7):
        a7, _ = _visc(tp, T / 7, h, u, np.zeros(1), np.zeros(1), vs, a7)
    ref = 1.2 * np.exp(-0.05 * c * T / H)
    assert np.allclose(a1, ref, rtol=1e-14) and np.allclose(a7, ref, rtol=1e-13)
    # S = v_sig^2 gives alpha_loc = alpha_max / 2, taken at once from below
    dt = 1e-3
    div = -(vs * vs) * dt / (H * H)
    a, dp = _visc(tp, dt, h, u, div, np.zeros(1), vs, np.zeros(1))
    assert np.allclose(a, tp.alpha_v_max / 2, rtol=1e-14) and np.array_equal(dp, div)
    # very strong compression: alpha -> alpha_max
    a, _ = _visc(tp, dt, h, u, 1e6 * div, np.zeros(1), vs, np.zeros(1))
    assert tp.alpha_v_max * (1 - 1e-5) < a[0] <= tp.alpha_v_max
    # expansion is not compression: decay only
    a, _ = _visc(tp, dt, h, u, -div, np.zeros(1), vs, np.array([0.8]))
    assert np.allclose(a, 0.8 * np.exp(-0.05 * c * dt / H), rtol=1e-14)
    # above alpha_loc it relaxes toward alpha_loc, staying between the two
    a, _ = _visc(tp, dt, h, u, div, np.zeros(1), vs, np.array([1.5]))
    assert 1.0 < a[0] < 1.5
    # dt = 0: alpha unchanged, div_prev refreshed
    a, dp = _visc(tp, 0.0, h, u, np.array([7.0]), np.array([1.0]), vs, np.array([0.3]))
    assert a[0] == 0.3 and dp[0] == 7.0


def test_diffusion_switch_converges_to_exponentials():
    tp = I.TimeParams(alpha_c_max=100.0)
    h, u = np.array([0.02]), np.array([4.0])
    H = KG * h
    T = 0.01

    def run(nsteps, lapu, vsig, a0):
        a = np.array([a0])
        for _ in range(nsteps):
            a = I.diffusion_switch(tp, KG, T / nsteps, h, u, np.array([lapu]), np.array([vsig]), np.zeros(1), a)
        return a[0]

    # decay toward alpha_min = 0 at rate v/H
    ref = 0.7 * np.exp(-5.0 * T / H[0])
    e1, e2 = abs(run(20, 0.0, 5.0, 0.7) - ref), abs(run(40, 0.0, 5.0, 0.7) - ref)
    assert 1.8 < e1 / e2 < 2.2  # first order
    # growth at rate beta_c H lap(u) / sqrt(u) (Eq. 21 as printed)
    g = 30.0
    ref = 0.1 * np.exp(tp.beta_c * H[0] * g / np.sqrt(4.0) * T)
    e1, e2 = abs(run(20, g, 0.0, 0.1) - ref), abs(run(40, g, 0.0, 0.1) - ref)
    assert 1.8 < e1 / e2 < 2.2 and run(400, g, 0.0, 0.1) == pytest.approx(ref, rel=1e-3)


def test_diffusion_cap_follows_viscosity():
    tp = I.TimeParams()
    h, u = np.array([0.02, 0.02]), np.array([1.0, 1.0])
    a = I.diffusion_switch(tp, KG, 1e-4, h, u, np.zeros(2), np.zeros(2),
                           np.array([tp.alpha_v_max, tp.alpha_v_max / 2]), np.array([0.9, 0.9]))
    assert a[0] == tp.alpha_c_min and np.isclose(a[1], tp.alpha_c_max / 2, rtol=1e-15)


def test_step_size():
    tp = I.TimeParams(cfl=0.2)
    h = np.array([0.01, 0.02, 0.005])
    vs = np.array([2.0, 1.0, 0.0])  # the last particle sets no bound
    assert I.step_size(tp, KG, h, vs) == pytest.approx(0.2 * 2 * KG * 0.01 / 2.0, rel=1e-15)
    assert I.step_size(I.TimeParams(cfl=0.2, dt_max=1e-4), KG, h, vs) == 1e-4
    assert I.step_size(tp, KG, h, vs, t=0.1, t_end=0.1 + 1e-6) == pytest.approx(1e-6, rel=1e-9)
    assert I.step_size(tp, KG, h, vs, t=0.2, t_end=0.1) == 0.0


def test_full_steps_conserve_momentum_and_energy(O):
    """Whole SPH steps (loops from the C++ oracle): momentum to rounding, energy to O(dt^2)."""
    from paper_2505_14538_b300 import ics
    d = ics.lattice(8, jitter=0.2, index=11)
    rng = np.random.default_rng(5)
    n = len(d["pos"])
    v = rng.normal(0, 0.3, size=(n, 3))
    u = rng.uniform(0.5, 1.5, n)
    p = O.Params(h_tol=1e-12)
    tp = I.TimeParams()
    st = I.prime(p, tp, d["pos"], v, d["m"], u, d["h"], np.full(n, 1.0), np.full(n, 0.5))
    m = st["m"]
    P0 = (m[:, None] * st["v"]).sum(0)
    scale = (m[:, None] * np.abs(st["v"])).sum()
    E = lambda s: (m * (0.5 * (s["v"] ** 2).sum(1) + s["u"])).sum()
    E0 = E(st)
    for _ in range(3):
        st = I.step(p, tp, st)
        assert np.abs((m[:, None] * st["v"]).sum(0) - P0).max() < 1e-13 * scale
    assert abs(E(st) / E0 - 1) < 1e-4
    assert st["t"] > 0 and np.all(st["alpha_v"] >= 0) and np.all(st["alpha_c"] >= 0)
