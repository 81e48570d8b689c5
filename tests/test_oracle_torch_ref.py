"""Pins of the PyTorch FP64 gradient reference (CPU only).

Its forward must reproduce the C++ oracle's accelerations and du/dt at fixed
h, and its autograd gradient must match central finite differences of the
C++ oracle's loss: the two are independent restatements of the equations.
"""
import numpy as np
import pytest

from paper_2505_14538_b300 import ics


def _state(seed=0, n_side=8, jitter=0.3):
    d = ics.lattice(n_side, jitter=jitter)
    rng = np.random.default_rng(seed)
    n = len(d["pos"])
    x = d["pos"].astype(np.float64)
    v = rng.normal(0, 0.3, (n, 3))
    u = d["u"] * rng.uniform(0.5, 1.5, n)
    h = d["h"].astype(np.float64) * rng.uniform(0.9, 1.1, n)
    w = rng.normal(size=(n, 3))
    cw = rng.normal(size=n)
    return x, v, u, d["m"].astype(np.float64), h, w, cw


def _oracle_loss(O, x, v, u, m, h, w, cw):
    s = O.step(O.Params(), x, v, m, u, h, solve=False)
    return float((w * s["accel"]).sum() + (cw * s["dudt"]).sum()), s


def test_torch_forward_matches_oracle(O):
    from oracle import torch_ref as T
    x, v, u, m, h, w, cw = _state()
    L, gx, gv, gu, a, du = T.loss_and_grad(x, v, u, m, h, w, cw)
    L0, s = _oracle_loss(O, x, v, m=m, u=u, h=h, w=w, cw=cw)
    assert np.all(np.linalg.norm(a - s["accel"], axis=1) <= 1e-11 * s["s_a"])
    assert np.all(np.abs(du - s["dudt"]) <= 1e-11 * s["s_u"])
    assert abs(L - L0) <= 1e-10 * (np.abs(w).sum(1) @ s["s_a"] + np.abs(cw) @ s["s_u"])


def test_torch_gradient_matches_oracle_finite_differences(O):
    """Central differences of the C++ oracle's loss (fixed h) on sampled components."""
    from oracle import torch_ref as T
    x, v, u, m, h, w, cw = _state(seed=3)
    n = len(x)
    L, gx, gv, gu, a, du = T.loss_and_grad(x, v, u, m, h, w, cw)
    rng = np.random.default_rng(9)
    scale = {"x": np.abs(gx).max(), "v": np.abs(gv).max(), "u": np.abs(gu).max()}
    checked = 0
    for k in rng.choice(n, 6, replace=False):
        for name, comp in (("x", 0), ("x", 2), ("v", 1), ("u", None)):
            arr = {"x": x, "v": v, "u": u}[name]
            ref = {"x": gx, "v": gv, "u": gu}[name]
            base = arr[k, comp] if comp is not None else arr[k]
            fd = []
            for delta in (1e-6 * max(abs(base), 0.05), 5e-7 * max(abs(base), 0.05)):
                vals = []
                for sgn in (1, -1):
                    a2 = arr.copy()
                    if comp is None:
                        a2[k] += sgn * delta
                    else:
                        a2[k, comp] += sgn * delta
                    args = dict(x=x, v=v, u=u)
                    args[name] = a2
                    vals.append(_oracle_loss(O, args["x"], args["v"], args["u"], m, h, w, cw)[0])
                fd.append((vals[0] - vals[1]) / (2 * delta))
            if abs(fd[0] - fd[1]) > 1e-5 * scale[name]:
                continue  # a kink (support edge, mu = 0, |.|) inside the stencil
            g = ref[k, comp] if comp is not None else ref[k]
            assert abs(g - fd[0]) <= 1e-5 * scale[name], (name, k, comp, g, fd[0])
            checked += 1
    assert checked >= 18


@pytest.mark.parametrize("kind", [1, 2])
def test_torch_forward_matches_oracle_wendland(O, kind):
    """The two restatements agree for the Wendland kernels too (same pair set, kernel's own H/h)."""
    from oracle import torch_ref as T
    x, v, u, m, h, w, cw = _state(seed=kind)
    kg = O.KERNEL_GAMMAS[kind]
    L, gx, gv, gu, a, du = T.loss_and_grad(x, v, u, m, h, w, cw, kernel_gamma=kg, kernel=kind)
    s = O.step(O.Params(kernel=kind, kernel_gamma=kg), x, v, m, u, h, solve=False)
    assert np.all(np.linalg.norm(a - s["accel"], axis=1) <= 1e-11 * s["s_a"])
    assert np.all(np.abs(du - s["dudt"]) <= 1e-11 * s["s_u"])


def test_hsolved_gradient_matches_oracle_finite_differences(O):
    """h = h(x) (the root of the h iteration): the IFT gradient against central differences of the C++
    oracle's loss with h re-solved at every perturbed position (to 1e-13)."""
    from oracle import torch_ref as T
    x, v, u, m, h0, w, cw = _state(seed=3, n_side=7, jitter=0.3)
    p = O.Params(h_tol=1e-14, max_iter=80, h_max=0.4)
    h = O.solve_h(p, x, v, m, h0)["h"]
    L, gx, gv, gu, gh, lam = T.loss_and_grad_hsolved(x, v, u, m, h, w, cw)
    assert np.abs(gh).max() > 0 and np.abs(lam).max() > 0

    def loss(xx, vv, uu):
        s = O.step(p, xx, vv, m, uu, h)  # solve=True: h re-solved from h as the start
        return float((w * s["accel"]).sum() + (cw * s["dudt"]).sum())

    assert abs(loss(x, v, u) - L) < 1e-9 * abs(L) + 1e-12
    rng = np.random.default_rng(9)
    scale = np.abs(gx).max()
    fixed_h = T.loss_and_grad(x, v, u, m, h, w, cw)[1]
    moved = 0
    for k in rng.choice(len(x), 6, replace=False):
        for c in range(3):
            fds = []
            for delta in (2e-6, 1e-6):
                xp, xm = x.copy(), x.copy()
                xp[k, c] += delta
                xm[k, c] -= delta
                fds.append((loss(xp, v, u) - loss(xm, v, u)) / (2 * delta))
            assert abs(fds[0] - fds[1]) < 1e-4 * scale  # smooth here (no support edge crossed)
            assert abs(gx[k, c] - fds[1]) < 1e-5 * scale, (k, c, gx[k, c], fds[1])
            moved += abs(gx[k, c] - fixed_h[k, c]) > 1e-3 * scale
    assert moved > 0  # the h term matters at this tolerance
