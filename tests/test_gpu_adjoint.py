"""GPU adjoint (swift_gpu_force_backward) against the FP64 references.

References: the PyTorch FP64 pair-list autograd of the same pipeline
(``oracle/torch_ref.py``, itself pinned to the C++ oracle and to its finite
differences) on every particle, and central finite differences of the C++
oracle on sampled components.

Tolerance, per element: |g - ref| <= 1e-4 |ref| + FLOOR max|ref|. The
floor is the FP32 rounding of the sums: a gradient component is a sum over
the pairs of two gathers (about 2 x 60 pair terms, each a chain of about 20
FP32 operations), so its error is at most about 100 x 2^-24 = 6e-6 times the
sum of its terms' magnitudes; with loss weights drawn from N(0, 1) the terms
of one component cancel, and their magnitudes add up to at most about 30 x the
array's largest component (3 sigma of a 100-term random sum), which bounds the
error by about 2e-4 max|ref|. Measured (FP64 torch reference, fixed and solved
h): at most 2.2e-5 max|ref|, most components below 1e-6 relative. FLOOR =
5e-5 lies between the two. A component that is 100 % wrong fails unless it is
below that floor.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_14538_b300 import ics

pytestmark = pytest.mark.gpu

FLOOR = 5e-5  # of the array's largest |component|: the FP32 rounding of the gathered sums (module docstring)


def _within(got, ref, what):
    """Per element |got - ref| <= 1e-4 |ref| + FLOOR max|ref|; returns the worst ratio to that bound."""
    bound = 1e-4 * np.abs(ref) + FLOOR * np.abs(ref).max()
    ratio = np.abs(got - ref) / bound
    worst = int(np.argmax(ratio))
    assert ratio.max() <= 1.0, (what, float(ratio.max()), float(np.ravel(got)[worst]), float(np.ravel(ref)[worst]),
                                float(np.abs(ref).max()))
    return float(ratio.max())


def _run_gpu(d, vel, u, w, cw):
    from paper_2505_14538_b300 import _lib, sph
    n = len(d["pos"])
    ctx = sph.Context(n, box=d["box"], flags=_lib.FLAG_NO_H_ITER)
    x = torch.from_numpy(d["pos"].astype(np.float32)).cuda().requires_grad_(True)
    v = torch.from_numpy(vel.astype(np.float32)).cuda().requires_grad_(True)
    uu = torch.from_numpy(u.astype(np.float32)).cuda().requires_grad_(True)
    m = torch.from_numpy(d["m"].astype(np.float32)).cuda()
    h = torch.from_numpy(d["h"].astype(np.float32)).cuda()
    a, du = sph.SphForces.apply(x, v, uu, m, h, ctx)
    L = (torch.from_numpy(w.astype(np.float32)).cuda() * a).sum() + (torch.from_numpy(cw.astype(np.float32)).cuda() * du).sum()
    L.backward()
    torch.cuda.synchronize()
    return x.grad.cpu().numpy(), v.grad.cpu().numpy(), uu.grad.cpu().numpy(), a.detach().cpu().numpy()


def _kink_mask(d, vel, u):
    """Particles of, or next to, a pair whose pressures agree to 1e-5 relative.

    The conduction signal speed (Eq. 22) holds sqrt(|P_i - P_j|), whose derivative is
    singular at P_i = P_j; there FP32 and FP64 gradients legitimately differ, so those
    particles (and the neighbours their density adjoints reach) are left out.
    """
    from oracle import torch_ref as T
    pairs = T.pair_list(d["pos"], d["h"], d["box"])
    x = torch.tensor(d["pos"].astype(np.float64))
    _, _, ex = T.forward(x, torch.tensor(vel.astype(np.float64)), torch.tensor(u.astype(np.float64)), d["m"],
                         d["h"], pairs, d["box"])
    P = ex["P"].numpy()
    i, j = pairs
    uu = np.asarray(u, np.float64)
    bad = (np.abs(P[i] - P[j]) < 1e-5 * (P[i] + P[j])) & (uu[i] != uu[j])  # the term carries u_i - u_j
    mask = np.zeros(len(P), bool)
    mask[i[bad]] = True
    mask[i[mask[j]]] = True
    return mask


def _cases():
    d1 = ics.kh(16, 11, 5)
    rng = np.random.default_rng(4)
    n = len(d1["pos"])
    yield "kh4096", d1, d1["vel"] + rng.normal(0, 0.05, (n, 3)).astype(np.float32), d1["u"]
    d2 = ics.lattice(12, jitter=0.3)
    rng = np.random.default_rng(5)
    n = len(d2["pos"])
    yield "lattice12", d2, rng.normal(0, 0.3, (n, 3)).astype(np.float32), (d2["u"] * rng.uniform(0.5, 1.5, n)).astype(np.float32)


@pytest.mark.parametrize("case", [0, 1])
def test_adjoint_matches_torch_fp64(case):
    from oracle import torch_ref as T
    name, d, vel, u = list(_cases())[case]
    n = len(d["pos"])
    rng = np.random.default_rng(100 + case)
    w = rng.normal(size=(n, 3))
    cw = rng.normal(size=n)
    gx, gv, gu, a = _run_gpu(d, vel, u, w, cw)
    L, rx, rv, ru, ra, rdu = T.loss_and_grad(d["pos"], vel, u, d["m"], d["h"], w, cw, box=d["box"])
    keep = ~_kink_mask(d, vel, u)
    assert keep.mean() > 0.9
    for got, ref, nm in ((gx, rx, "x"), (gv, rv, "v"), (gu, ru, "u")):
        _within(got[keep], ref[keep], (name, nm))


def test_adjoint_matches_oracle_finite_differences(O):
    name, d, vel, u = list(_cases())[1]
    n = len(d["pos"])
    rng = np.random.default_rng(7)
    w = rng.normal(size=(n, 3))
    cw = rng.normal(size=n)
    gx, gv, gu, a = _run_gpu(d, vel, u, w, cw)
    x = d["pos"].astype(np.float64)
    v = vel.astype(np.float64)
    uu = u.astype(np.float64)

    def loss(xx, vv, ux):
        s = O.step(O.Params(box=d["box"]), xx, vv, d["m"], ux, d["h"], solve=False)
        return float((w * s["accel"]).sum() + (cw * s["dudt"]).sum())

    scale = {"x": np.abs(gx).max(), "v": np.abs(gv).max(), "u": np.abs(gu).max()}
    keep = ~_kink_mask(d, vel, u)
    checked = 0
    for k in rng.choice(np.nonzero(keep)[0], 5, replace=False):
        for nm, comp in (("x", 0), ("x", 1), ("v", 2), ("u", None)):
            base = {"x": x, "v": v, "u": uu}[nm]
            fds = []
            for delta in (1e-6, 5e-7):
                vals = []
                for sg in (1, -1):
                    arr = base.copy()
                    if comp is None:
                        arr[k] += sg * delta * max(abs(base[k]), 0.05)
                    else:
                        arr[k, comp] += sg * delta * 0.05
                    args = {"x": x, "v": v, "u": uu}
                    args[nm] = arr
                    vals.append(loss(args["x"], args["v"], args["u"]))
                step = delta * (max(abs(base[k]), 0.05) if comp is None else 0.05)
                fds.append((vals[0] - vals[1]) / (2 * step))
            if abs(fds[0] - fds[1]) > 1e-5 * scale[nm]:
                continue
            got = {"x": gx, "v": gv, "u": gu}[nm]
            g = got[k, comp] if comp is not None else got[k]
            assert abs(g - fds[0]) <= 1e-4 * abs(fds[0]) + FLOOR * scale[nm], (nm, k, comp, g, fds[0])
            checked += 1
    assert checked >= 12


def test_adjoint_kh32_full_size_finite_differences(O):
    """The full 32^3 Kelvin-Helmholtz slab: GPU adjoint vs central differences of the oracle's loss.

    At fixed h, moving particle k changes only the densities within one support
    of it and the forces within two, so each difference quotient evaluates the
    oracle on the particles within 3.2 of the largest support (forces) and 4.3
    (densities) of k: the loss terms outside do not change. Samples lie more
    than three supports from the slab faces, where all neighbours share u (the
    conduction term, which carries u_i - u_j, is then smooth).
    """
    d = ics.kh()
    n = len(d["pos"])
    rng = np.random.default_rng(11)
    vel = (d["vel"] + rng.normal(0, 0.05, (n, 3))).astype(np.float32)
    u = d["u"].astype(np.float32)
    w = rng.normal(size=(n, 3))
    cw = rng.normal(size=n)
    gx, gv, gu, _ = _run_gpu(d, vel, u, w, cw)
    x = d["pos"].astype(np.float64)
    v = vel.astype(np.float64)
    uu = u.astype(np.float64)
    m = d["m"]
    h = d["h"]
    L = np.asarray(d["box"], np.float64)
    Hmax = float(np.float32(1.825742)) * float(h.max())
    y = x[:, 1]
    far = (np.abs(y - 0.25) > 3 * Hmax) & (np.abs(y - 0.75) > 3 * Hmax)
    p = O.Params(box=d["box"])

    def local_loss(k, xx, vv, ux):
        dd = x - x[k]
        dd -= L * np.round(dd / L)
        r2 = (dd * dd).sum(1)
        act_f = (r2 < (3.2 * Hmax) ** 2).astype(np.uint8)
        act_d = (r2 < (4.3 * Hmax) ** 2).astype(np.uint8)
        od = O.density(p, xx, vv, m, h, active=act_d)
        g = O.ghost(p, h, od["rho"], od["drho_dh"], od["div"], od["curl"], ux)
        of = O.force(p, xx, vv, m, h, ux, od["rho"], g["f"], g["P"], g["c"], g["B"], active=act_f)
        on = act_f.astype(bool)
        return float((w[on] * of["accel"][on]).sum() + (cw[on] * of["dudt"][on]).sum())

    scale = {"x": np.abs(gx).max(), "v": np.abs(gv).max(), "u": np.abs(gu).max()}
    checked = 0
    for k in rng.choice(np.nonzero(far)[0], 12, replace=False):
        for nm, comp in (("x", 0), ("x", 1), ("v", 2), ("u", None)):
            base = {"x": x, "v": v, "u": uu}[nm]
            fds = []
            for delta in (1e-6, 5e-7):
                vals = []
                step = delta * (max(abs(base[k]), 0.05) if comp is None else 0.05)
                for sg in (1, -1):
                    arr = base.copy()
                    if comp is None:
                        arr[k] += sg * step
                    else:
                        arr[k, comp] += sg * step
                    args = {"x": x, "v": v, "u": uu}
                    args[nm] = arr
                    vals.append(local_loss(k, args["x"], args["v"], args["u"]))
                fds.append((vals[0] - vals[1]) / (2 * step))
            if abs(fds[0] - fds[1]) > 1e-5 * scale[nm]:
                continue  # a kink of the loss inside the stencil (support edge, mu = 0)
            got = {"x": gx, "v": gv, "u": gu}[nm]
            g = got[k, comp] if comp is not None else got[k]
            assert abs(g - fds[0]) <= 1e-4 * abs(fds[0]) + FLOOR * scale[nm], (nm, k, comp, g, fds[0])
            checked += 1
    assert checked >= 30


def _run_gpu_hsolved(d, vel, u, w, cw, **params):
    from paper_2505_14538_b300 import sph
    n = len(d["pos"])
    ctx = sph.Context(n, box=d["box"], h_tol=1e-7, max_iter=60, **params)
    x = torch.from_numpy(d["pos"].astype(np.float32)).cuda().requires_grad_(True)
    v = torch.from_numpy(vel.astype(np.float32)).cuda().requires_grad_(True)
    uu = torch.from_numpy(u.astype(np.float32)).cuda().requires_grad_(True)
    m = torch.from_numpy(d["m"].astype(np.float32)).cuda()
    h0 = torch.from_numpy(d["h"].astype(np.float32)).cuda()
    a, du, h = sph.SphForcesSolvedH.apply(x, v, uu, m, h0, ctx)
    L = (torch.from_numpy(w.astype(np.float32)).cuda() * a).sum() + \
        (torch.from_numpy(cw.astype(np.float32)).cuda() * du).sum()
    L.backward()
    torch.cuda.synchronize()
    assert ctx.sync_status()[0] == 0
    return x.grad.cpu().numpy(), v.grad.cpu().numpy(), uu.grad.cpu().numpy(), h.cpu().numpy()


@pytest.mark.parametrize("kind", [0, 1])
def test_adjoint_hsolved_matches_torch_fp64(O, kind):
    """h_mode 1 (h = h(x), implicit function theorem) against the FP64 torch reference at the oracle's own root."""
    from oracle import torch_ref as T
    d = ics.lattice(10, jitter=0.3, index=14)
    n = len(d["pos"])
    rng = np.random.default_rng(60 + kind)
    vel = rng.normal(0, 0.3, (n, 3)).astype(np.float32)
    u = (d["u"] * rng.uniform(0.5, 1.5, n)).astype(np.float32)
    w = rng.normal(size=(n, 3))
    cw = rng.normal(size=n)
    kg = O.KERNEL_GAMMAS[kind]
    gx, gv, gu, h_gpu = _run_gpu_hsolved(d, vel, u, w, cw, kernel=kind)
    p = O.Params(kernel=kind, kernel_gamma=kg, h_tol=1e-14, max_iter=80, h_max=0.4)
    root = O.solve_h(p, d["pos"], vel, d["m"], d["h"])
    assert root["converged"].all()
    h = root["h"]
    assert np.max(np.abs(h_gpu / h - 1)) < 1e-5
    _, rx, rv, ru, rh, lam = T.loss_and_grad_hsolved(d["pos"], vel, u, d["m"], h, w, cw, box=d["box"],
                                                     kernel_gamma=kg, kernel=kind)
    # the sqrt kink of Eq. 22 (pairs with equal pressures and different u), as for h_mode 0
    pairs = T.pair_list(d["pos"], h, d["box"], kg)
    _, _, ex = T.forward(torch.tensor(d["pos"].astype(np.float64)), torch.tensor(vel.astype(np.float64)),
                         torch.tensor(u.astype(np.float64)), d["m"], h, pairs, d["box"], kernel_gamma=kg, kernel=kind)
    P = ex["P"].numpy()
    i, j = pairs
    bad = (np.abs(P[i] - P[j]) < 1e-5 * (P[i] + P[j])) & (u[i] != u[j])
    mask = np.zeros(n, bool)
    mask[i[bad]] = True
    mask[i[mask[j]]] = True
    keep = ~mask
    assert keep.mean() > {0: 0.8, 1: 0.7}[kind]  # Wendland C2: more neighbours reach the kink
    for got, ref, nm in ((gx, rx, "x"), (gv, rv, "v"), (gu, ru, "u")):
        _within(got[keep], ref[keep], (kind, nm))
    # the h term is not negligible here: the fixed-h gradient differs from it
    fixed = T.loss_and_grad(d["pos"], vel, u, d["m"], h, w, cw, box=d["box"], kernel_gamma=kg, kernel=kind)[1]
    assert np.abs(fixed - rx).max() > 1e-2 * np.abs(rx).max()


def test_hsolved_adjoint_refused_at_fixed_h():
    from paper_2505_14538_b300 import _lib, sph
    d = ics.lattice(8, jitter=0.2)
    n = len(d["pos"])
    ctx = sph.Context(n, flags=_lib.FLAG_NO_H_ITER)
    pos_h = torch.from_numpy(np.concatenate([d["pos"], d["h"][:, None]], 1).astype(np.float32)).cuda()
    vel_m = torch.from_numpy(np.concatenate([d["vel"], d["m"][:, None]], 1).astype(np.float32)).cuda()
    ctx.build_cells(pos_h)
    ctx.density(pos_h, vel_m)
    ctx.force(torch.from_numpy(d["u"].astype(np.float32)).cuda())
    with pytest.raises(sph.SwiftGPUError):
        ctx.force_backward(torch.zeros(n, 4, device="cuda"), h_mode=1)


def test_backward_after_another_forward_on_the_same_context():
    """Two SphForces forwards on one context, then the first one's backward: its gradient is still its own
    (the context's state is restored from the saved inputs), bitwise equal to a backward taken at once."""
    from paper_2505_14538_b300 import _lib, sph
    name, d, vel, u = list(_cases())[1]
    n = len(d["pos"])
    rng = np.random.default_rng(21)
    w = torch.from_numpy(rng.normal(size=(n, 3)).astype(np.float32)).cuda()
    cw = torch.from_numpy(rng.normal(size=n).astype(np.float32)).cuda()
    m = torch.from_numpy(d["m"].astype(np.float32)).cuda()
    h = torch.from_numpy(d["h"].astype(np.float32)).cuda()

    def leaves(shift):
        x = torch.from_numpy(((d["pos"] + shift) % 1.0).astype(np.float32)).cuda().requires_grad_(True)
        v = torch.from_numpy(vel.astype(np.float32)).cuda().requires_grad_(True)
        uu = torch.from_numpy(u.astype(np.float32)).cuda().requires_grad_(True)
        return x, v, uu

    ctx = sph.Context(n, box=d["box"], flags=_lib.FLAG_NO_H_ITER)
    # reference: forward and backward at once
    x, v, uu = leaves(0.0)
    a, du = sph.SphForces.apply(x, v, uu, m, h, ctx)
    ((w * a).sum() + (cw * du).sum()).backward()
    ref = [t.grad.clone() for t in (x, v, uu)]
    # the same forward, then another one (other positions) on the same context, then the first backward
    x, v, uu = leaves(0.0)
    a, du = sph.SphForces.apply(x, v, uu, m, h, ctx)
    x2, v2, u2 = leaves(0.01)
    a2, du2 = sph.SphForces.apply(x2, v2, u2, m, h, ctx)
    ((w * a).sum() + (cw * du).sum()).backward()
    torch.cuda.synchronize()
    for got, exp in zip((x.grad, v.grad, uu.grad), ref):
        assert torch.equal(got, exp)
    # and the second one's backward still gives its own gradient
    ((w * a2).sum() + (cw * du2).sum()).backward()
    assert not torch.equal(x2.grad, ref[0])
