"""PyTorch FP64 reference of the fixed-h density + ghost + force pipeline, for gradients.

TEST INFRASTRUCTURE: only ``tests/`` may import this module. It restates the
equations of the C++ oracle (``sph_oracle.cpp``; the paper's Sec. 2.1,
Eqs. 2-11, 16-20, 22 with the readings listed there) with plain torch CPU ops
over an explicit list of interacting pairs, so that autograd gives the exact
FP64 gradient of a loss of the outputs with respect to positions, velocities
and internal energies at fixed smoothing lengths. The pair list is found by
brute force over all pairs (O(N^2)), in FP64, with the oracle's predicate.

``loss_and_grad_hsolved`` is the gradient when each h_i is the solution of
the h iteration (Sec. 2.1.2), F_i(x, h_i) = n_i(x, h_i) - (eta/h_i)^3 = 0:
by the implicit function theorem dh_i/dx = -(dF_i/dx) / (dF_i/dh_i), so
dL/dx = dL/dx|_h - sum_i lambda_i dn_i/dx with lambda_i = (dL/dh_i|_x) / F'_i
(n_i depends on h_i alone, so the Jacobian of F in h is diagonal).
"""
from __future__ import annotations

import math

import numpy as np
import torch

KERNEL_GAMMA = float(np.float32(1.825742))


def pair_list(x, h, box, kernel_gamma=KERNEL_GAMMA, block=512):
    """Ordered pairs (i, j), i != j, with r_ij < max(H_i, H_j) (periodic minimum image)."""
    x = np.asarray(x, np.float64)
    h = np.asarray(h, np.float64)
    L = np.asarray(box, np.float64)
    H = kernel_gamma * h
    n = len(x)
    I, J = [], []
    for s in range(0, n, block):
        d = x[s:s + block, None, :] - x[None, :, :]
        d = d - L * np.round(d / L)
        r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
        Hi = H[s:s + block, None]
        m = (r2 < Hi * Hi) | (r2 < H[None, :] ** 2)
        m[np.arange(m.shape[0]), np.arange(s, s + m.shape[0])] = False
        ii, jj = np.nonzero(m)
        I.append(ii + s)
        J.append(jj)
    return np.concatenate(I), np.concatenate(J)


def _w(q, kernel=0):
    """Kernel shape on the support (the caller masks q >= 1): cubic spline, Wendland C2 or C4."""
    s = torch.clamp(1.0 - q, min=0.0)
    if kernel == 1:
        return s ** 4 * (1.0 + 4.0 * q)
    if kernel == 2:
        return s ** 6 * (1.0 + 6.0 * q + (35.0 / 3.0) * q * q)
    return torch.where(q < 0.5, 1.0 - 6.0 * q * q + 6.0 * q * q * q, 2.0 * s * s * s)


def _dw(q, kernel=0):
    s = torch.clamp(1.0 - q, min=0.0)
    if kernel == 1:
        return -20.0 * q * s ** 3
    if kernel == 2:
        return (-56.0 / 3.0) * q * (1.0 + 5.0 * q) * s ** 5
    return torch.where(q < 0.5, -12.0 * q + 18.0 * q * q, -6.0 * s * s)


def _norm(kernel=0):
    """3-D normalisation of W = C H^-3 w(r/H)."""
    return {0: 8.0 / math.pi, 1: 21.0 / (2.0 * math.pi), 2: 495.0 / (32.0 * math.pi)}[kernel]


def _safe_sqrt(x):
    return torch.where(x > 0, torch.sqrt(torch.clamp(x, min=1e-300)), torch.zeros_like(x))


def forward(x, v, u, m, h, pairs, box=(1.0, 1.0, 1.0), gamma=5.0 / 3.0, alpha_v=1.0, beta=3.0, alpha_c=1.0,
            kernel_gamma=KERNEL_GAMMA, kernel=0):
    """accel (n, 3) and du/dt (n,) at fixed h; x, v, u are torch float64 (may require grad)."""
    n = x.shape[0]
    i = torch.as_tensor(pairs[0], dtype=torch.long)
    j = torch.as_tensor(pairs[1], dtype=torch.long)
    m = torch.as_tensor(m, dtype=torch.float64)
    h = torch.as_tensor(h, dtype=torch.float64)
    L = torch.as_tensor(box, dtype=torch.float64)
    H = kernel_gamma * h
    d = x[i] - x[j]
    d = d - L * torch.round((d / L).detach())
    r = torch.sqrt((d * d).sum(1))
    e = d / r[:, None]
    Hi, Hj = H[i], H[j]
    qi, qj = r / Hi, r / Hj
    c3 = _norm(kernel) / H ** 3
    Wi = c3[i] * _w(qi, kernel)
    dWi = c3[i] / Hi * _dw(qi, kernel)
    dWj = c3[j] / Hj * _dw(qj, kernel)
    in_i = (r < Hi).detach().to(torch.float64)  # pairs in i's density sums
    # density sums (self term: W(0) = c3, r dW/dr = 0)
    rho = m * c3 + torch.zeros(n, dtype=torch.float64).index_add(0, i, in_i * m[j] * Wi)
    D = 3.0 * m * c3 + torch.zeros(n, dtype=torch.float64).index_add(0, i, in_i * m[j] * (3.0 * Wi + r * dWi))
    g = in_i * m[j] * dWi / r
    dv = v[j] - v[i]
    S = torch.zeros(n, dtype=torch.float64).index_add(0, i, g * (dv * d).sum(1))
    C = -torch.zeros(n, 3, dtype=torch.float64).index_add(0, i, g[:, None] * torch.cross(dv, d, dim=1))
    div = S / rho
    curl = C / rho[:, None]
    # ghost step
    f = 1.0 / (1.0 - D / (3.0 * rho))
    P = (gamma - 1.0) * rho * u
    c = torch.sqrt(gamma * (gamma - 1.0) * u)
    A = f * P / rho ** 2
    ad = torch.abs(div)
    acurl = _safe_sqrt((curl * curl).sum(1))
    B = torch.where(ad > 0, ad / (ad + acurl + 1e-4 * c / h), torch.zeros_like(ad))
    # force pairs
    vij = v[i] - v[j]
    vr = (vij * e).sum(1)
    fsum = f[i] * dWi + f[j] * dWj
    ps = m[j] * (A[i] * dWi + A[j] * dWj)
    du1 = m[j] * A[i] * dWi * vr
    mu = torch.clamp(vr, max=0.0)
    vsig = c[i] + c[j] - beta * mu
    al = 0.25 * (2.0 * alpha_v) * (B[i] + B[j])
    rs = rho[i] + rho[j]
    nu = -al * mu * vsig / rs
    vs = 0.5 * m[j] * nu * fsum
    du2 = 0.5 * vs * vr
    Ps = P[i] + P[j]
    ac = (P[i] * alpha_c + P[j] * alpha_c) / Ps
    vc = torch.abs(vr) + _safe_sqrt(2.0 * torch.abs(P[i] - P[j]) / rs)
    du3 = ac * vc * m[j] * (u[i] - u[j]) * fsum / rs
    as_ = ps + vs
    accel = -torch.zeros(n, 3, dtype=torch.float64).index_add(0, i, as_[:, None] * e)
    dudt = torch.zeros(n, dtype=torch.float64).index_add(0, i, du1 + du2 + du3)
    return accel, dudt, dict(rho=rho, D=D, div=div, curl=curl, f=f, P=P, c=c, B=B)


def loss_and_grad(x, v, u, m, h, w, cw, box=(1.0, 1.0, 1.0), pairs=None, **kw):
    """L = sum w_i . a_i + c_i du_i/dt and (dL/dx, dL/dv, dL/du) at fixed h, all FP64 numpy."""
    x = torch.tensor(np.asarray(x, np.float64), requires_grad=True)
    v = torch.tensor(np.asarray(v, np.float64), requires_grad=True)
    u = torch.tensor(np.asarray(u, np.float64), requires_grad=True)
    if pairs is None:
        pairs = pair_list(x.detach().numpy(), h, box, kw.get("kernel_gamma", KERNEL_GAMMA))
    a, du, _ = forward(x, v, u, m, h, pairs, box, **kw)
    Lv = (torch.as_tensor(np.asarray(w, np.float64)) * a).sum() + (torch.as_tensor(np.asarray(cw, np.float64)) * du).sum()
    gx, gv, gu = torch.autograd.grad(Lv, (x, v, u))
    return float(Lv.detach()), gx.numpy(), gv.numpy(), gu.numpy(), a.detach().numpy(), du.detach().numpy()


def number_density(x, h, pairs, box=(1.0, 1.0, 1.0), kernel_gamma=KERNEL_GAMMA, kernel=0):
    """n_i = W(0, h_i) + sum over pairs with r < H_i of W(r_ij, h_i) (Eq. 5), differentiable in x and h."""
    n = x.shape[0]
    i = torch.as_tensor(pairs[0], dtype=torch.long)
    j = torch.as_tensor(pairs[1], dtype=torch.long)
    L = torch.as_tensor(box, dtype=torch.float64)
    H = kernel_gamma * h
    d = x[i] - x[j]
    d = d - L * torch.round((d / L).detach())
    r = torch.sqrt((d * d).sum(1))
    q = r / H[i]
    c3 = _norm(kernel) / H ** 3
    inside = (q < 1.0).detach().to(torch.float64)
    w = c3[i] * _w(q, kernel) * inside
    return c3 * 1.0 + torch.zeros(n, dtype=torch.float64).index_add(0, i, w)


def loss_and_grad_hsolved(x, v, u, m, h, w, cw, box=(1.0, 1.0, 1.0), eta=1.2348, **kw):
    """(L, dL/dx, dL/dv, dL/du) with h = h(x) the root of the h iteration; h must be that root."""
    kg = kw.get("kernel_gamma", KERNEL_GAMMA)
    kernel = kw.get("kernel", 0)
    xt = torch.tensor(np.asarray(x, np.float64), requires_grad=True)
    vt = torch.tensor(np.asarray(v, np.float64), requires_grad=True)
    ut = torch.tensor(np.asarray(u, np.float64), requires_grad=True)
    ht = torch.tensor(np.asarray(h, np.float64), requires_grad=True)
    pairs = pair_list(x, h, box, kg)
    a, du, _ = forward(xt, vt, ut, m, ht, pairs, box, **kw)
    Lv = (torch.as_tensor(np.asarray(w, np.float64)) * a).sum() + \
        (torch.as_tensor(np.asarray(cw, np.float64)) * du).sum()
    gx, gv, gu, gh = torch.autograd.grad(Lv, (xt, vt, ut, ht))
    # F' = dn_i/dh_i + 3 eta^3 / h_i^4 (n_i depends on h_i only)
    h2 = torch.tensor(np.asarray(h, np.float64), requires_grad=True)
    nn = number_density(xt.detach(), h2, pairs, box, kg, kernel)
    dn_dh = torch.autograd.grad(nn.sum(), h2)[0]
    Fp = dn_dh + 3.0 * eta ** 3 / h2.detach() ** 4
    lam = (gh / Fp).detach()
    x2 = torch.tensor(np.asarray(x, np.float64), requires_grad=True)
    nx = number_density(x2, torch.tensor(np.asarray(h, np.float64)), pairs, box, kg, kernel)
    gx_ift = torch.autograd.grad((lam * nx).sum(), x2)[0]
    return float(Lv.detach()), (gx - gx_ift).numpy(), gv.numpy(), gu.numpy(), gh.numpy(), lam.numpy()
