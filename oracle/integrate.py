"""Plain FP64 oracle for time integration and the switch evolution (kick, drift,
Eqs. 12-15, 21, 23, 24 of arXiv 2505.14538), in NumPy.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module. It never imports the
CUDA package and the CUDA package never imports it. The pair loops of a full
step come from ``oracle.py`` (the FP64 C++ oracle).

The paper names the "kick" and "drift" tasks (Sec. 2.2.2) and prints the
switch equations (Sec. 2.1.3-2.1.4) but fixes neither the integrator nor the
time step, and several switch equations are garbled as printed. The readings
taken here (each one also listed in the design notes):

- Integrator: kick-drift-kick leapfrog with one global time step. A half
  kick v += a dt/2, u += du/dt dt/2; a drift x += v dt (wrapped into the
  periodic box) and h *= exp((dh/dt) dt / h); the loops of the new step see
  the predicted v + a dt/2 and u + du/dt dt/2 (the values the second half
  kick would give with the old rates). The second half kick uses the new
  rates. A half kick never lowers u below ``u_min_frac`` (0.5) of its value
  before the kick.
- Time step: dt_i = cfl * 2 H_i / v_sig,i with H_i = kernel_gamma h_i and
  v_sig,i the gradient loop's maximum signal velocity (Eq. 10); the step is
  the minimum over particles, further capped by ``dt_max`` and by the time
  left to ``t_end``. Particles with v_sig,i = 0 set no bound.
- Eq. 15: the rate of change of div v is the difference of div v between the
  two steps divided by the step.
- Eq. 14: S_i = H_i^2 max(0, -d(div v_i)/dt).
- Eq. 13: alpha_loc,i = alpha_v,max S_i / (v_sig,i^2 + S_i), with the
  particle's v_sig,i from the gradient loop of the previous step. The
  trailing "dt" of the printed equation is dropped: the ratio is already
  dimensionless and so is alpha.
- Eq. 12: alpha_v relaxes toward alpha_loc: when alpha_loc >= alpha_v it is
  taken at once; otherwise alpha_v <- alpha_loc + (alpha_v - alpha_loc)
  exp(-l c_i dt / H_i) with the decay length l = 0.05 (the paper's value) and
  c_i = sqrt(gamma (gamma - 1) u_i). The result is kept in
  [alpha_v,min, alpha_v,max].
- Eq. 21, as printed (the source term carries alpha_c,i):
  d alpha_c / dt = beta_c H_i lap(u)_i alpha_c / sqrt(u_i)
                   - (alpha_c - alpha_c,min) v_c,i / H_i,
  with v_c,i read as the particle's v_sig,i and lap(u)_i the gradient loop's
  Laplacian; integrated with one forward-Euler step over dt, using u_i after
  the second half kick; the source term is taken only where u_i > 0.
- Eq. 24: alpha_c,max,i = alpha_c,max (1 - alpha_v,i / alpha_v,max) (the
  printed recursion read with the global alpha_c,max on the right and the
  particle's current alpha_v,i); Eq. 23 caps alpha_c,i at it, and alpha_c,i
  is kept >= alpha_c,min.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import oracle as O


@dataclass
class TimeParams:
    cfl: float = 0.1
    dt_max: float = 0.0          # 0: no cap
    alpha_v_max: float = 2.0
    alpha_v_min: float = 0.0
    visc_length: float = 0.05    # l of Eq. 12
    alpha_c_max: float = 1.0
    alpha_c_min: float = 0.0
    beta_c: float = 1.0
    u_min_frac: float = 0.5


def _f(a, shape=None):
    a = np.array(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def step_size(tp: TimeParams, kernel_gamma, h, vsig, t=0.0, t_end=0.0):
    """Global step: min_i cfl 2 H_i / v_sig,i, capped by dt_max and by t_end - t (readings above)."""
    H = kernel_gamma * _f(h).ravel()
    vs = _f(vsig).ravel()
    dt = np.inf
    for Hi, vi in zip(H, vs):
        if vi > 0.0:
            dt = min(dt, tp.cfl * 2.0 * Hi / vi)
    if tp.dt_max > 0.0:
        dt = min(dt, tp.dt_max)
    if t_end > 0.0:
        dt = min(dt, max(t_end - t, 0.0))
    return dt


def half_kick_u(tp: TimeParams, u, dudt, dt):
    """u + du/dt dt/2, never below u_min_frac u."""
    u = _f(u)
    return np.maximum(u + _f(dudt) * (0.5 * dt), tp.u_min_frac * u)


def kick_drift(tp: TimeParams, box, dt, x, v, u, a, dudt, h, dhdt):
    """First half kick, drift and prediction of one leapfrog step (Sec. 2.2.2 "kick"/"drift").

    Returns x (wrapped into [0, L)), h (drifted), v and u after the half
    kick, and the predicted v, u the loops of the step read.
    """
    x, v, a = _f(x, (-1, 3)), _f(v, (-1, 3)), _f(a, (-1, 3))
    u, dudt, h, dhdt = _f(u), _f(dudt), _f(h), _f(dhdt)
    L = _f(box, (3,))
    v_half = v + a * (0.5 * dt)
    u_half = half_kick_u(tp, u, dudt, dt)
    x_new = np.mod(x + v_half * dt, L)
    h_new = h * np.exp(dhdt * dt / h)
    v_pred = v_half + a * (0.5 * dt)
    u_pred = half_kick_u(tp, u_half, dudt, dt)
    return {"x": x_new, "h": h_new, "v": v_half, "u": u_half, "v_pred": v_pred, "u_pred": u_pred}


def viscosity_switch(tp: TimeParams, gamma_eos, kernel_gamma, dt, h, u, div, div_prev, vsig, alpha_v):
    """Eqs. 12-15: new alpha_v from the change of div v over the step; returns (alpha_v, div_prev).

    With dt = 0 alpha_v is unchanged and only div_prev is set.
    """
    h, u, div, div_prev, vsig = _f(h), _f(u), _f(div), _f(div_prev), _f(vsig)
    alpha = _f(alpha_v).copy()
    if dt > 0.0:
        H = kernel_gamma * h
        c = np.sqrt(gamma_eos * (gamma_eos - 1.0) * np.maximum(u, 0.0))
        ddiv = (div - div_prev) / dt                           # Eq. 15
        S = H * H * np.maximum(0.0, -ddiv)                     # Eq. 14
        den = vsig * vsig + S
        a_loc = np.where(den > 0.0, tp.alpha_v_max * S / np.where(den > 0.0, den, 1.0), 0.0)  # Eq. 13
        decayed = a_loc + (alpha - a_loc) * np.exp(-tp.visc_length * c * dt / H)            # Eq. 12
        alpha = np.where(a_loc >= alpha, a_loc, decayed)
        alpha = np.clip(alpha, tp.alpha_v_min, tp.alpha_v_max)
    return alpha, div.copy()


def diffusion_switch(tp: TimeParams, kernel_gamma, dt, h, u, lapu, vsig, alpha_v, alpha_c):
    """Eqs. 21, 23, 24: one forward-Euler step of alpha_c, capped by the viscosity-dependent maximum."""
    h, u, lapu, vsig = _f(h), _f(u), _f(lapu), _f(vsig)
    av, ac = _f(alpha_v), _f(alpha_c)
    H = kernel_gamma * h
    source = np.where(u > 0.0, tp.beta_c * H * lapu * ac / np.sqrt(np.where(u > 0.0, u, 1.0)), 0.0)
    decay = (ac - tp.alpha_c_min) * vsig / H
    ac = ac + dt * (source - decay)                            # Eq. 21
    cap = tp.alpha_c_max * (1.0 - av / tp.alpha_v_max)         # Eq. 24
    ac = np.minimum(ac, cap)                                   # Eq. 23
    return np.maximum(ac, tp.alpha_c_min)


def kick_finish(tp: TimeParams, kernel_gamma, dt, h, v, u, a, dudt, vsig, lapu, alpha_v, alpha_c,
                t=0.0, t_end=0.0):
    """Second half kick, alpha_c update and the next step size (from this step's v_sig)."""
    v = _f(v, (-1, 3)) + _f(a, (-1, 3)) * (0.5 * dt)
    u = half_kick_u(tp, u, dudt, dt)
    ac = None if alpha_c is None else diffusion_switch(tp, kernel_gamma, dt, h, u, lapu, vsig, alpha_v, alpha_c)
    dt_next = step_size(tp, kernel_gamma, h, vsig, t + dt, t_end)
    return {"v": v, "u": u, "alpha_c": ac, "dt_next": dt_next}


def prime(p: "O.Params", tp: TimeParams, x, v, m, u, h0, alpha_v, alpha_c, t_end=0.0):
    """Loop evaluation at t = 0 that starts the integration: rates, v_sig, div v and the first step."""
    s = O.step(p, x, v, m, u, h0, alpha_v=alpha_v, alpha_c=alpha_c)
    dt = step_size(tp, p.kernel_gamma, s["h"], s["vsig"], 0.0, t_end)
    return {"x": _f(x, (-1, 3)).copy(), "v": _f(v, (-1, 3)).copy(), "m": _f(m).copy(), "u": _f(u).copy(),
            "h": s["h"], "a": s["accel"], "dudt": s["dudt"], "dhdt": s["dhdt"], "vsig": s["vsig"],
            "lapu": s["lapu"], "div_prev": s["div"], "alpha_v": _f(alpha_v).copy(),
            "alpha_c": _f(alpha_c).copy(), "t": 0.0, "dt_next": dt, "loops": s}


def step(p: "O.Params", tp: TimeParams, st: dict, t_end=0.0):
    """One full leapfrog step of the SPH system in the order the library runs it.

    kick + drift, h iteration + density at the predicted state, viscosity
    switch (Eqs. 12-15), ghost, gradient and force loops with the new alpha_v
    and the old alpha_c, second half kick, alpha_c update (Eqs. 21, 23, 24)
    and the next step size. Returns the new state dict.
    """
    dt = st["dt_next"]
    kd = kick_drift(tp, p.box, dt, st["x"], st["v"], st["u"], st["a"], st["dudt"], st["h"], st["dhdt"])
    s1 = O.solve_h(p, kd["x"], kd["v_pred"], st["m"], kd["h"])
    av, div_prev = viscosity_switch(tp, p.gamma_eos, p.kernel_gamma, dt, s1["h"], kd["u_pred"], s1["div"],
                                    st["div_prev"], st["vsig"], st["alpha_v"])
    g = O.ghost(p, s1["h"], s1["rho"], s1["drho_dh"], s1["div"], s1["curl"], kd["u_pred"])
    gr = O.gradient(p, kd["x"], kd["v_pred"], st["m"], s1["h"], s1["rho"], g["c"], kd["u_pred"])
    fo = O.force(p, kd["x"], kd["v_pred"], st["m"], s1["h"], kd["u_pred"], s1["rho"], g["f"], g["P"], g["c"],
                 g["B"], av, st["alpha_c"])
    kf = kick_finish(tp, p.kernel_gamma, dt, s1["h"], kd["v"], kd["u"], fo["accel"], fo["dudt"], gr["vsig"],
                     gr["lapu"], av, st["alpha_c"], st["t"], t_end)
    return {"x": kd["x"], "v": kf["v"], "m": st["m"], "u": kf["u"], "h": s1["h"], "a": fo["accel"],
            "dudt": fo["dudt"], "dhdt": fo["dhdt"], "vsig": gr["vsig"], "lapu": gr["lapu"],
            "div_prev": div_prev, "alpha_v": av, "alpha_c": kf["alpha_c"], "t": st["t"] + dt,
            "dt_next": kf["dt_next"], "dt": dt,
            "loops": {**s1, **g, **gr, **fo, "v_pred": kd["v_pred"], "u_pred": kd["u_pred"]}}
