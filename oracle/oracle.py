"""ctypes wrapper of the FP64 CPU oracle (``sph_oracle.cpp``).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module. It never imports the CUDA
package and the CUDA package never imports it.

Every function takes NumPy arrays (any float dtype; converted to float64) and
returns float64 results. Positions are ``(n, 3)``; ``h``, ``m``, ``u`` are
``(n,)``. The equations, and every reading of the paper they rest on, are
listed in the header of ``sph_oracle.cpp`` (Sec. 2.1, Eqs. 1-11, 16-20, 22).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

# H/h of the cubic spline from the second-moment definition h = 2 sigma,
# rounded to float32 so both sides of a parity test use the same support.
KERNEL_GAMMA = float(np.float32(1.825742))
ETA = 1.2348

# Kernel shapes (Sec. 2.1.1 names the cubic spline and the Wendland kernels):
# 0 cubic spline, 1 Wendland C2, 2 Wendland C4, each with its own H/h from the
# same definition (sqrt(30)/3, sqrt(15)/2, sqrt(78)/4), rounded to float32.
CUBIC, WENDLAND_C2, WENDLAND_C4 = 0, 1, 2
KERNEL_GAMMAS = {CUBIC: KERNEL_GAMMA, WENDLAND_C2: float(np.float32(np.sqrt(15.0) / 2.0)),
                 WENDLAND_C4: float(np.float32(np.sqrt(78.0) / 4.0))}


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source; returns its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", _LIB + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _CParams(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double * 3),
        ("periodic", ctypes.c_int),
        ("gamma_eos", ctypes.c_double),
        ("eta", ctypes.c_double),
        ("kernel_gamma", ctypes.c_double),
        ("alpha_v", ctypes.c_double),
        ("beta_v", ctypes.c_double),
        ("alpha_c", ctypes.c_double),
        ("h_tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("h_max", ctypes.c_double),
        ("use_cells", ctypes.c_int),
        ("nthreads", ctypes.c_int),
        ("terms", ctypes.c_int),
        ("kernel", ctypes.c_int),
    ]


@dataclass
class Params:
    box: tuple = (1.0, 1.0, 1.0)
    periodic: bool = True
    gamma_eos: float = 5.0 / 3.0
    eta: float = ETA
    kernel_gamma: float = KERNEL_GAMMA
    alpha_v: float = 1.0
    beta_v: float = 3.0
    alpha_c: float = 1.0
    h_tol: float = 1e-13
    max_iter: int = 60
    h_max: float = 0.0
    use_cells: bool = True
    nthreads: int = 0
    terms: int = 7
    kernel: int = CUBIC

    def c(self) -> _CParams:
        p = _CParams()
        p.box = (ctypes.c_double * 3)(*[float(b) for b in self.box])
        p.periodic = int(self.periodic)
        p.gamma_eos = float(self.gamma_eos)
        p.eta = float(self.eta)
        p.kernel_gamma = float(self.kernel_gamma)
        p.alpha_v = float(self.alpha_v)
        p.beta_v = float(self.beta_v)
        p.alpha_c = float(self.alpha_c)
        p.h_tol = float(self.h_tol)
        p.max_iter = int(self.max_iter)
        p.h_max = float(self.h_max)
        p.use_cells = int(self.use_cells)
        p.nthreads = int(self.nthreads)
        p.terms = int(self.terms)
        p.kernel = int(self.kernel)
        return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
    return _lib


def _d(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _act(active, n):
    if active is None:
        return None
    a = np.ascontiguousarray(np.asarray(active, dtype=np.uint8))
    assert a.shape == (n,)
    return a


def cell_ids(x, box, nc):
    """Linear cell id per particle (wrap, floor(x nc / L), clamp)."""
    x = _d(x, (-1, 3))
    out = np.zeros(len(x), np.uint32)
    b = _d(box, (3,))
    rc = lib().oracle_cell_ids(ctypes.c_int64(len(x)), _p(x), _p(b), ctypes.c_int(nc), _p(out))
    assert rc == 0
    return out


def kernel(r, h, kernel_gamma=KERNEL_GAMMA, kind=CUBIC):
    """W(r, h) and dW/dr of the cubic spline (kind 0) or a Wendland kernel (1: C2, 2: C4)."""
    r = _d(r).ravel()
    W = np.zeros_like(r)
    dW = np.zeros_like(r)
    rc = lib().oracle_kernel(ctypes.c_int64(len(r)), _p(r), ctypes.c_double(h), ctypes.c_double(kernel_gamma),
                             ctypes.c_int(kind), _p(W), _p(dW))
    assert rc == 0
    return W, dW


def density(p: Params, x, v, m, h, active=None):
    """Density loop at fixed h (Eq. 2-6): n, dn/dh, rho, drho/dh, div v, curl v, neighbour count."""
    x = _d(x, (-1, 3))
    n = len(x)
    v, m, h = _d(v, (n, 3)), _d(m, (n,)), _d(h, (n,))
    act = _act(active, n)
    out = {k: np.zeros(n) for k in ("n", "dn_dh", "rho", "drho_dh", "div")}
    out["curl"] = np.zeros((n, 3))
    out["ngb"] = np.zeros(n, np.int64)
    pc = p.c()
    rc = lib().oracle_density(ctypes.byref(pc), ctypes.c_int64(n), _p(x), _p(v), _p(m), _p(h), _p(act),
                              _p(out["n"]), _p(out["dn_dh"]), _p(out["rho"]), _p(out["drho_dh"]),
                              _p(out["div"]), _p(out["curl"]), _p(out["ngb"]))
    assert rc == 0
    return out


def solve_h(p: Params, x, v, m, h0, active=None):
    """Newton iteration on h (Sec. 2.1.2) then the density outputs at the final h."""
    x = _d(x, (-1, 3))
    n = len(x)
    v, m, h0 = _d(v, (n, 3)), _d(m, (n,)), _d(h0, (n,))
    act = _act(active, n)
    out = {k: np.zeros(n) for k in ("h", "n", "dn_dh", "rho", "drho_dh", "div")}
    out["curl"] = np.zeros((n, 3))
    out["ngb"] = np.zeros(n, np.int64)
    out["pass_pairs"] = np.zeros(n, np.int64)
    out["iters"] = np.zeros(n, np.int32)
    out["converged"] = np.zeros(n, np.int32)
    pc = p.c()
    rc = lib().oracle_solve_h(ctypes.byref(pc), ctypes.c_int64(n), _p(x), _p(v), _p(m), _p(h0), _p(act),
                              _p(out["h"]), _p(out["iters"]), _p(out["converged"]), _p(out["n"]),
                              _p(out["dn_dh"]), _p(out["rho"]), _p(out["drho_dh"]), _p(out["div"]),
                              _p(out["curl"]), _p(out["ngb"]), _p(out["pass_pairs"]))
    assert rc == 0
    return out


def ghost(p: Params, h, rho, drho_dh, div, curl, u):
    """Per-particle ghost step: f = 1/Omega (Eq. 8), P, c, Balsara B."""
    h = _d(h).ravel()
    n = len(h)
    rho, drho_dh, div, u = _d(rho, (n,)), _d(drho_dh, (n,)), _d(div, (n,)), _d(u, (n,))
    curl = _d(curl, (n, 3))
    out = {k: np.zeros(n) for k in ("f", "P", "c", "B")}
    pc = p.c()
    rc = lib().oracle_ghost(ctypes.byref(pc), ctypes.c_int64(n), _p(h), _p(rho), _p(drho_dh), _p(div),
                            _p(curl), _p(u), _p(out["f"]), _p(out["P"]), _p(out["c"]), _p(out["B"]))
    assert rc == 0
    return out


def gradient(p: Params, x, v, m, h, rho, c, u, active=None):
    """Gradient loop: v_sig,max (Eq. 10-11) and the Laplacian of u."""
    x = _d(x, (-1, 3))
    n = len(x)
    v, m, h, rho, c, u = _d(v, (n, 3)), _d(m, (n,)), _d(h, (n,)), _d(rho, (n,)), _d(c, (n,)), _d(u, (n,))
    act = _act(active, n)
    vsig, lapu = np.zeros(n), np.zeros(n)
    pc = p.c()
    rc = lib().oracle_gradient(ctypes.byref(pc), ctypes.c_int64(n), _p(x), _p(v), _p(m), _p(h), _p(rho),
                               _p(c), _p(u), _p(act), _p(vsig), _p(lapu))
    assert rc == 0
    return {"vsig": vsig, "lapu": lapu}


def force(p: Params, x, v, m, h, u, rho, f, P, c, B, alpha_v=None, alpha_c=None, active=None):
    """Force loop (Eq. 7, 9-11, 16-20, 22): accel, du/dt, dh/dt, force scales, pair count."""
    x = _d(x, (-1, 3))
    n = len(x)
    v = _d(v, (n, 3))
    m, h, u, rho, f, P, c, B = (_d(a, (n,)) for a in (m, h, u, rho, f, P, c, B))
    av = None if alpha_v is None else _d(alpha_v, (n,))
    ac = None if alpha_c is None else _d(alpha_c, (n,))
    act = _act(active, n)
    out = {"accel": np.zeros((n, 3))}
    for k in ("dudt", "dhdt", "s_a", "s_u"):
        out[k] = np.zeros(n)
    out["npairs"] = np.zeros(n, np.int64)
    pc = p.c()
    rc = lib().oracle_force(ctypes.byref(pc), ctypes.c_int64(n), _p(x), _p(v), _p(m), _p(h), _p(u),
                            _p(rho), _p(f), _p(P), _p(c), _p(B), _p(av), _p(ac), _p(act),
                            _p(out["accel"]), _p(out["dudt"]), _p(out["dhdt"]), _p(out["s_a"]),
                            _p(out["s_u"]), _p(out["npairs"]))
    assert rc == 0
    return out


def interpolate(p: Params, x, m, h, rho, Q):
    """SPH interpolant (Eq. 1) of a scalar field Q."""
    x = _d(x, (-1, 3))
    n = len(x)
    m, h, rho, Q = _d(m, (n,)), _d(h, (n,)), _d(rho, (n,)), _d(Q, (n,))
    out = np.zeros(n)
    pc = p.c()
    lib().oracle_interpolate(ctypes.byref(pc), ctypes.c_int64(n), _p(x), _p(m), _p(h), _p(rho), _p(Q),
                             _p(out))
    return out


def count_flops(loop: int, q: float = 0.75, approaching: bool = True, kind: int = CUBIC):
    """Ops of one interaction of loop 0 density / 1 gradient / 2 force / 3 h-iteration step (Eqs. 5-6)."""
    out = (ctypes.c_longlong * 5)()
    rc = lib().oracle_count_flops(ctypes.c_int(loop), ctypes.c_double(q), ctypes.c_int(int(approaching)),
                                  ctypes.c_int(kind), out)
    assert rc == 0
    return dict(zip(("add", "mul", "div", "sqrt", "cmp"), list(out)))


def step(p: Params, x, v, m, u, h0, alpha_v=None, alpha_c=None, active=None, solve=True):
    """Whole hot path in order: h iteration + density, ghost, gradient, force.

    With ``solve=False`` the given h is used as is (fixed-h pipeline).
    Returns one dict with every intermediate.
    """
    x = _d(x, (-1, 3))
    if solve:
        d = solve_h(p, x, v, m, h0, active=active)
    else:
        d = density(p, x, v, m, h0, active=active)
        d["h"] = _d(h0).ravel().copy()
    g = ghost(p, d["h"], d["rho"], d["drho_dh"], d["div"], d["curl"], u)
    gr = gradient(p, x, v, m, d["h"], d["rho"], g["c"], u, active=active)
    fo = force(p, x, v, m, d["h"], u, d["rho"], g["f"], g["P"], g["c"], g["B"], alpha_v, alpha_c,
               active=active)
    out = dict(d)
    out.update(g)
    out.update(gr)
    out.update(fo)
    return out
