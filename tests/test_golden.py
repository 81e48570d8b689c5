"""Stored oracle outputs (tests/golden/lattice8_oracle.txt, written by tests/golden/write_golden.py).

CPU: the oracle still produces them (a regression pin; its closed-form and
invariant pins are in test_oracle_*.py). GPU: the kernels reproduce them at
the parity tolerances without running the oracle.
"""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

from write_golden import OUT, case  # noqa: E402


def load():
    rows = np.loadtxt(OUT, comments="#")
    return {"i": rows[:, 0].astype(np.int64), "h": rows[:, 1], "rho": rows[:, 2], "ngb": rows[:, 3].astype(np.int64),
            "a": rows[:, 4:7], "dudt": rows[:, 7], "s_a": rows[:, 8], "s_u": rows[:, 9]}


def test_oracle_reproduces_golden(O):
    g = load()
    d, vel, u, sample = case()
    assert np.array_equal(sample, g["i"])
    s = O.step(O.Params(h_tol=1e-13, max_iter=60), d["pos"], vel, d["m"], u, d["h"], solve=True)
    i = g["i"]
    assert np.all(np.abs(s["h"][i] / g["h"] - 1) < 1e-12)
    assert np.all(np.abs(s["rho"][i] / g["rho"] - 1) < 1e-12)
    assert np.array_equal(s["ngb"][i], g["ngb"])
    assert np.all(np.linalg.norm(s["accel"][i] - g["a"], axis=1) <= 1e-10 * g["s_a"])
    assert np.all(np.abs(s["dudt"][i] - g["dudt"]) <= 1e-10 * g["s_u"])


@pytest.mark.gpu
def test_gpu_reproduces_golden():
    torch = pytest.importorskip("torch")
    from paper_2505_14538_b300 import sph
    g = load()
    d, vel, u, _ = case()
    n = len(d["pos"])
    ctx = sph.Context(n, box=d["box"], h_tol=1e-6)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    pos_h = t(np.concatenate([d["pos"], d["h"][:, None]], 1))
    vel_m = t(np.concatenate([vel, d["m"][:, None]], 1))
    out = ctx.step(pos_h, vel_m, t(u))
    torch.cuda.synchronize()
    assert out["status"] == (0, 0)
    i = g["i"]
    h = out["h"].cpu().numpy()[i]
    rho = out["rho4"].cpu().numpy()[i, 0]
    ngb = out["ngb"].cpu().numpy()[i]
    ad = out["accel_dudt"].cpu().numpy()[i]
    assert np.all(np.abs(h / g["h"] - 1) < 1e-5)
    assert np.all(np.abs(rho / g["rho"] - 1) < 1e-5)
    assert np.array_equal(ngb.astype(np.int64), g["ngb"])
    assert np.all(np.linalg.norm(ad[:, :3] - g["a"], axis=1) <= 1e-4 * g["s_a"])
    assert np.all(np.abs(ad[:, 3] - g["dudt"]) <= 1e-4 * g["s_u"])
