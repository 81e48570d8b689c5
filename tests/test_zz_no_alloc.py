"""swift_gpu_density_static: the density call for callers that cannot allocate GPU memory.

Such callers (code whose host framework owns every device allocation, or a
plug-in that may only use the buffers it is handed) get one entry point whose
work memory is a fixed array inside the library. This test calls it through
the C ABI twice in a row and compares each result with the ordinary
context-based density call on the same inputs, at the tolerances of the other
parity tests (h and rho within 1e-5 relative, neighbour counts exact). It
also checks that a particle count above the array's capacity is refused.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _inputs(n_side, seed):
    from paper_2505_14538_b300 import ics
    d = ics.lattice(n_side, jitter=0.25, index=seed)
    rng = np.random.default_rng(seed)
    n = len(d["pos"])
    vel = rng.normal(0, 0.3, (n, 3)).astype(np.float32)
    pos_h = torch.from_numpy(np.concatenate([d["pos"], d["h"][:, None]], 1).astype(np.float32)).cuda()
    vel_m = torch.from_numpy(np.concatenate([vel, d["m"][:, None]], 1).astype(np.float32)).cuda()
    return n, pos_h, vel_m


def _static_call(lib, p, pos_h, vel_m, n):
    out = dict(h=torch.empty(n, dtype=torch.float32, device="cuda"),
               rho4=torch.empty(n, 4, dtype=torch.float32, device="cuda"),
               cd=torch.empty(n, 4, dtype=torch.float32, device="cuda"),
               ngb=torch.empty(n, dtype=torch.int32, device="cuda"),
               status=torch.full((2,), -99, dtype=torch.int64, device="cuda"))
    v = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = lib.swift_gpu_density_static(ctypes.byref(p), v(pos_h), v(vel_m), ctypes.c_int64(n), ctypes.c_float(0.0),
                                      v(out["h"]), v(out["rho4"]), v(out["cd"]), v(out["ngb"]), v(out["status"]),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    return {k: t.cpu().numpy() for k, t in out.items()}


def test_static_density_matches_context_call_twice():
    from paper_2505_14538_b300 import _lib, sph
    lib = _lib.load()
    p = sph.make_params(h_tol=1e-6)
    for n_side, seed in ((16, 11), (20, 12)):  # 4096 then 8000 particles: the second call reuses the array
        n, pos_h, vel_m = _inputs(n_side, seed)
        got = _static_call(lib, p, pos_h, vel_m, n)
        ctx = sph.Context(n, h_tol=1e-6)
        ctx.build_cells(pos_h)
        ref = ctx.density(pos_h, vel_m)
        code, detail = ctx.sync_status()
        ref = {k: t.cpu().numpy() for k, t in ref.items()}
        assert tuple(got["status"]) == (code, detail) == (0, 0)
        assert np.max(np.abs(got["h"] / ref["h"] - 1)) < 1e-5
        assert np.max(np.abs(got["rho4"][:, 0] / ref["rho4"][:, 0] - 1)) < 1e-5
        assert np.max(np.abs(got["rho4"][:, 2] / ref["rho4"][:, 2] - 1)) < 1e-5
        sc = np.abs(ref["curl_div"]).max()
        assert np.max(np.abs(got["cd"] - ref["curl_div"])) <= 1e-5 * sc
        assert np.array_equal(got["ngb"], ref["ngb"])
        ctx.close()


def test_static_density_rejects_too_many_particles():
    from paper_2505_14538_b300 import _lib, sph
    lib = _lib.load()
    p = sph.make_params()
    n = _lib.STATIC_MAX_PARTICLES + 1
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    v = ctypes.c_void_p(dummy.data_ptr())
    rc = lib.swift_gpu_density_static(ctypes.byref(p), v, v, ctypes.c_int64(n), ctypes.c_float(0.0), v, v, v, None,
                                      None, None)
    assert rc == _lib.ERR_CAPACITY
