"""Context set-up rules: which arrays a context holds, and what swift_gpu_set_params may change.

A context created for the uniform grid holds no adaptive-tree arrays, so
turning adaptive leaves on afterwards is refused. Its kept-list store is
sized for the kernel shape it was created with; a later, wider shape keeps
no lists (the gradient and force loops then scan the cells) and still gives
the results of a context created for that shape.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from test_gpu_parity import dev_arrays, lattice_state  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    from paper_2505_14538_b300 import sph as S
    assert torch.cuda.is_available()
    return S


def _step(ctx, d, vel, u):
    pos_h, vel_m, ut = dev_arrays(d, vel, u)
    ctx.build_cells(pos_h, 0.0)
    out = ctx.density(pos_h, vel_m)
    out["vsig_lapu"] = ctx.gradient(ut)
    out.update(ctx.force(ut))
    torch.cuda.synchronize()
    assert ctx.sync_status() == (0, 0)
    return {k: v.cpu().numpy() for k, v in out.items() if torch.is_tensor(v)}


def test_adaptive_needs_a_context_created_for_it(sph):
    from paper_2505_14538_b300 import _lib
    ctx = sph.Context(4096)
    with pytest.raises(sph.SwiftGPUError):
        ctx.set_params(flags=_lib.FLAG_ADAPTIVE)
    ctx2 = sph.Context(4096, flags=_lib.FLAG_ADAPTIVE)
    ctx2.set_params(flags=0)  # the other way round is allowed: the uniform grid then scans its cells
    ctx2.set_params(flags=_lib.FLAG_ADAPTIVE)


def test_wider_kernel_shape_after_create(sph):
    d, vel, u = lattice_state(16, seed=5, jitter=0.2)
    n = len(d["pos"])
    made = sph.Context(n, box=d["box"], kernel=2, h_tol=1e-6)  # Wendland C4 from the start
    ref = _step(made, d, vel, u)
    assert made.info()["interactions"][0] > 0
    ctx = sph.Context(n, box=d["box"], h_tol=1e-6)  # cubic spline: the store holds 92 entries a lane
    ctx.set_params(kernel=2, kernel_gamma=made.params.kernel_gamma)
    got = _step(ctx, d, vel, u)
    assert np.array_equal(got["ngb"], ref["ngb"])
    for k in ("h", "rho4"):
        assert np.max(np.abs(got[k] - ref[k]) / np.maximum(np.abs(ref[k]), 1e-30)) < 1e-5, k
    sc = np.abs(ref["accel_dudt"]).max(0)
    assert np.all(np.abs(got["accel_dudt"] - ref["accel_dudt"]) <= 1e-4 * sc + 1e-30)
