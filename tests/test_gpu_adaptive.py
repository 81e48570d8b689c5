"""Adaptive leaves (SWIFT_GPU_ADAPTIVE) on the GPU against the FP64 oracle, through the C ABI.

Same tolerances as the uniform-grid parity tests (test_gpu_parity.py). The
leaf structure is checked against its definition: the leaves partition the
sorted particles into contiguous runs inside one cell; every cell is in
Morton order (10 bits per axis of the position inside the cell, ties by
input index); a leaf holds at most leaf_max particles unless it lies at the
deepest level; each leaf's h cap bounds the final h of its particles.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_14538_b300 import ics
from test_gpu_parity import check_against_oracle, dev_arrays, lattice_state, run_gpu

pytestmark = pytest.mark.gpu

ADAPTIVE = 8


@pytest.fixture(scope="module")
def sph():
    from paper_2505_14538_b300 import sph as S
    assert torch.cuda.is_available()
    return S


def _spread3(v):
    v = v.astype(np.uint64) & 0x3FF
    out = np.zeros_like(v)
    for b in range(10):
        out |= ((v >> b) & 1) << (3 * b)
    return out


def morton_in_cell(pos, box, nc):
    """30-bit Morton code of each position inside its cell (FP64: t = x nc / L, q = floor(1024 (t - floor t)))."""
    code = np.zeros(len(pos), np.uint64)
    for a in range(3):
        x = np.mod(pos[:, a].astype(np.float64), box[a])
        t = x * nc[a] / box[a]
        c = np.clip(np.floor(t), 0, nc[a] - 1)
        q = np.clip(np.floor((t - c) * 1024.0), 0, 1023).astype(np.uint64)
        code |= _spread3(q) << a
    return code


def clustered_state(n_total=2 ** 14, n_spheres=8, seed=0):
    d = ics.plummer(n_total=n_total, n_spheres=n_spheres, a_min=0.01, a_max=0.05, h_grid=16)
    rng = np.random.default_rng(seed)
    u = (d["u"] * rng.uniform(0.5, 1.5, len(d["pos"]))).astype(np.float32)
    return d, d["vel"].astype(np.float32), u


def run_step(sph, d, vel, u, **params):
    n = len(d["pos"])
    ctx = sph.Context(n, box=d["box"], **params)
    pos_h, vel_m, ut = dev_arrays(d, vel, u)
    out = ctx.step(pos_h, vel_m, ut)
    torch.cuda.synchronize()
    res = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}
    res["info"] = ctx.info()
    res["ctx"] = ctx
    return res


def test_adaptive_lattice_full_pipeline(sph, O):
    """16^3 lattice, 4^3 cells of 64 split into leaves of <= 8: every output against the oracle."""
    d, vel, u = lattice_state(16)
    g = run_gpu(sph, d, vel, u, min_cell_width=0.25, h_tol=1e-6, flags=ADAPTIVE, leaf_max=8)
    assert g["status"] == (0, 0), g["status"]
    info = g["info"]
    assert info["n_leaves"] >= 4096 // 8 and info["tree_depth"] >= 1
    check_against_oracle(O, d, vel, u, g, g["ctx"])
    ref = run_gpu(sph, d, vel, u, min_cell_width=0.25, h_tol=1e-6)
    assert np.array_equal(g["ngb"], ref["ngb"])
    assert np.max(np.abs(g["h"] / ref["h"] - 1)) < 1e-6
    # fewer candidates than the 27-cell scan
    assert info["candidates"][2] < ref["info"]["candidates"][2]


def test_adaptive_clustered_matches_oracle(sph, O):
    """Plummer spheres in a uniform background (h contrast > 10): step() with adaptive leaves vs the oracle."""
    d, vel, u = clustered_state()
    g = run_step(sph, d, vel, u, h_tol=1e-6, flags=ADAPTIVE)
    assert g["status"][0] == 0, g["status"]
    info = g["info"]
    assert info["tree_depth"] >= 2
    h = g["h"]
    assert h.max() / h.min() > 10.0
    check_against_oracle(O, d, vel, u, g, g["ctx"])


def test_adaptive_far_start_with_a_small_leaf_margin(sph, O):
    """Starting h at half the initial guess with leaf_margin 0.01: 32 rebuilds at a fixed margin
    reach only 1.01^32 = 1.37 times the start, so step() doubles the margin on each rebuild after
    the first and puts the caller's margin back afterwards."""
    d, vel, u = clustered_state(seed=3)
    d = dict(d, h=(0.5 * d["h"]).astype(np.float32))
    g = run_step(sph, d, vel, u, h_tol=1e-6, flags=ADAPTIVE, leaf_margin=0.01)
    assert g["status"][0] == 0, g["status"]
    assert abs(float(g["ctx"].params.leaf_margin) - 0.01) < 1e-9
    check_against_oracle(O, d, vel, u, g, g["ctx"])


def test_tune_leaf_max_keeps_a_timed_candidate(sph):
    """tune_leaf_max times each candidate from settled h, keeps the fastest, and the step after it
    solves the same h."""
    d, vel, u = clustered_state(seed=2)
    g = run_step(sph, d, vel, u, h_tol=1e-6, flags=ADAPTIVE)
    ctx = g["ctx"]
    pos_h, vel_m, ut = dev_arrays(d, vel, u)
    pos_h[:, 3] = torch.from_numpy(g["h"]).cuda()
    t = ctx.tune_leaf_max(pos_h, vel_m, ut, candidates=(16, 32, 64), steps=1)
    assert set(t["step_ms"]) == {16, 32, 64} and t["leaf_max"] == min(t["step_ms"], key=t["step_ms"].get)
    assert int(ctx.params.leaf_max) == t["leaf_max"]
    out = ctx.step(pos_h, vel_m, ut)
    torch.cuda.synchronize()
    assert ctx.sync_status()[0] == 0
    assert np.max(np.abs(out["h"].cpu().numpy() / g["h"] - 1)) < 1e-5
    with pytest.raises(ValueError):
        sph.Context(8).tune_leaf_max(pos_h[:8], vel_m[:8], ut[:8])


def test_adaptive_leaf_structure(sph):
    d, vel, u = clustered_state(seed=1)
    leaf_max = 16
    g = run_step(sph, d, vel, u, h_tol=1e-6, flags=ADAPTIVE, leaf_max=leaf_max)
    ctx, info = g["ctx"], g["info"]
    n = len(d["pos"])
    rng_t, hcap_t, cnt_t = ctx.leaves()
    cid, perm = ctx.cells()
    rng, hcap, cnt = rng_t.cpu().numpy(), hcap_t.cpu().numpy(), cnt_t.cpu().numpy()
    cid, perm = cid.cpu().numpy().astype(np.int64), perm.cpu().numpy().astype(np.int64)
    assert len(rng) == info["n_leaves"] > 0
    assert np.all(cnt >= 1) and cnt.sum() == info["leaf_pairs"]  # every leaf got its list here
    # a partition of the sorted positions into contiguous runs
    order = np.argsort(rng[:, 0])
    r = rng[order]
    assert r[0, 0] == 0 and r[-1, 1] == n
    assert np.array_equal(r[1:, 0], r[:-1, 1]) and np.all(r[:, 1] > r[:, 0])
    # each run inside one cell; leaf_max respected below the deepest level
    sc = cid[perm]
    for a, b in r:
        assert sc[a] == sc[b - 1]
    if info["tree_depth"] < 10:
        assert np.all(r[:, 1] - r[:, 0] <= leaf_max)
    # cells in Morton order, ties by input index
    mk = morton_in_cell(d["pos"], d["box"], info["nc"])[perm]
    same = sc[1:] == sc[:-1]
    assert np.all(sc[1:] >= sc[:-1])
    inc = (mk[1:] > mk[:-1]) | ((mk[1:] == mk[:-1]) & (perm[1:] > perm[:-1]))
    assert np.all(inc[same])
    # the caps bound the final h
    hs = g["h"][perm]
    for (a, b), c in zip(rng, hcap):
        assert hs[a:b].max() <= c <= info["h_cap"]


def test_adaptive_deterministic_and_backward(sph):
    """Adaptive runs repeat bit for bit, and the adjoint matches the uniform grid's."""
    d, vel, u = lattice_state(12, seed=4, jitter=0.3)
    n = len(d["pos"])
    rng = np.random.default_rng(2)
    ga = torch.from_numpy(rng.normal(size=(n, 4)).astype(np.float32)).cuda()
    outs = []
    for flags, reps in ((ADAPTIVE, 2), (0, 1)):
        for _ in range(reps):
            ctx = sph.Context(n, box=d["box"], flags=flags | 2, leaf_max=8)
            pos_h, vel_m, ut = dev_arrays(d, vel, u)
            ctx.build_cells(pos_h, 0.25)
            r = ctx.density(pos_h, vel_m)
            f = ctx.force(ut)
            gx, gv, gu = ctx.force_backward(ga)
            torch.cuda.synchronize()
            assert ctx.sync_status() == (0, 0)
            outs.append({"rho4": r["rho4"].cpu().numpy(), "a": f["accel_dudt"].cpu().numpy(),
                         "gx": gx.cpu().numpy(), "gv": gv.cpu().numpy(), "gu": gu.cpu().numpy()})
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
        sc = np.abs(outs[2][k]).max()
        assert np.max(np.abs(outs[0][k] - outs[2][k])) <= 1e-5 * sc, k


def test_adaptive_edge_cases(sph):
    ctx = sph.Context(8, flags=ADAPTIVE)
    e = torch.zeros(0, 4, dtype=torch.float32, device="cuda")
    ctx.build_cells(e)
    out = ctx.density(e, e.clone())
    assert out["h"].numel() == 0 and ctx.sync_status() == (0, 0)
    assert ctx.info()["n_leaves"] == 0
    one = torch.tensor([[0.3, 0.4, 0.5, 0.01]], dtype=torch.float32, device="cuda")
    vm = torch.tensor([[0.0, 0.0, 0.0, 1.0]], dtype=torch.float32, device="cuda")
    ctx.build_cells(one)
    out = ctx.density(one, vm)
    code, detail = ctx.sync_status()
    assert code == -5 and detail == 1  # capped by its leaf: a rebuild would widen it
    assert ctx.info()["n_leaves"] == 1
    assert out["ngb"].item() == 0
    with pytest.raises(sph.SwiftGPUError):
        sph.Context(8, flags=ADAPTIVE | 1)  # not with the per-task path
    with pytest.raises(sph.SwiftGPUError):
        sph.Context(8, flags=ADAPTIVE, leaf_max=4)
