"""GPU parity of the sm_103a kernels against the FP64 oracle, through the C ABI.

Tolerances (written here, from the arithmetic): cell ids, permutation and
neighbour counts bit-exact; rho and h within 1e-5 relative; acceleration and
du/dt within 1e-4 of each particle's force scale (sum over pairs of the
magnitude of the pair term); total momentum within 1e-6 of sum |m a|.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_14538_b300 import ics

pytestmark = pytest.mark.gpu

KG = float(np.float32(1.825742))


@pytest.fixture(scope="module")
def sph():
    from paper_2505_14538_b300 import sph as S
    assert torch.cuda.is_available()
    return S


def dev_arrays(d, vel=None, u=None):
    n = len(d["pos"])
    pos_h = np.concatenate([d["pos"], d["h"][:, None]], 1).astype(np.float32)
    v = d["vel"] if vel is None else vel
    vel_m = np.concatenate([v, d["m"][:, None]], 1).astype(np.float32)
    uu = d["u"] if u is None else u
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t(pos_h), t(vel_m), t(uu.astype(np.float32))


def oracle_params(O, ctx_params, **kw):
    p = O.Params(box=tuple(float(b) for b in ctx_params.box), gamma_eos=float(ctx_params.gamma_eos),
                 eta=float(ctx_params.eta), kernel_gamma=float(ctx_params.kernel_gamma),
                 alpha_v=float(ctx_params.alpha_v), beta_v=float(ctx_params.beta_v),
                 alpha_c=float(ctx_params.alpha_c), kernel=int(ctx_params.kernel))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# the density call's engines on the uniform grid, as tuning knobs: cell items (a warp shares a cell's
# candidates), and lane per particle with the shared-row or the pair-axis-window collect
ENGINES = {"cells": dict(lanes=32), "rows": dict(lanes=1, collect=0), "windows": dict(lanes=1, collect=1)}


def run_gpu(sph, d, vel=None, u=None, min_cell_width=0.0, active=None, lanes=None, collect=None, engine=None,
            **params):
    """One build, density, gradient and force pass; ``lanes`` sets the tuning's lanes per particle
    (1: the lane-per-particle path of the uniform grid; 2-32: cell items) and ``collect`` its
    candidate search; ``engine`` names one of ENGINES instead."""
    if engine is not None:
        lanes, collect = ENGINES[engine]["lanes"], ENGINES[engine].get("collect")
    n = len(d["pos"])
    ctx = sph.Context(max(n, 1), box=d["box"], **params)
    if lanes is not None:
        ctx.set_tuning(max_lanes_per_particle=lanes)
    if collect is not None:
        ctx.set_tuning(group_collect=collect)
    pos_h, vel_m, ut = dev_arrays(d, vel, u)
    act = None if active is None else torch.from_numpy(active.astype(np.uint8)).cuda()
    ctx.build_cells(pos_h, min_cell_width)
    out = ctx.density(pos_h, vel_m, act)
    status = ctx.sync_status()
    out["vsig_lapu"] = ctx.gradient(ut)
    out.update(ctx.force(ut))
    status2 = ctx.sync_status()
    torch.cuda.synchronize()
    res = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}
    res["status"] = status
    res["status2"] = status2
    res["info"] = ctx.info()
    res["ctx"] = ctx
    return res


def lattice_state(n_side=16, seed=0, jitter=0.1):
    d = ics.lattice(n_side, jitter=jitter)
    rng = np.random.default_rng(seed)
    n = len(d["pos"])
    vel = rng.normal(0, 0.3, size=(n, 3)).astype(np.float32)
    u = (d["u"] * rng.uniform(0.5, 1.5, n)).astype(np.float32)
    return d, vel, u


def check_against_oracle(O, d, vel, u, g, ctx, solve_tol=1e-13):
    """Compare a GPU run with the oracle: h (own solve), then every output at the GPU's h."""
    n = len(d["pos"])
    x = d["pos"]
    info = g["info"]
    # h: the oracle solves its own h from the same start with the same cap
    po = oracle_params(O, ctx.params, h_tol=solve_tol, max_iter=60, h_max=float(info["h_cap"]))
    so = O.solve_h(po, x, vel, d["m"], d["h"])
    assert np.all(so["converged"] == 1)
    h_gpu = g["h"].astype(np.float64)
    assert np.max(np.abs(h_gpu / so["h"] - 1)) < 1e-5
    # rho from the oracle at its own h
    assert np.max(np.abs(g["rho4"][:, 0] / so["rho"] - 1)) < 1e-5
    # everything else at the GPU's final float h
    pf = oracle_params(O, ctx.params)
    st = O.step(pf, x, vel, d["m"], u, g["h"], solve=False)
    assert np.array_equal(g["ngb"].astype(np.int64), st["ngb"])
    assert np.max(np.abs(g["rho4"][:, 0] / st["rho"] - 1)) < 1e-5
    assert np.max(np.abs(g["rho4"][:, 2] / st["n"] - 1)) < 1e-5
    sc_dn = np.abs(st["dn_dh"]).max()
    assert np.max(np.abs(g["rho4"][:, 3] - st["dn_dh"])) < 1e-5 * sc_dn
    sc_dr = np.abs(st["drho_dh"]).max()
    assert np.max(np.abs(g["rho4"][:, 1] - st["drho_dh"])) < 1e-5 * sc_dr
    cd = g["curl_div"]
    sc_v = max(np.abs(st["div"]).max(), np.abs(st["curl"]).max(), 1e-30)
    assert np.max(np.abs(cd[:, 3] - st["div"])) < 1e-5 * sc_v
    assert np.max(np.abs(cd[:, :3] - st["curl"])) < 1e-5 * sc_v
    # gradient loop
    vs = g["vsig_lapu"]
    assert np.max(np.abs(vs[:, 0] / st["vsig"] - 1)) < 1e-5
    sc_l = max(np.abs(st["lapu"]).max(), 1e-30)
    assert np.max(np.abs(vs[:, 1] - st["lapu"])) < 1e-4 * sc_l
    # force loop: per-particle scale
    a = g["accel_dudt"]
    err_a = np.linalg.norm(a[:, :3] - st["accel"], axis=1)
    assert np.all(err_a <= 1e-4 * st["s_a"] + 1e-30)
    err_u = np.abs(a[:, 3] - st["dudt"])
    assert np.all(err_u <= 1e-4 * st["s_u"] + 1e-30)
    # dh/dt uses the same sum as div v: dh/dt = h f div / 3
    ref_dh = st["dhdt"]
    assert np.max(np.abs(g["dh_dt"] - ref_dh)) < 1e-4 * max(np.abs(ref_dh).max(), 1e-30)
    # FP64 momentum reduction on the device
    red = g["reductions"]
    assert np.all(np.abs(red[:3]) <= 1e-6 * red[4])
    ma = d["m"][:, None].astype(np.float64) * a[:, :3].astype(np.float64)
    assert abs(red[4] / np.linalg.norm(ma, axis=1).sum() - 1) < 1e-6
    assert red[7] == st["npairs"].sum()
    return st


def test_cells_bit_exact(sph, O):
    d, vel, u = lattice_state(16)
    g = run_gpu(sph, d, vel, u, min_cell_width=0.25)
    ctx = g["ctx"]
    info = g["info"]
    assert info["nc"] == (4, 4, 4)
    cid, perm = ctx.cells()
    cid = cid.cpu().numpy().astype(np.uint32)
    perm = perm.cpu().numpy()
    ref = O.cell_ids(d["pos"], d["box"], 4)
    assert np.array_equal(cid, ref)
    assert np.array_equal(perm, np.argsort(ref, kind="stable"))


@pytest.mark.parametrize("engine", ["rows", "windows", "cells"])
def test_lattice16_full_pipeline(sph, O, engine):
    """Jittered 16^3 lattice with random v and u, 4^3 cells (64 particles a cell, more than a cell
    replica holds, so the windowed collect reads them whole; a group of 32 is half a cell, and its
    shared rows wrap periodically at both ends of the 4-cell rows): every output against the oracle,
    with every engine."""
    d, vel, u = lattice_state(16)
    g = run_gpu(sph, d, vel, u, min_cell_width=0.25, h_tol=1e-6, engine=engine)
    assert g["status"] == (0, 0), g["status"]
    check_against_oracle(O, d, vel, u, g, g["ctx"])
    inter = g["info"]["interactions"]
    assert inter[1] == g["ngb"].sum()


@pytest.mark.parametrize("engine", ["rows", "windows", "cells"])
def test_sedov_small_auto_cells(sph, O, engine):
    """Sedov blast at 16^3 with automatic cell width (strong u contrast, viscosity, conduction), with
    every engine; about 13 particles a cell, so the windowed collect reads its neighbour cells through
    the pair-axis windows, and a group of 32 spans three or four cells, some of them across the end
    of a row (two shared runs)."""
    d = ics.sedov(16)
    rng = np.random.default_rng(1)
    vel = rng.normal(0, 0.05, size=(len(d["pos"]), 3)).astype(np.float32)
    g = run_gpu(sph, d, vel, d["u"], h_tol=1e-6, engine=engine)
    assert g["status"][0] in (0,), g["status"]
    check_against_oracle(O, d, vel, d["u"], g, g["ctx"])


@pytest.mark.parametrize("engine", ["rows", "windows", "cells"])
def test_ragged_uniform_random(sph, O, engine):
    """3001 uniform random particles (ragged item sizes and tails: the last group of 32 is partial),
    non-cubic box, random h, with every engine."""
    rng = np.random.default_rng(7)
    n = 3001
    box = (1.0, 0.8, 1.25)
    pos = (rng.uniform(0, 1, (n, 3)) * np.array(box)).astype(np.float32)
    h = (rng.uniform(0.9, 1.1, n) * 1.2348 * (np.prod(box) / n) ** (1 / 3)).astype(np.float32)
    d = dict(pos=pos, h=h, m=np.full(n, 1.0 / n, np.float32), u=rng.uniform(0.5, 2, n).astype(np.float32),
             vel=rng.normal(0, 0.2, (n, 3)).astype(np.float32), box=box)
    g = run_gpu(sph, d, d["vel"], d["u"], h_tol=1e-6, engine=engine)
    assert g["status"][0] == 0, g["status"]
    check_against_oracle(O, d, d["vel"], d["u"], g, g["ctx"])


def test_rows_engine_smallest_grid(sph, O):
    """The shared-row collect on the smallest grid (the build never makes fewer than 3 cells a
    side): an 8^3 jittered lattice in cells of width 1/3. With 3 cells a row, a run
    covering x = 0..2 reads the row's images at x = -1 and x = 3, which are cells of the row itself
    (shifted by -L and +L). Every output against the oracle; candidates past a list's width take
    the multi-pass route."""
    d, vel, u = lattice_state(8, seed=11)
    g = run_gpu(sph, d, vel, u, min_cell_width=0.3, h_tol=1e-6, engine="rows")
    assert tuple(g["info"]["nc"]) == (3, 3, 3), g["info"]["nc"]
    assert g["status"] == (0, 0), g["status"]
    check_against_oracle(O, d, vel, u, g, g["ctx"])


def test_fixed_h_counts_at_input_h(sph, O):
    """NO_H_ITER: one density pass at the input h; counts bit-exact at that h."""
    d, vel, u = lattice_state(12, jitter=0.3)
    g = run_gpu(sph, d, vel, u, flags=2)
    assert np.array_equal(g["h"], d["h"])
    st = O.density(O.Params(), d["pos"], vel, d["m"], d["h"])
    assert np.array_equal(g["ngb"].astype(np.int64), st["ngb"])
    assert np.max(np.abs(g["rho4"][:, 0] / st["rho"] - 1)) < 1e-5


@pytest.mark.parametrize("engine", ["rows", "windows", "cells"])
def test_fixed_h_kept_lists_with_overflow(sph, O, engine):
    """NO_H_ITER keeps the density call's candidate lists for the gradient and force loops. On the
    Kelvin-Helmholtz slab (density ratio 2.2, the cells sized by the light layer's h) some lanes of
    the dense layer collect more candidates than a list holds: with cell items their items take the
    27-cell scan as a whole warp; lane per particle, such a particle scans its cells in the density
    call and its group does in the gradient and force loops. Every output against the oracle at the
    input h."""
    d = ics.kh(16, 11, 5)
    rng = np.random.default_rng(4)
    n = len(d["pos"])
    vel = d["vel"] + rng.normal(0, 0.05, (n, 3)).astype(np.float32)
    u = d["u"]
    g = run_gpu(sph, d, vel, u, flags=2, engine=engine)
    assert g["status"] == (0, 0) and g["status2"] == (0, 0)
    assert np.array_equal(g["h"], d["h"])
    pf = oracle_params(O, g["ctx"].params)
    st = O.step(pf, d["pos"], vel, d["m"], u, d["h"], solve=False)
    assert np.array_equal(g["ngb"].astype(np.int64), st["ngb"])
    assert np.max(np.abs(g["rho4"][:, 0] / st["rho"] - 1)) < 1e-5
    vs = g["vsig_lapu"]
    assert np.max(np.abs(vs[:, 0] / st["vsig"] - 1)) < 1e-5
    assert np.max(np.abs(vs[:, 1] - st["lapu"])) < 1e-4 * max(np.abs(st["lapu"]).max(), 1e-30)
    a = g["accel_dudt"]
    assert np.all(np.linalg.norm(a[:, :3] - st["accel"], axis=1) <= 1e-4 * st["s_a"] + 1e-30)
    assert np.all(np.abs(a[:, 3] - st["dudt"]) <= 1e-4 * st["s_u"] + 1e-30)
    # the overflowing items (groups) scanned in the density call and again in the gradient and
    # force loops; the others read their kept lists
    cand = g["info"]["candidates"]
    assert cand[1] == cand[2], cand
    if engine != "windows":
        assert cand[2] < cand[0], cand
    # on a lattice no list overflows: the loops read kept lists only, fewer candidates than the
    # density call tested (the cell items' 27-cell scan, or lane per particle the pair-axis windows,
    # whose kept entries are its hits), with the same outputs as the iterating path's loops at that h
    d, vel, u = lattice_state(12, jitter=0.3)
    g = run_gpu(sph, d, vel, u, flags=2, engine=engine)
    cand = g["info"]["candidates"]
    assert cand[2] < (cand[0] / 3 if engine != "windows" else cand[0]), cand
    st = O.step(oracle_params(O, g["ctx"].params), d["pos"], vel, d["m"], u, d["h"], solve=False)
    a = g["accel_dudt"]
    assert np.all(np.linalg.norm(a[:, :3] - st["accel"], axis=1) <= 1e-4 * st["s_a"] + 1e-30)
    assert np.all(np.abs(a[:, 3] - st["dudt"]) <= 1e-4 * st["s_u"] + 1e-30)


def test_deterministic(sph):
    d, vel, u = lattice_state(16, seed=3)
    a = run_gpu(sph, d, vel, u, h_tol=1e-6)
    b = run_gpu(sph, d, vel, u, h_tol=1e-6)
    for k in ("h", "rho4", "curl_div", "ngb", "vsig_lapu", "accel_dudt", "dh_dt"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("engine", ["rows", "cells"])
def test_active_subset_matches_full(sph, O, engine):
    """Only active particles are recomputed; with the inactive state from a full pass they match it.
    Lane per particle with shared rows, a group of 32 active particles spreads over many rows: two
    shared runs, the other lanes each scanning its own 27 cells."""
    d, vel, u = lattice_state(16, seed=5)
    n = len(d["pos"])
    full = run_gpu(sph, d, vel, u, h_tol=1e-6, engine=engine)
    act = ics.active_hash(n, 123, 4)
    ctx = sph.Context(n, box=d["box"], h_tol=1e-6)
    ctx.set_tuning(max_lanes_per_particle=ENGINES[engine]["lanes"], group_collect=ENGINES[engine].get("collect", 0))
    # previous state: converged h for everybody, rho4/curl_div from the full pass
    d2 = dict(d)
    d2["h"] = full["h"]
    pos_h, vel_m, ut = dev_arrays(d2, vel, u)
    rho4 = torch.from_numpy(full["rho4"]).cuda()
    cd = torch.from_numpy(full["curl_div"]).cuda()
    ctx.build_cells(pos_h)
    out = ctx.density(pos_h, vel_m, torch.from_numpy(act).cuda(), rho4=rho4, curl_div=cd)
    f = ctx.force(ut)
    torch.cuda.synchronize()
    on = act.astype(bool)
    h = out["h"].cpu().numpy()
    assert np.array_equal(h[~on], full["h"][~on])
    assert np.max(np.abs(h[on] / full["h"][on] - 1)) < 1e-6
    a = f["accel_dudt"].cpu().numpy()
    st = O.step(O.Params(), d["pos"], vel, d["m"], u, h, solve=False)
    err = np.linalg.norm(a[on, :3] - st["accel"][on], axis=1)
    assert np.all(err <= 1e-4 * st["s_a"][on])


def test_edge_cases(sph):
    """n = 0 and a single isolated particle (h runs into the cell cap: not converged, status set)."""
    ctx = sph.Context(8)
    e = torch.zeros(0, 4, dtype=torch.float32, device="cuda")
    ctx.build_cells(e)
    out = ctx.density(e, e.clone())
    assert out["h"].numel() == 0
    assert ctx.sync_status() == (0, 0)
    one = torch.tensor([[0.3, 0.4, 0.5, 0.01]], dtype=torch.float32, device="cuda")
    vm = torch.tensor([[0.0, 0.0, 0.0, 1.0]], dtype=torch.float32, device="cuda")
    ctx.build_cells(one)
    out = ctx.density(one, vm)
    code, detail = ctx.sync_status()
    assert code in (-4, -5) and detail == 1
    info = ctx.info()
    assert abs(out["h"].item() - info["h_cap"]) < 1e-7
    assert out["ngb"].item() == 0


def test_argument_errors(sph):
    ctx = sph.Context(16)
    empty = torch.zeros(0, 4, dtype=torch.float32, device="cuda")
    with pytest.raises(sph.SwiftGPUError) as e:
        ctx.density(empty, empty)  # before build_cells
    assert e.value.code == -2
    with pytest.raises(sph.SwiftGPUError):
        ctx.build_cells(torch.zeros(32, 4, dtype=torch.float32, device="cuda"))  # n > n_max
    nan = torch.full((4, 4), float("nan"), dtype=torch.float32, device="cuda")
    ctx.build_cells(nan)
    code, _ = ctx.sync_status()
    assert code == -1


def test_plain_per_task_path(sph, O):
    """SWIFT_GPU_PLAIN (one launch per self/pair task, host-driven h passes): same checks as the persistent path."""
    d, vel, u = lattice_state(12, seed=9)
    g = run_gpu(sph, d, vel, u, h_tol=1e-6, flags=1)
    assert g["status"][0] == 0, g["status"]
    check_against_oracle(O, d, vel, u, g, g["ctx"])
    p = run_gpu(sph, d, vel, u, h_tol=1e-6)
    assert np.max(np.abs(g["h"] / p["h"] - 1)) < 1e-6
    assert np.array_equal(g["ngb"], p["ngb"])


def test_step_graph_replays_bit_identically(sph):
    """The step captured in a CUDA graph gives bitwise the outputs of the direct calls, replay after replay."""
    d, vel, u = lattice_state(16, seed=11)
    n = len(d["pos"])
    pos_h, vel_m, ut = dev_arrays(d, vel, u)
    direct = sph.Context(n)
    ref = direct.step(pos_h, vel_m, ut, check=False)
    torch.cuda.synchronize()
    ctx = sph.Context(n)
    g = sph.StepGraph(ctx, pos_h, vel_m, ut)
    for _ in range(3):
        out = g.replay()
        torch.cuda.synchronize()
        for k in ("h", "rho4", "curl_div", "ngb", "vsig_lapu", "accel_dudt", "dh_dt"):
            assert torch.equal(out[k], ref[k]), k
    assert g.launches_per_step > 5


def test_info_and_status_wait_for_graph_replays(sph):
    """After replays of a graph captured on another stream, info() and sync_status() see all of them."""
    d = ics.sedov(32)
    n = len(d["pos"])
    pos_h, vel_m, ut = dev_arrays(d)
    ctx = sph.Context(n)
    g = sph.StepGraph(ctx, pos_h, vel_m, ut)
    torch.cuda.synchronize()
    i0 = ctx.info()
    g.replay()
    torch.cuda.synchronize()
    i1 = ctx.info()
    per = [i1["interactions"][j] - i0["interactions"][j] for j in range(3)]
    assert per[1] > 0
    for _ in range(5):
        g.replay()
    i2 = ctx.info()  # no host synchronisation before it
    assert [i2["interactions"][j] - i1["interactions"][j] for j in range(3)] == [5 * x for x in per]
    for _ in range(3):
        g.replay()
    assert ctx.sync_status() == (0, 0)
    i3 = ctx.info()
    assert i3["interactions"][1] - i2["interactions"][1] == 3 * per[1]


@pytest.mark.parametrize("flags", [0, 8])
def test_gradient_force_fused_equals_separate(sph, flags):
    """swift_gpu_gradient_force evaluates the pairs of gradient() then force(): v_sig bitwise (a max of the same
    terms); the Laplacian, a and du/dt to a few FP32 roundings (the fused loop may sum the pairs in another
    order); the FP64 sums to their own rounding (uniform grid and adaptive leaves)."""
    d, vel, u = lattice_state(16, seed=13, jitter=0.3)
    n = len(d["pos"])
    rng = np.random.default_rng(4)
    av = torch.from_numpy(rng.uniform(0.1, 2.0, n).astype(np.float32)).cuda()
    ac = torch.from_numpy(rng.uniform(0.0, 1.0, n).astype(np.float32)).cuda()
    outs = []
    for fused in (False, True):
        ctx = sph.Context(n, box=d["box"], flags=flags, leaf_max=8)
        pos_h, vel_m, ut = dev_arrays(d, vel, u)
        ctx.build_cells(pos_h)
        ctx.density(pos_h, vel_m)
        if fused:
            o = ctx.gradient_force(ut, av, ac)
        else:
            o = {"vsig_lapu": ctx.gradient(ut)}
            o.update(ctx.force(ut, av, ac))
        torch.cuda.synchronize()
        assert ctx.sync_status() == (0, 0)
        outs.append((o, ctx.info()))
    (a, ia), (b, ib) = outs
    assert torch.equal(a["vsig_lapu"][:, 0], b["vsig_lapu"][:, 0])  # a max of identical terms
    la, lb = a["vsig_lapu"][:, 1].cpu().numpy(), b["vsig_lapu"][:, 1].cpu().numpy()
    assert np.max(np.abs(la - lb)) <= 1e-5 * np.abs(lb).max()
    ad_a, ad_b = a["accel_dudt"].cpu().numpy(), b["accel_dudt"].cpu().numpy()
    sc_a = np.abs(ad_b[:, :3]).max()
    assert np.max(np.abs(ad_a[:, :3] - ad_b[:, :3])) <= 1e-6 * sc_a
    assert np.max(np.abs(ad_a[:, 3] - ad_b[:, 3])) <= 1e-6 * np.abs(ad_b[:, 3]).max()
    dh_a, dh_b = a["dh_dt"].cpu().numpy(), b["dh_dt"].cpu().numpy()
    assert np.max(np.abs(dh_a - dh_b)) <= 1e-6 * np.abs(dh_b).max()
    ra, rb = a["reductions"].cpu().numpy(), b["reductions"].cpu().numpy()
    assert np.all(np.abs(ra[:3] - rb[:3]) <= 1e-6 * rb[4])  # momentum: against sum |m a|
    assert abs(ra[3] - rb[3]) <= 1e-6 * rb[5] and abs(ra[6] - rb[6]) <= 1e-6 * rb[5]  # energy: against its abs sum
    assert np.all(np.abs(ra[[4, 5]] - rb[[4, 5]]) <= 1e-6 * rb[[4, 5]]) and ra[7] == rb[7]
    assert ia["interactions"][1:] == ib["interactions"][1:]


def test_out_of_box_positions_are_wrapped(sph, O):
    """Positions shifted by whole box lengths are wrapped into [0, L) (FP64) and give the oracle's answers there."""
    d, vel, u = lattice_state(12, seed=21)
    n = len(d["pos"])
    rng = np.random.default_rng(21)
    L = np.asarray(d["box"], np.float64)
    shifted = (d["pos"].astype(np.float64) + L * rng.integers(-2, 3, size=(n, 3))).astype(np.float32)
    wrapped = (shifted.astype(np.float64) - L * np.floor(shifted.astype(np.float64) / L)).astype(np.float32)
    assert np.any(shifted != wrapped)
    dg = dict(d)
    dg["pos"] = shifted
    g = run_gpu(sph, dg, vel, u, h_tol=1e-6)
    assert g["status"][0] == 0, g["status"]
    dw = dict(d)
    dw["pos"] = wrapped
    check_against_oracle(O, dw, vel, u, g, g["ctx"])


def test_injected_faults_report_status(sph):
    """Host-side fault injection: h <= 0, max_iter = 1, a grid barrier that gives up at once. No GPU fault."""
    d, vel, u = lattice_state(12, seed=23)
    n = len(d["pos"])
    # h <= 0 on one particle: the build reports ERR_ARG
    bad = dict(d)
    bad["h"] = d["h"].copy()
    bad["h"][7] = 0.0
    ctx = sph.Context(n, box=d["box"])
    pos_h, vel_m, ut = dev_arrays(bad, vel, u)
    ctx.build_cells(pos_h)
    assert ctx.sync_status()[0] == -1
    # one Newton step only: the unconverged particles are counted
    ctx = sph.Context(n, box=d["box"], max_iter=1, h_tol=1e-9)
    pos_h, vel_m, ut = dev_arrays(d, vel, u)
    ctx.build_cells(pos_h)
    ctx.density(pos_h, vel_m)
    code, detail = ctx.sync_status()
    assert code == -4 and 0 < detail <= n
    # the density launch's grid barrier gives up at once: ERR_TIMEOUT, and the context stays usable
    ctx = sph.Context(n, box=d["box"], h_tol=1e-6)
    ref = sph.Context(n, box=d["box"], h_tol=1e-6)
    ctx.set_tuning(wait_limit_us=-1)
    ctx.build_cells(pos_h)
    ctx.density(pos_h, vel_m)
    assert ctx.sync_status()[0] == -6
    ctx.set_tuning(wait_limit_us=0)
    out = ctx.step(pos_h, vel_m, ut)
    exp = ref.step(pos_h, vel_m, ut)
    torch.cuda.synchronize()
    assert out["status"] == (0, 0)
    for k in ("h", "rho4", "accel_dudt"):
        assert torch.equal(out[k], exp[k]), k


def test_autotune_picks_a_valid_setting_and_keeps_results(sph, O):
    """The autotuner times the loops over its candidates, keeps a valid setting, and the step still matches."""
    d, vel, u = lattice_state(16, seed=31)
    n = len(d["pos"])
    ctx = sph.Context(n, box=d["box"], h_tol=1e-6)
    pos_h, vel_m, ut = dev_arrays(d, vel, u)
    ref = ctx.step(pos_h, vel_m, ut)
    ref = {k: v.clone() for k, v in ref.items() if torch.is_tensor(v)}
    for loop in (0, 3):
        t = ctx.autotune(loop)
        assert t["max_lanes_per_particle"] in (1, 2, 4, 8, 16, 32) and 0 <= t["blocks_per_sm"] <= 2
    assert ctx.sync_status() == (0, 0)
    out = ctx.step(pos_h, vel_m, ut)
    torch.cuda.synchronize()
    assert torch.equal(out["ngb"], ref["ngb"])
    assert torch.max(torch.abs(out["h"] / ref["h"] - 1)).item() < 1e-5
    r_out, r_ref = out["rho4"], ref["rho4"]
    for c in (0, 2):  # rho and n: relative
        assert torch.max(torch.abs(r_out[:, c] / r_ref[:, c] - 1)).item() < 1e-5, c
    for c in (1, 3):  # h-derivatives (sums with cancellation): against the column's largest
        sc = torch.abs(r_ref[:, c]).max().item()
        assert torch.max(torch.abs(r_out[:, c] - r_ref[:, c])).item() < 1e-5 * sc, c
    sa = torch.abs(ref["accel_dudt"]).max().item()
    assert torch.max(torch.abs(out["accel_dudt"] - ref["accel_dudt"])).item() < 1e-4 * sa


@pytest.mark.parametrize("flags", [0, 8])
def test_repeated_loop_calls_and_builds_leave_their_counters_ready(sph, flags):
    """Each loop launch's last block sets its work ticket back to zero, and the cell build's h scan
    its max-h words, with no memset between launches. So the gradient, force and fused calls
    repeated after one density call fill fresh (NaN-filled) outputs bit-identically, and a build
    after one with twice the h gets the cell grid a fresh context gets."""
    d, vel, u = lattice_state(16, seed=21, jitter=0.3)
    n = len(d["pos"])
    ctx = sph.Context(n, box=d["box"], flags=flags, leaf_max=8)
    pos_h, vel_m, ut = dev_arrays(d, vel, u)
    ctx.build_cells(pos_h)
    ctx.density(pos_h, vel_m)
    nan = float("nan")
    runs = []
    for _ in range(3):
        o = ctx.gradient_force(ut, vsig_lapu=torch.full((n, 2), nan, device="cuda"),
                               accel_dudt=torch.full((n, 4), nan, device="cuda"))
        g = ctx.gradient(ut, vsig_lapu=torch.full((n, 2), nan, device="cuda"))
        f = ctx.force(ut, accel_dudt=torch.full((n, 4), nan, device="cuda"))
        runs.append((o["vsig_lapu"], o["accel_dudt"], g, f["accel_dudt"]))
    torch.cuda.synchronize()
    assert ctx.sync_status() == (0, 0)
    for r in runs:
        assert all(bool(torch.isfinite(t).all()) for t in r)
        for t, t0 in zip(r, runs[0]):
            assert torch.equal(t, t0)
    big = pos_h.clone()
    big[:, 3] *= 2.0
    ctx.build_cells(big)
    nc_big = ctx.info()["nc"]
    ctx.build_cells(pos_h)
    fresh = sph.Context(n, box=d["box"], flags=flags, leaf_max=8)
    fresh.build_cells(pos_h)
    assert ctx.info()["nc"] == fresh.info()["nc"] != nc_big
    assert ctx.info()["cell_width"] == fresh.info()["cell_width"]
