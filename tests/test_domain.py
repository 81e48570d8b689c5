"""Slab domain decomposition (paper_2505_14538_b300.domain) on two and three gloo ranks (CPU).

Every rank runs decomposed_step with a backend that evaluates its local set
(owned particles + the ghost layers it received) with the FP64 oracle; the
assembled per-particle outputs and the all-reduced sums must equal the
single-domain oracle step on the whole set. This checks the host-side
decomposition (ownership, ghost layers, both halo exchanges, the order in
which the owners' density results come back, the global sums); on GPUs the
same step runs with ContextBackend.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _state(n_side=16, seed=31):
    sys.path.insert(0, ROOT)
    from paper_2505_14538_b300 import ics
    d = ics.lattice(n_side, jitter=0.25)
    rng = np.random.default_rng(seed)
    n = len(d["pos"])
    vel = rng.normal(0, 0.3, (n, 3))
    u = d["u"] * rng.uniform(0.5, 1.5, n)
    return d, vel, u


class OracleBackend:
    """density / set_inactive / gradient_force of a decomposed step, evaluated by the FP64 oracle."""

    def __init__(self, O, p):
        import torch
        self.O, self.p, self.torch = O, p, torch

    def density(self, pos_h, vel_m, active):
        t = self.torch
        x = pos_h[:, :3].double().numpy()
        v = vel_m[:, :3].double().numpy()
        m = vel_m[:, 3].double().numpy()
        h0 = pos_h[:, 3].double().numpy()
        act = active.numpy()
        s = self.O.solve_h(self.p, x, v, m, h0, active=act)
        self.x, self.v, self.m, self.act = x, v, m, act
        self.h = np.where(act > 0, s["h"], h0)
        self.rho4 = np.stack([s["rho"], s["drho_dh"], s["n"], s["dn_dh"]], 1)
        self.cd = np.concatenate([s["curl"], s["div"][:, None]], 1)
        return {"h": t.from_numpy(self.h), "rho4": t.from_numpy(self.rho4), "curl_div": t.from_numpy(self.cd),
                "ngb": t.from_numpy(s["ngb"])}

    def set_inactive(self, mask, h, rho4, curl_div):
        mk = mask.numpy() > 0
        self.h[mk] = h.numpy()[mk]
        self.rho4[mk] = rho4.numpy()[mk]
        self.cd[mk] = curl_div.numpy()[mk]

    def gradient_force(self, u):
        t, O, p = self.torch, self.O, self.p
        uu = u.double().numpy()
        g = O.ghost(p, self.h, self.rho4[:, 0], self.rho4[:, 1], self.cd[:, 3], self.cd[:, :3], uu)
        gr = O.gradient(p, self.x, self.v, self.m, self.h, self.rho4[:, 0], g["c"], uu, active=self.act)
        fo = O.force(p, self.x, self.v, self.m, self.h, uu, self.rho4[:, 0], g["f"], g["P"], g["c"], g["B"],
                     active=self.act)
        on = self.act > 0
        ma = self.m[on, None] * fo["accel"][on]
        va = (self.v[on] * fo["accel"][on]).sum(1)
        du = fo["dudt"][on]
        mm = self.m[on]
        red = np.array([*ma.sum(0), (mm * (va + du)).sum(), np.linalg.norm(ma, axis=1).sum(),
                        (mm * (np.abs(va) + np.abs(du))).sum(), (mm * du).sum(), float(fo["npairs"][on].sum())])
        return {"vsig_lapu": t.from_numpy(np.stack([gr["vsig"], gr["lapu"]], 1)),
                "accel_dudt": t.from_numpy(np.concatenate([fo["accel"], fo["dudt"][:, None]], 1)),
                "dh_dt": t.from_numpy(fo["dhdt"]), "reductions": t.from_numpy(red)}


def _params(O, slabs):
    # the h cap of the slab layers, as the library derives it from its cells
    return O.Params(h_tol=1e-12, max_iter=60, h_max=slabs.width * (1 - 2 ** -20) / O.KERNEL_GAMMA)


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2505_14538_b300 import domain
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d, vel, u = _state()
    slabs = domain.Slabs(1.0, domain.slab_count(1.0, float(d["h"].max()), O.KERNEL_GAMMA), world)
    pos_h = torch.from_numpy(np.c_[d["pos"], d["h"]].astype(np.float32))
    vel_m = torch.from_numpy(np.c_[vel, d["m"]].astype(np.float32))
    uu = torch.from_numpy(u.astype(np.float32))
    mine = slabs.owner(pos_h[:, 2]) == rank
    ids = torch.nonzero(mine)[:, 0]
    out = domain.decomposed_step(OracleBackend(O, _params(O, slabs)), slabs, rank, pos_h[mine], vel_m[mine], uu[mine],
                                 ids=ids)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), ids=ids.numpy(), ghosts=out["ghosts"], nc=slabs.nc,
             **{k: out[k].numpy() for k in ("h", "rho4", "curl_div", "ngb", "vsig_lapu", "accel_dudt", "dh_dt",
                                            "reductions")})
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_decomposed_step_equals_single_domain(tmp_path, O, world):
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    d, vel, u = _state()
    n = len(d["pos"])
    ids = np.concatenate([q["ids"] for q in parts])
    assert np.array_equal(np.sort(ids), np.arange(n))  # every particle owned exactly once
    assert all(int(q["ghosts"]) > 0 for q in parts)
    from paper_2505_14538_b300 import domain
    slabs = domain.Slabs(1.0, int(parts[0]["nc"]), world)
    # the single-domain oracle at the same (FP32-rounded) inputs and h cap
    x = d["pos"].astype(np.float32).astype(np.float64)
    st = O.step(_params(O, slabs), x, vel.astype(np.float32), d["m"].astype(np.float32), u.astype(np.float32),
                d["h"].astype(np.float32))
    got = {k: np.zeros((n,) + parts[0][k].shape[1:]) for k in ("h", "rho4", "ngb", "accel_dudt", "vsig_lapu", "dh_dt")}
    for q in parts:
        for k in got:
            got[k][q["ids"]] = q[k]
    assert np.max(np.abs(got["h"] / st["h"] - 1)) < 1e-12
    assert np.array_equal(got["ngb"].astype(np.int64), st["ngb"])
    assert np.max(np.abs(got["rho4"][:, 0] / st["rho"] - 1)) < 1e-12
    assert np.max(np.abs(got["vsig_lapu"][:, 0] / st["vsig"] - 1)) < 1e-12
    scale = st["s_a"][:, None]
    assert np.all(np.abs(got["accel_dudt"][:, :3] - st["accel"]) <= 1e-10 * scale)
    assert np.all(np.abs(got["accel_dudt"][:, 3] - st["dudt"]) <= 1e-10 * st["s_u"] + 1e-300)
    assert np.max(np.abs(got["dh_dt"] - st["dhdt"])) <= 1e-10 * np.abs(st["dhdt"]).max()
    # the all-reduced sums are the whole set's, and every rank holds them
    ma = d["m"][:, None] * st["accel"]
    red = parts[0]["reductions"]
    for q in parts[1:]:
        assert np.array_equal(q["reductions"], red)
    assert np.allclose(red[:3], ma.sum(0), rtol=0, atol=1e-12 * np.linalg.norm(ma, axis=1).sum())
    assert red[7] == st["npairs"].sum()
    assert abs(red[4] - np.linalg.norm(ma, axis=1).sum()) <= 1e-12 * red[4]


def test_slab_ownership_and_ghost_layers():
    """Layers split evenly; each rank sends its bottom layer down and its top layer up (periodically)."""
    sys.path.insert(0, ROOT)
    import torch
    from paper_2505_14538_b300 import domain
    s = domain.Slabs(1.0, 9, 3)
    assert s.bounds == [0, 3, 6, 9]
    z = (torch.arange(9, dtype=torch.float64) + 0.5) / 9
    assert s.owner(z).tolist() == [0, 0, 0, 1, 1, 1, 2, 2, 2]
    m = s.send_masks(0, z[:3])
    assert m[2].tolist() == [True, False, False] and m[1].tolist() == [False, False, True]
    m = s.send_masks(1, torch.tensor([1.0]))  # z = L wraps to layer 0: not rank 1's, but masks are by layer
    s2 = domain.Slabs(1.0, 6, 2)
    m = s2.send_masks(0, (torch.arange(3, dtype=torch.float64) + 0.5) / 6)
    assert list(m) == [1] and m[1].tolist() == [True, False, True]  # both layers to the one neighbour
    assert s2.layer(torch.tensor([-1e-9, 1.0, 0.5])).tolist() == [5, 0, 3]
    with pytest.raises(ValueError):
        domain.Slabs(1.0, 5, 3)
