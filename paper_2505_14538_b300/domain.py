"""Slab domain decomposition of one hot-path step over ranks, with its halo exchanges.

SWIFT keeps its CPU code's domain decomposition over MPI ranks when it
off-loads the pair loops to GPUs (Sec. 5); this is that layer for this
library, one rank per GPU:

* the cell layers along z are split into ``world`` contiguous slabs; a rank
  owns the particles whose layer lies in its slab (the layer of a position is
  taken as the cell id is, ``floor(z nc / L)`` after the periodic wrap);
* the ghost layer of a rank is the layer just below and just above its slab
  (periodically): with layers no thinner than the largest support, every
  neighbour of an owned particle is owned or a ghost;
* one step: (1) exchange the ghosts' positions, velocities, masses and u with
  the two neighbouring ranks; (2) the density call on owned + ghosts with only
  the owned particles active; (3) exchange the ghosts' final h, rho4 and
  curl/div, which their owners computed; (4) put them in place
  (``swift_gpu_set_inactive``); (5) the gradient and force loops for the
  owned particles; (6) one all-reduce of the eight FP64 sums.

Exchanges are point-to-point sends into the receiver's own buffers
(``torch.distributed`` isend/irecv: NCCL between GPUs, gloo on CPU); no rank
reads another's memory. The compute is a backend with three calls
(``density``, ``set_inactive``, ``gradient_force``): :class:`ContextBackend`
runs them through the CUDA library.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, Optional

import torch


@dataclass
class Slabs:
    """``nc`` cell layers along z of a box of height ``Lz``, split into ``world`` contiguous slabs."""

    Lz: float
    nc: int
    world: int

    def __post_init__(self):
        if self.world > 1 and self.nc < 2 * self.world:
            raise ValueError(f"{self.nc} layers cannot give {self.world} ranks two layers each")
        self.bounds = [(r * self.nc) // self.world for r in range(self.world + 1)]

    @property
    def width(self) -> float:
        return self.Lz / self.nc

    def layer(self, z: torch.Tensor) -> torch.Tensor:
        """Layer index of each z (FP64: wrap into [0, L), floor(z nc / L), clamp)."""
        zd = z.double()
        zd = zd - self.Lz * torch.floor(zd / self.Lz)
        return torch.clamp(torch.floor(zd * self.nc / self.Lz).long(), 0, self.nc - 1)

    def owner(self, z: torch.Tensor) -> torch.Tensor:
        """Rank owning each z."""
        b = torch.tensor(self.bounds[1:-1], device=z.device, dtype=torch.long)
        return torch.bucketize(self.layer(z), b, right=True)

    def send_masks(self, rank: int, z: torch.Tensor) -> Dict[int, torch.Tensor]:
        """For each neighbouring rank, the owned particles (z of this rank's particles) in its ghost layer:
        the slab's bottom layer for the rank below, its top layer for the rank above (periodically)."""
        if self.world == 1:
            return {}
        lay = self.layer(z)
        lo, hi = self.bounds[rank], self.bounds[rank + 1]
        below, above = (rank - 1) % self.world, (rank + 1) % self.world
        masks = {below: lay == lo}
        masks[above] = masks.get(above, torch.zeros_like(lay, dtype=torch.bool)) | (lay == hi - 1)
        return masks


def slab_count(Lz: float, h_max: float, kernel_gamma: float, cell_margin: float = 0.05) -> int:
    """Layers along z as the library sizes cells: width >= (1 + margin) kernel_gamma max h."""
    return max(3, int(math.floor(Lz / ((1.0 + cell_margin) * kernel_gamma * h_max))))


def _exchange(rank: int, world: int, sends: Dict[int, torch.Tensor], width: int, dtype, device):
    """Send sends[dst] (rows of `width` values) to each dst, receive one block from each neighbour.

    Returns {src: tensor}. Counts first, then the rows, all as nonblocking
    point-to-point pairs (the neighbour sets are symmetric)."""
    import torch.distributed as dist
    peers = sorted(sends)
    cnt_out = {p: torch.tensor([sends[p].shape[0]], dtype=torch.int64, device=device) for p in peers}
    cnt_in = {p: torch.zeros(1, dtype=torch.int64, device=device) for p in peers}
    reqs = [dist.isend(cnt_out[p], p) for p in peers] + [dist.irecv(cnt_in[p], p) for p in peers]
    for r in reqs:
        r.wait()
    recv = {p: torch.empty((int(cnt_in[p].item()), width), dtype=dtype, device=device) for p in peers}
    reqs = [dist.isend(sends[p].contiguous(), p) for p in peers if sends[p].numel()]
    reqs += [dist.irecv(recv[p], p) for p in peers if recv[p].numel()]
    for r in reqs:
        r.wait()
    return recv


class ContextBackend:
    """The three calls of a decomposed step through the CUDA library (one context per rank).

    ``min_cell_width`` is the slab layer width, so the local cells (and the h
    cap they give) match the ghost layer; the local grid is the whole box,
    whose periodic images serve the ghosts across the box edge.
    """

    def __init__(self, n_max: int, min_cell_width: float, **params):
        from . import sph
        self.ctx = sph.Context(n_max, **params)
        # a hair below the layer width, so that the library's nc = floor(L / width) is the slab count
        # whatever the rounding of L / width (its cells are then exactly the layers)
        self.width = float(min_cell_width) * (1.0 - 2.0 ** -20)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def density(self, pos_h, vel_m, active):
        n = pos_h.shape[0]
        self.ctx.build_cells(pos_h, self.width)
        rho4 = torch.zeros(n, 4, dtype=torch.float32, device=pos_h.device)
        cd = torch.zeros(n, 4, dtype=torch.float32, device=pos_h.device)
        return self.ctx.density(pos_h, vel_m, active, rho4=rho4, curl_div=cd)

    def set_inactive(self, mask, h, rho4, curl_div):
        self.ctx.set_inactive(mask, h, rho4, curl_div)

    def gradient_force(self, u, alpha_v=None, alpha_c=None):
        return self.ctx.gradient_force(u, alpha_v, alpha_c)

    def status(self):
        return self.ctx.sync_status()


def decomposed_step(backend, slabs: Slabs, rank: int, pos_h: torch.Tensor, vel_m: torch.Tensor, u: torch.Tensor,
                    ids: Optional[torch.Tensor] = None) -> dict:
    """One step (density with the h iteration, gradient, force) of the particles this rank owns.

    pos_h, vel_m (n, 4) float32 and u (n,) are the owned particles (their z
    in this rank's slab), on the backend's device. Returns their h, rho4,
    curl_div, ngb, vsig_lapu, accel_dudt, dh_dt in the same order, the global
    FP64 sums (``reductions``, all-reduced) and the ghost count.
    """
    import torch.distributed as dist
    world = slabs.world
    n = pos_h.shape[0]
    dev = pos_h.device
    if ids is None:
        ids = torch.arange(n, device=dev)
    # (1) the ghosts' inputs from the neighbouring ranks
    masks = slabs.send_masks(rank, pos_h[:, 2])
    payload = torch.cat([pos_h, vel_m, u[:, None]], 1)  # 9 columns
    sends = {p: payload[m] for p, m in masks.items()}
    recv = _exchange(rank, world, sends, 9, torch.float32, dev) if world > 1 else {}
    peers = sorted(masks)
    ghost = torch.cat([recv[p] for p in peers], 0) if peers else payload[:0]
    ng = ghost.shape[0]
    loc_pos = torch.cat([pos_h, ghost[:, 0:4]], 0).contiguous()
    loc_vel = torch.cat([vel_m, ghost[:, 4:8]], 0).contiguous()
    loc_u = torch.cat([u, ghost[:, 8]], 0).contiguous()
    active = torch.cat([torch.ones(n, dtype=torch.uint8, device=dev), torch.zeros(ng, dtype=torch.uint8, device=dev)])
    # (2) density of the owned particles
    d = backend.density(loc_pos, loc_vel, active)
    # (3) the ghosts' density results from their owners, in the order of (1)
    res = torch.cat([d["h"][:n, None], d["rho4"][:n], d["curl_div"][:n]], 1)  # 9 columns, the backend's dtype
    back = _exchange(rank, world, {p: res[masks[p]] for p in peers}, 9, res.dtype, dev) if world > 1 else {}
    if ng:
        got = torch.cat([back[p] for p in peers], 0)
        h_all = torch.cat([d["h"][:n], got[:, 0]]).contiguous()
        rho_all = torch.cat([d["rho4"][:n], got[:, 1:5]], 0).contiguous()
        cd_all = torch.cat([d["curl_div"][:n], got[:, 5:9]], 0).contiguous()
        # (4) in place for the later loops
        backend.set_inactive((1 - active).contiguous(), h_all, rho_all, cd_all)
    # (5) gradient and force of the owned particles
    f = backend.gradient_force(loc_u)
    red = f["reductions"]
    # (6) the global sums
    if world > 1:
        dist.all_reduce(red)
    out = {"h": d["h"][:n], "rho4": d["rho4"][:n], "curl_div": d["curl_div"][:n],
           "ngb": d["ngb"][:n] if d.get("ngb") is not None else None,
           "vsig_lapu": f["vsig_lapu"][:n], "accel_dudt": f["accel_dudt"][:n], "dh_dt": f["dh_dt"][:n],
           "reductions": red, "ghosts": ng}
    return out
