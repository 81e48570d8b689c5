"""The slab decomposition through the CUDA library (swift_gpu_set_inactive), two ranks in one process.

The two ranks' contexts run one after the other on one GPU, and the host
moves the halo data between them (the same steps decomposed_step takes with
torch.distributed between processes): ghost inputs, the density of each
rank's owned particles, the owners' results for the ghosts put in place with
swift_gpu_set_inactive, then the fused gradient + force of the owned
particles. The assembled outputs meet every tolerance of the single-domain
parity test against the FP64 oracle, and the summed reductions match the
whole set's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_14538_b300 import ics

pytestmark = pytest.mark.gpu


def test_two_slabs_match_the_oracle(O):
    from paper_2505_14538_b300 import domain, sph
    from test_gpu_parity import check_against_oracle, lattice_state
    d, vel, u = lattice_state(20, seed=41, jitter=0.3)
    n = len(d["pos"])
    dev = torch.device("cuda")
    pos_h = torch.from_numpy(np.c_[d["pos"], d["h"]].astype(np.float32)).to(dev)
    vel_m = torch.from_numpy(np.c_[vel, d["m"]].astype(np.float32)).to(dev)
    uu = torch.from_numpy(u.astype(np.float32)).to(dev)
    slabs = domain.Slabs(1.0, domain.slab_count(1.0, float(d["h"].max()), O.KERNEL_GAMMA), 2)
    owner = slabs.owner(pos_h[:, 2])
    own = [torch.nonzero(owner == r)[:, 0] for r in range(2)]
    masks = [slabs.send_masks(r, pos_h[own[r], 2])[1 - r] for r in range(2)]
    # rank r's local set: its owned particles, then the other rank's boundary layers
    ghosts = [own[1 - r][masks[1 - r]] for r in range(2)]
    loc = [torch.cat([own[r], ghosts[r]]) for r in range(2)]
    be = [domain.ContextBackend(len(loc[r]), slabs.width, h_tol=1e-6) for r in range(2)]
    act = [torch.cat([torch.ones(len(own[r]), dtype=torch.uint8, device=dev),
                      torch.zeros(len(ghosts[r]), dtype=torch.uint8, device=dev)]) for r in range(2)]
    dens = [be[r].density(pos_h[loc[r]].contiguous(), vel_m[loc[r]].contiguous(), act[r]) for r in range(2)]
    out = {}
    for r in range(2):
        no = len(own[r])
        src = dens[1 - r]  # the owner's results for the particles it sent, in its owned order
        m = masks[1 - r]
        h_all = torch.cat([dens[r]["h"][:no], src["h"][:len(own[1 - r])][m]]).contiguous()
        rho_all = torch.cat([dens[r]["rho4"][:no], src["rho4"][:len(own[1 - r])][m]]).contiguous()
        cd_all = torch.cat([dens[r]["curl_div"][:no], src["curl_div"][:len(own[1 - r])][m]]).contiguous()
        be[r].set_inactive((1 - act[r]).contiguous(), h_all, rho_all, cd_all)
        f = be[r].gradient_force(uu[loc[r]].contiguous())
        assert be[r].status() == (0, 0)
        for k, v in (("h", dens[r]["h"]), ("rho4", dens[r]["rho4"]), ("curl_div", dens[r]["curl_div"]),
                     ("ngb", dens[r]["ngb"]), ("vsig_lapu", f["vsig_lapu"]), ("accel_dudt", f["accel_dudt"]),
                     ("dh_dt", f["dh_dt"])):
            a = out.setdefault(k, np.zeros((n,) + tuple(v.shape[1:]), np.float32 if k != "ngb" else np.int64))
            a[own[r].cpu().numpy()] = v[:no].cpu().numpy()
        out.setdefault("red", []).append(f["reductions"].cpu().numpy())
    red = out.pop("red")
    out["reductions"] = red[0] + red[1]
    ref = sph.Context(n, h_tol=1e-6)
    ref.build_cells(pos_h, be[0].width)
    ref.density(pos_h, vel_m)
    out["info"] = ref.info()  # the same cell grid, hence the same h cap as the slabs
    assert out["info"]["nc"][2] == slabs.nc
    check_against_oracle(O, d, vel, u, out, ref)
