"""Write tests/golden/lattice8_oracle.txt: FP64 oracle outputs on a small seeded case.

The paper prints no worked example of Eqs. 2-22, so this fixture is a stored
regression of the oracle itself (the oracle is pinned to closed forms and
invariants in tests/test_oracle_*.py). It calls only oracle/ and the seeded
input generator. Run from the repository root:

    python tests/golden/write_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2505_14538_b300 import ics  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lattice8_oracle.txt")


def case():
    """8^3 lattice, jitter 0.2 spacing, v ~ N(0, 0.3^2), u ~ U(0.5, 1.5), seeds fixed."""
    d = ics.lattice(8, jitter=0.2)
    rng = np.random.default_rng(20250514)
    n = len(d["pos"])
    vel = rng.normal(0, 0.3, (n, 3)).astype(np.float32)
    u = rng.uniform(0.5, 1.5, n).astype(np.float32)
    sample = np.sort(rng.choice(n, 32, replace=False))
    return d, vel, u, sample


def main():
    O.build()
    d, vel, u, sample = case()
    p = O.Params(h_tol=1e-13, max_iter=60)
    s = O.step(p, d["pos"], vel, d["m"], u, d["h"], solve=True)
    with open(OUT, "w") as f:
        f.write("# FP64 oracle on tests/golden/write_golden.py:case() (8^3 jittered lattice, 512 particles),\n")
        f.write("# h solved to h_tol 1e-13 (Sec. 2.1.2), then Eqs. 2-11, 16-20, 22 at that h.\n")
        f.write("# columns: index h rho ngb ax ay az dudt s_a s_u\n")
        for i in sample:
            a = s["accel"][i]
            f.write(f"{i} {s['h'][i]:.17g} {s['rho'][i]:.17g} {int(s['ngb'][i])} {a[0]:.17g} {a[1]:.17g} "
                    f"{a[2]:.17g} {s['dudt'][i]:.17g} {s['s_a'][i]:.17g} {s['s_u'][i]:.17g}\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
