"""Write the per-interaction flop counts of the three loops to profiles/flops_per_interaction.json.

The counts come from the oracle's own pair functions instantiated on an
op-counting scalar (add/sub/mul/div/sqrt = 1 flop each; comparisons are not
flops). A hit falls in the inner spline branch (q < 1/2) with probability
1/8 (hits are uniform in the support volume), so each loop's figure is
1/8 inner + 7/8 outer. The Wendland kernels have one branch; their counts
are written under "wendland_c2" and "wendland_c4". The neighbour test is not
part of those counts; its own cost, the distance of the predicate
(r^2 = dx^2 + dy^2 + dz^2 from the three coordinate differences: 3 sub, 3 mul,
2 add; the comparison is not a flop, and the periodic image is applied once
per cell, not per pair), is written under "neighbour_test".
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from oracle import oracle as O  # noqa: E402


def main():
    out = {}
    for loop, name in ((0, "density"), (1, "gradient"), (2, "force"), (3, "h_iteration")):
        tot = {}
        for q, w in ((0.3, 0.125), (0.75, 0.875)):
            c = O.count_flops(loop, q, True)
            tot[q] = c["add"] + c["mul"] + c["div"] + c["sqrt"]
        out[name] = {"inner": tot[0.3], "outer": tot[0.75], "mean": 0.125 * tot[0.3] + 0.875 * tot[0.75]}
    for kind, key in ((O.WENDLAND_C2, "wendland_c2"), (O.WENDLAND_C4, "wendland_c4")):
        out[key] = {}
        for loop, name in ((0, "density"), (1, "gradient"), (2, "force"), (3, "h_iteration")):
            c = O.count_flops(loop, 0.5, True, kind)
            out[key][name] = c["add"] + c["mul"] + c["div"] + c["sqrt"]
    out["neighbour_test"] = 3 + 3 + 2
    out["_how"] = ("oracle pair functions on an op-counting scalar; cubic spline mean = 1/8 inner-branch + 7/8 "
                   "outer-branch count; neighbour_test: the predicate's squared distance (3 sub, 3 mul, 2 add); "
                   "written by oracle/write_flop_counts.py")
    path = os.path.join(os.path.dirname(HERE), "profiles", "flops_per_interaction.json")
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
