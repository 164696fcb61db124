"""Write the stored oracle trajectories under tests/golden/.

Calls only the CPU oracle.  The small parity workload: 2D square lattice,
L = 16, J = 1, T = T_c = 2 / ln(1 + sqrt 2), random start from seed 1,
10^4 updates.  Also a 3D simple-cubic L = 8 run at T = 4.5115, seed 3.
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402

TC2 = 2.0 / math.log(1.0 + math.sqrt(2.0))
KEEP = 1000


def write(name, dim, L, T, seed, n):
    thr = oracle.bond_threshold(1.0, T)
    s = oracle.init_lattice(dim, L, seed)
    rec = oracle.run(dim, L, thr, seed, 0, n, s)
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        f.write("# oracle trajectory: dim=%d L=%d J=1 T=%.17g seed=%d updates=%d thr=%d\n"
                % (dim, L, T, seed, n, thr))
        f.write("# final lattice sum of (i+1)*(s_i+1)/2 mod 2^61-1: %d\n"
                % (int(((np.arange(len(s), dtype=np.int64) + 1) * ((s.astype(np.int64) + 1) // 2)).sum())
                   % (2**61 - 1)))
        f.write("# sums over all updates: C=%d levels=%d E_bond=%d M=%d\n"
                % (int(rec["C"].astype(np.int64).sum()), int(rec["levels"].astype(np.int64).sum()),
                   int(rec["E"].sum()), int(rec["M"].sum())))
        f.write("# t C levels E_bond M  (first %d updates)\n" % KEEP)
        for t, r in enumerate(rec[:KEEP]):
            f.write("%d %d %d %d %d\n" % (t, r["C"], r["levels"], r["E"], r["M"]))
    return path


if __name__ == "__main__":
    print(write("c1_2d_L16_seed1.txt", 2, 16, TC2, 1, 10_000))
    print(write("c3small_3d_L8_seed3.txt", 3, 8, 4.5115, 3, 2_000))
