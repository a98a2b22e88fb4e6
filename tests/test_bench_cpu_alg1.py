"""The benchmark's numpy restatement of Algorithm 1 (a CPU comparison program, not the
oracle) agrees with the oracle's exact radial values, so its timing is of correct work."""
import os
import sys

import numpy as np

from oracle import radial

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_alg1_numpy_column_matches_the_oracle():
    sys.path.insert(0, ROOT)
    import bench

    r = np.array([0.0, 0.1, 0.37, 0.5, 0.93, 1.0])
    for m, n_max in ((0, 40), (1, 41), (2, 30), (7, 37), (30, 60), (100, 100)):
        blk = bench.alg1_numpy_column(r, n_max, m)
        assert blk.shape == (4, (n_max - m) // 2 + 1, r.size)
        for j in range(blk.shape[1]):
            n = m + 2 * j
            for k in range(4):
                for p, rv in enumerate(r):
                    want = radial.radial(n, m, float(rv), k)
                    assert abs(blk[k, j, p] - want) <= 1e-11 * max(n, 1) ** (2 * k)
