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


def test_bench_parity_check_reports_planted_errors():
    """The benchmark's parity leg (timed GPU output against the exact oracle at sampled points)
    passes values within the tolerance and flags a planted error beyond it: on the CPU, with
    the oracle's own values standing in for the GPU output."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2409_19156_gb300 import inputs

    ns, ms = (list(map(int, v)) for v in inputs.radial_modes(12))
    rs = [0.0, 0.25, 0.8, 1.0]
    exact = np.array(radial.radial_table(ns, ms, rs, 3))
    max_abs, worst = bench._oracle_parity_chunk((ns, ms, rs, exact))
    assert max_abs == [0.0, 0.0, 0.0, 0.0] and worst == 0.0
    planted = exact.copy()
    j = ns.index(12)
    planted[2, j, 1] += 2e-11 * 12 ** 4  # twice the k = 2 tolerance at n = 12
    max_abs, worst = bench._oracle_parity_chunk((ns, ms, rs, planted))
    assert abs(worst - 2.0) < 1e-6 and max_abs[2] > 0 and max_abs[0] == 0.0
