"""Shared helpers for the GPU parity tests (not collected: no test_ prefix)."""
from __future__ import annotations

import numpy as np


def radial_tolerance(n, k: int) -> np.ndarray:
    """Parity bound for d^k/drho^k R_n^m: 1e-11 * max(n, 1)^(2k) (n = 0 has exact-zero derivatives)."""
    n = np.maximum(np.asarray(n, dtype=np.float64), 1.0)
    return 1e-11 * n ** (2 * k)


def assert_radial_close(got: np.ndarray, want: np.ndarray, ns, what: str = "") -> dict:
    """got/want [K][J][P]; per-mode tolerances; returns max abs error per k."""
    K = got.shape[0]
    stats = {}
    for k in range(K):
        err = np.abs(got[k] - want[k])
        tol = radial_tolerance(ns, k)[:, None]
        bad = err > tol
        if bad.any():
            j, p = np.argwhere(bad)[0]
            raise AssertionError(f"{what} k={k}: mode index {j} (n={ns[j]}) point {p}: got {got[k][j][p]!r} "
                                 f"want {want[k][j][p]!r} err {err[j][p]:.3e} tol {tol[j][0]:.3e}")
        stats[k] = float(err.max()) if err.size else 0.0
    return stats
