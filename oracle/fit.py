"""Weighted least-squares fit of Zernike series coefficients.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Definition: C = argmin_C  sum_p w_p || sum_j Z_j(p) C[j, :] - Y[p, :] ||^2 + ridge ||C||^2,
whose minimiser solves the normal equations (Z W Z^T + ridge I) C = Z W Y (Z = basis [J][P],
W = diag(w)).  Z comes from oracle.basis (correctly rounded); the products and the solve use
numpy's float64 matmul and LAPACK-backed solve as library steps.
"""
from __future__ import annotations

import numpy as np

from . import basis as _basis


def normal_matrix(ns, ms, rs, thetas, weights=None):
    """Z W Z^T [J][J] and Z [J][P]."""
    Z = np.array(_basis.basis_table(ns, ms, rs, thetas, 0)[0][0])
    w = np.ones(len(rs)) if weights is None else np.asarray(weights, dtype=np.float64)
    return (Z * w) @ Z.T, Z


def series_fit(ns, ms, rs, thetas, samples, weights=None, ridge: float = 0.0) -> np.ndarray:
    """C [J][S] for samples Y [P][S]."""
    A, Z = normal_matrix(ns, ms, rs, thetas, weights)
    w = np.ones(len(rs)) if weights is None else np.asarray(weights, dtype=np.float64)
    b = (Z * w) @ np.asarray(samples, dtype=np.float64)
    return np.linalg.solve(A + ridge * np.eye(len(A)), b)
