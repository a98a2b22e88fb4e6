"""GB300-native (sm_103a) Zernike basis and series library.

The compute lives in a C-ABI CUDA library (include/zernike_gb300.h, sources in csrc/);
this package is its build step and a thin torch-facing binding.
"""
from .api import (PREC, Batch, Plan, ZernikeSeries, basis, radial, radial_per_mode, series_adjoint,  # noqa: F401
                  series_eval, series_fit, series_point_hessian, series_point_hvp, zernike_series)
from ._lib import ZernikeError, library_path, load  # noqa: F401
