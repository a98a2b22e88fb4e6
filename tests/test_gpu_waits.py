"""Failure detection without a GPU fault: a bounded device wait that runs out is reported to
the host as ZP_ERR_TIMEOUT and the context keeps working."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2409_19156_gb300 as zp  # noqa: E402
from paper_2409_19156_gb300 import _lib, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_is_reported():
    lib = _lib.load()
    assert lib.zp_device_wait_status(1) == 0  # clear
    assert lib.zp_device_wait_selftest(50, None) == 0
    torch.cuda.synchronize()
    assert lib.zp_device_wait_status(0) == 5  # ZP_ERR_TIMEOUT
    assert b"gave up" in lib.zp_last_error()
    assert lib.zp_device_wait_status(1) == 5  # read and clear
    assert lib.zp_device_wait_status(0) == 0
    # the context is still usable: a normal evaluation works afterwards
    ns, ms = inputs.full_zernike_modes(4)
    r, th = inputs.uniform_points(64, 1)
    out, _ = zp.basis(ns, ms, torch.as_tensor(r, device="cuda"), torch.as_tensor(th, device="cuda"), 0)
    torch.cuda.synchronize()
    assert np.isfinite(out.cpu().numpy()).all()
    assert lib.zp_device_wait_selftest(0, None) == 1  # argument checked on the host
