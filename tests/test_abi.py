"""The C-ABI library builds, loads and exports every symbol declared in include/*.h; host-side
validation paths that need no GPU behave as documented."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_2409_19156_gb300 import _lib, build as zbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"^ZP_API\s+[\w\s\*]+?\b(zp_\w+)\s*\(", text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    zbuild.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["zp_radial", "zp_basis", "zp_series_eval", "zp_series_adjoint", "zp_plan_create",
                     "zp_plan_destroy", "zp_status_string"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (zp_\w+)", out))
    missing = declared_symbols() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    for name in declared_symbols():
        assert hasattr(lib, name)


def test_binding_signatures_cover_header(lib):
    assert declared_symbols() <= set(_lib.SIGNATURES)


def test_library_targets_sm_103a_only():
    assert zbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings_and_version(lib):
    assert lib.zp_status_string(0) == b"ok"
    assert b"mode" in lib.zp_status_string(2)
    assert lib.zp_version() >= 100


def _i32(vals):
    arr = (ctypes.c_int32 * len(vals))(*vals)
    return ctypes.cast(arr, _lib.c_i32p), arr


@pytest.mark.parametrize("n,m", [([3], [0]), ([2], [4]), ([-1], [0]), ([4, 5], [0, 2]), ([2000], [0])])
def test_invalid_modes_rejected_before_any_device_work(lib, n, m):
    pn, keep_n = _i32(n)
    pm, keep_m = _i32(m)
    h = ctypes.c_void_p()
    st = lib.zp_plan_create(pn, pm, len(n), ctypes.byref(h))
    assert st == 2  # ZP_ERR_INVALID_MODE
    assert h.value is None
    assert b"mode" in lib.zp_last_error()


def test_derivative_order_rejected(lib):
    pn, keep_n = _i32([2])
    pm, keep_m = _i32([0])
    for k in (-1, 4):
        assert lib.zp_radial(pn, pm, 1, None, 10, k, None, None) == 3  # ZP_ERR_DERIV_ORDER


def test_negative_sizes_rejected(lib):
    pn, keep_n = _i32([2])
    pm, keep_m = _i32([0])
    assert lib.zp_radial(pn, pm, 1, None, -1, 0, None, None) == 1
    h = ctypes.c_void_p()
    assert lib.zp_plan_create(pn, pm, -1, ctypes.byref(h)) == 1
    assert lib.zp_plan_create(None, None, 3, ctypes.byref(h)) == 1


def test_no_cpu_fallback_anywhere(monkeypatch, tmp_path):
    """The Python layer refuses host tensors instead of computing on the CPU, and a missing
    shared library raises instead of falling back."""
    torch = pytest.importorskip("torch")
    import paper_2409_19156_gb300 as zp

    r = torch.linspace(0, 1, 8, dtype=torch.float64)
    for call in (lambda: zp.radial([2], [0], r, 1),
                 lambda: zp.basis([2], [0], r, r, 0),
                 lambda: zp.series_eval([2], [0], r, r, torch.ones(1, 3, dtype=torch.float64), "bf16x3"),
                 lambda: zp.series_fit([2], [0], r, r, torch.ones(8, 3, dtype=torch.float64))):
        with pytest.raises(TypeError, match="CUDA tensor"):
            call()
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(zbuild, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load()


def test_probe_and_static_entry_validate_on_the_host(lib):
    res = (ctypes.c_double * 6)()
    assert lib.zp_probe_fp64(3, 100, None, res) == 1  # unknown operation
    assert lib.zp_probe_fp64(0, 0, None, res) == 1  # no iterations
    assert lib.zp_probe_fp64(0, 100, None, None) == 1
    pn, keep_n = _i32([0, 1])
    pm, keep_m = _i32([0, 1])
    # Sizes whose products would wrap around in 64 bits are refused before anything else.
    for sets in (1 << 40, (1 << 62) // 3):
        assert lib.zp_series_eval_static(pn, pm, 2, None, None, 10, None, sets, 1, None, None) == 1
        assert b"ZP_STATIC_SCRATCH_BYTES" in lib.zp_last_error()
    assert lib.zp_series_eval_static(pn, pm, 2, None, None, 10, None, 4, 0, None, None) == 1  # float64
