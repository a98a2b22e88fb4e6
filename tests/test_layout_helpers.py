"""Host-side helpers of the tensor-core series path, against independent definitions (CPU):
the float64 -> float32 conversion by significand truncation that feeds the split operands,
and the byte offsets of the 128- and 64-byte swizzled K-major operand layouts.  A small
driver (tests/layout_helpers_check.cu) is compiled for the host with nvcc."""
import os
import random
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2409_19156_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("layout") / "check")
    src = os.path.join(ROOT, "tests", "layout_helpers_check.cu")
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", os.path.join(ROOT, "include"),
                    "-I", CSRC, src, "-o", exe], check=True, capture_output=True)
    return exe


def run(exe, text):
    return subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split()


def trunc_reference(x: float) -> int:
    """float32 bits of a float64 by truncation of its significand, from the IEEE layouts."""
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    sign, e, mant = b >> 63, (b >> 52) & 0x7FF, b & ((1 << 52) - 1)
    if e == 0x7FF:
        return (sign << 31) | 0x7F800000 | (0x400000 if mant else 0)
    if e <= 1023 - 127:  # below the float32 normal range
        return sign << 31
    if e >= 1023 + 128:  # above it
        return (sign << 31) | 0x7F800000
    return (sign << 31) | ((e - 1023 + 127) << 23) | (mant >> 29)


def test_truncating_conversion(driver):
    rng = random.Random(7)
    xs = [0.0, -0.0, 1.0, -1.0, 0.5, 1.5, 2.0 ** -126, 2.0 ** -127, -(2.0 ** -126), 2.0 ** 127,
          3.4028234663852886e38, 3.5e38, -3.5e38, float("inf"), float("-inf"), 1e-300, 5e-324,
          1.0 + 2.0 ** -23, 1.0 + 2.0 ** -24, 1.0 - 2.0 ** -53, 0.1, -0.7, 123456.789]
    xs += [rng.uniform(-1, 1) for _ in range(2000)]
    xs += [rng.uniform(-1, 1) * 2.0 ** rng.randint(-160, 160) for _ in range(4000)]
    bits = [struct.unpack("<Q", struct.pack("<d", x))[0] for x in xs]
    bits += [0x7FF8000000000000, 0x7FF0000000000001, 0xFFF4000000000000]  # NaNs
    got = run(driver, "".join(f"t {b:016x}\n" for b in bits))
    for b, g in zip(bits, got):
        x = struct.unpack("<d", struct.pack("<Q", b))[0]
        want = trunc_reference(x)
        assert int(g, 16) == want, (hex(b), g, hex(want))
        f = struct.unpack("<f", struct.pack("<I", int(g, 16)))[0]
        if np.isfinite(x) and 2.0 ** -126 <= abs(x) < 2.0 ** 128:
            # truncation: |f| <= |x| < |f| + ulp(f), same sign
            assert abs(f) <= abs(x) and np.copysign(1.0, f) == np.copysign(1.0, x)
            ulp = 2.0 ** (((int(g, 16) >> 23) & 0xFF) - 127 - 23)
            assert abs(x) < abs(f) + ulp
        if np.isnan(x):
            assert np.isnan(f)


@pytest.mark.parametrize("row_bytes", [128, 64])
def test_swizzled_offsets(driver, row_bytes):
    """Element (row, k) sits at logical byte row * R + k * size, with address bits 4.. of the
    16-byte unit XORed with the bits above the 8-row group's row index: bits [6:4] ^= [9:7] for
    128-byte rows, [5:4] ^= [8:7] for 64-byte rows; every offset is distinct and inside the tile."""
    got = [int(v) for v in run(driver, f"s {row_bytes}\n")]
    n16, n32 = 256 * (row_bytes // 2), 256 * (row_bytes // 4)
    assert len(got) == n16 + n32
    bbits = 3 if row_bytes == 128 else 2
    mask = ((1 << bbits) - 1) << 7

    def swizzle(logical):
        return logical ^ ((logical & mask) >> 3)

    want16 = [swizzle(r * row_bytes + k * 2) for r in range(256) for k in range(row_bytes // 2)]
    want32 = [swizzle(r * row_bytes + k * 4) for r in range(256) for k in range(row_bytes // 4)]
    assert got[:n16] == want16 and got[n16:] == want32
    assert sorted(got[:n16]) == list(range(0, 256 * row_bytes, 2))
    assert sorted(got[n16:]) == list(range(0, 256 * row_bytes, 4))
