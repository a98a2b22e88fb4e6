"""Host logic of the fused float64-accurate series kernel (CPU): the balanced base-32 digits
it cuts every fixed-point value into, against exact integer arithmetic, and the exactness
bounds its shape rests on (diagonal sums below 2^24, Horner chains within int64).  A small
driver (tests/fused_digits_check.cu) is compiled for the host with nvcc."""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2409_19156_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("fused") / "check")
    src = os.path.join(ROOT, "tests", "fused_digits_check.cu")
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", os.path.join(ROOT, "include"),
                    "-I", CSRC, src, "-o", exe], check=True, capture_output=True)
    return exe


def run(exe, text):
    return subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")


def constants(exe):
    beta, digits, sets, max_modes, chunk, bias = (int(v) for v in run(exe, "c\n")[0].split())
    return beta, digits, sets, max_modes, chunk, bias


def test_constants_and_exactness_bounds(driver):
    beta, s, sets, max_modes, chunk, bias = constants(driver)
    assert beta * s >= 55  # at least 55 fraction bits: float64 accuracy with the scale 2^1 on |Z| <= 1
    assert chunk == s * sets * 64
    assert bias == sum((1 << (beta - 1)) << (beta * t) for t in range(s - 1))
    # Diagonal d sums over K modes: two pairs with the top digit (|a_1| <= 2^beta, the rest
    # below 2^(beta-1)) and d - 3 pairs of lower digits, largest at d = s + 1.
    per_k = 2 * (1 << beta) * (1 << (beta - 1)) + (s - 2) * (1 << (beta - 1)) ** 2
    assert max_modes * per_k < 1 << 24 <= (max_modes + 1) * per_k
    # Horner chains: diagonals 2..6 and 7..s+1 with |T_d| < 2^24 stay within int64.
    split = 5
    hi = sum((1 << 24) << (beta * (split - 1 - i)) for i in range(split))
    lo = sum((1 << 24) << (beta * (s - split - 1 - i)) for i in range(s - split))
    assert hi < 1 << 63 and lo < 1 << 63
    # ... and the joined 128-bit value is their exact combination.
    assert (hi << (beta * (s - split))) + lo < 1 << 127


def balanced_digits(x, beta, s):
    """Exact balanced digits of x, least significant position cut first, top digit the rest."""
    out = []
    half, full = 1 << (beta - 1), 1 << beta
    for _ in range(s - 1):
        low = x & (full - 1)
        d = low - full if low >= half else low
        out.append(d)
        x = (x - d) >> beta
    out.append(x)
    return out[::-1]


def test_digits_against_exact_arithmetic(driver):
    beta, s, _, _, _, _ = constants(driver)
    rng = random.Random(11)
    lim = 1 << (beta * s)
    xs = [0, 1, -1, 15, 16, -16, -17, lim - 1, -(lim - 1), lim, -lim, (1 << 54), -(1 << 54), 12345678901234567]
    xs += [rng.randrange(-lim, lim + 1) for _ in range(3000)]
    out = run(driver, "".join(f"d {x}\n" for x in xs))
    for x, line in zip(xs, out):
        got = [int(v) for v in line.split()]
        assert got == balanced_digits(x, beta, s), x
        assert sum(d << (beta * (s - 1 - t)) for t, d in enumerate(got)) == x
        assert all(-(1 << (beta - 1)) <= d < (1 << (beta - 1)) for d in got[1:])
        assert abs(got[0]) <= (1 << beta) + 1


def test_short_shape_bounds_and_digits(driver):
    """The 9-digit shape (6-bit digits) for contractions of at most 1489 positions: at least 54
    fraction bits, diagonal sums below 2^24 up to the limit and not one position beyond, Horner
    chains (4 and 5 diagonals) within int64, the shape chosen exactly up to the limit, and its
    digits against exact arithmetic."""
    beta, s, max_modes, bias, at_limit, past_limit = (int(v) for v in run(driver, "c9\n")[0].split())
    assert (beta, s) == (6, 9) and beta * s >= 54
    assert bias == sum((1 << (beta - 1)) << (beta * t) for t in range(s - 1))
    # the last kept diagonal (t + u = s + 1) holds two pairs with a top digit (|a_1| <= 2^beta)
    # and s - 2 pairs of lower digits (< 2^(beta-1) in magnitude)
    per_k = 2 * (1 << beta) * (1 << (beta - 1)) + (s - 2) * (1 << (beta - 1)) ** 2
    assert max_modes * per_k < 1 << 24 <= (max_modes + 1) * per_k
    assert (at_limit, past_limit) == (9, 11)
    split = 4
    hi = sum((1 << 24) << (beta * (split - 1 - i)) for i in range(split))
    lo = sum((1 << 24) << (beta * (s - split - 1 - i)) for i in range(s - split))
    assert hi < 1 << 63 and lo < 1 << 63
    rng = random.Random(12)
    lim = 1 << (beta * s)
    xs = [0, 1, -1, 31, 32, -32, -33, lim - 1, -(lim - 1), lim, -lim, 98765432109876]
    xs += [rng.randrange(-lim, lim + 1) for _ in range(3000)]
    out = run(driver, "".join(f"d9 {x}\n" for x in xs))
    for x, line in zip(xs, out):
        got = [int(v) for v in line.split()]
        assert got == balanced_digits(x, beta, s), x
        assert sum(d << (beta * (s - 1 - t)) for t, d in enumerate(got)) == x
        assert all(-(1 << (beta - 1)) <= d < (1 << (beta - 1)) for d in got[1:])
        assert abs(got[0]) <= (1 << beta) + 1
