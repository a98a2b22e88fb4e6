"""Shape choice of the float64-emulating tensor-core GEMM (CPU; host driver built with g++):
every float32 sum of slice-digit products stays an exact integer below 2^24, the slices carry
at least 54 fraction bits, the K batches cover K, and the two int64 Horner chains of the
recombination cannot overflow.  The digit bound the exactness rests on (|a_1| <= 2^beta,
|a_t| <= 2^(beta-1) for t >= 2) is checked by cutting random numbers into balanced digits."""
import math
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2409_19156_gb300", "csrc")
BK = 64  # K values per chunk


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("emu") / "emu_shape")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, os.path.join(ROOT, "tests", "emu_shape_check.cpp"), "-o", exe],
                   check=True, capture_output=True)
    return exe


CASES = [(k, t) for k in (1, 7, 63, 64, 65, 325, 384, 561, 576, 2601, 50000, 100000, 1_000_000, 4_000_000, 16_000_000)
         for t in (1, 3, 6, 100, 303, 304, 10_000)]


def test_shapes_are_exact_and_cover_k(driver):
    text = "".join(f"{k} {t} 152\n" for k, t in CASES)
    out = subprocess.run([driver], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    for (K, tiles), line in zip(CASES, out):
        ok, beta, s, KC, cpb, nb, split, paired, planes, psplit = map(int, line.split())
        assert ok, (K, tiles)
        assert KC == -(-K // BK)
        assert beta * s >= 54
        # largest diagonal (t + u = s + 1): two products with the first digit, s - 2 without
        per_k = 2 * 2 ** beta * 2 ** (beta - 1) + (s - 2) * 2 ** (2 * beta - 2)
        assert cpb * BK * per_k < 2 ** 24, (K, tiles, beta, s, cpb)
        assert nb * cpb >= KC and (nb - 1) * cpb < KC and nb <= 1024
        tb = 24 + max(0, math.ceil(math.log2(nb)))  # bits of a diagonal summed over batches
        assert tb + beta * (split - 1) + 1 <= 63
        if s > split:
            assert tb + beta * (s - split - 1) + 1 <= 63
        if paired:
            # two neighbouring diagonals in one int32: T_d 2^beta + T_(d+1) below 2^31
            assert cpb * BK * per_k * (2 ** beta + 1) < 2 ** 31, (K, tiles, beta, s, cpb)
            assert planes == (s + 1) // 2
            tp = 31 + max(0, math.ceil(math.log2(nb)))  # bits of a plane summed over batches
            assert 1 <= psplit <= planes
            assert tp + 2 * beta * (psplit - 1) + 1 <= 63
            if planes > psplit:
                assert tp + 2 * beta * (planes - psplit - 1) + 1 <= 63
        else:
            assert planes == s and psplit == split
        if tiles >= 2 * 152 and nb == 1:
            # a large output takes one batch with the fewest slice pairs K allows
            assert beta == max(b for b, ss in ((7, 8), (6, 9), (5, 11), (4, 14))
                               if KC * BK * (2 ** (2 * b) + (ss - 2) * 2 ** (2 * b - 2)) < 2 ** 24)


def test_mixed_n32_shape_pairs_its_diagonals(driver):
    """561 modes (K = 576) over many output tiles: beta = 6, s = 9, one batch, and the nine
    diagonals travel as five int32 planes (the largest pair sum, 9 chunks x 64 x 2^12 x 2.75 x
    65 = 4.2e8, is far below 2^31)."""
    out = subprocess.run([driver], input="561 100000 152\n", capture_output=True, text=True, check=True).stdout
    assert list(map(int, out.split())) == [1, 6, 9, 9, 9, 1, 7, 1, 5, 3]


def test_contraction_too_long_is_refused(driver):
    out = subprocess.run([driver], input="1000000000 1 152\n", capture_output=True, text=True, check=True).stdout
    assert out.split()[0] == "0"


@pytest.mark.parametrize("beta,s", [(7, 8), (6, 9), (5, 11), (4, 14)])
def test_balanced_digit_bounds(beta, s):
    """x in [-1, 1] as a fixed-point integer with beta * s fraction bits, cut from the lowest
    digit up into balanced base-2^beta digits: the later digits lie in [-2^(beta-1), 2^(beta-1)),
    the leading one within 2^beta, and the digits rebuild x exactly."""
    rng = random.Random(beta * 100 + s)
    half, full, mask = 1 << (beta - 1), 1 << beta, (1 << beta) - 1
    for _ in range(3000):
        x = rng.choice([rng.uniform(-1, 1), 1.0, -1.0, rng.uniform(-1e-3, 1e-3)])
        X = round(x * 2 ** (beta * s))
        digits = []
        for _t in range(s - 1):
            low = X & mask
            d = low - full if low >= half else low
            digits.append(d)
            X = (X - d) >> beta
        digits.append(X)  # leading digit
        assert all(-half <= d < half for d in digits[:-1])
        assert abs(digits[-1]) <= full
        assert sum(d * 2 ** (beta * i) for i, d in enumerate(digits)) == round(x * 2 ** (beta * s))


@pytest.mark.parametrize("beta,s", [(7, 8), (6, 9), (5, 11), (4, 14)])
def test_biased_field_digits_match_the_carry_cut(driver, beta, s):
    """The slice kernels read the digits off the biased word X + slice_bias(beta, s) (fields
    minus 2^(beta-1), the top digit the rest); they must be exactly the digits of the carry cut
    above, for values of either sign, at the fixed-point limits and at zero."""
    rng = random.Random(beta * 1000 + s)
    half, full, mask = 1 << (beta - 1), 1 << beta, (1 << beta) - 1
    lim = 1 << (beta * s)
    xs = [0, 1, -1, half, -half, half - 1, -half - 1, lim - 1, -(lim - 1), lim, -lim]
    xs += [rng.randrange(-lim, lim + 1) for _ in range(2000)]
    text = "".join(f"d {beta} {s} {x}\n" for x in xs)
    out = subprocess.run([driver], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    for x, line in zip(xs, out):
        X, want = x, []
        for _t in range(s - 1):
            low = X & mask
            d = low - full if low >= half else low
            want.append(d)
            X = (X - d) >> beta
        want.append(X)
        assert [int(v) for v in line.split()] == want[::-1], x
