"""The recombination's final rounding (CPU): join_to_double(H, L, ls, e2), the correctly
rounded float64 of (H 2^ls + L) 2^e2 formed with 64-bit words, against exact rational
arithmetic (Python's float of a Fraction rounds half to even) and against the 128-bit path it
replaces.  Cases cover both signs, carries of L into H, every rounding position (ties, the
mantissa overflowing to the next power of two), values of fewer than 54 bits, and exponents at
the edges of the normal range.  A small driver (tests/join_round_check.cu) is compiled for the
host with nvcc."""
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2409_19156_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("join") / "check")
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                    os.path.join(ROOT, "tests", "join_round_check.cu"), "-o", exe], check=True, capture_output=True)
    return exe


def exact(H, L, ls, e2):
    v = Fraction(H * 2 ** ls + L) * Fraction(2) ** e2
    try:
        return float(v)
    except OverflowError:
        return float("inf") if v > 0 else float("-inf")


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def cases():
    rng = random.Random(20240919)
    out = []
    for ls in (1, 5, 12, 24, 30, 40, 52, 53, 54, 62):
        for _ in range(300):
            hb = rng.randint(0, 61)
            H = rng.randint(-(2 ** hb), 2 ** hb)
            lb = rng.randint(0, min(61, ls + 20))
            L = rng.randint(-(2 ** lb), 2 ** lb)
            out.append((H, L, ls, rng.randint(-120, 40)))
        # ties and near-ties at the rounding position
        for _ in range(60):
            nb = rng.randint(30, 61)
            H = rng.choice([-1, 1]) * rng.randint(2 ** (nb - 1), 2 ** nb - 1)
            r = nb + ls - 53
            if r >= 1:
                base = (abs(H) * 2 ** ls) >> r << r
                for delta in (2 ** (r - 1), 2 ** (r - 1) - 1, 2 ** (r - 1) + 1, 0, 2 ** r - 1):
                    N = (base + delta) * (1 if H > 0 else -1)
                    Hq, Lq = divmod(N, 2 ** ls)
                    out.append((Hq, Lq, ls, rng.randint(-80, 20)))
        # mantissa of all ones rounding up to the next power of two
        for nb in (54, 60):
            N = (2 ** 53 - 1) * 2 ** (nb - 53) + 2 ** (nb - 54)
            Hq, Lq = divmod(N, 2 ** ls)
            if abs(Hq) < 2 ** 61:
                out.append((Hq, Lq, ls, -10))
                out.append((-Hq - 1, 2 ** ls - Lq, ls, -10))
    # small values (fewer than 54 bits), zero, and the edges of the normal range
    out += [(0, 0, 24, 0), (0, 5, 24, -3), (0, -(2 ** 40), 24, 7), (1, 0, 24, -1100), (-3, 7, 24, -1060),
            (2 ** 60, 0, 24, 1000), (2 ** 60, 123, 24, 939), (-(2 ** 60), -1, 24, 938), (1, 1, 62, -1136),
            (2 ** 62 + 5, 3, 20, -100), (-(2 ** 62) - 5, -3, 20, -100), (2 ** 63 - 1, 2 ** 40, 30, -120),
            (-(2 ** 63), -(2 ** 40), 30, -120)]
    return out


def test_join_matches_exact_rounding(driver):
    cs = cases()
    text = "".join(f"{H} {L} {ls} {e2}\n" for H, L, ls, e2 in cs)
    lines = subprocess.run([driver], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    assert len(lines) >= len(cs)
    for (H, L, ls, e2), line in zip(cs, lines):
        a, b = (int(w, 16) for w in line.split())
        want = exact(H, L, ls, e2)
        assert a == b, (H, L, ls, e2)
        assert a == bits(want), (H, L, ls, e2, hex(a), want)
