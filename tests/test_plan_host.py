"""The plan builder's host tables (CPU; a host driver compiled with nvcc builds them without a
GPU): the grouping of modes into |m| columns ordered by recursion length, the slot lists of
output columns per (column, Jacobi degree) with the sin flag of m < 0, the rescaled recursion
coefficients against exact rational arithmetic from the Jacobi recursion of Sec. 2, the seed
constants, and the split basis's per-step descriptors."""
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2409_19156_gb300", "csrc")
K_ROW, K_HEADER = 8, 2


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_check")
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", os.path.join(ROOT, "include"),
                    "-I", CSRC, os.path.join(ROOT, "tests", "plan_host_check.cu"), os.path.join(CSRC, "zp_plan.cpp"),
                    "-o", exe], check=True, capture_output=True)
    return exe


def build(exe, ns, ms):
    text = f"{len(ns)}\n" + "".join(f"{a} {b}\n" for a, b in zip(ns, ms))
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    it = iter(out)
    status = int(next(it).split()[1])
    if status:
        return status, None
    plan = {}
    for name in ("cols", "table", "slot_ptr", "slot_idx", "split_step"):
        head = next(it).split()
        assert head[0] == name
        rows = [next(it) for _ in range(int(head[1]))]
        if name == "cols":
            plan[name] = [tuple(map(int, r.split())) for r in rows]
        elif name == "table":
            plan[name] = [struct.unpack("<d", struct.pack("<Q", int(r, 16)))[0] for r in rows]
        else:
            plan[name] = [int(r) for r in rows]
    head = next(it).split()
    assert head[0] == "fused"
    ns_, units, kpad, ep = map(int, head[1:])
    plan["fused"] = {"streams": ns_, "units": units, "kpad": kpad, "ep": ep,
                     "ncols": [int(next(it)) for _ in range(ns_)]}
    for name in ("fused_col", "fused_kperm"):
        head = next(it).split()
        assert head[0] == name
        plan[name] = [int(next(it)) for _ in range(int(head[1]))]
    return 0, plan


def exact_rows(m, n_steps):
    """(A_N, B_N, w_N) of the rescaled recursion Q_N = (A_N rho^2 - B_N) Q_{N-1} - Q_{N-2}, from
    the Jacobi three-term recursion with alpha = m, beta = 0 written for R_N = R_{m+2N}^m."""
    w = [Fraction(1), Fraction(1)]
    rows = [(Fraction(0), Fraction(0), Fraction(1)), (Fraction(0), Fraction(0), Fraction(1))]
    for N in range(2, n_steps):
        D = Fraction(2 * N * (N + m) * (2 * N + m - 2))
        a = Fraction((2 * N + m - 1) * (2 * N + m) * (2 * N + m - 2)) / D
        b = Fraction((2 * N + m - 1) * m * m) / D
        c = Fraction(2 * (N + m - 1) * (N - 1) * (2 * N + m)) / D
        w.append(c * w[N - 2])
        rows.append((2 * a * w[N - 1] / w[N], (a + b) * w[N - 1] / w[N], w[N]))
    return rows[:n_steps]


def close(x, exact):
    return abs(Fraction(x) - exact) <= abs(exact) * Fraction(1, 2 ** 52)


def trunc_bits(x):
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    sign, e, mant = b >> 63, (b >> 52) & 0x7FF, b & ((1 << 52) - 1)
    assert 896 < e < 1151
    return (sign << 31) | ((e - 896) << 23) | (mant >> 29)


def test_plan_tables(driver):
    ns = [30, 4, 4, 9, 30, 0, 17, 4, 22, 12, 12, 12, 40, 1, 40] + [10] * 26
    ms = [0, 2, -2, 9, -4, 0, 1, 2, 22, -4, 4, -4, 0, -1, 38] + [2, -2] * 13
    st, plan = build(driver, ns, ms)
    assert st == 0
    cols, table = plan["cols"], plan["table"]
    # columns: one per distinct |m|, n_steps = largest degree + 1, longest first (stable in m)
    want = {}
    for n, m in zip(ns, ms):
        want[abs(m)] = max(want.get(abs(m), 0), (n - abs(m)) // 2 + 1)
    assert sorted((c[0], c[1]) for c in cols) == sorted(want.items())
    steps = [c[1] for c in cols]
    assert steps == sorted(steps, reverse=True)
    # slots: each mode exactly once at (its column, its degree), sin flag for m < 0
    col_of = {c[0]: i for i, c in enumerate(cols)}
    seen = []
    for j, (n, m) in enumerate(zip(ns, ms)):
        c = cols[col_of[abs(m)]]
        s = c[3] + (n - abs(m)) // 2
        codes = plan["slot_idx"][plan["slot_ptr"][s]:plan["slot_ptr"][s + 1]]
        assert (j | (0x80000000 if m < 0 else 0)) in codes
        seen.append(j)
    assert sorted(v & 0x7FFFFFFF for v in plan["slot_idx"]) == sorted(seen)
    # tables: header seeds and rescaled coefficients, each within one rounding of the exact value
    for am, n_steps, row0, sbase in cols:
        h = table[row0 * K_ROW:(row0 + K_HEADER) * K_ROW]
        assert h[0] == 1.0 and h[4] == am + 2 and h[8] == am + 1
        for N, (A, B, W) in enumerate(exact_rows(am, n_steps)):
            r = table[(row0 + K_HEADER + N) * K_ROW:(row0 + K_HEADER + N + 1) * K_ROW]
            assert close(r[0], A) and close(r[1], B) and close(r[3], W), (am, N)
            assert r[2] == 2 * r[0] and r[7] == 0.0
            assert close(r[5], 2 * W) and close(r[6], 6 * W)
            # split-basis step descriptor: slot count, sin flags (or "irregular"), float32 weight
            s = sbase + N
            codes = plan["slot_idx"][plan["slot_ptr"][s]:plan["slot_ptr"][s + 1]]
            word = plan["split_step"][2 * (row0 + K_HEADER + N)]
            if len(codes) > 24:
                assert word == 255
            else:
                flags = sum(((c >> 31) & 1) << i for i, c in enumerate(codes))
                assert word == len(codes) | (flags << 8)
            assert plan["split_step"][2 * (row0 + K_HEADER + N) + 1] == trunc_bits(r[3])


def check_fused_layout(plan):
    """The fused kernel's contraction layout: columns dealt to the streams, each column's
    outputs in whole 8-value units of its stream, unit j of stream s at global unit S j + s,
    every output slot exactly once in the K order, padding elsewhere, whole 32-position stages."""
    f, cols = plan["fused"], plan["cols"]
    S, units, nc = f["streams"], f["units"], len(cols)
    rec = [plan["fused_col"][4 * c:4 * c + 4] for c in range(nc)]
    lists = plan["fused_col"][4 * nc:]
    assert len(lists) == nc and sorted(lists) == list(range(nc))
    at = 0
    used = [0] * S
    for s in range(S):
        mine = lists[at:at + f["ncols"][s]]
        at += f["ncols"][s]
        for c in mine:  # walk order within the stream, units consecutive
            assert rec[c][1] == s and rec[c][2] == used[s]
            used[s] += -(-rec[c][3] // 8)
    assert at == nc
    G = units  # global units: stream s owns the g < G with g = s mod S
    assert G % 4 == 0 and all(used[s] <= (G - s + S - 1) // S for s in range(S))
    assert G < 4 or any(used[s] > (G - 4 - s + S - 1) // S for s in range(S))  # no whole stage to spare
    assert f["kpad"] == len(plan["fused_kperm"]) == 8 * G and f["kpad"] % 32 == 0
    # balance: round robin unless a stream runs more than two units ahead of the least loaded
    biggest = max((-(-r[3] // 8) for r in rec), default=0)
    assert max(used) - min(used) <= biggest + 2
    kperm = plan["fused_kperm"]
    want = {}
    for c, (kind, s, first, nvals) in enumerate(rec):
        am, n_steps, row0, sbase = cols[c]
        slot0 = plan["slot_ptr"][sbase]
        assert plan["slot_ptr"][sbase + n_steps] - slot0 == nvals
        for i in range(nvals):
            want[8 * (S * (first + i // 8) + s) + i % 8] = slot0 + i
    assert {k: v for k, v in enumerate(kperm) if v >= 0} == want
    assert sorted(want.values()) == list(range(len(plan["slot_idx"])))


def test_fused_layout(driver):
    for nmax in (0, 3, 10, 24, 32):
        ns = [n for n in range(nmax + 1) for m in range(-n, n + 1, 2)]
        ms = [m for n in range(nmax + 1) for m in range(-n, n + 1, 2)]
        st, plan = build(driver, ns, ms)
        assert st == 0
        check_fused_layout(plan)
        # a full mode set is dealt round robin: each stream's |m| advance by the stream count
        S, cols = plan["fused"]["streams"], plan["cols"]
        assert all(plan["fused_col"][4 * c + 1] == c % S for c in range(len(cols)))
        assert [c[0] for c in cols] == list(range(nmax + 1))
    # scrambled, duplicated and one-sided mode lists (irregular steps)
    ns = [30, 4, 4, 9, 30, 0, 17, 4, 22, 12, 12, 12, 40, 1, 40] + [10] * 26
    ms = [0, 2, -2, 9, -4, 0, 1, 2, 22, -4, 4, -4, 0, -1, 38] + [2, -2] * 13
    st, plan = build(driver, ns, ms)
    assert st == 0
    check_fused_layout(plan)


def test_fused_padded_lengths_around_the_short_digit_shape(driver):
    """The fused kernel cuts values into 9 digits of 6 bits when the padded contraction has at
    most 1489 positions, else 11 of 5 bits: the full sets n <= 49 (1275 modes, 1472 positions)
    and n <= 50 (1326 modes, 1504 positions) fall on either side, which the GPU tests rely on."""
    kp = {}
    for nmax in (49, 50):
        ns = [n for n in range(nmax + 1) for m in range(-n, n + 1, 2)]
        ms = [m for n in range(nmax + 1) for m in range(-n, n + 1, 2)]
        st, plan = build(driver, ns, ms)
        assert st == 0
        kp[nmax] = plan["fused"]["kpad"]
    assert kp[49] <= 1489 < kp[50]


@pytest.mark.parametrize("n,m", [(3, 2), (-1, 1), (2, 3), (1001, 1)])
def test_plan_rejects_invalid_modes(driver, n, m):
    st, _ = build(driver, [4, n], [0, m])
    assert st == 2  # ZP_ERR_INVALID_MODE
