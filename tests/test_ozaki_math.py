"""The arithmetic of the FP64-accurate tensor-core products (csrc/ozaki_math.cuh), compiled for
the host and checked against exact rational arithmetic. The GPU runs the same functions; the
BF16 slice GEMMs between them are exact integer sums (each product below 2^14, each sum of at
most 1024 of them below 2^24), which this test forms with Python integers.

* oz_slices: every slice is an integer of at most 7 bits (exact in BF16) with the sign of x,
  and sum_p d_p 2^(-7 (p+1)) 2^(e+1) is |x| truncated to 56 bits below the scale 2^(e+1).
* oz_to_double: (th 2^28 + tl) 2^(s - 63) rounded to the nearest double, ties to even.
* A whole emulated dot product (slices, the 36 pairs with p + q <= 9, level sums th and tl as
  the epilogues form them, one rounding) is within 4 n 2^-53 2^(ex + ey + 2) of the exact
  one, the bound the GPU tests state, including graded vectors.
"""
import math
import shutil
import struct
import subprocess
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

CSRC = Path(__file__).resolve().parents[1] / "paper_2109_13655_gb300" / "csrc"

DRIVER = r"""
#include "ozaki_math.cuh"
#include <cstdio>
using namespace cmsvd;
int main() {
    char op;
    while (scanf(" %c", &op) == 1) {
        if (op == 'S') {            // S <x bits> <e>: the 8 slices
            unsigned long long b; int e;
            if (scanf("%llx %d", &b, &e) != 2) return 1;
            float d[OZ_S];
            oz_slices(oz_from_bits(b), e, d);
            for (int p = 0; p < OZ_S; ++p) printf("%.1f ", d[p]);
            printf("\n");
        } else if (op == 'I') {     // I <x bits>: oz_ilogb
            unsigned long long b;
            if (scanf("%llx", &b) != 1) return 1;
            printf("%d\n", oz_ilogb(oz_from_bits(b)));
        } else if (op == 'D') {     // D <th> <tl> <s>
            long long th, tl; int s;
            if (scanf("%lld %lld %d", &th, &tl, &s) != 3) return 1;
            printf("%016llx\n", (unsigned long long)oz_bits(oz_to_double(th, tl, s)));
        }
        fflush(stdout);
    }
    return 0;
}
"""


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def from_bits(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("oz")
    src = d / "oz.cpp"
    src.write_text(DRIVER)
    exe = d / "oz"
    subprocess.run([cxx, "-O2", "-std=c++17", f"-I{CSRC}", str(src), "-o", str(exe)], check=True)

    def run(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return out.stdout.strip().splitlines()
    return run


def ilogb(x):
    return math.frexp(abs(x))[1] - 1


def slices(driver, xs, es):
    out = driver([f"S {bits(float(x)):x} {e}" for x, e in zip(xs, es)])
    return [[int(float(v)) for v in line.split()] for line in out]


def test_ilogb_from_the_exponent_field(driver):
    xs = [1.0, 0.75, 3.0, -1e300, 2.0 ** -1022, 1.5e-310, 7.0e22]
    got = [int(v) for v in driver([f"I {bits(x):x}" for x in xs])]
    for x, g in zip(xs, got):
        if abs(x) >= 2.0 ** -1022:
            assert g == ilogb(x)
        else:
            assert g == -1023 and abs(x) < 2.0 ** (g + 1)   # a bound for subnormals


def test_slices_are_7_bit_integers_reconstructing_56_bits(driver):
    rng = np.random.default_rng(3)
    xs = list(rng.standard_normal(400) * 10.0 ** rng.uniform(-20, 20, 400))
    xs += [0.0, -0.0, 1.0, -1.0, 2.0 ** -1074, -3.5e-310]
    cases = []
    for x in xs:
        e0 = ilogb(x) if x != 0 else 0
        for de in (0, 1, 9, 40, 60):                  # the scale of a larger entry in the group
            cases.append((x, e0 + de))
    got = slices(driver, [c[0] for c in cases], [c[1] for c in cases])
    for (x, e), d in zip(cases, got):
        assert all(abs(v) <= 127 for v in d)
        assert all(v == 0 or (v > 0) == (math.copysign(1.0, x) > 0) for v in d)
        V = sum(abs(v) << (7 * (7 - p)) for p, v in enumerate(d))
        exact = math.floor(abs(Fraction(x)) * Fraction(2) ** (56 - e - 1))
        assert V == exact, (x, e)


def test_to_double_rounds_once_to_nearest_even(driver):
    rng = np.random.default_rng(4)
    cases = []
    for _ in range(300):
        th = int(rng.integers(-2 ** 52, 2 ** 52))
        tl = int(rng.integers(-2 ** 52, 2 ** 52))
        cases.append((th, tl, int(rng.integers(-900, 900))))
    # ties: T = 2^53 + 1 (odd last place) and 2^53 + 3 scaled so one bit is dropped
    cases += [(0, (1 << 53) + 1, 0), (0, (1 << 53) + 3, 0), (1, 1, 0), (0, 0, 5), (-1, 0, -2000), (1, 0, 2000)]
    out = driver([f"D {th} {tl} {s}" for th, tl, s in cases])
    for (th, tl, s), got in zip(cases, out):
        g = from_bits(int(got, 16))
        exact = Fraction(th * (1 << 28) + tl) * Fraction(2) ** (s - 63)
        if exact == 0:
            assert g == 0.0
        elif abs(exact) < Fraction(2) ** -1022:
            assert g == 0.0 or abs(g) == 2.0 ** -1022
        elif abs(exact) >= Fraction(2) ** 1024:
            assert math.isinf(g)
        else:
            assert g == float(exact), (th, tl, s)   # Fraction -> float rounds to nearest even


def emulated_dot(driver, x, y):
    """x . y as the GPU forms it: slices on the scales of max|x| and max|y|, the 36 pairs with
    p + q <= 9, exact level sums, th / tl, one rounding."""
    ex = max(ilogb(v) for v in x if v != 0)
    ey = max(ilogb(v) for v in y if v != 0)
    dx = slices(driver, x, [ex] * len(x))
    dy = slices(driver, y, [ey] * len(y))
    s = {k: 0 for k in range(2, 10)}
    for p in range(8):
        for q in range(8):
            k = p + q + 2
            if k > 9:
                continue
            # the tensor cores sum at most 1024 of these products exactly in FP32
            part = 0
            for i in range(len(x)):
                part += dx[i][p] * dy[i][q]
                if (i + 1) % 1024 == 0 or i + 1 == len(x):
                    assert abs(part) < 2 ** 24
                    s[k] += part
                    part = 0
    th = sum(s[k] << (7 * (5 - k)) for k in range(2, 6))
    tl = sum(s[k] << (7 * (9 - k)) for k in range(6, 10))
    assert abs(th) < 2 ** 53 and abs(tl) < 2 ** 53
    g = from_bits(int(driver([f"D {th} {tl} {ex + ey + 2}"])[0], 16))
    return g, ex, ey


@pytest.mark.parametrize("n,graded", [(50, False), (2500, False), (2500, True)])
def test_emulated_dot_within_the_bound(driver, n, graded):
    rng = np.random.default_rng(n + graded)
    for _ in range(3):
        x = rng.standard_normal(n)
        y = rng.standard_normal(n)
        if graded:
            x *= 10.0 ** rng.uniform(-3, 3, n)
            y *= 10.0 ** rng.uniform(-3, 3, n)
        g, ex, ey = emulated_dot(driver, list(x), list(y))
        exact = sum(Fraction(a) * Fraction(b) for a, b in zip(x, y))
        err = abs(Fraction(g) - exact)
        assert err <= Fraction(4 * n) * Fraction(2) ** (-53 + ex + ey + 2)
