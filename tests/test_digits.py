"""The split's digit step (csrc/oz_digits.cuh), host-compiled, against its definition in exact
rational arithmetic: for an entry x of a column whose largest magnitude is c, E = ilogb(c) + 2,
N = round(x 2^(6 s - E)) to nearest with ties to even, and the balanced base-64 digits of N
(d_{s-1}, ..., d_1 in [-32, 31] taken from the least significant end, d_0 the rest), so that
N = sum_i d_i 64^(s-1-i) and |x - 2^(E-6s) N| <= 2^(E-6s-1).  The scale 2^(6 s - E) is clamped
to [2^-1022, 2^1023] (a column whose largest magnitude is below 2^-975 keeps fewer bits)."""
import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _bf16(h):
    return struct.unpack("<f", struct.pack("<I", int(h, 16) << 16))[0]


def _expected(x, c, s):
    """E and the digits by the definition (Fractions: exact)."""
    if c == 0.0:
        E = -400
    else:
        E = math.frexp(abs(c))[1] - 1 + 2            # ilogb(c) + 2 for normal c
        if abs(c) < 2.0 ** -1022:
            E = -1023 + 2                             # subnormal columns count as 2^-1023
    sh = max(-1022, min(1023, 6 * s - E))
    N = round(Fraction(x) * Fraction(2) ** sh)       # Fraction rounding: half to even
    digits = []
    n = N
    for _ in range(s - 1):
        d = (n + 32) % 64 - 32
        digits.append(d)
        n = (n - d) // 64
    digits.append(n)
    return E, N, digits[::-1]


def _cases(rng):
    out = []
    for _ in range(4000):
        s = rng.randint(3, 8)
        ex = rng.randint(-1070, 1020)
        c = math.ldexp(0.5 + 0.5 * rng.random(), ex)
        kind = rng.randrange(6)
        if kind == 0:
            x = c * rng.uniform(-1.0, 1.0)
        elif kind == 1:
            x = math.ldexp(rng.uniform(-1.0, 1.0), ex - rng.randrange(60))
        elif kind == 2:                               # an exact tie after scaling
            E = math.frexp(c)[1] + 1
            x = math.ldexp(2 * rng.randrange(1 << (6 * s - 3)) + 1, E - 6 * s - 1) * rng.choice((1, -1))
            x = max(-c, min(c, x))
        elif kind == 3:
            x = rng.choice((0.0, -0.0))
        elif kind == 4:
            x = math.ldexp(rng.uniform(-1.0, 1.0), -1074 + rng.randrange(60))
        else:
            x = rng.choice((c, -c))
        out.append((x, c, s))
    out += [(0.0, 0.0, s) for s in range(3, 9)]      # an all-zero column
    return out


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("ozd") / "oz_digits_host")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "host", "oz_digits_host.cu")],
                   check=True, capture_output=True)
    return exe


def test_digit_step_matches_definition(driver):
    cases = _cases(random.Random(20250923))
    inp = "".join(f"{_bits(x):016x} {_bits(c):016x} {s}\n" for x, c, s in cases)
    out = subprocess.run([driver], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for (x, c, s), line in zip(cases, out):
        f = line.split()
        E, N, digits = _expected(x, c, s)
        assert int(f[0]) == E, (x, c, s)
        got = [_bf16(h) for h in f[1:]]
        assert got == digits, (x, c, s, got, digits)
        assert all(-32 <= d <= 31 for d in digits[1:])
        assert sum(d * 64 ** (s - 1 - i) for i, d in enumerate(digits)) == N
        if c != 0.0 and 6 * s - E <= 1023:            # the scale is clamped to 2^1023 (columns below 2^-975)
            assert abs(Fraction(x) - Fraction(N) * Fraction(2) ** (E - 6 * s)) <= Fraction(2) ** (E - 6 * s - 1)
