"""The double-double arithmetic of the refinement residual (dd.cuh),
compiled for the host and checked in exact rational arithmetic: the
error-free transformations are exact, and sums and products of
double-double numbers are within a few units of 2^-106 of the exact result,
also under cancellation (Knuth; Dekker; Joldes, Muller & Popescu, ACM TOMS
44, 2017, for the bounds)."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("dd") / "dd_host_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe,
                    os.path.join(HERE, "dd_host_check.cpp")], check=True)
    return exe


def _run(exe, rows):
    text = "".join(f"{op} {a.hex()} {b.hex()} {c.hex()} {d.hex()}\n" for op, a, b, c, d in rows)
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
    return [tuple(float.fromhex(t) for t in line.split()) for line in out.splitlines()]


def _dd(g, n, lo_exp=-30, hi_exp=30):
    hi = g.uniform(1, 2, n) * 2.0 ** g.integers(lo_exp, hi_exp, n) * g.choice([-1, 1], n)
    lo = hi * g.uniform(-1, 1, n) * 2.0 ** -54          # |lo| < ulp(hi) / 2
    return hi, lo


def _f(*xs):
    return sum((Fraction(float(x)) for x in xs), Fraction(0))


def test_error_free_transformations_are_exact(harness):
    g = np.random.default_rng(71)
    a, _ = _dd(g, 400)
    b, _ = _dd(g, 400)
    rows = [("S", x, 0.0, y, 0.0) for x, y in zip(a, b)]
    rows += [("P", x, 0.0, y, 0.0) for x, y in zip(a, b)]
    res = _run(harness, rows)
    for (op, x, _, y, _), (hi, lo) in zip(rows, res):
        exact = _f(x) + _f(y) if op == "S" else _f(x) * _f(y)
        assert _f(hi, lo) == exact, (op, x, y)
        assert hi == (x + y if op == "S" else x * y)   # the leading part is the FP64 result


def test_double_double_sum_and_product_bounds(harness):
    g = np.random.default_rng(72)
    ah, al = _dd(g, 500)
    bh, bl = _dd(g, 500)
    # cancellation: b close to -a, so that the sum is decided by the low parts
    ch, cl = ah.copy(), al.copy()
    dh, dl = -ah, -al + al * g.uniform(-1, 1, al.size) * 2.0 ** -3
    # deeper cancellation: the high parts cancel to one ulp, the first low
    # part nearly cancels that ulp, and the second carries a tail 2^-67 below
    # the result, which a sum of the low parts without its error term drops
    sig = 2.0 ** g.integers(-30, 30, 200).astype(float)
    eh, fh = sig, -sig * (1 - 2.0 ** -52)
    el = -sig * 2.0 ** -53 * (1 - 2.0 ** -40 * g.integers(1, 2 ** 10, 200))
    fl = sig * 2.0 ** -120 * g.uniform(1, 2, 200)
    rows = [("A", *v) for v in zip(ah, al, bh, bl)] + [("A", *v) for v in zip(ch, cl, dh, dl)]
    rows += [("A", *v) for v in zip(eh, el, fh, fl)]
    rows += [("M", *v) for v in zip(ah, al, bh, bl)]
    res = _run(harness, rows)
    for (op, a1, a2, b1, b2), (hi, lo) in zip(rows, res):
        a, b = _f(a1, a2), _f(b1, b2)
        exact = a + b if op == "A" else a * b
        got = _f(hi, lo)
        bound = Fraction(1, 2 ** (103 if op == "A" else 101)) * abs(exact)
        assert abs(got - exact) <= bound, (op, float((got - exact) / exact))
        assert abs(lo) <= abs(hi) * 2.0 ** -52    # normalised pair
