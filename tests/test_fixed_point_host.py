"""The exact fixed-point accumulator behind the packed S-apply's projection sums (host build).

The packed S-apply forms the constraint sums C^T q_raw of the projection (Eq. 9) as sums of its
float32 products in a 128-bit fixed-point integer (units of 2^-88), so that the charges stay
neutral to float64 rounding although the sums never touch a float64 adder.  The header compiles
for the host too; here it is built with the host compiler and checked against exact rational sums:
every float enters exactly up to its part below 2^-88, the sum is independent of the order and of
the split into partial accumulators, cancellation loses nothing, and the documented exclusions
(zero, subnormal and non-finite values, magnitudes of 2^39 and more) add nothing.
"""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
UNIT = Fraction(1, 2 ** 88)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("fx") / "fixed_point_host")
    subprocess.run([cxx, "-std=c++17", "-O2", "-o", exe, os.path.join(HERE, "fixed_point_host.cpp")], check=True)

    def run(x, k=None):
        x = np.asarray(x, np.float32)
        k = len(x) if k is None else k
        inp = f"{k} {len(x)}\n" + "\n".join(f"{v:08x}" for v in x.view(np.uint32)) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
        return float(out[0]), (int(out[1], 16), int(out[2], 16))
    return run


def _exact(x):
    """Exact sum of the floats' values truncated toward zero to multiples of 2^-88."""
    tot = Fraction(0)
    for v in np.asarray(x, np.float32):
        f = Fraction(float(v))
        q = abs(f) // UNIT
        tot += (q if f >= 0 else -q) * UNIT
    return tot


def _state(total):
    """The 128-bit two's-complement state of an exact multiple of 2^-88."""
    n = int(total / UNIT) % (1 << 128)
    return n >> 64, n & ((1 << 64) - 1)


def test_sums_are_exact_across_magnitudes(harness):
    rng = np.random.default_rng(11)
    x = (rng.standard_normal(3000) * np.exp(rng.uniform(-40, 20, 3000))).astype(np.float32)
    x = x[np.abs(x) < 2.0 ** 39]
    v, st = harness(x)
    ex = _exact(x)
    assert st == _state(ex)
    assert abs(Fraction(v) - ex) <= abs(ex) * Fraction(2, 2 ** 53)


def test_order_and_split_do_not_matter(harness):
    rng = np.random.default_rng(12)
    x = (rng.standard_normal(2000) * 10.0 ** rng.uniform(-6, 2, 2000)).astype(np.float32)
    v0, s0 = harness(x)
    for k in (0, 1, 777, len(x)):
        assert harness(x, k) == (v0, s0)
    assert harness(x[::-1]) == (v0, s0)
    assert harness(rng.permutation(x), 1000) == (v0, s0)


def test_cancellation_leaves_the_exact_residual(harness):
    # tile products near 1 that cancel to a charge near 1e-2, as in the packed S-apply, and a pair
    # of values far apart in magnitude
    rng = np.random.default_rng(13)
    big = rng.standard_normal(5000).astype(np.float32)
    resid = np.float32([1e-2, -3e-9, 7.25e-20])
    x = np.concatenate([big, -big[::-1], resid, np.float32([2.0 ** 30, 1e-25, -2.0 ** 30])])
    v, st = harness(x)
    ex = _exact(x)
    assert st == _state(ex)
    assert abs(Fraction(v) - ex) <= abs(ex) * Fraction(2, 2 ** 53)


def test_excluded_values_add_nothing(harness):
    base = np.float32([0.5, -0.25, 3.0])
    v0, s0 = harness(base)
    excluded = np.float32([0.0, -0.0, 1e-40, np.inf, -np.inf, np.nan, 2.0 ** 39, -(2.0 ** 40)])
    assert harness(np.concatenate([base, excluded])) == (v0, s0)
    # just inside the range, and below the unit: kept exactly, and dropped
    v, st = harness(np.float32([2.0 ** 38, 2.0 ** -88, 2.0 ** -89]))
    assert st == _state(Fraction(2 ** 38) + UNIT)
    assert v == 2.0 ** 38 + 2.0 ** -88
    assert harness(np.float32([-2.0 ** -87]))[1] == _state(-2 * UNIT)
