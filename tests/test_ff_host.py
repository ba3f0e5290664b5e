"""The float-float helpers that the mixed form's QR, R^{-*} solve and Cholesky run on
(csrc/ff.cuh), compiled for the host from the same source and checked against exact
rational arithmetic: TwoSum is exact, and sums, products, reciprocals, square roots, dot
products and the double <-> float-float conversions are accurate to the bounds the
kernels rely on (about 2^-48 relative; asserted at 2^-44 with room for the operation
count)."""
import os
import shutil
import subprocess
from fractions import Fraction as F

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
U = F(1, 2 ** 44)


@pytest.fixture(scope="module")
def ffh(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("ffh") / "ffh")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-w", "-I",
                    os.path.join(ROOT, "paper_0912_1135_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "ff_host_check.cpp"), "-o", exe], check=True)

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return [[float.fromhex(v) for v in ln.split()] for ln in out.stdout.splitlines()]
    return run


def f32(x):
    return float(np.float32(x))


def ff_values(rng, n, emin=-20, emax=20):
    """Normalised float-float pairs: hi a float, |lo| <= ulp(hi) / 2."""
    hi = [f32(s * m * 2.0 ** e) for s, m, e in zip(rng.choice([-1.0, 1.0], n), rng.uniform(1, 2, n),
                                                   rng.integers(emin, emax, n))]
    lo = [f32(h * u * 2.0 ** -24) for h, u in zip(hi, rng.uniform(-1, 1, n))]
    return list(zip(hi, lo))


def val(p):
    return F(p[0]) + F(p[1])


def test_two_sum_is_exact(ffh):
    rng = np.random.default_rng(1)
    a = [f32(v) for v in rng.standard_normal(400) * 2.0 ** rng.integers(-30, 30, 400)]
    b = [f32(v) for v in rng.standard_normal(400) * 2.0 ** rng.integers(-30, 30, 400)]
    a += [1.0, 3.0, f32(1 + 2 ** -23)]
    b += [-1.0, -f32(3.0000002), f32(2 ** -24)]
    res = ffh([f"two_sum {x.hex()} {y.hex()}" for x, y in zip(a, b)])
    for x, y, (s, e) in zip(a, b, res):
        assert F(s) + F(e) == F(x) + F(y)
        assert s == f32(x + y)                        # the high part is the rounded sum


def test_sum_product_reciprocal_square_root(ffh):
    rng = np.random.default_rng(2)
    xs, ys = ff_values(rng, 300), ff_values(rng, 300)
    lines = [f"add {x[0].hex()} {x[1].hex()} {y[0].hex()} {y[1].hex()}" for x, y in zip(xs, ys)]
    lines += [f"mul {x[0].hex()} {x[1].hex()} {y[0].hex()} {y[1].hex()}" for x, y in zip(xs, ys)]
    lines += [f"recip {x[0].hex()} {x[1].hex()}" for x in xs]
    pos = [(abs(x[0]), x[1] if x[0] > 0 else -x[1]) for x in xs]
    lines += [f"sqrt {x[0].hex()} {x[1].hex()}" for x in pos]
    res = ffh(lines)
    n = len(xs)
    for i, (x, y) in enumerate(zip(xs, ys)):
        X, Y = val(x), val(y)
        assert abs(val(res[i]) - (X + Y)) <= U * (abs(X) + abs(Y))
        assert abs(val(res[n + i]) - X * Y) <= U * abs(X * Y)
        assert abs(val(res[2 * n + i]) * X - 1) <= U
        P = val(pos[i])
        s = val(res[3 * n + i])
        assert s > 0 and abs(s * s - P) <= 2 * U * P
    for r in res:                                      # every result normalised
        assert r[1] == 0 or abs(r[1]) <= abs(r[0]) * 2.0 ** -23


def test_dot_product_accumulation(ffh):
    rng = np.random.default_rng(3)
    lines, cases = [], []
    for n in (1, 2, 16, 32, 33, 500):
        xs, ys = ff_values(rng, n, -4, 4), ff_values(rng, n, -4, 4)
        cases.append((xs, ys))
        lines.append(f"dot {n} " + " ".join(f"{x[0].hex()} {x[1].hex()} {y[0].hex()} {y[1].hex()}"
                                             for x, y in zip(xs, ys)))
    for (xs, ys), r in zip(cases, ffh(lines)):
        exact = sum(val(x) * val(y) for x, y in zip(xs, ys))
        scale = sum(abs(val(x) * val(y)) for x, y in zip(xs, ys))
        assert abs(val(r) - exact) <= len(xs) * U * scale


def test_double_round_trip(ffh):
    rng = np.random.default_rng(4)
    ds = list(rng.standard_normal(200) * 2.0 ** rng.integers(-100, 100, 200)) + [1.0, -3.0, 2.0 ** -120]
    res = ffh([f"split {float(d).hex()}" for d in ds])
    for d, (hi, lo, back) in zip(ds, res):
        assert hi == f32(d)                            # the high part is the float rounding
        assert F(hi) + F(lo) == F(back)                # ff_to_double sums the parts exactly here
        assert abs(F(back) - F(float(d))) <= F(1, 2 ** 47) * abs(F(float(d)))
