"""The dual-number arithmetic behind pf_tangent (csrc/dual.cuh), on the host:
each derivative against its closed form, and a composite against central
differences of plain double arithmetic."""
import math
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))

CLOSED = {
    "sqrt": (lambda x: math.sqrt(x), lambda x: 0.5 / math.sqrt(x)),
    "rsqrt": (lambda x: 1 / math.sqrt(x), lambda x: -0.5 * x ** -1.5),
    "exp": (math.exp, math.exp),
    "expm1": (math.expm1, math.exp),
    "exp2": (lambda x: 2.0 ** x, lambda x: math.log(2.0) * 2.0 ** x),
    "log2": (math.log2, lambda x: 1.0 / (x * math.log(2.0))),
    "neg": (lambda x: abs(-x), lambda x: 1.0),
    "quot": (lambda x: (x * x + 1) / (2 - 0.25 * x),
             lambda x: (2 * x * (2 - 0.25 * x) + 0.25 * (x * x + 1)) / (2 - 0.25 * x) ** 2),
}


def chain(x):
    s = x * math.exp(-x) / (1 + x * x) + math.sqrt(x) * math.log2(1 + x)
    return s - math.expm1(-0.5 * x) / x


@pytest.fixture(scope="module")
def rows(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("dual") / "dual_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", os.path.join(HERE, "dual_check.cu"), "-o", exe], check=True,
                   capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    return [(r.split()[0], *map(float, r.split()[1:])) for r in out if r.strip()]


def test_elementary_derivatives(rows):
    n = 0
    for name, x, v, d in rows:
        if name in CLOSED:
            f, df = CLOSED[name]
            assert abs(v - f(x)) <= 1e-15 * max(1.0, abs(f(x))), (name, x)
            assert abs(d - df(x)) <= 1e-14 * max(1.0, abs(df(x))), (name, x, d, df(x))
            n += 1
    assert n == 3 * len(CLOSED)


def test_composite_against_central_differences(rows):
    for name, x, v, d in rows:
        if name != "chain":
            continue
        assert abs(v - chain(x)) <= 1e-14 * max(1.0, abs(v))
        h = 1e-5
        fd = (chain(x + h) - chain(x - h)) / (2 * h)
        assert abs(d - fd) <= 1e-8 * max(1.0, abs(d)), (x, d, fd)
