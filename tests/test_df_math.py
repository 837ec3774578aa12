"""The double-float (pair-of-floats) arithmetic of the mixed form's per-point
coefficient stage: the device header is plain C++ besides its qualifiers, so it
is compiled here for the host (FP32 with exactly rounded FMA, as on the GPU)
and its exp, log, sin, cos, square root, reciprocal and double -> double-float
conversion are checked against 60-digit references over the ranges the stage
uses. The device build of the same code is checked by the GPU parity tests."""
import math
import os
import random
import shutil
import subprocess

import pytest

mp = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_24949_gb300", "csrc")

DRIVER = r"""
#include <stdio.h>
#include <stdlib.h>
#include "gwns_df.cuh"
using namespace gwns;
static dfl rd() { double v; if (scanf("%lf", &v) != 1) exit(1); return df_from_double(v); }
int main() {
    char op[16];
    while (scanf("%15s", op) == 1) {
        dfl x = rd(), r = {0, 0}, r2 = {0, 0};
        switch (op[0]) {
            case 'e': r = df_exp(x); break;
            case 'l': r = df_log(x); break;
            case 's': df_sincos(x, r, r2); break;
            case 'q': r = df_sqrt(x); break;
            case 'r': r = df_rcp(x); break;
            case 'c': r = x; break;
            case 'm': { dfl y = rd(); r = df_mul(x, y); r2 = df_add(x, y); break; }
        }
        printf("%a %a %a %a\n", (double)r.h, (double)r.l, (double)r2.h, (double)r2.l);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def df_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("dfmath")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    # no contraction, no fast math: every float operation rounds once, as the
    # device's __fadd_rn / __fmul_rn / __fmaf_rn do
    subprocess.run([cxx, "-O1", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-I", CSRC,
                    str(src), "-o", str(exe), "-lm"], check=True)
    return str(exe)


def run(exe, lines):
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    res = []
    for ln in out:
        if ln.strip():
            h, l, h2, l2 = (float.fromhex(t) for t in ln.split())
            res.append((mp.mpf(h) + mp.mpf(l), mp.mpf(h2) + mp.mpf(l2), h, l))
    return res


def test_conversion_and_normalisation(df_exe):
    rng = random.Random(1)
    xs = [0.0, 1.0, 0.5, 2.0 ** -60, -3.25, 1e-20] + [rng.random() for _ in range(200)] + \
         [rng.uniform(-1e6, 1e6) for _ in range(100)] + [2.0 ** -80]
    res = run(df_exe, [f"c {x!r}" for x in xs])
    for x, (v, _, h, l) in zip(xs, res):
        if abs(x) < 2.0 ** -74:
            assert v == 0
            continue
        assert abs(v - mp.mpf(x)) <= abs(mp.mpf(x)) * mp.mpf(2) ** -47, x
        # normalised: |l| <= ulp(h) / 2, ulp of a float h = 2^(exponent - 23)
        assert abs(l) <= 2.0 ** (math.frexp(h)[1] - 1 - 23) / 2, x


def test_exp_relative_error(df_exe):
    rng = random.Random(2)
    xs = [0.0, 1e-9, -1e-9, 0.0054, -0.0054, 1.0, -1.0, -33.8, 10.0, -60.0, 40.0]
    xs += [rng.uniform(-60.0, 10.0) for _ in range(3000)]
    res = run(df_exe, [f"e {x!r}" for x in xs])
    worst = 0.0
    with mp.workdps(60):
        for x, (v, *_) in zip(xs, res):
            # the double argument reaches the function as a double-float within
            # 2^-47 |x| of it, which moves e^x by that much relative
            ref = mp.exp(mp.mpf(x))
            worst = max(worst, float(abs(v / ref - 1)) / (1.0 + abs(x) / 8.0))
    assert worst < 2.0 ** -44, worst


def test_log_absolute_error(df_exe):
    rng = random.Random(3)
    xs = [1.0, 2.0, 0.5, 1.0 + 2 ** -20, 1.0 - 2 ** -20, 0.25, 0.16, 5.4e-6, 2e-4, 100.0, 2000.0, 8e9, 1e3]
    xs += [math.exp(rng.uniform(math.log(1e-7), math.log(1e11))) for _ in range(3000)]
    xs += [rng.uniform(0.9, 1.1) for _ in range(500)]
    res = run(df_exe, [f"l {x!r}" for x in xs])
    worst = 0.0
    with mp.workdps(60):
        for x, (v, *_) in zip(xs, res):
            ref = mp.log(mp.mpf(x))
            worst = max(worst, float(abs(v - ref) / max(1, abs(ref))))
    assert worst < 2.0 ** -45, worst


def test_sincos_absolute_error(df_exe):
    rng = random.Random(4)
    xs = [0.0, math.pi / 4, math.pi / 2, math.pi, 1.5 * math.pi, 2 * math.pi, 1e-8, 3 * math.pi / 4,
          -1.0, -math.pi / 2]
    xs += [rng.uniform(0.0, 2 * math.pi) for _ in range(3000)]
    xs += [rng.uniform(-100.0, 100.0) for _ in range(500)]
    res = run(df_exe, [f"s {x!r}" for x in xs])
    worst = 0.0
    with mp.workdps(60):
        for x, (s, c, *_) in zip(xs, res):
            # the double argument reaches the function as a double-float within
            # 2^-47 |x| of it, which moves sin and cos by as much
            err = max(float(abs(s - mp.sin(mp.mpf(x)))), float(abs(c - mp.cos(mp.mpf(x)))))
            worst = max(worst, err / (4e-15 + abs(x) * 2.0 ** -46))
    assert worst < 1.0, worst


def test_sqrt_rcp_mul_add(df_exe):
    rng = random.Random(5)
    xs = [rng.uniform(0.0, 1.0) for _ in range(500)] + [rng.uniform(1.0, 2.0) for _ in range(500)] + \
         [1.0, 0.25, 1e-12, 7.0]
    rs = run(df_exe, [f"q {x!r}" for x in xs])
    rr = run(df_exe, [f"r {x!r}" for x in xs if x > 0])
    with mp.workdps(60):
        for x, (v, *_) in zip(xs, rs):
            assert abs(v - mp.sqrt(mp.mpf(x))) <= mp.sqrt(mp.mpf(x)) * mp.mpf(2) ** -45, x
        for x, (v, *_) in zip([x for x in xs if x > 0], rr):
            assert abs(v * mp.mpf(x) - 1) <= mp.mpf(2) ** -45, x
    pairs = [(rng.uniform(-1e3, 1e3), rng.uniform(-1e3, 1e3)) for _ in range(1000)]
    rm = run(df_exe, [f"m {a!r} {b!r}" for a, b in pairs])
    with mp.workdps(60):
        for (a, b), (p, s, *_) in zip(pairs, rm):
            A, B = mp.mpf(a), mp.mpf(b)
            assert abs(p - A * B) <= abs(A * B) * mp.mpf(2) ** -45
            assert abs(s - (A + B)) <= (abs(A) + abs(B)) * mp.mpf(2) ** -46


def test_a_planted_slip_is_caught(df_exe, tmp_path):
    """The exp check fails when a Taylor coefficient of e^r is mistyped (1/24 -> 1/25)."""
    src = open(os.path.join(CSRC, "gwns_df.cuh")).read()
    bad = src.replace("1.0f / 24.0f), rh, 1.0f / 6.0f)", "1.0f / 25.0f), rh, 1.0f / 6.0f)")
    assert bad != src
    (tmp_path / "gwns_df.cuh").write_text(bad)
    shutil.copy(os.path.join(CSRC, "gwns_tables.cuh"), tmp_path / "gwns_tables.cuh")
    (tmp_path / "drv.cpp").write_text(DRIVER)
    cxx = shutil.which("g++") or shutil.which("c++")
    exe = tmp_path / "drv"
    subprocess.run([cxx, "-O1", "-std=c++17", "-ffp-contract=off", "-I", str(tmp_path), str(tmp_path / "drv.cpp"),
                    "-o", str(exe), "-lm"], check=True)
    res = run(str(exe), ["e 0.005", "e -0.0054"])
    worst = max(float(abs(v / mp.exp(mp.mpf(x)) - 1)) for x, (v, *_) in zip([0.005, -0.0054], res))
    assert worst > 2.0 ** -44
