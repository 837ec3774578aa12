"""The table-driven FP64 exp and log of the per-point coefficient stage (Tang's
method): the committed table header is what its generator writes, and the
algorithm the device code follows, run here in Python with an exactly rounded
fused multiply-add, is within 1 ulp of 60-digit references over the ranges the
coefficient stage uses (exp of [-60, 10]; log of [1e-7, 1e11]). The device code
itself is checked by the GPU parity tests (FP64 log L within 1e-9)."""
import importlib.util
import math
import os
import random
import re
import struct

import pytest

mp = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_24949_gb300", "csrc")
HEADER = os.path.join(CSRC, "gwns_tables.cuh")


def _tables():
    src = open(HEADER).read()

    def tab(name):
        body = re.search(name + r"\[\d+\] = \{(.*?)\};", src, re.S).group(1)
        return [float.fromhex(t.strip()) for t in body.replace("\n", " ").split(",") if t.strip()]

    return {n: tab(n) for n in ("EXP_T_HI", "EXP_T_LO", "LOG_INV_C", "LOG_NLN_HI", "LOG_NLN_LO")}


def test_header_is_the_generator_output(tmp_path, monkeypatch):
    spec = importlib.util.spec_from_file_location("gen_tables", os.path.join(CSRC, "gen_tables.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    monkeypatch.setattr(gen, "HERE", str(tmp_path))
    gen.main()
    assert (tmp_path / "gwns_tables.cuh").read_text() == open(HEADER).read()


def _fma(a, b, c):
    with mp.workdps(80):
        return float(mp.mpf(a) * mp.mpf(b) + mp.mpf(c))


def _head(x: float) -> float:
    """x with the low 20 mantissa bits cleared (the device's 33-bit heads)."""
    b = struct.unpack("<Q", struct.pack("<d", x))[0] & ~((1 << 20) - 1)
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def test_exp_and_log_within_one_ulp():
    t = _tables()
    mp.mp.dps = 40
    l64 = mp.log(2) / 64
    # the device's literal constants are the heads and tails of these values
    assert _head(float(l64)) == float.fromhex("0x1.62e42fef00000p-7")
    assert float(l64 - mp.mpf(_head(float(l64)))) == float.fromhex("0x1.473de6af278edp-40")
    assert _head(float(mp.log(2))) == float.fromhex("0x1.62e42fef00000p-1")
    assert float(mp.log(2) - mp.mpf(_head(float(mp.log(2))))) == float.fromhex("0x1.473de6af278edp-34")
    assert float(64 / mp.log(2)) == float.fromhex("0x1.71547652b82fep+6")
    shift = 6755399441055744.0
    inv_l, lh, ll = 64 / math.log(2), _head(float(l64)), float(l64 - mp.mpf(_head(float(l64))))
    ln2h, ln2l = _head(float(mp.log(2))), float(mp.log(2) - mp.mpf(_head(float(mp.log(2)))))

    def exp_t(x):
        kk = _fma(x, float.fromhex("0x1.71547652b82fep+6"), shift)
        k = kk - shift
        ki = int(k)
        r = _fma(-k, lh, x)
        r = _fma(-k, ll, r)
        j, m = ki & 63, ki >> 6
        q = _fma(r, 1 / 120, 1 / 24)
        q = _fma(q, r, 1 / 6)
        q = _fma(q, r, 0.5)
        p = _fma(r * r, q, r)
        res = t["EXP_T_HI"][j] + _fma(t["EXP_T_HI"][j], p, t["EXP_T_LO"][j])
        return math.ldexp(res, m)

    def log_t(x):
        mant, e = math.frexp(x)
        m, e = mant * 2, e - 1
        j = int((m - 1) * 128)
        r = _fma(m, t["LOG_INV_C"][j], -1.0)
        q = _fma(r, -1 / 6, 0.2)
        q = _fma(q, r, -0.25)
        q = _fma(q, r, 1 / 3)
        q = _fma(q, r, -0.5)
        p = _fma(r * r, q, r)
        h = _fma(float(e), ln2h, t["LOG_NLN_HI"][j])
        lo = _fma(float(e), ln2l, t["LOG_NLN_LO"][j]) + p
        return h + lo

    assert inv_l == pytest.approx(float.fromhex("0x1.71547652b82fep+6"), rel=1e-16)
    rng = random.Random(7)
    ulp = 2.0 ** -52
    for _ in range(3000):
        x = rng.uniform(-60.0, 10.0)
        ref = mp.exp(x)
        assert abs(float((mp.mpf(exp_t(x)) - ref) / ref)) < ulp
        y = 10 ** rng.uniform(-7.0, 11.0)
        ref = mp.log(y)
        assert abs(float(mp.mpf(log_t(y)) - ref)) < ulp * max(1.0, abs(float(ref)))
    # table points and interval ends
    for j in range(128):
        for m in (1 + j / 128, 1 + (j + 1) / 128 - 2 ** -40):
            assert abs(float(mp.mpf(log_t(m)) - mp.log(m))) < ulp
