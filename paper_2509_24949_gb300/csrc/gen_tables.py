"""Write gwns_tables.cuh: the tables of the table-driven exp and log used by
the per-point coefficient stage (Tang, ACM TOMS 15 (1989) 144 and 16 (1990)
378: reduce the argument against a table point, then a short polynomial), in
FP64 and in double-float (pairs of floats).

exp: T[j] = 2^(j/64), j = 0..63, as a double (hi) and the rounding remainder (lo);
and as a double-float (the float nearest, then the float nearest the remainder).
log: for the mantissa interval j = 0..127 of [1, 2) (top 7 fraction bits),
inv_c[j] = the double nearest 1/(1 + (j + 1/2)/128), and nlninv[j] = -ln(inv_c[j])
as hi + lo, so that ln m = ln(m inv_c) - ln(inv_c) holds exactly for the stored
inv_c; and the same with inv_c the float nearest and -ln(inv_c) as a
double-float. Values are computed with 60-digit arithmetic (mpmath) and rounded.

    python paper_2509_24949_gb300/csrc/gen_tables.py
"""
import os
import struct

import mpmath as mp
import numpy as np

mp.mp.dps = 60
HERE = os.path.dirname(os.path.abspath(__file__))


def split(x):
    hi = float(x)
    lo = float(x - mp.mpf(hi))
    return hi, lo


def hexd(v: float) -> str:
    return float.hex(v)


def f32(x) -> float:
    """x rounded to the nearest float (binary32), returned as a Python float."""
    return struct.unpack("<f", struct.pack("<f", float(x)))[0]


def split_f(x):
    """x as a double-float: the float nearest x, then the float nearest the rest."""
    hi = f32(mp.mpf(x))
    # rounding x to double first, then to float, could round twice; pick the
    # nearest float of the exact value by checking the neighbours
    cands = [hi, float(np.nextafter(np.float32(hi), np.float32(np.inf))),
             float(np.nextafter(np.float32(hi), np.float32(-np.inf)))]
    hi = min(cands, key=lambda c: abs(mp.mpf(c) - x))
    lo = f32(x - mp.mpf(hi))
    return hi, lo


def hexf(v: float) -> str:
    return float.hex(v) + "f"


def main():
    lines = ["// gwns_tables.cuh -- generated by gen_tables.py (do not edit): tables of the",
             "// table-driven exp and log of the per-point coefficient stage, in FP64 and",
             "// in double-float.",
             "#pragma once", "",
             "#ifndef GWNS_TABLE",
             "#if defined(__CUDACC__)",
             "#define GWNS_TABLE __device__ const",
             "#else",
             "#define GWNS_TABLE static const",
             "#endif",
             "#endif", "", "namespace gwns {", ""]
    exp_hi, exp_lo = [], []
    for j in range(64):
        hi, lo = split(mp.power(2, mp.mpf(j) / 64))
        exp_hi.append(hexd(hi))
        exp_lo.append(hexd(lo))
    inv, nl_hi, nl_lo = [], [], []
    for j in range(128):
        c = 1 + (mp.mpf(j) + mp.mpf(1) / 2) / 128
        ic = float(1 / c)
        hi, lo = split(-mp.log(mp.mpf(ic)))
        inv.append(hexd(ic))
        nl_hi.append(hexd(hi))
        nl_lo.append(hexd(lo))

    exf_hi, exf_lo = [], []
    for j in range(64):
        hi, lo = split_f(mp.power(2, mp.mpf(j) / 64))
        exf_hi.append(hexf(hi))
        exf_lo.append(hexf(lo))
    invf, nlf_hi, nlf_lo = [], [], []
    for j in range(128):
        c = 1 + (mp.mpf(j) + mp.mpf(1) / 2) / 128
        icf = split_f(1 / c)[0]
        hi, lo = split_f(-mp.log(mp.mpf(icf)))
        invf.append(hexf(icf))
        nlf_hi.append(hexf(hi))
        nlf_lo.append(hexf(lo))

    def arr(name, vals, ty="double"):
        out = [f"GWNS_TABLE {ty} {name}[{len(vals)}] = {{"]
        for i in range(0, len(vals), 4):
            out.append("    " + ", ".join(vals[i:i + 4]) + ",")
        out.append("};")
        return out

    lines += arr("EXP_T_HI", exp_hi) + arr("EXP_T_LO", exp_lo)
    lines += arr("LOG_INV_C", inv) + arr("LOG_NLN_HI", nl_hi) + arr("LOG_NLN_LO", nl_lo)
    lines += arr("EXPF_T_HI", exf_hi, "float") + arr("EXPF_T_LO", exf_lo, "float")
    lines += arr("LOGF_INV_C", invf, "float") + arr("LOGF_NLN_HI", nlf_hi, "float")
    lines += arr("LOGF_NLN_LO", nlf_lo, "float")
    lines += ["", "}  // namespace gwns", ""]
    with open(os.path.join(HERE, "gwns_tables.cuh"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
