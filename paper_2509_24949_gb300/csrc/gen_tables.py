"""Write gwns_tables.cuh: the tables of the table-driven FP64 exp and log used
by the per-point coefficient stage (Tang, ACM TOMS 15 (1989) 144 and 16 (1990)
378: reduce the argument against a table point, then a short polynomial).

exp: T[j] = 2^(j/64), j = 0..63, as a double (hi) and the rounding remainder (lo).
log: for the mantissa interval j = 0..127 of [1, 2) (top 7 fraction bits),
inv_c[j] = the double nearest 1/(1 + (j + 1/2)/128), and nlninv[j] = -ln(inv_c[j])
as hi + lo, so that ln m = ln(m inv_c) - ln(inv_c) holds exactly for the stored
inv_c. Values are computed with 60-digit arithmetic (mpmath) and rounded.

    python paper_2509_24949_gb300/csrc/gen_tables.py
"""
import os

import mpmath as mp

mp.mp.dps = 60
HERE = os.path.dirname(os.path.abspath(__file__))


def split(x):
    hi = float(x)
    lo = float(x - mp.mpf(hi))
    return hi, lo


def hexd(v: float) -> str:
    return float.hex(v)


def main():
    lines = ["// gwns_tables.cuh -- generated by gen_tables.py (do not edit): tables of the",
             "// table-driven FP64 exp and log of the per-point coefficient stage.",
             "#pragma once", "", "namespace gwns {", ""]
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

    def arr(name, vals):
        out = [f"__device__ const double {name}[{len(vals)}] = {{"]
        for i in range(0, len(vals), 4):
            out.append("    " + ", ".join(vals[i:i + 4]) + ",")
        out.append("};")
        return out

    lines += arr("EXP_T_HI", exp_hi) + arr("EXP_T_LO", exp_lo)
    lines += arr("LOG_INV_C", inv) + arr("LOG_NLN_HI", nl_hi) + arr("LOG_NLN_LO", nl_lo)
    lines += ["", "}  // namespace gwns", ""]
    with open(os.path.join(HERE, "gwns_tables.cuh"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
