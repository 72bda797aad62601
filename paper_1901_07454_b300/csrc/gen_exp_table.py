"""Writes arb_exp_table.h: 2^(j/64), j = 0..63, rounded to the nearest double, and the
Cody-Waite split of ln(2)/64 used by the table-driven exponential in arb_hh.cuh (Tang, "Table-
driven implementation of the exponential function in IEEE floating-point arithmetic", ACM TOMS
15(2), 1989). Values come from 60-digit arithmetic; the split keeps 32 significant bits in the
high part so that k * hi is exact for |k| < 2^20.

    python gen_exp_table.py > arb_exp_table.h
"""
import mpmath

mpmath.mp.dps = 60


def hexd(v):
    return float(v).hex()


def main():
    rows = [hexd(mpmath.power(2, mpmath.mpf(j) / 64)) for j in range(64)]
    l = mpmath.log(2) / 64
    hi = mpmath.mpf(float(l))
    # keep 32 significant bits of the high part
    m, e = mpmath.frexp(hi)
    hi = mpmath.ldexp(mpmath.floor(m * 2 ** 32), e - 32)
    lo = l - hi
    inv = 64 / mpmath.log(2)
    print("// Generated by gen_exp_table.py: 2^(j/64) for j = 0..63 and ln(2)/64 = kExpLn2Hi + kExpLn2Lo.")
    print("#pragma once")
    print("namespace arbk {")
    print("__device__ const double kExpTable[64] = {")
    for i in range(0, 64, 4):
        print("    " + ", ".join(rows[i:i + 4]) + ",")
    print("};")
    print("constexpr double kExpInvLn2x64 = %s;   // 64 / ln(2)" % hexd(inv))
    print("constexpr double kExpLn2Hi = %s;" % hexd(hi))
    print("constexpr double kExpLn2Lo = %s;" % hexd(lo))
    print("}  // namespace arbk")


if __name__ == "__main__":
    main()
