"""Generate exp2_table.h: the tables of the kernels' exponential and logarithm.

Exponential (Tang, "Table-driven implementation of the exponential function
in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989): correctly rounded
2^(j/256), j = 0..255, and ln2/256 split in two (256 intervals keep the
reduced argument within ln2/512, where a degree-4 polynomial of e^r - 1 is
accurate below an ulp).  Logarithm (Tang,
"Table-driven implementation of the logarithm function in IEEE
floating-point arithmetic", ACM TOMS 16(4), 1990): for the 128 intervals
[1 + j/128, 1 + (j+1)/128) of the significand, the reciprocal of the
interval's centre rounded to binary64 (inv_c) and -ln(inv_c) of that rounded
value, and ln2 split in two.  Values are computed with 60-digit decimal
arithmetic and rounded once to binary64.

    python paper_1712_00953_gb300/csrc/gen_exp_table.py > paper_1712_00953_gb300/csrc/exp2_table.h
"""

import struct
from decimal import Decimal, getcontext

N = 256  # exponential table
NL = 128  # logarithm tables


def main():
    getcontext().prec = 60
    ln2 = Decimal(2).ln()
    lines = ["// Generated by gen_exp_table.py: RK_EXP2_TABLE_VALUES[j] = 2^(j/256) rounded to binary64;",
             "// RK_LOG_INV_C_VALUES[j] = 1/(1 + (j + 1/2)/128) rounded, RK_LOG_LN_C_VALUES[j] = -ln of it.",
             "#pragma once", f"#define RK_EXP2_TABLE_N {N}", f"#define RK_LOG_TABLE_N {NL}",
             "#define RK_EXP2_TABLE_VALUES \\"]
    for j in range(N):
        v = (ln2 * j / N).exp()
        f = float(v)  # Decimal -> nearest binary64
        sep = ", \\" if j + 1 < N else ""
        lines.append(f"    {f.hex()}{sep}")
    # ln2 / N split into a head with trailing zero bits and a tail
    ln2n = ln2 / N
    head = float(ln2n)
    # clear the low 32 bits of the head so that k * head is exact for |k| < 2^20
    bits = struct.unpack("<Q", struct.pack("<d", head))[0] & ~((1 << 32) - 1)
    head = struct.unpack("<d", struct.pack("<Q", bits))[0]
    tail = float(ln2n - Decimal(head))
    lines.append(f"constexpr double RK_LN2_OVER_N_HI = {head.hex()};")
    lines.append(f"constexpr double RK_LN2_OVER_N_LO = {tail.hex()};")
    lines.append(f"constexpr double RK_N_OVER_LN2 = {float(Decimal(N) / ln2).hex()};")
    # logarithm: inv_c_j = 1 / (1 + (j + 1/2) / NL) rounded, ln_c_j = -ln(inv_c_j) of the rounded value
    inv_c = [float(1 / (1 + (Decimal(j) + Decimal(1) / 2) / NL)) for j in range(NL)]
    ln_c = [float(-Decimal(v).ln()) for v in inv_c]  # Decimal(v) is the binary64 value exactly
    lines.append(f"#define RK_LOG_INV_C_VALUES {', '.join(v.hex() for v in inv_c)}")
    lines.append(f"#define RK_LOG_LN_C_VALUES {', '.join(v.hex() for v in ln_c)}")
    bits = struct.unpack("<Q", struct.pack("<d", float(ln2)))[0] & ~((1 << 32) - 1)
    ln2_hi = struct.unpack("<d", struct.pack("<Q", bits))[0]
    lines.append(f"constexpr double RK_LN2_HI = {ln2_hi.hex()};")
    lines.append(f"constexpr double RK_LN2_LO = {float(ln2 - Decimal(ln2_hi)).hex()};")
    lines.append(f"constexpr double RK_INV_LN10 = {float(1 / Decimal(10).ln()).hex()};")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
