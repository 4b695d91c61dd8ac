"""Generate exp2_table.h: correctly rounded 2^(j/128), j = 0..127, as hex literals.

Used by the table-driven exponential of the kernels (Tang, "Table-driven
implementation of the exponential function in IEEE floating-point arithmetic",
ACM TOMS 15(2), 1989).  The values are computed with 50-digit decimal
arithmetic and rounded once to binary64.

    python paper_1712_00953_gb300/csrc/gen_exp_table.py > paper_1712_00953_gb300/csrc/exp2_table.h
"""

from decimal import Decimal, getcontext

N = 128


def main():
    getcontext().prec = 60
    ln2 = Decimal(2).ln()
    lines = ["// Generated by gen_exp_table.py: RK_EXP2_TABLE_VALUES[j] = 2^(j/128) rounded to binary64.",
             "#pragma once", f"#define RK_EXP2_TABLE_N {N}", "#define RK_EXP2_TABLE_VALUES \\"]
    for j in range(N):
        v = (ln2 * j / N).exp()
        f = float(v)  # Decimal -> nearest binary64
        sep = ", \\" if j + 1 < N else ""
        lines.append(f"    {f.hex()}{sep}")
    # ln2 / N split into a head with trailing zero bits and a tail
    ln2n = ln2 / N
    head = float(ln2n)
    # clear the low 32 bits of the head so that k * head is exact for |k| < 2^20
    import struct
    bits = struct.unpack("<Q", struct.pack("<d", head))[0] & ~((1 << 32) - 1)
    head = struct.unpack("<d", struct.pack("<Q", bits))[0]
    tail = float(ln2n - Decimal(head))
    lines.append(f"constexpr double RK_LN2_OVER_N_HI = {head.hex()};")
    lines.append(f"constexpr double RK_LN2_OVER_N_LO = {tail.hex()};")
    lines.append(f"constexpr double RK_N_OVER_LN2 = {float(Decimal(N) / ln2).hex()};")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
