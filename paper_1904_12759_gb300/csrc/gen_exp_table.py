"""Write exp_table.cuh: the table and reduction constants of the FP64 exponential
of an FP32 argument used by the control-variate coefficients (exp_of_f32 in
expd.cuh, Tang's table-driven method: ACM TOMS 15(2), 1989).

    T_j = 2^(j/64) rounded to FP64, j = 0..63;
    L   = ln(2)/64 split as L1 + L2: L1 keeps the leading 36 significant bits of
          L (so that N * L1 is exact for |N| < 2^17), L2 = L - L1 rounded to FP64.
All values come from 50-digit decimal arithmetic (Python's decimal module) and
are rounded to FP64 once.

Run: python gen_exp_table.py  (rewrites exp_table.cuh beside it).
"""
import os
import struct
from decimal import Decimal, getcontext

ROWS = 64
L1_BITS = 36


def f64_bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def constants():
    getcontext().prec = 50
    ln2 = Decimal(2).ln()
    table = [float((Decimal(j) / ROWS * ln2).exp()) for j in range(ROWS)]
    L = ln2 / ROWS
    # L1: L truncated to L1_BITS significant bits (L lies in [2^-7, 2^-6))
    scale = Decimal(2) ** (L1_BITS + 6)
    L1 = Decimal(int(L * scale)) / scale
    L2 = float(L - L1)
    assert float(L1) == L1 and 2.0 ** -7 <= float(L1) < 2.0 ** -6
    return table, float(L1), L2


def main():
    table, L1, L2 = constants()
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "// Table and reduction constants of exp_of_f32 (expd.cuh).  Written by",
        "// gen_exp_table.py: T_j = 2^(j/64) as FP64 bit patterns; ln(2)/64 = L1 + L2",
        "// with L1 of 36 significant bits.",
        "#pragma once",
        "",
        "#include <stdint.h>",
        "",
        "namespace mcx {",
        "",
        f"constexpr int EXP_TABLE_ROWS = {ROWS};",
        f"constexpr double EXP_L1 = {L1!r};  // 0x{f64_bits(L1):016x}",
        f"constexpr double EXP_L2 = {L2!r};  // 0x{f64_bits(L2):016x}",
        "",
        "static __device__ const unsigned long long c_exp_table[EXP_TABLE_ROWS] = {",
    ]
    for j, x in enumerate(table):
        lines.append(f"    0x{f64_bits(x):016x}ull,  // 2^({j}/64) = {x!r}")
    lines += ["};", "", "}  // namespace mcx", ""]
    with open(os.path.join(here, "exp_table.cuh"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
