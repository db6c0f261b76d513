"""Write ln_table.cuh: the breakpoint table of the walkers' FP32 logarithm.

Row j = 0..64 of the table belongs to the breakpoint c_j = 1 + j/64 of the
mantissa M in [1, 2):
    inv_j = 1/c_j rounded to FP32,
    L_j   = -ln(inv_j)      rounded to FP32   (j <= 26),
    L_j   = -ln(2 inv_j)    rounded to FP32   (j >= 27: the row takes one factor
                                               2 of x into the exponent).
The logarithms are taken in FP64 and checked against 50-digit decimal
logarithms, so that no row sits on an FP32 rounding tie.

Run: python gen_ln_table.py  (rewrites ln_table.cuh beside it).
"""
import math
import os
import struct
from decimal import Decimal, getcontext

ROWS = 65
BINADE_SPLIT = 27


def f32(x: float) -> float:
    return struct.unpack("<f", struct.pack("<f", x))[0]


def bits(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def table():
    getcontext().prec = 50
    out = []
    for j in range(ROWS):
        inv = f32(1.0 / (1.0 + j / 64.0))
        a = 2.0 * inv if j >= BINADE_SPLIT else inv
        lj = f32(0.0 - math.log(a))
        assert f32(float(-Decimal(a).ln())) == lj or (lj == 0.0), j
        out.append((inv, lj))
    return out


def main():
    rows = table()
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "// Breakpoint table of the walkers' FP32 logarithm (ln_f32 in mcx_internal.cuh).",
        "// Written by gen_ln_table.py; row j = {1/c_j, L_j} for c_j = 1 + j/64 as FP32 bit",
        "// patterns: L_j = -ln(1/c_j as rounded) for j <= 26 and -ln(2/c_j as rounded) for",
        "// j >= 27.",
        "#pragma once",
        "",
        "#include <stdint.h>",
        "",
        "namespace mcx {",
        "",
        f"constexpr int LN_TABLE_ROWS = {ROWS};",
        f"constexpr int LN_TABLE_BINADE_SPLIT = {BINADE_SPLIT};",
        "",
        "static __device__ const uint2 c_ln_table[LN_TABLE_ROWS] = {",
    ]
    for j, (inv, lj) in enumerate(rows):
        lines.append(f"    {{0x{bits(inv):08x}u, 0x{bits(lj):08x}u}},  // j = {j:2d}: 1/c = {inv:.9g}, L = {lj:.9g}")
    lines += ["};", "", "}  // namespace mcx", ""]
    with open(os.path.join(here, "ln_table.cuh"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
