"""Build-time generator of the sin/cos constant tables used by the CUDA kernels.

Everything is computed with exact Python integers at 320 fractional bits and rounded once:
  * pi from Machin's formula pi = 16 atan(1/5) - 4 atan(1/239), atan(1/x) by its alternating series;
  * cos and sin of 2 pi c / 2^8 and 2 pi c / 2^16 (c = 0..255) by their Taylor series;
  * reciprocal factorials 1/n!.
Outputs (written to gen/tables.h):
  * fixed-point tables: signed two's-complement Q2.126 in four little-endian 32-bit limbs, cos then sin;
  * double-double tables: (hi, lo) pairs with hi = nearest double, lo = nearest double to the rest.
The CUDA library's sincos of a phase in turns is t = c1/2^8 + c2/2^16 + r with |r| < 2^-16:
e^{2 pi i t} = A[c1] * B[c2] * e^{2 pi i r}, the last factor from a short Taylor series.
"""
from __future__ import annotations

import os
import sys
from fractions import Fraction

P = 320
ONE = 1 << P


def atan_inv(x: int) -> int:
    """atan(1/x) * 2^P by the alternating series (x >= 2)."""
    total, term, k, x2 = 0, ONE // x, 0, x * x
    while term:
        total += term // (2 * k + 1) if k % 2 == 0 else -(term // (2 * k + 1))
        term //= x2
        k += 1
    return total


PI = 16 * atan_inv(5) - 4 * atan_inv(239)


def cos_sin(theta: int) -> tuple[int, int]:
    """cos and sin of theta (all values scaled by 2^P) by Taylor series."""
    c, s = 0, 0
    term, n = ONE, 0       # theta^n / n!
    while term:
        r = n % 4
        if r == 0:
            c += term
        elif r == 1:
            s += term
        elif r == 2:
            c -= term
        else:
            s -= term
        n += 1
        term = term * theta // ONE // n
    return c, s


def q126(x: int) -> int:
    """Round x / 2^P to signed Q2.126 (range [-2, 2), resolution 2^-126)."""
    return (x + (1 << (P - 127))) >> (P - 126)


def limbs(v: int, n: int = 4) -> list[int]:
    v &= (1 << (32 * n)) - 1
    return [(v >> (32 * i)) & 0xFFFFFFFF for i in range(n)]


def to_dd(x: int) -> tuple[float, float]:
    f = Fraction(x, ONE)
    hi = float(f)
    lo = float(f - Fraction(hi))
    return hi, lo


def main(out_path: str) -> None:
    rows = []
    rows.append("// Generated by gen_tables.py (exact integer arithmetic); do not edit.")
    rows.append("#pragma once")
    rows.append("#include <stdint.h>")
    rows.append("#ifndef SSH_TABLE_QUAL")
    rows.append("#define SSH_TABLE_QUAL static")
    rows.append("#endif")
    fx_a, fx_b, dd_a, dd_b = [], [], [], []
    for c in range(256):
        ca, sa = cos_sin(2 * PI * c // 256)
        cb, sb = cos_sin(2 * PI * c // 65536)
        fx_a.append(limbs(q126(ca)) + limbs(q126(sa)))
        fx_b.append(limbs(q126(cb)) + limbs(q126(sb)))
        dd_a.append(to_dd(ca) + to_dd(sa))
        dd_b.append(to_dd(cb) + to_dd(sb))

    def emit_u32(name, tab):
        rows.append(f"SSH_TABLE_QUAL const uint32_t {name}[256][8] = {{")
        for r in tab:
            rows.append("  {" + ", ".join(f"0x{w:08x}u" for w in r) + "},")
        rows.append("};")

    def emit_dd(name, tab):
        rows.append(f"SSH_TABLE_QUAL const double {name}[256][4] = {{")
        for r in tab:
            rows.append("  {" + ", ".join(f"{v!r}" for v in r) + "},")
        rows.append("};")

    emit_u32("SSH_FX_TAB_A", fx_a)
    emit_u32("SSH_FX_TAB_B", fx_b)
    emit_dd("SSH_DD_TAB_A", dd_a)
    emit_dd("SSH_DD_TAB_B", dd_b)
    # pi * 2^125: for a turn remainder r (integer, value r / 2^128) the Q2.126 angle 2 pi r / 2^128 is
    # (r * pi 2^125) >> 126
    pi_q3_125 = (PI + (1 << (P - 126))) >> (P - 125)
    rows.append("SSH_TABLE_QUAL const uint32_t SSH_FX_PI_Q3_125[4] = {" + ", ".join(f"0x{w:08x}u" for w in limbs(pi_q3_125)) + "};")
    two_pi = to_dd(2 * PI)
    rows.append(f"SSH_TABLE_QUAL const double SSH_DD_2PI[2] = {{{two_pi[0]!r}, {two_pi[1]!r}}};")
    rows.append(f"#define SSH_DD_2PI_HI {two_pi[0]!r}")
    rows.append(f"#define SSH_DD_2PI_LO {two_pi[1]!r}")
    fact = 1
    inv_fx, inv_dd = [], []
    for n in range(0, 12):
        fact = fact * n if n > 0 else 1
        inv = ONE // fact
        inv_fx.append(limbs(q126(inv)))
        inv_dd.append(to_dd(inv))
    rows.append("SSH_TABLE_QUAL const uint32_t SSH_FX_INV_FACT[12][4] = {")
    for r in inv_fx:
        rows.append("  {" + ", ".join(f"0x{w:08x}u" for w in r) + "},")
    rows.append("};")
    rows.append("SSH_TABLE_QUAL const double SSH_DD_INV_FACT[12][2] = {")
    for r in inv_dd:
        rows.append(f"  {{{r[0]!r}, {r[1]!r}}},")
    rows.append("};")
    os.makedirs(os.path.dirname(out_path), exist_ok=True)
    tmp = out_path + ".tmp"
    with open(tmp, "w") as f:
        f.write("\n".join(rows) + "\n")
    os.replace(tmp, out_path)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(__file__), "gen", "tables.h"))
