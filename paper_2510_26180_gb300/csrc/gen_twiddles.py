"""Writes twiddles.h: cos(2 pi t / 128) for t = 0..32 as exact double
literals (the first quadrant; the transforms get every other t by symmetry).

The values are computed in 40-digit decimal arithmetic (pi by Machin's
formula, cos by its Taylor series) and rounded once to the nearest double,
so each literal is the correctly rounded value.  Run from this directory:
    python gen_twiddles.py > twiddles.h
"""
from decimal import Decimal, getcontext

getcontext().prec = 40


def arctan_inv(n: int) -> Decimal:
    """arctan(1/n) by its Taylor series."""
    x = Decimal(1) / n
    x2 = x * x
    term, total, k = x, x, 1
    while True:
        term *= -x2
        add = term / (2 * k + 1)
        if abs(add) < Decimal(10) ** -45:
            return total
        total += add
        k += 1


def cos_dec(x: Decimal) -> Decimal:
    term, total, k = Decimal(1), Decimal(1), 0
    while True:
        term *= -x * x / ((2 * k + 1) * (2 * k + 2))
        if abs(term) < Decimal(10) ** -45:
            return total
        total += term
        k += 1


PI = 16 * arctan_inv(5) - 4 * arctan_inv(239)   # Machin's formula


def main() -> None:
    vals = []
    for t in range(33):
        v = 0.0 if t == 32 else float(cos_dec(2 * PI * t / 128))
        vals.append(repr(v))
    print("// Generated by gen_twiddles.py: cos(2 pi t / 128), t = 0..32, each the")
    print("// correctly rounded double.  Do not edit by hand.")
    print("#pragma once")
    print("")
    print("namespace klecgc {")
    print("")
    print("// A constexpr function (not an array) so that device code can use it and,")
    print("// called with a compile-time argument, it folds to the literal.")
    print("__host__ __device__ constexpr double twiddle_cos_q1(int t) {")
    print("    constexpr double v[33] = {")
    for i in range(0, 33, 3):
        print("        " + ", ".join(vals[i:i + 3]) + ",")
    print("    };")
    print("    return v[t];")
    print("}")
    print("")
    print("}  // namespace klecgc")


if __name__ == "__main__":
    main()
