"""Write expm1_table.cuh: the constants of the table-driven e^a - 1 used by the
solver's Bernoulli function (see expm1_table.cuh for the method).

2^(j/64), j = 0..63, and ln(2)/64 are evaluated with 60 significant decimal
digits (Python's decimal module) and split into a double and the double
nearest to the remainder. Run from this directory:

    python gen_expm1_table.py > expm1_table.cuh
"""
from decimal import Decimal, getcontext

getcontext().prec = 60


def split(d: Decimal):
    hi = float(d)
    lo = float(d - Decimal(hi))
    return hi, lo


def main():
    ln2 = Decimal(2).ln()
    l1, l2 = split(ln2 / 64)
    inv = float(64 / ln2)
    rows = []
    for j in range(64):
        hi, lo = split((ln2 * j / 64).exp())
        rows.append(f"    {{{hi.hex()}, {lo.hex()}}},   // 2^({j}/64)")
    print("// Generated by gen_expm1_table.py (60-digit decimal arithmetic); do not edit.")
    print("#pragma once")
    print("namespace sdcef {")
    print(f"constexpr double kExpInvL = {inv.hex()};   // 64 / ln 2")
    print(f"constexpr double kExpL1 = {l1.hex()};   // ln 2 / 64, leading double")
    print(f"constexpr double kExpL2 = {l2.hex()};   // ln 2 / 64 - kExpL1")
    print("// 2^(j/64) = hi + lo")
    print("__device__ const double2 kExp2Tab[64] = {")
    print("\n".join(rows))
    print("};")
    print("}  // namespace sdcef")


if __name__ == "__main__":
    main()
