"""Write expm1_table.cuh: the constants of the table-driven e^a - 1 used by the
solver's Bernoulli function (see solver.cuh: expm1_pos for the method).

2^(j/N), j = 0..N-1 (N = 1024), and ln(2)/N are evaluated with 60 significant
decimal digits (Python's decimal module) and split into a double and the
double nearest to the remainder. Run from this directory:

    python gen_expm1_table.py > expm1_table.cuh
"""
from decimal import Decimal, getcontext

getcontext().prec = 60

TABLE_BITS = 10
N = 1 << TABLE_BITS


def split(d: Decimal):
    hi = float(d)
    lo = float(d - Decimal(hi))
    return hi, lo


def main():
    ln2 = Decimal(2).ln()
    l1, l2 = split(ln2 / N)
    inv = float(N / ln2)
    rows = []
    for j in range(N):
        hi, lo = split((ln2 * j / N).exp())
        rows.append(f"    {{{hi.hex()}, {lo.hex()}}},   // 2^({j}/{N})")
    print("// Generated by gen_expm1_table.py (60-digit decimal arithmetic); do not edit.")
    print("#pragma once")
    print("namespace sdcef {")
    print(f"constexpr int kExpTabBits = {TABLE_BITS};")
    print(f"constexpr double kExpInvL = {inv.hex()};   // {N} / ln 2")
    print(f"constexpr double kExpL1 = {l1.hex()};   // ln 2 / {N}, leading double")
    print(f"constexpr double kExpL2 = {l2.hex()};   // ln 2 / {N} - kExpL1")
    print(f"// 2^(j/{N}) = hi + lo")
    print(f"__device__ const double2 kExp2Tab[{N}] = {{")
    print("\n".join(rows))
    print("};")
    print("}  // namespace sdcef")


if __name__ == "__main__":
    main()
