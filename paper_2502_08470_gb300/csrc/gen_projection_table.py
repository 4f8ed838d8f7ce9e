#!/usr/bin/env python3
"""Generate sk_projection_table.h: the interpolation projection of the polynomial interpolation
scheme (Definition "def:polyinterpscheme", operator Omega^N of Definition "interpooperator"), in
the factorial-scaled coordinates used by the CUDA wavefront.

For order N the Chebyshev extrema of [0, 1] are u_r = (1 + cos(pi r / N)) / 2, r = 0..N.  A series
f(u) = sum_j c_j u^j / j! sampled at the nodes and interpolated by a degree-N polynomial has
factorial-scaled coefficients a'_n = sum_j P[n][j] c_j with P = D V^{-1} W D_ext^{-1},
V_{rn} = u_r^n (n <= N), W_{rj} = u_r^j, D = diag(n!).  Columns j <= N of P are the identity; the
table stores columns j = N+1 .. N+kJMax.  Everything is computed with 60-digit decimals (cos by
its Taylor series, Gauss-Jordan elimination with partial pivoting) and rounded once to double.

Run from this directory:  python3 gen_projection_table.py > sk_projection_table.h
"""
from decimal import Decimal, getcontext
from math import factorial

getcontext().prec = 60
NMAX, JMAX = 12, 12


def pi_dec():
    # Machin's formula: pi = 16 atan(1/5) - 4 atan(1/239)
    def atan_inv(x):
        x = Decimal(x)
        term = 1 / x
        total = term
        x2 = x * x
        k = 1
        while True:
            term /= -x2
            t = term / (2 * k + 1)
            if abs(t) < Decimal(10) ** -70:
                break
            total += t
            k += 1
        return total
    return 16 * atan_inv(5) - 4 * atan_inv(239)


PI = pi_dec()


def cos_dec(x):
    x = Decimal(x)
    term = Decimal(1)
    total = term
    k = 0
    while True:
        term *= -x * x / ((2 * k + 1) * (2 * k + 2))
        k += 1
        if abs(term) < Decimal(10) ** -70:
            break
        total += term
    return total


def projection(N):
    n1 = N + 1
    u = [(1 + cos_dec(PI * r / N)) / 2 for r in range(n1)]
    def power(x, k):  # x^k with 0^0 = 1
        v = Decimal(1)
        for _ in range(k):
            v *= x
        return v
    V = [[power(u[r], n) for n in range(n1)] for r in range(n1)]
    Wm = [[power(u[r], N + 1 + jj) for jj in range(JMAX)] for r in range(n1)]
    for col in range(n1):  # Gauss-Jordan on [V | W]
        piv = max(range(col, n1), key=lambda r: abs(V[r][col]))
        V[col], V[piv] = V[piv], V[col]
        Wm[col], Wm[piv] = Wm[piv], Wm[col]
        for r in range(n1):
            if r == col:
                continue
            f = V[r][col] / V[col][col]
            V[r] = [a - f * b for a, b in zip(V[r], V[col])]
            Wm[r] = [a - f * b for a, b in zip(Wm[r], Wm[col])]
    out = []
    for n in range(n1):
        row = []
        for jj in range(JMAX):
            j = N + 1 + jj
            g = Wm[n][jj] / V[n][n]
            row.append(g * factorial(n) / factorial(j))
        out.append(row)
    return out


def main():
    print("// Generated by gen_projection_table.py; do not edit.  Interpolation projection of the")
    print("// polynomial interpolation scheme in factorial-scaled coordinates: proj_coef(N, n, jj) is the")
    print("// weight of series coefficient j = N + 1 + jj in interpolant coefficient n (order N).  A")
    print("// constexpr function of its indices, so unrolled device loops fold it into immediates.")
    print("#pragma once")
    print("")
    print("namespace sk {")
    print("")
    print(f"constexpr int kProjNMax = {NMAX};")
    print(f"constexpr int kProjJMax = {JMAX};")
    print("__host__ __device__ constexpr double proj_coef(int N, int n, int jj) {")
    print("    switch (N * 1024 + n * 32 + jj) {")
    for N in range(2, NMAX + 1):
        P = projection(N)
        for n in range(N + 1):
            for jj in range(JMAX):
                v = float(P[n][jj])
                if v != 0.0:
                    print(f"        case {N * 1024 + n * 32 + jj}: return {v:.17g};")
    print("        default: return 0.0;")
    print("    }")
    print("}")
    print("")
    print("}  // namespace sk")


if __name__ == "__main__":
    main()
