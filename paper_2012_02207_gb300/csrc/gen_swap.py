"""Generate the x<->z swap matrices used by the rotation-accelerated M2L.

Sec. 2.4 of Mukherjee et al. (2021): the M2L rotates the source expansion
about z, swaps x and z, rotates about z again and swaps back, so that the
translation runs along z; the swap matrices are generated once and saved for
p <= 30.

The library works with hat-normalised regular harmonics
    Shat_n^m(r) = sqrt((n+m)!(n-m)!) * Upsilon_n^m(r),
(Upsilon in the normalisation of Sec. 2.2), split into real parts
c_n^m = Re Shat_n^m (m = 0..n) and s_n^m = Im Shat_n^m (m = 1..n). The swap
(x, y, z) -> (z, y, x) keeps y, so it maps cosine parts to cosine parts and
sine parts to sine parts:
    c_n^m(z, y, x) = sum_{m'} A_n[m][m'] c_n^{m'}(x, y, z)
    s_n^m(z, y, x) = sum_{m'} B_n[m][m'] s_n^{m'}(x, y, z)
This script finds A_n and B_n exactly: it builds Upsilon_n^m as polynomials
with rational coefficients, swaps the exponents of x and z, and solves for
the coefficients in the basis using the 2n+1 monomials of z-degree <= 1 (a
harmonic polynomial is fixed by them). The hat normalisation introduces
square roots of rationals, which are rounded once, correctly, to FP64.

Run:  python gen_swap.py > swap_table.inc
"""
from __future__ import annotations

import sys
from fractions import Fraction
from math import factorial, isqrt

PMAX = 30


def poly_add(a, b, cb=Fraction(1)):
    out = dict(a)
    for k, v in b.items():
        out[k] = out.get(k, Fraction(0)) + cb * v
        if out[k] == 0:
            del out[k]
    return out


def poly_scale(a, c):
    return {k: v * c for k, v in a.items()} if c != 0 else {}


def poly_mulmono(a, dx, dy, dz):
    return {(i + dx, j + dy, k + dz): v for (i, j, k), v in a.items()}


def regular_polys(pmax):
    """Re and Im of Upsilon_n^m as {(i,j,k): Fraction} for x^i y^j z^k."""
    U = {}
    U[(0, 0)] = ({(0, 0, 0): Fraction(1)}, {})
    for m in range(1, pmax + 1):
        re, im = U[(m - 1, m - 1)]
        # (x + i y)(re + i im) / (2m)
        nre = poly_add(poly_mulmono(re, 1, 0, 0), poly_mulmono(im, 0, 1, 0), Fraction(-1))
        nim = poly_add(poly_mulmono(im, 1, 0, 0), poly_mulmono(re, 0, 1, 0))
        c = Fraction(1, 2 * m)
        U[(m, m)] = (poly_scale(nre, c), poly_scale(nim, c))
    for m in range(0, pmax):
        re, im = U[(m, m)]
        U[(m + 1, m)] = (poly_mulmono(re, 0, 0, 1), poly_mulmono(im, 0, 0, 1))
    for m in range(0, pmax + 1):
        for n in range(m + 2, pmax + 1):
            c = Fraction(1, (n + m) * (n - m))
            parts = []
            for q in range(2):
                a = U[(n - 1, m)][q]
                b = U[(n - 2, m)][q]
                za = poly_scale(poly_mulmono(a, 0, 0, 1), Fraction(2 * n - 1))
                r2b = poly_add(poly_add(poly_mulmono(b, 2, 0, 0), poly_mulmono(b, 0, 2, 0)), poly_mulmono(b, 0, 0, 2))
                parts.append(poly_scale(poly_add(za, r2b, Fraction(-1)), c))
            U[(n, m)] = (parts[0], parts[1])
    return U


def swap_xz(a):
    return {(k, j, i): v for (i, j, k), v in a.items()}


def solve(mat, rhs):
    """Solve mat @ X = rhs exactly (Gauss-Jordan on Fractions)."""
    n = len(mat)
    aug = [list(mat[i]) + list(rhs[i]) for i in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if aug[r][col] != 0)
        aug[col], aug[piv] = aug[piv], aug[col]
        pv = aug[col][col]
        aug[col] = [v / pv for v in aug[col]]
        for r in range(n):
            if r != col and aug[r][col] != 0:
                f = aug[r][col]
                aug[r] = [vr - f * vc for vr, vc in zip(aug[r], aug[col])]
    return [row[n:] for row in aug]


def signed_sqrt_to_float(sign: int, q: Fraction) -> float:
    """Correctly rounded sign * sqrt(q) for a non-negative rational q."""
    if q == 0:
        return 0.0
    num, den = q.numerator, q.denominator
    shift = 240
    root = isqrt((num << (2 * shift)) // den)  # floor(sqrt(q) * 2^shift)
    return sign * float(Fraction(root, 1 << shift))


def swap_blocks(U, n):
    """Exact A_n (cos) and B_n (sin) blocks in the plain Upsilon basis."""
    blocks = []
    for q, ms in ((0, list(range(0, n + 1))), (1, list(range(1, n + 1)))):
        par = q  # cosine parts are even in y, sine parts odd
        monos = [(n - c - j, j, c) for c in (0, 1) for j in range(0, n - c + 1) if j % 2 == par]
        assert len(monos) == len(ms)
        if not ms:
            blocks.append([])
            continue
        basis = [U[(n, mp)][q] for mp in ms]
        mat = [[basis[col].get(mono, Fraction(0)) for col in range(len(ms))] for mono in monos]
        tgt = [swap_xz(U[(n, m)][q]) for m in ms]
        rhs = [[tgt[col].get(mono, Fraction(0)) for col in range(len(ms))] for mono in monos]
        X = solve(mat, rhs)  # column j of X: coefficients of target j
        # T[m][m'] = X[m'][m]
        blocks.append([[X[j][i] for j in range(len(ms))] for i in range(len(ms))])
    return blocks


def hat_blocks(n, blocks):
    out = []
    for blk, ms in zip(blocks, (list(range(0, n + 1)), list(range(1, n + 1)))):
        rows = []
        for i, m in enumerate(ms):
            row = []
            for j, mp in enumerate(ms):
                v = blk[i][j]
                ratio = Fraction(factorial(n + m) * factorial(n - m), factorial(n + mp) * factorial(n - mp))
                row.append(signed_sqrt_to_float(1 if v >= 0 else -1, v * v * ratio))
            rows.append(row)
        out.append(rows)
    return out


def translation_coefficients(pmax):
    """(n+k)!/(w_n^m w_k^m) with w_n^m = sqrt((n+m)!(n-m)!), correctly rounded."""
    out = {}
    for n in range(pmax + 1):
        for k in range(pmax + 1):
            for m in range(min(n, k) + 1):
                q = Fraction(factorial(n + k) ** 2,
                             factorial(n + m) * factorial(n - m) * factorial(k + m) * factorial(k - m))
                out[(n, k, m)] = signed_sqrt_to_float(1, q)
    return out


def main(pmax=PMAX, out=sys.stdout):
    U = regular_polys(pmax)
    cos_vals, sin_vals = [], []
    for n in range(pmax + 1):
        a, b = hat_blocks(n, swap_blocks(U, n))
        cos_vals += [v for row in a for v in row]
        sin_vals += [v for row in b for v in row]
    w = out.write
    w("// Generated by gen_swap.py; do not edit.\n")
    w("// x<->z swap of the hat-normalised regular harmonics, degrees 0..%d.\n" % pmax)
    w("// Degree n: cosine block (n+1)x(n+1) at offset sum_{k<n}(k+1)^2, rows m = 0..n;\n")
    w("// sine block n x n at offset sum_{k<n} k^2, rows m = 1..n. Row-major.\n")
    w("#define GBFMM_SWAP_PMAX %d\n" % pmax)
    for name, vals in (("kSwapCos", cos_vals), ("kSwapSin", sin_vals)):
        w("static const double %s[%d] = {\n" % (name, len(vals)))
        for i in range(0, len(vals), 4):
            w("  " + ", ".join(float.hex(v) for v in vals[i:i + 4]) + ",\n")
        w("};\n")



if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else PMAX)
