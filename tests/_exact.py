"""Exact rational brute force of Eq. 1 for tiny inputs (independent of the oracle).

Uses Python Fractions throughout: mean, N-1 covariance and the quadratic form
by Gauss-Jordan elimination (not Cholesky), so no rounding enters at all.
"""
from fractions import Fraction


def exact_mean_cov(rows):
    n, b = len(rows), len(rows[0])
    mu = [sum(Fraction(r[j]) for r in rows) / n for j in range(b)]
    cov = [[sum((Fraction(r[i]) - mu[i]) * (Fraction(r[j]) - mu[j]) for r in rows) / (n - 1)
            for j in range(b)] for i in range(b)]
    return mu, cov


def exact_solve(A, rhs):
    """Solve A z = rhs exactly by Gauss-Jordan with row pivoting on non-zero entries."""
    n = len(A)
    M = [[Fraction(A[i][j]) for j in range(n)] + [Fraction(rhs[i])] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [v / piv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [M[i][n] for i in range(n)]


def exact_scores(stat_rows, scored_rows):
    mu, cov = exact_mean_cov(stat_rows)
    out = []
    for s in scored_rows:
        d = [Fraction(s[j]) - mu[j] for j in range(len(mu))]
        z = exact_solve(cov, d)
        out.append(sum(a * b for a, b in zip(d, z)))
    return out
