"""Pins of the oracle's basis and time integrator (CPU only).

Each check compares the oracle with something fixed outside it: closed-form LGL
nodes and weights, exactness of D and of the quadrature on polynomials, the SBP
property, and the Runge-Kutta order conditions.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def test_lgl_closed_forms():
    # N = 3: nodes +-1, +-1/sqrt(5); weights 1/6, 5/6.  N = 4: 0, +-sqrt(3/7), +-1;
    # weights 1/10, 49/90, 32/45 (standard Gauss-Lobatto tables).
    xi, w, _, _ = O.lgl(3)
    s = 1 / np.sqrt(5)
    assert np.allclose(xi, [-1, -s, s, 1], atol=1e-15, rtol=0)
    assert np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15, rtol=0)
    xi, w, _, _ = O.lgl(4)
    t = np.sqrt(3 / 7)
    assert np.allclose(xi, [-1, -t, 0, t, 1], atol=1e-15, rtol=0)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15, rtol=0)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7])
def test_D_exact_on_polynomials(N):
    xi, _, D, _ = O.lgl(N)
    for k in range(N + 1):
        f = xi ** k
        df = k * xi ** (k - 1) if k > 0 else np.zeros_like(xi)
        assert np.allclose(D @ f, df, atol=1e-12 * max(1, k * N), rtol=0)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7])
def test_quadrature_exactness_and_sbp(N):
    xi, w, D, Dt = O.lgl(N)
    for k in range(2 * N):  # LGL integrates degree <= 2N-1 exactly
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(w @ xi ** k - exact) < 1e-14
    W = np.diag(w)
    Bm = np.zeros((N + 1, N + 1))
    Bm[0, 0], Bm[N, N] = -1, 1
    assert np.allclose(W @ D + D.T @ W, Bm, atol=1e-13, rtol=0)
    # Dt = 2D - W^-1 B: zero diagonal and W Dt antisymmetric
    assert np.allclose(Dt, 2 * D - np.linalg.inv(W) @ Bm, atol=1e-12, rtol=0)
    assert np.all(np.diag(Dt) == 0)
    assert np.allclose(W @ Dt, -(W @ Dt).T, atol=1e-12, rtol=0)


def test_lgl_long_double_agrees():
    for N in (3, 4, 7):
        a = O.lgl(N)
        b = O.lgl(N, precision="long")
        for x, y in zip(a, b):
            assert np.allclose(x, y, atol=1e-14, rtol=0)


def _butcher_from_2n(A, B):
    """Butcher tableau of the 2N-storage scheme dq_s = A_s dq_{s-1} + dt f(Y_s),
    q_s = q_{s-1} + B_s dq_s, Y_{s+1} = q_s, in exact rational arithmetic."""
    s = len(A)
    a = [[Fraction(0)] * s for _ in range(s)]
    b = [Fraction(0)] * s

    def coef(j, r):  # coefficient of k_j in dq_r
        c = Fraction(1)
        for m in range(j + 1, r + 1):
            c *= A[m]
        return c

    for i in range(1, s):          # stage i uses q_{i-1}
        for j in range(i):
            a[i][j] = sum(B[r] * coef(j, r) for r in range(j, i))
    for j in range(s):
        b[j] = sum(B[r] * coef(j, r) for r in range(j, s))
    return a, b


def test_lsrk_order_conditions():
    # The oracle's coefficients (doubles) are converted exactly to rationals and the
    # eight conditions of order <= 4 evaluated without rounding: the published rationals
    # meet them to ~1e-26 and their doubles to ~1e-17, while a one-digit typo in any
    # 13-digit numerator or denominator leaves residuals of ~1e-14 to 1e-13.
    A, B, c = (list(map(Fraction, v)) for v in O.lsrk_coeffs())
    a, b = _butcher_from_2n(A, B)
    s = len(A)
    cc = [sum(row) for row in a]
    assert max(abs(float(x - y)) for x, y in zip(cc, c)) < 1e-15

    def dot(x, y):
        return sum(p * q for p, q in zip(x, y))

    def amul(v):
        return [dot(a[i], v) for i in range(s)]

    ac = amul(cc)
    conds = [
        (sum(b), Fraction(1)),
        (dot(b, cc), Fraction(1, 2)),
        (dot(b, [x ** 2 for x in cc]), Fraction(1, 3)),
        (dot(b, ac), Fraction(1, 6)),
        (dot(b, [x ** 3 for x in cc]), Fraction(1, 4)),
        (dot(b, [x * y for x, y in zip(cc, ac)]), Fraction(1, 8)),
        (dot(b, amul([x ** 2 for x in cc])), Fraction(1, 12)),
        (dot(b, amul(ac)), Fraction(1, 24)),
    ]
    for got, want in conds:
        assert abs(float(got - want)) < 1e-15, float(got - want)
    # a fifth-order condition is not met: the scheme is exactly fourth order
    assert abs(float(dot(b, [x ** 4 for x in cc]) - Fraction(1, 5))) > 1e-6


def test_lsrk_fourth_order_on_linear_ode():
    A, B, _ = O.lsrk_coeffs()

    def integrate(lam, T, n):
        y, dt, dy = 1.0 + 0j, T / n, 0j
        for _ in range(n):
            for s in range(5):
                dy = A[s] * dy + dt * lam * y
                y = y + B[s] * dy
        return y

    lam, T = -1.0 + 2.0j, 1.0
    e1 = abs(integrate(lam, T, 20) - np.exp(lam * T))
    e2 = abs(integrate(lam, T, 40) - np.exp(lam * T))
    assert 14.0 < e1 / e2 < 18.0
