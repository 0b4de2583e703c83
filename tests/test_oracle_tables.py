"""Pins of the oracle's acceptance tables.

T(x) is checked against a 50-digit evaluation of 2^32 e^{-x} (mpmath, an
implementation independent of libm), for monotonicity and for its boundary
values; Jperp against the closed form 1/2 ln coth(beta A / L) in mpmath; the
table layouts against the scalar functions.
"""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle as O

mp.mp.dps = 50


def test_threshold_boundaries():
    assert O.threshold(0.0) == 0xFFFFFFFF
    assert O.threshold(-3.0) == 0xFFFFFFFF
    assert O.threshold(-math.inf) == 0xFFFFFFFF
    assert O.threshold(math.inf) == 0
    assert O.threshold(1e-300) == 0xFFFFFFFE       # x > 0 never reaches "always"
    assert O.threshold(23.0) == 0                  # 2^32 e^-23 < 1
    assert O.threshold(22.0) > 0                   # 2^32 e^-22 > 1


@pytest.mark.parametrize("x", [1e-9, 1e-3, 0.05, 0.5, 1.0, math.log(2), 2.5, 7.25, 15.0, 21.9])
def test_threshold_matches_high_precision(x):
    exact = mp.mpf(2) ** 32 * mp.exp(-mp.mpf(x))
    T = O.threshold(x)
    # floor of the exact value, up to one unit from the double rounding of exp
    assert abs(T - int(mp.floor(exact))) <= 1
    assert T <= 0xFFFFFFFE


def test_threshold_monotone():
    xs = np.concatenate([np.linspace(-1, 25, 4001), np.geomspace(1e-12, 1e-2, 500)])
    xs.sort()
    Ts = np.array([O.threshold(x) for x in xs], np.int64)
    assert np.all(np.diff(Ts) <= 0)


@pytest.mark.parametrize("beta,A,L", [(10 / 3, 0.99, 32), (1.0, 0.5, 64), (20.0, 1e-3, 64),
                                      (0.1, 1.0, 16)])
def test_jperp_closed_form(beta, A, L):
    a = mp.mpf(beta) * A / L
    want = mp.log(mp.coth(a)) / 2                  # e^{2 Jperp} = coth(beta A / L)
    assert abs(O.jperp(beta, A, L) - float(want)) <= 1e-12 * max(1.0, float(want))
    assert O.jperp(beta, 0.0, L) == math.inf


def test_sqa_x_terms():
    # x = alpha*delta + 2*Jperp*m; m = 0 removes the temporal term even when Jperp is infinite
    assert O.sqa_x(0.25, math.inf, 8, 0) == 2.0
    assert O.sqa_x(0.25, math.inf, 8, 2) == math.inf
    assert O.sqa_x(0.25, math.inf, 8, -2) == -math.inf
    assert O.sqa_x(0.5, 1.5, -4, 2) == -2.0 + 6.0


def test_sqa_table_layout():
    S, L, beta = 50, 32, 10 / 3
    A, B = O.linear_schedule(S)
    dmin, dmax = -12, 16
    T = O.sqa_table(A, B, beta, L, 10, 20, dmin, dmax)
    assert T.shape == (10, (dmax - dmin) // 2 + 1, 3)
    for t in (10, 13, 19):
        alpha = beta * B[t] / L
        jp = O.jperp(beta, A[t], L)
        for di, delta in enumerate(range(dmin, dmax + 1, 2)):
            for mi, m in enumerate((-2, 0, 2)):
                assert T[t - 10, di, mi] == O.threshold(O.sqa_x(alpha, jp, delta, m))
    # larger delta or larger m never raises the acceptance
    assert np.all(np.diff(T.astype(np.int64), axis=1) <= 0)
    assert np.all(np.diff(T.astype(np.int64), axis=2) <= 0)


def test_linear_schedule_midpoints():
    A, B = O.linear_schedule(4)
    assert np.allclose(B, [0.125, 0.375, 0.625, 0.875])
    assert np.allclose(A + B, 1.0)
    assert A.min() > 0                               # A never reaches 0


def test_pt_and_swap_tables():
    betas = np.array([2.0, 1.0, 0.5])
    T = O.pt_table(betas, -6, 6)
    for p, b in enumerate(betas):
        for di, d in enumerate(range(-6, 7, 2)):
            assert T[p, di] == O.threshold(b * d)
    assert O.swap_threshold(2.0, 1.0, 3) == O.threshold(3.0)
    assert O.swap_threshold(2.0, 1.0, 0) == 0xFFFFFFFF
