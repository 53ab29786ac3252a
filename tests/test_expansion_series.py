"""The separable series the tensor-core expansion of the exact model and of virtual snapshots
uses for the coupling factor e^{j x t}, x = 2 pi eps m' n_h (row) and t = n' / n_h in [-1, 1)
(column), checked on the CPU against the exponential itself and scipy's Bessel functions.

  Taylor:    sum_{p<P} (j x)^p t^p / p!                  remainder <= theta^P / P!
  Chebyshev: J_0(x) + 2 sum_{1<=p<P} j^p J_p(x) T_p(t)   remainder <= 2 (theta/2)^P / P! /
                                                                      (1 - theta / (2 (P + 1)))

The kernel sums J_p(x) = (x/2)^p / p! sum_{k<=K} (-x^2/4)^k / (k! (p+1)_k) to K = 2, 4, 6 for
P = 4, 6, 8, and its term chooser uses the two bounds above.  These tests check that the bounds
hold at the largest theta each P is chosen for, that the short Bessel series is close enough
there, and that Chebyshev terms reach further than Taylor terms at every P."""
import math

import numpy as np
import pytest

special = pytest.importorskip("scipy.special")

K_OF_P = {4: 2, 6: 4, 8: 6}


def taylor_bound(theta, P):
    return theta ** P / math.factorial(P)


def chebyshev_bound(theta, P):
    return 2.0 * (theta / 2.0) ** P / math.factorial(P) / (1.0 - theta / (2.0 * (P + 1)))


def largest_theta(bound, P, tol):
    lo, hi = 0.0, 3.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if bound(mid, P) <= tol else (lo, mid)
    return lo


def bessel_short(p, x, K):
    w = -x * x / 4.0
    s = np.zeros_like(x)
    for k in range(K, -1, -1):
        c = 1.0
        for i in range(1, k + 1):
            c /= i * (p + i)
        s = s * w + c
    return (x / 2.0) ** p / math.factorial(p) * s


def grid(theta, n=4001, m=257):
    x = np.linspace(-theta, theta, n)[:, None]
    t = np.linspace(-1.0, 1.0, m)[None, :]
    return x, t


@pytest.mark.parametrize("tol", [1e-6, 1e-5])
@pytest.mark.parametrize("P", [4, 6, 8])
def test_chebyshev_remainder_within_bound(P, tol):
    theta = largest_theta(chebyshev_bound, P, tol)
    x, t = grid(theta)
    series = sum((1.0 if p == 0 else 2.0) * (1j ** p) * special.jv(p, x) * special.eval_chebyt(p, t) for p in range(P))
    err = np.abs(np.exp(1j * x * t) - series).max()
    assert err <= chebyshev_bound(theta, P)
    assert err >= 0.5 * chebyshev_bound(theta, P)  # the bound is not loose


@pytest.mark.parametrize("tol", [1e-6, 1e-5])
@pytest.mark.parametrize("P", [4, 6, 8])
def test_short_bessel_series_where_each_P_is_used(P, tol):
    theta = largest_theta(chebyshev_bound, P, tol)
    x = np.linspace(-theta, theta, 20001)
    for p in range(P):
        ref = special.jv(p, x)
        assert np.abs(bessel_short(p, x, K_OF_P[P]) - ref).max() <= 5e-8 * max(np.abs(special.jv(0, x)).max(), 1.0)


@pytest.mark.parametrize("P", [4, 6, 8])
def test_taylor_remainder_within_bound(P):
    theta = largest_theta(taylor_bound, P, 1e-6)
    x, t = grid(theta)
    series = sum((1j * x * t) ** p / math.factorial(p) for p in range(P))
    assert np.abs(np.exp(1j * x * t) - series).max() <= taylor_bound(theta, P)


def test_chebyshev_reaches_further_than_taylor():
    for tol in (1e-6, 1e-5):
        for P in (4, 6, 8):
            assert largest_theta(chebyshev_bound, P, tol) > 1.6 * largest_theta(taylor_bound, P, tol)
    # the moving-box snapshot scene (theta ~0.072 at split precision) needs six Taylor terms
    # but only four Chebyshev terms
    assert taylor_bound(0.072, 4) > 1e-6 >= chebyshev_bound(0.072, 4)
