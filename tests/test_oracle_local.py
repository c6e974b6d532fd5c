"""Pins of the oracle's local solve (the root of Eq. 2 at one node).

Each check holds the root against something other than its own formula:
closed forms, the equation itself with its max(., 0) clamps, an independent
bisection of the equation, and the unshifted textbook quadratic.
"""
import math

import numpy as np
import pytest

import oracle

INF = math.inf


def eq2_lhs(u, a, s):
    """sum_d max(u - a_d, 0)^2 - s^2: zero at the root of Eq. 2 (scaled by h^2)."""
    return sum(max(u - ad, 0.0) ** 2 for ad in a) - s * s


def bisect_root(a, s):
    """Root of eq2_lhs by bisection on [min a, min a + s] (the left side
    increases strictly there and changes sign on that interval)."""
    lo = min(a)
    hi = lo + s
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if eq2_lhs(mid, a, s) < 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("s", [1.0, 1.0 / 64, 1.0 / 512, 3.7])
def test_closed_forms(s):
    # one finite neighbour: U = a + s
    assert oracle.local_solve(0.0, INF, INF, s) == s
    assert oracle.local_solve(INF, 2.0, INF, s) == 2.0 + s
    # two equal neighbours, third absent: U = a + s / sqrt(2)
    assert oracle.local_solve(0.0, 0.0, INF, s) == pytest.approx(s / math.sqrt(2), rel=1e-15)
    # three equal neighbours: U = a + s / sqrt(3)
    assert oracle.local_solve(1.0, 1.0, 1.0, s) == pytest.approx(1.0 + s / math.sqrt(3), rel=1e-15)
    # a neighbour that is not smaller than the 1D root is ignored
    assert oracle.local_solve(0.0, s, s * 10, s) == s
    # no information
    assert oracle.local_solve(INF, INF, INF, s) == INF


def test_point_source_corner_values():
    # F = 1 source at the origin: U(1,0,0) = h, U(1,1,0) = h (1 + 1/sqrt 2),
    # U(1,1,1) from three equal neighbours = U(1,1,0) + h / sqrt 3
    h = 1.0 / 64
    u100 = oracle.local_solve(0.0, INF, INF, h)
    u110 = oracle.local_solve(u100, u100, INF, h)
    u111 = oracle.local_solve(u110, u110, u110, h)
    assert u100 == h
    assert u110 == pytest.approx(h * (1 + 1 / math.sqrt(2)), rel=1e-15)
    assert u111 == pytest.approx(h * (1 + 1 / math.sqrt(2)) + h / math.sqrt(3), rel=1e-15)


def _random_triples(rng, n):
    out = []
    for _ in range(n):
        s = float(10 ** rng.uniform(-4, 1))
        base = float(rng.uniform(-2, 5))
        kind = rng.integers(0, 5)
        a = base + rng.uniform(0, 1.5, 3) * s
        if kind == 1:
            a[rng.integers(0, 3)] = INF
        elif kind == 2:
            a[:2] = INF
        elif kind == 3:
            a[1] = a[0]  # ties
        elif kind == 4:
            a[:] = a[0]
        out.append((tuple(float(v) for v in rng.permutation(a)), s))
    return out


def test_root_satisfies_eq2_and_matches_bisection():
    rng = np.random.default_rng(1)
    for a, s in _random_triples(rng, 4000):
        u = oracle.local_solve(*a, s)
        assert math.isfinite(u)
        # the root exceeds the smallest neighbour and solves Eq. 2
        assert u > min(a)
        assert abs(eq2_lhs(u, a, s)) <= 1e-13 * s * s + 1e-15 * max(abs(u), 1) * s
        ub = bisect_root(a, s)
        assert u == pytest.approx(ub, rel=2e-15, abs=4e-16 * max(abs(u), 1.0))


def test_symmetric_in_arguments():
    rng = np.random.default_rng(2)
    for a, s in _random_triples(rng, 500):
        u = oracle.local_solve(*a, s)
        for perm in ((1, 0, 2), (2, 1, 0), (0, 2, 1), (1, 2, 0), (2, 0, 1)):
            assert oracle.local_solve(*(a[p] for p in perm), s) == u


def test_monotone_and_shift_invariant():
    rng = np.random.default_rng(3)
    for a, s in _random_triples(rng, 500):
        u = oracle.local_solve(*a, s)
        # raising one neighbour never lowers the root
        for d in range(3):
            b = list(a)
            if math.isfinite(b[d]):
                b[d] += s * 0.3
                assert oracle.local_solve(*b, s) >= u
        # Lambda(a + c) = Lambda(a) + c for exactly representable shifts
        c = 2.0 ** int(rng.integers(-3, 3))
        shifted = oracle.local_solve(*(v + c for v in a), s)
        assert shifted == pytest.approx(u + c, rel=4e-15)


def test_textbook_quadratic_agrees_within_cancellation():
    rng = np.random.default_rng(4)
    for a, s in _random_triples(rng, 2000):
        u = oracle.local_solve(*a, s)
        ut = oracle.local_solve_textbook(*a, s)
        finite = [v for v in a if math.isfinite(v)]
        scale = max(abs(v) for v in finite) + s
        # unshifted form loses ~ (scale / s)^2 ulps of the discriminant
        tol = 1e-15 * scale * (1.0 + scale / s)
        assert abs(u - ut) <= tol, (a, s, u, ut)
