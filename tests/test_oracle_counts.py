"""Pins for the oracle's line enumeration and truncation (CPU).

Sources: Section 3.2 (Farey series F^1, F^2, line counts A^1, Figure 1),
Lemma 3.1, Section 4 (stated Ntilde values).  The 3D count is pinned to the
textbook Moebius count of primitive vectors in a box, because the printed
formula A^2 = 24(|F^2| - |F^1|) - 2 A^1 does not count lines (it gives 16 for
m = 1, where the 13 lines through 0 in [-1,1]^3 are easy to list).
"""
import math
import os
from math import gcd

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([int(x) for x in line.split()])
    return rows


def farey1(n):
    """F^1_n by its definition (Section 3.2)."""
    return [(p, q) for q in range(1, n + 1) for p in range(0, q + 1) if gcd(p, q) == 1]


def farey2(n):
    """F^2_n by its definition (Section 3.2)."""
    return [(p, q, r) for r in range(1, n + 1) for q in range(0, r + 1) for p in range(0, q + 1)
            if gcd(gcd(p, q), r) == 1]


def mobius(n):
    if n == 1:
        return 1
    res, x, p = 1, n, 2
    while p * p <= x:
        if x % p == 0:
            x //= p
            if x % p == 0:
                return 0
            res = -res
        p += 1
    if x > 1:
        res = -res
    return res


def primitive_lines_closed_form(d, m):
    """Number of lines through 0 with a primitive direction in [-m,m]^d:
    (1/2) sum_k mu(k) ((2 floor(m/k) + 1)^d - 1)."""
    return sum(mobius(k) * ((2 * (m // k) + 1) ** d - 1) for k in range(1, m + 1)) // 2


def test_ntilde_matches_section4():
    for N, Nt in _read_table("ntilde_section4.txt"):
        assert oracle.default_ntilde(N) == Nt


def test_figure1_farey_order3():
    golden = sorted(tuple(r) for r in _read_table("farey_figure1.txt"))
    assert sorted(farey1(3)) == golden
    assert len(oracle.lines(2, 3)) == 16 == 4 * (len(golden) - 1)


@pytest.mark.parametrize("m", range(1, 13))
def test_2d_line_count_is_4_farey_minus_1(m):
    # A^1 = 4 (|F^1| - 1), Section 3.2
    assert len(oracle.lines(2, m)) == 4 * (len(farey1(m)) - 1)
    # |F^1_m| = 1 + phi(1) + ... + phi(m)  (Euler totient)
    phi_sum = sum(sum(1 for a in range(1, n + 1) if gcd(a, n) == 1) for n in range(1, m + 1))
    assert len(farey1(m)) == 1 + phi_sum


@pytest.mark.parametrize("d,m", [(2, m) for m in range(1, 15)] + [(3, m) for m in range(1, 9)])
def test_line_count_moebius(d, m):
    assert len(oracle.lines(d, m)) == primitive_lines_closed_form(d, m)


def test_3d_small_counts_by_hand():
    # [-1,1]^3: 26 non-zero vectors, all primitive, 13 lines.
    assert len(oracle.lines(3, 1)) == 13
    # the corrected Farey identity 24(|F2| - |F1|) - 3 A1 + 1 holds for small m
    for m in range(1, 7):
        A1 = len(oracle.lines(2, m))
        assert len(oracle.lines(3, m)) == 24 * (len(farey2(m)) - len(farey1(m))) - 3 * A1 + 1


@pytest.mark.parametrize("d,m", [(2, 6), (3, 4)])
def test_lines_are_canonical_primitive_and_ordered(d, m):
    L = oracle.lines(d, m)
    seen = set()
    prev = None
    for e in L:
        e = tuple(int(x) for x in e)
        assert max(abs(x) for x in e) <= m
        g = 0
        for x in e:
            g = gcd(g, abs(x))
        assert g == 1
        first = next(x for x in e if x != 0)
        assert first > 0
        assert e not in seen and tuple(-x for x in e) not in seen
        seen.add(e)
        key = (max(abs(x) for x in e), e)
        if prev is not None:
            assert key > prev
        prev = key


def test_lemma31_asymptotics():
    # |F^1_n| ~ 3 n^2 / pi^2, Lemma 3.1.
    n = 60
    f1 = len(farey1(n))
    assert abs(f1 / (3 * n * n / math.pi ** 2) - 1) < 0.05
    # 3D: the ordered triples 0 <= p <= q <= r <= n number ~ n^3/6, so the
    # primitive ones number ~ n^3 / (6 zeta(3)); the constant printed in
    # Lemma 3.1 (1/(12 zeta(3))) is half of that.  Brute force converges to
    # the 1/6 constant (ratio 1.150, 1.075 at n = 30, 60).
    zeta3 = sum(1.0 / k ** 3 for k in range(1, 100000))
    ratios = [len(farey2(n)) / (n ** 3 / (6 * zeta3)) for n in (30, 60)]
    assert ratios[1] < ratios[0] and abs(ratios[1] - 1) < 0.08


def test_terms_per_point_first_workload():
    # 2D, N = 16 (Ntilde = 3), all lines: 16 lines with j in +-1..3 along the
    # axes/diagonals and fewer on the others; the count is the number of
    # orthogonal pairs (k, l) in [-3,3]^2 \ {0}.
    brute = 0
    for k0 in range(-3, 4):
        for k1 in range(-3, 4):
            for l0 in range(-3, 4):
                for l1 in range(-3, 4):
                    if (k0, k1) != (0, 0) and (l0, l1) != (0, 0) and k0 * l0 + k1 * l1 == 0:
                        brute += 1
    assert oracle.terms_count(2, 3, 3) == brute == 192
