"""Pins of the oracle's generator: Philox4x32-10 known answers, the own ln and
sin/cos against the C library, and the distribution of the Box-Muller normals
(the KL inputs xi of Sec. 3.1.1, drawn from a counter-based Philox stream)."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from helpers import read_golden


def test_philox_known_answers():
    rows = read_golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        assert r[0] == "philox4x32" and r[1] == "10"
        vals = [int(x, 16) for x in r[2:]]
        out = O.philox4x32_10(vals[0:4], vals[4:6])
        assert out.tolist() == vals[6:10]


def test_ln_matches_libm():
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.random(20000), 2.0 ** -rng.uniform(0, 53, 2000),
                         [2.0 ** -53, 0.5, 1.0, np.nextafter(1.0, 0.0), 0.7071067811865476]])
    for x in xs:
        ref = math.log(x)
        got = O.ln(x)
        assert abs(got - ref) <= 4e-16 * max(1.0, abs(ref)), (x, got, ref)
    assert O.ln(1.0) == 0.0


def test_sincos_matches_libm():
    rng = np.random.default_rng(2)
    us = np.concatenate([rng.random(20000), np.arange(16) / 16.0, [np.nextafter(1.0, 0.0)]])
    for u in us:
        s, c = O.sincos_2pi(u)
        assert abs(s - math.sin(2 * math.pi * u)) <= 1e-15
        assert abs(c - math.cos(2 * math.pi * u)) <= 1e-15
    # exact quadrant points
    assert O.sincos_2pi(0.0) == (0.0, 1.0)
    assert O.sincos_2pi(0.25) == (1.0, 0.0)


def test_xi_is_standard_normal():
    M = 64
    X = np.concatenate([O.xi(7, 1, i, M) for i in range(4000)])
    n = X.size
    assert abs(X.mean()) < 5.0 / math.sqrt(n)
    assert abs(X.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert abs(stats.kurtosis(X, fisher=False) - 3.0) < 0.1
    assert stats.kstest(X, "norm").pvalue > 1e-4


def test_xi_counter_layout_independent_streams():
    a = O.xi(0, 0, 0, 16)
    assert np.array_equal(a, O.xi(0, 0, 0, 16))           # deterministic
    assert not np.allclose(a, O.xi(0, 0, 1, 16))           # sample id
    assert not np.allclose(a, O.xi(0, 1, 0, 16))           # level pair
    assert not np.allclose(a, O.xi(1, 0, 0, 16))           # seed
    # a prefix of a longer draw: mode pairs are counter-indexed
    assert np.array_equal(O.xi(3, 2, 5, 7), O.xi(3, 2, 5, 16)[:7])
    # modes 2j and 2j+1 come from one Philox block: (r cos, r sin) with r^2 = sum
    x = O.xi(0, 0, 0, 2)
    w = O.philox4x32_10([0, 0, 0, 0], [0, 0]).astype(np.uint64)
    k1 = (int(w[0]) >> 5) * 2 ** 26 + (int(w[1]) >> 6)
    u1 = (k1 + 1) * 2.0 ** -53
    assert math.isclose(x[0] ** 2 + x[1] ** 2, -2.0 * math.log(u1), rel_tol=1e-13)


def test_xi_modes_uncorrelated():
    X = np.stack([O.xi(0, 0, i, 8) for i in range(5000)])
    C = np.corrcoef(X.T)
    off = C - np.diag(np.diag(C))
    assert np.abs(off).max() < 5.0 / math.sqrt(5000)
