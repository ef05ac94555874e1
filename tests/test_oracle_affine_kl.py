"""Pins of the oracle's version of the paper's KL variant (Sec. 3.1.1,
Eq. KL-expansion-deterministic; Sec. 4): uniform inputs psi ~ U(-1, 1), the
pivoted Cholesky factor of the Gaussian covariance and its extension to other
points, the ellipticity cap on s, the field's covariance, and the isotropic
conductivity G = G0 (1 + Z) in the assembly."""
import math

import numpy as np
import pytest

import oracle as O
from helpers import gauss3_assembly


def gauss_cov(X, Y, sigma2, ell):
    d2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    return sigma2 * np.exp(-d2 / ell ** 2)


def test_uniform_inputs():
    P = np.stack([O.psi_uniform(7, 2, i, 9) for i in range(4000)])
    assert P.min() >= -1.0 and P.max() <= 1.0
    assert abs(P.mean()) < 0.02 and abs(P.var() - 1.0 / 3.0) < 0.01
    from scipy import stats
    assert stats.kstest((P[:, 3] + 1) / 2, "uniform").pvalue > 1e-3
    # the same counters as the normals: one Philox block per mode pair, so
    # changing the level, the id or the seed changes every value
    a = O.psi_uniform(7, 2, 5, 9)
    for other in (O.psi_uniform(7, 3, 5, 9), O.psi_uniform(7, 2, 6, 9), O.psi_uniform(8, 2, 5, 9)):
        assert np.all(a != other)


def test_full_rank_factor_is_the_cholesky_factor():
    X = O.cell_centroids(2, [1.0, 1.0], [4, 3])
    C = gauss_cov(X, X, 0.7, 0.8)
    n = len(X)
    m, piv, Lp, L = O.pivoted_cholesky(X, 0.7, 0.8, n, 0.0, want_L=True)
    assert m == n and sorted(piv.tolist()) == list(range(n))
    np.testing.assert_allclose(L @ L.T, C, atol=1e-12)
    # the pivot rows form the ordinary Cholesky factor of the permuted matrix
    np.testing.assert_allclose(Lp[:m, :m], np.linalg.cholesky(C[np.ix_(piv, piv)]), atol=1e-10)


def test_low_rank_factor_interpolates_at_the_pivots_and_greedy_order():
    X = O.cell_centroids(3, [1.0, 1.0, 1.0], [5, 4, 3])
    sigma2, ell = 1.3, 0.5
    C = gauss_cov(X, X, sigma2, ell)
    m, piv, Lp, L = O.pivoted_cholesky(X, sigma2, ell, 12, 0.0, want_L=True)
    assert m == 12
    R = C - L @ L.T
    # exact on the pivot rows and columns; the remainder is positive semidefinite
    assert np.abs(R[piv]).max() < 1e-12 and np.abs(R[:, piv]).max() < 1e-12
    assert np.linalg.eigvalsh(R).min() > -1e-10
    # greedy: every diagonal equals sigma2, so the first pivot is index 0 and
    # the second the point farthest from it (largest remainder 1 - k^2)
    assert piv[0] == 0
    d = ((X - X[0]) ** 2).sum(1)
    assert piv[1] == int(np.argmax(d))
    # each pivot is the largest remainder diagonal at its step
    for k in range(1, m):
        Lk = L[:, :k]
        rem = np.diag(C) - (Lk ** 2).sum(1)
        assert math.isclose(rem[piv[k]], rem.max(), rel_tol=1e-12)


def test_trace_tolerance_stops_the_factor():
    X = O.cell_centroids(2, [1.0, 1.0], [8, 8])
    C = gauss_cov(X, X, 1.0, 0.5)
    for tol in (1e-2, 1e-4, 1e-6):
        m, piv, Lp, L = O.pivoted_cholesky(X, 1.0, 0.5, 64, tol, want_L=True)
        rem = np.trace(C - L @ L.T) / np.trace(C)
        assert rem <= tol
        if m > 1:
            Lm = L[:, :m - 1]
            assert np.trace(C - Lm @ Lm.T) / np.trace(C) > tol   # not stopped earlier


def test_extension_reproduces_the_factor_and_the_kernel():
    X = O.cell_centroids(3, [1.0, 1.0, 1.0], [6, 6, 6])
    sigma2, ell, M = 1.0, 0.5, 40
    m, piv, Lp, L = O.pivoted_cholesky(X, sigma2, ell, M, 0.0, want_L=True)
    Phi = O.pc_eval(X, X[piv], sigma2, ell, M, m, Lp)
    np.testing.assert_allclose(Phi, L, atol=1e-12)
    # at new points (a finer grid) the remainder kernel C - l l^T stays
    # positive semidefinite: |C(x, x') - l(x).l(x')| <= sqrt(r(x) r(x')),
    # r(x) = C(x, x) - |l(x)|^2 >= 0 (Cauchy-Schwarz)
    Y = O.cell_centroids(3, [1.0, 1.0, 1.0], [12, 12, 12])[::37]
    PY = O.pc_eval(Y, X[piv], sigma2, ell, M, m, Lp)
    R = gauss_cov(Y, Y, sigma2, ell) - PY @ PY.T
    r = np.diag(R)
    assert r.min() > -1e-12
    assert np.all(np.abs(R) <= np.sqrt(np.outer(np.maximum(r, 0), np.maximum(r, 0))) + 1e-12)
    assert np.linalg.eigvalsh(R).min() > -1e-10
    # and it is exact between a new point and every pivot
    np.testing.assert_allclose(PY @ L[piv].T,
                               gauss_cov(Y, X[piv], sigma2, ell), atol=1e-10)


def test_ellipticity_cap_and_field_covariance():
    akl = O.AffineKL(2, [1.0, 1.0], (6, 6), [(6, 6), (12, 12)], 1.0, 0.5, 20, 0.0, 0.3, 0.5)
    bound = np.abs(akl.Phi[0]).sum(1).max()       # level 0 is the candidate grid
    assert akl.s_eff == pytest.approx(min(0.3, 0.5 / bound))
    # the extreme inputs psi_k = sign(l_k(x)) reach the cap exactly at the
    # maximising candidate and nowhere there exceed it; on a finer grid the
    # field stays within a few per cent of the cap (the sup is taken on the
    # candidates)
    P = akl.Phi[0]
    i = int(np.argmax(np.abs(P).sum(1)))
    z = akl.s_eff * np.sign(P[i]) @ P.T
    assert abs(z.max() - 0.5) < 1e-12
    assert akl.s_eff * np.abs(akl.Phi[1]).sum(1).max() <= 0.5 * 1.05
    # covariance of Z: s_eff^2 / 3 Phi Phi^T (psi uniform, variance 1/3)
    rng_ids = range(6000)
    Zs = np.stack([akl.field(1, O.psi_uniform(3, 1, i, 20))[0] for i in rng_ids])
    C_emp = np.cov(Zs[:, ::17].T)
    C_th = akl.s_eff ** 2 / 3.0 * akl.Phi[1][::17] @ akl.Phi[1][::17].T
    assert np.abs(C_emp - C_th).max() < 0.06 * np.abs(C_th).max()


def test_affine_isotropic_conductivity_assembly():
    rng = np.random.default_rng(3)
    lv = O.make_level(2, (5, 4), 3, (1.0, 0.8), 1.0, 18.5, 0.24, 9.0, 2e-3, 35.0, cond_kind=1)
    Z = rng.uniform(-0.4, 0.4, lv.cells)
    mass, kst = O.assemble(lv, Z)
    K = gauss3_assembly(2, [5, 4], [1.0, 0.8], [2e-3 * (1 + z) * np.eye(2) for z in Z])
    from helpers import dense_K
    np.testing.assert_allclose(dense_K(lv, kst), K, atol=1e-15)
