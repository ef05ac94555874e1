"""Pins of the oracle's Karhunen-Loeve expansion (Sec. 3.1.1, Eq. KL-expansion)
for the separable exponential covariance: closed-form eigenpairs against a
Nystrom eigen-solve of the kernel, the trace identity, orthonormality, the
mode ordering and the covariance of the synthesised field."""
import math

import numpy as np
import pytest

import oracle as O


def nystrom(length, ell, n=2000):
    """Midpoint-rule Nystrom discretisation of exp(-|x-y|/ell) on [0, length]."""
    h = length / n
    x = (np.arange(n) + 0.5) * h
    Kmat = np.exp(-np.abs(x[:, None] - x[None, :]) / ell) * h
    w, V = np.linalg.eigh(Kmat)
    order = np.argsort(w)[::-1]
    return x, w[order], V[:, order] / math.sqrt(h)


@pytest.mark.parametrize("length,ell", [(1.0, 0.2), (1.0, 0.1), (0.25, 0.1)])
def test_eigenpairs_match_nystrom(length, ell):
    om, lam, nrm = O.kl_1d(length, ell, 8)
    x, wn, Vn = nystrom(length, ell)
    np.testing.assert_allclose(lam, wn[:8], rtol=2e-5)
    for k in range(8):
        phi = np.array([O.kl_phi_1d(length, k, om[k], nrm[k], xx) for xx in x])
        s = np.sign(phi @ Vn[:, k])
        assert np.abs(phi - s * Vn[:, k]).max() < 2e-3
        # parity: cosine modes even, sine modes odd about the centre
        assert math.isclose(O.kl_phi_1d(length, k, om[k], nrm[k], 0.0),
                            (1 if k % 2 == 0 else -1) * O.kl_phi_1d(length, k, om[k], nrm[k], length),
                            rel_tol=1e-12, abs_tol=1e-14)


def test_eigenvalues_decrease_and_roots_bracketed():
    om, lam, _ = O.kl_1d(1.0, 0.2, 40)
    assert np.all(np.diff(lam) < 0)
    A = 0.5
    for k in range(40):
        assert k * math.pi / 2 < om[k] * A < (k + 1) * math.pi / 2


def test_trace_identity():
    # sum of all eigenvalues of a unit-variance kernel = length of the interval
    om, lam, _ = O.kl_1d(1.0, 0.2, 4000)
    c = 1.0 / 0.2
    # tail beyond mode n: lam ~ 2c/w^2 with w ~ n pi: sum_{k>n} 2c/(k pi)^2 ~ 2c/(pi^2 n)
    tail = 2 * c / (math.pi ** 2 * 4000)
    assert abs(lam.sum() + tail - 1.0) < 0.2 * tail


def test_orthonormality():
    length, ell = 1.0, 0.1
    om, lam, nrm = O.kl_1d(length, ell, 10)
    n = 4000
    x = (np.arange(n) + 0.5) * length / n
    Phi = np.array([[O.kl_phi_1d(length, k, om[k], nrm[k], xx) for xx in x] for k in range(10)])
    G = Phi @ Phi.T * (length / n)
    np.testing.assert_allclose(G, np.eye(10), atol=1e-5)


def test_table_order_and_ties():
    idx, sl = O.kl_table(2, [1.0, 1.0], 0.04, 0.2, 18)
    _, lam, _ = O.kl_1d(1.0, 0.2, 18)
    prod = np.array([0.04 * lam[i] * lam[j] for i, j, _ in idx])
    np.testing.assert_allclose(sl ** 2, prod, rtol=1e-14)
    assert np.all(np.diff(sl) <= 0)
    assert idx[0].tolist() == [0, 0, 0]
    # (i,j) and (j,i) are exact ties; the tie-break puts the smaller first index first
    for q in range(17):
        if sl[q] == sl[q + 1]:
            assert idx[q, 0] < idx[q + 1, 0] and idx[q, 0] == idx[q + 1, 1]
    # brute force: the 18 largest of all products with indices < 18
    allp = np.sort((lam[:, None] * lam[None, :]).ravel())[::-1]
    np.testing.assert_allclose(prod / 0.04, allp[:18], rtol=1e-14)


def test_table_3d_uses_both_intervals():
    idx, sl = O.kl_table(3, [1.0, 1.0, 0.25], 0.04, 0.1, 256)
    _, lx, _ = O.kl_1d(1.0, 0.1, 256)
    _, lz, _ = O.kl_1d(0.25, 0.1, 256)
    prod = np.array([0.04 * lx[i] * lx[j] * lz[k] for i, j, k in idx])
    np.testing.assert_allclose(sl ** 2, prod, rtol=1e-13)
    # brute force over a generous index box
    cand = np.sort((lx[:40, None, None] * lx[None, :40, None] * lz[None, None, :12]).ravel())[::-1]
    np.testing.assert_allclose(np.sort(prod / 0.04)[::-1], cand[:256], rtol=1e-13)


def test_field_covariance():
    """Empirical covariance of Z between cell centroids = sum_k lam_k phi_k phi_k."""
    dim, L, n, s2, ell, M = 2, [1.0, 1.0], [8, 8], 0.04, 0.2, 16
    xis = np.stack([O.xi(11, 0, i, M) for i in range(6000)])
    Z = O.kl_field(dim, L, n, s2, ell, M, xis)
    idx, sl = O.kl_table(dim, L, s2, ell, M)
    om, lam, nrm = O.kl_1d(1.0, ell, M)
    cells = [(0, 0), (3, 4), (7, 7)]
    phis = []
    for (i, j) in cells:
        x, y = (i + 0.5) / 8, (j + 0.5) / 8
        phis.append(np.array([O.kl_phi_1d(1.0, a, om[a], nrm[a], x) * O.kl_phi_1d(1.0, b, om[b], nrm[b], y)
                              for a, b, _ in idx]))
    for p, (i, j) in enumerate(cells):
        for q, (k, l) in enumerate(cells):
            theo = np.sum(sl ** 2 * phis[p] * phis[q])
            emp = np.mean(Z[:, j * 8 + i] * Z[:, l * 8 + k])
            assert abs(emp - theo) < 5 * 0.04 * math.sqrt(2.0 / 6000) + 1e-4, (p, q, emp, theo)
    # truncated variance below the full variance sigma2, and close to it on average
    var = np.array([np.sum(sl ** 2 * ph * ph) for ph in phis])
    assert np.all(var < 0.04)
