"""Pins of the oracle's Q1 discretisation (Sec. 3.2, Eq. semi-disc) with lumped
mass and the anisotropic fiber conductivity: textbook stencils, invariants, an
independent higher-order quadrature, tensor-product structure and the exact
implicit-Euler decay of a discrete cosine mode."""
import math

import numpy as np
import pytest

import oracle as O
from helpers import dense_K, gauss3_assembly, read_golden


def level(dim, n, m=4, T=1.0, c=0.0, s_t=1.0, s_l0=1.0, th0=0.0, th1=None, L=None):
    L = L or [1.0] * dim
    return O.make_level(dim, n, m, L, T, c, 0.1, s_t, s_l0, th0, th1)


def test_textbook_laplacian_stencils():
    rows = read_golden("q1_laplacian_stencils.txt")
    gold = {(int(r[0]), r[1]): float(r[2]) for r in rows}
    for dim, n in ((2, (6, 6)), (3, (4, 4, 4))):
        h = 0.25 if dim == 3 else 1.0 / 6
        lv = level(dim, n, L=[n[0] * h] * dim)
        _, kst = O.assemble(lv, np.zeros(lv.cells))
        no = 27 if dim == 3 else 9
        N = n[0] + 1
        centre = (N // 2) * (1 + N + (N * N if dim == 3 else 0))
        row = kst.reshape(-1, no)[centre] / h ** (dim - 2)
        for o in range(no):
            off = [o % 3 - 1, (o // 3) % 3 - 1] + ([o // 9 - 1] if dim == 3 else [])
            nz = sum(1 for v in off if v != 0)
            cls = {0: "centre", 1: "face", 2: "corner" if dim == 2 else "edge", 3: "corner"}[nz]
            assert math.isclose(row[o], gold[(dim, cls)], abs_tol=1e-14), (dim, off, row[o])


@pytest.mark.parametrize("dim,n", [(2, (5, 3)), (3, (3, 2, 2))])
def test_invariants(dim, n):
    rng = np.random.default_rng(3)
    L = [1.0, 0.7, 0.4][:dim]
    lv = level(dim, n, s_t=2.5e-4, s_l0=1e-3, th0=30.0, th1=-45.0, L=L)
    Z = rng.normal(0, 0.3, lv.cells)
    mass, kst = O.assemble(lv, Z)
    K = dense_K(lv, kst)
    np.testing.assert_allclose(K, K.T, atol=1e-18)
    assert np.abs(K @ np.ones(lv.nodes)).max() < 1e-17          # Neumann: constants in the kernel
    assert np.linalg.eigvalsh(K).min() > -1e-17                  # positive semidefinite
    assert math.isclose(mass.sum(), float(np.prod(L)), rel_tol=1e-14)
    h = [L[d] / n[d] for d in range(dim)]
    vol = float(np.prod(h))
    # interior / face / corner lumped masses: vol * 2^(#interior axes) / 2^dim ... checked by counts
    N = [n[d] + 1 for d in range(dim)]
    for A in range(lv.nodes):
        idx = [A % N[0], (A // N[0]) % N[1]] + ([A // (N[0] * N[1])] if dim == 3 else [])
        ncell = np.prod([1 if idx[d] in (0, n[d]) else 2 for d in range(dim)])
        assert math.isclose(mass[A], vol * ncell / 2 ** dim, rel_tol=1e-14)


@pytest.mark.parametrize("dim,n,L", [(2, (3, 4), [1.0, 1.2]), (3, (2, 3, 2), [1.0, 1.0, 0.25])])
def test_against_independent_quadrature(dim, n, L):
    rng = np.random.default_rng(4)
    th0, th1 = 30.0, (60.0 if dim == 3 else 30.0)
    lv = level(dim, n, s_t=2.5e-4, s_l0=1e-3, th0=th0, th1=th1, L=L)
    Z = rng.normal(0, 0.5, lv.cells)
    _, kst = O.assemble(lv, Z)
    Dc = []
    h = [L[d] / n[d] for d in range(dim)]
    for ci in range(lv.cells):
        kz = ci // (n[0] * n[1]) if dim == 3 else 0
        th = th0 if dim == 2 else th0 + (th1 - th0) * (kz + 0.5) * h[2] / L[2]
        f = np.array([math.cos(math.radians(th)), math.sin(math.radians(th)), 0.0])[:dim]
        sl = 1e-3 * math.exp(Z[ci])
        Dc.append(2.5e-4 * np.eye(dim) + (sl - 2.5e-4) * np.outer(f, f))
    K_ref = gauss3_assembly(dim, n, L, Dc)
    np.testing.assert_allclose(dense_K(lv, kst), K_ref, rtol=0, atol=1e-17)


def test_axis_aligned_fibers_tensor_structure():
    """theta = 0, Z = 0:  K = s_l K1x(x)M1y + s_t M1x(x)K1y with 1D Q1 matrices."""
    nx, ny, L = 5, 4, (1.0, 0.8)
    lv = level(2, (nx, ny), s_t=2.5e-4, s_l0=1e-3, th0=0.0, L=list(L))
    _, kst = O.assemble(lv, np.zeros(lv.cells))

    def k1m1(n, length):
        h = length / n
        K1 = np.zeros((n + 1, n + 1)); M1 = np.zeros((n + 1, n + 1))
        for e in range(n):
            K1[e:e + 2, e:e + 2] += np.array([[1, -1], [-1, 1]]) / h
            M1[e:e + 2, e:e + 2] += np.array([[2, 1], [1, 2]]) * h / 6
        return K1, M1
    Kx, Mx = k1m1(nx, L[0]); Ky, My = k1m1(ny, L[1])
    K_ref = 1e-3 * np.kron(My, Kx) + 2.5e-4 * np.kron(Ky, Mx)
    np.testing.assert_allclose(dense_K(lv, kst), K_ref, atol=1e-18)
    # rotating the fibers by 90 degrees swaps the roles of x and y
    lv90 = level(2, (nx, ny), s_t=2.5e-4, s_l0=1e-3, th0=90.0, L=list(L))
    _, k90 = O.assemble(lv90, np.zeros(lv90.cells))
    K90 = 2.5e-4 * np.kron(My, Kx) + 1e-3 * np.kron(Ky, Mx)
    np.testing.assert_allclose(dense_K(lv90, k90), K90, atol=1e-17)


@pytest.mark.parametrize("dim", [2, 3])
def test_cosine_mode_implicit_euler_exact(dim):
    """c = 0, D = I: nodal cos(pi x)cos(pi y)(cos(pi z)) is an eigenvector of
    M_L^{-1} K with eigenvalue dim-sum of 2 kappa mu^(dim-1) per axis,
    kappa = 2(1-cos pi h)/h^2, mu = (2 + cos pi h)/3, so each implicit-Euler
    step divides it by (1 + dt lambda_h)."""
    n = 8
    m, T = 5, 0.05
    lv = level(dim, (n,) * dim, m=m, T=T, c=0.0)
    h = 1.0 / n
    x = np.arange(n + 1) * h
    v1 = np.cos(math.pi * x)
    u0 = v1
    for _ in range(dim - 1):
        u0 = np.kron(v1, u0)
    kappa = 2 * (1 - math.cos(math.pi * h)) / h ** 2
    mu = (2 + math.cos(math.pi * h)) / 3
    lam_h = dim * kappa * mu ** (dim - 1)
    slab, _, _ = O.solve_sample(lv, np.zeros(lv.cells), u0=u0)
    for k in range(m + 1):
        np.testing.assert_allclose(slab[k], u0 / (1 + (T / m) * lam_h) ** k, atol=1e-13)


def test_stimulus_nodes():
    lv = O.make_level(2, (32, 32), 64, (1, 1), 5.0, 100, 0.1, 2.5e-4, 1e-3, 30.0)
    u0 = O.initial(lv).reshape(33, 33)
    # nodes (i, j) with i^2 + j^2 < (0.1 * 32)^2 = 10.24
    expect = np.array([[1.0 if i * i + j * j <= 10 else 0.0 for i in range(33)] for j in range(33)])
    assert np.array_equal(u0, expect) and u0.sum() == 13


@pytest.mark.parametrize("dim,ns", [(2, (4, 8, 16, 32)), (3, (4, 8, 16))])
def test_spatial_convergence_rate_against_the_heat_equation(dim, ns):
    """Manufactured solution: with c = 0 and D = I, u = exp(-dim pi^2 t)
    prod_d cos(pi x_d) solves u_t = div grad u with Neumann data on the unit
    box.  Implicit Euler with the exact spatial operator maps the mode by
    1 / (1 + dt dim pi^2) per step, so comparing the oracle's slab with that
    factor isolates the spatial error, which for Q1 with lumped mass must
    fall as h^2 (ratio 4 per halving)."""
    m, T = 10, 0.05
    dt = T / m
    errs = []
    for n in ns:
        lv = level(dim, (n,) * dim, m=m, T=T, c=0.0)
        x = np.arange(n + 1) / n
        v1 = np.cos(math.pi * x)
        u0 = v1
        for _ in range(dim - 1):
            u0 = np.kron(v1, u0)
        slab, _, _ = O.solve_sample(lv, np.zeros(lv.cells), u0=u0)
        exact = u0 / (1 + dt * dim * math.pi ** 2) ** m
        errs.append(np.abs(slab[m] - exact).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.8 < r < 4.2 for r in ratios[1:]), (errs, ratios)
    assert 3.5 < ratios[0] < 4.5, (errs, ratios)


@pytest.mark.parametrize("dim,n", [(2, (6, 5)), (3, (4, 3, 3))])
def test_each_coupling_pair_is_symmetric_and_out_of_domain_couplings_are_zero(dim, n):
    """The coupling of node A to offset o equals the coupling of node A + o to
    offset -o (to rounding: the quadrature here multiplies the gradient
    factors of (a, b) and (b, a) in different orders), and an offset that
    leaves the domain carries exactly zero -- the two facts that let the 3D
    global-memory sweeps store each pair once and read the partner's entry."""
    rng = np.random.default_rng(11)
    L = [1.0, 0.7, 0.4][:dim]
    lv = level(dim, n, s_t=2.5e-4, s_l0=1e-3, th0=30.0, th1=-45.0, L=L)
    _, kst = O.assemble(lv, rng.normal(0, 0.4, lv.cells))
    NO = 3 ** dim
    K = kst.reshape(lv.nodes, NO)
    N = [n[d] + 1 for d in range(dim)] + [1] * (3 - dim)
    for A in range(lv.nodes):
        i, j, k = A % N[0], (A // N[0]) % N[1], A // (N[0] * N[1])
        for o in range(NO):
            dx, dy, dz = o % 3 - 1, (o // 3) % 3 - 1 if dim >= 2 else 0, o // 9 - 1 if dim == 3 else 0
            ii, jj, kk = i + dx, j + dy, k + dz
            if not (0 <= ii < N[0] and 0 <= jj < N[1] and 0 <= kk < N[2]):
                assert K[A, o] == 0.0
                continue
            B = (kk * N[1] + jj) * N[0] + ii
            # rounding of sums of terms of both signs: against the row's scale
            assert abs(K[A, o] - K[B, NO - 1 - o]) <= 1e-15 * np.abs(K[A]).max(), (A, o)
