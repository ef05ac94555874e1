"""Pins of the oracle's nonlinear space-time solve (Sec. 3.3, Eq. mono_disc, in
the implicit-Euler variant): the reaction ODE's closed form and first-order
rate, the all-at-once residual rebuilt independently, the root-selection
rule (a local minimum of the step energy reached by descent), the Newton-CG
direction against a dense solve, and the bistable travelling-wave speed."""
import math

import numpy as np
import pytest

import oracle as O
from helpers import fiber_D, gauss3_assembly


def G_closed(u, a):
    """Antiderivative of 1/(u(1-u)(u-a)) by partial fractions."""
    return -math.log(u) / a - math.log(1 - u) / (1 - a) + math.log(u - a) / (a * (1 - a))


def test_reaction_ode_rate():
    """Spatially uniform state: K 1 = 0, so each node follows the implicit-Euler
    discretisation of u' = c u (1-u)(u-a); the activation time converges to
    t* = (G(1/2) - G(u0))/c at first order in dt."""
    c, a, u0 = 100.0, 0.1, 0.2
    tstar = (G_closed(0.5, a) - G_closed(u0, a)) / c
    errs = []
    for m in (50, 100, 200, 400):
        lv = O.make_level(2, (2, 2), m, (1, 1), 0.2, c, a, 2.5e-4, 1e-3, 30.0)
        slab, t, _ = O.solve_sample(lv, np.zeros(lv.cells), u0=np.full(lv.nodes, u0))
        assert np.ptp(t) < 1e-12
        errs.append(abs(t[0] - tstar))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(1.7 < r < 2.3 for r in ratios), (errs, ratios)
    assert errs[-1] < 1e-2 * tstar


def independent_operators(lv, Z):
    """Lumped mass and stiffness rebuilt with 3-point Gauss quadrature."""
    dim = lv.dim
    n = [lv.n[d] for d in range(dim)]
    L = [lv.L[d] for d in range(dim)]
    D = fiber_D(dim, n, L, lv.theta0, lv.theta1, lv.s_t, lv.s_l0, Z)
    K = gauss3_assembly(dim, n, L, D)
    h = [L[d] / n[d] for d in range(dim)]
    N = [n[d] + 1 for d in range(dim)]
    idx = np.indices(N[::-1]).reshape(dim, -1)[::-1]     # x fastest
    ncell = np.ones(lv.nodes)
    for d in range(dim):
        ncell *= np.where((idx[d] == 0) | (idx[d] == n[d]), 1.0, 2.0)
    mass = np.prod(h) * ncell / 2 ** dim
    return mass, K


def independent_residual(lv, Z, slab):
    mass, K = independent_operators(lv, Z)
    dt = lv.T / lv.m
    F = []
    for k in range(1, lv.m + 1):
        u, up = slab[k], slab[k - 1]
        F.append(mass / dt * (u - up) + K @ u - mass * lv.c * u * (1 - u) * (u - lv.a))
    return np.array(F), mass, K


@pytest.mark.parametrize("dim,n,m,T", [(2, (12, 12), 12, 5.0), (2, (10, 14), 40, 3.0),
                                       (3, (4, 4, 2), 6, 5.0)])
def test_solution_is_root_and_local_minimum(dim, n, m, T):
    rng = np.random.default_rng(5)
    L = (1.0, 1.0) if dim == 2 else (1.0, 1.0, 0.25)
    lv = O.make_level(dim, n, m, L, T, 100.0, 0.1, 2.5e-4, 1e-3, 30.0,
                      theta1=(-60.0 if dim == 3 else None), stim_r=0.45)
    Z = rng.normal(0, 0.3, lv.cells)
    slab, t, per = O.solve_sample(lv, Z)
    F, mass, K = independent_residual(lv, Z, slab)
    assert np.abs(F / mass).max() < 1e-9
    # the all-at-once residual of the oracle agrees with the rebuilt one
    mo, ko = O.assemble(lv, Z)
    np.testing.assert_allclose(O.slab_residual(lv, mo, ko, slab), F, atol=1e-14)
    # each step is a local minimum of its step energy (Hessian positive definite)
    dt = lv.T / lv.m
    for k in range(1, lv.m + 1):
        u = slab[k]
        rp = lv.c * (-3 * u * u + 2 * (1 + lv.a) * u - lv.a)
        H = K + np.diag(mass / dt - mass * rp)
        assert np.linalg.eigvalsh(H).min() > 0.0, k
    assert t.min() == 0.0 and t.max() <= lv.T


def test_rebuilt_slab_system_block_structure():
    """C u + r(u) = f with C block lower-bidiagonal (A on, -M/dt below)."""
    import scipy.sparse as sp
    lv = O.make_level(2, (6, 6), 5, (1, 1), 1.0, 100.0, 0.1, 2.5e-4, 1e-3, 30.0, stim_r=0.4)
    Z = np.zeros(lv.cells)
    slab, _, _ = O.solve_sample(lv, Z)
    mass, kst = O.assemble(lv, Z)
    F, massi, K = independent_residual(lv, Z, slab)
    dt = lv.T / lv.m
    A = sp.csr_matrix(np.diag(massi / dt) + K)
    B = sp.csr_matrix(-np.diag(massi / dt))
    m, n = lv.m, lv.nodes
    blocks = [[A if i == j else (B if i == j + 1 else None) for j in range(m)] for i in range(m)]
    Cm = sp.bmat(blocks).tocsr()
    u = slab[1:].ravel()
    f = np.zeros(m * n)
    f[:n] = massi / dt * slab[0]
    r = -np.tile(massi, m) * lv.c * u * (1 - u) * (u - lv.a)
    res = Cm @ u + r - f
    np.testing.assert_allclose(res.reshape(m, n), O.slab_residual(lv, mass, kst, slab), atol=1e-14)
    assert np.abs(res).max() < 1e-12


def test_newton_cg_direction_spd_matches_dense_solve():
    rng = np.random.default_rng(6)
    lv = O.make_level(2, (9, 7), 400, (1, 1), 1.0, 100.0, 0.1, 2.5e-4, 1e-3, 30.0)
    Z = rng.normal(0, 0.3, lv.cells)
    mass, kst = O.assemble(lv, Z)
    u = rng.random(lv.nodes)
    up = rng.random(lv.nodes)
    F = O.step_residual(lv, mass, kst, u, up)
    d, it, tr = O.newton_cg(lv, mass, kst, u, F)
    massi, K = independent_operators(lv, Z)
    dt = lv.T / lv.m
    rp = lv.c * (-3 * u * u + 2.2 * u - 0.1)
    H = K + np.diag(massi / dt - massi * rp)
    assert np.linalg.eigvalsh(H).min() > 0 and not tr
    np.testing.assert_allclose(d, np.linalg.solve(H, -F), rtol=1e-9, atol=1e-14)


def test_newton_cg_truncates_to_descent_direction():
    rng = np.random.default_rng(7)
    lv = O.make_level(2, (9, 7), 8, (1, 1), 5.0, 100.0, 0.1, 2.5e-4, 1e-3, 30.0)
    mass, kst = O.assemble(lv, np.zeros(lv.cells))
    u = np.full(lv.nodes, 0.3) + 0.01 * rng.random(lv.nodes)    # inside the fold: H indefinite
    F = O.step_residual(lv, mass, kst, u, np.zeros(lv.nodes))
    d, it, tr = O.newton_cg(lv, mass, kst, u, F)
    assert tr and F @ d < 0


def test_deterministic():
    lv = O.make_level(2, (16, 16), 32, (1, 1), 5.0, 100.0, 0.1, 2.5e-4, 1e-3, 30.0, stim_r=0.3)
    Z = O.kl_field(2, [1, 1], [16, 16], 0.04, 0.2, 16, O.xi(0, 0, 3, 16))[0]
    a = O.solve_sample(lv, Z)[0]
    b = O.solve_sample(lv, Z)[0]
    assert np.array_equal(a, b)


def test_travelling_wave_speed():
    """Bistable front speed sqrt(c D / 2)(1 - 2a) as h, dt -> 0 (1D strip)."""
    c, a, D = 100.0, 0.1, 1e-3
    lv = O.make_level(2, (800, 1), 1500, (0.4, 0.0005), 1.5, c, a, D, D, 0.0, stim_r=0.1)
    slab, t, _ = O.solve_sample(lv, np.zeros(lv.cells))
    x = np.arange(801) * 0.0005
    i1, i2 = np.searchsorted(x, 0.2), np.searchsorted(x, 0.3)
    v = (x[i2] - x[i1]) / (t[i2] - t[i1])
    v_theory = math.sqrt(c * D / 2) * (1 - 2 * a)
    assert abs(v / v_theory - 1) < 0.03, (v, v_theory)
