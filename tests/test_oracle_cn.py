"""Pins of the oracle's Crank-Nicolson blocks and applied-current stimulus
(the paper's own discretisation, Sec. 3.2 Eq. st-system / Eq. system_C and
Sec. 3.3 Eq. mono_disc; the set-up of Sec. 4):

* a discrete cosine mode of the heat equation decays by exactly
  (1 - dt lambda_h / 2) / (1 + dt lambda_h / 2) per step;
* that decay is second-order accurate in time (errors fall 4x per halving of
  dt), where implicit Euler's fall 2x;
* the sequential solve satisfies the all-at-once system C u + r(u) = f rebuilt
  independently with A = M/dt + K/2 on the diagonal and B = -M/dt + K/2 below;
* the first step of a pure-diffusion problem driven by the pulse equals the
  dense solve of (M/dt + K/2) u_1 = M s_1, s_1 the current's exact step average;
* the step energy's gradient is the Crank-Nicolson residual."""
import math

import numpy as np
import pytest

import oracle as O
from helpers import dense_K, fiber_D, gauss3_assembly


def cn_level(dim, n, m, T, c=0.0, **kw):
    L = [1.0] * dim
    return O.make_level(dim, n, m, L, T, c, 0.1, 1.0, 1.0, 0.0, scheme=1, **kw)


def cosine(dim, n):
    x = np.arange(n + 1) / n
    v1 = np.cos(math.pi * x)
    u = v1
    for _ in range(dim - 1):
        u = np.kron(v1, u)
    return u


def lam_h(dim, n):
    h = 1.0 / n
    kappa = 2 * (1 - math.cos(math.pi * h)) / h ** 2
    mu = (2 + math.cos(math.pi * h)) / 3
    return dim * kappa * mu ** (dim - 1)


@pytest.mark.parametrize("dim", [2, 3])
def test_cosine_mode_crank_nicolson_exact(dim):
    n, m, T = 8, 5, 0.05
    lv = cn_level(dim, (n,) * dim, m, T)
    u0 = cosine(dim, n)
    slab, _, _ = O.solve_sample(lv, np.zeros(lv.cells), u0=u0)
    dt, lh = T / m, lam_h(dim, n)
    g = (1 - dt * lh / 2) / (1 + dt * lh / 2)
    for k in range(m + 1):
        np.testing.assert_allclose(slab[k], u0 * g ** k, atol=1e-13)


def test_crank_nicolson_is_second_order_in_time():
    n, T = 8, 0.1
    u0 = cosine(2, n)
    exact = math.exp(-lam_h(2, n) * T)
    errs = {0: [], 1: []}
    for scheme in (0, 1):
        for m in (4, 8, 16, 32):
            lv = O.make_level(2, (n, n), m, (1, 1), T, 0.0, 0.1, 1.0, 1.0, 0.0, scheme=scheme)
            slab, _, _ = O.solve_sample(lv, np.zeros(lv.cells), u0=u0)
            errs[scheme].append(abs(slab[m][0] / u0[0] - exact))
    cn = [errs[1][i] / errs[1][i + 1] for i in range(3)]
    ie = [errs[0][i] / errs[0][i + 1] for i in range(3)]
    assert all(3.8 < r < 4.2 for r in cn), cn
    assert all(1.8 < r < 2.2 for r in ie), ie


def test_all_at_once_crank_nicolson_system():
    import scipy.sparse as sp
    rng = np.random.default_rng(4)
    lv = O.make_level(2, (6, 6), 6, (1, 1), 1.0, 18.5, 0.2435, 3e-3, 3e-3, 0.0, scheme=1,
                      stim_kind=1, stim_amp=40.0, stim_sigma=0.3, stim_t1=0.25)
    Z = rng.normal(0, 0.3, lv.cells)
    slab, _, _ = O.solve_sample(lv, Z)
    assert np.abs(slab[1]).max() > 1e-3          # the pulse did drive the state
    D = fiber_D(2, [6, 6], [1, 1], 0.0, 0.0, 3e-3, 3e-3, Z)
    K = gauss3_assembly(2, [6, 6], [1, 1], D)
    mass, _ = O.assemble(lv, Z)
    dt, m, nn = lv.T / lv.m, lv.m, lv.nodes
    A = sp.csr_matrix(np.diag(mass / dt) + 0.5 * K)
    Bm = sp.csr_matrix(-np.diag(mass / dt) + 0.5 * K)
    C = sp.bmat([[A if i == j else (Bm if i == j + 1 else None) for j in range(m)] for i in range(m)])
    u = slab[1:].ravel()
    # f: the first block row's explicit part and the current's step averages
    xs = np.indices((7, 7))[::-1].reshape(2, -1) / 6.0
    g = 40.0 * np.exp(-(xs ** 2).sum(0) / 0.09)
    f = np.zeros(m * nn)
    f[:nn] = -(Bm @ slab[0])
    for k in range(1, m + 1):
        ov = max(0.0, min(k * dt, 0.25) - (k - 1) * dt)
        f[(k - 1) * nn:k * nn] += mass * g * ov / dt
    r = -np.tile(mass, m) * lv.c * u * (1 - u) * (u - lv.a)
    res = C @ u + r - f
    assert np.abs(res).max() < 1e-12
    np.testing.assert_allclose(res.reshape(m, nn), O.slab_residual(lv, mass, O.assemble(lv, Z)[1], slab),
                               atol=1e-13)


@pytest.mark.parametrize("t1_steps", [0.5, 1.0, 2.5])
def test_pulse_first_step_is_the_dense_solve(t1_steps):
    lv = O.make_level(2, (5, 4), 4, (1, 1), 0.4, 0.0, 0.1, 0.2, 0.2, 0.0, scheme=1,
                      stim_kind=1, stim_amp=3.0, stim_sigma=0.4, stim_t1=0.1 * t1_steps,
                      stim_c=(0.3, 0.6, 0.0))
    Z = np.zeros(lv.cells)
    slab, _, _ = O.solve_sample(lv, Z)
    assert np.array_equal(slab[0], np.zeros(lv.nodes))
    mass, kst = O.assemble(lv, Z)
    K = dense_K(lv, kst)
    dt = 0.1
    x = np.indices((5, 6))[::-1].reshape(2, -1) * np.array([[0.2], [0.25]])
    g = 3.0 * np.exp(-((x[0] - 0.3) ** 2 + (x[1] - 0.6) ** 2) / 0.16)
    s1 = g * min(dt, 0.1 * t1_steps) / dt
    u1 = np.linalg.solve(np.diag(mass / dt) + 0.5 * K, mass * s1)
    np.testing.assert_allclose(slab[1], u1, atol=1e-14)
    np.testing.assert_allclose(O.stimulus_step(lv, 1), s1, atol=1e-15)


def test_final_state_quantity_of_interest():
    lv = O.make_level(2, (6, 6), 5, (1, 1), 0.5, 18.5, 0.2435, 3e-3, 3e-3, 0.0, scheme=1,
                      stim_kind=1, stim_amp=1.0, stim_sigma=0.5, stim_t1=0.1, qoi=1)
    slab, q, _ = O.solve_sample(lv, np.zeros(lv.cells))
    assert np.array_equal(q, slab[-1])


def test_step_energy_gradient_is_the_cn_residual():
    """Finite differences of the step energy E (theta = 1/2) reproduce F_k."""
    rng = np.random.default_rng(2)
    lv = O.make_level(2, (4, 4), 3, (1, 1), 0.3, 18.5, 0.2435, 0.05, 0.08, 20.0, scheme=1,
                      stim_kind=1, stim_amp=2.0, stim_sigma=0.5, stim_t1=0.15)
    Z = rng.normal(0, 0.2, lv.cells)
    mass, kst = O.assemble(lv, Z)
    up, u = rng.random(lv.nodes), rng.random(lv.nodes)
    dt, c, a = lv.T / lv.m, lv.c, lv.a
    s1 = O.stimulus_step(lv, 1)

    def energy(v):
        R = c * (-v ** 4 / 4 + (1 + a) * v ** 3 / 3 - a * v ** 2 / 2)
        return (np.sum(mass * (v - up) ** 2) / (2 * dt) + 0.25 * v @ O.stiff_apply(lv, kst, v)
                + 0.5 * up @ O.stiff_apply(lv, kst, v) - np.sum(mass * (R + s1 * v)))

    F = O.step_residual(lv, mass, kst, u, up, 1)
    h = 1e-6
    g = np.array([(energy(u + h * e) - energy(u - h * e)) / (2 * h) for e in np.eye(lv.nodes)])
    np.testing.assert_allclose(g, F, rtol=1e-6, atol=1e-9)
