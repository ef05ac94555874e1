"""Pins of the oracle's activation-time QoI, grid transfer and the MC / MLMC
estimators (Sec. 3.1.2, Eq. MC-estimator and Eq. MLMC-estimator)."""
import math

import numpy as np

import oracle as O
from helpers import oracle_level, oracle_levels, small_workload


def test_activation_on_linear_ramps():
    m, T = 10, 5.0
    dt = T / m
    nodes = 5
    slopes = np.array([0.05, 0.2, 0.11, 0.0, 1.0])           # u(t) = slope * t
    slab = np.array([slopes * k * dt for k in range(m + 1)])
    slab[0, 4] = 0.7                                           # already active at t = 0
    t = O.activation(nodes, m, dt, T, slab)
    expect = [0.5 / 0.05 if 0.5 / 0.05 <= T else T, 0.5 / 0.2, 0.5 / 0.11, T, 0.0]
    np.testing.assert_allclose(t, expect, rtol=1e-14)
    # crossing exactly at a grid time is reported at that time
    slab2 = np.array([[0.1 * k] for k in range(m + 1)])
    assert O.activation(1, m, dt, T, slab2)[0] == 5 * dt
    # only the first crossing counts
    slab3 = np.array([[0.0], [0.6], [0.2], [0.9]] + [[0.9]] * (m - 3))
    assert math.isclose(O.activation(1, m, dt, T, slab3)[0], dt * 0.5 / 0.6)


def test_injection_picks_shared_vertices():
    w = small_workload(n0=(4, 4), levels=3)
    lvs = oracle_levels(w)
    for l in (0, 1, 2):
        lv = lvs[l]
        N = lv.n[0] + 1
        x = np.arange(N) / lv.n[0]
        f = (x[None, :] + 2 * x[:, None] ** 2).ravel()
        x0 = np.arange(5) / 4
        np.testing.assert_array_equal(O.inject(lv, lvs[0], f), (x0[None, :] + 2 * x0[:, None] ** 2).ravel())
    w3 = small_workload(dim=3, n0=(2, 2, 1), levels=2, M=8, ell=0.1)
    l3 = oracle_levels(w3)
    f = np.arange(l3[1].nodes, dtype=float)
    g = O.inject(l3[1], l3[0], f)
    # node (i,j,k) of level 0 is node (2i,2j,2k) of level 1 (5 x 5 x 3 grid)
    for k in range(2):
        for j in range(3):
            for i in range(3):
                assert g[(k * 3 + j) * 3 + i] == (2 * k * 5 + 2 * j) * 5 + 2 * i


def test_welford_matches_two_pass():
    rng = np.random.default_rng(8)
    Y = rng.normal(3.0, 2.0, (257, 11)) + 1e6
    w = O.Welford(11)
    for r in Y:
        w.add(r)
    assert w.n == 257
    np.testing.assert_allclose(w.mean, Y.mean(0), rtol=1e-15)
    np.testing.assert_allclose(w.var(), Y.var(0, ddof=1), rtol=1e-9)


def test_pair_shares_xi_and_level0_is_plain():
    """The coarse member of a level pair is the standalone coarse solve with the
    same xi; on level 0 the pair difference is the injected map itself."""
    w = small_workload(n0=(4, 4), m0=4, levels=2, M=8, stim_r=0.45)
    lvs = oracle_levels(w)
    y, y2, _ = O.sample_pair(lvs[1], lvs[0], lvs[0], w["sigma2"], w["ell"], w["M"], 5, 1, 3)
    xi = O.xi(5, 1, 3, w["M"])
    t = []
    for l in (1, 0):
        Z = O.kl_field(2, [1, 1], [lvs[l].n[0], lvs[l].n[1]], w["sigma2"], w["ell"], w["M"], xi)[0]
        t.append(O.inject(lvs[l], lvs[0], O.solve_sample(lvs[l], Z)[1]))
    np.testing.assert_array_equal(y, t[0] - t[1])
    np.testing.assert_array_equal(y2, t[0] ** 2 - t[1] ** 2)
    y0, y20, _ = O.sample_pair(lvs[0], None, lvs[0], w["sigma2"], w["ell"], w["M"], 5, 0, 3)
    xi0 = O.xi(5, 0, 3, w["M"])
    Z0 = O.kl_field(2, [1, 1], [4, 4], w["sigma2"], w["ell"], w["M"], xi0)[0]
    np.testing.assert_array_equal(y0, O.solve_sample(lvs[0], Z0)[1])


def test_mlmc_unbiased_against_brute_force_mc():
    """The MLMC estimate of E[t_L] and a plain MC estimate on level L agree within
    the sum of their standard errors (fixed seeds, CLT bound)."""
    w = small_workload(n0=(4, 4), m0=16, levels=2, M=8, stim_r=0.3, s_l0=0.02, s_t=0.005,
                       sigma2=0.25, T=1.5)
    lvs = oracle_levels(w, newton_max=500)
    est = O.mlmc_estimate(lvs, w["sigma2"], w["ell"], w["M"], 1, [160, 40], threads=4)
    # plain MC on level 1 with its own (independent) stream: level-pair index 7
    T1 = []
    for i in range(200):
        xi = O.xi(99, 7, i, w["M"])
        Z = O.kl_field(2, [1, 1], [8, 8], w["sigma2"], w["ell"], w["M"], xi)[0]
        T1.append(O.inject(lvs[1], lvs[0], O.solve_sample(lvs[1], Z)[1]))
    T1 = np.array(T1)
    se_mc = T1.std(0, ddof=1) / math.sqrt(200)
    se_ml = np.sqrt(est["var_l"][0] / 160 + est["var_l"][1] / 40)
    z = np.abs(est["mean"] - T1.mean(0)) / np.maximum(np.sqrt(se_mc ** 2 + se_ml ** 2), 1e-12)
    active = (se_mc > 0)
    assert active.sum() > 5
    assert z[active].max() < 4.5
    # the estimator's own bookkeeping
    assert math.isclose(est["rmse"] ** 2,
                        est["V_l"][0] / 160 + est["V_l"][1] / 40 + est["bias"] ** 2, rel_tol=1e-12)
    assert np.all(est["var"] >= 0)
