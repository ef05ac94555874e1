"""Pins of the root the oracle's step solver selects (Sec. 3.3, Eq. mono_disc,
implicit-Euler blocks).

When c dt max r' > 1 an implicit-Euler step has several roots.  The root is
defined without reference to any solver: the end point of the gradient flow
M v' = -F_k(v) of the step energy started at u_{k-1} -- the local minimum in
whose basin of attraction u_{k-1} lies -- integrated by fixed-length,
strictly convex implicit-Euler pseudo-steps (``O.step_gradient_flow``).  The
oracle's fast step solver (``O.step_solve``: a gradient-flow continuation by
linearly implicit pseudo-steps with adaptive length) must land on that root
from the same u_{k-1}, on every step of many samples of the workload levels
where the roots are not unique.  A one-ulp perturbation of the field must not
change the selected root either.
"""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle as O
from helpers import oracle_level
from paper_1911_06066_gb300 import workloads as W

THREADS = max(1, O.cores())


def _field(w, level, i, seed=0):
    n, _ = W.level_shape(w, level)
    return O.kl_field(w["dim"], w["L"], n, w["sigma2"], w["ell"], w["M"],
                      O.xi(seed, level, i, w["M"]))[0]


def _compare_steps(args):
    w, level, i, steps = args
    lv = oracle_level(w, level)
    Z = _field(w, level, i)
    mass, kst = O.assemble(lv, Z)
    u = O.initial(lv)
    worst, pseudo = 0.0, 0
    for k in range(1, steps + 1):
        un, _ = O.step_solve(lv, mass, kst, u)
        ugf, st = O.step_gradient_flow(lv, mass, kst, u)
        worst = max(worst, float(np.abs(un - ugf).max()))
        pseudo += st["pseudo"]
        u = un
    return i, worst, pseudo


def _multi_root(w, level):
    lv = oracle_level(w, level)
    return lv.c * ((1 + lv.a) ** 2 / 3 - lv.a) * lv.T / lv.m


@pytest.mark.parametrize("name,level,samples,steps", [
    ("2d", 0, 16, 64),      # 32^2, 64 steps (all): c dt max r' = 2.37
    ("2d", 1, 16, 16),      # 64^2, first 16 of 128 steps: c dt max r' = 1.18
    ("3d", 0, 16, 2),       # 32x32x8, first 2 of 32 steps: c dt max r' = 4.74
])
def test_step_solver_lands_on_the_gradient_flow_root(name, level, samples, steps):
    w = W.MLMC2D_3LVL if name == "2d" else W.SLAB3D_4LVL
    assert _multi_root(w, level) > 1.0           # several roots exist on these levels
    jobs = [(w, level, i, steps) for i in range(samples)]
    with cf.ThreadPoolExecutor(THREADS) as ex:
        res = list(ex.map(_compare_steps, jobs))
    worst = max(r[1] for r in res)
    assert worst <= 1e-9, res
    # the flow passes near saddles on these levels (many pseudo-steps), so
    # the agreement is not the trivial one of a unique root
    assert max(r[2] for r in res) > 20 * steps


def test_gradient_flow_root_does_not_depend_on_the_pseudo_step():
    """The reference is the flow's end point, not an artefact of its step
    length: tau and tau / 4 reach the same minimum on a step where the flow
    lingers near a saddle (sample 0, step 10 of the 32^2 level, where a
    Newton-CG iteration with a step limit reaches a different minimum)."""
    w = W.MLMC2D_3LVL
    lv = oracle_level(w, 0)
    Z = _field(w, 0, 0)
    mass, kst = O.assemble(lv, Z)
    slab, _, _ = O.solve_sample(lv, Z)
    s = lv.c * ((1 + lv.a) ** 2 / 3 - lv.a) - lv.m / lv.T
    u1, st1 = O.step_gradient_flow(lv, mass, kst, slab[9], tau=0.5 / s)
    u4, st4 = O.step_gradient_flow(lv, mass, kst, slab[9], tau=0.125 / s)
    assert np.abs(u1 - u4).max() <= 1e-10
    assert st4["pseudo"] > 3 * st1["pseudo"]
    np.testing.assert_allclose(u1, slab[10], atol=1e-9)


def test_gradient_flow_root_is_a_local_minimum_not_the_lowest_one():
    """The selected root is a local minimum of the step energy with positive
    definite Hessian; it need not be the global one (a step of this length
    could lower the energy by activating more nodes), which is why the
    definition is the basin of u_{k-1} and not the energy minimiser."""
    w = W.MLMC2D_3LVL
    lv = oracle_level(w, 0)
    Z = _field(w, 0, 0)
    mass, kst = O.assemble(lv, Z)
    slab, _, _ = O.solve_sample(lv, Z)
    dt = lv.T / lv.m
    u, up = slab[10], slab[9]
    rp = lv.c * (-3 * u * u + 2 * (1 + lv.a) * u - lv.a)
    from helpers import dense_K
    H = dense_K(lv, kst) + np.diag(mass / dt - mass * rp)
    assert np.linalg.eigvalsh(H).min() > 0.0

    def energy(v):
        R = lv.c * (-v ** 4 / 4 + (1 + lv.a) * v ** 3 / 3 - lv.a * v ** 2 / 2)
        return np.sum(mass * (v - up) ** 2) / (2 * dt) + 0.5 * v @ O.stiff_apply(lv, kst, v) - np.sum(mass * R)

    # activating one more node at the front gives a deeper minimum of the same
    # step: the flow from the selected root with that node set to 1 settles
    # at another root whose energy is lower
    N0 = lv.n[0] + 1
    act = u >= 0.5
    front = [i for i in range(lv.nodes) if not act[i] and
             any(0 <= j < lv.nodes and act[j] for j in (i - 1, i + 1, i - N0, i + N0))]
    assert front
    start = u.copy()
    start[front[0]] = 1.0
    v, _ = O.step_gradient_flow(lv, mass, kst, up, v0=start)
    F = O.step_residual(lv, mass, kst, v, up)
    lower = np.abs(F / mass).max() < 1e-9 and energy(v) < energy(u) - 1e-6 and (v >= 0.5).sum() > act.sum()
    assert lower


@pytest.mark.parametrize("name,level,samples,steps", [("2d", 0, 64, 64), ("3d", 0, 4, 16)])
def test_selected_root_is_insensitive_to_one_ulp_in_the_field(name, level, samples, steps):
    """The continuation never jumps between basins, so rounding-level changes
    of the problem leave the selected roots where they are (all 64 steps of
    64 samples of the 32^2 level; the first 16 of 32 steps of 4 samples of the
    32x32x8 level)."""
    w = W.MLMC2D_3LVL if name == "2d" else W.SLAB3D_4LVL
    lv = oracle_level(w, level)

    def states(Z):
        mass, kst = O.assemble(lv, Z)
        u = O.initial(lv)
        out = []
        for _ in range(steps):
            u, _ = O.step_solve(lv, mass, kst, u)
            out.append(u)
        return np.array(out)

    def one(i):
        Z = _field(w, level, i)
        return float(np.abs(states(Z) - states(np.nextafter(Z, np.inf))).max())

    with cf.ThreadPoolExecutor(THREADS) as ex:
        diffs = list(ex.map(one, range(samples)))
    assert max(diffs) <= 1e-9, diffs
