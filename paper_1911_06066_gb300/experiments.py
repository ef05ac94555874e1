"""Experiments of the paper run through the C ABI (no arithmetic of the method
here: every sample is solved and accumulated by the library).

* controlled_convergence_1d: the 1D+1 controlled-convergence experiment of
  Sec. 4.1 (Table 1d-levels, Fig. Controlled-Convergence-1D): an interval with
  n_l = 31 2^l cells and m_l = 4 2^l Crank-Nicolson steps over T = 0.64
  (dt_l = 0.16 2^-l), l = 0..5; a reference mean from 20,000 samples on the
  finest level; plain MC on level l with N_l = 2^(4l) samples; MLMC with fine
  level L, N_0 = 2^(4L) and the ideal sampling ratio 16 between levels; the
  RMSE of each estimator against the reference in the L2(D) norm of the
  coarsest grid at the final time (the paper's space-time norm needs the whole
  slab; the final state is the quantity the library estimates), averaged
  over independent repetitions.
* work_report: the work model of Sec. 4.2 from measured per-sample costs:
  gamma_d = log2(W'_{l+1} / W'_l) (Eq. complexity), W_l = W'_{l-1} + W'_l,
  W_MC,L = W'_L N_L and W_MLMC,L = sum_l W_l N_l (Eq. work), and the
  asymptotic forms 2^((gamma d + 4) L) and Eq. Work-MLMC.
"""
import math

import numpy as np

# The 1D+1 problem: the stochastic heat equation (Eq. stochastic-heat; no
# reaction) with the paper's affine KL conductivity (at most 16 modes; the
# factor stops once the remainder trace is 1e-10 of the covariance's -- the
# Gaussian kernel's spectrum decays so fast that further columns would only
# carry rounding), a forcing held on for the whole interval, u(x, 0) = 0, and
# the final state as quantity of interest.
HEAT1D_6LVL = dict(
    name="heat1d_cc_31-992_m4-128_affineKL",
    dim=1, L=(1.0,), n0=(31,), m0=4, levels=6, T=0.64,
    c=0.0, a=0.0, s_t=0.1, s_l0=0.1, theta0=0.0, theta1=0.0,
    stim_r=0.0, stim_c=(0.3, 0.0, 0.0), sigma2=1.0, ell=0.5, M=16, N=[1] * 6, seed=0,
    scheme=1, stim_kind=1, stim_amp=1.0, stim_sigma=0.15, stim_t1=0.64, qoi=1,
    kl_kind=1, kl_tol=1e-10, kl_s=0.3, kl_delta=0.5, kl_cand_n=(248, 0, 0))


def _weights(n0):
    """Lumped mass of the coarsest 1D grid (trapezoid weights)."""
    h = 1.0 / n0
    w = np.full(n0 + 1, h)
    w[0] = w[-1] = 0.5 * h
    return w


def controlled_convergence_1d(B, w=HEAT1D_6LVL, reps=4, n_ref=20000, mc_levels=4, mlmc_levels=5,
                              precision=None, seed=0, batch=4096):
    """Runs the experiment; returns a dict of RMSEs per level for MC and MLMC."""
    precision = B.MLMC_PREC_FP64 if precision is None else precision
    wts = _weights(w["n0"][0])
    # every context below shares the random field: the same candidate grid
    # for the pivoted Cholesky, the same (seed, level, id) -> psi map
    def one_level(l):
        return dict(w, n0=(w["n0"][0] * 2 ** l,), m0=w["m0"] * 2 ** l, levels=1)

    # reference: the plain MC mean of n_ref samples on the finest level
    ref_ctx = B.Context(B.make_config(one_level(w["levels"] - 1), precision))
    r = ref_ctx.run([n_ref], seed=seed + 10 ** 6, batch=min(batch, n_ref))
    stride = 2 ** (w["levels"] - 1)
    v_ref = r["mean"][::stride]
    out = {"workload": w["name"], "reference_samples": n_ref, "reps": reps, "mc": [], "mlmc": []}

    def rmse_of(means):
        e2 = [float(np.sum(wts * (m - v_ref) ** 2)) for m in means]
        return math.sqrt(sum(e2) / len(e2))

    for l in range(mc_levels):
        ctx = B.Context(B.make_config(one_level(l), precision))
        N = 2 ** (4 * l)
        means = []
        for k in range(reps):
            rr = ctx.run([N], seed=seed + 1000 * (k + 1) + l, batch=min(batch, N))
            means.append(rr["mean"][::2 ** l])
        out["mc"].append({"level": l, "N": N, "rmse": rmse_of(means)})
    for L in range(mlmc_levels):
        ctx = B.Context(B.make_config(dict(w, levels=L + 1), precision))
        N = [max(1, 2 ** (4 * L) // 16 ** l) for l in range(L + 1)]
        means = []
        for k in range(reps):
            rr = ctx.run(N, seed=seed + 7919 * (k + 1) + L, batch=min(batch, max(N)))
            means.append(rr["mean"])
        out["mlmc"].append({"L": L, "N_l": N, "rmse": rmse_of(means)})
    for key in ("mc", "mlmc"):
        e = [x["rmse"] for x in out[key]]
        out[key + "_rate_per_level"] = [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)
                                        if e[i + 1] > 0]
    return out


def work_report(W_prime, N_l=None, ratio=16.0):
    """Sec. 4.2's work model from measured per-sample costs W'_l (seconds).
    Returns gamma_d per level step, W_l, W_MC and W_MLMC for the counts N_l
    (default: the ideal ratio from one fine sample), and the asymptotic work
    for the mean gamma_d."""
    Wp = np.asarray(W_prime, float)
    L = len(Wp) - 1
    gd = [math.log2(Wp[l + 1] / Wp[l]) for l in range(L) if Wp[l] > 0 and Wp[l + 1] > 0]
    Wl = Wp + np.concatenate([[0.0], Wp[:-1]])
    if N_l is None:
        N_l = [ratio ** (L - l) for l in range(L + 1)]
    N_l = np.asarray(N_l, float)
    g = float(np.mean(gd)) if gd else float("nan")

    def w_mlmc_asym(Lf):
        if abs(g - 4.0) < 1e-9:
            return Lf * 2.0 ** (4 * Lf)
        return (2.0 ** (g * Lf) - 2.0 ** (4 * Lf)) / (2.0 ** (g - 4) - 1.0)

    return {"W_prime_l": Wp.tolist(), "gamma_d_l": gd, "gamma_d": g, "W_l": Wl.tolist(),
            "N_l": N_l.tolist(), "W_MC": float(Wp[-1] * N_l[0]),
            "W_MLMC": float(np.sum(Wl * N_l)),
            "asymptotic": {"W_MC": 2.0 ** ((g + 4) * L), "W_MLMC": w_mlmc_asym(L),
                           "L": L}}


if __name__ == "__main__":
    # python -m paper_1911_06066_gb300.experiments [reps]: the full 1D+1
    # controlled-convergence experiment on cuda:0, one JSON line
    import json
    import sys
    import time

    from . import binding as _B
    from . import build as _build
    _build.build()
    t0 = time.perf_counter()
    res = controlled_convergence_1d(_B, reps=int(sys.argv[1]) if len(sys.argv) > 1 else 4)
    res["seconds"] = time.perf_counter() - t0
    print(json.dumps(res))
