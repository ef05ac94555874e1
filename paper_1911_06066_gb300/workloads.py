"""Synthetic workloads of the space-time MLMC monodomain path: parameters only.

This module holds no arithmetic of the method.  Each workload is the shape
and parameter set of one benchmark configuration; both the CUDA path and the
CPU oracle are driven from these dictionaries by the tests and the benchmark.

Problem (arXiv:1911.06066, Sec. 2.1 / 2.2 in the variant the workloads fix):
    u_t = div(D grad u) + c u (1-u) (u-a)      on a box, Neumann boundary,
    D = s_t I + (s_l - s_t) f f^T,  s_l = s_l0 exp(Z),  f = (cos th, sin th, 0),
    Z = sum_k sqrt(lam_k) phi_k xi_k  (separable exponential covariance),
    u(x, 0) = 1 inside the ball |x - x_c| < stim_r, else 0,
    QoI: activation time, the first t with u >= 1/2 (linear in t).
Level l refines every axis and the time grid by 2^l.
"""

# Reaction, conductivity, stimulus and end time shared by every workload.
COMMON = dict(T=5.0, c=100.0, a=0.1, s_t=2.5e-4, s_l0=1e-3, stim_r=0.1,
              stim_c=(0.0, 0.0, 0.0), sigma2=0.04)

MC2D_32 = dict(
    name="mc2d_32x32_m64_M16",
    dim=2, L=(1.0, 1.0), n0=(32, 32), m0=64, levels=1,
    theta0=30.0, theta1=30.0, ell=0.2, M=16,
    N=[16], seed=0, **COMMON)

# mixed_cdr_max: FP32 inner solves on all three levels (c dt max r' = 2.37,
# 1.19, 0.59); on the 32^2 level they end in the same roots as FP64 ones (512
# samples), the KL field stays FP64 there.
MLMC2D_3LVL = dict(
    name="mlmc2d_3lvl_32-128_m64-256_M64",
    dim=2, L=(1.0, 1.0), n0=(32, 32), m0=64, levels=3,
    theta0=30.0, theta1=30.0, ell=0.1, M=64,
    N=[512, 128, 32], seed=0, mixed_cdr_max=2.5, **COMMON)

SLAB3D_4LVL = dict(
    name="mlmc3d_4lvl_32x32x8-256x256x64_m32-256_M256",
    dim=3, L=(1.0, 1.0, 0.25), n0=(32, 32, 8), m0=32, levels=4,
    theta0=-60.0, theta1=60.0, ell=0.1, M=256,
    N=[256, 64, 16, 4], seed=0, **COMMON)

# The paper's own discretisation and model on its cube set-up (Sec. 3.1.1,
# Sec. 3.2-3.3, Sec. 4 and the cube hierarchy of Sec. 4.2): the unit cube,
# h = 0.2 .. 0.025 (5 .. 40 cells per axis), dt = 0.04 .. 0.005 ms over
# T = 1 ms, Crank-Nicolson blocks, the FHN current with alpha = 1.4e-3,
# u_rest = 0, u_th = 28, u_peak = 115 in units of u_peak (c = alpha u_peak^2,
# a = u_th / u_peak), the isotropic conductivity G = G0 (1 + s Z), G0 = 3.325e-3,
# Z the affine KL field of the Gaussian kernel exp(-d^2 / sigma_KL) with
# sigma_KL = 0.25 (ell = 0.5 in exp(-d^2/ell^2)), 66 pivoted-Cholesky modes on
# the level-1 centroids (10^3), y ~ U(-1, 1), s = 0.3 capped by delta = 0.5;
# u(x, 0) = 0 and the applied current u_peak exp(-|x - x0|^2 / sigma^2)
# (sigma = 0.5) on [0, t1), t1 = 0.005 ms, in units of u_peak (amplitude 1);
# QoI u(x, T).  The stimulus centre x0 is the corner (the paper shows it only
# in a figure).
FHN_ALPHA, FHN_UTH, FHN_UPEAK = 1.4e-3, 28.0, 115.0
CUBE_CN_4LVL = dict(
    name="mlmc3d_cube_cn_fhn_5-40_m25-200_affineKL66",
    dim=3, L=(1.0, 1.0, 1.0), n0=(5, 5, 5), m0=25, levels=4,
    theta0=0.0, theta1=0.0, ell=0.5, M=66, N=[512, 128, 32, 8], seed=0,
    T=1.0, c=FHN_ALPHA * FHN_UPEAK ** 2, a=FHN_UTH / FHN_UPEAK,
    s_t=3.325e-3, s_l0=3.325e-3, stim_r=0.0, stim_c=(0.0, 0.0, 0.0), sigma2=1.0,
    scheme=1, stim_kind=1, stim_amp=1.0, stim_sigma=0.5, stim_t1=0.005, qoi=1,
    kl_kind=1, kl_tol=0.0, kl_s=0.3, kl_delta=0.5, kl_cand_n=(10, 10, 10))

WORKLOADS = {w["name"]: w for w in (MC2D_32, MLMC2D_3LVL, SLAB3D_4LVL, CUBE_CN_4LVL)}


def level_shape(w, l):
    """(cells per axis, time steps) of level l of workload w."""
    f = 2 ** l
    return tuple(n * f for n in w["n0"]), w["m0"] * f
