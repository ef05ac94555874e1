"""Shared test helpers: build oracle levels from the workload dictionaries."""
import itertools
import math

import numpy as np

import oracle as O
from paper_1911_06066_gb300 import workloads as W


def oracle_level(w, l, **kw):
    n, m = W.level_shape(w, l)
    for key in ("scheme", "stim_kind", "stim_amp", "stim_sigma", "stim_t1", "qoi"):
        if key in w and key not in kw:
            kw[key] = w[key]
    if w.get("kl_kind", 0) == 1 and "cond_kind" not in kw:
        kw["cond_kind"] = 1
    return O.make_level(w["dim"], n, m, w["L"], w["T"], w["c"], w["a"], w["s_t"], w["s_l0"],
                        w["theta0"], w["theta1"], w["stim_r"], w["stim_c"], **kw)


def oracle_levels(w, **kw):
    return [oracle_level(w, l, **kw) for l in range(w["levels"])]


def small_workload(dim=2, n0=(8, 8), m0=8, levels=2, M=8, ell=0.2, **over):
    """A workload of the same structure, shrunk so the oracle finishes in seconds."""
    base = W.MC2D_32 if dim == 2 else W.SLAB3D_4LVL
    w = dict(base)
    w.update(dict(name="small", n0=tuple(n0), m0=m0, levels=levels, M=M, ell=ell,
                  N=[4] * levels))
    w.update(over)
    return w


def read_golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def dense_K(lv, kst):
    dim = lv.dim
    N = [lv.n[d] + 1 for d in range(dim)] + [1] * (3 - dim)
    nodes = lv.nodes
    no = 3 ** dim
    K = np.zeros((nodes, nodes))
    kst = kst.reshape(nodes, no)
    for A in range(nodes):
        i, j, k = A % N[0], (A // N[0]) % N[1], A // (N[0] * N[1])
        for o in range(no):
            di = o % 3 - 1
            dj = (o // 3) % 3 - 1 if dim >= 2 else 0
            dk = (o // 9 - 1) if dim == 3 else 0
            ii, jj, kk = i + di, j + dj, k + dk
            if 0 <= ii < N[0] and 0 <= jj < N[1] and 0 <= kk < N[2]:
                K[A, (kk * N[1] + jj) * N[0] + ii] += kst[A, o]
            else:
                assert kst[A, o] == 0.0
    return K


def gauss3_assembly(dim, n, L, Dcells):
    """Independent assembly: 3-point Gauss per axis, basis from tensor products."""
    g = np.array([-math.sqrt(0.6), 0.0, math.sqrt(0.6)]) * 0.5 + 0.5
    wg = np.array([5.0, 8.0, 5.0]) / 18.0
    h = [L[d] / n[d] for d in range(dim)]
    N = [n[d] + 1 for d in range(dim)]
    nodes = int(np.prod(N))
    K = np.zeros((nodes, nodes))
    for cell in itertools.product(*[range(n[d]) for d in range(dim)]):
        ci = cell[0] + n[0] * cell[1] + (n[0] * n[1] * cell[2] if dim == 3 else 0)
        D = Dcells[ci]
        loc = list(itertools.product(*[(0, 1)] * dim))
        gl = [cell[0] + a[0] + N[0] * (cell[1] + a[1]) + (N[0] * N[1] * (cell[2] + a[2]) if dim == 3 else 0)
              for a in loc]
        for q in itertools.product(range(3), repeat=dim):
            xi = [g[q[d]] for d in range(dim)]
            w = np.prod([wg[q[d]] for d in range(dim)]) * np.prod(h)
            grads = []
            for a in loc:
                gr = []
                for d in range(dim):
                    v = (1.0 if a[d] else -1.0) / h[d]
                    for e in range(dim):
                        if e != d:
                            v *= xi[e] if a[e] else 1 - xi[e]
                    gr.append(v)
                grads.append(np.array(gr))
            for p_, a in enumerate(loc):
                for q_, b in enumerate(loc):
                    K[gl[p_], gl[q_]] += w * grads[p_] @ D @ grads[q_]
    return K


def fiber_D(dim, n, L, th0, th1, s_t, s_l0, Z):
    """Per-cell conductivity tensors D = s_t I + (s_l - s_t) f f^T."""
    h = [L[d] / n[d] for d in range(dim)]
    out = []
    for ci in range(len(Z)):
        kz = ci // (n[0] * n[1]) if dim == 3 else 0
        th = th0 if dim == 2 else th0 + (th1 - th0) * (kz + 0.5) * h[2] / L[2]
        f = np.array([math.cos(math.radians(th)), math.sin(math.radians(th)), 0.0])[:dim]
        sl = s_l0 * math.exp(Z[ci])
        out.append(s_t * np.eye(dim) + (sl - s_t) * np.outer(f, f))
    return out


def affine_kl(w):
    """The oracle's KL of a workload with the paper's variant (kl_kind 1)."""
    ns = [W.level_shape(w, l)[0] for l in range(w["levels"])]
    cand = tuple(c if c else n for c, n in zip(w["kl_cand_n"][:w["dim"]], w["n0"]))
    return O.AffineKL(w["dim"], w["L"], cand, ns, w["sigma2"], w["ell"], w["M"],
                      w["kl_tol"], w["kl_s"], w["kl_delta"])


def oracle_field(w, level, seed, pair_level, sample_id, akl=None):
    """The oracle's KL field of one sample on `level` (xi / psi drawn for the
    pair `pair_level`), for either KL kind."""
    if w.get("kl_kind", 0) == 1:
        akl = akl or affine_kl(w)
        return akl.field(level, O.psi_uniform(seed, pair_level, sample_id, w["M"]))[0]
    n, _ = W.level_shape(w, level)
    return O.kl_field(w["dim"], w["L"], n, w["sigma2"], w["ell"], w["M"],
                      O.xi(seed, pair_level, sample_id, w["M"]))[0]
