"""Test-side helpers: handle setup through the binding, and initial data built with numpy."""
import numpy as np

import paper_2007_10196_gb300 as P
from paper_2007_10196_gb300 import inputs


def shapes_from_levels(nr, levels):
    return [tuple(int(nr) << int(l) for l in lev) for lev in levels]


def sine_grid(nr, lev, lo, hi, ic, dtype=np.float64):
    """u0 = b + a sin(w sum_k x_k + phi) at the nodes x_k = lo + j (hi-lo)/n_k, flat, axis 0 fastest."""
    b, a, w, phi = ic
    n = [int(nr) << int(l) for l in lev]
    xs = [lo + np.arange(nk) * ((hi - lo) / nk) for nk in n]
    S = sum(np.meshgrid(*xs, indexing="ij"))
    v = b + a * np.sin(w * S + phi)
    return np.ascontiguousarray(v.transpose(tuple(reversed(range(len(n))))).reshape(-1), dtype=dtype)


def random_grids(seed, nr, levels, kind="mixed", scale=1.0, offset=0.0):
    return [offset + scale * inputs.random_field(seed + 17 * g, tuple(int(nr) << int(l) for l in lev), kind)
            for g, lev in enumerate(levels)]


def make(dim, nr, nl, pde, **kw):
    return P.create(dim, nr, nl, pde, **kw)


def read_grids(h, sizes):
    out = P.sg_read(h, P.SG_WHICH_ALL_GRIDS, count=int(sum(sizes)))
    res, off = [], 0
    for s in sizes:
        res.append(out[off:off + s].copy())
        off += s
    return res


def oracle_problem(orc, dim, nr, nl, pde, scheme=0, prolong=0, eps=1e-3, lo=0.0, hi=4.0, adv=1.0):
    return orc.problem(dim, nr, nl, pde=pde, scheme=scheme, prolong=prolong, eps=eps, lo=lo, hi=hi, adv=adv)
