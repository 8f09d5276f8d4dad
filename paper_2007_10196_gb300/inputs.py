"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds the workload definitions (analytic initial conditions, domains, end times, time-step
rules) and seeded random draws; none of the method's arithmetic.  Every random value comes
from numpy's PCG64 generator with a fixed seed.

The paper's experiments use analytic initial data only (Section 3), so every workload here
is synthetic by construction; no dataset stands behind any of them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PI = math.pi


@dataclass
class Workload:
    name: str
    dim: int
    nr: int
    nl: int
    pde: int                  # 0 advection, 1 Burgers
    ic: tuple                 # (b, a, w, phi): u0 = b + a sin(w sum x + phi)
    t_end: float
    dt_rule: int              # 0: dt = coef h^{5/3}, 1: CFL
    dt_coef: float = 0.5
    cfl: float = 0.4
    lo: float = 0.0
    hi: float = 4.0
    scheme: int = 0           # WENO5
    prolong: int = 0          # WENO5 interpolation
    note: str = ""


# Domain [0, 4]^d: sin(pi sum x / 2) has period 4 in every coordinate, so it is periodic on
# [0, 4]^d (on [0, 2]^d it is not: a shift by 2 flips its sign).
WORKLOADS = {
    "adv2d_nr10_nl4": Workload("adv2d_nr10_nl4", 2, 10, 4, 0, (0.0, 1.0, PI / 2, 0.0), 1.0, 0, 0.5,
                               note="2-D linear advection, finest 160^2, dt = 0.5 h^{5/3}, t = 1"),
    "burgers2d_nr16_nl6_smooth": Workload("burgers2d_nr16_nl6_smooth", 2, 16, 6, 1, (0.5, 1.0, PI / 2, 0.0),
                                          0.5 / PI, 0, 0.5,
                                          note="2-D Burgers, finest 1024^2, smooth (t = 0.5/pi)"),
    "burgers2d_nr16_nl6_shock": Workload("burgers2d_nr16_nl6_shock", 2, 16, 6, 1, (0.5, 1.0, PI / 2, 0.0),
                                         1.5 / PI, 1, cfl=0.4,
                                         note="2-D Burgers, finest 1024^2, after the shock (t = 1.5/pi), CFL 0.4"),
    "adv3d_nr8_nl6": Workload("adv3d_nr8_nl6", 3, 8, 6, 0, (0.0, 1.0, PI / 2, 0.0), 0.5, 0, 0.5,
                              note="3-D linear advection, finest 512^3"),
    "adv4d_nr8_nl5": Workload("adv4d_nr8_nl5", 4, 8, 5, 0, (0.0, 1.0, PI / 2, 0.0), 0.5, 0, 0.5,
                              note="4-D linear advection, finest 256^4"),
}


@dataclass
class BatchMember:
    nr: int
    nl: int
    a: float


def burgers3d_batch(n: int = 256, seed: int = 2007):
    """Uneven batch of independent 3-D Burgers problems u0 = 0.5 + a sin(pi sum x / 2) on
    [0, 4]^3: per member, in this order, root cells from {8, 12, 16}, finest level from
    {3, 4, 5} and amplitude a ~ U[0.5, 1]; all run to t = 0.3 with CFL 0.4."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nr = int(rng.choice([8, 12, 16]))
        nl = int(rng.choice([3, 4, 5]))
        a = float(rng.uniform(0.5, 1.0))
        out.append(BatchMember(nr, nl, a))
    return out


BATCH_T_END = 0.3
BATCH_CFL = 0.4


def random_field(seed: int, shape, kind: str = "smooth", dtype=np.float64):
    """A seeded random periodic field on an index grid of `shape` (axis 0 fastest; returned
    flat).  kind: 'smooth' (a few random Fourier modes), 'rough' (uniform noise in [-1, 1]),
    'steps' (piecewise constant with jumps), 'mixed' (smooth plus steps)."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    idx = np.meshgrid(*[np.arange(s) / s for s in shape], indexing="ij")
    if kind == "rough":
        v = rng.uniform(-1.0, 1.0, size=shape)
    elif kind in ("smooth", "steps", "mixed"):
        v = np.zeros(shape)
        if kind != "steps":
            v += 0.5
            for _ in range(4):
                kvec = rng.integers(-2, 3, size=len(shape))
                ph = rng.uniform(0, 2 * PI)
                amp = rng.uniform(0.1, 0.5)
                v += amp * np.sin(2 * PI * sum(int(kk) * x for kk, x in zip(kvec, idx)) + ph)
        if kind != "smooth":
            for _ in range(3):
                ax = int(rng.integers(0, len(shape)))
                cut = rng.uniform(0, 1)
                v += rng.uniform(-0.8, 0.8) * (idx[ax] >= cut)
    else:
        raise ValueError(kind)
    # to axis-0-fastest flat order
    return np.ascontiguousarray(v.transpose(tuple(reversed(range(len(shape))))).reshape(-1), dtype=dtype)
