"""2-D Burgers at the full sparse-grid size: u0 = 0.5 + sin(pi (x + y) / 2) on [0, 4]^2, N_r = 16,
N_L = 6 (finest grid 1024^2, 13 component grids, 163,840 points) -- Example 3 (a) of the paper
(Section 3.2) on a finer sparse grid.

Smooth run to t = 0.5/pi with dt = 0.5 h^{5/3}: the first steps of every grid and the whole
combined solution bit for bit against the oracle (FP64); the full run's L1 error against the
characteristic solution in FP64 and in FP32.
Shock run to t = 1.5/pi with CFL 0.4 and WENO5 prolongation (Eqs. 8-11): the first steps bit
for bit; the full run's undershoot and overshoot of the combined solution against the data
range [-0.5, 1.5], against the oracle's own full run (identical in FP64) and in FP32.  Bounds
are not guaranteed by the method (Remark 1, after Example 4), so the overshoot is reported
and checked against the oracle, not against a bound.
"""
import numpy as np
import pytest

import paper_2007_10196_gb300 as P
from paper_2007_10196_gb300 import inputs

pytestmark = pytest.mark.gpu

SMOOTH = inputs.WORKLOADS["burgers2d_nr16_nl6_smooth"]
SHOCK = inputs.WORKLOADS["burgers2d_nr16_nl6_shock"]


def _setup(orc, w):
    lev, co = orc.grid_set(w.dim, w.nl)
    p = orc.problem(w.dim, w.nr, w.nl, pde=w.pde, eps=1e-3, lo=w.lo, hi=w.hi)
    b, a, om, phi = w.ic
    g0 = [orc.restrict_sine(p, lv, b, a, om, phi) for lv in lev]
    return p, lev, co, g0


def _gpu(w, g0, prec):
    """A handle of workload w; initial grids from the host (g0) or restricted on the device."""
    kw = dict(precision=prec, exec=P.SG_BATCHED, dt_rule=w.dt_rule, dt_coef=w.dt_coef, cfl=w.cfl,
              lo=w.lo, hi=w.hi, prolong=w.prolong)
    h = P.create(w.dim, w.nr, w.nl, w.pde, **kw)
    if g0 is None:
        P.sg_init(h, P.SG_IC_SINE, w.ic)  # also sets the exact solution's parameters
    else:
        flat = np.concatenate(g0)
        P.sg_init_grids(h, flat if prec == P.SG_F64 else flat.astype(np.float32))
    return h


def _pow53_steps(w):
    """Steps of the h^{5/3} rule to t_end, the last one shortened (the device's time loop)."""
    dt = w.dt_coef * (4.0 / (w.nr << w.nl)) ** (5.0 / 3.0)
    t, n = 0.0, 0
    while t < w.t_end:
        t = w.t_end if dt >= w.t_end - t else t + dt
        n += 1
    return n


def _grids(h, sizes):
    out = P.sg_read(h, P.SG_WHICH_ALL_GRIDS, count=int(sum(sizes)))
    return np.split(out.astype(np.float64), np.cumsum(sizes)[:-1])


@pytest.mark.parametrize("w", [SMOOTH, SHOCK], ids=["smooth", "shock"])
def test_c2_first_steps_and_combination_fp64_bitwise(sg, orc, w):
    p, lev, co, g0 = _setup(orc, w)
    sizes = [len(g) for g in g0]
    h = _gpu(w, g0, P.SG_F64)
    try:
        P.sg_step(h, w.t_end, 3)
        got = _grids(h, sizes)
        P.sg_prolong_combine(h)
        uhat = P.sg_read(h, P.SG_WHICH_COMBINED, count=(w.nr << w.nl) ** 2)
        t, steps = P.sg_time(h)
    finally:
        P.sg_destroy(h)
    ref, osteps, ot = orc.solve(p, lev, g0, w.t_end, max_steps=3, rule=w.dt_rule, coef=w.dt_coef, cfl=w.cfl)
    assert steps == osteps == 3 and t == ot
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)
    assert np.array_equal(uhat, orc.combine(p, lev, co, ref))


def test_c2_smooth_full_run_l1(sg):
    w = SMOOTH
    res = {}
    for prec in (P.SG_F64, P.SG_F32):
        h = _gpu(w, None, prec)
        try:
            t = P.sg_step(h, w.t_end)
            _, steps = P.sg_time(h)
            P.sg_prolong_combine(h)
            l1 = P.sg_reduce(h, P.SG_WHICH_COMBINED, P.SG_REDUCE_L1_EXACT)
            linf = P.sg_reduce(h, P.SG_WHICH_COMBINED, P.SG_REDUCE_LINF_EXACT)
        finally:
            P.sg_destroy(h)
        assert t == w.t_end
        res[prec] = (l1, linf, steps)
    (l64, i64, s64), (l32, i32, s32) = res[P.SG_F64], res[P.SG_F32]
    print("C2 smooth (t = 0.5/pi, %d steps): L1 FP64 %.4e, FP32 %.4e; Linf FP64 %.4e, FP32 %.4e"
          % (s64, l64, l32, i64, i32))
    assert s64 == s32 == _pow53_steps(w)
    assert l64 < 1e-6
    # FP32 against FP64 at equal resolution: within 1.5x where the FP64 error exceeds 1e-5,
    # else within the float floor of the combined data (|u| <= 1.5)
    assert l32 <= max(1.5 * l64, l64 + 2e-6)


def test_c2_shock_full_run_overshoot(sg, orc):
    w = SHOCK
    p, lev, co, g0 = _setup(orc, w)
    lo_b, hi_b = w.ic[0] - w.ic[1], w.ic[0] + w.ic[1]
    res = {}
    for prec in (P.SG_F64, P.SG_F32):
        h = _gpu(w, g0, prec)
        try:
            t = P.sg_step(h, w.t_end)
            _, steps = P.sg_time(h)
            sizes = [len(g) for g in g0]
            grids = _grids(h, sizes)
            P.sg_prolong_combine(h)
            mn = P.sg_reduce(h, P.SG_WHICH_COMBINED, P.SG_REDUCE_MIN)
            mx = P.sg_reduce(h, P.SG_WHICH_COMBINED, P.SG_REDUCE_MAX)
            uhat = P.sg_read(h, P.SG_WHICH_COMBINED, count=(w.nr << w.nl) ** 2) if prec == P.SG_F64 else None
        finally:
            P.sg_destroy(h)
        assert t == w.t_end
        gmin = min(g.min() for g in grids)
        gmax = max(g.max() for g in grids)
        res[prec] = (mn, mx, gmin, gmax, steps, uhat, grids)
    mn64, mx64, gmin64, gmax64, s64, uhat64, grids64 = res[P.SG_F64]
    mn32, mx32, gmin32, gmax32, s32, _, _ = res[P.SG_F32]
    over = lambda a, b: max(lo_b - a, b - hi_b, 0.0)
    print("C2 shock (t = 1.5/pi, %d/%d steps): combined range FP64 [%.6f, %.6f] overshoot %.3e, "
          "FP32 [%.6f, %.6f] overshoot %.3e; component grids FP64 [%.6f, %.6f] overshoot %.3e; "
          "criterion 1e-3 %s"
          % (s64, s32, mn64, mx64, over(mn64, mx64), mn32, mx32, over(mn32, mx32), gmin64, gmax64,
             over(gmin64, gmax64), "met" if over(mn64, mx64) <= 1e-3 else "not met"))
    # the oracle's own full run: identical grids, combined solution and range
    ref, osteps, ot = orc.solve(p, lev, g0, w.t_end, rule=w.dt_rule, coef=w.dt_coef, cfl=w.cfl)
    assert osteps == s64 and ot == w.t_end
    for g, r in zip(grids64, ref):
        assert np.array_equal(g, r)
    refhat = orc.combine(p, lev, co, ref)
    assert np.array_equal(uhat64, refhat)
    assert refhat.min() == mn64 and refhat.max() == mx64
    # FP32 follows FP64 after the shock to float accuracy of the range
    assert abs(mn32 - mn64) <= 1e-4 and abs(mx32 - mx64) <= 1e-4
