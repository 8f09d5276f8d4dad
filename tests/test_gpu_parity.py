"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 path: bit-exact.  Both sides evaluate the paper's formulas as the same sequence of
IEEE-754 double operations (no fused multiply-add on either side), so every grid value after
any number of steps, and every combined value, must be identical.  Where the GPU evaluates
sin() itself (on-device restriction), values differ by an ulp and a tolerance of 1e-12
relative L-infinity applies.

FP32 path: the bulk WENO arithmetic is float; the tolerance is derived in each test from the
float unit roundoff (2^-24) and the number of roundings that reach the result.
"""
import math

import numpy as np
import pytest

import paper_2007_10196_gb300 as P
from paper_2007_10196_gb300 import inputs

from _helpers import make, oracle_problem, random_grids, read_grids, shapes_from_levels, sine_grid

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _levels(h, dim):
    G = P.sg_num_grids(h)
    info = [P.sg_grid_info(h, g, dim) for g in range(G)]
    return [i[0] for i in info], [i[1] for i in info], [i[2] for i in info]


@pytest.mark.parametrize("dim,nl", [(1, 3), (2, 0), (2, 4), (3, 3), (4, 3), (5, 2), (6, 2)])
def test_grid_table_matches_oracle(sg, orc, dim, nl):
    h = make(dim, 5, nl, P.SG_PDE_ADVECTION)
    try:
        lev, shp, co = _levels(h, dim)
        olev, oco = orc.grid_set(dim, nl)
        assert [tuple(x) for x in olev] == lev
        assert list(oco) == co
        assert shp == shapes_from_levels(5, lev)
    finally:
        P.sg_destroy(h)


@pytest.mark.parametrize("prec", [P.SG_F64, P.SG_F32])
def test_restriction_matches_oracle(sg, orc, prec):
    dim, nr, nl = 3, 6, 2
    ic = (0.5, 0.8, 1.3, 0.2)
    h = make(dim, nr, nl, P.SG_PDE_BURGERS, precision=prec, lo=[0.0, -1.0, 2.0], hi=[4.0, 3.0, 5.0])
    try:
        P.sg_init(h, P.SG_IC_SINE, ic)
        lev, shp, _ = _levels(h, dim)
        got = read_grids(h, [int(np.prod(s)) for s in shp])
        p = orc.problem(dim, nr, nl, pde=1, lo=(0.0, -1.0, 2.0), hi=(4.0, 3.0, 5.0))
        for l, g in zip(lev, got):
            ref = orc.restrict_sine(p, l, *ic)
            if prec == P.SG_F64:
                assert np.max(np.abs(g - ref)) <= 4 * np.finfo(float).eps * 1.3
            else:
                assert np.max(np.abs(g.astype(np.float64) - ref)) <= U32 * 1.3 * 1.01
    finally:
        P.sg_destroy(h)


SWEEP = -1  # tile column: the d = 3 sweep kernel; 0: autotuned; else the tiled kernel's tile

# (dim, nr, nl, pde, scheme, adv, exec, tile_points, dt_rule, steps)
STEP_CASES = [
    (1, 7, 3, 1, 0, 1.0, P.SG_PLAIN, 0, 1, 3),
    (2, 10, 3, 0, 0, (1.0, -0.7), P.SG_BATCHED, 256, 1, 2),
    (2, 5, 4, 1, 1, 1.0, P.SG_PLAIN, 512, 0, 2),
    (2, 6, 3, 1, 0, 1.0, P.SG_BATCHED, 1024, 1, 4),
    (3, 6, 2, 1, 0, 1.0, P.SG_BATCHED, 1024, 1, 2),
    (3, 12, 2, 1, 0, 1.0, P.SG_PLAIN, 512, 1, 1),
    (3, 12, 2, 1, 0, 1.0, P.SG_PLAIN, SWEEP, 1, 1),
    (3, 5, 3, 0, 1, (0.5, -1.0, 2.0), P.SG_BATCHED, 256, 0, 1),
    (3, 5, 3, 0, 1, (0.5, -1.0, 2.0), P.SG_BATCHED, SWEEP, 0, 1),
    (3, 13, 1, 1, 0, 1.0, P.SG_BATCHED, SWEEP, 1, 2),  # ragged 3-D tiles (13 = 8 + 5, 26 = 8 + 8 + 8 + 2)
    (3, 13, 1, 1, 0, 1.0, P.SG_BATCHED, 0, 1, 2),
    (4, 5, 2, 0, 0, (1.0, -1.0, 0.5, 2.0), P.SG_BATCHED, 512, 1, 1),
    (5, 5, 1, 1, 0, 1.0, P.SG_PLAIN, 256, 1, 1),
    (6, 5, 1, 0, 0, (1.0, -0.5, 0.25, 2.0, -1.5, 1.0), P.SG_BATCHED, 1024, 1, 1),
]


def _step_case(orc, case, prec, kind="mixed", seed=11):
    dim, nr, nl, pde, scheme, adv, exe, tp, rule, nsteps = case
    advv = tuple(np.broadcast_to(np.asarray(adv, float), (dim,)))
    kern = dict(stage_kernel=P.SG_STAGE_SWEEP, tile_points=0) if tp == SWEEP else dict(tile_points=tp)
    h = make(dim, nr, nl, pde, precision=prec, exec=exe, scheme=scheme, **kern,
             adv_speed=list(advv) + [1.0] * (6 - dim), dt_rule=rule, dt_coef=0.7, cfl=0.45)
    try:
        lev, shp, _ = _levels(h, dim)
        sizes = [int(np.prod(s)) for s in shp]
        g0 = random_grids(seed, nr, lev, kind, scale=0.6, offset=0.2)
        if prec == P.SG_F32:
            g0 = [g.astype(np.float32).astype(np.float64) for g in g0]  # both sides start equal
        P.sg_init_grids(h, np.concatenate(g0))
        t = P.sg_step(h, 10.0, nsteps)
        got = read_grids(h, sizes)
        _, steps = P.sg_time(h)
    finally:
        P.sg_destroy(h)
    p = oracle_problem(orc, dim, nr, nl, pde, scheme=scheme, adv=advv)
    ref, osteps, ot = orc.solve(p, lev, g0, 10.0, max_steps=nsteps, rule=rule, coef=0.7, cfl=0.45)
    return got, ref, steps, osteps, t, ot, g0


@pytest.mark.parametrize("case", STEP_CASES, ids=lambda c: "d%d_nr%d_nl%d_pde%d_s%d_x%d_tp%d" % (c[0], c[1], c[2], c[3], c[4], c[6], c[7]))
def test_steps_fp64_bitwise(sg, orc, case):
    got, ref, steps, osteps, t, ot, _ = _step_case(orc, case, P.SG_F64)
    assert steps == osteps and t == ot
    for g, r in zip(got, ref):
        assert np.array_equal(g, r), np.max(np.abs(g - r))


@pytest.mark.parametrize("case", [c for c in STEP_CASES if c[0] <= 3], ids=lambda c: "d%d_nr%d_nl%d_pde%d_s%d_x%d_tp%d" % (c[0], c[1], c[2], c[3], c[4], c[6], c[7]))
def test_steps_fp32_within_tolerance(sg, orc, case):
    got, ref, steps, osteps, t, ot, g0 = _step_case(orc, case, P.SG_F32)
    assert steps == osteps
    # Each stage rounds the state once per RK update plus the flux arithmetic, whose
    # rounding enters multiplied by dt/h <= 1: bound 64 u32 per stage relative to max|u|.
    umax = max(np.abs(g).max() for g in g0)
    tol = 64 * U32 * 3 * steps * max(umax, 1.0)
    for g, r in zip(got, ref):
        assert np.max(np.abs(g.astype(np.float64) - r)) <= tol


def test_graph_and_direct_launch_agree(sg, orc):
    res = []
    for gs in (0, -1, 3):
        h = make(2, 6, 3, P.SG_PDE_BURGERS, graph_steps=gs, dt_rule=P.SG_DT_CFL)
        try:
            lev, shp, _ = _levels(h, 2)
            P.sg_init_grids(h, np.concatenate(random_grids(5, 6, lev)))
            P.sg_step(h, 0.2, 1 << 40)
            res.append((P.sg_time(h), read_grids(h, [int(np.prod(s)) for s in shp])))
        finally:
            P.sg_destroy(h)
    for r in res[1:]:
        assert r[0] == res[0][0]
        assert all(np.array_equal(a, b) for a, b in zip(r[1], res[0][1]))


def test_adv2d_nr10_nl4_full_run_fp64(sg, orc):
    """The 2-D advection workload end to end (936 steps): grids and combination bit-exact
    with the oracle from the same initial arrays; the on-device restriction within 1e-12."""
    W = inputs.WORKLOADS["adv2d_nr10_nl4"]
    p = orc.problem(2, W.nr, W.nl, pde=W.pde, eps=1e-3, lo=W.lo, hi=W.hi)
    lev, co = orc.grid_set(2, W.nl)
    g0 = [sine_grid(W.nr, l, W.lo, W.hi, W.ic) for l in lev]
    ref, osteps, ot = orc.solve(p, lev, g0, W.t_end, rule=W.dt_rule, coef=W.dt_coef)
    refhat = orc.combine(p, lev, co, ref)
    ol1, olinf = orc.error_norms(p, refhat, *W.ic, W.t_end)
    for mode in ("host", "device"):
        h = make(2, W.nr, W.nl, W.pde, dt_coef=W.dt_coef)
        try:
            if mode == "host":
                P.sg_init_grids(h, np.concatenate(g0))
            else:
                P.sg_init(h, P.SG_IC_SINE, W.ic)
            P.sg_step(h, W.t_end)
            t, steps = P.sg_time(h)
            assert steps == osteps == 936 and t == ot
            got = read_grids(h, [len(g) for g in g0])
            P.sg_prolong_combine(h)
            uhat = P.sg_read(h, P.SG_WHICH_COMBINED, count=refhat.size)
            if mode == "host":  # exact-solution norms need the analytic initial condition
                with pytest.raises(P.SgError) as e:
                    P.sg_reduce(h, -1, P.SG_REDUCE_L1_EXACT)
                assert e.value.status == P.SG_ERR_STATE
            else:
                l1 = P.sg_reduce(h, -1, P.SG_REDUCE_L1_EXACT)
                linf = P.sg_reduce(h, -1, P.SG_REDUCE_LINF_EXACT)
        finally:
            P.sg_destroy(h)
        if mode == "host":
            for g, r in zip(got, ref):
                assert np.array_equal(g, r)
            assert np.array_equal(uhat, refhat)
        else:
            scale = max(np.abs(r).max() for r in ref)
            for g, r in zip(got, ref):
                assert np.max(np.abs(g - r)) <= 1e-12 * scale
            assert np.max(np.abs(uhat - refhat)) <= 1e-12 * np.abs(refhat).max()
            assert abs(l1 - ol1) <= 1e-9 * ol1 and abs(linf - olinf) <= 1e-9 * olinf


@pytest.mark.parametrize("dim,nr,nl,prolong,kind", [
    (1, 7, 3, 0, "mixed"), (2, 6, 3, 0, "mixed"), (2, 5, 3, 1, "smooth"), (3, 5, 2, 0, "steps"),
    (3, 6, 2, 1, "mixed"), (4, 5, 1, 0, "mixed")])
@pytest.mark.parametrize("budget", [0.0, -1.0], ids=["one_pass", "grid_by_grid"])
def test_prolong_combine_fp64_bitwise(sg, orc, dim, nr, nl, prolong, kind, budget):
    h = make(dim, nr, nl, P.SG_PDE_ADVECTION, prolong=prolong, combine_budget_gb=budget)
    try:
        lev, shp, co = _levels(h, dim)
        g0 = random_grids(3, nr, lev, kind)
        P.sg_init_grids(h, np.concatenate(g0))
        P.sg_prolong_combine(h)
        nf = (nr << nl) ** dim
        got = P.sg_read(h, P.SG_WHICH_COMBINED, count=nf)
    finally:
        P.sg_destroy(h)
    p = orc.problem(dim, nr, nl, pde=0, prolong=prolong, eps=1e-3)
    ref = orc.combine(p, lev, co, g0)
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))


# last-axis ratios r = 2^(N_L - l_{d-1}) up to 4 with ragged 8-node chunks (N_f = 20), and up
# to 16 (d = 3, N_L = 4) and 64 (d = 2, N_L = 6) on whole chunks: every chunk schedule of the
# FP32 last-axis kernel (r = 1, 2, 4, 8, >= 16, ragged); N_L = 0 with odd N_r: an odd number of
# columns (no 8-byte column pairs)
@pytest.mark.parametrize("dim,nr,nl,prolong", [(2, 6, 3, 0), (3, 5, 2, 0), (3, 5, 2, 1), (3, 5, 4, 0), (3, 5, 4, 1),
                                               (2, 5, 6, 0), (2, 5, 0, 0), (3, 7, 0, 1)])
@pytest.mark.parametrize("budget", [0.0, -1.0], ids=["one_pass", "grid_by_grid"])
def test_prolong_combine_fp32_within_tolerance(sg, orc, dim, nr, nl, prolong, budget):
    h = make(dim, nr, nl, P.SG_PDE_ADVECTION, prolong=prolong, precision=P.SG_F32, combine_budget_gb=budget)
    try:
        lev, shp, co = _levels(h, dim)
        g0 = [g.astype(np.float32).astype(np.float64) for g in random_grids(4, nr, lev, "mixed")]
        P.sg_init_grids(h, np.concatenate(g0))
        P.sg_prolong_combine(h)
        got = P.sg_read(h, P.SG_WHICH_COMBINED, count=(nr << nl) ** dim)
    finally:
        P.sg_destroy(h)
    ref = orc.combine(orc.problem(dim, nr, nl, pde=0, prolong=prolong, eps=1e-3), lev, co, g0)
    # d interpolation passes, each a few float roundings of values <= max|u| times the weights'
    # condition; summed with |c_g| over the grids
    umax = max(np.abs(g).max() for g in g0)
    tol = 32 * U32 * dim * umax * sum(abs(c) for c in co)
    assert np.max(np.abs(got - ref)) <= tol


def test_reductions_match_oracle(sg, orc):
    W = inputs.WORKLOADS["burgers2d_nr16_nl6_smooth"]
    nl = 3
    h = make(2, W.nr, nl, W.pde, dt_coef=W.dt_coef)
    try:
        P.sg_init(h, P.SG_IC_SINE, W.ic)
        lev, shp, co = _levels(h, 2)
        m0 = [P.sg_reduce(h, g, P.SG_REDUCE_MASS) for g in range(len(lev))]
        P.sg_step(h, W.t_end)
        grids = read_grids(h, [int(np.prod(s)) for s in shp])
        m1 = [P.sg_reduce(h, g, P.SG_REDUCE_MASS) for g in range(len(lev))]
        e1 = [P.sg_reduce(h, g, P.SG_REDUCE_ENERGY) for g in range(len(lev))]
        mn = [P.sg_reduce(h, g, P.SG_REDUCE_MIN) for g in range(len(lev))]
        P.sg_prolong_combine(h)
        l1 = P.sg_reduce(h, -1, P.SG_REDUCE_L1_EXACT)
        linf = P.sg_reduce(h, -1, P.SG_REDUCE_LINF_EXACT)
        uhat = P.sg_read(h, -1, count=(W.nr << nl) ** 2)
        t, _ = P.sg_time(h)
    finally:
        P.sg_destroy(h)
    p = orc.problem(2, W.nr, nl, pde=1, eps=1e-3, lo=W.lo, hi=W.hi)
    for l, g, a, b, e, m in zip(lev, grids, m0, m1, e1, mn):
        om = orc.mass(p, l, g)
        assert abs(b - om) <= 1e-13 * abs(om) + 1e-13
        assert abs(a - b) <= 1e-12 * abs(a)  # periodic: mass conserved
        hv = np.prod([4.0 / (W.nr << int(x)) for x in l])
        assert abs(e - np.sum(g * g) * hv) <= 1e-12 * abs(e)
        assert m == g.min()
    ol1, olinf = orc.error_norms(p, uhat, *W.ic, t)
    assert abs(l1 - ol1) <= 1e-11 * ol1 and abs(linf - olinf) <= 1e-11 * olinf


@pytest.mark.parametrize("kernel", [P.SG_STAGE_SWEEP, P.SG_STAGE_TILED])
def test_batch_matches_members_and_oracle(sg, orc, kernel):
    """Uneven members, each with its own CFL time step, advanced by one persistent launch per
    stage: every member equals the same problem run alone, and (FP64) the oracle bit for bit."""
    specs = [(8, 2, 0.6), (5, 3, 1.0), (6, 1, 0.8)]
    for prec in (P.SG_F64, P.SG_F32):
        solo, hs = [], []
        for nr, nl, a in specs:
            for rep in range(2):
                h = make(3, nr, nl, P.SG_PDE_BURGERS, precision=prec, exec=P.SG_BATCHED, dt_rule=P.SG_DT_CFL,
                         stage_kernel=kernel)
                P.sg_init(h, P.SG_IC_SINE, (0.5, a, math.pi / 2, 0.0))
                (hs if rep == 0 else solo).append(h)
        b = P.sg_batch_create(hs)
        try:
            P.sg_step(b, 0.12)
            res_b = [(P.sg_time(h), read_grids(h, [int(np.prod(s)) for s in _levels(h, 3)[1]])) for h in hs]
            for h in solo:
                P.sg_step(h, 0.12)
            res_s = [(P.sg_time(h), read_grids(h, [int(np.prod(s)) for s in _levels(h, 3)[1]])) for h in solo]
        finally:
            P.sg_destroy(b)
            for h in hs + solo:
                P.sg_destroy(h)
        for (tb, gb), (ts, gs_) in zip(res_b, res_s):
            assert tb == ts
            assert all(np.array_equal(x, y) for x, y in zip(gb, gs_))
        if prec == P.SG_F64:
            for (nr, nl, a), ((t, steps), grids) in zip(specs, res_b):
                p = orc.problem(3, nr, nl, pde=1, eps=1e-3)
                lev, _ = orc.grid_set(3, nl)
                g0 = [orc.restrict_sine(p, l, 0.5, a, math.pi / 2) for l in lev]
                ref, osteps, ot = orc.solve(p, lev, g0, 0.12, rule=1, cfl=0.4)
                assert steps == osteps and t == ot
                scale = max(np.abs(r).max() for r in ref)
                for g, r in zip(grids, ref):  # device sin() differs by an ulp
                    assert np.max(np.abs(g - r)) <= 1e-12 * scale


def test_error_paths(sg):
    h = make(2, 6, 2, P.SG_PDE_BURGERS)
    try:
        with pytest.raises(P.SgError) as e:
            P.sg_step(h, 0.1)
        assert e.value.status == P.SG_ERR_STATE
        with pytest.raises(P.SgError) as e:
            P.sg_prolong_combine(h)
        assert e.value.status == P.SG_ERR_STATE
        with pytest.raises(P.SgError) as e:
            P.sg_init_grid(h, 0, np.zeros(3))
        assert e.value.status == P.SG_ERR_ARG
        with pytest.raises(P.SgError) as e:
            P.sg_init_grid(h, 99, np.zeros(3))
        assert e.value.status == P.SG_ERR_ARG
        lev, shp, _ = _levels(h, 2)
        g = [np.full(int(np.prod(s)), 0.5) for s in shp]
        g[1][7] = np.nan
        P.sg_init_grids(h, np.concatenate(g))
        with pytest.raises(P.SgError) as e:
            P.sg_step(h, 0.1, 2)
        assert e.value.status == P.SG_ERR_NONFINITE
        with pytest.raises(P.SgError) as e:
            P.sg_read(h, -1, count=10)
        assert e.value.status == P.SG_ERR_STATE
        # an infinite value under the CFL rule makes alpha infinite and the step zero: the
        # call must stop with an error at the first check instead of stepping forever
        for prec in (P.SG_F64, P.SG_F32):
            c = make(2, 6, 2, P.SG_PDE_BURGERS, precision=prec, dt_rule=P.SG_DT_CFL)
            try:
                g = [np.full(int(np.prod(s)), 0.5) for s in shp]
                g[0][3] = np.inf
                P.sg_init_grids(c, np.concatenate(g))
                with pytest.raises(P.SgError) as e:
                    P.sg_step(c, 1e6)
                assert e.value.status == P.SG_ERR_NONFINITE
                assert P.sg_time(c)[1] <= 16  # at most one captured graph of steps
            finally:
                P.sg_destroy(c)
        # the handle stays usable after errors
        P.sg_init(h, P.SG_IC_SINE, (0.5, 1.0, math.pi / 2, 0.0))
        P.sg_step(h, 0.01)
        with pytest.raises(P.SgError) as e:
            P.sg_read(h, 0, out=np.empty(3))
        assert e.value.status == P.SG_ERR_ARG
    finally:
        P.sg_destroy(h)
    a = make(2, 6, 2, P.SG_PDE_BURGERS)
    b = make(2, 6, 2, P.SG_PDE_BURGERS, precision=P.SG_F32)
    try:
        with pytest.raises(P.SgError) as e:
            P.sg_batch_create([a, b])
        assert e.value.status == P.SG_ERR_ARG
    finally:
        P.sg_destroy(a)
        P.sg_destroy(b)


def test_max_steps_and_time_reached(sg):
    h = make(2, 6, 2, P.SG_PDE_ADVECTION, dt_coef=1.0)
    try:
        P.sg_init(h, P.SG_IC_SINE, (0.0, 1.0, math.pi / 2, 0.0))
        hf = 4.0 / (6 << 2)
        dt = hf ** (5.0 / 3.0)
        t = P.sg_step(h, 1.0, 3)
        assert P.sg_time(h)[1] == 3 and abs(t - 3 * dt) < 1e-15
        t = P.sg_step(h, 4.5 * dt)  # the shortened last step lands exactly on t_end
        assert P.sg_time(h)[1] == 5 and t == 4.5 * dt
        t = P.sg_step(h, 4.5 * dt)  # already there: no step
        assert P.sg_time(h)[1] == 5
        assert P.sg_launch_count(h) > 0
    finally:
        P.sg_destroy(h)


@pytest.mark.parametrize("nr,nl", [(10, 3), (20, 3)])
def test_fp32_error_matches_fp64_on_table4_rows(sg, orc, nr, nl):
    """Example 3(a) sparse rows of Table 4 (2-D Burgers, WENO prolongation): FP64 reproduces
    the printed L1 to five digits; the FP32 batched path's L1 is within 1.5x of the FP64 one
    (the discretisation error, 7.1e-05 and 2.7e-07, dominates float rounding)."""
    ic = (1.0, 0.5, 1.0, 0.0)
    two_pi = 2 * math.pi
    printed = {10: 7.1354e-05, 20: 2.7404e-07}[nr]
    res = {}
    for prec, exe in ((P.SG_F64, P.SG_PLAIN), (P.SG_F32, P.SG_BATCHED)):
        h = make(2, nr, nl, P.SG_PDE_BURGERS, precision=prec, exec=exe, lo=[0.0] * 6, hi=[two_pi] * 6,
                 dt_coef=1.0)
        try:
            P.sg_init(h, P.SG_IC_SINE, ic)
            P.sg_step(h, 0.3)
            P.sg_prolong_combine(h)
            res[prec] = (P.sg_reduce(h, -1, P.SG_REDUCE_L1_EXACT),
                         P.sg_read(h, -1, count=(nr << nl) ** 2))
        finally:
            P.sg_destroy(h)
    l64, u64 = res[P.SG_F64]
    l32, u32 = res[P.SG_F32]
    unit = 10.0 ** (math.floor(math.log10(printed)) - 4)
    assert abs(l64 - printed) <= 0.5 * unit
    if nr == 10:  # truncation error above 1e-5: FP32 must reproduce the same L1 within 1.5x
        assert l64 / 1.5 <= l32 <= 1.5 * l64, (l32, l64)
    # the FP32 result differs from FP64 by float rounding only (compensated state): 64 u32
    assert np.max(np.abs(u32 - u64)) <= 64 * U32 * 1.5, np.max(np.abs(u32 - u64))


def test_fp32_long_run_stays_close_to_fp64(sg, orc):
    """936 steps of dt = 0.5 h^{5/3} (the 2-D advection workload): with the float-pair state
    the FP32 solution stays within a few float ulps of the FP64 one instead of drifting with
    the number of steps."""
    W = inputs.WORKLOADS["adv2d_nr10_nl4"]
    out = {}
    for prec, exe in ((P.SG_F64, P.SG_PLAIN), (P.SG_F32, P.SG_BATCHED)):
        h = make(2, W.nr, W.nl, W.pde, precision=prec, exec=exe, dt_coef=W.dt_coef)
        try:
            P.sg_init(h, P.SG_IC_SINE, W.ic)
            P.sg_step(h, W.t_end)
            P.sg_prolong_combine(h)
            out[prec] = (P.sg_read(h, -1, count=(W.nr << W.nl) ** 2), P.sg_reduce(h, -1, P.SG_REDUCE_L1_EXACT))
        finally:
            P.sg_destroy(h)
    d = np.max(np.abs(out[P.SG_F32][0] - out[P.SG_F64][0]))
    print("fp32-fp64 max diff after 936 steps: %.3e; L1 %.4e vs %.4e" % (d, out[P.SG_F32][1], out[P.SG_F64][1]))
    assert d <= 64 * U32
    assert abs(out[P.SG_F32][1] - out[P.SG_F64][1]) <= 0.05 * out[P.SG_F64][1]


def test_fp32_mass_conserved_by_float_pair(sg):
    """Periodic mass is conserved to float-pair precision over many steps."""
    h = make(3, 6, 2, P.SG_PDE_BURGERS, precision=P.SG_F32, exec=P.SG_BATCHED, dt_rule=P.SG_DT_CFL)
    try:
        P.sg_init(h, P.SG_IC_SINE, (0.5, 0.9, math.pi / 2, 0.0))
        G = P.sg_num_grids(h)
        m0 = [P.sg_reduce(h, g, P.SG_REDUCE_MASS) for g in range(G)]
        P.sg_step(h, 0.5)  # about 32 steps, through the shock (t_s = 0.24)
        steps = P.sg_time(h)[1]
        m1 = [P.sg_reduce(h, g, P.SG_REDUCE_MASS) for g in range(G)]
    finally:
        P.sg_destroy(h)
    assert steps > 20
    for a, b in zip(m0, m1):
        # the flux differences telescope; each step adds at most one float rounding of the
        # increment per point to the pair
        assert abs(a - b) <= 1e-6 * 64.0, (a, b)


def test_shocked_member_fp64_bitwise(sg, orc):
    """A benchmark-batch member past its shock time (3-D Burgers, N_r = 8, N_L = 3, a = 1,
    t = 0.3, CFL 0.4): the FP64 path equals the oracle bit for bit through the shock and the
    combination, including the combined solution's overshoot of the initial bounds — the
    overshoot is the combination technique at this root resolution, not the implementation."""
    nr, nl, a = 8, 3, 1.0
    ic = (0.5, a, math.pi / 2, 0.0)
    p = orc.problem(3, nr, nl, pde=1, eps=1e-3)
    lev, co = orc.grid_set(3, nl)
    g0 = [sine_grid(nr, l, 0.0, 4.0, ic) for l in lev]
    ref, osteps, ot = orc.solve(p, lev, g0, 0.3, rule=1, cfl=0.4)
    refhat = orc.combine(p, lev, co, ref)
    h = make(3, nr, nl, P.SG_PDE_BURGERS, exec=P.SG_BATCHED, dt_rule=P.SG_DT_CFL)
    try:
        P.sg_init_grids(h, np.concatenate(g0))
        P.sg_step(h, 0.3)
        t, steps = P.sg_time(h)
        got = read_grids(h, [len(g) for g in g0])
        P.sg_prolong_combine(h)
        uhat = P.sg_read(h, -1, count=refhat.size)
        lo, hi = P.sg_reduce(h, -1, P.SG_REDUCE_MIN), P.sg_reduce(h, -1, P.SG_REDUCE_MAX)
    finally:
        P.sg_destroy(h)
    assert steps == osteps and t == ot == 0.3
    assert all(np.array_equal(g, r) for g, r in zip(got, ref))
    assert np.array_equal(uhat, refhat)
    assert lo == refhat.min() and hi == refhat.max()
    assert max(g.max() for g in ref) <= 0.5 + a and min(g.min() for g in ref) >= 0.5 - a  # grids stay bounded
    assert lo < 0.5 - a - 0.1  # the combination overshoots


def test_autotuner_choice_is_cached_and_shared_by_a_batch(sg, orc):
    """The first sg_step of an autotuned handle times the candidates and keeps one; a second
    handle of the same kind reuses the cached choice; a batch puts every member on its own
    tuned configuration, and the results stay bit-exact (FP64) whichever kernel was chosen."""
    spec = (3, 6, 2, P.SG_PDE_BURGERS)
    h1 = make(*spec, dt_rule=P.SG_DT_CFL)
    h2 = make(*spec, dt_rule=P.SG_DT_CFL)
    try:
        assert P.sg_stage_config(h1) == (P.SG_STAGE_SWEEP, 512, 0.0)  # starting point for d = 3
        for h in (h1, h2):
            P.sg_init(h, P.SG_IC_SINE, (0.5, 1.0, math.pi / 2, 0.0))
            P.sg_step(h, 0.05)
        k1, tp1, ms1 = P.sg_stage_config(h1)
        assert k1 in (P.SG_STAGE_SWEEP, P.SG_STAGE_TILED) and tp1 in (256, 512, 1024) and ms1 > 0.0
        assert P.sg_stage_config(h2) == (k1, tp1, ms1)
        lev, shp, _ = _levels(h1, 3)
        sizes = [int(np.prod(x)) for x in shp]
        g1, g2 = read_grids(h1, sizes), read_grids(h2, sizes)
        assert all(np.array_equal(a, b) for a, b in zip(g1, g2))
        p = orc.problem(3, 6, 2, pde=1, eps=1e-3)
        g0 = [orc.restrict_sine(p, l, 0.5, 1.0, math.pi / 2) for l in lev]
        ref, _, _ = orc.solve(p, lev, g0, 0.05, rule=1, cfl=0.4)
        scale = max(np.abs(r).max() for r in ref)
        for g, r in zip(g1, ref):  # device sin() differs by an ulp
            assert np.max(np.abs(g - r)) <= 1e-12 * scale
        b = P.sg_batch_create([h1, h2])
        try:
            P.sg_step(b, 0.1)
            kb = P.sg_stage_config(b)
            assert kb[2] > 0.0
            assert P.sg_stage_config(h1)[:2] == kb[:2] and P.sg_stage_config(h2)[:2] == kb[:2]
            assert all(np.array_equal(a, c) for a, c in zip(read_grids(h1, sizes), read_grids(h2, sizes)))
        finally:
            P.sg_destroy(b)
    finally:
        P.sg_destroy(h1)
        P.sg_destroy(h2)
