"""Zero boundary (SG_BC_ZERO) for advection and Burgers against the oracle, through the C ABI.

u = 0 beyond the nodes of a zero-boundary axis, in the WENO5 stencils (Section 2.1) and in the
interpolation of Eqs. (8)-(11) (the zero boundary treatment of Example 5 applied to Eq. 1).
FP64: every grid value after several steps, and every combined value, bit for bit, for each
stage kernel (d = 3 line sweep with its vectorised and scalar gathers, the padded box for
d <= 3, the line buffer for d = 4), with zero and periodic axes mixed.  FP32: within the
float-rounding bound of the other FP32 tests.
"""
import numpy as np
import pytest

import paper_2007_10196_gb300 as P

from _helpers import make, oracle_problem, random_grids, read_grids

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
SWEEP, SWEEP2 = -1, -2
Z, PER = P.SG_BC_ZERO, P.SG_BC_PERIODIC

# (dim, nr, nl, pde, bc, exec, tile, dt_rule, steps)
CASES = [
    (1, 7, 3, 1, (Z,), P.SG_PLAIN, 0, 1, 3),
    (2, 6, 3, 1, (Z, Z), P.SG_BATCHED, 256, 1, 3),
    (2, 10, 2, 0, (Z, PER), P.SG_PLAIN, 512, 0, 2),
    (3, 8, 2, 1, (Z, Z, Z), P.SG_BATCHED, SWEEP, 1, 2),      # float4 gather (8-wide tiles)
    (3, 8, 2, 0, (PER, Z, Z), P.SG_BATCHED, SWEEP, 1, 2),
    (3, 13, 1, 1, (Z, PER, Z), P.SG_BATCHED, SWEEP, 1, 2),   # ragged tiles, scalar gather
    (3, 6, 2, 1, (Z, PER, Z), P.SG_BATCHED, 1024, 1, 2),
    (4, 5, 2, 0, (Z, PER, Z, PER), P.SG_BATCHED, 512, 1, 1),
]


def _levels(h, dim):
    G = P.sg_num_grids(h)
    info = [P.sg_grid_info(h, g, dim) for g in range(G)]
    return [i[0] for i in info], [i[1] for i in info], [i[2] for i in info]


def _run(orc, case, prec):
    dim, nr, nl, pde, bc, exe, tile, rule, nsteps = case
    adv = (1.0, -0.7, 0.5, 2.0)[:dim]
    kern = (dict(stage_kernel=P.SG_STAGE_SWEEP, tile_points=0) if tile == SWEEP else
            dict(stage_kernel=P.SG_STAGE_SWEEP2, tile_points=0) if tile == SWEEP2 else dict(tile_points=tile))
    h = make(dim, nr, nl, pde, precision=prec, exec=exe, bc=list(bc) + [PER] * (6 - dim),
             adv_speed=list(adv) + [1.0] * (6 - dim), dt_rule=rule, dt_coef=0.7, cfl=0.45, **kern)
    try:
        lev, shp, co = _levels(h, dim)
        sizes = [int(np.prod(s)) for s in shp]
        g0 = random_grids(31, nr, lev, "mixed", scale=0.6, offset=0.2)
        if prec == P.SG_F32:
            g0 = [g.astype(np.float32).astype(np.float64) for g in g0]
        P.sg_init_grids(h, np.concatenate(g0))
        P.sg_step(h, 10.0, nsteps)
        got = read_grids(h, sizes)
        _, steps = P.sg_time(h)
        P.sg_prolong_combine(h)
        uhat = P.sg_read(h, P.SG_WHICH_COMBINED, count=(nr << nl) ** dim)
        with pytest.raises(P.SgError) as e:  # the exact solution is the periodic one
            P.sg_reduce(h, P.SG_WHICH_COMBINED, P.SG_REDUCE_L1_EXACT)
        assert e.value.status == P.SG_ERR_STATE
    finally:
        P.sg_destroy(h)
    p = oracle_problem(orc, dim, nr, nl, pde, eps=1e-3, adv=adv)
    for k in range(dim):
        p.bc[k] = int(bc[k])
    ref, osteps, _ = orc.solve(p, lev, g0, 10.0, max_steps=nsteps, rule=rule, coef=0.7, cfl=0.45)
    refhat = orc.combine(p, lev, co, ref)
    return got, ref, steps, osteps, uhat, refhat, co, g0


def _id(c):
    return "d%d_nr%d_pde%d_bc%s_x%d_tp%d" % (c[0], c[1], c[3], "".join("z" if b == Z else "p" for b in c[4]), c[5], c[6])


@pytest.mark.parametrize("case", CASES, ids=_id)
def test_zero_bc_fp64_bitwise(sg, orc, case):
    got, ref, steps, osteps, uhat, refhat, _, _ = _run(orc, case, P.SG_F64)
    assert steps == osteps
    for g, r in zip(got, ref):
        assert np.array_equal(g, r), np.max(np.abs(g - r))
    assert np.array_equal(uhat, refhat), np.max(np.abs(uhat - refhat))


FP32_CASES = [c for c in CASES if c[0] <= 3] + [
    (3, 8, 2, 1, (Z, Z, Z), P.SG_BATCHED, SWEEP2, 1, 2),
    (3, 13, 1, 1, (Z, PER, Z), P.SG_BATCHED, SWEEP2, 1, 2),
]


@pytest.mark.parametrize("case", FP32_CASES, ids=_id)
def test_zero_bc_fp32_within_tolerance(sg, orc, case):
    got, ref, steps, osteps, uhat, refhat, co, g0 = _run(orc, case, P.SG_F32)
    assert steps == osteps
    umax = max(np.abs(g).max() for g in g0)
    tol = 64 * U32 * 3 * steps * max(umax, 1.0)
    for g, r in zip(got, ref):
        assert np.max(np.abs(g.astype(np.float64) - r)) <= tol
    tolc = (tol + 32 * U32 * case[0] * umax) * sum(abs(c) for c in co)
    assert np.max(np.abs(uhat - refhat)) <= tolc


@pytest.mark.parametrize("budget", [0.0, -1.0], ids=["one_pass", "grid_by_grid"])
@pytest.mark.parametrize("dim,nr,nl,prolong,bc", [(2, 6, 3, 0, (Z, Z)), (3, 5, 2, 1, (PER, Z, Z)),
                                                  (3, 5, 2, 0, (Z, PER, PER))])
def test_zero_bc_combination_fp64_bitwise(sg, orc, dim, nr, nl, prolong, bc, budget):
    h = make(dim, nr, nl, P.SG_PDE_BURGERS, prolong=prolong, combine_budget_gb=budget,
             bc=list(bc) + [PER] * (6 - dim))
    try:
        lev, shp, co = _levels(h, dim)
        g0 = random_grids(8, nr, lev, "mixed")
        P.sg_init_grids(h, np.concatenate(g0))
        P.sg_prolong_combine(h)
        got = P.sg_read(h, P.SG_WHICH_COMBINED, count=(nr << nl) ** dim)
    finally:
        P.sg_destroy(h)
    p = orc.problem(dim, nr, nl, pde=1, prolong=prolong, eps=1e-3, bc=bc)
    assert np.array_equal(got, orc.combine(p, lev, co, g0))


# FP32 last-axis kernel with zeros beyond the ends of the last axis: ratios r up to 16 (d = 3,
# N_L = 4) and 64 (d = 2, N_L = 6), so the window rows of every chunk schedule reach past
# both ends; within the FP32 combination bound (d interpolation passes, summed with |c_g|)
@pytest.mark.parametrize("dim,nr,nl,prolong,bc", [(3, 5, 4, 0, (PER, Z, Z)), (3, 5, 4, 1, (Z, PER, Z)),
                                                  (2, 5, 6, 0, (Z, Z)), (2, 6, 3, 0, (PER, Z))])
def test_zero_bc_combination_fp32_large_ratios(sg, orc, dim, nr, nl, prolong, bc):
    h = make(dim, nr, nl, P.SG_PDE_BURGERS, prolong=prolong, precision=P.SG_F32, bc=list(bc) + [PER] * (6 - dim))
    try:
        lev, shp, co = _levels(h, dim)
        g0 = [g.astype(np.float32).astype(np.float64) for g in random_grids(9, nr, lev, "mixed")]
        P.sg_init_grids(h, np.concatenate(g0))
        P.sg_prolong_combine(h)
        got = P.sg_read(h, P.SG_WHICH_COMBINED, count=(nr << nl) ** dim)
    finally:
        P.sg_destroy(h)
    p = orc.problem(dim, nr, nl, pde=1, prolong=prolong, eps=1e-3, bc=bc)
    ref = orc.combine(p, lev, co, g0)
    umax = max(np.abs(g).max() for g in g0)
    tol = 32 * U32 * dim * umax * sum(abs(c) for c in co)
    assert np.max(np.abs(got - ref)) <= tol


def test_zero_bc_batch_matches_members(sg, orc):
    case = (3, 8, 2, 1, (Z, Z, PER), P.SG_BATCHED, SWEEP, 1, 2)
    single = _run(orc, case, P.SG_F64)
    dim, nr, nl = 3, 8, 2
    hs = [make(dim, nr, nl, 1, exec=P.SG_BATCHED, bc=[Z, Z, PER, PER, PER, PER], dt_rule=1, cfl=0.45,
               stage_kernel=P.SG_STAGE_SWEEP) for _ in range(2)]
    other = make(dim, nr, nl, 1, exec=P.SG_BATCHED, dt_rule=1, cfl=0.45, stage_kernel=P.SG_STAGE_SWEEP)
    try:
        with pytest.raises(P.SgError) as e:
            P.sg_batch_create([hs[0], other])
        assert e.value.status == P.SG_ERR_ARG and "bc" in P.sg_last_error()
        lev, shp, _ = _levels(hs[0], dim)
        sizes = [int(np.prod(s)) for s in shp]
        g0 = random_grids(31, nr, lev, "mixed", scale=0.6, offset=0.2)
        for h in hs:
            P.sg_init_grids(h, np.concatenate(g0))
        b = P.sg_batch_create(hs)
        try:
            P.sg_step(b, 10.0, 2)
        finally:
            P.sg_destroy(b)
        for h in hs:
            got = read_grids(h, sizes)
            for g, r in zip(got, single[1]):
                assert np.array_equal(g, r)
    finally:
        for h in hs + [other]:
            P.sg_destroy(h)
