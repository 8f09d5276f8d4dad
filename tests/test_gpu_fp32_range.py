"""FP32 path against the FP64 oracle across data scales and epsilon (Section 2.1, Eqs. 3-6;
Section 2.2.1, Eqs. 8-11).

The nonlinear weights of Eqs. (5) and (9) depend on the data only through the ratios of the
three (eps + beta_r), so the scheme is scale-covariant apart from eps.  The FP32 kernels form
the weights from rescaled smoothness terms; these tests step and prolong float grids whose
values span 1e-3 to 1e3 (mixed smooth + jump data, so that the weights are far from linear)
and smooth data with small differences at eps down to 1e-8, where unscaled products of the
squared smoothness terms would overflow or fall into subnormals.  Every value must be finite
and within a bound derived from the float unit roundoff (2^-24), the number of roundings that
reach it, and the data's scale.
"""
import numpy as np
import pytest

import paper_2007_10196_gb300 as P

from _helpers import make, oracle_problem, random_grids, read_grids

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
SWEEP, SWEEP2 = -1, -2

# (dim, nr, nl, pde, tile): tile SWEEP = the d = 3 line-sweep kernel, SWEEP2 its two-line form,
# else the tiled kernel with that tile (d <= 3 padded box, d = 4 line buffer)
KERNELS = [
    (3, 6, 2, 1, SWEEP),
    (3, 6, 2, 1, SWEEP2),
    (3, 8, 2, 0, SWEEP2),
    (3, 13, 1, 1, SWEEP2),
    (3, 6, 2, 1, 512),
    (2, 6, 3, 1, 256),
    (2, 6, 3, 0, 1024),
    (4, 5, 1, 1, 512),
]


def _levels(h, dim):
    G = P.sg_num_grids(h)
    info = [P.sg_grid_info(h, g, dim) for g in range(G)]
    return [i[0] for i in info], [i[1] for i in info], [i[2] for i in info]


def _run(orc, dim, nr, nl, pde, tile, kind, scale, eps, nsteps=3):
    kern = (dict(stage_kernel=P.SG_STAGE_SWEEP, tile_points=0) if tile == SWEEP else
            dict(stage_kernel=P.SG_STAGE_SWEEP2, tile_points=0) if tile == SWEEP2 else dict(tile_points=tile))
    adv = (1.0, -0.7, 0.5, 2.0)[:dim]
    h = make(dim, nr, nl, pde, precision=P.SG_F32, exec=P.SG_BATCHED, eps=eps, dt_rule=P.SG_DT_CFL,
             cfl=0.45, adv_speed=list(adv) + [1.0] * (6 - dim), **kern)
    try:
        lev, shp, co = _levels(h, dim)
        sizes = [int(np.prod(s)) for s in shp]
        g0 = [g.astype(np.float32).astype(np.float64)
              for g in random_grids(23, nr, lev, kind, scale=scale, offset=0.3 * scale)]
        P.sg_init_grids(h, np.concatenate(g0).astype(np.float32))
        P.sg_step(h, 1e30, nsteps)
        got = read_grids(h, sizes)
        _, steps = P.sg_time(h)
        P.sg_prolong_combine(h)
        uhat = P.sg_read(h, P.SG_WHICH_COMBINED, count=(nr << nl) ** dim)
    finally:
        P.sg_destroy(h)
    p = oracle_problem(orc, dim, nr, nl, pde, eps=eps, adv=adv)
    ref, osteps, _ = orc.solve(p, lev, g0, 1e30, max_steps=nsteps, rule=orc.DT_CFL, cfl=0.45)
    refhat = orc.combine(p, lev, co, ref)
    return got, ref, steps, osteps, uhat, refhat, co, g0


def _check(got, ref, steps, osteps, uhat, refhat, co, g0, dim):
    assert steps == osteps
    umax = max(np.abs(g).max() for g in g0)
    # per RK stage: the state update rounds once, the flux arithmetic a few tens of times at
    # values <= max|u| (entering multiplied by dt/h <= 1)
    tol = 64 * U32 * 3 * steps * umax
    for g, r in zip(got, ref):
        assert np.all(np.isfinite(g))
        err = np.max(np.abs(g.astype(np.float64) - r))
        assert err <= tol, (err, tol, err / (U32 * umax))
    # prolongation: d interpolation passes of the stepped grids (themselves within tol), summed
    # with |c_g| over the grids
    assert np.all(np.isfinite(uhat))
    tolc = (tol + 32 * U32 * dim * umax) * sum(abs(c) for c in co)
    errc = np.max(np.abs(uhat - refhat))
    assert errc <= tolc, (errc, tolc, errc / (U32 * umax))


@pytest.mark.parametrize("scale", [1e-3, 1.0, 30.0, 1e3])
@pytest.mark.parametrize("kernel", KERNELS, ids=lambda k: "d%d_nr%d_nl%d_pde%d_tp%d" % k)
def test_fp32_mixed_data_any_scale(sg, orc, kernel, scale):
    dim, nr, nl, pde, tile = kernel
    out = _run(orc, dim, nr, nl, pde, tile, "mixed", scale, 1e-3)
    _check(*out, dim)


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-8])
@pytest.mark.parametrize("kernel", KERNELS[:4] + KERNELS[5:6], ids=lambda k: "d%d_nr%d_nl%d_pde%d_tp%d" % k)
def test_fp32_smooth_small_differences_small_eps(sg, orc, kernel, eps):
    # smooth data of amplitude 1e-2: neighbouring differences ~1e-4, smoothness terms ~1e-8,
    # their squared products far below the float normal range unless rescaled
    dim, nr, nl, pde, tile = kernel
    out = _run(orc, dim, nr, nl, pde, tile, "smooth", 1e-2, eps)
    _check(*out, dim)


@pytest.mark.parametrize("eps", [1e-6, 1e-8])
@pytest.mark.parametrize("scale", [1.0, 1e3])
@pytest.mark.parametrize("tile", [SWEEP, SWEEP2])
def test_fp32_mixed_data_small_eps(sg, orc, scale, eps, tile):
    # jumps with a tiny eps: the smoothness terms of one interface span many decades
    out = _run(orc, 3, 6, 2, 1, tile, "mixed", scale, eps)
    _check(*out, 3)


@pytest.mark.parametrize("budget", [0.0, -1.0], ids=["one_pass", "grid_by_grid"])
@pytest.mark.parametrize("scale,eps", [(1e3, 1e-3), (1e-2, 1e-8), (1.0, 1e-6)])
def test_fp32_prolongation_any_scale(sg, orc, scale, eps, budget):
    dim, nr, nl = 3, 5, 2
    h = make(dim, nr, nl, P.SG_PDE_ADVECTION, precision=P.SG_F32, eps=eps, combine_budget_gb=budget)
    try:
        lev, shp, co = _levels(h, dim)
        g0 = [g.astype(np.float32).astype(np.float64)
              for g in random_grids(5, nr, lev, "mixed" if scale != 1e-2 else "smooth", scale=scale)]
        P.sg_init_grids(h, np.concatenate(g0).astype(np.float32))
        P.sg_prolong_combine(h)
        got = P.sg_read(h, P.SG_WHICH_COMBINED, count=(nr << nl) ** dim)
    finally:
        P.sg_destroy(h)
    ref = orc.combine(orc.problem(dim, nr, nl, pde=0, eps=eps), lev, co, g0)
    umax = max(np.abs(g).max() for g in g0)
    tol = 32 * U32 * dim * umax * sum(abs(c) for c in co)
    assert np.all(np.isfinite(got))
    err = np.max(np.abs(got - ref))
    assert err <= tol, (err, tol, err / (U32 * umax))
