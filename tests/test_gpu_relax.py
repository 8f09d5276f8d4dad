"""The Vlasov-Boltzmann relaxation model (Example 5) on the GPU against the FP64 oracle.

f_t + v . grad_x f - x . grad_v f = (mu_inf(v) rho(x) - f) / tau on [-5, 5]^{2d}, zero
boundaries, d = 1 (2-D phase space) and d = 2 (4-D).  FP64: bit for bit after several CFL
steps (plain and batched execution, several tiles, theta and tau away from 1) and through the
combination (one pass and grid by grid); FP32 within derived tolerances; the initial-condition
kernel and the entropy reductions; and the paper's two runs: (a) N_r = 40, N_L = 3 against the
320^2 single grid (the entropy functionals decay alike) and (b) N_r = 10, N_L = 3 in 4-D against
the 80^4 single grid, with their GPU times beside the paper's CPU times.
"""
import math
import time

import numpy as np
import pytest

import paper_2007_10196_gb300 as P

from _helpers import make, read_grids

pytestmark = pytest.mark.gpu

LO, HI = -5.0, 5.0
U32 = 2.0 ** -24


def _levels(h, dim):
    G = P.sg_num_grids(h)
    info = [P.sg_grid_info(h, g, dim) for g in range(G)]
    return [i[0] for i in info], [i[1] for i in info], [i[2] for i in info]


def _orc_p(orc, dim, nr, nl, theta=1.0, tau=1.0):
    return orc.problem(dim, nr, nl, pde=orc.VLASOV_BOLTZMANN, eps=1e-3, lo=LO, hi=HI, theta=theta, tau=tau)


def _make(dim, nr, nl, prec=P.SG_F64, exe=P.SG_PLAIN, tp=0, **kw):
    return make(dim, nr, nl, P.SG_PDE_VLASOV_BOLTZMANN, precision=prec, exec=exe, tile_points=tp, lo=LO, hi=HI,
                dt_rule=P.SG_DT_CFL, cfl=0.4, **kw)


def _run(orc, dim, nr, nl, prec, exe, tp, nsteps, theta=1.0, tau=1.0, budget=0.0):
    h = _make(dim, nr, nl, prec, exe, tp, theta=theta, tau=tau, combine_budget_gb=budget)
    try:
        lev, shp, co = _levels(h, dim)
        p = _orc_p(orc, dim, nr, nl, theta, tau)
        s = orc.relax_norm(p)
        g0 = [orc.restrict_relax(p, l, s) for l in lev]
        if prec == P.SG_F32:
            g0 = [g.astype(np.float32).astype(np.float64) for g in g0]
        P.sg_init_grids(h, np.concatenate(g0))
        t = P.sg_step(h, 100.0, nsteps)
        got = read_grids(h, [int(np.prod(s)) for s in shp])
        P.sg_prolong_combine(h)
        uh = P.sg_read(h, P.SG_WHICH_COMBINED, count=(nr << nl) ** dim)
        steps = P.sg_time(h)[1]
    finally:
        P.sg_destroy(h)
    ref, osteps, ot = orc.solve(p, lev, g0, 100.0, max_steps=nsteps, rule=orc.DT_CFL, cfl=0.4)
    return dict(lev=lev, co=co, p=p, got=got, uh=uh, t=t, steps=steps, ref=ref, osteps=osteps, ot=ot)


CASES = [(2, 8, 2, P.SG_PLAIN, 256, 1.0, 1.0), (2, 8, 2, P.SG_BATCHED, 512, 1.5, 0.5),
         (2, 10, 3, P.SG_BATCHED, 1024, 1.0, 1.0), (2, 6, 3, P.SG_PLAIN, 0, 0.8, 2.0),
         (4, 6, 2, P.SG_BATCHED, 256, 1.0, 1.0), (4, 5, 1, P.SG_PLAIN, 512, 1.5, 0.5)]


@pytest.mark.parametrize("dim,nr,nl,exe,tp,theta,tau", CASES, ids=lambda c: str(c))
def test_relax_steps_and_combination_fp64_bitwise(sg, orc, dim, nr, nl, exe, tp, theta, tau):
    r = _run(orc, dim, nr, nl, P.SG_F64, exe, tp, 3, theta, tau)
    assert r["steps"] == r["osteps"] == 3 and r["t"] == r["ot"]
    for g, ref in zip(r["got"], r["ref"]):
        assert np.array_equal(g, ref), np.max(np.abs(g - ref))
    expect = orc.combine(r["p"], r["lev"], r["co"], r["ref"])
    assert np.array_equal(r["uh"], expect), np.max(np.abs(r["uh"] - expect))


@pytest.mark.parametrize("dim,nr,nl", [(2, 8, 3), (4, 5, 2)])
def test_relax_combination_grid_by_grid_fp64_bitwise(sg, orc, dim, nr, nl):
    r = _run(orc, dim, nr, nl, P.SG_F64, P.SG_BATCHED, 0, 2, budget=-1.0)
    assert np.array_equal(r["uh"], orc.combine(r["p"], r["lev"], r["co"], r["ref"]))


@pytest.mark.parametrize("dim,nr,nl,exe,tp,theta,tau", CASES[1:3] + CASES[4:5], ids=lambda c: str(c))
def test_relax_steps_fp32_within_tolerance(sg, orc, dim, nr, nl, exe, tp, theta, tau):
    r = _run(orc, dim, nr, nl, P.SG_F32, exe, tp, 4, theta, tau)
    assert r["steps"] == r["osteps"]
    # |f| <= 0.5: 64 float roundings per stage on the state scale, three stages per step; the
    # relaxation term adds a few roundings of mu rho (~ |f|) per stage
    tol = 80 * U32 * 3 * r["steps"] * 0.5
    for g, ref in zip(r["got"], r["ref"]):
        assert np.max(np.abs(g.astype(np.float64) - ref)) <= tol
    expect = orc.combine(r["p"], r["lev"], r["co"], r["ref"])
    assert np.max(np.abs(r["uh"] - expect)) <= 2 * tol


@pytest.mark.parametrize("dim,nr,nl", [(2, 8, 3), (4, 5, 2)])
def test_relax_initial_condition_and_entropy_reductions(sg, orc, dim, nr, nl):
    """SG_IC_RELAX (device sin/cos/exp, the library's own normalisation) against the oracle's
    restriction; the entropy functionals of a grid and of the combined solution against the
    oracle's (device exp/log: relative 1e-12)."""
    h = _make(dim, nr, nl)
    try:
        lev, shp, co = _levels(h, dim)
        P.sg_init(h, P.SG_IC_RELAX, ())
        got = read_grids(h, [int(np.prod(s)) for s in shp])
        P.sg_prolong_combine(h)
        uh = P.sg_read(h, P.SG_WHICH_COMBINED, count=(nr << nl) ** dim)
        red = {(w, k): P.sg_reduce(h, w, k) for w in (-1, 0, len(lev) - 1)
               for k in (P.SG_REDUCE_ENTROPY_H2, P.SG_REDUCE_ENTROPY_LOG)}
    finally:
        P.sg_destroy(h)
    p = _orc_p(orc, dim, nr, nl)
    ref = [orc.restrict_relax(p, l) for l in lev]
    for g, r in zip(got, ref):
        assert np.max(np.abs(g - r)) <= 1e-13 * np.max(np.abs(r))
    pf = _orc_p(orc, dim, nr << nl, 0)
    for w, arr, lv, pp in ((-1, uh, [0] * dim, pf), (0, got[0], lev[0], p), (len(lev) - 1, got[-1], lev[-1], p)):
        h2, hl = orc.relax_entropy(pp, lv, arr)
        assert abs(red[(w, P.SG_REDUCE_ENTROPY_H2)] - h2) <= 1e-12 * abs(h2)
        assert abs(red[(w, P.SG_REDUCE_ENTROPY_LOG)] - hl) <= 1e-12 * max(abs(hl), 1e-3)


def test_relax_arguments(sg):
    """dim must be even, the IC needs dim 2 or 4, the entropy needs the model, tau > 0."""
    with pytest.raises(P.SgError):
        _make(3, 8, 1)
    with pytest.raises(P.SgError):
        _make(2, 8, 1, tau=0.0)
    h = _make(6, 5, 0)
    try:
        with pytest.raises(P.SgError):
            P.sg_init(h, P.SG_IC_RELAX, ())
    finally:
        P.sg_destroy(h)
    h = make(2, 8, 1, P.SG_PDE_BURGERS)
    try:
        P.sg_init(h, P.SG_IC_SINE, (0.5, 1.0, math.pi / 2, 0.0))
        with pytest.raises(P.SgError):
            P.sg_reduce(h, 0, P.SG_REDUCE_ENTROPY_H2)
    finally:
        P.sg_destroy(h)


def _evolve(dim, nr, nl, times, prec=P.SG_F32):
    """Runs Example 5 to each time in `times`; returns (H2, Hlog, mass, cumulative step seconds,
    steps) of the combined solution at each, and the handle's point count."""
    h = _make(dim, nr, nl, prec, P.SG_BATCHED)
    out = []
    try:
        P.sg_init(h, P.SG_IC_RELAX, ())
        pts = sum(int(np.prod(s)) for s in _levels(h, dim)[1])
        P.sg_step(h, 1e-9, 1)  # one 1e-9 step: the autotuner and the graph capture run outside the timing
        t_step = 0.0
        for t in times:
            t0 = time.perf_counter()
            P.sg_step(h, t)
            t_step += time.perf_counter() - t0
            P.sg_prolong_combine(h)
            out.append((P.sg_reduce(h, -1, P.SG_REDUCE_ENTROPY_H2), P.sg_reduce(h, -1, P.SG_REDUCE_ENTROPY_LOG),
                        P.sg_reduce(h, -1, P.SG_REDUCE_MASS), t_step, P.sg_time(h)[1]))
    finally:
        P.sg_destroy(h)
    return out, pts


def test_relax_example5a_sparse_vs_single_grid(sg):
    """Example 5 (a): N_r = 40, N_L = 3 (finest 320^2) against the 320^2 single grid, CFL 0.4,
    FP32 batched.  Both entropy functionals decrease towards equilibrium and the sparse-grid
    curves follow the single-grid ones (the paper's Figure: 'agree very well'); mass stays 1
    up to the outflow through |x|, |v| = 5."""
    times = [0.5, 1.0, 2.0, 3.0, 6.0]
    sp, sp_pts = _evolve(2, 40, 3, times)
    si, si_pts = _evolve(2, 320, 0, times)
    for t, a, b in zip(times, sp, si):
        print("example5a t=%.1f sparse H2 %.6f Hlog %.6f mass %.6f (%.3f s, %d steps) | single H2 %.6f Hlog %.6f "
              "mass %.6f (%.3f s)" % (t, a[0], a[1], a[2], a[3], a[4], b[0], b[1], b[2], b[3]))
    print("example5a points: sparse %d, single %d" % (sp_pts, si_pts))
    for run in (sp, si):
        assert all(y[0] < x[0] and y[1] < x[1] for x, y in zip(run, run[1:]))
        assert all(abs(x[2] - 1.0) < 1e-3 for x in run)
    for a, b in zip(sp, si):  # distance from equilibrium (H2 -> 1, Hlog -> 0) agrees within 10%
        assert abs((a[0] - 1.0) - (b[0] - 1.0)) <= 0.1 * abs(b[0] - 1.0) + 1e-4
        assert abs(a[1] - b[1]) <= 0.1 * abs(b[1]) + 1e-4


def _cut(h, dim, n):
    """The x1-v1 plane through x2 = v2 = 0 of the combined 4-D solution (n^4 finest nodes;
    node n/2 is 0 on [-5, 5)), read at sample points on the device."""
    i = np.arange(n)
    I1, I3 = np.meshgrid(i, i, indexing="ij")
    idx = I1 + n * (n // 2) + n * n * I3 + n ** 3 * (n // 2)
    return P.sg_read_points(h, P.SG_WHICH_COMBINED, idx.reshape(-1)).reshape(n, n)


def test_relax_example5b_4d_sparse_vs_single_grid(sg):
    """Example 5 (b): 4-D, N_r = 10, N_L = 3 (finest 80^4) to t = 3, and the 80^4 single grid to
    t = 0.5 (FP32 batched).  The paper compares 2-D cuts of f.  The combined initial condition
    matches the single grid's to a fraction of a percent, but after the evolution the x1-v1
    cuts through x2 = v2 = 0 differ by about 10% of the cut's maximum: the component grids are
    coarse (10 nodes, h = 1, on the axes at level 0) for a solution that rotates in phase
    space.  A sparse set with finer component grids and the same finest grid (N_r = 20,
    N_L = 2) comes closer, which attributes the gap to the resolution of the components (the
    FP64 path matches the oracle bit for bit in 4-D).  H_log agrees within 10%, decays, and the
    mass stays near 1.  (H_2 = sum f^2 / M of the sparse solution is dominated by the
    combination's small values at the corners, where M ~ e^{-50}: printed, not compared.)"""
    times = [0.5, 1.0, 2.0, 3.0]
    res = {}
    for name, nr, nl, ts in (("sparse", 10, 3, times), ("sparse_nr20_nl2", 20, 2, times[:1]),
                             ("single", 80, 0, times[:1])):
        h = _make(4, nr, nl, P.SG_F32, P.SG_BATCHED)
        out = []
        try:
            P.sg_init(h, P.SG_IC_RELAX, ())
            pts = sum(int(np.prod(s)) for s in _levels(h, 4)[1])
            P.sg_prolong_combine(h)
            cut0 = _cut(h, 4, 80)
            P.sg_step(h, 1e-9, 1)  # one 1e-9 step: the autotuner and the graph capture run outside the timing
            t_step, cut = 0.0, None
            for t in ts:
                t0 = time.perf_counter()
                P.sg_step(h, t)
                t_step += time.perf_counter() - t0
                P.sg_prolong_combine(h)
                if t == 0.5:
                    cut = _cut(h, 4, 80)
                out.append((P.sg_reduce(h, -1, P.SG_REDUCE_ENTROPY_H2), P.sg_reduce(h, -1, P.SG_REDUCE_ENTROPY_LOG),
                            P.sg_reduce(h, -1, P.SG_REDUCE_MASS), t_step, P.sg_time(h)[1]))
        finally:
            P.sg_destroy(h)
        res[name] = (out, pts, cut, cut0)
        for t, a in zip(ts, out):
            print("example5b %s t=%.1f H2 %.6g Hlog %.6f mass %.6f (%.3f s, %d steps)" % ((name, t) + a))
        print("example5b %s points %d" % (name, pts))
    sp, si = res["sparse"][0], res["single"][0]
    def rel(name, j):
        cs, cg = res[name][j], res["single"][j]
        return np.max(np.abs(cs - cg)) / np.max(np.abs(cg))

    r0, r5, rf = rel("sparse", 3), rel("sparse", 2), rel("sparse_nr20_nl2", 2)
    print("example5b x1-v1 cut: max|sparse - single| / max|single| = %.4f at t = 0, %.4f at t = 0.5; "
          "N_r = 20, N_L = 2: %.4f at t = 0.5" % (r0, r5, rf))
    assert r0 < 0.01 and r5 < 0.2 and rf < r5
    assert all(y[1] < x[1] for x, y in zip(sp, sp[1:]))
    assert all(abs(x[2] - 1.0) < 2e-3 for x in sp + si)
    assert abs(sp[0][1] - si[0][1]) <= 0.1 * abs(si[0][1])
