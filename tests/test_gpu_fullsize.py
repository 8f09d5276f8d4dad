"""Parity at full workload sizes, through the C ABI, against the FP64 oracle.

* The 3-D and 4-D linear advection workloads (finest 512^3 and 256^4; 64 and 121 component
  grids): the first time steps of every grid bit for bit (FP64), the combined solution bit for
  bit at sampled finest-grid points (the full 256^4 FP64 solution is 34 GB, so it is gathered
  on the device at the sample), and the whole run to t = 0.5 in FP32 (batched, autotuned)
  against FP64 (plain per-grid launches): the same L1 error against the exact solution.
* Every row of the paper's tables stored in tests/golden (2-D and 3-D, single grids and sparse
  grids, both schemes and prolongations): the GPU FP64 path reproduces the printed L1 and
  L-infinity errors to the printed digits, as the oracle does; the FP32 path's L1 is within
  1.5x of FP64's where the discretisation error exceeds 1e-5 and within float rounding of it
  elsewhere.
"""
import json
import math
import os

import numpy as np
import pytest

import paper_2007_10196_gb300 as P
from paper_2007_10196_gb300 import inputs

from _helpers import make, read_grids, sine_grid

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def _levels(h, dim):
    G = P.sg_num_grids(h)
    info = [P.sg_grid_info(h, g, dim) for g in range(G)]
    return [i[0] for i in info], [i[1] for i in info], [i[2] for i in info]


def _sample(dim, Nf, m, seed):
    """m random finest-grid multi-indices plus the two corners (the periodic wrap)."""
    rng = np.random.default_rng(seed)
    J = rng.integers(0, Nf, size=(m, dim))
    J = np.vstack([J, np.zeros(dim, np.int64), np.full(dim, Nf - 1, np.int64)])
    flat = sum(J[:, k] * Nf ** k for k in range(dim))  # axis 0 fastest
    return J, flat


@pytest.mark.parametrize("name,nsteps", [("adv3d_nr8_nl6", 2), ("adv4d_nr8_nl5", 2)])
def test_full_size_first_steps_and_sampled_combination_fp64(sg, orc, name, nsteps):
    W = inputs.WORKLOADS[name]
    d, Nf = W.dim, W.nr << W.nl
    h = make(d, W.nr, W.nl, W.pde, dt_rule=W.dt_rule, dt_coef=W.dt_coef)
    try:
        lev, shp, coeff = _levels(h, d)
        g0 = [sine_grid(W.nr, l, W.lo, W.hi, W.ic) for l in lev]
        P.sg_init_grids(h, np.concatenate(g0))
        P.sg_step(h, W.t_end, nsteps)
        got = read_grids(h, [int(np.prod(s)) for s in shp])
        P.sg_prolong_combine(h)
        J, flat = _sample(d, Nf, 768, seed=d)
        uh = P.sg_read_points(h, P.SG_WHICH_COMBINED, flat)
    finally:
        P.sg_destroy(h)
    p = orc.problem(d, W.nr, W.nl, pde=W.pde, eps=1e-3, lo=W.lo, hi=W.hi)
    olev, oco = orc.grid_set(d, W.nl)
    assert [list(x) for x in olev] == [list(x) for x in lev] and list(oco) == list(coeff)
    ref, steps, _ = orc.solve(p, olev, g0, W.t_end, max_steps=nsteps, rule=W.dt_rule, coef=W.dt_coef)
    assert steps == nsteps
    for g, r in zip(got, ref):
        assert np.array_equal(g, r), np.max(np.abs(g - r))
    expect = orc.combine_points(p, olev, oco, ref, J)
    assert np.array_equal(uh, expect), np.max(np.abs(uh - expect))


@pytest.mark.parametrize("name", ["adv3d_nr8_nl6", "adv4d_nr8_nl5"])
def test_full_run_fp32_batched_matches_fp64_accuracy(sg, name):
    """The whole workload to t = 0.5: FP32 state (compensated), all grids in one persistent
    launch per stage with the autotuned kernel, against FP64 with one launch per grid."""
    W = inputs.WORKLOADS[name]
    d, Nf = W.dim, W.nr << W.nl
    _, flat = _sample(d, Nf, 4096, seed=10 + d)
    import time
    res = {}
    for prec, exe in ((P.SG_F64, P.SG_PLAIN), (P.SG_F32, P.SG_BATCHED)):
        h = make(d, W.nr, W.nl, W.pde, precision=prec, exec=exe, dt_rule=W.dt_rule, dt_coef=W.dt_coef)
        try:
            P.sg_init(h, P.SG_IC_SINE, W.ic)
            t0 = time.perf_counter()
            t = P.sg_step(h, W.t_end)
            t1 = time.perf_counter()
            assert t == W.t_end
            P.sg_prolong_combine(h)
            t2 = time.perf_counter()
            pts = sum(int(np.prod(x)) for x in _levels(h, d)[1])
            print("%s %s: %d points, %d steps, step %.2f s (%.3g point-updates/s, first call includes "
                  "autotuning), combine %.2f s" % (name, "f64 plain" if prec == P.SG_F64 else "f32 batched", pts,
                                                   P.sg_time(h)[1], t1 - t0, pts * P.sg_time(h)[1] / (t1 - t0),
                                                   t2 - t1))
            res[prec] = (P.sg_reduce(h, -1, P.SG_REDUCE_L1_EXACT), P.sg_reduce(h, -1, P.SG_REDUCE_LINF_EXACT),
                         P.sg_read_points(h, P.SG_WHICH_COMBINED, flat), P.sg_time(h)[1])
        finally:
            P.sg_destroy(h)
    l64, i64, s64, n64 = res[P.SG_F64]
    l32, i32, s32, n32 = res[P.SG_F32]
    assert n32 == n64
    # the sparse-grid solution converges: error far below the O(1) data
    assert 0 < l64 < 1e-2 and i64 < 1e-1
    # FP32 - FP64 bound: per step and axis the float flux difference carries at most
    # 16 u32 max|u| / h of rounding, i.e. 16 u32 dt/h in the state; summed over the steps,
    # axes and three stages without cancellation, plus the initial rounding, and amplified by
    # sum |c_g| = 2^(d-1) in the combination
    h = (W.hi - W.lo) / Nf
    dt = W.dt_coef * h ** (5.0 / 3.0)
    tol = 2 ** (d - 1) * (64 * U32 + n64 * d * 3 * 16 * U32 * dt / h)
    assert np.max(np.abs(s32 - s64)) <= tol, (np.max(np.abs(s32 - s64)), tol)
    assert abs(l32 - l64) <= tol
    if l64 > 1e-5:
        assert l64 / 1.5 <= l32 <= 1.5 * l64, (l32, l64)


def _rows():
    with open(GOLDEN) as fh:
        return json.load(fh)["rows"]


@pytest.mark.parametrize("row", _rows(), ids=lambda r: r["cite"])
def test_paper_table_rows_on_gpu(sg, row):
    dim, nr, nl, T = row["dim"], row["nr"], row["nl"], row["T"]
    pde = P.SG_PDE_BURGERS if row["pde"] == "burgers" else P.SG_PDE_ADVECTION
    scheme = P.SG_LINEAR5 if row["scheme"] == "linear" else P.SG_WENO5
    prol = P.SG_PROLONG_LAGRANGE5 if row["prolong"] == "lagrange" else P.SG_PROLONG_WENO5
    lo, hi = row["domain"]
    b, a, w = row["ic"]
    res = {}
    for prec, exe in ((P.SG_F64, P.SG_PLAIN), (P.SG_F32, P.SG_BATCHED)):
        h = make(dim, nr, nl, pde, precision=prec, exec=exe, scheme=scheme, prolong=prol,
                 lo=[lo] * 6, hi=[hi] * 6)
        try:
            P.sg_init(h, P.SG_IC_SINE, (b, a, w, 0.0))
            assert P.sg_step(h, T) == T
            P.sg_prolong_combine(h)
            res[prec] = (P.sg_reduce(h, -1, P.SG_REDUCE_L1_EXACT), P.sg_reduce(h, -1, P.SG_REDUCE_LINF_EXACT))
        finally:
            P.sg_destroy(h)
    l64, i64 = res[P.SG_F64]
    l32, _ = res[P.SG_F32]
    if row["exact_digits"]:
        for ours, printed in ((l64, row["l1"]), (i64, row["linf"])):
            unit = 10.0 ** (math.floor(math.log10(printed)) - (row["exact_digits"] - 1))
            assert abs(ours - printed) <= 0.5 * unit * (1 + 1e-9), (ours, printed)
    else:
        f = row["loose"]
        assert row["l1"] / f <= l64 <= row["l1"] * f
        assert row["linf"] / f <= i64 <= row["linf"] * f
    if l64 > 1e-5:
        assert l64 / 1.5 <= l32 <= 1.5 * l64, (l32, l64)
    else:
        assert abs(l32 - l64) <= 64 * U32 * (abs(b) + abs(a)) * (2 ** (dim - 1)), (l32, l64)


def test_example4_shock_sparse_vs_single_grid(sg):
    """Example 4 (Section 3): 3-D Burgers, u0 = 0.3 + 0.7 sin(x + y + z) on [0, 2pi]^3 to
    T = 0.52 (after the shocks form), CFL 0.4, WENO prolongation; sparse N_r = 40, N_L = 3 and
    the 320^3 single grid.  Checks what the paper shows for it: every component grid conserves
    its mass, the solutions stay within the data's range up to a small shock overshoot, and the
    sparse-grid solution is close to the single-grid one.  Prints the run times (the paper:
    17893.4 s sparse, 86549.8 s single, on one CPU core)."""
    import time
    two_pi = 2 * math.pi
    ic = (0.3, 0.7, 1.0, 0.0)
    kw = dict(lo=[0.0] * 6, hi=[two_pi] * 6, dt_rule=P.SG_DT_CFL, cfl=0.4)
    Nf = 320
    _, flat = _sample(3, Nf, 200000, seed=4)
    res = {}
    for name, nr, nl, prec, exe in (("sparse_f64", 40, 3, P.SG_F64, P.SG_PLAIN),
                                    ("sparse_f32", 40, 3, P.SG_F32, P.SG_BATCHED),
                                    ("single_f32", 320, 0, P.SG_F32, P.SG_BATCHED)):
        h = make(3, nr, nl, P.SG_PDE_BURGERS, precision=prec, exec=exe, **kw)
        try:
            P.sg_init(h, P.SG_IC_SINE, ic)
            G = P.sg_num_grids(h)
            m0 = [P.sg_reduce(h, g, P.SG_REDUCE_MASS) for g in range(G)]
            t0 = time.perf_counter()
            t = P.sg_step(h, 0.52)
            step_s = time.perf_counter() - t0
            assert t == 0.52
            m1 = [P.sg_reduce(h, g, P.SG_REDUCE_MASS) for g in range(G)]
            t0 = time.perf_counter()
            P.sg_prolong_combine(h)
            comb_s = time.perf_counter() - t0
            lo_, hi_ = P.sg_reduce(h, -1, P.SG_REDUCE_MIN), P.sg_reduce(h, -1, P.SG_REDUCE_MAX)
            res[name] = P.sg_read_points(h, P.SG_WHICH_COMBINED, flat)
            print("example4 %s: %d grids, %d steps, step %.3f s, combine %.3f s, range [%.4f, %.4f]"
                  % (name, G, P.sg_time(h)[1], step_s, comb_s, lo_, hi_))
        finally:
            P.sg_destroy(h)
        vol = two_pi ** 3
        for a, b in zip(m0, m1):  # conservative update on a periodic grid
            assert abs(a - b) <= (1e-12 if prec == P.SG_F64 else 1e-5) * vol
        assert abs(m0[0] - 0.3 * vol) < 1e-6 * vol
        # WENO keeps a single grid within the data's range [-0.4, 1] up to a small overshoot;
        # the signed combination of grids that resolve the shock differently may add more
        slack = 0.05 if nl == 0 else 0.3
        assert -0.4 - slack <= lo_ and hi_ <= 1.0 + slack
    # sparse vs single grid: close away from the shocks, in the mean
    assert np.mean(np.abs(res["sparse_f64"] - res["single_f32"])) < 0.02
    assert np.mean(np.abs(res["sparse_f32"] - res["sparse_f64"])) < 1e-5
