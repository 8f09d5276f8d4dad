"""Pins of the oracle's zero boundary for advection and Burgers (the zero boundary treatment
of Example 5 applied to Eq. (1); u = 0 at the ghost nodes beyond x_0 and x_{n-1}).

Each check reaches the oracle's zero-boundary operator through something other than itself:
- data supported away from the boundary: the zero-boundary operator, RK3 step and combination
  must equal the (separately pinned) periodic ones bit for bit, since every stencil then sees
  the same values;
- the flux difference telescopes: per line, sum_j L_j h = F_{-1/2} - F_{n-1/2}, with the two
  boundary fluxes formed here from the WENO5 side function (pinned by Tables 3-6 and the
  closed forms) on the explicit ghost stencils;
- a smooth pulse advected out through the boundary converges to the exact translate
  u_0(x - a t) restricted to the domain, and the mass left in the domain tracks the exact one;
- zero data stay zero.
A sign or index slip in the ghost handling (a wrapped neighbour, a dropped boundary interface,
the mirror stencil shifted by one) fails one of them.
"""
import numpy as np
import pytest

import oracle as O


def _bump(x, c, w, p=8):
    z = (x - c) / w
    return np.where(np.abs(z) < 1.0, (1.0 - z * z) ** p, 0.0)


def _grid_values(nx, f, lo, hi):
    """f(x_0, x_1, ...) at the nodes lo + j h, j < n (axis 0 fastest, flat)."""
    xs = [lo[k] + np.arange(n) * ((hi[k] - lo[k]) / n) for k, n in enumerate(nx)]
    X = np.meshgrid(*xs, indexing="ij")
    v = f(*X)
    return np.ascontiguousarray(v.transpose(tuple(reversed(range(len(nx))))).reshape(-1))


@pytest.mark.parametrize("pde", [O.ADVECTION, O.BURGERS])
def test_interior_support_equals_periodic(pde):
    dim, nr = 2, 40
    lev = np.array([0, 0], np.int32)
    f = lambda x, y: _bump(x, 2.0, 0.5) * _bump(y, 2.1, 0.6)
    u = _grid_values((nr, nr), f, (0.0, 0.0), (4.0, 4.0))
    pz = O.problem(dim, nr, 0, pde=pde, eps=1e-3, adv=(1.0, -0.6), bc=O.BC_ZERO)
    pp = O.problem(dim, nr, 0, pde=pde, eps=1e-3, adv=(1.0, -0.6), bc=O.BC_PERIODIC)
    assert np.array_equal(O.spatial_operator(pz, lev, u), O.spatial_operator(pp, lev, u))
    # one RK3 step spreads the support by at most 9 nodes: still 3 away from either end
    assert np.array_equal(O.rk3_step(pz, lev, u, 0.02), O.rk3_step(pp, lev, u, 0.02))


def test_interior_support_combination_equals_periodic():
    dim, nr, nl = 2, 16, 2
    lev, co = O.grid_set(dim, nl)
    f = lambda x, y: _bump(x, 2.0, 0.9) * _bump(y, 1.9, 0.8)
    grids = [_grid_values(tuple(nr << int(l) for l in lv), f, (0.0, 0.0), (4.0, 4.0)) for lv in lev]
    for prolong in (O.PROLONG_WENO5, O.PROLONG_LAGRANGE5):
        pz = O.problem(dim, nr, nl, prolong=prolong, eps=1e-3, bc=O.BC_ZERO)
        pp = O.problem(dim, nr, nl, prolong=prolong, eps=1e-3, bc=O.BC_PERIODIC)
        assert np.array_equal(O.combine(pz, lev, co, grids), O.combine(pp, lev, co, grids))


def _boundary_fluxes(fp, fm, eps, linear=False):
    """F_{-1/2} and F_{n-1/2} of one line from its split values, ghosts zero."""
    z = 0.0
    F_left = (O.weno5_side(z, z, z, fp[0], fp[1], eps, linear)
              + O.weno5_side(fm[2], fm[1], fm[0], z, z, eps, linear))
    F_right = (O.weno5_side(fp[-3], fp[-2], fp[-1], z, z, eps, linear)
               + O.weno5_side(z, z, z, fm[-1], fm[-2], eps, linear))
    return F_left, F_right


@pytest.mark.parametrize("pde,scheme", [(O.ADVECTION, O.WENO5), (O.BURGERS, O.WENO5), (O.BURGERS, O.LINEAR5)])
def test_flux_difference_telescopes_to_boundary_fluxes(pde, scheme):
    # 2-D, axis 0 zero and axis 1 periodic: summed over the grid, the axis-1 differences cancel
    # and the axis-0 ones leave F_{-1/2} - F_{n-1/2} of every axis-0 line
    rng = np.random.default_rng(5)
    n, lo, hi, eps, adv = 13, (0.0, -1.0), (2.0, 1.5), 1e-3, (0.7, -1.3)
    p = O.problem(2, n, 0, pde=pde, scheme=scheme, eps=eps, adv=adv, lo=lo, hi=hi,
                  bc=(O.BC_ZERO, O.BC_PERIODIC))
    u = rng.uniform(-1.0, 1.5, size=n * n)
    L = O.spatial_operator(p, np.array([0, 0], np.int32), u)
    U = u.reshape(n, n)  # [j (axis 1), i (axis 0)]
    alpha = np.abs(U).max() if pde == O.BURGERS else abs(adv[0])
    tot = 0.0
    for j in range(n):
        line = U[j]
        f = 0.5 * line * line if pde == O.BURGERS else adv[0] * line
        Fl, Fr = _boundary_fluxes(0.5 * (f + alpha * line), 0.5 * (f - alpha * line), eps, scheme == O.LINEAR5)
        tot += Fl - Fr
    h0 = (hi[0] - lo[0]) / n
    assert abs(L.sum() * h0 - tot) <= 1e-13 * np.abs(L).sum() * h0
    assert abs(tot) > 1e-2


@pytest.mark.parametrize("pde", [O.ADVECTION, O.BURGERS])
def test_flux_difference_telescopes_1d(pde):
    rng = np.random.default_rng(9)
    n, lo, hi, eps = 11, -1.0, 2.0, 1e-3
    u = rng.uniform(-1.0, 1.0, size=n)
    p = O.problem(1, n, 0, pde=pde, eps=eps, adv=-0.8, lo=lo, hi=hi, bc=O.BC_ZERO)
    L = O.spatial_operator(p, np.array([0], np.int32), u)
    alpha = np.abs(u).max() if pde == O.BURGERS else 0.8
    f = 0.5 * u * u if pde == O.BURGERS else -0.8 * u
    Fl, Fr = _boundary_fluxes(0.5 * (f + alpha * u), 0.5 * (f - alpha * u), eps)
    h = (hi - lo) / n
    assert abs(L.sum() * h - (Fl - Fr)) <= 1e-13 * np.abs(L).sum() * h
    # and the periodic operator on the same data telescopes to zero instead
    pp = O.problem(1, n, 0, pde=pde, eps=eps, adv=-0.8, lo=lo, hi=hi)
    Lp = O.spatial_operator(pp, np.array([0], np.int32), u)
    assert abs(Lp.sum() * h) <= 1e-13 * np.abs(Lp).sum() * h
    assert abs(Fl - Fr) > 1e-3  # the boundary fluxes of this data are far from cancelling


def test_zero_data_stay_zero():
    lev = np.array([1, 0, 2], np.int32)
    for pde in (O.ADVECTION, O.BURGERS):
        p = O.problem(3, 6, 2, pde=pde, eps=1e-6, bc=O.BC_ZERO)
        u = np.zeros(O.state_points(p, lev))
        assert not np.any(O.rk3_step(p, lev, u, 0.01))


def _outflow_run(n, t_end):
    """1-D advection a = 1 on [0, 1], zero boundary, a smooth pulse crossing x = 1."""
    lo, hi = 0.0, 1.0
    p = O.problem(1, n, 0, pde=O.ADVECTION, eps=1e-6, adv=1.0, lo=lo, hi=hi, bc=O.BC_ZERO)
    x = lo + np.arange(n) * ((hi - lo) / n)
    u0 = _bump(x, 0.75, 0.2)
    lev = [np.array([0], np.int32)]
    out, steps, t = O.solve(p, lev, [u0], t_end, rule=O.DT_CFL, cfl=0.4)
    exact = _bump(x - t, 0.75, 0.2)
    h = (hi - lo) / n
    return np.abs(out[0] - exact).sum() * h, out[0].sum() * h, exact.sum() * h


def test_outflow_converges_to_exact_translate():
    # the pulse (support [0.55, 0.95]) is half outside the domain at t = 0.2
    errs = []
    for n in (80, 160, 320):
        e, m, me = _outflow_run(n, 0.2)
        errs.append(e)
        assert abs(m - me) <= 2 * e + 1e-14
    assert errs[0] / errs[1] > 6.0 and errs[1] / errs[2] > 6.0, errs
    assert errs[2] < 3e-6, errs


def test_outflow_2d_sparse_combination_converges():
    # oblique advection out through two faces; the combined solution against the exact translate
    errs = []
    for nr in (10, 20, 40):
        dim, nl = 2, 2
        lev, co = O.grid_set(dim, nl)
        p = O.problem(dim, nr, nl, pde=O.ADVECTION, eps=1e-6, adv=(1.0, 0.5), lo=0.0, hi=1.0, bc=O.BC_ZERO)
        f = lambda x, y: _bump(x, 0.7, 0.25) * _bump(y, 0.7, 0.25)
        g0 = [_grid_values(tuple(nr << int(l) for l in lv), f, (0.0, 0.0), (1.0, 1.0)) for lv in lev]
        out, steps, t = O.solve(p, lev, g0, 0.15, rule=O.DT_CFL, cfl=0.4)
        uh = O.combine(p, lev, co, out)
        nf = nr << nl
        ex = _grid_values((nf, nf), lambda x, y: _bump(x - t, 0.7, 0.25) * _bump(y - 0.5 * t, 0.7, 0.25),
                          (0.0, 0.0), (1.0, 1.0))
        errs.append(np.abs(uh - ex).mean())
    assert errs[0] / errs[1] > 4.0 and errs[1] / errs[2] > 4.0, errs
