"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here retypes an oracle formula.  Each test derives its expectation another way:
values printed in the paper's tables (tests/golden/paper_tables.json), Fourier closed
forms of the linear scheme and of Lagrange prolongation, first-principles constructions
of the WENO5 reconstruction and interpolation from their definitions (cell-average /
point-value interpolation, the smoothness integral of Eq. (10)), the printed combination
formulas (12), (14), (15), brute-force enumeration, invariants and special cases.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")
EPS = 1e-3  # epsilon of Eqs. (5) and (9); pinned by test_paper_table_rows


# --------------------------------------------------------------------------------------
# helpers written from the mathematics (not from the oracle)
# --------------------------------------------------------------------------------------
def _cell_avg_matrix(cells, deg):
    """Rows: cell averages over [j-1/2, j+1/2] (unit spacing) of x^p, p = 0..deg."""
    M = np.zeros((len(cells), deg + 1))
    for r, j in enumerate(cells):
        for p in range(deg + 1):
            M[r, p] = ((j + 0.5) ** (p + 1) - (j - 0.5) ** (p + 1)) / (p + 1)
    return M


def _point_matrix(nodes, deg):
    return np.array([[float(x) ** p for p in range(deg + 1)] for x in nodes])


def _smoothness(coef):
    """sum_{l=1,2} int_{-1/2}^{1/2} (p^{(l)}(x))^2 dx for p = sum coef_p x^p (h = 1), Eq. (10)."""
    P = np.polynomial.Polynomial(coef)
    tot = 0.0
    for l in (1, 2):
        d = P.deriv(l)
        I = (d * d).integ()
        tot += I(0.5) - I(-0.5)
    return tot


def _weno_reconstruct_first_principles(f, eps, linear):
    """fhat_{i+1/2} from Shu's finite-volume view of the finite-difference flux: the
    values f_{i-2..i+2} are cell averages of a function whose value at x_{i+1/2} is
    reconstructed.  Candidates are the quadratics matching three averages; the linear
    weights make their combination equal the quartic matching all five; beta_r is the
    smoothness integral over cell i."""
    f = np.asarray(f, dtype=np.float64)
    cells = [-2, -1, 0, 1, 2]
    q, beta, rows = [], [], []
    for r in range(3):
        sub = cells[r:r + 3]
        M = _cell_avg_matrix(sub, 2)
        Minv = np.linalg.inv(M)
        coef = Minv @ f[r:r + 3]
        row = np.zeros(5)
        row[r:r + 3] = np.array([0.5 ** p for p in range(3)]) @ Minv
        rows.append(row)
        q.append(float(row @ f))
        beta.append(_smoothness(coef))
    big = np.array([0.5 ** p for p in range(5)]) @ np.linalg.inv(_cell_avg_matrix(cells, 4))
    d, *_ = np.linalg.lstsq(np.array(rows).T, big, rcond=None)
    if linear:
        a = d
    else:
        a = np.array([d[r] / (eps + beta[r]) ** 2 for r in range(3)])
    return float(np.dot(a, q) / a.sum()), d


def _weno_interp_first_principles(v, s, eps, lagrange):
    """Point-value WENO interpolation at x = s (nodes -2..2): P_k quadratics through the
    substencils, C_k(s) the weights making sum C_k P_k equal the quartic interpolant,
    beta_k from Eq. (10)."""
    v = np.asarray(v, dtype=np.float64)
    nodes = [-2, -1, 0, 1, 2]
    P, beta, rows = [], [], []
    for k in range(3):
        Minv = np.linalg.inv(_point_matrix(nodes[k:k + 3], 2))
        coef = Minv @ v[k:k + 3]
        row = np.zeros(5)
        row[k:k + 3] = np.array([s ** p for p in range(3)]) @ Minv
        rows.append(row)
        P.append(float(row @ v))
        beta.append(_smoothness(coef))
    big = np.array([s ** p for p in range(5)]) @ np.linalg.inv(_point_matrix(nodes, 4))
    C, *_ = np.linalg.lstsq(np.array(rows).T, big, rcond=None)
    w = C if lagrange else np.array([C[k] / (eps + beta[k]) ** 2 for k in range(3)])
    return float(np.dot(w, P) / w.sum()), C


def _rk3_amplification(z):
    # a three-stage, third-order explicit RK method applied to u' = lambda u is exact through z^3
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0


def _upwind5_symbol(theta):
    """Linear-weight flux fhat_{i+1/2} = sum_m c_m u_{i+m} for a positive wind, from the
    first-principles reconstruction above; returns F(theta) with fhat = F(theta) e^{i theta i}."""
    _, d = _weno_reconstruct_first_principles(np.zeros(5), 1.0, True)
    # coefficients of the linear combination on u_{i-2..i+2}
    cells = [-2, -1, 0, 1, 2]
    coef = np.array([0.5 ** p for p in range(5)]) @ np.linalg.inv(_cell_avg_matrix(cells, 4))
    return sum(coef[m] * np.exp(1j * theta * (m - 2)) for m in range(5)), coef


def _advection_mode_factor(theta, h, a):
    """lambda with L u = lambda u for u_j = e^{i theta j} and flux a u, LF split with alpha=|a|.
    Positive part uses the upwind stencil; the negative part its mirror image about x_{i+1/2}."""
    F, coef = _upwind5_symbol(theta)
    if a >= 0:
        fh = a * F
    else:
        # mirror: fhat_{i+1/2} = a * sum_m coef[m] u_{i+1-(m-2)}
        fh = a * sum(coef[m] * np.exp(1j * theta * (1 - (m - 2))) for m in range(5))
    return -(1.0 - np.exp(-1j * theta)) * fh / h


def _march(lmb, T, dt):
    A, t = 1.0 + 0j, 0.0
    n = 0
    while t < T:
        d = min(dt, T - t)
        A *= _rk3_amplification(d * lmb)
        t = T if d == T - t else t + d
        n += 1
    return A, n


def _lagrange_basis(s):
    nodes = [-2, -1, 0, 1, 2]
    return np.array([np.prod([(s - n) / (m - n) for n in nodes if n != m]) for m in nodes])


def _fine_to_coarse(jf, r):
    i, m = divmod(jf, r)
    return (i, m / r) if 2 * m < r else (i + 1, (m - r) / r)


def _burgers_exact(S, t, b, a, w, d):
    """u = b + a sin(w (S - d u t)), Newton per point (characteristics)."""
    u = b + a * np.sin(w * S)
    for _ in range(60):
        arg = w * (S - d * u * t)
        F = u - b - a * np.sin(arg)
        u = u - F / (1.0 + a * w * d * t * np.cos(arg))
    return u


# --------------------------------------------------------------------------------------
# Section 2.1: the WENO5 flux (Eqs. 3-6) and the LF split (7)
# --------------------------------------------------------------------------------------
def test_weno5_side_matches_first_principles(orc):
    rng = np.random.default_rng(1)
    for trial in range(300):
        scale = 10.0 ** rng.uniform(-4, 1)
        f = rng.normal(size=5) * scale
        if trial % 3 == 0:  # smooth data
            x = np.arange(-2, 3) * 0.05
            f = np.sin(x + rng.uniform(0, 6)) * scale
        for linear in (False, True):
            exp, d = _weno_reconstruct_first_principles(f, EPS, linear)
            got = orc.weno5_side(*f, eps=EPS, linear=linear)
            assert abs(got - exp) <= 1e-12 * (np.abs(f).max() + 1e-300), (f, linear, got, exp)
    # the linear weights the construction finds are the printed d_r
    np.testing.assert_allclose(d, [0.1, 0.6, 0.3], atol=1e-13)


def test_linear_flux_difference_exact_for_quintics(orc):
    """(fhat_{i+1/2} - fhat_{i-1/2})/h equals f'(x_i) for polynomial data of degree <= 5."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        c = rng.normal(size=6)
        p = np.polynomial.Polynomial(c)
        h = 0.1
        x = np.arange(-3, 4) * h
        f = p(x)
        fr = orc.weno5_side(*f[1:6], eps=EPS, linear=True)
        fl = orc.weno5_side(*f[0:5], eps=EPS, linear=True)
        assert abs((fr - fl) / h - p.deriv()(0.0)) < 1e-9 * np.abs(c).sum() / h


def test_weno5_weights_linear_on_quadratic_data(orc):
    """Quadratic data give beta_0 = beta_1 = beta_2, hence w_r = d_r (Eq. 5)."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        c = rng.normal(size=3)
        f = np.polynomial.Polynomial(c)(np.arange(-2, 3) * 0.3)
        a = orc.weno5_side(*f, eps=EPS, linear=False)
        b = orc.weno5_side(*f, eps=EPS, linear=True)
        assert abs(a - b) < 1e-13 * np.abs(f).max()


# --------------------------------------------------------------------------------------
# Section 2.2.1: WENO5 / Lagrange interpolation (Eqs. 8-11)
# --------------------------------------------------------------------------------------
def test_weno5_interp_matches_first_principles(orc):
    rng = np.random.default_rng(4)
    for trial in range(300):
        v = rng.normal(size=5) * 10.0 ** rng.uniform(-3, 1)
        s = float(rng.choice([-0.5, -0.375, -0.25, 0.125, 0.25, 0.375, rng.uniform(-0.5, 0.5)]))
        for lag in (False, True):
            exp, C = _weno_interp_first_principles(v, s, EPS, lag)
            got = orc.weno5_interp(*v, s, eps=EPS, lagrange=lag)
            assert abs(got - exp) <= 1e-12 * np.abs(v).max(), (v, s, lag)
        assert np.all(C > 0)  # positive linear weights on [x_{i-1/2}, x_{i+1/2})
    _, C = _weno_interp_first_principles(np.zeros(5), -0.5, EPS, True)
    np.testing.assert_allclose(C, [5 / 16, 5 / 8, 1 / 16], atol=1e-14)


def test_interp_exactness_and_coincident_node(orc):
    rng = np.random.default_rng(5)
    nodes = np.arange(-2, 3).astype(float)
    for _ in range(20):
        q4 = np.polynomial.Polynomial(rng.normal(size=5))
        q2 = np.polynomial.Polynomial(rng.normal(size=3))
        s = float(rng.uniform(-0.5, 0.5))
        assert abs(orc.weno5_interp(*q4(nodes), s, eps=EPS, lagrange=True) - q4(s)) < 1e-12 * 50
        assert abs(orc.weno5_interp(*q2(nodes), s, eps=EPS, lagrange=False) - q2(s)) < 1e-12 * 50
        v = rng.normal(size=5)
        assert orc.weno5_interp(*v, 0.0, eps=EPS) == v[2]


# --------------------------------------------------------------------------------------
# Section 2.2: grid set and combination coefficients (Eqs. 12-15)
# --------------------------------------------------------------------------------------
PRINTED = {2: [1, -1], 3: [1, -2, 1], 4: [1, -3, 3, -1]}


@pytest.mark.parametrize("dim,nl", [(1, 3), (2, 0), (2, 4), (2, 6), (3, 3), (3, 6), (4, 3), (4, 5), (5, 4), (6, 3)])
def test_grid_set_enumeration(orc, dim, nl):
    lev, co = orc.grid_set(dim, nl)
    exp_lev, exp_co = [], []
    for q in range(dim):
        for l in itertools.product(range(nl + 1), repeat=dim):  # lexicographic, l_0 slowest
            if sum(l) == nl - q:
                exp_lev.append(l)
                exp_co.append((-1) ** q * math.comb(dim - 1, q))
    assert [tuple(x) for x in lev] == exp_lev
    assert list(co) == exp_co
    assert abs(sum(co) - 1.0) < 1e-15  # constants are reproduced
    if dim in PRINTED:
        for l, c in zip(lev, co):
            q = nl - int(sum(l))
            assert c == PRINTED[dim][q]
    if dim == 2:
        assert len(lev) == 2 * nl + 1 if nl >= 1 else len(lev) == 1
    if (dim, nl) == (3, 6):
        assert len(lev) == 64
    if (dim, nl) == (4, 5):
        assert len(lev) == 121


# --------------------------------------------------------------------------------------
# Whole-pipeline closed forms (linear scheme, linear advection)
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("N,adv", [(20, (1.0, 1.0)), (16, (1.0, -0.5)), (13, (-1.0, 2.0))])
def test_single_grid_fourier_closed_form(orc, N, adv):
    """Linear scheme + RK3 on one Fourier mode: u^n = G(z)^n u^0 with the upwind-5 symbol
    (mirrored for a negative wind).  Pins Eq. (2)-(4), (7), RK3 and the dt rule."""
    b, a, w, T = 0.3, 0.7, math.pi / 2, 0.37
    p = orc.problem(2, N, 0, pde=orc.ADVECTION, scheme=orc.LINEAR5, eps=EPS, lo=0.0, hi=4.0, adv=adv)
    lev, co = orc.grid_set(2, 0)
    u0 = orc.restrict_sine(p, lev[0], b, a, w)
    (u,), steps, t = orc.solve(p, lev, [u0], T, rule=orc.DT_POW53, coef=0.8)
    h = 4.0 / N
    dt = 0.8 * h ** (5.0 / 3.0)
    th = w * h
    lmb = _advection_mode_factor(th, h, adv[0]) + _advection_mode_factor(th, h, adv[1])
    A, n = _march(lmb, T, dt)
    assert n == steps and abs(t - T) < 1e-15
    j = np.arange(N)
    J0, J1 = np.meshgrid(j, j, indexing="xy")  # axis 0 fastest
    exp = b + a * np.imag(A * np.exp(1j * th * (J0 + J1)))
    assert np.max(np.abs(u.reshape(N, N) - exp)) < 1e-13


@pytest.mark.parametrize("nr,nl", [(10, 3), (6, 4)])
def test_sparse_lagrange_fourier_closed_form(orc, nr, nl):
    """Whole sparse pipeline for the linear scheme with Lagrange prolongation: every grid
    evolves its own Fourier factor, prolongation of a mode is the degree-4 Lagrange
    interpolant of e^{i theta x} (product formula), combination with Eq. (12)."""
    b, a, w, T = 0.3, 0.7, math.pi / 2, 0.5
    p = orc.problem(2, nr, nl, pde=orc.ADVECTION, scheme=orc.LINEAR5, prolong=orc.PROLONG_LAGRANGE5,
                    eps=EPS, lo=0.0, hi=4.0)
    lev, co = orc.grid_set(2, nl)
    grids = [orc.restrict_sine(p, l, b, a, w) for l in lev]
    out, steps, t = orc.solve(p, lev, grids, T)
    uh = orc.combine(p, lev, co, out)
    Nf = nr << nl
    hf = 4.0 / Nf
    dt = hf ** (5.0 / 3.0)
    exp = np.zeros((Nf, Nf))
    for l, c in zip(lev, co):
        hs = [4.0 / (nr << int(lk)) for lk in l]
        ths = [w * hk for hk in hs]
        lmb = sum(_advection_mode_factor(th, hk, 1.0) for th, hk in zip(ths, hs))
        A, n = _march(lmb, T, dt)
        E = []
        for k in range(2):
            r = 1 << (nl - int(l[k]))
            e = np.zeros(Nf, dtype=complex)
            for jf in range(Nf):
                ic, s = _fine_to_coarse(jf, r)
                if s == 0.0:
                    e[jf] = np.exp(1j * ths[k] * ic)
                else:
                    e[jf] = np.dot(_lagrange_basis(s), np.exp(1j * ths[k] * (ic + np.arange(-2, 3))))
            E.append(e)
        exp += c * (b + a * np.imag(A * np.outer(E[1], E[0])))  # row = axis 1, column = axis 0
    assert np.max(np.abs(uh.reshape(Nf, Nf) - exp)) < 1e-12


# --------------------------------------------------------------------------------------
# Paper tables (Section 3): pin epsilon, the LF-alpha convention and the whole pipeline
# --------------------------------------------------------------------------------------
def _rows():
    with open(GOLDEN) as fh:
        return json.load(fh)["rows"]


@pytest.mark.parametrize("row", _rows(), ids=lambda r: r["cite"])
def test_paper_table_rows(orc, row):
    dim, nr, nl = row["dim"], row["nr"], row["nl"]
    pde = orc.BURGERS if row["pde"] == "burgers" else orc.ADVECTION
    scheme = orc.LINEAR5 if row["scheme"] == "linear" else orc.WENO5
    prol = orc.PROLONG_LAGRANGE5 if row["prolong"] == "lagrange" else orc.PROLONG_WENO5
    lo, hi = row["domain"]
    b, a, w = row["ic"]
    p = orc.problem(dim, nr, nl, pde=pde, scheme=scheme, prolong=prol, eps=EPS, lo=lo, hi=hi)
    lev, co = orc.grid_set(dim, nl)
    grids = [orc.restrict_sine(p, l, b, a, w) for l in lev]
    out, steps, t = orc.solve(p, lev, grids, row["T"])
    uh = orc.combine(p, lev, co, out)
    # error norms computed here from the exact solution, and by the oracle
    Nf = nr << nl
    x = lo + np.arange(Nf) * ((hi - lo) / Nf)
    S = sum(np.meshgrid(*([x] * dim), indexing="ij"))
    if pde == orc.BURGERS:
        ex = _burgers_exact(S, row["T"], b, a, w, dim)
    else:
        ex = b + a * np.sin(w * (S - dim * row["T"]))
    err = np.abs(uh - ex.transpose().reshape(-1))
    l1, linf = err.mean(), err.max()
    ol1, olinf = orc.error_norms(p, uh, b, a, w, 0.0, row["T"])
    assert abs(ol1 - l1) < 1e-9 * l1 and abs(olinf - linf) < 1e-9 * linf
    if row["exact_digits"]:
        for ours, printed in ((l1, row["l1"]), (linf, row["linf"])):
            # agree to exact_digits significant digits: within half a unit of that digit
            unit = 10.0 ** (math.floor(math.log10(printed)) - (row["exact_digits"] - 1))
            assert abs(ours - printed) <= 0.5 * unit * (1 + 1e-9), (ours, printed)
    else:
        f = row["loose"]
        assert row["l1"] / f <= l1 <= row["l1"] * f
        assert row["linf"] / f <= linf <= row["linf"] * f


# --------------------------------------------------------------------------------------
# Invariants and special cases
# --------------------------------------------------------------------------------------
def test_mass_conservation_periodic(orc):
    rng = np.random.default_rng(6)
    p = orc.problem(2, 8, 2, pde=orc.BURGERS, scheme=orc.WENO5, eps=EPS, lo=0.0, hi=4.0)
    lev, co = orc.grid_set(2, 2)
    grids = [0.5 + rng.uniform(-1, 1, size=int(np.prod(orc.shape(p, l)))) for l in lev]
    m0 = [orc.mass(p, l, g) for l, g in zip(lev, grids)]
    out, steps, t = orc.solve(p, lev, grids, 1.0, max_steps=6, rule=orc.DT_CFL, cfl=0.4)
    assert steps == 6
    for l, g, m in zip(lev, out, m0):
        hs = [4.0 / n for n in orc.shape(p, l)]
        assert abs(orc.mass(p, l, g) - m) < 1e-13 * abs(np.prod(hs)) * g.size
    for l, g0 in zip(lev, grids):
        hs = [4.0 / n for n in orc.shape(p, l)]
        assert abs(orc.mass(p, l, g0) - g0.sum() * np.prod(hs)) < 1e-12


def test_cfl_time_step_closed_form(orc):
    p = orc.problem(3, 6, 2, pde=orc.BURGERS, eps=EPS, lo=0.0, hi=4.0)
    lev, co = orc.grid_set(3, 2)
    rng = np.random.default_rng(7)
    grids = [rng.uniform(-1.5, 1.2, size=int(np.prod(orc.shape(p, l)))) for l in lev]
    amax = max(np.abs(g).max() for g in grids)
    hf = 4.0 / (6 << 2)
    assert abs(orc.dt(p, lev, grids, rule=orc.DT_CFL, cfl=0.4) - 0.4 / (3 * amax / hf)) < 1e-15
    assert abs(orc.dt(p, lev, grids, rule=orc.DT_POW53, coef=0.5) - 0.5 * hf ** (5 / 3)) < 1e-16
    pa = orc.problem(2, 6, 2, pde=orc.ADVECTION, eps=EPS, adv=(1.0, -3.0))
    lev2, _ = orc.grid_set(2, 2)
    g2 = [np.zeros(int(np.prod(orc.shape(pa, l)))) for l in lev2]
    assert abs(orc.dt(pa, lev2, g2, rule=orc.DT_CFL, cfl=0.4) - 0.4 / (1.0 / hf + 3.0 / hf)) < 1e-15


def test_restriction_and_burgers_exact(orc):
    p = orc.problem(3, 5, 1, pde=orc.BURGERS, eps=EPS, lo=(0.0, -1.0, 2.0), hi=(4.0, 3.0, 5.0))
    lev, _ = orc.grid_set(3, 1)
    for l in lev:
        n = orc.shape(p, l)
        xs = [lo + np.arange(nk) * (hi - lo) / nk for lo, hi, nk in zip((0.0, -1.0, 2.0), (4.0, 3.0, 5.0), n)]
        S = sum(np.meshgrid(*xs, indexing="ij"))
        exp = 0.5 + 0.8 * np.sin(1.3 * S + 0.2)
        np.testing.assert_allclose(orc.restrict_sine(p, l, 0.5, 0.8, 1.3, 0.2),
                                   exp.transpose().reshape(-1), rtol=0, atol=1e-14)
    rng = np.random.default_rng(8)
    for _ in range(50):
        x = rng.uniform(0, 4, size=3)
        t = rng.uniform(0, 0.9) / (0.8 * 1.3 * 3)  # before the shock time 1/(a w d)
        u = orc.exact_sine(p, 0.5, 0.8, 1.3, 0.2, x, t)
        assert abs(u - (0.5 + 0.8 * np.sin(1.3 * (x.sum() - 3 * u * t) + 0.2))) < 1e-13
        assert orc.exact_sine(p, 0.5, 0.8, 1.3, 0.2, x, 0.0) == pytest.approx(
            0.5 + 0.8 * np.sin(1.3 * x.sum() + 0.2), abs=1e-15)


def test_constant_state_is_steady_and_reproduced(orc):
    """A constant is a steady state of every grid and the combination reproduces it
    (sum of coefficients is 1)."""
    for prol in (orc.PROLONG_WENO5, orc.PROLONG_LAGRANGE5):
        p = orc.problem(3, 5, 2, pde=orc.BURGERS, eps=EPS, prolong=prol)
        lev, co = orc.grid_set(3, 2)
        grids = [np.full(int(np.prod(orc.shape(p, l))), 0.75) for l in lev]
        out, steps, t = orc.solve(p, lev, grids, 0.2, max_steps=3, rule=orc.DT_CFL)
        for g in out:
            assert np.all(g == 0.75)
        uh = orc.combine(p, lev, co, out)
        assert np.max(np.abs(uh - 0.75)) < 1e-15


def test_pointwise_prolongation_equals_array_prolongation(orc):
    rng = np.random.default_rng(9)
    for dim, nr, nl in [(2, 5, 3), (3, 5, 2)]:
        for prol in (orc.PROLONG_WENO5, orc.PROLONG_LAGRANGE5):
            p = orc.problem(dim, nr, nl, eps=EPS, prolong=prol)
            lev, co = orc.grid_set(dim, nl)
            grids = [rng.normal(size=int(np.prod(orc.shape(p, l)))) for l in lev]
            uh = orc.combine(p, lev, co, grids)
            Nf = nr << nl
            Js = rng.integers(0, Nf, size=(40, dim))
            got = orc.combine_points(p, lev, co, grids, Js)
            idx = [sum(int(J[k]) * Nf ** k for k in range(dim)) for J in Js]
            assert np.array_equal(got, uh[idx])


def test_burgers_convergence_order_single_grid(orc):
    """Measured order of the WENO scheme on smooth Burgers data approaches 5 (Table 4)."""
    b, a, w, T = 1.0, 0.5, 1.0, 0.3
    errs = []
    for N in (40, 80):
        p = orc.problem(2, N, 0, pde=orc.BURGERS, eps=EPS, lo=0.0, hi=2 * math.pi)
        lev, co = orc.grid_set(2, 0)
        g = [orc.restrict_sine(p, lev[0], b, a, w)]
        out, steps, t = orc.solve(p, lev, g, T)
        x = np.arange(N) * (2 * math.pi / N)
        S = x[None, :] + x[:, None]
        ex = _burgers_exact(S, T, b, a, w, 2)
        errs.append(np.abs(out[0].reshape(N, N) - ex).mean())
    order = math.log2(errs[0] / errs[1])
    assert 4.3 < order < 6.5, errs


# --------------------------------------------------------------------------------------
# Vlasov-Poisson workload (1D1V Landau damping; not in the paper): field solve, steady
# states, zero-inflow prolongation and the linear damping rate
# --------------------------------------------------------------------------------------
VP_LO, VP_HI = [0.0, -2 * math.pi], [4 * math.pi, 2 * math.pi]


def _vp(orc, nr, nl, **kw):
    return orc.problem(2, nr, nl, pde=orc.VLASOV, eps=EPS, lo=VP_LO, hi=VP_HI, **kw)


def test_vlasov_field_solve_second_order(orc):
    """rho = h_v sum_j f = 1 + a cos(k x) (up to the Maxwellian's truncated tail) gives
    E = (a/k) sin(k x); the trapezoid integration converges at second order."""
    errs = []
    for n in (32, 64, 128):
        p = _vp(orc, n, 0)
        u = orc.restrict_landau(p, [0, 0], 0.05, 0.5)
        E = orc.efield(p, [0, 0], u)
        x = np.arange(n) * (4 * math.pi / n)
        errs.append(np.max(np.abs(E - 0.1 * np.sin(0.5 * x))))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def test_vlasov_uniform_maxwellian_is_steady(orc):
    """a = 0: the density is uniform, so E vanishes up to the rounding of the mean, and f is
    independent of x: L(f) vanishes to rounding (the x fluxes cancel exactly)."""
    p = _vp(orc, 16, 0)
    u = orc.restrict_landau(p, [0, 0], 0.0, 0.5)
    assert np.max(np.abs(orc.efield(p, [0, 0], u))) < 1e-13
    L = orc.spatial_operator(p, [0, 0], u).reshape(16, 16)
    assert np.max(np.abs(L)) < 1e-13
    # with E ~ 0 the operator is the x-transport alone, which cancels exactly on each v line
    p2 = orc.problem(2, 16, 0, pde=orc.ADVECTION, eps=EPS, lo=VP_LO, hi=VP_HI, adv=(1.0, 0.0))
    assert np.all(orc.spatial_operator(p2, [0, 0], u) == 0.0)


def test_vlasov_zero_inflow_prolongation_matches_periodic_inside(orc):
    """For data that vanish within five cells of both v ends, the zero-inflow prolongation
    along v equals the periodic one (a different code path: the wrap-around branch)."""
    rng = np.random.default_rng(21)
    nr, nl = 10, 3
    pv = _vp(orc, nr, nl)
    pp = orc.problem(2, nr, nl, pde=orc.ADVECTION, eps=EPS, lo=VP_LO, hi=VP_HI)
    lev, co = orc.grid_set(2, nl)
    grids = []
    for l in lev:
        n0, n1 = orc.shape(pv, l)
        g = rng.normal(size=(n1, n0))
        g[:5, :] = 0.0
        g[-5:, :] = 0.0
        grids.append(g.reshape(-1))
    assert np.array_equal(orc.combine(pv, lev, co, grids), orc.combine(pp, lev, co, grids))


def test_vlasov_landau_damping_rate_and_mass(orc):
    """Linear Landau damping, k = 0.5, a = 0.01: the field amplitude decays at the rate of
    linear theory, 0.1533 (the root of the dispersion relation), within 3% on a 64^2 grid;
    mass is conserved up to the Maxwellian's outflow at |v| = 2 pi (~1e-9)."""
    p = _vp(orc, 64, 0)
    lev = [0, 0]
    u = orc.restrict_landau(p, lev, 0.01, 0.5)
    m0 = orc.mass(p, lev, u)
    ts, amp, t = [], [], 0.0
    for _ in range(40):
        out, _, t = orc.solve(p, [lev], [u], t + 0.5, t0=t, rule=orc.DT_CFL, cfl=0.4)
        u = out[0]
        ts.append(t)
        amp.append(0.5 * math.log(orc.field_energy(p, lev, u)))
    assert abs(orc.mass(p, lev, u) - m0) < 1e-8 * m0
    pk = [i for i in range(1, len(amp) - 1) if amp[i] > amp[i - 1] and amp[i] > amp[i + 1]]
    rate = -np.polyfit(np.array(ts)[pk], np.array(amp)[pk], 1)[0]
    assert abs(rate - 0.1533) < 0.03 * 0.1533, rate
