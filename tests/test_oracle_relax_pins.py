"""Pins of the oracle's Vlasov-Boltzmann relaxation model (Example 5) against the mathematics.

f_t + v . grad_x f - x . grad_v f = (mu_inf(v) rho(x) - f) / tau on [-5, 5]^{2d} with zero
boundary values.  None of these tests retypes an oracle formula:
  - the normalisation of the initial condition against a closed form (error function of a
    complex argument);
  - with the relaxation switched off (tau -> infinity) the exact solution is a rigid
    rotation of phase space (the characteristics of x' = v, v' = -x), and the scheme
    converges to it at high order;
  - the velocity moments of L(f) obey the moment equations of the model (mass, momentum,
    energy) with the Maxwellian's moments taken on the truncated velocity nodes;
  - the stationary state M makes L vanish as h -> 0;
  - with the linear scheme (linear weights) the 4-D transport of a product g(x1, v1)
    h(x2, v2) separates exactly into two 2-D transports;
  - the relaxation term alone (L_tau - L_inf) has the exact moments per space node;
  - closed forms of the entropy functionals at multiples of M.
"""
import math

import numpy as np
import pytest

EPS = 1e-3
LO, HI = -5.0, 5.0


def _p(orc, dim, n, nl=0, **kw):
    return orc.problem(dim, n, nl, pde=orc.VLASOV_BOLTZMANN, eps=EPS, lo=LO, hi=HI, **kw)


def _nodes(n):
    h = (HI - LO) / n
    return LO + np.arange(n) * h, h


def _flat2(a):
    """[i_x, i_v] array -> flat index i_x + n i_v (axis 0 fastest)."""
    return np.ascontiguousarray(a.T.reshape(-1))


def _flat4(a):
    """[i_x1, i_x2, i_v1, i_v2] array -> flat index, axis 0 fastest."""
    return np.ascontiguousarray(a.transpose(3, 2, 1, 0).reshape(-1))


def _mu_moments(v, h, theta):
    """sum_j v_j^m mu(v_j) h for m = 0, 1, 2: the Maxwellian's moments on the truncated nodes."""
    mu = np.exp(-v * v / (2 * theta)) / math.sqrt(2 * math.pi * theta)
    return [float((v ** m * mu).sum() * h) for m in range(3)]


def test_relax_normalisation_closed_form(orc):
    """int_{-5}^{5} exp(-a x^2) dx = sqrt(pi/a) erf(5 sqrt(a)) for complex a; with
    sin^2(x^2/2) = (1 - Re e^{i x^2})/2 and cos^2 = (1 + Re e^{i x^2})/2 the normalisation s
    is a product of such integrals."""
    from scipy.special import erf
    a = 0.5 - 1.0j
    gauss = math.sqrt(2 * math.pi) * erf(5 / math.sqrt(2))
    osc = (np.sqrt(np.pi / a) * erf(5 * np.sqrt(a))).real
    s_sin, s_cos = 0.5 * (gauss - osc), 0.5 * (gauss + osc)
    assert abs(orc.relax_norm(_p(orc, 2, 8)) / (s_sin * gauss) - 1) < 1e-12
    assert abs(orc.relax_norm(_p(orc, 4, 8)) / (s_sin * s_cos * gauss * gauss) - 1) < 1e-12
    # the restricted initial condition then has unit mass up to quadrature error
    p = _p(orc, 2, 128)
    u = orc.restrict_relax(p, [0, 0])
    assert abs(orc.mass(p, [0, 0], u) - 1.0) < 1e-5


def test_relax_free_transport_is_a_phase_space_rotation(orc):
    """tau -> infinity: f(t, x, v) = f_0(x cos t - v sin t, x sin t + v cos t).  After a
    quarter turn a Gaussian centred at (1, 0) sits at (0, -1); the error falls by more
    than 16x from 64^2 to 128^2 (a wrong sign of E or v gives an O(1) error)."""
    errs = []
    f0 = lambda X, V: np.exp(-((X - 1.0) ** 2 + V ** 2) / (2 * 0.6 ** 2))
    for n in (64, 128):
        p = _p(orc, 2, n, tau=1e300)
        x, _ = _nodes(n)
        X, V = np.meshgrid(x, x, indexing="ij")
        out, _, t = orc.solve(p, [[0, 0]], [_flat2(f0(X, V))], math.pi / 2, rule=orc.DT_CFL, cfl=0.4)
        assert t == math.pi / 2
        ex = _flat2(f0(X * math.cos(t) - V * math.sin(t), X * math.sin(t) + V * math.cos(t)))
        errs.append(np.max(np.abs(out[0] - ex)))
    assert errs[1] < 1e-3 and errs[0] / errs[1] > 16, errs


def test_relax_moment_equations_2d(orc):
    """d/dt of int f, int v f, int v^2 f under the model: transport gives 0, -int x f and
    -2 int x v f; relaxation gives (M_m rho - int v^m f) / tau with M_m the Maxwellian's
    moments.  theta = 1.5, tau = 0.5 so that a misplaced theta or tau is an O(1) error;
    the residuals fall at high order (boundary outflow ~1e-6 is the floor)."""
    th, tau = 1.5, 0.5
    res = []
    for n in (32, 64, 128):
        p = _p(orc, 2, n, theta=th, tau=tau)
        x, h = _nodes(n)
        X, V = np.meshgrid(x, x, indexing="ij")
        u = _flat2(np.exp(-((X - 0.7) ** 2 + (V - 0.4) ** 2) / (2 * 0.8 ** 2)))
        Xf, Vf = _flat2(X), _flat2(V)
        L = orc.spatial_operator(p, [0, 0], u)
        dV = h * h
        M0, M1, M2 = _mu_moments(x, h, th)
        mass = u.sum() * dV
        r0 = L.sum() * dV - (M0 * mass - mass) / tau
        r1 = (Vf * L).sum() * dV - (-(Xf * u).sum() * dV + (M1 * mass - (Vf * u).sum() * dV) / tau)
        r2 = (Vf ** 2 * L).sum() * dV - (-2 * (Xf * Vf * u).sum() * dV
                                         + (M2 * mass - (Vf ** 2 * u).sum() * dV) / tau)
        res.append((abs(r0), abs(r1), abs(r2)))
    # scale of the terms: |int x f| ~ 3, |int v^2 f / tau| ~ 3
    assert res[2][0] < 1e-5 and res[2][1] < 1e-5 and res[2][2] < 2e-4, res
    assert res[0][2] / res[1][2] > 16 and res[1][2] / res[2][2] > 16, res


def test_relax_stationary_state(orc):
    """M = exp(-(x^2 + v^2)/2) / (2 pi) is the stationary state: L(M) -> 0 at high order."""
    r = []
    for n in (32, 64):
        p = _p(orc, 2, n)
        x, _ = _nodes(n)
        X, V = np.meshgrid(x, x, indexing="ij")
        L = orc.spatial_operator(p, [0, 0], _flat2(np.exp(-(X ** 2 + V ** 2) / 2) / (2 * math.pi)))
        r.append(np.max(np.abs(L)))
    assert r[1] < 1e-4 and r[0] / r[1] > 20, r


def test_relax_4d_transport_separates(orc):
    """Linear weights make the scheme linear, so for f = g(x1, v1) h(x2, v2) the 4-D
    transport is T2(g) h + g T2(h) to rounding: this fixes the axis pairing (x_k with v_k)
    and the zero boundaries of the 4-D operator against the 2-D one."""
    n = 12
    p4 = _p(orc, 4, n, scheme=orc.LINEAR5, tau=1e300)
    p2 = _p(orc, 2, n, scheme=orc.LINEAR5, tau=1e300)
    x, _ = _nodes(n)
    X, V = np.meshgrid(x, x, indexing="ij")
    g = np.exp(-((X - 0.5) ** 2 + (V + 0.3) ** 2) / 2) * (1 + 0.2 * np.cos(X))
    hh = np.exp(-((X + 0.4) ** 2 + (V - 0.6) ** 2) / 1.5)
    f4 = np.einsum("ac,bd->abcd", g, hh)  # axes (x1, x2, v1, v2)
    L4 = orc.spatial_operator(p4, [0] * 4, _flat4(f4)).reshape(n, n, n, n).transpose(3, 2, 1, 0)
    Tg = orc.spatial_operator(p2, [0, 0], _flat2(g)).reshape(n, n).T
    Th = orc.spatial_operator(p2, [0, 0], _flat2(hh)).reshape(n, n).T
    expect = np.einsum("ac,bd->abcd", Tg, hh) + np.einsum("ac,bd->abcd", g, Th)
    assert np.max(np.abs(L4 - expect)) < 1e-13 * np.max(np.abs(expect))


def test_relax_4d_relaxation_moments_per_space_node(orc):
    """R = L_tau - L_inf is the relaxation term alone.  Per space node its velocity moments
    are exact: sum_v R dv = (M0^2 - 1) rho / tau, sum_v v1 R dv = (M1 M0 rho - j1) / tau,
    sum_v v2^2 R dv = (M2 M0 rho - e2) / tau, with rho, j1, e2 the moments of f."""
    th, tau, n = 1.5, 0.5, 10
    p = _p(orc, 4, n, theta=th, tau=tau)
    pinf = _p(orc, 4, n, theta=th, tau=1e300)
    x, h = _nodes(n)
    X1, X2, V1, V2 = np.meshgrid(x, x, x, x, indexing="ij")
    rng = np.random.default_rng(5)
    f = np.exp(-((X1 - 0.7) ** 2 + (X2 + 0.5) ** 2 + (V1 - 0.4) ** 2 + (V2 - 0.3) ** 2) / 2)
    f = f * (1 + 0.3 * rng.random(f.shape))
    R = (orc.spatial_operator(p, [0] * 4, _flat4(f))
         - orc.spatial_operator(pinf, [0] * 4, _flat4(f))).reshape(n, n, n, n).transpose(3, 2, 1, 0)
    M0, M1, M2 = _mu_moments(x, h, th)
    dv = h * h
    rho = f.sum(axis=(2, 3)) * dv
    j1 = (f * V1).sum(axis=(2, 3)) * dv
    e2 = (f * V2 ** 2).sum(axis=(2, 3)) * dv
    scale = np.max(np.abs(rho)) / tau
    tol = 1e-12 * scale
    assert np.max(np.abs(R.sum(axis=(2, 3)) * dv - (M0 * M0 - 1) * rho / tau)) < tol
    assert np.max(np.abs((R * V1).sum(axis=(2, 3)) * dv - (M1 * M0 * rho - j1) / tau)) < 10 * tol
    assert np.max(np.abs((R * V2 ** 2).sum(axis=(2, 3)) * dv - (M2 * M0 * rho - e2) / tau)) < 30 * tol


def test_relax_density_and_zero_boundary_prolongation(orc):
    """rho of a product f = a(x) b(v) is a(x) h sum_v b; and for data that vanish within
    five cells of every end, the zero-boundary combination equals the periodic one."""
    p = _p(orc, 2, 16)
    x, h = _nodes(16)
    a, b = np.cos(x) + 2.0, np.exp(-x * x / 3)
    rho = orc.vb_density(p, [0, 0], _flat2(np.outer(a, b)))
    assert np.allclose(rho, a * b.sum() * h, rtol=1e-14, atol=0)
    rng = np.random.default_rng(22)
    nr, nl = 12, 3
    pv = _p(orc, 2, nr, nl)
    pp = orc.problem(2, nr, nl, pde=orc.ADVECTION, eps=EPS, lo=LO, hi=HI)
    lev, co = orc.grid_set(2, nl)
    grids = []
    for l in lev:
        n0, n1 = orc.shape(pv, l)
        g = rng.normal(size=(n1, n0))
        g[:5, :] = g[-5:, :] = 0.0
        g[:, :5] = g[:, -5:] = 0.0
        grids.append(g.reshape(-1))
    assert np.array_equal(orc.combine(pv, lev, co, grids), orc.combine(pp, lev, co, grids))


def test_relax_entropy_closed_forms(orc):
    """At f = c M: H_2 = c^2 sum M dV and H_log = c log(c) sum M dV (exactly 0 at c = 1);
    sum M dV -> 1 (M is normalised over the domain in x and over the line in v).
    Negative values add nothing to H_log; H_2 >= (int f)^2 / int M (Cauchy-Schwarz)."""
    n = 64
    p = _p(orc, 2, n)
    x, h = _nodes(n)
    X, V = np.meshgrid(x, x, indexing="ij")
    from scipy.special import erf
    Z = math.sqrt(math.pi / 2) * (erf(HI / math.sqrt(2)) - erf(LO / math.sqrt(2)))
    M = _flat2(np.exp(-(X ** 2 + V ** 2) / 2) / (math.sqrt(2 * math.pi) * Z))
    sM = M.sum() * h * h
    assert abs(sM - 1) < 1e-5
    h2, hl = orc.relax_entropy(p, [0, 0], M)
    assert abs(h2 - sM) < 1e-12 and abs(hl) < 1e-15
    h2, hl = orc.relax_entropy(p, [0, 0], 2.0 * M)
    assert abs(h2 - 4 * sM) < 1e-12 and abs(hl - 2 * math.log(2) * sM) < 1e-12
    h2, hl = orc.relax_entropy(p, [0, 0], -M)
    assert abs(h2 - sM) < 1e-12 and hl == 0.0
    f = orc.restrict_relax(p, [0, 0])
    h2, hl = orc.relax_entropy(p, [0, 0], f)
    assert h2 >= (f.sum() * h * h) ** 2 / sM and hl > 0


@pytest.mark.slow
def test_relax_entropy_decays(orc):
    """Example 5 (a) on a 64^2 single grid: both entropy functionals decrease towards their
    equilibrium values (H_2 -> 1, H_log -> 0) and the mass stays within the outflow bound."""
    p = _p(orc, 2, 64)
    u = orc.restrict_relax(p, [0, 0])
    m0 = orc.mass(p, [0, 0], u)
    h2s, hls = [], []
    t = 0.0
    for _ in range(6):
        out, _, t = orc.solve(p, [[0, 0]], [u], t + 0.5, t0=t, rule=orc.DT_CFL, cfl=0.4)
        u = out[0]
        h2, hl = orc.relax_entropy(p, [0, 0], u)
        h2s.append(h2)
        hls.append(hl)
    assert all(b < a for a, b in zip(h2s, h2s[1:])) and all(b < a for a, b in zip(hls, hls[1:]))
    assert h2s[-1] > 0.99 and hls[-1] > -1e-3
    assert abs(orc.mass(p, [0, 0], u) - m0) < 1e-3
