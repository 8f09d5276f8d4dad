"""FP64 CPU oracle for the sparse-grid WENO5 method (Zhu & Zhang, arXiv 2007.10196).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The product (``paper_2007_10196_gb300``) never imports it, and the two share no code.

The arithmetic lives in ``sgweno_oracle.c`` (plain scalar C, compiled with
``-ffp-contract=off``); this module only compiles it, loads it with ctypes and marshals
numpy arrays.  Grid arrays are flat, axis 0 fastest (index = i_0 + n_0 (i_1 + n_1 ...)).

Pins (tests/test_oracle_pins.py): Table 1 single-grid rows and the Fourier closed form of
the linear scheme (operator + RK3 + time-step rule), the sparse-grid Fourier closed form
with Lagrange prolongation (grid set, coefficients, prolongation, combination), Tables 3,
4 and 6 single-grid rows (epsilon and the LF alpha convention), the smoothness-indicator
integrals of Eq. (10), polynomial exactness of the flux difference and the interpolants,
the printed 2-D/3-D/4-D combination formulas, mass conservation and the Burgers
characteristic equation.  The kinetic workloads: the Vlasov-Poisson field solve and Landau
damping rate (tests/test_oracle_pins.py), and the Vlasov-Boltzmann relaxation model of
Example 5 (tests/test_oracle_relax_pins.py: phase-space rotation, moment equations,
stationary state, 4-D separability, entropy closed forms).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgweno_oracle.c")
_LIB = os.path.join(_HERE, "libsgweno_oracle.so")
MAXD = 6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add) into oracle/libsgweno_oracle.so."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Problem(C.Structure):
    """Mirror of ``orc_problem`` (oracle/sgweno_oracle.c)."""

    _fields_ = [
        ("dim", C.c_int), ("nr", C.c_int), ("nl", C.c_int), ("pde", C.c_int),
        ("scheme", C.c_int), ("prolong", C.c_int), ("eps", C.c_double),
        ("lo", C.c_double * MAXD), ("hi", C.c_double * MAXD), ("adv", C.c_double * MAXD),
        ("theta", C.c_double), ("tau", C.c_double), ("bc", C.c_int * MAXD),
    ]


ADVECTION, BURGERS, VLASOV, VLASOV_BOLTZMANN, VLASOV_MAXWELL = 0, 1, 2, 3, 4
WENO5, LINEAR5 = 0, 1
PROLONG_WENO5, PROLONG_LAGRANGE5 = 0, 1
DT_POW53, DT_CFL = 0, 1

_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER(Problem)
        sig = {
            "orc_grid_set": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
            "orc_grid_points": (C.c_long, [P, _ip]),
            "orc_weno5_side": (C.c_double, [C.c_double] * 6 + [C.c_int]),
            "orc_weno5_interp": (C.c_double, [C.c_double] * 7 + [C.c_int]),
            "orc_lf_alpha": (C.c_double, [P, _ip, _dp, C.c_int]),
            "orc_spatial_operator": (None, [P, _ip, _dp, _dp]),
            "orc_rk3_step": (None, [P, _ip, _dp, C.c_double, _dp]),
            "orc_dt": (C.c_double, [P, C.c_int, _ip, _dp, C.c_int, C.c_double, C.c_double]),
            "orc_solve": (C.c_long, [P, C.c_int, _ip, _dp, C.c_double, C.c_double, C.c_long,
                                     C.c_int, C.c_double, C.c_double,
                                     C.POINTER(C.c_double)]),
            "orc_restrict_sine": (None, [P, _ip] + [C.c_double] * 4 + [_dp]),
            "orc_prolong_grid": (None, [P, _ip, _dp, _dp, _dp]),
            "orc_combine": (None, [P, C.c_int, _ip, _dp, _dp, _dp, _dp]),
            "orc_prolong_point": (C.c_double, [P, _ip, _dp, _lp]),
            "orc_combine_point": (C.c_double, [P, C.c_int, _ip, _dp, _dp, _lp]),
            "orc_mass": (C.c_double, [P, _ip, _dp]),
            "orc_efield": (None, [P, _ip, _dp, _dp]),
            "orc_restrict_landau": (None, [P, _ip, C.c_double, C.c_double, _dp]),
            "orc_field_energy": (C.c_double, [P, _ip, _dp]),
            "orc_vb_density": (None, [P, _ip, _dp, _dp]),
            "orc_state_points": (C.c_long, [P, _ip]),
            "orc_vm_currents": (None, [P, _ip, _dp, _dp, _dp]),
            "orc_restrict_vm": (None, [P, _ip] + [C.c_double] * 6 + [_dp]),
            "orc_vm_energy": (None, [P, _ip, _dp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "orc_relax_norm": (C.c_double, [P]),
            "orc_restrict_relax": (None, [P, _ip, C.c_double, _dp]),
            "orc_relax_entropy": (None, [P, _ip, _dp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "orc_exact_sine": (C.c_double, [P] + [C.c_double] * 4 + [_dp, C.c_double]),
            "orc_error_norms": (None, [P, _dp] + [C.c_double] * 5
                                + [C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


BC_PERIODIC, BC_ZERO = 0, 1


def problem(dim, nr, nl, pde=ADVECTION, scheme=WENO5, prolong=PROLONG_WENO5, eps=1e-6,
            lo=0.0, hi=4.0, adv=1.0, theta=1.0, tau=1.0, bc=BC_PERIODIC) -> Problem:
    p = Problem()
    p.dim, p.nr, p.nl, p.pde = dim, nr, nl, pde
    p.scheme, p.prolong, p.eps = scheme, prolong, eps
    p.theta, p.tau = theta, tau
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (dim,))
    hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), (dim,))
    adv = np.broadcast_to(np.asarray(adv, dtype=np.float64), (dim,))
    bc = np.broadcast_to(np.asarray(bc, dtype=np.int64), (dim,))
    for k in range(dim):
        p.lo[k], p.hi[k], p.adv[k], p.bc[k] = lo[k], hi[k], adv[k], int(bc[k])
    return p


def grid_set(dim: int, nl: int):
    """(levels[G, dim] int32, coeff[G] float64) in enumeration order (Eq. 13)."""
    L = lib()
    G = L.orc_grid_set(dim, nl, None, None)
    lev = np.zeros((max(G, 0), dim), dtype=np.int32)
    co = np.zeros(max(G, 0), dtype=np.float64)
    L.orc_grid_set(dim, nl, lev.ctypes.data, co.ctypes.data)
    return lev, co


def shape(p: Problem, levels) -> tuple:
    """Per-axis node counts (n_0, ..., n_{d-1}) of a grid."""
    return tuple(int(p.nr) << int(l) for l in levels)


def _lev(levels):
    return np.ascontiguousarray(levels, dtype=np.int32).reshape(-1)


def weno5_side(a, b, c, d, e, eps=1e-6, linear=False) -> float:
    return lib().orc_weno5_side(a, b, c, d, e, eps, int(bool(linear)))


def weno5_interp(a, b, c, d, e, s, eps=1e-6, lagrange=False) -> float:
    return lib().orc_weno5_interp(a, b, c, d, e, s, eps, int(bool(lagrange)))


def lf_alpha(p, levels, u, k) -> float:
    return lib().orc_lf_alpha(C.byref(p), _lev(levels), np.ascontiguousarray(u, np.float64), k)


def spatial_operator(p, levels, u):
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    out = np.empty_like(u)
    lib().orc_spatial_operator(C.byref(p), _lev(levels), u, out)
    return out


def rk3_step(p, levels, u, dt):
    u = np.array(u, dtype=np.float64).reshape(-1)
    assert u.size == state_points(p, levels)
    work = np.empty(3 * u.size, dtype=np.float64)
    lib().orc_rk3_step(C.byref(p), _lev(levels), u, dt, work)
    return u


def restrict_sine(p, levels, b, a, w, phi=0.0):
    n = shape(p, levels)
    u = np.empty(int(np.prod(n)), dtype=np.float64)
    lib().orc_restrict_sine(C.byref(p), _lev(levels), b, a, w, phi, u)
    return u


def concat(grids):
    return np.ascontiguousarray(np.concatenate([np.asarray(g, np.float64).reshape(-1)
                                                for g in grids]))


def state_points(p, levels) -> int:
    """Values of one grid's state (its nodes; Vlasov-Maxwell: and its three field arrays)."""
    return int(lib().orc_state_points(C.byref(p), _lev(levels)))


def split(p, levels, flat):
    out, off = [], 0
    for lv in np.asarray(levels).reshape(-1, p.dim):
        n = state_points(p, lv)
        out.append(flat[off:off + n].copy())
        off += n
    return out


def dt(p, levels, grids, rule=DT_POW53, coef=1.0, cfl=0.4):
    levels = np.asarray(levels).reshape(-1, p.dim)
    flat = concat(grids)
    return lib().orc_dt(C.byref(p), len(levels), _lev(levels), flat, rule, coef, cfl)


def solve(p, levels, grids, t_end, t0=0.0, max_steps=1 << 62, rule=DT_POW53, coef=1.0,
          cfl=0.4):
    """Step 2 of the algorithm.  Returns (grids_out list, steps, t_reached)."""
    levels = np.asarray(levels).reshape(-1, p.dim)
    flat = concat(grids)
    t_out = C.c_double(0.0)
    steps = lib().orc_solve(C.byref(p), len(levels), _lev(levels), flat, t0, t_end,
                            max_steps, rule, coef, cfl, C.byref(t_out))
    return split(p, levels, flat), int(steps), float(t_out.value)


def fine_points(p) -> int:
    return (int(p.nr) << int(p.nl)) ** int(p.dim)


def prolong_grid(p, levels, u):
    tot = fine_points(p)
    out = np.empty(tot, dtype=np.float64)
    work = np.empty(2 * tot, dtype=np.float64)
    lib().orc_prolong_grid(C.byref(p), _lev(levels), np.ascontiguousarray(u, np.float64),
                           out, work)
    return out


def combine(p, levels, coeff, grids):
    levels = np.asarray(levels).reshape(-1, p.dim)
    tot = fine_points(p)
    out = np.empty(tot, dtype=np.float64)
    work = np.empty(3 * tot, dtype=np.float64)
    lib().orc_combine(C.byref(p), len(levels), _lev(levels),
                      np.ascontiguousarray(coeff, np.float64), concat(grids), out, work)
    return out


def prolong_point(p, levels, u, J) -> float:
    return lib().orc_prolong_point(C.byref(p), _lev(levels), np.ascontiguousarray(u, np.float64),
                                   np.ascontiguousarray(J, np.int64))


def combine_points(p, levels, coeff, grids, Js):
    """uhat at each finest-grid multi-index in Js (array [M, dim])."""
    levels = np.asarray(levels).reshape(-1, p.dim)
    flat = concat(grids)
    co = np.ascontiguousarray(coeff, np.float64)
    lv = _lev(levels)
    L = lib()
    Js = np.asarray(Js, dtype=np.int64).reshape(-1, p.dim)
    return np.array([L.orc_combine_point(C.byref(p), len(levels), lv, co, flat,
                                         np.ascontiguousarray(J)) for J in Js])


def mass(p, levels, u) -> float:
    return lib().orc_mass(C.byref(p), _lev(levels), np.ascontiguousarray(u, np.float64))


def exact_sine(p, b, a, w, phi, x, t) -> float:
    return lib().orc_exact_sine(C.byref(p), b, a, w, phi, np.ascontiguousarray(x, np.float64), t)


def error_norms(p, uhat, b, a, w, phi, t):
    l1, li = C.c_double(), C.c_double()
    lib().orc_error_norms(C.byref(p), np.ascontiguousarray(uhat, np.float64), b, a, w, phi, t,
                          C.byref(l1), C.byref(li))
    return float(l1.value), float(li.value)


def efield(p: Problem, levels, u):
    """Vlasov-Poisson field E_i of one grid (pde VLASOV)."""
    n0 = int(p.nr) << int(levels[0])
    E = np.empty(n0, dtype=np.float64)
    lib().orc_efield(C.byref(p), _lev(levels), np.ascontiguousarray(u, np.float64), E)
    return E


def restrict_landau(p: Problem, levels, a, k):
    """f_0 = (1 + a cos(k x)) exp(-v^2/2) / sqrt(2 pi) on one grid (pde VLASOV)."""
    u = np.empty(int(np.prod(shape(p, levels))), dtype=np.float64)
    lib().orc_restrict_landau(C.byref(p), _lev(levels), float(a), float(k), u)
    return u


def field_energy(p: Problem, levels, u) -> float:
    return float(lib().orc_field_energy(C.byref(p), _lev(levels), np.ascontiguousarray(u, np.float64)))


def vb_density(p: Problem, levels, u):
    """rho(x) of one grid of the Vlasov-Boltzmann model (pde VLASOV_BOLTZMANN), flattened
    over the space axes."""
    n = shape(p, levels)
    rho = np.empty(int(np.prod(n[:p.dim // 2])), dtype=np.float64)
    lib().orc_vb_density(C.byref(p), _lev(levels), np.ascontiguousarray(u, np.float64), rho)
    return rho


def relax_norm(p: Problem) -> float:
    """Normalisation s of the Example 5 initial condition (integral over the domain)."""
    return float(lib().orc_relax_norm(C.byref(p)))


def restrict_relax(p: Problem, levels, s_norm=None):
    """Example 5 initial condition on one grid (pde VLASOV_BOLTZMANN, dim 2 or 4)."""
    if s_norm is None:
        s_norm = relax_norm(p)
    u = np.empty(int(np.prod(shape(p, levels))), dtype=np.float64)
    lib().orc_restrict_relax(C.byref(p), _lev(levels), float(s_norm), u)
    return u


def relax_entropy(p: Problem, levels, u):
    """(H_2, H_log) of Example 5 over one grid's nodes (the finest grid for the combined
    solution: levels all N_L)."""
    h2, hl = C.c_double(), C.c_double()
    lib().orc_relax_entropy(C.byref(p), _lev(levels), np.ascontiguousarray(u, np.float64),
                            C.byref(h2), C.byref(hl))
    return float(h2.value), float(hl.value)


def vm_state(p: Problem, levels, beta=0.01, delta=0.5, v1=0.3, v2=0.3, b=0.001, k0=0.2):
    """Example 6 initial state of one grid (pde VLASOV_MAXWELL): f, then E_1, E_2, B_3."""
    u = np.empty(state_points(p, levels), dtype=np.float64)
    lib().orc_restrict_vm(C.byref(p), _lev(levels), beta, delta, v1, v2, b, k0, u)
    return u


def vm_currents(p: Problem, levels, u):
    nx = int(p.nr) << int(levels[0])
    j1, j2 = np.empty(nx), np.empty(nx)
    lib().orc_vm_currents(C.byref(p), _lev(levels), np.ascontiguousarray(u, np.float64), j1, j2)
    return j1, j2


def vm_energy(p: Problem, levels, u):
    """(kinetic, field) energy of one Vlasov-Maxwell grid."""
    k, f = C.c_double(), C.c_double()
    lib().orc_vm_energy(C.byref(p), _lev(levels), np.ascontiguousarray(u, np.float64), C.byref(k), C.byref(f))
    return float(k.value), float(f.value)
