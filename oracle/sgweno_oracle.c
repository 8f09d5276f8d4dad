/*
 * sgweno_oracle.c -- plain, slow FP64 CPU oracle for the sparse-grid fifth-order WENO
 * method of Zhu & Zhang, "Fast sparse grid simulations of fifth order WENO scheme for
 * high dimensional hyperbolic PDEs" (arXiv 2007.10196).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  The CUDA library never calls it, and the two
 * share no code, headers or tables.
 *
 * Every routine is scalar double arithmetic written in the order the paper prints the
 * formula, with no blocking, fusion or reordering.  It must be compiled with
 * -ffp-contract=off so that no multiply-add is fused; then each line below is a fixed
 * sequence of IEEE-754 double operations.
 *
 * Equation numbers are the paper's (global numbering): (2) flux difference, (3)-(6) the
 * WENO5 reconstruction, (7) Lax-Friedrichs splitting, (8)-(11) WENO5 interpolation,
 * (12)-(15) the combination formulas.
 *
 * Readings where the paper is silent (all shared with the CUDA path by specification):
 *  - grid nodes are vertex-centred and periodic: n_k = N_r 2^{l_k} unique nodes
 *    x_j = lo_k + j h_k, h_k = (hi_k - lo_k)/n_k (Section 2.2);
 *  - the TVD-RK3 scheme cited in Section 2.2 is the Shu-Osher form;
 *  - the LF alpha of (7) is max |f_k'(u)| over one component grid, recomputed from the
 *    input of every RK stage;
 *  - the time step is common to all grids and set by the finest grid (Section 3):
 *    dt = coef * h^{5/3} (accuracy tests) or dt = cfl / sum_k(alpha_k / h_k) with
 *    alpha_k the maximum over all grids; the last step is shortened to land on T;
 *  - the WENO interpolation for x in [x_{i-1/2}, x_{i+1/2}) assigns a fine node to the
 *    nearest coarse node, a midpoint to the right-hand node; at a coincident node (s = 0)
 *    the interpolant is the node value itself, and an axis already at the finest level
 *    is copied, not interpolated;
 *  - prolongation runs axis 0, 1, ..., d-1 (Section 2.2.1);
 *  - the combination sums grids in enumeration order (q = 0, 1, ...; lexicographic
 *    levels within each q, l_0 most significant), into an accumulator that starts at 0.
 *  - zero boundary (bc[k] = 1, advection and Burgers): the nodes are the same, x_j = lo_k +
 *    j h_k, j = 0..n_k-1, and u is zero beyond them (three ghost nodes on either side in
 *    the stencils, two in the interpolation), as for the kinetic models' zero boundaries;
 *  - the flux difference of Eq. (2) multiplies by 1/h_k, formed once per grid and axis,
 *    instead of dividing by h_k at every node (the product and the quotient differ by at
 *    most one rounding; both sides of the parity tests use the product).
 * Vlasov-Poisson (pde 2; not in the paper, the 1D1V kinetic workload run on the same
 * method):
 *  - x is periodic as above; v nodes are v_j = lo_1 + j h_v, j = 0..n_v-1, and f is zero
 *    outside them (zero inflow): stencils and interpolation read 0 beyond either end;
 *  - rho_i = h_v sum_j f_ij (j ascending); E solves dE/dx = rho - mean(rho) by the
 *    trapezoid rule, E_0 = 0, E_i = E_{i-1} + h_x ((rho_{i-1} + rho_i) / 2 - mean(rho)),
 *    then the mean of E is subtracted (periodic E with zero mean);
 *  - E is recomputed from the input of every RK stage; the LF alpha of axis 0 is
 *    max_j |v_j| of the grid, of axis 1 max_i |E_i|.
 * Vlasov-Boltzmann relaxation model (pde 3; Example 5), dim = 2 d with space axes 0..d-1
 * and velocity axes d..2d-1:
 *  - every axis has nodes lo_k + j h_k, j = 0..n_k-1, and f is zero outside them (the
 *    zero boundary condition): stencils and interpolation read 0 beyond either end;
 *  - the transport speed along x_k is the line's v_k, along v_k it is E_k = -x_k (the
 *    potential |x|^2/2); the LF alpha of an axis is the largest |speed| over the grid;
 *  - rho(x) = (h_{v_1} ... h_{v_d}) sum_v f(x, v), the velocity nodes in ascending
 *    flattened order; mu_inf(v) = exp(-(|v|^2 / (2 theta))) / (2 pi theta)^{d/2} with |v|^2
 *    summed in axis order; the relaxation term (mu_inf rho - f) / tau is added to the
 *    transport operator after all axes, from the same stage input.
 * Vlasov-Maxwell (pde 4; Example 6), dim = 3: axis 0 = x_2 (periodic), axes 1, 2 = xi_1, xi_2
 * (periodic, as the example states):
 *  - the state of a grid is f followed by its own fields E_1, E_2, B_3 on its x_2 nodes;
 *  - f: transport speed xi_2 along x_2, E_1 + xi_2 B_3 along xi_1, E_2 - xi_1 B_3 along xi_2,
 *    each constant on a grid line; LF alpha of an axis = the largest |speed| over the grid;
 *  - currents j_m = (h_1 h_2) sum_xi f xi_m (velocity nodes in ascending flattened order);
 *  - Maxwell: w+ = E_1 + B_3 moves at speed -1 and w- = E_1 - B_3 at +1, both with source
 *    -j_1 (the characteristic form of dB_3/dt = dE_1/dx_2, dE_1/dt = dB_3/dx_2 - j_1), each
 *    by the LF-split WENO5 operator with alpha = 1; then dE_1/dt = (L+ + L-)/2,
 *    dB_3/dt = (L+ - L-)/2 and dE_2/dt = -j_2; all from the same stage input;
 *  - the CFL step takes max(max|xi_2|, 1) along x_2 (the fields' speed is 1).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXD 6

typedef struct {
    int dim;           /* d, 1..6 */
    int nr;            /* N_r, root cells per axis */
    int nl;            /* N_L, finest level */
    int pde;           /* 0: linear advection f_k = a_k u;  1: Burgers f_k = u^2/2;
                          2: Vlasov-Poisson (d = 2, axis 0 = x, axis 1 = v): f_x = v u,
                          f_v = E(x) u, E from the grid's own density (see orc_efield);
                          3: Vlasov-Boltzmann relaxation (dim = 2d, see vb_operator);
                          4: Vlasov-Maxwell (dim = 3, see vm_operator) */
    int scheme;        /* 0: WENO5-JS weights (5);  1: fifth-order linear scheme, w_r = d_r */
    int prolong;       /* 0: WENO5 interpolation (11);  1: fifth-order Lagrange (8) */
    double eps;        /* epsilon of (5) and (9) */
    double lo[ORC_MAXD], hi[ORC_MAXD];
    double adv[ORC_MAXD];   /* a_k for linear advection */
    double theta, tau;      /* pde 3: temperature and relaxation time of L(f) */
    int bc[ORC_MAXD];       /* pde 0 and 1, per axis: 0 periodic, 1 zero beyond the nodes */
} orc_problem;

static int zero_axis(const orc_problem *P, int k);

/* ------------------------------------------------------------------------------------
 * Grid set, Section 2.2 and combination formula (13):
 *   coefficient of every grid with |l| = N_L - q is (-1)^q C(d-1, q), q = 0..d-1.
 * ---------------------------------------------------------------------------------- */
static long binom(int n, int k)
{
    long r = 1;
    int i;
    if (k < 0 || k > n) return 0;
    for (i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

/* Enumerates the grids; writes levels[g*dim + k] and coeff[g] if non-NULL.  Returns G. */
int orc_grid_set(int dim, int nl, int *levels, double *coeff)
{
    int g = 0, q, k;
    int l[ORC_MAXD];
    if (dim < 1 || dim > ORC_MAXD || nl < 0) return -1;
    for (q = 0; q < dim; ++q) {
        int target = nl - q;
        if (target < 0) break;
        /* lexicographic walk over l in [0, nl]^dim, l_0 most significant */
        for (k = 0; k < dim; ++k) l[k] = 0;
        for (;;) {
            int s = 0;
            for (k = 0; k < dim; ++k) s += l[k];
            if (s == target) {
                if (levels) for (k = 0; k < dim; ++k) levels[g * dim + k] = l[k];
                if (coeff) coeff[g] = (double)((q % 2 == 0) ? 1 : -1) * (double)binom(dim - 1, q);
                ++g;
            }
            /* increment the last axis first so that l_0 varies slowest */
            k = dim - 1;
            while (k >= 0) {
                if (l[k] < nl) { ++l[k]; break; }
                l[k] = 0;
                --k;
            }
            if (k < 0) break;
        }
    }
    return g;
}

static long grid_points(const orc_problem *P, const int *levels, long *n)
{
    long tot = 1;
    int k;
    for (k = 0; k < P->dim; ++k) {
        n[k] = (long)P->nr << levels[k];
        tot *= n[k];
    }
    return tot;
}

/* Values of one grid's state: its nodes, and for pde 4 the fields E_1, E_2, B_3 (n_0 each). */
long orc_state_points(const orc_problem *P, const int *levels)
{
    long n[ORC_MAXD];
    long N = grid_points(P, levels, n);
    return P->pde == 4 ? N + 3 * n[0] : N;
}

long orc_grid_points(const orc_problem *P, const int *levels)
{
    long n[ORC_MAXD];
    return grid_points(P, levels, n);
}

/* Node spacing of one axis: h_k = (hi_k - lo_k) / n_k. */
static double spacing(const orc_problem *P, int k, long nk)
{
    return (P->hi[k] - P->lo[k]) / (double)nk;
}

/* ------------------------------------------------------------------------------------
 * One-sided WENO5 reconstruction, Section 2.1, Eqs. (3)-(6).
 * (a, b, c, d, e) = (f_{i-2}, f_{i-1}, f_i, f_{i+1}, f_{i+2}) gives fhat_{i+1/2} for the
 * positive wind; the negative wind uses the mirror image (f_{i+3}, ..., f_{i-1}).
 * ---------------------------------------------------------------------------------- */
double orc_weno5_side(double a, double b, double c, double d, double e, double eps, int linear)
{
    /* candidate fluxes, Eq. (4) */
    double q0 = (1.0 / 3.0) * a - (7.0 / 6.0) * b + (11.0 / 6.0) * c;
    double q1 = -(1.0 / 6.0) * b + (5.0 / 6.0) * c + (1.0 / 3.0) * d;
    double q2 = (1.0 / 3.0) * c + (5.0 / 6.0) * d - (1.0 / 6.0) * e;
    double al0, al1, al2;
    if (linear) {
        /* fifth-order linear scheme: w_r = d_r (Section 3) */
        al0 = 0.1;
        al1 = 0.6;
        al2 = 0.3;
    } else {
        /* smoothness indicators, Eq. (6) */
        double t0 = a - 2.0 * b + c, s0 = a - 4.0 * b + 3.0 * c;
        double t1 = b - 2.0 * c + d, s1 = b - d;
        double t2 = c - 2.0 * d + e, s2 = 3.0 * c - 4.0 * d + e;
        double b0 = (13.0 / 12.0) * (t0 * t0) + 0.25 * (s0 * s0);
        double b1 = (13.0 / 12.0) * (t1 * t1) + 0.25 * (s1 * s1);
        double b2 = (13.0 / 12.0) * (t2 * t2) + 0.25 * (s2 * s2);
        /* unnormalised weights, Eq. (5): alpha_r = d_r / (eps + beta_r)^2 */
        al0 = 0.1 / ((eps + b0) * (eps + b0));
        al1 = 0.6 / ((eps + b1) * (eps + b1));
        al2 = 0.3 / ((eps + b2) * (eps + b2));
    }
    /* Eq. (3) with w_r = alpha_r / sum alpha */
    return (al0 * q0 + al1 * q1 + al2 * q2) / (al0 + al1 + al2);
}

/* Vlasov-Poisson field of one grid (pde 2): E_i, i = 0..n_x-1, from the density of u. */
void orc_efield(const orc_problem *P, const int *levels, const double *u, double *E)
{
    long n[ORC_MAXD];
    long i, j;
    double hx, hv, mean = 0.0, meanE = 0.0;
    double *rho;
    grid_points(P, levels, n);
    hx = spacing(P, 0, n[0]);
    hv = spacing(P, 1, n[1]);
    rho = (double *)malloc(sizeof(double) * n[0]);
    for (i = 0; i < n[0]; ++i) {
        double sum = 0.0;
        for (j = 0; j < n[1]; ++j) sum = sum + u[i + n[0] * j];
        rho[i] = hv * sum;
    }
    for (i = 0; i < n[0]; ++i) mean = mean + rho[i];
    mean = mean / (double)n[0];
    E[0] = 0.0;
    for (i = 1; i < n[0]; ++i) E[i] = E[i - 1] + hx * (0.5 * (rho[i - 1] + rho[i]) - mean);
    for (i = 0; i < n[0]; ++i) meanE = meanE + E[i];
    meanE = meanE / (double)n[0];
    for (i = 0; i < n[0]; ++i) E[i] = E[i] - meanE;
    free(rho);
}

/* Velocity node j of a Vlasov-Poisson grid. */
static double vnode(const orc_problem *P, long j, long nv)
{
    return P->lo[1] + (double)j * spacing(P, 1, nv);
}

/* Vlasov-Boltzmann (pde 3): the velocity axis of space axis k and vice versa. */
static int vb_partner(const orc_problem *P, int k)
{
    int d = P->dim / 2;
    return k < d ? k + d : k - d;
}

/* Node j of axis k on a grid with nk nodes on that axis. */
static double node(const orc_problem *P, int k, long j, long nk)
{
    return P->lo[k] + (double)j * spacing(P, k, nk);
}

/* Transport speed along axis k on the lines through node jp of the partner axis:
 * v_k along x_k, E_k = -x_k along v_k. */
static double vb_speed(const orc_problem *P, int k, long jp, long np)
{
    double c = node(P, vb_partner(P, k), jp, np);
    return k < P->dim / 2 ? c : -c;
}

/* Flux of one axis, Eq. (1): f_k(u) = a_k u (advection) or u^2/2 (Burgers). */
static double flux(const orc_problem *P, int k, double u)
{
    if (P->pde == 1) return (0.5 * u) * u;
    return P->adv[k] * u;
}

/* |f_k'(u)|: |a_k| (advection) or |u| (Burgers). */
static double wave_speed(const orc_problem *P, int k, double u)
{
    if (P->pde == 1) return fabs(u);
    return fabs(P->adv[k]);
}

/* Lax-Friedrichs alpha of Eq. (7) for axis k over one grid: max_j |f_k'(u_j)|. */
double orc_lf_alpha(const orc_problem *P, const int *levels, const double *u, int k)
{
    long n[ORC_MAXD];
    long N = grid_points(P, levels, n), p;
    double a = 0.0;
    if (P->pde == 2) {  /* axis 0: max |v_j|; axis 1: max |E_i| */
        if (k == 0) {
            for (p = 0; p < n[1]; ++p) {
                double s = fabs(vnode(P, p, n[1]));
                if (s > a) a = s;
            }
        } else {
            double *E = (double *)malloc(sizeof(double) * n[0]);
            orc_efield(P, levels, u, E);
            for (p = 0; p < n[0]; ++p) {
                double s = fabs(E[p]);
                if (s > a) a = s;
            }
            free(E);
        }
        return a;
    }
    if (P->pde == 4) {  /* xi_2 along x_2; E_1 + xi_2 B_3 along xi_1; E_2 - xi_1 B_3 along xi_2 */
        const double *E1 = u + N, *E2 = E1 + n[0], *B3 = E2 + n[0];
        long i, j;
        if (k == 0) {
            for (j = 0; j < n[2]; ++j) {
                double s = fabs(node(P, 2, j, n[2]));
                if (s > a) a = s;
            }
        } else {
            for (i = 0; i < n[0]; ++i)
                for (j = 0; j < n[3 - k]; ++j) {
                    double xi = node(P, 3 - k, j, n[3 - k]);
                    double s = fabs(k == 1 ? E1[i] + xi * B3[i] : E2[i] - xi * B3[i]);
                    if (s > a) a = s;
                }
        }
        return a;
    }
    if (P->pde == 3) {  /* the largest |speed| of the axis: |v_k| or |x_k| at the nodes */
        int pk = vb_partner(P, k);
        for (p = 0; p < n[pk]; ++p) {
            double s = fabs(vb_speed(P, k, p, n[pk]));
            if (s > a) a = s;
        }
        return a;
    }
    for (p = 0; p < N; ++p) {
        double s = wave_speed(P, k, u[p]);
        if (s > a) a = s;
    }
    return a;
}

/* Vlasov-Poisson spatial operator: as below, with the line's own wave speed (v_j along x,
 * E_i along v) in the split (7), and zero values beyond the ends of v (n_v + 1 interfaces). */
static void vp_operator(const orc_problem *P, const int *levels, const double *u, const long *n,
                        double *L)
{
    long nx = n[0], nv = n[1], i, j;
    double *E = (double *)malloc(sizeof(double) * nx);
    double ax = orc_lf_alpha(P, levels, u, 0);
    double av;
    double rdx = 1.0 / spacing(P, 0, nx), rdv = 1.0 / spacing(P, 1, nv);
    long nmax = nx > nv ? nx : nv;
    double *fp = (double *)malloc(sizeof(double) * (nmax + 6));
    double *fm = (double *)malloc(sizeof(double) * (nmax + 6));
    double *F = (double *)malloc(sizeof(double) * (nmax + 1));
    orc_efield(P, levels, u, E);
    av = 0.0;
    for (i = 0; i < nx; ++i)
        if (fabs(E[i]) > av) av = fabs(E[i]);
    /* axis 0 (x, periodic): line j has speed v_j */
    for (j = 0; j < nv; ++j) {
        double a = vnode(P, j, nv);
        for (i = 0; i < nx; ++i) {
            double uj = u[i + nx * j];
            double fj = a * uj;
            fp[i] = 0.5 * (fj + ax * uj);
            fm[i] = 0.5 * (fj - ax * uj);
        }
        for (i = 0; i < nx; ++i) {
            long im2 = (i - 2 + 2 * nx) % nx, im1 = (i - 1 + nx) % nx;
            long ip1 = (i + 1) % nx, ip2 = (i + 2) % nx, ip3 = (i + 3) % nx;
            double fplus = orc_weno5_side(fp[im2], fp[im1], fp[i], fp[ip1], fp[ip2], P->eps, P->scheme == 1);
            double fminus = orc_weno5_side(fm[ip3], fm[ip2], fm[ip1], fm[i], fm[im1], P->eps, P->scheme == 1);
            F[i] = fplus + fminus;
        }
        for (i = 0; i < nx; ++i) {
            long il = (i - 1 + nx) % nx;
            L[i + nx * j] = L[i + nx * j] - (F[i] - F[il]) * rdx;
        }
    }
    /* axis 1 (v, zero beyond the ends): line i has speed E_i; fp/fm hold nodes -3..nv+2
       at offset 3, interfaces m + 1/2 for m = -1..nv-1 at F[m + 1] */
    for (i = 0; i < nx; ++i) {
        double a = E[i];
        long m;
        for (m = -3; m < nv + 3; ++m) {
            double uj = (m < 0 || m >= nv) ? 0.0 : u[i + nx * m];
            double fj = a * uj;
            fp[m + 3] = 0.5 * (fj + av * uj);
            fm[m + 3] = 0.5 * (fj - av * uj);
        }
        for (m = -1; m < nv; ++m) {
            const double *P5 = fp + m + 3, *M5 = fm + m + 3;
            double fplus = orc_weno5_side(P5[-2], P5[-1], P5[0], P5[1], P5[2], P->eps, P->scheme == 1);
            double fminus = orc_weno5_side(M5[3], M5[2], M5[1], M5[0], M5[-1], P->eps, P->scheme == 1);
            F[m + 1] = fplus + fminus;
        }
        for (m = 0; m < nv; ++m) L[i + nx * m] = L[i + nx * m] - (F[m + 1] - F[m]) * rdv;
    }
    free(E);
    free(fp);
    free(fm);
    free(F);
}

/* Density of one grid (pde 3): rho[ix] = (h_{v_1} ... h_{v_d}) sum_jv f[ix + nx jv] over the
 * flattened velocity index jv in ascending order; ix is the flattened space index. */
void orc_vb_density(const orc_problem *P, const int *levels, const double *u, double *rho)
{
    long n[ORC_MAXD], nx = 1, nv = 1, ix, jv;
    double hv = 1.0;
    int k, d = P->dim / 2;
    grid_points(P, levels, n);
    for (k = 0; k < d; ++k) nx *= n[k];
    for (k = d; k < P->dim; ++k) {
        nv *= n[k];
        hv = hv * spacing(P, k, n[k]);
    }
    for (ix = 0; ix < nx; ++ix) {
        double s = 0.0;
        for (jv = 0; jv < nv; ++jv) s = s + u[ix + nx * jv];
        rho[ix] = hv * s;
    }
}

/* Absolute Maxwellian mu_inf at the flattened velocity node jv (pde 3). */
double orc_vb_maxwellian(const orc_problem *P, const long *n, long jv)
{
    int k, d = P->dim / 2;
    double s = 0.0;
    for (k = d; k < P->dim; ++k) {
        double v = node(P, k, jv % n[k], n[k]);
        jv /= n[k];
        s = s + v * v;
    }
    return exp(-(s / (2.0 * P->theta))) / pow(2.0 * 3.14159265358979323846 * P->theta, 0.5 * (double)d);
}

/* Vlasov-Boltzmann operator (pde 3): for axes 0, 1, ... the LF-split WENO5 flux difference
 * of f_k = speed * u, the speed constant on each line (v_k along x_k, -x_k along v_k),
 * values zero beyond both ends (n_k + 1 interfaces per line); then
 * L += (mu_inf(v) rho(x) - u) / tau. */
static void vb_operator(const orc_problem *P, const int *levels, const double *u, const long *n,
                        double *L)
{
    long stride[ORC_MAXD], N = 1, nmax = 0, nx = 1, p;
    int k, d = P->dim / 2;
    double *fp, *fm, *F, *rho;
    for (k = 0; k < P->dim; ++k) {
        stride[k] = N;
        N *= n[k];
        if (n[k] > nmax) nmax = n[k];
    }
    for (k = 0; k < d; ++k) nx *= n[k];
    fp = (double *)malloc(sizeof(double) * (nmax + 6));
    fm = (double *)malloc(sizeof(double) * (nmax + 6));
    F = (double *)malloc(sizeof(double) * (nmax + 1));
    for (k = 0; k < P->dim; ++k) {
        int pk = vb_partner(P, k);
        long nk = n[k], sk = stride[k], nlines = N / nk, line, m;
        double alpha = orc_lf_alpha(P, levels, u, k);
        double rdx = 1.0 / spacing(P, k, nk);
        for (line = 0; line < nlines; ++line) {
            long below = line % sk, above = line / sk;
            long base = below + above * sk * nk;
            double a = vb_speed(P, k, (base / stride[pk]) % n[pk], n[pk]);
            /* fp/fm hold nodes -3..nk+2 at offset 3; interface m + 1/2 (m = -1..nk-1) at F[m + 1] */
            for (m = -3; m < nk + 3; ++m) {
                double uj = (m < 0 || m >= nk) ? 0.0 : u[base + m * sk];
                double fj = a * uj;
                fp[m + 3] = 0.5 * (fj + alpha * uj);
                fm[m + 3] = 0.5 * (fj - alpha * uj);
            }
            for (m = -1; m < nk; ++m) {
                const double *P5 = fp + m + 3, *M5 = fm + m + 3;
                double fplus = orc_weno5_side(P5[-2], P5[-1], P5[0], P5[1], P5[2], P->eps, P->scheme == 1);
                double fminus = orc_weno5_side(M5[3], M5[2], M5[1], M5[0], M5[-1], P->eps, P->scheme == 1);
                F[m + 1] = fplus + fminus;
            }
            for (m = 0; m < nk; ++m) L[base + m * sk] = L[base + m * sk] - (F[m + 1] - F[m]) * rdx;
        }
    }
    rho = (double *)malloc(sizeof(double) * nx);
    orc_vb_density(P, levels, u, rho);
    for (p = 0; p < N; ++p) {
        double mu = orc_vb_maxwellian(P, n, p / nx);
        L[p] = L[p] + (mu * rho[p % nx] - u[p]) / P->tau;
    }
    free(rho);
    free(fp);
    free(fm);
    free(F);
}

/* Currents of one Vlasov-Maxwell grid (pde 4): j_m[i] = (h_1 h_2) sum_xi f xi_m over the
 * velocity nodes in ascending flattened order (xi_1 fastest). */
void orc_vm_currents(const orc_problem *P, const int *levels, const double *u, double *j1, double *j2)
{
    long n[ORC_MAXD], i, a, b;
    double hv;
    grid_points(P, levels, n);
    hv = 1.0;
    hv = hv * spacing(P, 1, n[1]);
    hv = hv * spacing(P, 2, n[2]);
    for (i = 0; i < n[0]; ++i) {
        double s1 = 0.0, s2 = 0.0;
        for (b = 0; b < n[2]; ++b)
            for (a = 0; a < n[1]; ++a) {
                double fv = u[i + n[0] * (a + n[1] * b)];
                s1 = s1 + fv * node(P, 1, a, n[1]);
                s2 = s2 + fv * node(P, 2, b, n[2]);
            }
        j1[i] = hv * s1;
        j2[i] = hv * s2;
    }
}

/* -(F_{i+1/2} - F_{i-1/2}) / h of the LF-split WENO5 flux of f = a u on a periodic line of n
 * values (alpha = |a|), into out. */
static void weno_periodic_line(const orc_problem *P, const double *u, long n, double a, double rdx,
                               double *out)
{
    double alpha = fabs(a);
    double *fp = (double *)malloc(sizeof(double) * n);
    double *fm = (double *)malloc(sizeof(double) * n);
    double *F = (double *)malloc(sizeof(double) * n);
    long i;
    for (i = 0; i < n; ++i) {
        double fj = a * u[i];
        fp[i] = 0.5 * (fj + alpha * u[i]);
        fm[i] = 0.5 * (fj - alpha * u[i]);
    }
    for (i = 0; i < n; ++i) {
        long im2 = (i - 2 + 2 * n) % n, im1 = (i - 1 + n) % n;
        long ip1 = (i + 1) % n, ip2 = (i + 2) % n, ip3 = (i + 3) % n;
        double fplus = orc_weno5_side(fp[im2], fp[im1], fp[i], fp[ip1], fp[ip2], P->eps, P->scheme == 1);
        double fminus = orc_weno5_side(fm[ip3], fm[ip2], fm[ip1], fm[i], fm[im1], P->eps, P->scheme == 1);
        F[i] = fplus + fminus;
    }
    for (i = 0; i < n; ++i) out[i] = 0.0 - (F[i] - F[(i - 1 + n) % n]) * rdx;
    free(fp);
    free(fm);
    free(F);
}

/* Vlasov-Maxwell operator (pde 4): f by the periodic LF-split WENO5 flux differences of
 * speed * f along each axis (axis order, L = ((0 - D_0) - D_1) - D_2), the speed constant on
 * each line; the fields by the characteristic form of Maxwell's equations (see the header). */
static void vm_operator(const orc_problem *P, const int *levels, const double *u, const long *n,
                        double *L)
{
    long N = n[0] * n[1] * n[2], nx = n[0], stride[3], k, i;
    const double *E1 = u + N, *E2 = E1 + nx, *B3 = E2 + nx;
    double *LE1 = L + N, *LE2 = LE1 + nx, *LB3 = LE2 + nx;
    long nmax = n[0] > n[1] ? n[0] : n[1];
    double *fp, *fm, *F, *j1, *j2, *wp, *wm, *Lp, *Lm;
    if (n[2] > nmax) nmax = n[2];
    stride[0] = 1;
    stride[1] = n[0];
    stride[2] = n[0] * n[1];
    fp = (double *)malloc(sizeof(double) * nmax);
    fm = (double *)malloc(sizeof(double) * nmax);
    F = (double *)malloc(sizeof(double) * nmax);
    for (k = 0; k < 3; ++k) {
        long nk = n[k], sk = stride[k], nlines = N / nk, line;
        double alpha = orc_lf_alpha(P, levels, u, (int)k);
        double rdx = 1.0 / spacing(P, (int)k, nk);
        for (line = 0; line < nlines; ++line) {
            long below = line % sk, above = line / sk;
            long base = below + above * sk * nk;
            long ix = base % n[0];
            double a;
            if (k == 0) a = node(P, 2, (base / stride[2]) % n[2], n[2]);
            else if (k == 1) a = E1[ix] + node(P, 2, (base / stride[2]) % n[2], n[2]) * B3[ix];
            else a = E2[ix] - node(P, 1, (base / stride[1]) % n[1], n[1]) * B3[ix];
            for (i = 0; i < nk; ++i) {
                double uj = u[base + i * sk];
                double fj = a * uj;
                fp[i] = 0.5 * (fj + alpha * uj);
                fm[i] = 0.5 * (fj - alpha * uj);
            }
            for (i = 0; i < nk; ++i) {
                long im2 = (i - 2 + 2 * nk) % nk, im1 = (i - 1 + nk) % nk;
                long ip1 = (i + 1) % nk, ip2 = (i + 2) % nk, ip3 = (i + 3) % nk;
                double fplus = orc_weno5_side(fp[im2], fp[im1], fp[i], fp[ip1], fp[ip2], P->eps, P->scheme == 1);
                double fminus = orc_weno5_side(fm[ip3], fm[ip2], fm[ip1], fm[i], fm[im1], P->eps, P->scheme == 1);
                F[i] = fplus + fminus;
            }
            for (i = 0; i < nk; ++i) {
                long il = (i - 1 + nk) % nk;
                L[base + i * sk] = L[base + i * sk] - (F[i] - F[il]) * rdx;
            }
        }
    }
    free(fp);
    free(fm);
    free(F);
    /* fields */
    j1 = (double *)malloc(sizeof(double) * nx);
    j2 = (double *)malloc(sizeof(double) * nx);
    wp = (double *)calloc((size_t)nx, sizeof(double));
    wm = (double *)calloc((size_t)nx, sizeof(double));
    Lp = (double *)malloc(sizeof(double) * nx);
    Lm = (double *)malloc(sizeof(double) * nx);
    orc_vm_currents(P, levels, u, j1, j2);
    for (i = 0; i < nx; ++i) {
        wp[i] = E1[i] + B3[i];
        wm[i] = E1[i] - B3[i];
    }
    weno_periodic_line(P, wp, nx, -1.0, 1.0 / spacing(P, 0, nx), Lp);
    weno_periodic_line(P, wm, nx, 1.0, 1.0 / spacing(P, 0, nx), Lm);
    for (i = 0; i < nx; ++i) {
        double lp = Lp[i] - j1[i], lm = Lm[i] - j1[i];
        LE1[i] = 0.5 * (lp + lm);
        LE2[i] = 0.0 - j2[i];
        LB3[i] = 0.5 * (lp - lm);
    }
    free(j1);
    free(j2);
    free(wp);
    free(wm);
    free(Lp);
    free(Lm);
}

/* ------------------------------------------------------------------------------------
 * Spatial operator L(u) = - sum_k (fhat_{i+1/2} - fhat_{i-1/2}) / h_k, Eq. (2) applied
 * dimension by dimension (Section 2.1), with the LF split (7) and fhat = fhat^+ + fhat^-.
 * L accumulates axis 0 first: L = ((0 - D_0) - D_1) - ..., D_k = (F_r - F_l) * (1/h_k).
 * ---------------------------------------------------------------------------------- */
void orc_spatial_operator(const orc_problem *P, const int *levels, const double *u, double *L)
{
    long n[ORC_MAXD], stride[ORC_MAXD];
    long N = grid_points(P, levels, n), p;
    int k;
    stride[0] = 1;
    for (k = 1; k < P->dim; ++k) stride[k] = stride[k - 1] * n[k - 1];
    for (p = 0; p < N; ++p) L[p] = 0.0;
    if (P->pde == 2) {
        vp_operator(P, levels, u, n, L);
        return;
    }
    if (P->pde == 3) {
        vb_operator(P, levels, u, n, L);
        return;
    }
    if (P->pde == 4) {
        for (p = N; p < orc_state_points(P, levels); ++p) L[p] = 0.0;
        vm_operator(P, levels, u, n, L);
        return;
    }

    for (k = 0; k < P->dim; ++k) {
        long nk = n[k], sk = stride[k], i, line;
        double alpha = orc_lf_alpha(P, levels, u, k);
        double rdx = 1.0 / spacing(P, k, nk);
        double *fp = (double *)malloc(sizeof(double) * (nk + 6));
        double *fm = (double *)malloc(sizeof(double) * (nk + 6));
        double *F = (double *)malloc(sizeof(double) * (nk + 1));
        long nlines = N / nk;
        if (zero_axis(P, k)) {
            /* zero boundary: u = 0 at the three ghost nodes beyond either end, so f = 0 and
               f^+- = 0 there; interfaces m + 1/2, m = -1..n_k-1, at F[m + 1] */
            for (line = 0; line < nlines; ++line) {
                long below = line % sk, above = line / sk;
                long base = below + above * sk * nk, m;
                for (m = -3; m < nk + 3; ++m) {
                    double uj = (m < 0 || m >= nk) ? 0.0 : u[base + m * sk];
                    double fj = flux(P, k, uj);
                    fp[m + 3] = 0.5 * (fj + alpha * uj);
                    fm[m + 3] = 0.5 * (fj - alpha * uj);
                }
                for (m = -1; m < nk; ++m) {
                    const double *P5 = fp + m + 3, *M5 = fm + m + 3;
                    double fplus = orc_weno5_side(P5[-2], P5[-1], P5[0], P5[1], P5[2], P->eps,
                                                  P->scheme == 1);
                    double fminus = orc_weno5_side(M5[3], M5[2], M5[1], M5[0], M5[-1], P->eps,
                                                   P->scheme == 1);
                    F[m + 1] = fplus + fminus;
                }
                for (m = 0; m < nk; ++m)
                    L[base + m * sk] = L[base + m * sk] - (F[m + 1] - F[m]) * rdx;
            }
            free(fp);
            free(fm);
            free(F);
            continue;
        }
        for (line = 0; line < nlines; ++line) {
            /* base offset of this line: the index with i_k = 0 */
            long below = line % sk, above = line / sk;
            long base = below + above * sk * nk;
            for (i = 0; i < nk; ++i) {
                double uj = u[base + i * sk];
                double fj = flux(P, k, uj);
                fp[i] = 0.5 * (fj + alpha * uj);
                fm[i] = 0.5 * (fj - alpha * uj);
            }
            for (i = 0; i < nk; ++i) {
                /* interface i+1/2, periodic neighbours */
                long im2 = (i - 2 + 2 * nk) % nk, im1 = (i - 1 + nk) % nk;
                long ip1 = (i + 1) % nk, ip2 = (i + 2) % nk, ip3 = (i + 3) % nk;
                double fplus = orc_weno5_side(fp[im2], fp[im1], fp[i], fp[ip1], fp[ip2],
                                              P->eps, P->scheme == 1);
                double fminus = orc_weno5_side(fm[ip3], fm[ip2], fm[ip1], fm[i], fm[im1],
                                               P->eps, P->scheme == 1);
                F[i] = fplus + fminus;
            }
            for (i = 0; i < nk; ++i) {
                long il = (i - 1 + nk) % nk;
                L[base + i * sk] = L[base + i * sk] - (F[i] - F[il]) * rdx;
            }
        }
        free(fp);
        free(fm);
        free(F);
    }
}

/* ------------------------------------------------------------------------------------
 * Third-order TVD Runge-Kutta (Shu-Osher form), cited in Section 2.2:
 *   u1 = u + dt L(u)
 *   u2 = 3/4 u + 1/4 (u1 + dt L(u1))
 *   u  = 1/3 u + 2/3 (u2 + dt L(u2))
 * work must hold 3 * N doubles, N the grid's state size (orc_state_points).
 * ---------------------------------------------------------------------------------- */
void orc_rk3_step(const orc_problem *P, const int *levels, double *u, double dt, double *work)
{
    long N = orc_state_points(P, levels), p;
    double *u1 = work, *u2 = work + N, *L = work + 2 * N;
    orc_spatial_operator(P, levels, u, L);
    for (p = 0; p < N; ++p) u1[p] = u[p] + dt * L[p];
    orc_spatial_operator(P, levels, u1, L);
    for (p = 0; p < N; ++p) u2[p] = 0.75 * u[p] + 0.25 * (u1[p] + dt * L[p]);
    orc_spatial_operator(P, levels, u2, L);
    for (p = 0; p < N; ++p) u[p] = (1.0 / 3.0) * u[p] + (2.0 / 3.0) * (u2[p] + dt * L[p]);
}

/* Finest-grid spacing per axis: (hi_k - lo_k) / (N_r 2^{N_L}). */
static double fine_spacing(const orc_problem *P, int k)
{
    return (P->hi[k] - P->lo[k]) / (double)((long)P->nr << P->nl);
}

/* Nominal time step, Section 3.
 * rule 0: dt = coef * (min_k h_k)^{5/3} on the finest grid.
 * rule 1: dt = cfl / sum_k (alpha_k / h_k), alpha_k = max over all grids of max|f_k'(u)|.
 * grids: all component grids concatenated in enumeration order. */
double orc_dt(const orc_problem *P, int G, const int *levels, const double *grids,
              int rule, double coef, double cfl)
{
    int k, g;
    if (rule == 0) {
        double h = fine_spacing(P, 0);
        for (k = 1; k < P->dim; ++k) {
            double hk = fine_spacing(P, k);
            if (hk < h) h = hk;
        }
        return coef * pow(h, 5.0 / 3.0);
    } else {
        double s = 0.0;
        for (k = 0; k < P->dim; ++k) {
            double a = 0.0;
            const double *u = grids;
            for (g = 0; g < G; ++g) {
                double ag = orc_lf_alpha(P, levels + g * P->dim, u, k);
                if (ag > a) a = ag;
                u += orc_state_points(P, levels + g * P->dim);
            }
            if (P->pde == 4 && k == 0 && a < 1.0) a = 1.0;  /* the fields move at speed 1 */
            s = s + a / fine_spacing(P, k);
        }
        return cfl / s;
    }
}

/* ------------------------------------------------------------------------------------
 * Step 2 of the algorithm (Section 2.2.2): march every component grid with the common
 * time step until t_end (last step shortened) or max_steps steps.  Returns the number of
 * steps taken; *t_out receives the time reached.
 * ---------------------------------------------------------------------------------- */
long orc_solve(const orc_problem *P, int G, const int *levels, double *grids, double t0,
               double t_end, long max_steps, int rule, double coef, double cfl, double *t_out)
{
    long Nmax = 0, steps = 0;
    int g;
    double t = t0;
    double *work;
    for (g = 0; g < G; ++g) {
        long Ng = orc_state_points(P, levels + g * P->dim);
        if (Ng > Nmax) Nmax = Ng;
    }
    work = (double *)malloc(sizeof(double) * 3 * Nmax);
    while (t < t_end && steps < max_steps) {
        double dt = orc_dt(P, G, levels, grids, rule, coef, cfl);
        double *u = grids;
        int last = 0;
        if (dt >= t_end - t) {  /* shortened last step: the run ends exactly at t_end */
            dt = t_end - t;
            last = 1;
        }
        for (g = 0; g < G; ++g) {
            orc_rk3_step(P, levels + g * P->dim, u, dt, work);
            u += orc_state_points(P, levels + g * P->dim);
        }
        t = last ? t_end : t + dt;
        ++steps;
    }
    free(work);
    if (t_out) *t_out = t;
    return steps;
}

/* ------------------------------------------------------------------------------------
 * Step 1: restriction of u_0(x) = b + a sin(w * (x_0 + ... + x_{d-1}) + phi) to a grid: the
 * pointwise restriction of Section 2.2.2, Step 1 (u_0 sampled at the nodes).  The sum runs
 * over axes in order.
 * ---------------------------------------------------------------------------------- */
void orc_restrict_sine(const orc_problem *P, const int *levels, double b, double a, double w,
                       double phi, double *u)
{
    long n[ORC_MAXD], idx[ORC_MAXD];
    long N = grid_points(P, levels, n), p;
    int k;
    for (p = 0; p < N; ++p) {
        long r = p;
        double S = 0.0;
        for (k = 0; k < P->dim; ++k) {
            idx[k] = r % n[k];
            r /= n[k];
            S = S + (P->lo[k] + (double)idx[k] * spacing(P, k, n[k]));
        }
        u[p] = b + a * sin(w * S + phi);
    }
}

/* Landau-damping initial condition of the Vlasov-Poisson workload (pde 2):
 * f_0(x, v) = (1 + a cos(k x)) exp(-v^2 / 2) / sqrt(2 pi) at the nodes of one grid. */
void orc_restrict_landau(const orc_problem *P, const int *levels, double a, double kx, double *u)
{
    long n[ORC_MAXD], i, j;
    grid_points(P, levels, n);
    for (j = 0; j < n[1]; ++j) {
        double v = vnode(P, j, n[1]);
        double m = exp(-0.5 * (v * v)) / sqrt(2.0 * 3.14159265358979323846);
        for (i = 0; i < n[0]; ++i) {
            double x = P->lo[0] + (double)i * spacing(P, 0, n[0]);
            u[i + n[0] * j] = (1.0 + a * cos(kx * x)) * m;
        }
    }
}

/* Electric field energy of one grid, (1/2) sum_i E_i^2 h_x (pde 2). */
double orc_field_energy(const orc_problem *P, const int *levels, const double *u)
{
    long n[ORC_MAXD], i;
    double s = 0.0, *E;
    grid_points(P, levels, n);
    E = (double *)malloc(sizeof(double) * n[0]);
    orc_efield(P, levels, u, E);
    for (i = 0; i < n[0]; ++i) s = s + E[i] * E[i];
    free(E);
    return 0.5 * s * spacing(P, 0, n[0]);
}

/* Example 5 initial condition, without its normalisation: the factor of space axis k,
 * g_0(x) = sin(x^2/2)^2 exp(-x^2/2), g_1(x) = cos(x^2/2)^2 exp(-x^2/2), and of a velocity
 * axis, exp(-v^2/2). */
static double relax_factor(const orc_problem *P, int k, double x)
{
    double e = exp(-0.5 * (x * x));
    if (k >= P->dim / 2) return e;
    if (k == 0) {
        double sn = sin(0.5 * (x * x));
        return (sn * sn) * e;
    } else {
        double cs = cos(0.5 * (x * x));
        return (cs * cs) * e;
    }
}

/* Normalisation s of Example 5: the integral over the domain of the product of the factors
 * above, one composite Simpson rule per axis (the integrand is a product of one-axis
 * functions), 2 * 10^5 intervals per axis. */
double orc_relax_norm(const orc_problem *P)
{
    const long m = 200000;
    double s = 1.0;
    int k;
    for (k = 0; k < P->dim; ++k) {
        double a = P->lo[k], b = P->hi[k], h = (b - a) / (double)m, acc;
        long i;
        acc = relax_factor(P, k, a) + relax_factor(P, k, b);
        for (i = 1; i < m; ++i) acc = acc + (i % 2 ? 4.0 : 2.0) * relax_factor(P, k, a + (double)i * h);
        s = s * (acc * h / 3.0);
    }
    return s;
}

/* Example 5 initial condition at the nodes of one grid (pde 3, dim 2 or 4):
 * f_0 = (1/s) prod_k factor_k(x_k). */
void orc_restrict_relax(const orc_problem *P, const int *levels, double s_norm, double *u)
{
    long n[ORC_MAXD];
    long N = grid_points(P, levels, n), p;
    int k;
    for (p = 0; p < N; ++p) {
        long r = p;
        double f = 1.0;
        for (k = 0; k < P->dim; ++k) {
            f = f * relax_factor(P, k, node(P, k, r % n[k], n[k]));
            r /= n[k];
        }
        u[p] = f / s_norm;
    }
}

/* Entropy functionals of Example 5 on one grid's nodes (pde 3):
 *   H_2 = sum f^2 / M dV,  H_log = sum f log(f / M) dV (nodes with f <= 0 add 0),
 * with the stationary state M = exp(-(|v|^2/2 + |x|^2/2)/theta) / ((2 pi theta)^{d/2} Z),
 * Z = prod_k int_{lo_k}^{hi_k} exp(-x^2 / (2 theta)) dx = prod_k sqrt(pi theta / 2)
 * (erf(hi_k / sqrt(2 theta)) - erf(lo_k / sqrt(2 theta))), and dV the cell volume. */
void orc_relax_entropy(const orc_problem *P, const int *levels, const double *u, double *h2,
                       double *hlog)
{
    long n[ORC_MAXD];
    long N = grid_points(P, levels, n), p;
    int k, d = P->dim / 2;
    double Z = 1.0, vol = 1.0, c, s2 = 0.0, sl = 0.0;
    double rt = sqrt(2.0 * P->theta);
    for (k = 0; k < d; ++k)
        Z = Z * (sqrt(3.14159265358979323846 * P->theta / 2.0) * (erf(P->hi[k] / rt) - erf(P->lo[k] / rt)));
    for (k = 0; k < P->dim; ++k) vol = vol * spacing(P, k, n[k]);
    c = pow(2.0 * 3.14159265358979323846 * P->theta, 0.5 * (double)d) * Z;
    for (p = 0; p < N; ++p) {
        long r = p;
        double q = 0.0, M, f = u[p];
        for (k = 0; k < P->dim; ++k) {
            double x = node(P, k, r % n[k], n[k]);
            r /= n[k];
            q = q + 0.5 * (x * x);
        }
        M = exp(-(q / P->theta)) / c;
        s2 = s2 + (f * f) / M;
        if (f > 0.0) sl = sl + f * log(f / M);
    }
    *h2 = s2 * vol;
    *hlog = sl * vol;
}

/* Example 6 initial state of one Vlasov-Maxwell grid (pde 4): f = exp(-xi_2^2/beta)
 * (delta exp(-(xi_1 - v1)^2/beta) + (1 - delta) exp(-(xi_1 + v2)^2/beta)) / (pi beta) at the
 * nodes, E_1 = E_2 = 0, B_3 = b sin(k0 x_2). */
void orc_restrict_vm(const orc_problem *P, const int *levels, double beta, double delta, double v1,
                     double v2, double b, double k0, double *u)
{
    long n[ORC_MAXD];
    long N = grid_points(P, levels, n), i, a, c;
    double *E1 = u + N, *E2 = E1 + n[0], *B3 = E2 + n[0];
    for (c = 0; c < n[2]; ++c) {
        double x2 = node(P, 2, c, n[2]);
        double g2 = exp(-((x2 * x2) / beta));
        for (a = 0; a < n[1]; ++a) {
            double x1 = node(P, 1, a, n[1]);
            double d1 = x1 - v1, d2 = x1 + v2;
            double g1 = delta * exp(-((d1 * d1) / beta)) + (1.0 - delta) * exp(-((d2 * d2) / beta));
            double f = (g2 * g1) / (3.14159265358979323846 * beta);
            for (i = 0; i < n[0]; ++i) u[i + n[0] * (a + n[1] * c)] = f;
        }
    }
    for (i = 0; i < n[0]; ++i) {
        E1[i] = 0.0;
        E2[i] = 0.0;
        B3[i] = b * sin(k0 * node(P, 0, i, n[0]));
    }
}

/* Energies of one Vlasov-Maxwell grid (pde 4): kinetic sum f |xi|^2/2 dV and field
 * sum (E_1^2 + E_2^2 + B_3^2)/2 dx. */
void orc_vm_energy(const orc_problem *P, const int *levels, const double *u, double *kinetic,
                   double *field)
{
    long n[ORC_MAXD];
    long N = grid_points(P, levels, n), i, a, c;
    const double *E1 = u + N, *E2 = E1 + n[0], *B3 = E2 + n[0];
    double sk = 0.0, sf = 0.0, hx = spacing(P, 0, n[0]);
    double dV = hx * spacing(P, 1, n[1]) * spacing(P, 2, n[2]);
    for (c = 0; c < n[2]; ++c) {
        double x2 = node(P, 2, c, n[2]);
        for (a = 0; a < n[1]; ++a) {
            double x1 = node(P, 1, a, n[1]);
            double e = 0.5 * (x1 * x1 + x2 * x2);
            for (i = 0; i < n[0]; ++i) sk = sk + u[i + n[0] * (a + n[1] * c)] * e;
        }
    }
    for (i = 0; i < n[0]; ++i) sf = sf + 0.5 * (E1[i] * E1[i] + E2[i] * E2[i] + B3[i] * B3[i]);
    *kinetic = sk * dV;
    *field = sf * hx;
}

/* ------------------------------------------------------------------------------------
 * One-dimensional fifth-order interpolation at x = x_i + s h, s in [-1/2, 1/2),
 * Section 2.2.1, Eqs. (8)-(11).  (a..e) = (u_{i-2}, ..., u_{i+2}).
 * P_k are the quadratics through the substencils S_0, S_1, S_2; C_k the linear weights
 * printed after (8); beta_k of (10) evaluate to the formulas of Eq. (6).
 * lagrange != 0 gives the Lagrange interpolant (8); otherwise the WENO interpolant (11).
 * ---------------------------------------------------------------------------------- */
double orc_weno5_interp(double a, double b, double c, double d, double e, double s, double eps,
                        int lagrange)
{
    double g0 = 0.5 * (a - 4.0 * b + 3.0 * c), k0 = 0.5 * (a - 2.0 * b + c);
    double g1 = 0.5 * (d - b), k1 = 0.5 * (b - 2.0 * c + d);
    double g2 = 0.5 * (-3.0 * c + 4.0 * d - e), k2 = 0.5 * (c - 2.0 * d + e);
    double P0 = c + s * (g0 + s * k0);
    double P1 = c + s * (g1 + s * k1);
    double P2 = c + s * (g2 + s * k2);
    double C0 = ((s - 1.0) * (s - 2.0)) / 12.0;
    double C1 = (4.0 - s * s) / 6.0;
    double C2 = ((s + 1.0) * (s + 2.0)) / 12.0;
    double w0, w1, w2;
    if (s == 0.0) return c;  /* coincident node */
    if (lagrange) {
        return C0 * P0 + C1 * P1 + C2 * P2;
    } else {
        double t0 = a - 2.0 * b + c, s0 = a - 4.0 * b + 3.0 * c;
        double t1 = b - 2.0 * c + d, s1 = b - d;
        double t2 = c - 2.0 * d + e, s2 = 3.0 * c - 4.0 * d + e;
        double b0 = (13.0 / 12.0) * (t0 * t0) + 0.25 * (s0 * s0);
        double b1 = (13.0 / 12.0) * (t1 * t1) + 0.25 * (s1 * s1);
        double b2 = (13.0 / 12.0) * (t2 * t2) + 0.25 * (s2 * s2);
        /* Eq. (9): tilde C_k = C_k / (eps + beta_k)^2, w_k = tilde C_k / sum */
        w0 = C0 / ((eps + b0) * (eps + b0));
        w1 = C1 / ((eps + b1) * (eps + b1));
        w2 = C2 / ((eps + b2) * (eps + b2));
        return (w0 * P0 + w1 * P1 + w2 * P2) / (w0 + w1 + w2);
    }
}

/* Axes with zero values beyond the ends: v of the Vlasov-Poisson workload, every axis of
 * the Vlasov-Boltzmann model; the others are periodic. */
static int zero_axis(const orc_problem *P, int k)
{
    return (P->pde == 2 && k == 1) || P->pde == 3 || (P->pde <= 1 && P->bc[k] == 1);
}

/* Coarse centre and offset of fine node jf on an axis refined by ratio r = 2^{N_L - l}:
 * t = jf / r, centre i = floor(t + 1/2), s = t - i in [-1/2, 1/2). */
static void fine_to_coarse(long jf, long r, long *ic, double *s)
{
    long i = jf / r, m = jf % r;
    if (2 * m < r) {
        *ic = i;
        *s = (double)m / (double)r;
    } else {
        *ic = i + 1;
        *s = (double)(m - r) / (double)r;
    }
}

/* ------------------------------------------------------------------------------------
 * Prolongation P^{N_L..N_L} U of one grid onto the finest grid, dimension by dimension,
 * axis 0 first (Section 2.2.1).  out holds (N_r 2^{N_L})^d values; work must hold two
 * arrays of that size.
 * ---------------------------------------------------------------------------------- */
void orc_prolong_grid(const orc_problem *P, const int *levels, const double *u, double *out,
                      double *work)
{
    long n[ORC_MAXD], m[ORC_MAXD];
    long Nf = (long)P->nr << P->nl;
    long N = grid_points(P, levels, n), p;
    int k, j;
    double *src = work, *dst = work + 0;
    double *bufA = work, *bufB = NULL;
    long tot;
    /* two ping-pong buffers of Nf^d each */
    tot = 1;
    for (k = 0; k < P->dim; ++k) tot *= Nf;
    bufB = work + tot;
    for (p = 0; p < N; ++p) bufA[p] = u[p];
    for (k = 0; k < P->dim; ++k) m[k] = n[k];
    src = bufA;
    dst = bufB;
    for (k = 0; k < P->dim; ++k) {
        long r, below, above, Min, Mout, q;
        if (levels[k] == P->nl) continue;  /* axis already at the finest level */
        r = 1L << (P->nl - levels[k]);
        below = 1;
        for (j = 0; j < k; ++j) below *= m[j];
        above = 1;
        for (j = k + 1; j < P->dim; ++j) above *= m[j];
        Min = m[k];
        Mout = Nf;
        for (q = 0; q < below * above; ++q) {
            long lo_i = q % below, hi_i = q / below, jf;
            const double *line = src + lo_i + hi_i * below * Min;
            double *oline = dst + lo_i + hi_i * below * Mout;
            for (jf = 0; jf < Mout; ++jf) {
                long ic;
                double s;
                fine_to_coarse(jf, r, &ic, &s);
                if (zero_axis(P, k)) {  /* zero beyond the ends */
                    double v5[5];
                    int t;
                    for (t = 0; t < 5; ++t) {
                        long c = ic - 2 + t;
                        v5[t] = (c < 0 || c >= Min) ? 0.0 : line[c * below];
                    }
                    oline[jf * below] = orc_weno5_interp(v5[0], v5[1], v5[2], v5[3], v5[4], s, P->eps,
                                                         P->prolong == 1);
                } else {
                    double a = line[((ic - 2) % Min + Min) % Min * below];
                    double b = line[((ic - 1) % Min + Min) % Min * below];
                    double c = line[((ic) % Min + Min) % Min * below];
                    double d = line[((ic + 1) % Min + Min) % Min * below];
                    double e = line[((ic + 2) % Min + Min) % Min * below];
                    oline[jf * below] = orc_weno5_interp(a, b, c, d, e, s, P->eps, P->prolong == 1);
                }
            }
        }
        m[k] = Nf;
        {
            double *t = src;
            src = dst;
            dst = t;
        }
    }
    tot = 1;
    for (k = 0; k < P->dim; ++k) tot *= Nf;
    for (p = 0; p < tot; ++p) out[p] = src[p];
}

/* Step 3 (combination), Eqs. (12)-(15): uhat = sum_g c_g P U_g, grids in enumeration
 * order.  grids: concatenated in enumeration order.  work: 3 * Nf^d doubles. */
void orc_combine(const orc_problem *P, int G, const int *levels, const double *coeff,
                 const double *grids, double *uhat, double *work)
{
    long Nf = (long)P->nr << P->nl, tot = 1, p;
    int k, g;
    const double *u = grids;
    double *pu = work, *pw = work + 0;
    for (k = 0; k < P->dim; ++k) tot *= Nf;
    pw = work + tot;
    for (p = 0; p < tot; ++p) uhat[p] = 0.0;
    for (g = 0; g < G; ++g) {
        orc_prolong_grid(P, levels + g * P->dim, u, pu, pw);
        for (p = 0; p < tot; ++p) uhat[p] = uhat[p] + coeff[g] * pu[p];
        u += orc_state_points(P, levels + g * P->dim);
    }
}

/* Pointwise prolongation: the value of P U at one finest-grid node J, evaluated by the
 * same dimension-by-dimension recursion (axis d-1 interpolates values that are fine in
 * axes 0..d-2).  Each intermediate value is computed by exactly the arithmetic of
 * orc_prolong_grid, so the two agree bit for bit. */
static double prolong_rec(const orc_problem *P, const int *levels, const long *n,
                          const double *u, int k, const long *J, long *ci)
{
    /* value of the array after prolonging axes 0..k, at fine indices J[0..k] and coarse
     * indices ci[k+1..d-1] */
    long Nf = (long)P->nr << P->nl;
    long ic, r, t;
    double s, v[5];
    if (k < 0) {
        long p = 0, st = 1;
        int j;
        for (j = 0; j < P->dim; ++j) {
            p += ci[j] * st;
            st *= n[j];
        }
        return u[p];
    }
    if (levels[k] == P->nl) {
        ci[k] = J[k];
        return prolong_rec(P, levels, n, u, k - 1, J, ci);
    }
    r = 1L << (P->nl - levels[k]);
    (void)Nf;
    fine_to_coarse(J[k], r, &ic, &s);
    if (s == 0.0) {
        ci[k] = ((ic % n[k]) + n[k]) % n[k];
        return prolong_rec(P, levels, n, u, k - 1, J, ci);
    }
    for (t = 0; t < 5; ++t) {
        if (zero_axis(P, k)) {  /* zero beyond the ends */
            long c = ic - 2 + t;
            if (c < 0 || c >= n[k]) {
                v[t] = 0.0;
                continue;
            }
            ci[k] = c;
        } else {
            ci[k] = (((ic - 2 + t) % n[k]) + n[k]) % n[k];
        }
        v[t] = prolong_rec(P, levels, n, u, k - 1, J, ci);
    }
    return orc_weno5_interp(v[0], v[1], v[2], v[3], v[4], s, P->eps, P->prolong == 1);
}

double orc_prolong_point(const orc_problem *P, const int *levels, const double *u, const long *J)
{
    long n[ORC_MAXD], ci[ORC_MAXD];
    grid_points(P, levels, n);
    return prolong_rec(P, levels, n, u, P->dim - 1, J, ci);
}

/* uhat at one finest-grid node, summed over grids in enumeration order. */
double orc_combine_point(const orc_problem *P, int G, const int *levels, const double *coeff,
                         const double *grids, const long *J)
{
    double acc = 0.0;
    const double *u = grids;
    int g;
    for (g = 0; g < G; ++g) {
        acc = acc + coeff[g] * orc_prolong_point(P, levels + g * P->dim, u, J);
        u += orc_state_points(P, levels + g * P->dim);
    }
    return acc;
}

/* ------------------------------------------------------------------------------------
 * Diagnostics: mass sum_j u_j prod_k h_k of one grid (conserved under periodic boundary
 * conditions, Eq. (2) telescopes), and the exact solutions the error norms use.
 * ---------------------------------------------------------------------------------- */
double orc_mass(const orc_problem *P, const int *levels, const double *u)
{
    long n[ORC_MAXD];
    long N = grid_points(P, levels, n), p;
    double vol = 1.0, s = 0.0;
    int k;
    for (k = 0; k < P->dim; ++k) vol = vol * spacing(P, k, n[k]);
    for (p = 0; p < N; ++p) s = s + u[p];
    return s * vol;
}

/* Exact solution for u_0 = b + a sin(w sum_k x_k + phi):
 *   advection:  u(x, t) = u_0(x - a t);
 *   Burgers:    u = u_0(x - u t 1), i.e. u = b + a sin(w (S - d u t) + phi), solved by
 *               Newton's method (valid before the shock time 1/(a w d)). */
double orc_exact_sine(const orc_problem *P, double b, double a, double w, double phi,
                      const double *x, double t)
{
    int k, it;
    double S = 0.0;
    if (P->pde == 0) {
        for (k = 0; k < P->dim; ++k) S = S + (x[k] - P->adv[k] * t);
        return b + a * sin(w * S + phi);
    }
    for (k = 0; k < P->dim; ++k) S = S + x[k];
    {
        double d = (double)P->dim, u = b + a * sin(w * S + phi);
        for (it = 0; it < 100; ++it) {
            double arg = w * (S - d * u * t) + phi;
            double F = u - b - a * sin(arg);
            double dF = 1.0 + a * w * d * t * cos(arg);
            double du = F / dF;
            u = u - du;
            if (fabs(du) <= 1e-16 * (1.0 + fabs(u))) break;
        }
        return u;
    }
}

/* L^1 (mean absolute) and L^inf errors of the combined solution on the finest grid. */
void orc_error_norms(const orc_problem *P, const double *uhat, double b, double a, double w,
                     double phi, double t, double *l1, double *linf)
{
    long Nf = (long)P->nr << P->nl, tot = 1, p;
    int k;
    double x[ORC_MAXD], s = 0.0, mx = 0.0;
    for (k = 0; k < P->dim; ++k) tot *= Nf;
    for (p = 0; p < tot; ++p) {
        long r = p;
        double err;
        for (k = 0; k < P->dim; ++k) {
            x[k] = P->lo[k] + (double)(r % Nf) * fine_spacing(P, k);
            r /= Nf;
        }
        err = fabs(uhat[p] - orc_exact_sine(P, b, a, w, phi, x, t));
        s = s + err;
        if (err > mx) mx = err;
    }
    *l1 = s / (double)tot;
    *linf = mx;
}
