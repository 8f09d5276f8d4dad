/*
 * sgweno.h -- C ABI of the GB300 sparse-grid fifth-order WENO library (libsgweno.so).
 *
 * The library advances a scalar conservation law u_t + div f(u) = 0 (Eq. 1 of Zhu &
 * Zhang, arXiv 2007.10196) on every semi-coarsened grid of the sparse-grid combination
 * technique with the fifth-order finite-difference WENO scheme and Lax-Friedrichs flux
 * splitting (Section 2.1, Eqs. 2-7) inside third-order TVD Runge-Kutta (Section 2.2),
 * then prolongs every grid onto the finest grid with fifth-order WENO interpolation
 * (Section 2.2.1, Eqs. 8-11) and forms the signed combination sum (Eqs. 12-15).  The
 * three steps are the algorithm of Section 2.2.2.
 *
 * Conventions shared by every call:
 *  - All functions return sg_status (SG_OK = 0).  Nothing aborts, traps or throws across
 *    the ABI.  After any error the handle stays valid and destroyable; sg_last_error()
 *    returns a message for the calling thread's last failure.
 *  - Handles are not thread safe: one host thread at a time per handle.
 *  - Host buffers passed in are owned by the caller and only read or written during the
 *    call.  Device memory is owned by the library (allocated through the allocator hook if
 *    one is installed, else cudaMalloc) and released by sg_destroy.
 *  - Grid arrays are stored axis 0 fastest: index = i_0 + n_0 (i_1 + n_1 (i_2 + ...)).
 *  - Grid g has levels l^g and n_k = N_r 2^{l^g_k} periodic nodes x_j = lo_k + j h_k,
 *    h_k = (hi_k - lo_k)/n_k, j = 0..n_k-1 (vertex-centred, Section 2.2).
 *  - Grids are enumerated q = 0..d-1, levels with |l| = N_L - q in lexicographic order
 *    (l_0 most significant); grid g has combination coefficient (-1)^q C(d-1, q), Eq. (13).
 *  - There is no CPU fallback.  Every computation runs in the library's CUDA kernels on
 *    the current CUDA device; SG_ERR_CUDA reports a CUDA runtime failure.
 */
#ifndef SGWENO_H
#define SGWENO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SG_OK = 0,
    SG_ERR_ARG = 1,         /* invalid argument (range, size, NULL pointer) */
    SG_ERR_STATE = 2,       /* call out of order (e.g. step before init) */
    SG_ERR_NOMEM = 3,       /* device or host allocation failed */
    SG_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    SG_ERR_NONFINITE = 5,   /* a NaN or Inf appeared in the solution */
    SG_ERR_TIMEOUT = 6,     /* a bounded wait ran out */
    SG_ERR_UNSUPPORTED = 7  /* valid request the library does not implement */
} sg_status;

/* PDE of Eq. (1): linear advection f_k(u) = a_k u, or Burgers f_k(u) = u^2/2 on every axis.
 * SG_PDE_VLASOV: the 1D1V Vlasov-Poisson system f_t + v f_x + E(x) f_v = 0 (not in the paper;
 * the kinetic workload run on the same method), dim = 2 with axis 0 = x (periodic) and axis 1
 * = v (f = 0 beyond the v nodes: zero inflow; bc is ignored).  Every component grid carries
 * its own field: rho_i = h_v sum_j f_ij, E from dE/dx = rho - mean(rho) integrated by the
 * trapezoid rule from E_0 = 0 and shifted to zero mean, recomputed at every RK stage; the LF
 * alpha of Eq. (7) is max|v_j| along x and max|E_i| along v. */
/* SG_PDE_VLASOV_BOLTZMANN: the relaxation model of Example 5,
 *   f_t + v . grad_x f + E(x) . grad_v f = (mu_inf(v) rho(x) - f) / tau,  E = -x,
 * dim = 2 d (d = 1, 2 or 3): axes 0..d-1 are x, axes d..2d-1 are v.  Every axis has nodes
 * lo_k + j h_k, j = 0..n_k-1, with f = 0 beyond them (the zero boundary condition; bc is
 * ignored).  The flux along x_k is v_k f and along v_k it is -x_k f, with the line's node on
 * the partner axis; the LF alpha of an axis is the largest |partner node| of the grid.
 * rho(x) = (h_{v_1} ... h_{v_d}) sum_v f(x, v) is formed from the input of every RK stage;
 * mu_inf(v) = exp(-(|v|^2 / (2 theta))) / (2 pi theta)^{d/2} at the velocity nodes (theta and
 * tau from sg_params). */
enum { SG_PDE_ADVECTION = 0, SG_PDE_BURGERS = 1, SG_PDE_VLASOV = 2, SG_PDE_VLASOV_BOLTZMANN = 3 };
/* Boundary conditions per axis, for SG_PDE_ADVECTION and SG_PDE_BURGERS (the kinetic PDEs imply
 * theirs: SG_PDE_VLASOV zero inflow in v, SG_PDE_VLASOV_BOLTZMANN zero on every axis; bc is
 * ignored for them).
 * SG_BC_PERIODIC: n_k periodic nodes x_j = lo_k + j h_k, j = 0..n_k-1.
 * SG_BC_ZERO: the same nodes, and u = 0 beyond them -- at x_{-3..-1} and x_{n_k..n_k+2} in the
 *   WENO5 stencils, at the two nodes beyond either end in the interpolation of Eqs. (8)-(11):
 *   the zero boundary treatment of Example 5 (Section 3.5) applied to Eq. (1). */
enum { SG_BC_PERIODIC = 0, SG_BC_ZERO = 1 };
/* Precision of the component-grid states and the WENO arithmetic.  The combination sum
 * (the finest-grid accumulator) and every reduction are FP64 in both. */
enum { SG_F64 = 0, SG_F32 = 1 };
/* SG_PLAIN: one kernel launch per component grid per RK stage.
 * SG_BATCHED: one persistent launch per RK stage over a (grid, tile) work queue covering
 * every grid of the handle (or of every member of a batch). */
enum { SG_PLAIN = 0, SG_BATCHED = 1 };
/* Spatial scheme: WENO5-JS nonlinear weights (Eq. 5) or the fifth-order linear scheme that
 * replaces them by d_r = (0.1, 0.6, 0.3) (Section 3). */
enum { SG_WENO5 = 0, SG_LINEAR5 = 1 };
/* Prolongation: WENO5 interpolation (Eq. 11) or fifth-order Lagrange (Eq. 8). */
enum { SG_PROLONG_WENO5 = 0, SG_PROLONG_LAGRANGE5 = 1 };
/* Time step, common to every grid and set by the finest grid (Section 3):
 * SG_DT_POW53: dt = dt_coef * h^{5/3}, h = min_k (hi_k - lo_k)/(N_r 2^{N_L});
 * SG_DT_CFL:   dt = cfl / sum_k (alpha_k / h_k), alpha_k = max over all grids of
 *              max |f_k'(u)| at the start of the step.
 * Either way the last step is shortened so that the run ends exactly at t_end. */
enum { SG_DT_POW53 = 0, SG_DT_CFL = 1 };
/* Stage kernel (an implementation choice; every choice computes the same values, bit for bit
 * in FP64):
 * SG_STAGE_AUTO:  tile_points = 0 lets the autotuner pick the kernel and the tile at the
 *                 first sg_step (see sg_stage_config); tile_points > 0 selects SG_STAGE_TILED
 *                 with that tile;
 * SG_STAGE_TILED: the tiled kernel of the dimension (d <= 3 padded box, d >= 4 line buffer),
 *                 tiles of tile_points points (0 = 512);
 * SG_STAGE_SWEEP: d = 3 only -- one thread per grid line of an 8 x 8 x 8 tile, sweeping it
 *                 with a register window; tile_points is ignored.
 * SG_STAGE_SWEEP2: d = 3 and SG_F32 only -- the same sweep with two lines of one axis per
 *                 thread, both in one packed two-lane FP32 instruction stream. */
enum { SG_STAGE_AUTO = 0, SG_STAGE_TILED = 1, SG_STAGE_SWEEP = 2, SG_STAGE_SWEEP2 = 3 };
/* Initial condition kinds for sg_init. SG_IC_SINE: u_0(x) = p0 + p1 sin(p2 (x_0+...+x_{d-1}) + p3).
 * SG_IC_LANDAU (SG_PDE_VLASOV only, 2 parameters a, k): f_0 = (1 + a cos(k x)) exp(-v^2/2)/sqrt(2 pi).
 * SG_IC_RELAX (SG_PDE_VLASOV_BOLTZMANN with dim 2 or 4, no parameters): the initial condition
 * of Example 5, f_0 = (1/s) sin(x_1^2/2)^2 [cos(x_2^2/2)^2] exp(-(|x|^2 + |v|^2)/2), s the
 * integral of the rest over the domain (so that f_0 has unit mass). */
enum { SG_IC_SINE = 0, SG_IC_LANDAU = 1, SG_IC_RELAX = 2 };
/* Reductions (FP64).  MASS = sum u prod h, ENERGY = sum u^2 prod h, MIN/MAX of the values;
 * L1_EXACT = mean |u - u_exact|, LINF_EXACT = max |u - u_exact| against the exact solution of
 * the SG_IC_SINE initial condition at the current time (advection: translation; Burgers:
 * characteristic solution by Newton's method, valid before the shock time; both need periodic
 * boundaries on every axis, SG_ERR_STATE otherwise). */
/* FIELD_ENERGY (SG_PDE_VLASOV only): (1/2) sum_i E_i^2 h_x of the field of grid `which` or of
 * the combined solution, E as described for SG_PDE_VLASOV. */
/* ENTROPY_H2 / ENTROPY_LOG (SG_PDE_VLASOV_BOLTZMANN only): the entropy functionals of
 * Example 5 over the nodes, sum f^2 / M dV and sum_{f > 0} f log(f / M) dV, with the stationary
 * state M = exp(-(|x|^2/2 + |v|^2/2) / theta) / ((2 pi theta)^{d/2} Z), Z = the integral of
 * exp(-|x|^2 / (2 theta)) over the space domain. */
enum {
    SG_REDUCE_MASS = 0, SG_REDUCE_ENERGY = 1, SG_REDUCE_MIN = 2, SG_REDUCE_MAX = 3,
    SG_REDUCE_L1_EXACT = 4, SG_REDUCE_LINF_EXACT = 5, SG_REDUCE_FIELD_ENERGY = 6,
    SG_REDUCE_ENTROPY_H2 = 7, SG_REDUCE_ENTROPY_LOG = 8
};

#define SG_MAX_DIM 6
#define SG_WHICH_COMBINED (-1)
#define SG_WHICH_ALL_GRIDS (-2)

typedef struct sg_ctx *sg_handle;

/* Parameters.  Fill with sg_params_init, then override fields. */
typedef struct {
    size_t struct_size;          /* sizeof(sg_params), set by sg_params_init */
    double lo[SG_MAX_DIM];       /* domain [lo_k, hi_k] per axis; default [0, 4] */
    double hi[SG_MAX_DIM];
    int bc[SG_MAX_DIM];          /* SG_BC_PERIODIC (default) or SG_BC_ZERO, per axis */
    double adv_speed[SG_MAX_DIM];/* a_k for linear advection; default 1 */
    int precision;               /* SG_F64 (default) or SG_F32 */
    int exec;                    /* SG_PLAIN (default) or SG_BATCHED */
    int scheme;                  /* SG_WENO5 (default) or SG_LINEAR5 */
    int prolong;                 /* SG_PROLONG_WENO5 (default) or SG_PROLONG_LAGRANGE5 */
    double eps;                  /* epsilon of Eqs. (5) and (9); default 1e-3 */
    int dt_rule;                 /* SG_DT_POW53 (default) or SG_DT_CFL */
    double dt_coef;              /* default 1.0 */
    double cfl;                  /* default 0.4 */
    void *cuda_stream;           /* cudaStream_t to run on; NULL = a stream the handle owns */
    int graph_steps;             /* time steps per captured CUDA graph; 0 = default (16), <0 = no graph */
    int tile_points;             /* points per work-queue tile: 0 (default), 256, 512 or 1024 */
    double combine_budget_gb;    /* device memory (GB) the one-pass prolongation + combination may
                                    use for intermediates; above it (or if < 0) uhat is accumulated
                                    grid by grid instead.  0 = default (8 GB) */
    int stage_kernel;            /* SG_STAGE_AUTO (default), SG_STAGE_TILED or SG_STAGE_SWEEP */
    double theta;                /* SG_PDE_VLASOV_BOLTZMANN: temperature of mu_inf; default 1 */
    double tau;                  /* SG_PDE_VLASOV_BOLTZMANN: relaxation time (> 0); default 1 */
} sg_params;

/* Fills *p with the defaults listed above.  SG_ERR_ARG if p is NULL. */
sg_status sg_params_init(sg_params *p);

/* Creates a sparse-grid problem (Section 2.2): dim in [1, 6], root_cells = N_r >= 5 (the
 * stencil needs five distinct points on every periodic line), level = N_L with
 * 0 <= N_L <= 16 and N_r 2^{N_L} <= 2^20, pde one of SG_PDE_*.  Allocates every component
 * grid's three RK arrays on the device.  *out receives the handle.  Errors: SG_ERR_ARG for
 * out-of-range arguments (a bc other than SG_BC_PERIODIC / SG_BC_ZERO among them),
 * SG_ERR_UNSUPPORTED for a component grid of 2^31 or more points, SG_ERR_NOMEM, SG_ERR_CUDA. */
sg_status sg_create(int dim, int root_cells, int level, int pde, const sg_params *params,
                    sg_handle *out);

/* Step 1 of the algorithm: restricts an analytic initial condition to every component grid
 * on the device (point values at the nodes) and sets t = 0.  ic_kind = SG_IC_SINE with
 * n_params = 4 (p0, p1, p2, p3).  SG_ERR_ARG on a wrong kind or count. */
sg_status sg_init(sg_handle h, int ic_kind, const double *ic_params, int n_params);

/* Sets component grid `grid` from a host array of its n_0 n_1 ... values in the handle's
 * precision (double for SG_F64, float for SG_F32), bytes = count * element size, and sets
 * t = 0.  SG_ERR_ARG if grid is out of range or bytes does not match. */
sg_status sg_init_grid(sg_handle h, int grid, const void *host_values, size_t bytes);

/* Sets every component grid at once from one host array holding the grids concatenated in
 * enumeration order (sum_g n^g_0 ... n^g_{d-1} values in the handle's precision), and sets
 * t = 0.  One host-to-device copy; SG_ERR_ARG if bytes does not match. */
sg_status sg_init_grids(sg_handle h, const void *host_values, size_t bytes);

/* Step 2: advances every component grid with the common time step until t = t_end (last
 * step shortened) or until max_steps further steps have been taken.  *t_reached (may be
 * NULL) receives the time reached (for a batch: the smallest over members).  Errors:
 * SG_ERR_STATE before init, SG_ERR_NONFINITE if a stage produced NaN/Inf or a time step came
 * out non-positive or non-finite (stepping stops at the next check, at most one captured graph
 * of steps later; the state then holds the last stage's output), SG_ERR_ARG if t_end is not
 * finite or max_steps < 0. */
sg_status sg_step(sg_handle h, double t_end, long max_steps, double *t_reached);

/* Step 3: prolongs every component grid onto the finest grid (axis 0 first) and forms
 * uhat = sum_g c_g P U_g in FP64 on the device.  For a batch, does so for every member.
 * SG_ERR_STATE before init. */
sg_status sg_prolong_combine(sg_handle h);

/* Copies to the host: which = SG_WHICH_COMBINED (-1) the FP64 combined solution on the
 * finest grid ((N_r 2^{N_L})^d doubles), which = g >= 0 component grid g in the handle's
 * precision, or which = SG_WHICH_ALL_GRIDS (-2) every grid concatenated in enumeration order.  dst_bytes must be at least the size.  Synchronises the handle's stream.
 * SG_ERR_STATE for -1 before sg_prolong_combine, SG_ERR_ARG for a small buffer. */
sg_status sg_read(sg_handle h, int which, void *host_dst, size_t dst_bytes);

/* Sampled read: dst[j] = value at flat index idx[j] (axis 0 fastest) of the combined solution
 * (which = SG_WHICH_COMBINED; doubles), grid `which` >= 0, or SG_WHICH_ALL_GRIDS (values in the
 * handle's precision), j < n.  idx and dst are host arrays owned by the caller; dst_bytes
 * must hold n values.  Gathers on the device, so a large combined solution (256^4 doubles is
 * 34 GB) can be checked at sample points without copying it.  SG_ERR_ARG for an index out of
 * range (nothing is read), SG_ERR_STATE as for sg_read.  Synchronises the handle's stream. */
sg_status sg_read_points(sg_handle h, int which, const long long *idx, size_t n, void *dst, size_t dst_bytes);

/* FP64 reduction of the combined solution (which = -1) or of grid g, kind one of
 * SG_REDUCE_*.  L1_EXACT / LINF_EXACT need which = -1 and an SG_IC_SINE initial condition
 * (SG_ERR_STATE otherwise). */
sg_status sg_reduce(sg_handle h, int which, int kind, double *out);

/* Number of component grids G. */
sg_status sg_num_grids(sg_handle h, int *n);

/* levels[dim], shape[dim] (node counts) and combination coefficient of grid g; any output
 * pointer may be NULL. */
sg_status sg_grid_info(sg_handle h, int g, int *levels, long *shape, double *coeff);

/* Time and number of steps taken since the last init. */
sg_status sg_time(sg_handle h, double *t, long *steps);

/* Groups n independent problems (each from sg_create) into one batch: sg_step on the batch
 * advances every member, each with its own time step, with one persistent launch per RK
 * stage over all members' grids; members that reach t_end drop out.  Members must share
 * dim, pde, precision, scheme, eps, adv_speed and bc.  The batch does not own its members: destroy the
 * batch first, then the members.  sg_read / sg_reduce / sg_init apply to members only. */
sg_status sg_batch_create(const sg_handle *members, int n, sg_handle *batch);

/* Releases the handle and its device memory.  NULL is accepted. */
sg_status sg_destroy(sg_handle h);

/* Message for the calling thread's last failed call ("" if none). */
const char *sg_last_error(void);

/* Optional device allocator hook (e.g. a framework's caching allocator).  alloc returns a
 * device pointer of at least `bytes` bytes aligned to 256, or NULL; release frees it.
 * Pass NULLs to restore cudaMalloc/cudaFree.  Must not be changed while handles exist. */
typedef void *(*sg_alloc_fn)(size_t bytes, void *ctx);
typedef void (*sg_free_fn)(void *ptr, size_t bytes, void *ctx);
sg_status sg_set_allocator(sg_alloc_fn alloc, sg_free_fn release, void *ctx);

/* Build and kernel information, for diagnostics and the benchmark: *n_launches receives the
 * number of kernels this handle launched since creation. */
sg_status sg_launch_count(sg_handle h, long *n_launches);

/* Profiling.  With profiling on, every RK-stage launch of sg_step is bracketed by CUDA
 * events recorded on the handle's stream (captured into the step graph), and their elapsed
 * times are accumulated after each graph replay.  sg_profile(kind = SG_PROF_STAGE) returns
 * the accumulated milliseconds and the number of stage kernel launches since profiling was
 * switched on (a plain handle counts one launch per grid per stage; the events then bracket
 * the group).  Switching profiling on or off re-captures the graph at the next sg_step. */
enum { SG_PROF_STAGE = 0 };
sg_status sg_set_profiling(sg_handle h, int on);
sg_status sg_profile(sg_handle h, int kind, double *ms, long *launches);

/* The stage-kernel configuration the handle (or batch) steps with: *kernel receives
 * SG_STAGE_TILED, SG_STAGE_SWEEP or SG_STAGE_SWEEP2, *tile_points the largest tile in points, *tune_ms the
 * measured time of one RK-stage launch of the chosen configuration when the autotuner picked
 * it (0 otherwise).  Under SG_STAGE_AUTO with tile_points = 0 the autotuner runs at the first
 * sg_step: it times one stage-0 launch with dt = 0 (which leaves the solution untouched) of
 * each candidate -- the tiled kernel with 256-, 512- and 1024-point tiles and, for d = 3, the
 * sweep kernels -- keeps the fastest and remembers it, for the life of the process, per
 * dimension, precision, PDE, scheme, execution mode and size class (total points rounded up
 * to a power of two).  Before that first step the query reports the starting configuration.
 * A batch puts all of its members on one configuration (the first member's at creation, the
 * tuned one after its first sg_step); any output pointer may be NULL. */
sg_status sg_stage_config(sg_handle h, int *kernel, int *tile_points, double *tune_ms);

/* One RK3 step of one grid without any device allocation.  The paper has no counterpart:
 * this is a library convenience.  It serves callers that cannot call cudaMalloc -- code
 * running inside a framework that owns all of the device memory, or a loop with real-time
 * constraints where an allocation (and the synchronisation that cudaMalloc/cudaFree can
 * bring) is not allowed.  The caller passes the grid in and gets the stepped grid back; all
 * scratch (the two intermediate RK stages, the grid descriptor, the work queue, the
 * Lax-Friedrichs alpha slots and the flags) lives in one static device array of the library,
 * sized for SG_NOALLOC_MAX_POINTS points (about 16.5 MB), which every GPU that loads the
 * library holds until the process exits.
 *
 * It advances one periodic FP64 grid by one TVD-RK3 step of the WENO5 / Lax-Friedrichs
 * scheme with the same stage kernel and tiles as sg_step, so the result equals that of a
 * level-0 handle stepped with the same dt, bit for bit.
 *   dim: 1..3 (SG_ERR_UNSUPPORTED otherwise); shape[k] >= 5 and prod shape[k] <=
 *   SG_NOALLOC_MAX_POINTS (SG_ERR_ARG otherwise, with a message in sg_last_error);
 *   lo, hi: the domain (node spacing (hi_k - lo_k)/shape[k]); pde, scheme, eps as in
 *   sg_create / sg_params; adv_speed: a_k for advection (NULL = all 1);
 *   u_in, u_out: device pointers to prod shape[k] doubles, axis 0 fastest: the same pointer
 *   (stepped in place) or two arrays that do not overlap (SG_ERR_ARG if they overlap otherwise);
 *   dt: the step; cuda_stream: the cudaStream_t to run on (NULL = default).
 * The call is asynchronous on that stream and calls no cudaMalloc, cudaFree or allocating
 * library routine.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture.  Every call uses the same scratch array and leaves its last contents there: calls
 * whose work overlaps on the GPU (other streams, other host threads) race and corrupt each
 * other's result.  Non-finite values are not reported (sg_step reports them). */
#define SG_NOALLOC_MAX_POINTS 1048576
sg_status sg_step_grid_noalloc(int dim, const long *shape, const double *lo, const double *hi, int pde,
                               const double *adv_speed, int scheme, double eps, const double *u_in,
                               double *u_out, double dt, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SGWENO_H */
