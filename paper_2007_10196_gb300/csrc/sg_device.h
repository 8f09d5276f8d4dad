// sg_device.h -- plain-data structures shared by the host API (sg_api.cu) and the kernels.
//
// Layout in HBM (one problem = one "instance"; a batch concatenates instances):
//   * every component grid owns three state arrays u0/u1/u2 of n_0*...*n_{d-1} elements
//     (axis 0 fastest), each 256-byte aligned inside the instance's arena;
//   * the work queue is an array of (grid, tile) items, grid-major, tiles in row-major
//     order of the tile grid;
//   * alpha slots: three per grid (the max |f'(u)| of the input of RK stage 0, 1, 2), kept
//     as the bit pattern of a non-negative number in the state precision (FP64: the double's
//     bits; FP32: the float's bits, zero-extended) so that atomicMax on the integer orders
//     them like the values;
//   * one InstState per instance carries its time, step size and step counters on the
//     device, so that graph-captured steps need no host round trip.
#pragma once
#include <cstdint>

#define SG_MAXD 6

struct GridDesc {
    // FP64: u0 = u^n (u^{n+1} written in place by the last stage), u1 = u^{(1)}, u2 = u^{(2)}.
    // FP32: (u0, u1) = ping-pong pair holding U (the float head of u^n) and the first stage
    // increment, u2 = second-stage increment, u3 = C (the float tail: u^n = U + C).
    // Between calls u0 always holds U.
    void* u0;
    void* u1;
    void* u2;
    void* u3;
    void* ef;            // Vlasov-Poisson: E_i of the current stage input, n[0] values;
                         // Vlasov-Boltzmann: rho(x) of the stage input, n_0 ... n_{d-1} values
    const void* mu;      // Vlasov-Boltzmann: mu_inf at the velocity nodes (flattened), else null
    long long npts;
    int n[SG_MAXD];      // nodes per axis
    int te[SG_MAXD];     // tile extent per axis
    int nt[SG_MAXD];     // tiles per axis
    unsigned long long ntmag[SG_MAXD];  // floor((2^64 - 1) / nt) + 1: division-free tile decomposition
    double h[SG_MAXD];   // node spacing (hi-lo)/n
    double rdx[SG_MAXD]; // 1/h
    float rdxf[SG_MAXD]; // (float)(1/h), for the FP32 kernels (no per-tile FP64 conversion)
    double lo[SG_MAXD];
    double coeff;        // combination coefficient (-1)^q C(d-1,q)
    int lev[SG_MAXD];
    int inst;            // instance (batch member) index
    int first_item;      // index of this grid's first work item
    int n_items;
    int pad_;
};

// Host side: the 64-bit multiplier of GridDesc.ntmag.
inline unsigned long long sg_div_magic64(unsigned d) { return d <= 1u ? 0ull : ~0ull / d + 1ull; }

struct WorkItem {
    int grid;
    int tile;
};

struct InstState {
    double t;
    double dt;
    float dtf;              // (float)dt, for the FP32 kernels
    double t_end;
    double dt_nom;          // dt of the h^{5/3} rule (host-computed)
    double cfl;
    double hf[SG_MAXD];     // finest-grid spacing per axis
    double alpha_vb[SG_MAXD];  // Vlasov-Boltzmann: max over the instance's grids of the axis's
                               // largest |partner node| (host-computed, the stage precision's arithmetic)
    long long steps;
    long long step0;        // steps at the start of the current sg_step call (FP32 ping-pong parity)
    long long step_limit;
    int active;             // 1 while a step is being taken
    int pending;            // dt set, step not yet added to t
    int grid0;              // first grid of this instance in the grid table
    int ngrids;
    int dt_rule;            // 0: h^{5/3}, 1: CFL
    int last;               // the pending step is the shortened last one (ends at t_end)
};

struct PhysParams {
    int dim;
    int pde;                 // 0 advection, 1 Burgers, 2 Vlasov-Poisson, 3 Vlasov-Boltzmann
    int scheme;              // 0 WENO5, 1 linear
    int prolong;             // 0 WENO5 interpolation, 1 Lagrange
    double eps;
    double adv[SG_MAXD];
    int alpha_f32;           // alpha slots hold float bits (FP32 state)
    double tau;              // Vlasov-Boltzmann: relaxation time of (mu rho - f) / tau
    int zmask;               // advection / Burgers: bit k set = u is 0 beyond the ends of axis k
                             // (zero boundary), else periodic; the kinetic PDEs imply theirs
};

struct StageArgs {
    const GridDesc* grids;
    const WorkItem* items;
    InstState* inst;
    unsigned long long* alpha;  // [grids][3]
    int* flags;                 // [0]: non-finite seen
    int item_begin;
    int item_end;
    int stage;                  // 0, 1, 2
    int box_elems;              // box kernel: elements of one padded box in shared memory
    PhysParams phys;
};

// Exact solution of u0 = b + a sin(w sum x + phi) on the finest grid (for error norms).
struct ExactSpec {
    int dim, pde, nf;
    double lo[SG_MAXD], h[SG_MAXD], adv[SG_MAXD];
    double b, a, w, phi, t;
    // entropy functionals of the Vlasov-Boltzmann model: node counts per axis of the reduced
    // array, temperature and the normalisation (2 pi theta)^{d/2} Z of the stationary state
    int n[SG_MAXD];
    double theta, mnorm;
};

// One grid's entry for the fused last-axis prolongation + combination kernel.
struct CombineGrid {
    const void* src;  // the grid prolonged over axes 0..d-2: shape (N_f^{d-1}, n), axis 0 fastest
    int n;            // coarse points of the last axis
    int r;            // refinement ratio 2^{N_L - l_{d-1}} of the last axis
    double coeff;     // combination coefficient
    float coeff_f;    // the same as a float (exact: |c| = C(d-1, q) <= 10)
};

// One grid's share of a prolongation pass over many grids (Step 3, axes 0..d-2): the array
// `in` of shape (below, n, above) (axis 0 fastest) is prolonged along its middle axis into
// `out` of shape (below, nf, above).  Its units -- chunks of J consecutive fine nodes of one
// line, numbered lo + below (chunk + nchunks hi) -- are the pass's global unit indices
// [unit0, unit0 + below nchunks above).
struct ProlongTask {
    const void* in;
    void* out;
    long long unit0;
    int below;        // < 2^31 (a pass's unit count is checked on the host)
    int above;
    int n;            // coarse points of the prolonged axis
    int nf;           // fine points of the prolonged axis
    int r;            // refinement ratio nf / n = 2^{N_L - l}
    int zero_bc;      // 0 beyond the ends of the axis, else periodic
    unsigned long long below_mag, nch_mag;  // sg_div_magic64 of below and of the chunks per line
};

// flags[0]: a non-finite value appeared; flags[1]: a time step came out non-positive or
// non-finite (the instance is stopped)
enum { SG_FLAG_NONFINITE = 0, SG_FLAG_BADDT = 1 };
