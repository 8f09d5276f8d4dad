// sg_launch.h -- host-side launchers of the kernels in sg_kernels.cuh.  Each precision is
// compiled in its own translation unit (sg_kernels_f64.cu without FMA contraction,
// sg_kernels_f32.cu with it); the API (sg_api.cu) sees only these declarations.
#pragma once
#include <cuda_runtime.h>

#include "sg_device.h"

namespace sg {

// Shared-memory footprint (elements) of the d <= 3 stage kernel for tile extents te[0..d-1]:
// two padded boxes (box) and the flux arrays of all axes (flux).
void box_footprint(int d, const int* te, long long* box, long long* flux);
// Shared memory (elements) of the line-sweep kernel (d >= 4; d = 2 variant 2) for tile extents
// te[0..d-1]: the line buffer of the widest axis, lines x ((te_k + 6) | 1) (box), and one
// accumulator per tile point (acc).
void line_footprint(int d, const int* te, long long* box, long long* acc);
// The same for the d = 3 line-sweep kernel (odd x stride; three 512-point difference arrays).
void sweep_footprint(const int* te, long long* box, long long* flux);
// Tile extents of the d = 3 line-sweep kernel: <= 8 per axis (at most 512 points, 192 lines),
// preferring a divisor of the axis length in [4, 8] so that no tile is ragged.
void sweep_tile(const int* n, int* te);

template <class T>
struct Launch {
    // Dynamic shared memory (bytes) of the stage kernel: the padded-box and one-line sweep
    // kernels (d <= 3) hold 2 box + flux elements, the two-line sweep kernel (d = 3, variant 3)
    // box + flux, the line-sweep kernel (d >= 4; variant 2) box + flux (line buffer and
    // accumulators, from line_footprint) and flux ints (per-line offsets).
    static size_t stage_smem(int dim, int ppt, long long box, long long flux, int variant = 0);
    // Raises the kernel's shared-memory limit and returns resident blocks per SM (0 if the
    // configuration cannot run).  variant: 0 = the default kernel of the dimension (d = 3:
    // line sweep), 1 = the padded-box kernel for d = 3, 2 = the line-buffer kernel for d = 2
    // (the Vlasov-Boltzmann model; d = 4 and 6 use it by default).
    static int stage_prepare(int dim, int ppt, size_t smem, int variant = 0);
    // One RK stage over work items [a.item_begin, a.item_end) with `nblocks` blocks.
    static cudaError_t stage(int dim, int ppt, const StageArgs& a, int nblocks, size_t smem, cudaStream_t s,
                             int variant = 0);
    static int stage_threads(int dim, int variant);
    // alpha slot 0 of every grid <- max |u0| (slots must be zero); flags non-finite values.
    static cudaError_t alpha_init(const GridDesc* grids, int ngrids, long long max_pts,
                                  unsigned long long* alpha, int* flags, cudaStream_t s);
    // u0 of every grid of the device table <- p0 + p1 sin(p2 sum x + p3) (FP32: also the
    // compensation term u3), one launch; max_npts = the largest grid's points.
    static cudaError_t restrict_sine(const GridDesc* grids, int ngrids, long long max_npts, int dim, const double* p,
                                     cudaStream_t s);
    // One prolongation axis; acc != nullptr fuses "acc += coeff * result"; zero_bc: values
    // beyond the ends of the axis are 0 (Vlasov-Poisson v, every Vlasov-Boltzmann axis), else
    // periodic.
    static cudaError_t prolong_axis(const T* in, T* out, double* acc, double coeff, long long below,
                                    int min_, int nf, long long above, int r, double eps,
                                    int lagrange, int zero_bc, cudaStream_t s);
    // Vlasov-Poisson: E of every grid from the input of RK stage `stage` into GridDesc.ef,
    // max|E| into the stage's alpha slot (pre_dt: launched before the step's dt control).
    static cudaError_t efield(const GridDesc* grids, int ngrids, const InstState* inst, unsigned long long* alpha,
                              int stage, int pre_dt, cudaStream_t s);
    // Field energy of one 2-D array (n0 x n1, comp may be null) into *out (device);
    // scratch holds n0 doubles.
    static cudaError_t field_energy(const T* u, const T* comp, int n0, int n1, double hx, double hv,
                                    double* scratch, double* out, cudaStream_t s);
    // Landau initial condition on one grid.
    static cudaError_t restrict_landau(const GridDesc& g, double a, double kx, cudaStream_t s);
    // Vlasov-Boltzmann: Example 5 initial condition on one grid (normalisation s_norm).
    static cudaError_t restrict_relax(const GridDesc& g, int dim, double s_norm, cudaStream_t s);
    // Vlasov-Boltzmann: rho(x) of every grid from the input of RK stage `stage` into GridDesc.ef.
    static cudaError_t density(const GridDesc* grids, int ngrids, long long max_nx, const InstState* inst,
                               int stage, int dim, cudaStream_t s);
    static cudaError_t accumulate(const T* u, double* acc, double coeff, long long n, cudaStream_t s);
    // out[j] = u[idx[j]], j < n (device arrays; indices already checked)
    static cudaError_t gather(const T* u, const long long* idx, T* out, long long n, cudaStream_t s);
    // One prolongation pass over the ntasks tasks of a device table (their unit ranges cover
    // [0, nunits)), J = 8 fine nodes per unit.
    static cudaError_t prolong_multi(const ProlongTask* tasks, int ntasks, long long nunits, double eps, int lagrange,
                                     cudaStream_t s);
    // The same for tasks whose lines pair up (below even, 8-byte aligned arrays; FP32): two
    // adjacent columns per thread in packed arithmetic.  FP64: the same as prolong_multi.
    static cudaError_t prolong_multi_pairs(const ProlongTask* tasks, int ntasks, long long nunits, double eps,
                                           int lagrange, cudaStream_t s);
    // uhat = sum_g c_g P_{d-1} I_g over the G entries of tab (device array), written once.
    // exact_coeffs: every |c_g| is a power of two (products c_g v are exact in the FP32 sum);
    // pairs_aligned: below is even and every tab[g].src is 8-byte aligned (FP32: both columns
    // of a pair with one 8-byte load)
    static cudaError_t combine_last_axis(const CombineGrid* tab, int G, double* uhat, long long below, int nf,
                                         int exact_coeffs, int zero_last, int pairs_aligned,
                                         double eps, int lagrange, cudaStream_t s);
    // FP64 reduction of n values u (+ comp if non-null); partial holds >= 1024 doubles.
    static cudaError_t reduce(const T* u, const T* comp, long long n, int kind, const ExactSpec& X,
                              double* partial, double* out, cudaStream_t s);
};

extern template struct Launch<double>;
extern template struct Launch<float>;

// flags: the device flag array (SG_FLAG_BADDT is set if a step comes out non-positive)
cudaError_t launch_dt(InstState* inst, int ninst, const GridDesc* grids, const unsigned long long* alpha,
                      const PhysParams& ph, int commit_only, int* flags, cudaStream_t s);

// Sets the calling thread's message returned by sg_last_error (defined in sg_api.cu).
void set_last_error(const char* msg);

}  // namespace sg
