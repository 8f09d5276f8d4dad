// sg_aux.cuh -- the kernels around the stage kernels: the initial alpha reduction, the
// device-side time-step control, Step 1 (restriction of the initial condition), Step 3
// (prolongation of each grid and the FP64 signed combination sum) and FP64 reductions.
#pragma once
#include "sg_stage.cuh"

// max |u| of the stage-0 input over every tile of the queue -> alpha slot 0 (the slots of
// stages 1 and 2 are cleared by the caller); also flags non-finite values.
template <class T>
__global__ void __launch_bounds__(SG_NT) sg_alpha_init_kernel(const GridDesc* grids, int ngrids,
                                                               unsigned long long* alpha, int* flags) {
    __shared__ double red[SG_NT / 32];
    for (int g = blockIdx.y; g < ngrids; g += gridDim.y) {
        const GridDesc* G = grids + g;
        const T* u = (const T*)G->u0;
        double mx = 0.0;
        bool bad = false;
        for (long long p = blockIdx.x * (long long)SG_NT + threadIdx.x; p < G->npts;
             p += (long long)gridDim.x * SG_NT) {
            const T v = u[p];
            if (!sg_isfinite(v)) bad = true;
            mx = fmax(mx, (double)sg_abs(v));
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags + SG_FLAG_NONFINITE, 1);
        const double m = block_max(mx, red);
        if (threadIdx.x == 0) atomicMax(alpha + g * 3, alpha_enc((T)m));  // m is a T value
    }
}

// max over a warp (every lane gets it); exact, and like fmax it ignores a NaN operand
__device__ __forceinline__ double warp_fmax(double a) {
    for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    return a;
}

// Per-instance time-step control, one warp per instance (the lanes split the maxima over the
// instance's grids; the max is exact in any order).  commit_only = 0 at the start of a step:
// adds the previous (pending) step to t, then sets dt for the next step or marks the instance
// inactive.  commit_only = 1 after the last step: only adds the pending step.
static __global__ void sg_dt_kernel(InstState* inst, int ninst, const GridDesc* grids,
                             const unsigned long long* alpha, PhysParams ph, int commit_only, int* flags) {
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= ninst) return;  // the whole warp
    InstState s = inst[i];
    if (s.pending) {
        s.t = s.last ? s.t_end : s.t + s.dt;
        s.steps += 1;
        s.pending = 0;
    }
    s.active = 0;
    if (!commit_only && s.t < s.t_end && s.steps < s.step_limit) {
        double dt;
        if (s.dt_rule == 0) {
            dt = s.dt_nom;
        } else {
            double sum = 0.0;
            for (int k = 0; k < ph.dim; ++k) {
                double a = 0.0;
                if (ph.pde == 1 || (ph.pde == 2 && k == 1)) {  // Burgers max|u|; Vlasov-Poisson max|E|
                    for (int g = s.grid0 + lane; g < s.grid0 + s.ngrids; g += 32)
                        a = fmax(a, ph.alpha_f32 ? (double)alpha_dec<float>(alpha[g * 3]) : bitsd(alpha[g * 3]));
                    a = warp_fmax(a);
                } else if (ph.pde == 2) {  // Vlasov-Poisson along x: max |v_j|, at an end node
                    for (int g = s.grid0 + lane; g < s.grid0 + s.ngrids; g += 32) {
                        const GridDesc& G = grids[g];
                        if (ph.alpha_f32) {
                            const float v0 = (float)G.lo[1], v1 = (float)G.lo[1] + (float)(G.n[1] - 1) * (float)G.h[1];
                            a = fmax(a, (double)fmaxf(fabsf(v0), fabsf(v1)));
                        } else {
                            const double v0 = G.lo[1], v1 = G.lo[1] + (double)(G.n[1] - 1) * G.h[1];
                            a = fmax(a, fmax(fabs(v0), fabs(v1)));
                        }
                    }
                    a = warp_fmax(a);
                } else if (ph.pde == 3) {  // Vlasov-Boltzmann: static, from the instance's grids
                    a = s.alpha_vb[k];
                } else {
                    a = ph.adv[k] < 0.0 ? -ph.adv[k] : ph.adv[k];
                }
                sum = sum + a / s.hf[k];
            }
            dt = s.cfl / sum;
        }
        s.last = 0;
        if (!(dt > 0.0) || !isfinite(dt)) {  // e.g. alpha overflowed: stop instead of stalling
            if (lane == 0) {
                atomicOr(flags + SG_FLAG_BADDT, 1);
                inst[i] = s;  // inactive, nothing pending
            }
            return;
        }
        if (dt >= s.t_end - s.t) {  // shortened last step: the run ends exactly at t_end
            dt = s.t_end - s.t;
            s.last = 1;
        }
        s.dt = dt;
        s.dtf = (float)dt;
        s.pending = 1;
        s.active = 1;
    }
    if (lane == 0) inst[i] = s;
}

// ------------------------------------------------------------------------------------
// Step 1: restriction of u0 = p0 + p1 sin(p2 sum_k x_k + p3), x_k = lo_k + j_k h_k.
// One launch for all grids of a problem: blockIdx.y = grid, the blocks along x stride over its
// points.  The node indices j_k come from 32-bit division when the grid has fewer than 2^31
// points (64-bit otherwise); the sum, sine and split are the same operations in the same order
// either way.
// ------------------------------------------------------------------------------------
template <class T>
__global__ void sg_restrict_sine_kernel(const GridDesc* __restrict__ grids, int dim, double p0, double p1, double p2,
                                        double p3) {
    const GridDesc& G = grids[blockIdx.y];
    const long long npts = G.npts;
    const bool narrow = npts < (1LL << 31);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts;
         p += (long long)gridDim.x * blockDim.x) {
        double S = 0.0;
        if (narrow) {
            unsigned r = (unsigned)p;
            for (int k = 0; k < dim; ++k) {
                const unsigned n = (unsigned)G.n[k], q = r / n;
                S = S + (G.lo[k] + (double)(r - q * n) * G.h[k]);
                r = q;
            }
        } else {
            long long r = p;
            for (int k = 0; k < dim; ++k) {
                const long long j = r % G.n[k];
                r /= G.n[k];
                S = S + (G.lo[k] + (double)j * G.h[k]);
            }
        }
        const double v = p0 + p1 * sin(p2 * S + p3);
        ((T*)G.u0)[p] = (T)v;
        if (sizeof(T) == 4) ((T*)G.u3)[p] = (T)(v - (double)(T)v);  // float pair: v = U + C
    }
}

// Landau initial condition of the Vlasov-Poisson workload (d = 2, axis 0 = x, axis 1 = v):
// f_0 = (1 + a cos(k x)) exp(-v^2/2) / sqrt(2 pi).
template <class T>
__global__ void sg_restrict_landau_kernel(GridDesc G, double a, double kx) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < G.npts;
         p += (long long)gridDim.x * blockDim.x) {
        const long long j = p / G.n[0], i = p - j * G.n[0];
        const double x = G.lo[0] + (double)i * G.h[0], v = G.lo[1] + (double)j * G.h[1];
        const double m = exp(-0.5 * (v * v)) / sqrt(2.0 * 3.14159265358979323846);
        const double f = (1.0 + a * cos(kx * x)) * m;
        ((T*)G.u0)[p] = (T)f;
        if (sizeof(T) == 4) ((T*)G.u3)[p] = (T)(f - (double)(T)f);
    }
}

// Example 5 initial condition of the Vlasov-Boltzmann model (dim = 2 d, d = 1 or 2):
// f_0 = (1/s) prod_k factor_k(x_k), factor_0 = sin(x^2/2)^2 exp(-x^2/2), factor_1 =
// cos(x^2/2)^2 exp(-x^2/2) on the space axes, exp(-v^2/2) on the velocity axes.
template <class T>
__global__ void sg_restrict_relax_kernel(GridDesc G, int dim, double s_norm) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < G.npts;
         p += (long long)gridDim.x * blockDim.x) {
        long long r = p;
        double f = 1.0;
        for (int k = 0; k < dim; ++k) {
            const long long j = r % G.n[k];
            r /= G.n[k];
            const double x = G.lo[k] + (double)j * G.h[k];
            const double e = exp(-0.5 * (x * x));
            double fac = e;
            if (k < dim / 2) {
                const double t = k == 0 ? sin(0.5 * (x * x)) : cos(0.5 * (x * x));
                fac = (t * t) * e;
            }
            f = f * fac;
        }
        const double v = f / s_norm;
        ((T*)G.u0)[p] = (T)v;
        if (sizeof(T) == 4) ((T*)G.u3)[p] = (T)(v - (double)(T)v);
    }
}

// Vlasov-Boltzmann density of every grid from the input of RK stage `stage`, into G->ef:
// rho[ix] = (h_{v_1} ... h_{v_d}) sum_jv f[ix + n_x jv] (ix the flattened space index, jv the
// flattened velocity index), summed in FP64.  Block (32, SG_DENS_ROWS).
//   FP64: one thread per space node, jv ascending (the order of the definition); the loads of
//   16 consecutive jv are issued before their adds, which keep their order.
//   FP32: threadIdx.x over 32 consecutive space nodes, threadIdx.y over the residues of jv
//   modulo SG_DENS_ROWS; the partial sums are added in y order and the density is rounded to
//   float once.
// ------------------------------------------------------------------------------------
#define SG_DENS_ROWS 16
template <class T>
__global__ void __launch_bounds__(32 * SG_DENS_ROWS) sg_density_kernel(const GridDesc* grids, int ngrids,
                                                                       const InstState* inst, int stage, int dim) {
    __shared__ double part[SG_DENS_ROWS][33];
    const int dx = dim / 2;
    for (int g = blockIdx.y; g < ngrids; g += gridDim.y) {
        const GridDesc* G = grids + g;
        const InstState* S = inst + G->inst;
        if (!S->active) continue;  // uniform over the block
        StageIO<T> io;
        io.setup(G, stage, stage_parity<T>(S));
        long long nx = 1, nv = 1;
        double hv = 1.0;
        for (int k = 0; k < dx; ++k) nx *= G->n[k];
        for (int k = dx; k < dim; ++k) {
            nv *= G->n[k];
            hv = hv * G->h[k];
        }
        T* rho = (T*)G->ef;
        if constexpr (sizeof(T) == 8) {
            const int per = 32 * SG_DENS_ROWS;
            for (long long ix = blockIdx.x * (long long)per + threadIdx.x + 32 * threadIdx.y; ix < nx;
                 ix += (long long)gridDim.x * per) {
                double sum = 0.0;
                long long jv = 0;
                for (; jv + 16 <= nv; jv += 16) {
                    T v[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = io.load(ix + nx * (jv + q));
#pragma unroll
                    for (int q = 0; q < 16; ++q) sum = sum + (double)v[q];
                }
                for (; jv < nv; ++jv) sum = sum + (double)io.load(ix + nx * jv);
                rho[ix] = (T)(hv * sum);
            }
        } else {
            for (long long ix0 = blockIdx.x * 32LL; ix0 < nx; ix0 += (long long)gridDim.x * 32) {  // uniform
                const long long ix = ix0 + threadIdx.x;
                double sum = 0.0;
                if (ix < nx) {
                    long long jv = threadIdx.y;
                    for (; jv + 3 * SG_DENS_ROWS < nv; jv += 4 * SG_DENS_ROWS) {
                        T v[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) v[q] = io.load(ix + nx * (jv + q * SG_DENS_ROWS));
#pragma unroll
                        for (int q = 0; q < 4; ++q) sum += (double)v[q];
                    }
                    for (; jv < nv; jv += SG_DENS_ROWS) sum += (double)io.load(ix + nx * jv);
                }
                part[threadIdx.y][threadIdx.x] = sum;
                __syncthreads();
                if (threadIdx.y == 0 && ix < nx) {
                    double t = 0.0;
#pragma unroll
                    for (int y = 0; y < SG_DENS_ROWS; ++y) t += part[y][threadIdx.x];
                    rho[ix] = (T)(hv * t);
                }
                __syncthreads();
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Vlasov-Poisson field of every grid from the input of RK stage `stage` (one block per
// grid): rho_i = h_v sum_j f_ij (j ascending, one thread per i), then by one thread, in the
// same order of operations as the definition: mean(rho), E_0 = 0, E_i = E_{i-1} +
// h_x ((rho_{i-1} + rho_i)/2 - mean), and the mean of E removed.  E goes to G->ef and
// max |E| to the grid's alpha slot of the stage (the LF alpha along v).  pre_dt: launched
// before the step's time-step control, which has not yet counted the previous step (FP32
// ping-pong parity).
// ------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) sg_efield_kernel(const GridDesc* grids, int ngrids, const InstState* inst,
                                                        unsigned long long* alpha, int stage, int pre_dt) {
    for (int g = blockIdx.x; g < ngrids; g += gridDim.x) {
        const GridDesc* G = grids + g;
        const InstState* S = inst + G->inst;
        const long long steps = S->steps + (pre_dt ? S->pending : 0);
        StageIO<T> io;
        io.setup(G, stage, (int)((steps - S->step0) & 1));
        const int n0 = G->n[0], n1 = G->n[1];
        T* E = (T*)G->ef;
        const T hv = (T)G->h[1], hx = (T)G->h[0];
        for (int i = threadIdx.x; i < n0; i += blockDim.x) {
            T sum = T(0);
            for (int j = 0; j < n1; ++j) sum = sum + io.load(i + (long long)n0 * j);
            E[i] = hv * sum;  // rho_i for now
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            T mean = T(0);
            for (int i = 0; i < n0; ++i) mean = mean + E[i];
            mean = mean / (T)n0;
            T prev = E[0], e = T(0), meanE = T(0);
            E[0] = T(0);
            for (int i = 1; i < n0; ++i) {
                const T rho = E[i];
                e = e + hx * ((T)0.5 * (prev + rho) - mean);
                prev = rho;
                E[i] = e;
            }
            for (int i = 0; i < n0; ++i) meanE = meanE + E[i];
            meanE = meanE / (T)n0;
            T mx = T(0);
            for (int i = 0; i < n0; ++i) {
                const T v = E[i] - meanE;
                E[i] = v;
                mx = sg_max(mx, sg_abs(v));
            }
            alpha[g * 3 + stage] = alpha_enc(mx);
        }
        __syncthreads();
    }
}

// Field energy (1/2) sum_i E_i^2 h_x of one 2-D array (a grid, or the combined solution), E
// as in sg_efield_kernel but in FP64 (FP32 grids: the float pair U + C).  One block; rho
// goes through `scratch` (n0 doubles).
template <class T>
__global__ void __launch_bounds__(256) sg_field_energy_kernel(const T* u, const T* comp, int n0, int n1, double hx,
                                                              double hv, double* scratch, double* out) {
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        double sum = 0.0;
        for (int j = 0; j < n1; ++j) {
            const long long p = i + (long long)n0 * j;
            double v = (double)u[p];
            if (comp) v = v + (double)comp[p];
            sum = sum + v;
        }
        scratch[i] = hv * sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mean = 0.0;
        for (int i = 0; i < n0; ++i) mean = mean + scratch[i];
        mean = mean / (double)n0;
        double prev = scratch[0], e = 0.0, meanE = 0.0;
        scratch[0] = 0.0;
        for (int i = 1; i < n0; ++i) {
            const double rho = scratch[i];
            e = e + hx * (0.5 * (prev + rho) - mean);
            prev = rho;
            scratch[i] = e;
        }
        for (int i = 0; i < n0; ++i) meanE = meanE + scratch[i];
        meanE = meanE / (double)n0;
        double s = 0.0;
        for (int i = 0; i < n0; ++i) {
            const double v = scratch[i] - meanE;
            s = s + v * v;
        }
        *out = 0.5 * s * hx;
    }
}

// ------------------------------------------------------------------------------------
// Prolongation of one axis (Section 2.2.1): in has shape (below, m_in, above) in the
// axis-0-fastest sense, out has (below, Nf, above).  Fine node jf on an axis refined by
// r = 2^{N_L - l}: centre i = floor(jf/r + 1/2), s = jf/r - i in [-1/2, 1/2).
// If acc != nullptr the result is added, times coeff, into the FP64 accumulator instead
// (the last prolonged axis, fused with the combination sum of Eq. 13).
// ------------------------------------------------------------------------------------
// 2^-e exactly (0 <= e <= 126), built from its bits: no division
template <class T>
__device__ __forceinline__ T pow2_neg(int e);
template <>
__device__ __forceinline__ float pow2_neg<float>(int e) { return __int_as_float((127 - e) << 23); }
template <>
__device__ __forceinline__ double pow2_neg<double>(int e) { return __longlong_as_double((long long)(1023 - e) << 52); }

// r is a power of two: shifts and masks instead of integer division, and s = m / r formed as
// m 2^-lr, the same value as the quotient (both exact)
template <class T>
__device__ __forceinline__ void fine_to_coarse(int jf, int r, int& ic, T& s) {
    const int lr = __ffs(r) - 1;
    const int i = jf >> lr, m = jf & (r - 1);
    const T inv = pow2_neg<T>(lr);
    if (2 * m < r) {
        ic = i;
        s = (T)m * inv;
    } else {
        ic = i + 1;
        s = (T)(m - r) * inv;
    }
}

// c in [-n, 2n) -> c mod n (a stencil index at most two cells outside [0, n))
__device__ __forceinline__ int wrap_index(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

template <class T>
__global__ void sg_prolong_axis_kernel(const T* __restrict__ in, T* __restrict__ out,
                                       double* __restrict__ acc, double coeff, long long below,
                                       int min_, int nf, long long above, int r, double eps,
                                       int lagrange, int zero_bc) {
    const long long tot = below * nf * above;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long lo = idx % below;
        const long long rest = idx / below;
        const int jf = (int)(rest % nf);
        const long long hi = rest / nf;
        int ic;
        T s;
        fine_to_coarse<T>(jf, r, ic, s);
        const T* line = in + lo + hi * below * min_;
        T v[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const int cr = ic - 2 + m;  // zero_bc: 0 beyond the ends, else periodic
            v[m] = zero_bc && (cr < 0 || cr >= min_) ? T(0) : line[(long long)wrap_index(cr, min_) * below];
        }
        T res;
        if constexpr (sizeof(T) == 8) {
            res = Weno<double>::interp(v[0], v[1], v[2], v[3], v[4], s, eps, lagrange);
        } else {
            res = Weno<float>::interp(v[0], v[1], v[2], v[3], v[4], s, sg_eps4<float>(eps), lagrange);
        }
        if (acc) acc[idx] = acc[idx] + coeff * (double)res;
        else out[idx] = res;
    }
}

// ------------------------------------------------------------------------------------
// Step 3, last axis fused with the combination: uhat = sum_g c_g P_{d-1} I_g, where I_g is
// grid g prolonged over axes 0..d-2 (shape (below, n_g) with below = N_f^{d-1}).  Each thread
// owns one fine position `lo` in axes 0..d-2 and a chunk of J consecutive fine indices of the
// last axis; it loops over the grids in enumeration order with a 5-value window sliding along
// the grid's coarse last axis, and writes uhat once.
//   T = double: acc = acc + c_g v in FP64, grids in enumeration order -- the same operations
//     as accumulating each grid's prolongation into uhat in turn.
//   T = float:  the sum is kept as an unevaluated float pair (error-free sums and products),
//     whose accuracy exceeds FP64's for these sums; GB300's FP64 rate is a small fraction of
//     its FP32 rate.
// ------------------------------------------------------------------------------------
template <class T>
struct CombineAcc;

template <>
struct CombineAcc<double> {
    double a = 0.0;
    template <bool EXACT = false>
    __device__ __forceinline__ void add(double c, double v) { a = a + c * v; }
    __device__ __forceinline__ double value() const { return a; }
};

template <>
struct CombineAcc<float> {
    float hi = 0.f, lo = 0.f;
    // EXACT: every coefficient is a power of two (d <= 3), so c v is exact and has no error term
    template <bool EXACT = false>
    __device__ __forceinline__ void add(float cf, float v) {  // cf: |c| <= C(5, 2), exact in float
        const float p = cf * v;
        const float pe = EXACT ? 0.f : fmaf(cf, v, -p);    // exact product error
        const float s = hi + p;              // two-sum of hi and p
        const float bb = s - hi;
        const float e = (hi - (s - bb)) + (p - bb);
        hi = s;                              // hi: the float sum; lo: the sum of its exact errors
        lo += e + pe;                        // (lo's own rounding is O(u^2) of the result)
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Interpolation window of one coarse line: the five values around the current coarse centre.
//   double: Eqs. (8)-(11) evaluated literally per output (Weno<double>::interp).
//   float:  the quantities that depend only on the five values (differences, the products of
//     the smoothness terms) are formed once per centre; each output then needs the linear
//     weights C_k(s), the three parabolas and one division.
template <class T>
struct InterpWin;

template <>
struct InterpWin<double> {
    double w0, w1, w2, w3, w4;
    __device__ __forceinline__ void prepare(double, int) {}
    __device__ __forceinline__ double eval(double s, double eps, int lagrange) const {
        return Weno<double>::interp(w0, w1, w2, w3, w4, s, eps, lagrange);
    }
};

template <>
struct InterpWin<float> {
    // Per centre, the interpolant of Eqs. (8)-(11) is w2 + (s/2) N(s) / D(s) with N cubic and D
    // quadratic in s: N = sum_k C_k(s) beta_w_k (s_k + s t_k), D = sum_k C_k(s) beta_w_k, where
    // beta_w_k = prod_{j != k} (eps + beta_j)^2 (up to a common factor) and C_k(s) the linear
    // weights.  prepare() forms their coefficients once; eval() is two Horner evaluations.
    float w0, w1, w2, w3, w4;
    float n0, n1, n2, n3, d0, d1, d2;
    __device__ __forceinline__ void prepare(float eps4, int lagrange) {
        const float d1_ = w1 - w0, d2_ = w2 - w1, d3_ = w3 - w2, d4_ = w4 - w3;
        const float t0 = d2_ - d1_, t1 = d3_ - d2_, t2 = d4_ - d3_;
        const float s0 = fmaf(3.f, d2_, -d1_), s1 = d2_ + d3_, s2 = fmaf(3.f, d3_, -d4_);
        float E0 = 1.f, E1 = 1.f, E2 = 1.f;  // beta_w_k; 1 for Lagrange
        if (!lagrange) {  // rescaled as in Weno<float>::side: every E in [1, 2^80], D >= 1/16
            float e0 = fmaf((13.f / 3.f) * t0, t0, fmaf(s0, s0, eps4));
            float e1 = fmaf((13.f / 3.f) * t1, t1, fmaf(s1, s1, eps4));
            float e2 = fmaf((13.f / 3.f) * t2, t2, fmaf(s2, s2, eps4));
            weno_scale3(e0, e1, e2);
            const float q0 = e0 * e0, q1 = e1 * e1, q2 = e2 * e2;
            E0 = q1 * q2;
            E1 = q0 * q2;
            E2 = q0 * q1;
        }
        // C_0 = 1/6 - s/4 + s^2/12, C_1 = 2/3 - s^2/6, C_2 = 1/6 + s/4 + s^2/12
        const float A0 = E0 * s0, A1 = E1 * s1, A2 = E2 * s2;
        const float B0 = E0 * t0, B1 = E1 * t1, B2 = E2 * t2;
        const float Ap = A0 + A2, Bp = B0 + B2, Ep = E0 + E2;
        n0 = fmaf(Ap, 1.f / 6.f, (2.f / 3.f) * A1);
        n1 = fmaf(Bp, 1.f / 6.f, fmaf(A2 - A0, 0.25f, (2.f / 3.f) * B1));
        n2 = fmaf(B2 - B0, 0.25f, fmaf(Ap, 1.f / 12.f, (-1.f / 6.f) * A1));
        n3 = fmaf(Bp, 1.f / 12.f, (-1.f / 6.f) * B1);
        d0 = fmaf(Ep, 1.f / 6.f, (2.f / 3.f) * E1);
        d1 = (E2 - E0) * 0.25f;
        d2 = fmaf(Ep, 1.f / 12.f, (-1.f / 6.f) * E1);
    }
    __device__ __forceinline__ float eval(float s, float, int) const {
        if (s == 0.f) return w2;
        const float N = fmaf(fmaf(fmaf(n3, s, n2), s, n1), s, n0);
        const float D = fmaf(fmaf(d2, s, d1), s, d0);
        return fmaf(0.5f * s, __fdividef(N, D), w2);
    }
};


template <class T, int J, bool EXACT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) sg_combine_last_axis_kernel(const CombineGrid* __restrict__ tab, int G,
                                                                    double* __restrict__ uhat, long long below,
                                                                    int nf, double eps, int lagrange, int zero_last) {
    const T e12 = sg_eps4<T>(eps);
    const int nchunks = (nf + J - 1) / J;
    // centre index and offset s of the chunk's J fine nodes for every refinement ratio
    // r = 2^lr (lr <= 16): the same for all grids with that ratio and all columns of the block
    __shared__ T s_tab[17 * J];
    __shared__ int c_tab[17 * J];
    for (int ch = blockIdx.y; ch < nchunks; ch += gridDim.y) {
        const int j0 = ch * J;
        __syncthreads();  // the previous chunk's readers are done
        for (int t = threadIdx.x; t < 17 * J; t += blockDim.x) {
            const int lr = t / J, jf = j0 + (t - lr * J), r = 1 << lr;
            const int i = jf >> lr, m = jf & (r - 1);  // jf = i r + m; centre i or i + 1
            const T inv_r = pow2_neg<T>(lr);
            if (2 * m < r) {
                c_tab[t] = i;
                s_tab[t] = (T)m * inv_r;
            } else {
                c_tab[t] = i + 1;
                s_tab[t] = (T)(m - r) * inv_r;
            }
        }
        __syncthreads();
        for (long long lo = blockIdx.x * (long long)blockDim.x + threadIdx.x; lo < below;
             lo += (long long)gridDim.x * blockDim.x) {
            CombineAcc<T> acc[J];
            for (int g = 0; g < G; ++g) {
                const CombineGrid cg = tab[g];
                const T* col = (const T*)cg.src + lo;
                const int n = cg.n, r = cg.r;
                const T cT = (T)cg.coeff;  // converted once per grid
                if (r == 1) {  // last axis already fine: values at coincident nodes
#pragma unroll
                    for (int j = 0; j < J; ++j) {
                        const int jf = j0 + j;
                        if (jf < nf) acc[j].template add<EXACT>(cT, col[(long long)jf * below]);
                    }
                    continue;
                }
                // r = 2^lr: centres and offsets of the chunk's nodes from the block's table
                const int lr = __ffs(r) - 1;
                const T* st = s_tab + lr * J;
                const int* ct = c_tab + lr * J;
                int cur = ct[0];
                // coarse value at index c of the last axis: periodic, or 0 beyond the ends
                auto at = [&](int c) -> T {
                    if (zero_last && (c < 0 || c >= n)) return T(0);
                    return col[(long long)wrap_index(c, n) * below];
                };
                InterpWin<T> W;
                W.w0 = at(cur - 2);
                W.w1 = at(cur - 1);
                W.w2 = at(cur);
                W.w3 = at(cur + 1);
                W.w4 = at(cur + 2);
                W.prepare(e12, lagrange);
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int jf = j0 + j;
                    if (jf >= nf) break;
                    const int ic = ct[j];
                    const T s = st[j];
                    if (ic != cur) {  // centres advance by one coarse node at a time (r >= 2)
                        W.w0 = W.w1;
                        W.w1 = W.w2;
                        W.w2 = W.w3;
                        W.w3 = W.w4;
                        W.w4 = at(ic + 2);
                        W.prepare(e12, lagrange);
                        cur = ic;
                    }
                    acc[j].template add<EXACT>(cT, W.eval(s, eps, lagrange));
                }
            }
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int jf = j0 + j;
                if (jf < nf) uhat[lo + (long long)jf * below] = acc[j].value();
            }
        }
    }
}

// One prolongation pass over many grids (Step 3, axes 0..d-2, Section 2.2.1): thread u of
// the pass takes unit u -- J consecutive fine nodes of one line -- of the task whose unit range
// holds it, and slides the five coarse values around the current centre along the line: their
// s-independent part is formed once per centre (InterpWin::prepare), so the r fine nodes that
// share a centre pay only for eval().  Consecutive units are consecutive columns (below > 1:
// the loads of a warp are coalesced) or consecutive chunks of one row (below = 1).
template <class T, int J>
__global__ void __launch_bounds__(256) sg_prolong_multi_kernel(const ProlongTask* __restrict__ tasks, int ntasks,
                                                               long long nunits, double eps, int lagrange) {
    const T e4 = sg_eps4<T>(eps);
    for (long long u = blockIdx.x * 256LL + threadIdx.x; u < nunits; u += gridDim.x * 256LL) {
        int a = 0, b = ntasks - 1;  // the last task with unit0 <= u
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if (tasks[mid].unit0 <= u) a = mid;
            else b = mid - 1;
        }
        const ProlongTask& tk = tasks[a];
        const unsigned v = (unsigned)(u - tk.unit0);
        const unsigned below = (unsigned)tk.below;
        const int nchunks = (tk.nf + J - 1) / J;
        const unsigned q = div_mag(v, below, tk.below_mag);
        const unsigned lo = v - q * below;
        const unsigned hi = div_mag(q, (unsigned)nchunks, tk.nch_mag);
        const int j0 = (int)(q - hi * (unsigned)nchunks) * J;
        const int n = tk.n, nf = tk.nf, r = tk.r, lr = __ffs(r) - 1;
        const T inv_r = pow2_neg<T>(lr);
        const T* col = (const T*)tk.in + (long long)hi * below * n + lo;
        T* ocol = (T*)tk.out + (long long)hi * below * nf + lo;
        auto centre = [&](int jf, int& ic, T& s) {  // as fine_to_coarse
            const int i = jf >> lr, m = jf & (r - 1);
            if (2 * m < r) {
                ic = i;
                s = (T)m * inv_r;
            } else {
                ic = i + 1;
                s = (T)(m - r) * inv_r;
            }
        };
        auto at = [&](int c) -> T {  // c in [-2, n + 2]
            if (tk.zero_bc && (c < 0 || c >= n)) return T(0);
            return col[(long long)wrap_index(c, n) * below];
        };
        int cur;
        T s0;
        centre(j0, cur, s0);
        InterpWin<T> W;
        W.w0 = at(cur - 2);
        W.w1 = at(cur - 1);
        W.w2 = at(cur);
        W.w3 = at(cur + 1);
        W.w4 = at(cur + 2);
        W.prepare(e4, lagrange);
#pragma unroll 1
        for (int j = 0; j < J; ++j) {
            const int jf = j0 + j;
            if (jf >= nf) break;
            int ic;
            T s;
            centre(jf, ic, s);
            if (ic != cur) {  // centres advance by one coarse node at a time (r >= 2)
                W.w0 = W.w1;
                W.w1 = W.w2;
                W.w2 = W.w3;
                W.w3 = W.w4;
                W.w4 = at(ic + 2);
                W.prepare(e4, lagrange);
                cur = ic;
            }
            ocol[(long long)jf * below] = W.eval(s, (T)eps, lagrange);
        }
    }
}

// uhat += coeff * u for a grid that is already the finest grid.
template <class T>
__global__ void sg_accumulate_kernel(const T* __restrict__ u, double* __restrict__ acc, double coeff,
                                     long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        acc[i] = acc[i] + coeff * (double)u[i];
}

// out[j] = u[idx[j]] (indices checked by the host).
template <class T>
__global__ void sg_gather_kernel(const T* __restrict__ u, const long long* __restrict__ idx, T* __restrict__ out,
                                 long long n) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x)
        out[j] = u[idx[j]];
}

// ------------------------------------------------------------------------------------
// FP64 reductions, deterministic two-pass (fixed grid, fixed order).
// kind: 0 sum u, 1 sum u^2, 2 min, 3 max, 4 sum |u - exact|, 5 max |u - exact|,
// 7 sum u^2 / M, 8 sum over u > 0 of u log(u / M) (M the Vlasov-Boltzmann stationary state)
// ------------------------------------------------------------------------------------

// Stationary state of the Vlasov-Boltzmann model at node p of an array shaped X.n:
// M = exp(-(sum_k x_k^2 / 2) / theta) / ((2 pi theta)^{d/2} Z).
__device__ __forceinline__ double sg_relax_state(const ExactSpec& X, long long p) {
    double q = 0.0;
    long long r = p;
    for (int k = 0; k < X.dim; ++k) {
        const long long j = r % X.n[k];
        r /= X.n[k];
        const double x = X.lo[k] + (double)j * X.h[k];
        q = q + 0.5 * (x * x);
    }
    return exp(-(q / X.theta)) / X.mnorm;
}


__device__ __forceinline__ double sg_exact(const ExactSpec& X, long long p) {
    double S = 0.0, St = 0.0;
    long long r = p;
    for (int k = 0; k < X.dim; ++k) {
        const long long j = r % X.nf;
        r /= X.nf;
        const double x = X.lo[k] + (double)j * X.h[k];
        S = S + x;
        St = St + (x - X.adv[k] * X.t);
    }
    if (X.pde == 0) return X.b + X.a * sin(X.w * St + X.phi);
    const double d = (double)X.dim;
    double u = X.b + X.a * sin(X.w * S + X.phi);
    for (int it = 0; it < 100; ++it) {
        const double arg = X.w * (S - d * u * X.t) + X.phi;
        const double F = u - X.b - X.a * sin(arg);
        const double dF = 1.0 + X.a * X.w * d * X.t * cos(arg);
        const double du = F / dF;
        u = u - du;
        if (fabs(du) <= 1e-16 * (1.0 + fabs(u))) break;
    }
    return u;
}

template <class T>
__global__ void __launch_bounds__(256) sg_reduce_pass1(const T* __restrict__ u, const T* __restrict__ comp,
                                                       long long n, int kind, ExactSpec X, double* partial) {
    __shared__ double sh[256];
    double v;
    const bool is_min = kind == 2, is_max = kind == 3 || kind == 5;
    v = is_min ? INFINITY : (is_max ? -INFINITY : 0.0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double x = comp ? (double)u[i] + (double)comp[i] : (double)u[i];
        double y;
        switch (kind) {
            case 0: y = x; break;
            case 1: y = x * x; break;
            case 4:
            case 5: y = fabs(x - sg_exact(X, i)); break;
            case 7: y = (x * x) / sg_relax_state(X, i); break;
            case 8: y = x > 0.0 ? x * log(x / sg_relax_state(X, i)) : 0.0; break;
            default: y = x; break;
        }
        if (is_min) v = fmin(v, y);
        else if (is_max) v = fmax(v, y);
        else v = v + y;
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double o = sh[threadIdx.x + s];
            double& m = sh[threadIdx.x];
            m = is_min ? fmin(m, o) : (is_max ? fmax(m, o) : m + o);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

static __global__ void __launch_bounds__(256) sg_reduce_pass2(const double* partial, int np, int kind, double* out) {
    __shared__ double sh[256];
    const bool is_min = kind == 2, is_max = kind == 3 || kind == 5;
    double v = is_min ? INFINITY : (is_max ? -INFINITY : 0.0);
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const double y = partial[i];
        v = is_min ? fmin(v, y) : (is_max ? fmax(v, y) : v + y);
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double o = sh[threadIdx.x + s];
            double& m = sh[threadIdx.x];
            m = is_min ? fmin(m, o) : (is_max ? fmax(m, o) : m + o);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}
