// sg_aux.cuh -- the kernels around the stage kernels: the initial alpha reduction, the
// device-side time-step control, Step 1 (restriction of the initial condition), Step 3
// (prolongation of each grid and the FP64 signed combination sum) and FP64 reductions.
#pragma once
#include "sg_weno.cuh"

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
        if (threadIdx.x == 0) atomicMax(alpha + g * 3, dbits(m));
    }
}

// Per-instance time-step control, one thread per instance.  commit_only = 0 at the start of
// a step: adds the previous (pending) step to t, then sets dt for the next step or marks the
// instance inactive.  commit_only = 1 after the last step: only adds the pending step.
static __global__ void sg_dt_kernel(InstState* inst, int ninst, const unsigned long long* alpha,
                             PhysParams ph, int commit_only) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ninst) return;
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
                if (ph.pde == 1) {
                    for (int g = s.grid0; g < s.grid0 + s.ngrids; ++g) a = fmax(a, bitsd(alpha[g * 3]));
                } else {
                    a = ph.adv[k] < 0.0 ? -ph.adv[k] : ph.adv[k];
                }
                sum = sum + a / s.hf[k];
            }
            dt = s.cfl / sum;
        }
        s.last = 0;
        if (dt >= s.t_end - s.t) {  // shortened last step: the run ends exactly at t_end
            dt = s.t_end - s.t;
            s.last = 1;
        }
        s.dt = dt;
        s.pending = 1;
        s.active = 1;
    }
    inst[i] = s;
}

// ------------------------------------------------------------------------------------
// Step 1: restriction of u0 = p0 + p1 sin(p2 sum_k x_k + p3), x_k = lo_k + j_k h_k.
// ------------------------------------------------------------------------------------
template <class T>
__global__ void sg_restrict_sine_kernel(GridDesc G, int dim, double p0, double p1, double p2,
                                        double p3) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < G.npts;
         p += (long long)gridDim.x * blockDim.x) {
        long long r = p;
        double S = 0.0;
        for (int k = 0; k < dim; ++k) {
            const long long j = r % G.n[k];
            r /= G.n[k];
            S = S + (G.lo[k] + (double)j * G.h[k]);
        }
        const double v = p0 + p1 * sin(p2 * S + p3);
        ((T*)G.u0)[p] = (T)v;
        if (sizeof(T) == 4) ((T*)G.u3)[p] = (T)(v - (double)(T)v);  // float pair: v = U + C
    }
}

// ------------------------------------------------------------------------------------
// Prolongation of one axis (Section 2.2.1): in has shape (below, m_in, above) in the
// axis-0-fastest sense, out has (below, Nf, above).  Fine node jf on an axis refined by
// r = 2^{N_L - l}: centre i = floor(jf/r + 1/2), s = jf/r - i in [-1/2, 1/2).
// If acc != nullptr the result is added, times coeff, into the FP64 accumulator instead
// (the last prolonged axis, fused with the combination sum of Eq. 13).
// ------------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void fine_to_coarse(int jf, int r, int& ic, T& s) {
    const int i = jf / r, m = jf - i * r;
    if (2 * m < r) {
        ic = i;
        s = (T)m / (T)r;
    } else {
        ic = i + 1;
        s = (T)(m - r) / (T)r;
    }
}

template <class T>
__global__ void sg_prolong_axis_kernel(const T* __restrict__ in, T* __restrict__ out,
                                       double* __restrict__ acc, double coeff, long long below,
                                       int min_, int nf, long long above, int r, double eps,
                                       int lagrange) {
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
            int c = ic - 2 + m;
            c %= min_;
            if (c < 0) c += min_;
            v[m] = line[(long long)c * below];
        }
        T res;
        if constexpr (sizeof(T) == 8) {
            res = Weno<double>::interp(v[0], v[1], v[2], v[3], v[4], s, eps, lagrange);
        } else {
            res = Weno<float>::interp(v[0], v[1], v[2], v[3], v[4], s, (float)(12.0 * eps), lagrange);
        }
        if (acc) acc[idx] = acc[idx] + coeff * (double)res;
        else out[idx] = res;
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

// ------------------------------------------------------------------------------------
// FP64 reductions, deterministic two-pass (fixed grid, fixed order).
// kind: 0 sum u, 1 sum u^2, 2 min, 3 max, 4 sum |u - exact|, 5 max |u - exact|
// ------------------------------------------------------------------------------------


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
