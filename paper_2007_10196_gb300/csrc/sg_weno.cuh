// sg_weno.cuh -- device arithmetic of the method: the Lax-Friedrichs split (Eq. 7), the
// one-sided WENO5 reconstruction (Eqs. 3-6) and the WENO5 / Lagrange interpolation
// (Eqs. 8-11), plus small device helpers.
//
// Weno<double> evaluates the paper's formulas literally; the translation unit that
// instantiates it is compiled with --fmad=false so each expression is a fixed sequence of
// IEEE-754 operations.  Weno<float> evaluates the same mathematics in first differences with
// rescaled smoothness terms and one division per side (see the comment above it).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sg_device.h"

#define SG_NT 256  // threads per block of the stage kernels

// Exact unsigned division by a run-time divisor d <= 2^16 for x < 2^16 (multiply-high by
// ceil(2^32 / d)).  x (d - 1) < 2^32 guarantees floor(x m / 2^32) = floor(x / d).
// ceil(2^32 / d) = floor((2^32 - 1) / d) + 1 for d >= 2.
// Multipliers of FDiv for divisors up to 1024, so that setting one up needs no division (an
// integer division by a run-time value is a long instruction sequence with a reciprocal).
struct SgMagic {
    unsigned v[1025];
};
constexpr SgMagic sg_make_magic() {
    SgMagic t{};
    for (unsigned d = 0; d <= 1024; ++d) t.v[d] = d <= 1 ? 0u : 0xFFFFFFFFu / d + 1u;
    return t;
}
static __constant__ SgMagic sg_magic = sg_make_magic();

struct FDiv {
    unsigned m, d;
    __device__ __forceinline__ void init(unsigned dd) {
        d = dd;
        m = dd <= 1024u ? sg_magic.v[dd] : 0xFFFFFFFFu / dd + 1u;
    }
    __device__ __forceinline__ unsigned div(unsigned x) const { return d <= 1u ? x : __umulhi(x, m); }
};

// x / d for any 32-bit x with the 64-bit multiplier mag = floor((2^64 - 1) / d) + 1 made on the
// host (exact: x (mag d - 2^64) < 2^64 for x, d < 2^32).
__device__ __forceinline__ unsigned div_mag(unsigned x, unsigned d, unsigned long long mag) {
    return d <= 1u ? x : (unsigned)__umul64hi((unsigned long long)x, mag);
}

// Work item tile -> tile coordinates along the first D axes of grid G (tile index row-major,
// axis 0 fastest).
template <int D>
__device__ __forceinline__ void tile_coords(const GridDesc* G, unsigned tile, int (&tc)[D]) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const unsigned nt = (unsigned)G->nt[k];
        const unsigned q = div_mag(tile, nt, G->ntmag[k]);
        tc[k] = (int)(tile - q * nt);
        tile = q;
    }
}

__device__ __forceinline__ unsigned long long dbits(double v) {
    return (unsigned long long)__double_as_longlong(v);
}
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

// Alpha slots: a non-negative max |u| stored as bits that unsigned atomicMax orders like the
// values -- the double's bits for FP64 state, the float's bits zero-extended for FP32 state
// (so the FP32 kernels never touch the FP64 pipe to read or write them).
__device__ __forceinline__ unsigned long long alpha_enc(double v) { return dbits(v); }
__device__ __forceinline__ unsigned long long alpha_enc(float v) { return (unsigned long long)__float_as_uint(v); }
template <class T>
__device__ __forceinline__ T alpha_dec(unsigned long long b);
template <>
__device__ __forceinline__ double alpha_dec<double>(unsigned long long b) { return bitsd(b); }
template <>
__device__ __forceinline__ float alpha_dec<float>(unsigned long long b) { return __uint_as_float((unsigned)b); }

// dt and 1/h in the state precision (FP32: host- or dt-kernel-rounded copies)
template <class T>
__device__ __forceinline__ T inst_dt(const InstState* S);
template <>
__device__ __forceinline__ double inst_dt<double>(const InstState* S) { return S->dt; }
template <>
__device__ __forceinline__ float inst_dt<float>(const InstState* S) { return S->dtf; }
template <class T>
__device__ __forceinline__ T grid_rdx(const GridDesc* G, int k);
template <>
__device__ __forceinline__ double grid_rdx<double>(const GridDesc* G, int k) { return G->rdx[k]; }
template <>
__device__ __forceinline__ float grid_rdx<float>(const GridDesc* G, int k) { return G->rdxf[k]; }

template <class T>
__device__ __forceinline__ T sg_abs(T v) { return v < T(0) ? -v : v; }

__device__ __forceinline__ bool sg_isfinite(double v) { return isfinite(v); }
__device__ __forceinline__ bool sg_isfinite(float v) { return isfinite(v); }

__device__ __forceinline__ double sg_fmax_(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float sg_fmax_(float a, float b) { return fmaxf(a, b); }

// Block-wide max of non-negative values; the result is valid in thread 0.  Contains two
// barriers, so every thread of the block must call it.
__device__ __forceinline__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;
}

// Block-wide max where any thread's `neg` forces the result to -1 (used to fold the
// non-finite flag into the alpha reduction); result valid in thread 0; two barriers.
template <class T>
__device__ __forceinline__ T block_max(T v, T* red, bool neg) {
    const unsigned anyneg = __ballot_sync(0xffffffffu, neg);
    for (int o = 16; o > 0; o >>= 1) v = sg_fmax_(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = anyneg ? T(-1) : v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : T(0);
        const unsigned n2 = __ballot_sync(0xffffffffu, v < T(0));
        for (int o = 16; o > 0; o >>= 1) v = sg_fmax_(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (n2) v = T(-1);
    }
    __syncthreads();
    return v;
}

// Float version: the FP32 kernels keep every per-point operation in FP32 (GB300's FP64 pipe
// runs at a small fraction of the FP32 rate); the block result is widened once.
__device__ __forceinline__ float block_max(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;
}

// 1/x to about one ulp (the hardware approximation; x normal)
__device__ __forceinline__ float sg_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Packed two-lane FP32 arithmetic (one instruction for both lanes; sm_100 and later), used by
// the kernels that carry two independent columns or lines per thread.
__device__ __forceinline__ float2 sg_f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sg_neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sg_add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sg_sub2(float2 a, float2 b) { return __fadd2_rn(a, sg_neg2(b)); }
__device__ __forceinline__ float2 sg_mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sg_fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <class T>
struct Weno;

// ------------------------------------------------------------------------------------
// FP64: Eqs. (3)-(7) and (8)-(11) evaluated literally; compile without contraction.
// ------------------------------------------------------------------------------------
template <>
struct Weno<double> {
    // fhat_{i+1/2} from (a..e) = (f_{i-2}, ..., f_{i+2}) (positive wind), Eqs. (3)-(6).
    static __device__ __forceinline__ double side(double a, double b, double c, double d, double e,
                                                  double eps, int linear) {
        const double q0 = (1.0 / 3.0) * a - (7.0 / 6.0) * b + (11.0 / 6.0) * c;
        const double q1 = -(1.0 / 6.0) * b + (5.0 / 6.0) * c + (1.0 / 3.0) * d;
        const double q2 = (1.0 / 3.0) * c + (5.0 / 6.0) * d - (1.0 / 6.0) * e;
        double w0 = 0.1, w1 = 0.6, w2 = 0.3;
        if (!linear) {
            const double r0 = a - 2.0 * b + c, g0 = a - 4.0 * b + 3.0 * c;
            const double r1 = b - 2.0 * c + d, g1 = b - d;
            const double r2 = c - 2.0 * d + e, g2 = 3.0 * c - 4.0 * d + e;
            const double b0 = (13.0 / 12.0) * (r0 * r0) + 0.25 * (g0 * g0);
            const double b1 = (13.0 / 12.0) * (r1 * r1) + 0.25 * (g1 * g1);
            const double b2 = (13.0 / 12.0) * (r2 * r2) + 0.25 * (g2 * g2);
            w0 = 0.1 / ((eps + b0) * (eps + b0));
            w1 = 0.6 / ((eps + b1) * (eps + b1));
            w2 = 0.3 / ((eps + b2) * (eps + b2));
        }
        return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2);
    }

    // Lax-Friedrichs split of one value, Eq. (7): f^{+-} = (f +- alpha u)/2.
    static __device__ __forceinline__ void split(double u, double alpha, double ak, int pde, double& fp,
                                                 double& fm) {
        const double f = pde == 1 ? (0.5 * u) * u : ak * u;
        fp = 0.5 * (f + alpha * u);
        fm = 0.5 * (f - alpha * u);
    }

    // fhat = fhat^+ + fhat^- at x_{L+1/2} from split values at L-2 .. L+3 (stride S):
    // fhat^+ on (L-2..L+2), fhat^- on the mirror image (L+3..L-1).
    static __device__ __forceinline__ double interface_split(const double* p, const double* m, int S,
                                                             const PhysParams& ph) {
        const double fplus = side(p[0], p[S], p[2 * S], p[3 * S], p[4 * S], ph.eps, ph.scheme);
        const double fminus = side(m[5 * S], m[4 * S], m[3 * S], m[2 * S], m[S], ph.eps, ph.scheme);
        return fplus + fminus;
    }

    // Same from raw values u_{L-2} .. u_{L+3} (stride S).
    static __device__ __forceinline__ double interface(const double* v, int S, double alpha, double ak,
                                                       const PhysParams& ph) {
        double fp[6], fm[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) split(v[j * S], alpha, ak, ph.pde, fp[j], fm[j]);
        const double fplus = side(fp[0], fp[1], fp[2], fp[3], fp[4], ph.eps, ph.scheme);
        const double fminus = side(fm[5], fm[4], fm[3], fm[2], fm[1], ph.eps, ph.scheme);
        return fplus + fminus;
    }

    // WENO5 / Lagrange interpolation at x_i + s h, Eqs. (8)-(11), literal order.
    static __device__ __forceinline__ double interp(double a, double b, double c, double d, double e,
                                                    double s, double eps, int lagrange) {
        if (s == 0.0) return c;
        const double g0 = 0.5 * (a - 4.0 * b + 3.0 * c), k0 = 0.5 * (a - 2.0 * b + c);
        const double g1 = 0.5 * (d - b), k1 = 0.5 * (b - 2.0 * c + d);
        const double g2 = 0.5 * (-3.0 * c + 4.0 * d - e), k2 = 0.5 * (c - 2.0 * d + e);
        const double P0 = c + s * (g0 + s * k0);
        const double P1 = c + s * (g1 + s * k1);
        const double P2 = c + s * (g2 + s * k2);
        const double C0 = ((s - 1.0) * (s - 2.0)) / 12.0;
        const double C1 = (4.0 - s * s) / 6.0;
        const double C2 = ((s + 1.0) * (s + 2.0)) / 12.0;
        if (lagrange) return C0 * P0 + C1 * P1 + C2 * P2;
        const double r0 = a - 2.0 * b + c, g0s = a - 4.0 * b + 3.0 * c;
        const double r1 = b - 2.0 * c + d, g1s = b - d;
        const double r2 = c - 2.0 * d + e, g2s = 3.0 * c - 4.0 * d + e;
        const double b0 = (13.0 / 12.0) * (r0 * r0) + 0.25 * (g0s * g0s);
        const double b1 = (13.0 / 12.0) * (r1 * r1) + 0.25 * (g1s * g1s);
        const double b2 = (13.0 / 12.0) * (r2 * r2) + 0.25 * (g2s * g2s);
        const double w0 = C0 / ((eps + b0) * (eps + b0));
        const double w1 = C1 / ((eps + b1) * (eps + b1));
        const double w2 = C2 / ((eps + b2) * (eps + b2));
        return (w0 * P0 + w1 * P1 + w2 * P2) / (w0 + w1 + w2);
    }
};

// ------------------------------------------------------------------------------------
// FP32: the same mathematics in first differences d_j = f_j - f_{j-1}:
//   q_r - f_i = (5/6 d2 - 1/3 d1, 1/6 d2 + 1/3 d3, 2/3 d3 - 1/6 d4)
//   e_r = 4 (eps + beta_r) = (13/3) t_r^2 + s_r^2 + 4 eps, t = second differences,
//   s = (3 d2 - d1, d2 + d3, 3 d3 - d4)
//   alpha_r / alpha_1 = (d_r / d_1) prod_{j != r} E_j / prod_{j != 1} E_j, E_r = e_r^2
// so a side needs no division of its own beyond num / den.
//
// Range.  The weights of Eq. (5) depend on the e_r only through their ratios, so the three
// are rescaled before they are squared and multiplied (weno_scale3): divided by the power of
// two at or below the smallest, exactly, which puts the smallest in [1, 2), and capped at
// 2^20.  A weight whose e was capped lies below 2^-38 of the largest weight before and after
// the cap, so the cap changes the result by less than 2^-38 of the candidate fluxes' spread.
// Every product of two E then lies in [1, 2^80]: the arithmetic neither overflows nor
// underflows for any eps > 0 (4 eps is raised to 2^-100 if smaller: sg_eps4) and split-flux
// differences below about 10^13; the quotient num / den is taken per side.
// ------------------------------------------------------------------------------------
// 4 eps, the eps term of e_r (FP32 kernels; the FP64 ones use eps itself)
template <class T>
__device__ __forceinline__ T sg_eps4(double eps);
template <>
__device__ __forceinline__ double sg_eps4<double>(double eps) { return 4.0 * eps; }
template <>
__device__ __forceinline__ float sg_eps4<float>(double eps) { return fmaxf((float)(4.0 * eps), 0x1p-100f); }

// e_k <- min(e_k 2^-floor(log2 min_j e_j), 2^20); the scale is built from the exponent bits of
// the smallest e (normal: e >= 4 eps >= 2^-100), so the division is exact.
__device__ __forceinline__ float sg_min3(float a, float b, float c) {  // three-input min (sm_100+)
    float m;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(m) : "f"(a), "f"(b), "f"(c));
    return m;
}
__device__ __forceinline__ void weno_scale3(float& e0, float& e1, float& e2) {
    const float m = sg_min3(e0, e1, e2);
    const float sc = __uint_as_float(0x7f000000u - (__float_as_uint(m) & 0x7f800000u));
    e0 = fminf(e0 * sc, 0x1p20f);
    e1 = fminf(e1 * sc, 0x1p20f);
    e2 = fminf(e2 * sc, 0x1p20f);
}

template <>
struct Weno<float> {
    static __device__ __forceinline__ void side(float a, float b, float c, float d, float e,
                                                float eps4, int linear, float& num, float& den) {
        // weights proportional to E_1 E_2 / 6, E_0 E_2, E_0 E_1 / 2 with E_k = e_k^2 (rescaled;
        // linear scheme: E_k = 1), num and den formed factored (as SweepSide<float>::value);
        // den >= 5/3, so num / den is in the accurate range of __fdividef
        const float d1 = b - a, d2 = c - b, d3 = d - c, d4 = e - d;
        const float p0s = fmaf(5.f / 36.f, d2, (-1.f / 18.f) * d1);  // p_0 / 6
        const float p1 = fmaf(1.f / 6.f, d2, (1.f / 3.f) * d3);
        const float p2h = fmaf(1.f / 3.f, d3, (-1.f / 12.f) * d4);   // p_2 / 2
        float E0 = 1.f, E1 = 1.f, E2 = 1.f;
        if (!linear) {
            const float t0 = d2 - d1, t1 = d3 - d2, t2 = d4 - d3;
            const float s0 = fmaf(3.f, d2, -d1), s1 = d2 + d3, s2 = fmaf(3.f, d3, -d4);
            float e0 = fmaf((13.f / 3.f) * t0, t0, fmaf(s0, s0, eps4));
            float e1 = fmaf((13.f / 3.f) * t1, t1, fmaf(s1, s1, eps4));
            float e2 = fmaf((13.f / 3.f) * t2, t2, fmaf(s2, s2, eps4));
            weno_scale3(e0, e1, e2);
            E0 = e0 * e0;
            E1 = e1 * e1;
            E2 = e2 * e2;
        }
        const float X = E0 * E2;
        num = fmaf(E1, fmaf(E2, p0s, E0 * p2h), X * p1);
        den = fmaf(E1, fmaf(E2, 1.f / 6.f, 0.5f * E0), X);
    }

    // Burgers split, Eq. (7): f^{+-} = u (u/4 +- alpha/2).
    static __device__ __forceinline__ void split_burgers(float u, float half_alpha, float& fp, float& fm) {
        fp = u * fmaf(0.25f, u, half_alpha);
        fm = u * fmaf(0.25f, u, -half_alpha);
    }

    // fhat = fhat^+ + fhat^- from the centres and the (num, den) of the two sides; each den lies
    // in [5/3, 2^81], inside the range where __fdividef is accurate
    static __device__ __forceinline__ float combine(float cp, float cm, float np, float dp, float nm, float dm) {
        return (cp + cm) + (__fdividef(np, dp) + __fdividef(nm, dm));
    }

    static __device__ __forceinline__ float interface_split(const float* p, const float* m, int S, float eps4,
                                                            int linear) {
        float np, dp, nm, dm;
        side(p[0], p[S], p[2 * S], p[3 * S], p[4 * S], eps4, linear, np, dp);
        side(m[5 * S], m[4 * S], m[3 * S], m[2 * S], m[S], eps4, linear, nm, dm);
        return combine(p[2 * S], m[3 * S], np, dp, nm, dm);
    }

    // raw values u_{L-2} .. u_{L+3} (stride S)
    static __device__ __forceinline__ float interface(const float* v, int S, float alpha, float ak,
                                                      const PhysParams& ph, float eps4) {
        float fp[6], fm[6];
        if (ph.pde == 1) {
            const float ha = 0.5f * alpha;
#pragma unroll
            for (int j = 0; j < 6; ++j) split_burgers(v[j * S], ha, fp[j], fm[j]);
        } else {
            const float cp = 0.5f * (ak + alpha), cm = 0.5f * (ak - alpha);
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                fp[j] = cp * v[j * S];
                fm[j] = cm * v[j * S];
            }
        }
        float np, dp, nm, dm;
        side(fp[0], fp[1], fp[2], fp[3], fp[4], eps4, ph.scheme, np, dp);
        side(fm[5], fm[4], fm[3], fm[2], fm[1], eps4, ph.scheme, nm, dm);
        return combine(fp[2], fm[3], np, dp, nm, dm);
    }

    static __device__ __forceinline__ float interp(float a, float b, float c, float d, float e,
                                                   float s, float eps4, int lagrange) {
        if (s == 0.f) return c;
        const float d1 = b - a, d2 = c - b, d3 = d - c, d4 = e - d;
        const float t0 = d2 - d1, t1 = d3 - d2, t2 = d4 - d3;
        const float s0 = fmaf(3.f, d2, -d1), s1 = d2 + d3, s2 = fmaf(3.f, d3, -d4);
        // P_k(s) - c = (s/2) (s_k + s t_k)
        const float p0 = fmaf(s, t0, s0), p1 = fmaf(s, t1, s1), p2 = fmaf(s, t2, s2);
        // linear weights C_k(s) of Eq. (9): (s-1)(s-2)/12, (4-s^2)/6, (s+1)(s+2)/12
        const float ss = s * s;
        const float q = fmaf(ss, 1.f / 12.f, 1.f / 6.f);
        const float C0 = fmaf(s, -0.25f, q), C2 = fmaf(s, 0.25f, q);
        const float C1 = fmaf(ss, -1.f / 6.f, 2.f / 3.f);
        float w0 = C0, w1 = C1, w2 = C2;
        if (!lagrange) {  // weights of Eq. (9), rescaled as in side(): sum >= 1/16
            float e0 = fmaf((13.f / 3.f) * t0, t0, fmaf(s0, s0, eps4));
            float e1 = fmaf((13.f / 3.f) * t1, t1, fmaf(s1, s1, eps4));
            float e2 = fmaf((13.f / 3.f) * t2, t2, fmaf(s2, s2, eps4));
            weno_scale3(e0, e1, e2);
            const float E0 = e0 * e0, E1 = e1 * e1, E2 = e2 * e2;
            w0 = C0 * (E1 * E2);
            w1 = C1 * (E0 * E2);
            w2 = C2 * (E0 * E1);
        }
        const float num = fmaf(w0, p0, fmaf(w1, p1, w2 * p2));
        return fmaf(0.5f * s, __fdividef(num, w0 + w1 + w2), c);
    }
};
