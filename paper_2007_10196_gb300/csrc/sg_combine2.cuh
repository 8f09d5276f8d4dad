// sg_combine2.cuh -- Step 3's last axis and the signed combination sum (Eqs. 12-15) in FP32
// for two adjacent columns per thread, with GB300's packed two-lane FP32 arithmetic.
//
// Every column of a grid's phase-1 array (the grid prolonged over axes 0..d-2) has the same
// last-axis structure: the same coarse length, refinement ratio, centres and offsets s of the
// fine nodes.  Two adjacent columns therefore follow one control flow, and each arithmetic
// instruction can serve both as a packed f32x2 operation: the interpolation of Eqs. (8)-(11)
// (the window preparation and the per-node evaluation) and the float-pair accumulation of
// c_g v.  Each coarse row is read as one 8-byte load per column pair.
//
// Thread layout: threadIdx.x = 32 column pairs (a warp reads 64 consecutive columns, 256
// bytes per coarse row), threadIdx.y = CY consecutive chunks of J fine nodes along the last
// axis; blockIdx.x walks the chunk groups of the last axis, blockIdx.y the column blocks.
// The warps of a block and the blocks with consecutive blockIdx.x read overlapping windows of
// the same columns, so the repeated window loads hit L1 or L2 instead of DRAM.
#pragma once
#include "sg_aux.cuh"
#include "sg_sweep2.cuh"  // weno_scale3x2

// InterpWin<float> for two columns: the same formulas lane by lane (the rescaling of the
// smoothness terms, weno_scale3, works per lane).  The denominator coefficients are kept
// doubled (d = 2 D, exact), so that eval needs the offset s only once per lane.
struct InterpWin2 {
    float2 w0, w1, w2, w3, w4;
    float2 n0, n1, n2, n3, d0, d1, d2;
    __device__ __forceinline__ void prepare(float eps4, int lagrange) {
        const float2 d1_ = sg_sub2(w1, w0), d2_ = sg_sub2(w2, w1), d3_ = sg_sub2(w3, w2), d4_ = sg_sub2(w4, w3);
        const float2 t0 = sg_sub2(d2_, d1_), t1 = sg_sub2(d3_, d2_), t2 = sg_sub2(d4_, d3_);
        const float2 s0 = sg_fma2(sg_f2(3.f), d2_, sg_neg2(d1_)), s1 = sg_add2(d2_, d3_);
        const float2 s2 = sg_fma2(sg_f2(3.f), d3_, sg_neg2(d4_));
        float2 E0 = sg_f2(1.f), E1 = sg_f2(1.f), E2 = sg_f2(1.f);  // 1 for Lagrange
        if (!lagrange) {
            const float2 c13 = sg_f2(13.f / 3.f), ep = sg_f2(eps4);
            float2 e0 = sg_fma2(sg_mul2(c13, t0), t0, sg_fma2(s0, s0, ep));
            float2 e1 = sg_fma2(sg_mul2(c13, t1), t1, sg_fma2(s1, s1, ep));
            float2 e2 = sg_fma2(sg_mul2(c13, t2), t2, sg_fma2(s2, s2, ep));
            weno_scale3x2(e0, e1, e2);
            const float2 q0 = sg_mul2(e0, e0), q1 = sg_mul2(e1, e1), q2 = sg_mul2(e2, e2);
            E0 = sg_mul2(q1, q2);
            E1 = sg_mul2(q0, q2);
            E2 = sg_mul2(q0, q1);
        }
        // C_0 = 1/6 - s/4 + s^2/12, C_1 = 2/3 - s^2/6, C_2 = 1/6 + s/4 + s^2/12
        const float2 A0 = sg_mul2(E0, s0), A1 = sg_mul2(E1, s1), A2 = sg_mul2(E2, s2);
        const float2 B0 = sg_mul2(E0, t0), B1 = sg_mul2(E1, t1), B2 = sg_mul2(E2, t2);
        const float2 Ap = sg_add2(A0, A2), Bp = sg_add2(B0, B2), Ep = sg_add2(E0, E2);
        n0 = sg_fma2(Ap, sg_f2(1.f / 6.f), sg_mul2(sg_f2(2.f / 3.f), A1));
        n1 = sg_fma2(Bp, sg_f2(1.f / 6.f), sg_fma2(sg_sub2(A2, A0), sg_f2(0.25f), sg_mul2(sg_f2(2.f / 3.f), B1)));
        n2 = sg_fma2(sg_sub2(B2, B0), sg_f2(0.25f), sg_fma2(Ap, sg_f2(1.f / 12.f), sg_mul2(sg_f2(-1.f / 6.f), A1)));
        n3 = sg_fma2(Bp, sg_f2(1.f / 12.f), sg_mul2(sg_f2(-1.f / 6.f), B1));
        d0 = sg_fma2(Ep, sg_f2(1.f / 3.f), sg_mul2(sg_f2(4.f / 3.f), E1));
        d1 = sg_mul2(sg_sub2(E2, E0), sg_f2(0.5f));
        d2 = sg_fma2(Ep, sg_f2(1.f / 6.f), sg_mul2(sg_f2(-1.f / 3.f), E1));
    }
    // w2 + s N(s) / d(s) = w2 + (s/2) N(s) / D(s); D >= 1/16 (see Weno<float>::interp), so
    // d >= 1/8 is normal and the hardware reciprocal is within about an ulp.  S = (s, s); at
    // s = 0 the value of the node itself (0 x a finite quotient added to w2).
    __device__ __forceinline__ float2 eval(float2 S) const {
        const float2 N = sg_fma2(sg_fma2(sg_fma2(n3, S, n2), S, n1), S, n0);
        const float2 D = sg_fma2(sg_fma2(d2, S, d1), S, d0);
        const float2 q = sg_mul2(N, make_float2(sg_rcp(D.x), sg_rcp(D.y)));
        return sg_fma2(S, q, w2);
    }
    // the window moved by one coarse node: v is the new last value
    __device__ __forceinline__ void shift(float2 v) {
        w0 = w1;
        w1 = w2;
        w2 = w3;
        w3 = w4;
        w4 = v;
    }
};

// CombineAcc<float> for two columns: an unevaluated float pair per column (error-free sums
// and products), lane by lane the same operations.  c = (c_g, c_g).
struct CombineAcc2 {
    float2 hi = make_float2(0.f, 0.f), lo = make_float2(0.f, 0.f);
    template <bool EXACT>
    __device__ __forceinline__ void add(float2 c, float2 v) {
        if (EXACT) {
            // c v is exact: the two-sum of hi and p = c v with p formed inside the fused
            // operations (s = hi + p and p - bb each rounded once, as with p stored)
            const float2 s = sg_fma2(c, v, hi);
            const float2 bb = sg_sub2(s, hi);
            const float2 e = sg_add2(sg_sub2(hi, sg_sub2(s, bb)), sg_fma2(c, v, sg_neg2(bb)));
            hi = s;
            lo = sg_add2(lo, e);
        } else {
            const float2 p = sg_mul2(c, v);
            const float2 s = sg_add2(hi, p);  // two-sum of hi and p
            const float2 bb = sg_sub2(s, hi);
            const float2 e = sg_add2(sg_sub2(hi, sg_sub2(s, bb)), sg_sub2(p, bb));
            const float2 pe = sg_fma2(c, v, sg_neg2(p));  // exact product error
            hi = s;
            lo = sg_add2(lo, sg_add2(e, pe));
        }
    }
};

// The values of a column pair at the 8 fine nodes j0..j0+7 of one axis for a ratio r = 2^LR <= 8,
// where j0 is a multiple of 8 (so j0 is a multiple of r): node j0 + j has the centre
// c0 + (j >> LR) (+1 in the upper half of its cell) and the offset s = m / r or (m - r) / r,
// m = j mod r -- all fixed at compile time.  W holds the rows c0 - 2 .. c0 + 2; the further rows
// the chunk needs are loaded first.  Nodes with s = 0 coincide with coarse node c0 + (j >> LR) and
// take its value.  sink(j, value) receives node j0 + j.
template <int LR, class Row, class Sink>
__device__ __forceinline__ void chunk_pow2(InterpWin2& W, int c0, float e4, int lagrange, const Row& row, Sink sink) {
    constexpr int R = 1 << LR;
    constexpr int NX = (7 >> LR) + (2 * (7 & (R - 1)) < R ? 0 : 1);  // centre offset of node 7
    float2 ex[NX];
#pragma unroll
    for (int k = 0; k < NX; ++k) ex[k] = row(c0 + k + 3);
    W.prepare(e4, lagrange);
    int at = 0;  // centre offset of the prepared window
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int m = j & (R - 1);
        const int cj = (j >> LR) + (2 * m < R ? 0 : 1);
        if (cj != at) {  // one coarse node further (r >= 2: the centres advance by one)
            W.shift(ex[cj - 1]);
            W.prepare(e4, lagrange);
            at = cj;
        }
        if (m == 0) sink(j, W.w2);
        else sink(j, W.eval(sg_f2((float)(2 * m < R ? m : m - R) / (float)R)));
    }
}

// The same for r = 2^lr >= 16: the chunk lies in one half of one coarse cell (j0 and r / 2 are
// multiples of 8), so one window (rows c0 - 2 .. c0 + 2 in W) serves all 8 nodes, at the
// offsets s_j = s_0 + j / r (exact steps).
template <class Sink>
__device__ __forceinline__ void chunk_one_window(InterpWin2& W, int j0, int lr, float e4, int lagrange, Sink sink) {
    W.prepare(e4, lagrange);
    const int m0 = j0 & ((1 << lr) - 1);
    const float inv_r = pow2_neg<float>(lr);
    float2 S = sg_f2((float)(2 * m0 < (1 << lr) ? m0 : m0 - (1 << lr)) * inv_r);
    const float2 dS = sg_f2(inv_r);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        sink(j, W.eval(S));
        S = sg_add2(S, dS);
    }
}

// centre of fine node j0 for r = 2^lr >= 2: the centre of the window of its first node
__device__ __forceinline__ int chunk_centre0(int j0, int lr) {
    const int i0 = j0 >> lr, m0 = j0 & ((1 << lr) - 1);
    return 2 * m0 < (1 << lr) ? i0 : i0 + 1;
}

// The grid table as the last-axis kernel keeps it in shared memory: one 16-byte entry per grid
// (the phase-1 array, n | lr << 26 with r = 2^lr, the float coefficient).
struct CombineEntry {
    const float* src;
    int nlr;
    float c;
};
#define SG_COMBINE_NLR_SHIFT 26

// Template flags: VEC -- below is even and every source array is 8-byte aligned (both columns
// of a pair with one 8-byte load); ZL -- zeros beyond the ends of the last axis (else periodic).
// Dynamic shared memory: G CombineEntry.
template <int J, int CY, bool EXACT, bool VEC, bool ZL>
__global__ void __launch_bounds__(32 * CY, 2) sg_combine_last_axis_f32x2_kernel(const CombineGrid* __restrict__ tab, int G,
                                                                         double* __restrict__ uhat, long long below,
                                                                         int nf, double eps, int lagrange) {
    static_assert(J == 8, "the chunk schedules assume 8 fine nodes per chunk");
    extern __shared__ __align__(16) unsigned char sg_smem_raw[];
    CombineEntry* s_grid = reinterpret_cast<CombineEntry*>(sg_smem_raw);
    for (int t = threadIdx.y * 32 + threadIdx.x; t < G; t += 32 * CY) {
        const CombineGrid& cg = tab[t];
        CombineEntry e;
        e.src = (const float*)cg.src;
        e.nlr = cg.n | ((__ffs(cg.r) - 1) << SG_COMBINE_NLR_SHIFT);
        e.c = cg.coeff_f;
        s_grid[t] = e;
    }
    __syncthreads();
    const float e4 = sg_eps4<float>(eps);
    constexpr int JB = J * CY;  // fine nodes of the last axis per block
    const int ngroups = (nf + JB - 1) / JB;
    const long long npairs = (below + 1) >> 1;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int j0 = grp * JB + threadIdx.y * J;  // this warp's chunk: a multiple of 8
        if (j0 >= nf) continue;
        const bool full = j0 + J <= nf;
        for (long long pr = blockIdx.y * 32LL + threadIdx.x; pr < npairs; pr += gridDim.y * 32LL) {
            const long long lo = 2 * pr;
            const bool two = lo + 1 < below;
            CombineAcc2 acc[J];
            // one grid's last axis for this column pair
            struct View {
                const float* col;
                int n, lr;
                float2 c;
            };
            auto view = [&](int g) -> View {
                const int4 e = *reinterpret_cast<const int4*>(s_grid + g);
                View v;
                v.col = reinterpret_cast<const float*>(((unsigned long long)(unsigned)e.y << 32) | (unsigned)e.x) + lo;
                v.n = e.z & ((1 << SG_COMBINE_NLR_SHIFT) - 1);
                v.lr = e.z >> SG_COMBINE_NLR_SHIFT;
                v.c = sg_f2(__int_as_float(e.w));
                return v;
            };
            auto row = [&](const View& v, int c) -> float2 {  // coarse row c (c in [-n, 2n))
                const float* p = v.col + (long long)wrap_index(c, v.n) * below;
                float2 x;
                if (VEC) x = __ldg(reinterpret_cast<const float2*>(p));
                else x = make_float2(__ldg(p), two ? __ldg(p + 1) : 0.f);
                if (ZL && (c < 0 || c >= v.n)) x = make_float2(0.f, 0.f);
                return x;
            };
            // centre of node j0: the rows c0 - 2 .. c0 + 2 of the first window (r >= 2), or the
            // first five fine rows j0 .. j0 + 4 (r = 1: c0 = j0 + 2)
            auto centre0 = [&](const View& v) -> int { return v.lr == 0 ? j0 + 2 : chunk_centre0(j0, v.lr); };
            auto first = [&](const View& v, float2 (&w)[5]) {
                const int c0 = centre0(v);
                if (VEC && c0 >= 2 && c0 + 2 < v.n) {  // interior rows: no wrap, no zero boundary
                    const float* p = v.col + (long long)(c0 - 2) * below;
#pragma unroll
                    for (int k = 0; k < 5; ++k, p += below) w[k] = __ldg(reinterpret_cast<const float2*>(p));
                } else {
#pragma unroll
                    for (int k = 0; k < 5; ++k) w[k] = row(v, c0 - 2 + k);
                }
            };
            View nv = view(0);
            float2 nw[5];
            first(nv, nw);
            for (int g = 0; g < G; ++g) {
                const View v = nv;
                InterpWin2 W;
                W.w0 = nw[0];
                W.w1 = nw[1];
                W.w2 = nw[2];
                W.w3 = nw[3];
                W.w4 = nw[4];
                const int c0 = centre0(v);
                if (g + 1 < G) {  // the next grid's first rows are in flight during this grid's work
                    nv = view(g + 1);
                    first(nv, nw);
                }
                auto rowv = [&](int c) { return row(v, c); };
                auto accv = [&](int j, float2 x) { acc[j].template add<EXACT>(v.c, x); };
                if (v.lr == 0) {  // last axis already fine: values at coincident nodes (rows
                                  // j0 + j < 2 nf, read also for j0 + j >= nf and not used)
                    const float2 w8[8] = {W.w0, W.w1, W.w2, W.w3, W.w4, row(v, j0 + 5), row(v, j0 + 6), row(v, j0 + 7)};
#pragma unroll
                    for (int j = 0; j < J; ++j)
                        if (j0 + j < nf) acc[j].template add<EXACT>(v.c, w8[j]);
                    continue;
                }
                if (full) {
                    if (v.lr == 1) {
                        chunk_pow2<1>(W, c0, e4, lagrange, rowv, accv);
                        continue;
                    }
                    if (v.lr == 2) {
                        chunk_pow2<2>(W, c0, e4, lagrange, rowv, accv);
                        continue;
                    }
                    if (v.lr == 3) {
                        chunk_pow2<3>(W, c0, e4, lagrange, rowv, accv);
                        continue;
                    }
                    chunk_one_window(W, j0, v.lr, e4, lagrange, accv);  // r >= 16
                    continue;
                }
                // the last, ragged chunk (r <= 4 only: N_f is a multiple of 8 when N_L >= 3):
                // centres and offsets node by node
                const int r = 1 << v.lr;
                const float inv_r = pow2_neg<float>(v.lr);
                int cur = c0;
                W.prepare(e4, lagrange);
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int jf = j0 + j;
                    if (jf >= nf) break;
                    const int i = jf >> v.lr, m = jf & (r - 1);
                    const int ic = 2 * m < r ? i : i + 1;
                    const float s = (float)(2 * m < r ? m : m - r) * inv_r;
                    if (ic != cur) {  // centres advance by one coarse node at a time (r >= 2)
                        W.shift(row(v, ic + 2));
                        W.prepare(e4, lagrange);
                        cur = ic;
                    }
                    acc[j].template add<EXACT>(v.c, W.eval(sg_f2(s)));
                }
            }
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int jf = j0 + j;
                if (jf >= nf) break;
                const double v0 = (double)acc[j].hi.x + (double)acc[j].lo.x;
                const double v1 = (double)acc[j].hi.y + (double)acc[j].lo.y;
                double* o = uhat + lo + (long long)jf * below;
                if (VEC) {
                    *reinterpret_cast<double2*>(o) = make_double2(v0, v1);
                } else {
                    o[0] = v0;
                    if (two) o[1] = v1;
                }
            }
        }
    }
}

// sg_prolong_multi_kernel for FP32 tasks whose lines come in adjacent pairs (below even, 8-byte
// aligned arrays): thread p takes units 2p and 2p + 1 -- the same chunk of two adjacent columns
// -- and runs the window arithmetic once for both in packed f32x2 form (InterpWin2), with
// 8-byte loads and stores.  The tasks' unit ranges are even-sized, so a pair never straddles
// two tasks.  A chunk starts at a multiple of 8, so whole chunks follow the compile-time
// schedules of chunk_pow2 (r <= 8) or one window (r >= 16); only a last, ragged chunk takes its
// centres node by node.  Every task has r >= 2 (axes already at the finest level are skipped).
template <int J>
__global__ void __launch_bounds__(256) sg_prolong_multi_x2_kernel(const ProlongTask* __restrict__ tasks, int ntasks,
                                                                  long long nunits, double eps, int lagrange) {
    static_assert(J == 8, "the chunk schedules assume 8 fine nodes per chunk");
    const float e4 = sg_eps4<float>(eps);
    const long long npairs = nunits >> 1;
    for (long long pp = blockIdx.x * 256LL + threadIdx.x; pp < npairs; pp += gridDim.x * 256LL) {
        const long long u = 2 * pp;
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
        const unsigned lo = v - q * below;  // even: below is even and v is even
        const unsigned hi = div_mag(q, (unsigned)nchunks, tk.nch_mag);
        const int j0 = (int)(q - hi * (unsigned)nchunks) * J;
        const int n = tk.n, nf = tk.nf, lr = __ffs(tk.r) - 1;
        const bool zero_bc = tk.zero_bc != 0;
        const float* col = (const float*)tk.in + (long long)hi * below * n + lo;
        float* ocol = (float*)tk.out + (long long)hi * below * nf + lo;
        auto at = [&](int c) -> float2 {  // both columns' coarse value c, c in [-n, 2n)
            float2 x = __ldg(reinterpret_cast<const float2*>(col + (long long)wrap_index(c, n) * below));
            if (zero_bc && (c < 0 || c >= n)) x = make_float2(0.f, 0.f);
            return x;
        };
        auto put = [&](int j, float2 x) { *reinterpret_cast<float2*>(ocol + (long long)(j0 + j) * below) = x; };
        const int c0 = chunk_centre0(j0, lr);
        InterpWin2 W;
        W.w0 = at(c0 - 2);
        W.w1 = at(c0 - 1);
        W.w2 = at(c0);
        W.w3 = at(c0 + 1);
        W.w4 = at(c0 + 2);
        if (j0 + J <= nf) {
            if (lr == 1) chunk_pow2<1>(W, c0, e4, lagrange, at, put);
            else if (lr == 2) chunk_pow2<2>(W, c0, e4, lagrange, at, put);
            else if (lr == 3) chunk_pow2<3>(W, c0, e4, lagrange, at, put);
            else chunk_one_window(W, j0, lr, e4, lagrange, put);
            continue;
        }
        const int r = 1 << lr;
        const float inv_r = pow2_neg<float>(lr);
        int cur = c0;
        W.prepare(e4, lagrange);
#pragma unroll 1
        for (int j = 0; j < J; ++j) {
            const int jf = j0 + j;
            if (jf >= nf) break;
            const int i = jf >> lr, m = jf & (r - 1);
            const int ic = 2 * m < r ? i : i + 1;
            const float sv = (float)(2 * m < r ? m : m - r) * inv_r;
            if (ic != cur) {  // centres advance by one coarse node at a time (r >= 2)
                W.shift(at(ic + 2));
                W.prepare(e4, lagrange);
                cur = ic;
            }
            put(j, W.eval(sg_f2(sv)));
        }
    }
}
