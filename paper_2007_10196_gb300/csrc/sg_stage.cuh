// sg_stage.cuh -- the TVD-RK3 stage kernels: LF split + WENO5 fluxes on every axis
// (Section 2.1), the conservative flux difference (Eq. 2), the Shu-Osher stage update and
// the per-grid max |u| of the result for the next stage's Lax-Friedrichs alpha, all fused.
//
// Both kernels are persistent: each block walks work items (grid, tile) of
// [item_begin, item_end) with a grid stride; a tile is a box of at most SG_NT * PPT points.
#pragma once
#include "sg_weno.cuh"

// ------------------------------------------------------------------------------------
// State storage and stage update.
//
// FP64 (Shu-Osher form, literal):  arrays u0 = u^n (and u^{n+1}, written in place by the
// last stage, which reads u0 only at its own point), u1 = u^{(1)}, u2 = u^{(2)}:
//   u1 = u + dt L(u);  u2 = 3/4 u + 1/4 (u1 + dt L(u1));  u = 1/3 u + 2/3 (u2 + dt L(u2)).
//
// FP32 (the same scheme in increment form with a compensated state): u^n = U + C with a
// float pair; stage increments are small and keep full float precision:
//   D1 = dt L(U)                        (u1 = U + D1)
//   D2 = (D1 + dt L(U + D1)) / 4        (u2 = U + D2)
//   u^{n+1} = U + C + 2/3 (D2 + dt L(U + D2)), added to (U, C) with an error-free sum.
// U and D1 share a ping-pong pair (u0, u1): the last stage writes the new U over D1 (no
// longer needed), so no array is read by a stencil while it is written.  `parity` selects
// which of the pair holds U this step; u2 holds D2, u3 holds C.
// ------------------------------------------------------------------------------------
template <class T>
struct StageIO;

template <>
struct StageIO<double> {
    const double* in;
    const double* un;
    double* out;
    int stage;
    __device__ __forceinline__ void setup(const GridDesc* G, int s, int /*parity*/) {
        stage = s;
        in = (const double*)(s == 0 ? G->u0 : s == 1 ? G->u1 : G->u2);
        un = (const double*)G->u0;
        out = (double*)(s == 0 ? G->u1 : s == 1 ? G->u2 : G->u0);
    }
    // advances every pointer by o elements (tile-relative indexing)
    __device__ __forceinline__ void shift(long long o) {
        in += o;
        un += o;
        out += o;
    }
    __device__ __forceinline__ double load(long long g) const { return in[g]; }
    // writes the stage result at g; returns it (for the alpha reduction)
    __device__ __forceinline__ double update(long long g, double L, double dt) const {
        const double us = in[g];
        double o;
        if (stage == 0) o = us + dt * L;
        else if (stage == 1) o = 0.75 * un[g] + 0.25 * (us + dt * L);
        else o = (1.0 / 3.0) * un[g] + (2.0 / 3.0) * (us + dt * L);
        out[g] = o;
        return o;
    }
};

template <>
struct StageIO<float> {
    const float* U;
    float* Ub;   // D1 during stages 0-1, the new U after stage 2
    float* D2;
    float* Cc;
    int stage;
    __device__ __forceinline__ void setup(const GridDesc* G, int s, int parity) {
        stage = s;
        U = (const float*)(parity ? G->u1 : G->u0);
        Ub = (float*)(parity ? G->u0 : G->u1);
        D2 = (float*)G->u2;
        Cc = (float*)G->u3;
    }
    // advances every pointer by o elements (tile-relative indexing)
    __device__ __forceinline__ void shift(long long o) {
        U += o;
        Ub += o;
        D2 += o;
        Cc += o;
    }
    // the arrays whose sum is the stencil input: U, and D1 (stage 1) or D2 (stage 2)
    __device__ __forceinline__ void stencil_src(const float*& a, const float*& b) const {
        a = U;
        b = stage == 0 ? nullptr : (stage == 1 ? Ub : D2);
    }
    __device__ __forceinline__ float load(long long g) const {
        if (stage == 0) return U[g];
        if (stage == 1) return U[g] + Ub[g];
        return U[g] + D2[g];
    }
    __device__ __forceinline__ float update(long long g, float L, float dt) const {
        const float d = dt * L;
        const float u = U[g];
        if (stage == 0) {
            Ub[g] = d;
            return u + d;
        }
        if (stage == 1) {
            const float nd = 0.25f * (Ub[g] + d);
            D2[g] = nd;
            return u + nd;
        }
        const float y = fmaf(2.f / 3.f, D2[g] + d, Cc[g]);
        // error-free sum (Knuth): u + y = s + err exactly
        const float s = u + y;
        const float bb = s - u;
        const float err = (u - (s - bb)) + (y - bb);
        Ub[g] = s;
        Cc[g] = err;
        return s;
    }
    // true if every array of the stage starts on a 16-byte boundary (update4 may be used)
    __device__ __forceinline__ bool aligned16() const {
        const unsigned long long a = reinterpret_cast<unsigned long long>(U) | reinterpret_cast<unsigned long long>(Ub) |
                                     reinterpret_cast<unsigned long long>(D2) | reinterpret_cast<unsigned long long>(Cc);
        return (a & 15) == 0;
    }
    // update() of four consecutive points g..g+3 (g a multiple of 4) with 16-byte accesses;
    // the same arithmetic per point
    __device__ __forceinline__ float4 update4(long long g, const float (&L)[4], float dt) const {
        const float4 u = *reinterpret_cast<const float4*>(U + g);
        const float uu[4] = {u.x, u.y, u.z, u.w};
        float o[4];
        if (stage == 0) {
            float dd[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                dd[l] = dt * L[l];
                o[l] = uu[l] + dd[l];
            }
            *reinterpret_cast<float4*>(Ub + g) = make_float4(dd[0], dd[1], dd[2], dd[3]);
        } else if (stage == 1) {
            const float4 b = *reinterpret_cast<const float4*>(Ub + g);
            const float bb[4] = {b.x, b.y, b.z, b.w};
            float nd[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const float d = dt * L[l];
                nd[l] = 0.25f * (bb[l] + d);
                o[l] = uu[l] + nd[l];
            }
            *reinterpret_cast<float4*>(D2 + g) = make_float4(nd[0], nd[1], nd[2], nd[3]);
        } else {
            const float4 d2 = *reinterpret_cast<const float4*>(D2 + g);
            const float4 c = *reinterpret_cast<const float4*>(Cc + g);
            const float dd2[4] = {d2.x, d2.y, d2.z, d2.w}, cc[4] = {c.x, c.y, c.z, c.w};
            float er[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const float d = dt * L[l];
                const float y = fmaf(2.f / 3.f, dd2[l] + d, cc[l]);
                const float sm = uu[l] + y;
                const float bb = sm - uu[l];
                er[l] = (uu[l] - (sm - bb)) + (y - bb);
                o[l] = sm;
            }
            *reinterpret_cast<float4*>(Ub + g) = make_float4(o[0], o[1], o[2], o[3]);
            *reinterpret_cast<float4*>(Cc + g) = make_float4(er[0], er[1], er[2], er[3]);
        }
        return make_float4(o[0], o[1], o[2], o[3]);
    }
};

template <class T>
__device__ __forceinline__ int stage_parity(const InstState* S) {
    return (int)((S->steps - S->step0) & 1);
}

__device__ __forceinline__ double sg_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float sg_max(float a, float b) { return fmaxf(a, b); }

// Epilogue shared by both kernels: non-finite flag, alpha slot of the next stage, and the
// clearing of the slot two stages ahead (by the grid's first item).  The block max is taken in
// the state precision and widened to double once per tile.
template <class T>
__device__ __forceinline__ void stage_epilogue(const StageArgs& A, const WorkItem& w, const GridDesc* G, int it,
                                               T mx, bool bad, T* red) {
    if (A.phys.pde == 1) {
        // one reduction for both: a non-finite value is carried as -1 (|u| >= 0 otherwise)
        const T m = block_max(bad ? T(-1) : mx, red, bad);
        if (threadIdx.x == 0) {
            if (m < T(0)) atomicOr(A.flags + SG_FLAG_NONFINITE, 1);
            else atomicMax(A.alpha + w.grid * 3 + (A.stage + 1) % 3, alpha_enc(m));
        }
    } else if (__syncthreads_or(bad) && threadIdx.x == 0) {
        atomicOr(A.flags + SG_FLAG_NONFINITE, 1);
    }
    if (threadIdx.x == 0 && it == G->first_item) A.alpha[w.grid * 3 + (A.stage + 2) % 3] = 0ull;
}

// Barrier-free variant for the sweep kernel: each warp folds its max |u| into the alpha slot
// with one atomicMax (max is exact and order-independent, so the slot gets the same value) and
// raises the non-finite flag itself; a warp holding a non-finite value leaves the slot alone.
template <class T>
__device__ __forceinline__ void stage_epilogue_warp(const StageArgs& A, const WorkItem& w, const GridDesc* G,
                                                    int it, T mx, bool bad) {
    const unsigned anybad = __ballot_sync(0xffffffffu, bad);
    if (A.phys.pde == 1) {
        for (int o = 16; o > 0; o >>= 1) mx = sg_fmax_(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0 && !anybad) atomicMax(A.alpha + w.grid * 3 + (A.stage + 1) % 3, alpha_enc(mx));
    }
    if ((threadIdx.x & 31) == 0 && anybad) atomicOr(A.flags + SG_FLAG_NONFINITE, 1);
    if (threadIdx.x == 0 && it == G->first_item) A.alpha[w.grid * 3 + (A.stage + 2) % 3] = 0ull;
}

// ------------------------------------------------------------------------------------
// d <= 3: padded-box kernel.  Per tile: one load of the tile with a 3-point halo on each face
// (periodic wrap, or zeros beyond the ends of a zero-boundary axis), the LF split computed once
// per loaded value (Burgers: the split is the
// same on every axis); one phase computing every interface flux of every axis once; one
// phase forming L = -sum_k (F_{i+1/2} - F_{i-1/2}) / h_k and the stage update.
// Shared memory: two box arrays of box_elems values (f^+, f^-; or u and unused) and the
// flux arrays of all axes (flux_elems), sized by the host for the largest tile.
// Flux layouts (x fastest where possible, for conflict-free shared-memory access):
//   axis 0: F0[(y + e1 z)(e0+1) + i];  axis 1: F1[x + e0 (i + (e1+1) z)];  axis 2: F2[x + e0 (y + e1 i)]
// where i indexes the interface between tile-local points i-1 and i.
// ------------------------------------------------------------------------------------
template <class T, int D, int PPT>
__global__ void __launch_bounds__(SG_NT) sg_stage_box_kernel(const StageArgs A) {
    static_assert(D >= 1 && D <= 3, "box kernel handles d <= 3");
    extern __shared__ __align__(16) unsigned char sg_smem_raw[];
    T* bp = reinterpret_cast<T*>(sg_smem_raw);
    T* bm = bp + A.box_elems;
    T* fb = bm + A.box_elems;
    __shared__ T red[SG_NT / 32];

    const int tid = threadIdx.x;
    const PhysParams& ph = A.phys;
    const bool burgers = ph.pde == 1;
    const bool vlasov = ph.pde == 2;  // d = 2: axis 0 = x (speed v_j), axis 1 = v (speed E_i, 0 beyond the ends)
    const T eps4 = sg_eps4<T>(ph.eps);
    const T adv0 = (T)ph.adv[0], adv1 = (T)ph.adv[1], adv2 = (T)ph.adv[2];
    const int zm = ph.zmask;  // zero boundary per axis (advection / Burgers)

    for (int it = A.item_begin + blockIdx.x; it < A.item_end; it += gridDim.x) {
        const WorkItem w = A.items[it];
        const GridDesc* G = A.grids + w.grid;
        const InstState* S = A.inst + G->inst;
        if (!S->active) continue;  // uniform: the state is not written during this kernel
        const T dt = inst_dt<T>(S);
        StageIO<T> io;
        io.setup(G, A.stage, stage_parity<T>(S));

        int org[3] = {0, 0, 0}, e[3] = {1, 1, 1}, n[3] = {1, 1, 1};
        long long gs[3] = {1, 0, 0};
        {
            int tc[D];
            tile_coords<D>(G, (unsigned)w.tile, tc);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                n[k] = G->n[k];
                org[k] = tc[k] * G->te[k];
                e[k] = min(G->te[k], n[k] - org[k]);
            }
            if (D >= 2) gs[1] = n[0];
            if (D >= 3) gs[2] = (long long)n[0] * n[1];
        }
        const int P = e[0] * e[1] * e[2];
        const int B0 = e[0] + 6, B1 = D >= 2 ? e[1] + 6 : 1;
        const T alpha_b = alpha_dec<T>(A.alpha[w.grid * 3 + A.stage]);
        const T half_alpha = (T)0.5 * alpha_b;
        FDiv fe0, fe1, fr0, fp0, fp1;
        fe0.init(e[0]);
        fe1.init(e[1]);
        fr0.init(e[0] + 6);
        fp0.init(e[0] + 1);
        fp1.init(e[1] + 1);

        // ---- 1) load the padded box (interior + face halos), split once per value
        auto put = [&](int bidx, long long g) {
            const T v = io.load(g);
            if (burgers) {
                if constexpr (sizeof(T) == 8) {
                    double fp, fm;
                    Weno<double>::split(v, alpha_b, 0.0, 1, fp, fm);
                    bp[bidx] = fp;
                    bm[bidx] = fm;
                } else {
                    float fp, fm;
                    Weno<float>::split_burgers(v, half_alpha, fp, fm);
                    bp[bidx] = fp;
                    bm[bidx] = fm;
                }
            } else {
                bp[bidx] = v;
            }
        };
        auto put0 = [&](int bidx) {  // a zero boundary value (its split values are 0 too)
            bp[bidx] = T(0);
            if (burgers) bm[bidx] = T(0);
        };
        {
            const int n0 = B0 * e[1] * e[2];  // interior rows extended by the axis-0 halos
            for (int q = tid; q < n0; q += SG_NT) {
                const int r = (int)fr0.div((unsigned)q);
                const int x = q - r * B0;
                int y = 0, z = 0;
                if (D >= 2) {
                    z = (int)fe1.div((unsigned)r);
                    y = r - z * e[1];
                }
                int gx = org[0] + x - 3;
                const int bidx = x + B0 * ((y + (D >= 2 ? 3 : 0)) + B1 * (z + (D >= 3 ? 3 : 0)));
                if ((zm & 1) && (gx < 0 || gx >= n[0])) {
                    put0(bidx);
                    continue;
                }
                if (gx < 0) gx += n[0];
                else if (gx >= n[0]) gx -= n[0];
                const long long g = gx + gs[1] * (org[1] + y) + gs[2] * (org[2] + z);
                put(bidx, g);
            }
            if (D >= 2) {
                const int n1 = e[0] * 6 * e[2];  // axis-1 halos
                for (int q = tid; q < n1; q += SG_NT) {
                    const int r = (int)fe0.div((unsigned)q);
                    const int x = q - r * e[0];
                    const int z = r / 6, h = r - z * 6;
                    const int y = h < 3 ? h - 3 : e[1] + h - 3;
                    int gy = org[1] + y;
                    const int bidx = (x + 3) + B0 * ((y + 3) + B1 * (z + (D >= 3 ? 3 : 0)));
                    if ((vlasov || (zm & 2)) && (gy < 0 || gy >= n[1])) {  // zero inflow in v / zero boundary
                        put0(bidx);
                        continue;
                    }
                    if (gy < 0) gy += n[1];
                    else if (gy >= n[1]) gy -= n[1];
                    const long long g = (org[0] + x) + gs[1] * gy + gs[2] * (org[2] + z);
                    put(bidx, g);
                }
            }
            if (D >= 3) {
                const int n2 = e[0] * e[1] * 6;  // axis-2 halos
                for (int q = tid; q < n2; q += SG_NT) {
                    const int r = (int)fe0.div((unsigned)q);
                    const int x = q - r * e[0];
                    const int h = (int)fe1.div((unsigned)r);
                    const int y = r - h * e[1];
                    const int z = h < 3 ? h - 3 : e[2] + h - 3;
                    int gz = org[2] + z;
                    const int bidx = (x + 3) + B0 * ((y + 3) + B1 * (z + 3));
                    if ((zm & 4) && (gz < 0 || gz >= n[2])) {
                        put0(bidx);
                        continue;
                    }
                    if (gz < 0) gz += n[2];
                    else if (gz >= n[2]) gz -= n[2];
                    const long long g = (org[0] + x) + gs[1] * (org[1] + y) + gs[2] * gz;
                    put(bidx, g);
                }
            }
        }
        __syncthreads();

        // ---- 2) every interface flux of every axis, once
        const int NF0 = (e[0] + 1) * e[1] * e[2];
        const int NF1 = D >= 2 ? e[0] * (e[1] + 1) * e[2] : 0;
        const int NF2 = D >= 3 ? e[0] * e[1] * (e[2] + 1) : 0;
        const int NF = NF0 + NF1 + NF2;
        // Vlasov-Poisson: the LF alpha along x is max_j |v_j| of the grid (an end node)
        T ax = T(0);
        if (vlasov) {
            const T v0 = (T)G->lo[1], v1 = (T)G->lo[1] + (T)(n[1] - 1) * (T)G->h[1];
            ax = sg_max(sg_abs(v0), sg_abs(v1));
        }
        for (int q = tid; q < NF; q += SG_NT) {
            int b, Sx;
            T ak, al;
            if (q < NF0) {
                Sx = 1;
                ak = adv0;
                const int r = (int)fp0.div((unsigned)q);
                const int i = q - r * (e[0] + 1);
                int y = 0, z = 0;
                if (D >= 2) {
                    z = (int)fe1.div((unsigned)r);
                    y = r - z * e[1];
                }
                b = i + B0 * ((y + (D >= 2 ? 3 : 0)) + B1 * (z + (D >= 3 ? 3 : 0)));
                if (vlasov) ak = (T)G->lo[1] + (T)(org[1] + y) * (T)G->h[1];  // v_j of the line
                al = vlasov ? ax : sg_abs(ak);
            } else if (D >= 2 && q < NF0 + NF1) {
                Sx = B0;
                ak = adv1;
                const int qq = q - NF0;
                const int r = (int)fe0.div((unsigned)qq);
                const int x = qq - r * e[0];
                const int z = (int)fp1.div((unsigned)r);
                const int i = r - z * (e[1] + 1);
                b = (x + 3) + B0 * (i + B1 * (z + (D >= 3 ? 3 : 0)));
                if (vlasov) ak = ((const T*)G->ef)[org[0] + x];  // E_i of the line
                al = vlasov ? alpha_b : sg_abs(ak);
            } else {
                Sx = B0 * B1;
                ak = adv2;
                const int qq = q - NF0 - NF1;
                const int r = (int)fe0.div((unsigned)qq);
                const int x = qq - r * e[0];
                const int i = (int)fe1.div((unsigned)r);
                const int y = r - i * e[1];
                b = (x + 3) + B0 * ((y + 3) + B1 * i);
                al = sg_abs(ak);
            }
            T F;
            if constexpr (sizeof(T) == 8) {
                if (burgers) {
                    F = Weno<double>::interface_split((const double*)bp + b, (const double*)bm + b, Sx, ph);
                } else {
                    F = Weno<double>::interface((const double*)bp + b, Sx, (double)al, (double)ak, ph);
                }
            } else {
                if (burgers) {
                    F = Weno<float>::interface_split((const float*)bp + b, (const float*)bm + b, Sx, eps4, ph.scheme);
                } else {
                    F = Weno<float>::interface((const float*)bp + b, Sx, (float)al, (float)ak, ph, eps4);
                }
            }
            fb[q] = F;
        }
        __syncthreads();

        // ---- 3) flux difference, stage update, alpha of the result
        T mx = T(0);
        bool bad = false;
        const T r0 = grid_rdx<T>(G, 0), r1 = grid_rdx<T>(G, 1), r2 = grid_rdx<T>(G, 2);
#pragma unroll
        for (int qq = 0; qq < PPT; ++qq) {
            const int p = tid + qq * SG_NT;
            if (p >= P) continue;
            const int r = (int)fe0.div((unsigned)p);
            const int c0 = p - r * e[0];
            int c1 = 0, c2 = 0;
            if (D >= 2) {
                c2 = (int)fe1.div((unsigned)r);
                c1 = r - c2 * e[1];
            }
            T L = T(0);
            {
                const T* F = fb + (c1 + e[1] * c2) * (e[0] + 1) + c0;
                L = L - (F[1] - F[0]) * r0;
            }
            if (D >= 2) {
                const T* F = fb + NF0 + c0 + e[0] * (c1 + (e[1] + 1) * c2);
                L = L - (F[e[0]] - F[0]) * r1;
            }
            if (D >= 3) {
                const T* F = fb + NF0 + NF1 + c0 + e[0] * (c1 + e[1] * c2);
                L = L - (F[e[0] * e[1]] - F[0]) * r2;
            }
            const long long g = (org[0] + c0) + gs[1] * (org[1] + c1) + gs[2] * (org[2] + c2);
            const T o = io.update(g, L, dt);
            if (!sg_isfinite(o)) bad = true;
            mx = sg_max(mx, sg_abs(o));
        }
        stage_epilogue(A, w, G, it, mx, bad, red);
        __syncthreads();  // the next tile overwrites the shared arrays
    }
}

// ------------------------------------------------------------------------------------
// d = 3: line-sweep kernel.  Per tile (extents <= 8 on every axis, so at most 8^3 points and
// 3 * 64 = 192 lines): one load of the padded box (as above, periodic or zero beyond the ends of
// a zero-boundary axis; x stride made odd so that threads
// on neighbouring x-lines hit different banks); then every thread takes one line of one axis
// and sweeps it, keeping the five-point windows of f^+ and f^- in registers, so each new
// interface costs one shared-memory load per side; the flux difference of each point goes to
// a per-axis array D_k; finally each point forms L = ((0 - D_0) - D_1) - D_2 (the axis order
// of the FP64 definition) and takes the stage update.
//
// SweepSide<T>: one side of the WENO5 reconstruction sliding along a line.  push_back shifts
// in a value at the far end (the positive-wind stencil f_{i-2..i+2}); push_front at the near
// end (the mirrored negative-wind stencil f_{i+3..i-1}).
//   double: keeps the raw window and evaluates Eqs. (3)-(6) literally per interface.
//   float: keeps first differences d1..d4 and T_j = (13/3) t_j^2 + 4 eps (t = second differences)
//     and updates them incrementally, so consecutive interfaces share them.
// ------------------------------------------------------------------------------------
template <class T>
struct SweepSide;

template <>
struct SweepSide<double> {
    double w0, w1, w2, w3, w4;
    __device__ __forceinline__ void init(double a, double b, double c, double d, double e, double) {
        w0 = a; w1 = b; w2 = c; w3 = d; w4 = e;
    }
    __device__ __forceinline__ void push_back(double v, double) {
        w0 = w1; w1 = w2; w2 = w3; w3 = w4; w4 = v;
    }
    __device__ __forceinline__ void push_front(double v, double) {
        w4 = w3; w3 = w2; w2 = w1; w1 = w0; w0 = v;
    }
};

template <>
struct SweepSide<float> {
    float w0, w1, c, w3, w4;    // the window (c = centre); shifted, never recomputed
    float d1, d2, d3, d4;       // first differences: the same values a fresh window would give
    float T0, T1, T2;           // (13/3) t^2 + 4 eps of the three second differences
    __device__ __forceinline__ void init(float a, float b, float cc, float d, float e, float eps4) {
        w0 = a; w1 = b; c = cc; w3 = d; w4 = e;
        d1 = b - a; d2 = cc - b; d3 = d - cc; d4 = e - d;
        const float t0 = d2 - d1, t1 = d3 - d2, t2 = d4 - d3;
        T0 = fmaf((13.f / 3.f) * t0, t0, eps4);
        T1 = fmaf((13.f / 3.f) * t1, t1, eps4);
        T2 = fmaf((13.f / 3.f) * t2, t2, eps4);
    }
    __device__ __forceinline__ void push_back(float v, float eps4) {
        w0 = w1; w1 = c; c = w3; w3 = w4;
        d1 = d2; d2 = d3; d3 = d4; d4 = v - w4;
        w4 = v;
        T0 = T1; T1 = T2;
        const float t2 = d4 - d3;
        T2 = fmaf((13.f / 3.f) * t2, t2, eps4);
    }
    __device__ __forceinline__ void push_front(float v, float eps4) {
        w4 = w3; w3 = c; c = w1; w1 = w0;
        d4 = d3; d3 = d2; d2 = d1; d1 = w0 - v;
        w0 = v;
        T2 = T1; T1 = T0;
        const float t0 = d2 - d1;
        T0 = fmaf((13.f / 3.f) * t0, t0, eps4);
    }
    // numerator and denominator of fhat - c (as in Weno<float>::side)
    // With E_k = e_k^2, e_k = 4 (eps + beta_k) rescaled by weno_scale3, the weights are proportional to
    // a_0 = E_1 E_2 / 6, a_1 = E_0 E_2, a_2 = E_0 E_1 / 2 (linear scheme: all E_k = 1, giving
    // 0.1, 0.6, 0.3), and num = sum a_k p_k, den = sum a_k are formed factored:
    // num = E_1 (E_2 p_0/6 + E_0 p_2/2) + E_0 E_2 p_1,  den = E_1 (E_2/6 + E_0/2) + E_0 E_2.
    __device__ __forceinline__ void value(int linear, float& num, float& den) const {
        const float p0s = fmaf(5.f / 36.f, d2, (-1.f / 18.f) * d1);  // p_0 / 6
        const float p1 = fmaf(1.f / 6.f, d2, (1.f / 3.f) * d3);
        const float p2h = fmaf(1.f / 3.f, d3, (-1.f / 12.f) * d4);   // p_2 / 2
        float E0 = 1.f, E1 = 1.f, E2 = 1.f;
        if (!linear) {
            const float s0 = fmaf(3.f, d2, -d1), s1 = d2 + d3, s2 = fmaf(3.f, d3, -d4);
            float e0 = fmaf(s0, s0, T0);
            float e1 = fmaf(s1, s1, T1);
            float e2 = fmaf(s2, s2, T2);
            weno_scale3(e0, e1, e2);  // ratios only: smallest in [1, 2), others capped at 2^20
            E0 = e0 * e0;
            E1 = e1 * e1;
            E2 = e2 * e2;
        }
        const float X = E0 * E2;
        num = fmaf(E1, fmaf(E2, p0s, E0 * p2h), X * p1);
        den = fmaf(E1, fmaf(E2, 1.f / 6.f, 0.5f * E0), X);
    }
};

__device__ __forceinline__ double sweep_flux(const SweepSide<double>& P, const SweepSide<double>& M,
                                             const PhysParams& ph) {
    const double fplus = Weno<double>::side(P.w0, P.w1, P.w2, P.w3, P.w4, ph.eps, ph.scheme);
    const double fminus = Weno<double>::side(M.w0, M.w1, M.w2, M.w3, M.w4, ph.eps, ph.scheme);
    return fplus + fminus;
}

__device__ __forceinline__ float sweep_flux(const SweepSide<float>& P, const SweepSide<float>& M,
                                            const PhysParams& ph) {
    float np, dp, nm, dm;
    P.value(ph.scheme, np, dp);
    M.value(ph.scheme, nm, dm);
    return Weno<float>::combine(P.c, M.c, np, dp, nm, dm);
}

#define SG_NT3 192  // threads of the d = 3 sweep kernel: one per line of an 8x8x8 tile
// Flux differences of axis k: line l of the tile (axis 0: y + e1 z; axis 1: x + e0 z; axis 2:
// x + e0 y), point i along it, at Dk[SG_DK_AXIS k + 9 l + i].  The odd line stride puts the
// lines a warp sweeps, and the points a warp updates, on distinct banks.
#define SG_DK_AXIS 576

// ZB: some axis has a zero boundary (the periodic instantiation carries no boundary tests)
template <class T, bool ZB>
__global__ void __launch_bounds__(SG_NT3, sizeof(T) == 4 ? 6 : 1) sg_stage_sweep3_kernel(const StageArgs A) {
    extern __shared__ __align__(16) unsigned char sg_smem_raw[];
    T* bp = reinterpret_cast<T*>(sg_smem_raw);   // f^+ (Burgers) or u (advection)
    T* bm = bp + A.box_elems;                     // f^-
    T* Dk = bm + A.box_elems;                     // 3 x SG_DK_AXIS flux differences

    const int tid = threadIdx.x;
    const PhysParams& ph = A.phys;
    const bool burgers = ph.pde == 1;
    const T eps4 = sg_eps4<T>(ph.eps);
    const T adv[3] = {(T)ph.adv[0], (T)ph.adv[1], (T)ph.adv[2]};
    const int zm = ZB ? ph.zmask : 0;  // zero boundary per axis (advection / Burgers)

    for (int it = A.item_begin + blockIdx.x; it < A.item_end; it += gridDim.x) {
        const WorkItem w = A.items[it];
        const GridDesc* G = A.grids + w.grid;
        const InstState* S = A.inst + G->inst;
        if (!S->active) continue;  // uniform: the state is not written during this kernel
        const T dt = inst_dt<T>(S);
        StageIO<T> io;
        io.setup(G, A.stage, stage_parity<T>(S));

        int org[3], e[3], n[3];
        {
            int tc[3];
            tile_coords<3>(G, (unsigned)w.tile, tc);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                n[k] = G->n[k];
                org[k] = tc[k] * G->te[k];
                e[k] = min(G->te[k], n[k] - org[k]);
            }
        }
        // global indices below are 32-bit offsets from the tile's first point (a grid holds
        // fewer than 2^31 points): one 64-bit address computation per tile
        const int n0 = n[0], n01 = n[0] * n[1];
        io.shift(org[0] + (long long)n0 * org[1] + (long long)n01 * org[2]);
        const int P = e[0] * e[1] * e[2];
        const int R0 = e[0] + 6;                 // valid row length along x
        const int B0 = R0 | 1;                   // odd row stride
        const int B1 = e[1] + 6;
        const T alpha_b = alpha_dec<T>(A.alpha[w.grid * 3 + A.stage]);
        const T half_alpha = (T)0.5 * alpha_b;
        FDiv fR0, fe0, fe1;
        fR0.init(R0);
        fe0.init(e[0]);
        fe1.init(e[1]);

        // split of one loaded stencil value into the box
        auto put = [&](int bidx, T v) {
            if (burgers) {
                if constexpr (sizeof(T) == 8) {
                    double fp, fm;
                    Weno<double>::split(v, alpha_b, 0.0, 1, fp, fm);
                    bp[bidx] = fp;
                    bm[bidx] = fm;
                } else {
                    float fp, fm;
                    Weno<float>::split_burgers(v, half_alpha, fp, fm);
                    bp[bidx] = fp;
                    bm[bidx] = fm;
                }
            } else {
                bp[bidx] = v;
            }
        };
        // FP32, tile 8 wide at an x origin and row length that are multiples of 4, on grids whose
        // arrays start on a 16-byte boundary (grids are packed back to back, so not all do):
        // every row segment the box needs is read as 16-byte float4 loads (4 per x-row with its
        // halos, 2 per halo row), wrapping whole chunks at the faces
        bool vec = false;
        const T* A0 = nullptr;
        const T* A1 = nullptr;
        if constexpr (sizeof(T) == 4) {
            io.stencil_src(A0, A1);
            const unsigned long long align = reinterpret_cast<unsigned long long>(A0) |
                                             reinterpret_cast<unsigned long long>(A1);
            vec = e[0] == 8 && (org[0] & 3) == 0 && (n[0] & 3) == 0 && (align & 15) == 0;
        }
        if constexpr (sizeof(T) == 4) {
            if (vec) {
                const int nr0 = e[1] * e[2] * 4, nr1 = 12 * e[2], nr2 = 12 * e[1];
                const int ntask = nr0 + nr1 + nr2;
                // task t: one float4 chunk; its box index with three flags (drop the chunk's first
                // value: x = -4; drop its last: x = 11; the chunk lies beyond the end of a
                // zero-boundary axis: all four values are 0) packed above bit 16.  Chunks never
                // straddle an end (x origins and row lengths are multiples of 4).
                auto chunk = [&](int t, long long& g) -> int {
                    int gx, gy, gz, bx, y, z, flags = 0;
                    if (t < nr0) {
                        const int c = t & 3, r = t >> 2;
                        z = (int)fe1.div(r);
                        y = r - z * e[1];
                        bx = 4 * c - 1;  // box x of the chunk's first value (x = 4c - 4)
                        flags = (c == 0 ? 1 : 0) | (c == 3 ? 2 : 0);
                        gx = org[0] + 4 * c - 4;
                        if ((zm & 1) && (gx < 0 || gx >= n[0])) flags |= 4;
                        gx = gx < 0 ? gx + n[0] : (gx >= n[0] ? gx - n[0] : gx);
                        gy = org[1] + y;
                        gz = org[2] + z;
                    } else if (t < nr0 + nr1) {
                        const int q = t - nr0, c = q & 1, r = q >> 1;
                        z = r / 6;
                        const int h = r - z * 6;
                        y = h < 3 ? h - 3 : e[1] + h - 3;
                        bx = 4 * c + 3;
                        gx = org[0] + 4 * c;
                        gy = org[1] + y;
                        if ((zm & 2) && (gy < 0 || gy >= n[1])) flags |= 4;
                        gy = gy < 0 ? gy + n[1] : (gy >= n[1] ? gy - n[1] : gy);
                        gz = org[2] + z;
                    } else {
                        const int q = t - nr0 - nr1, c = q & 1, r = q >> 1;
                        const int h = (int)fe1.div(r);
                        y = r - h * e[1];
                        z = h < 3 ? h - 3 : e[2] + h - 3;
                        bx = 4 * c + 3;
                        gx = org[0] + 4 * c;
                        gy = org[1] + y;
                        gz = org[2] + z;
                        if ((zm & 4) && (gz < 0 || gz >= n[2])) flags |= 4;
                        gz = gz < 0 ? gz + n[2] : (gz >= n[2] ? gz - n[2] : gz);
                    }
                    g = (gx - org[0]) + n0 * (gy - org[1]) + n01 * (gz - org[2]);
                    return (bx + 1 + B0 * ((y + 3) + B1 * (z + 3))) | (flags << 16);  // +1: >= 0
                };
                auto fetch = [&](int code, long long g) {
                    if (code & (4 << 16)) return make_float4(0.f, 0.f, 0.f, 0.f);  // zero boundary
                    float4 v = *reinterpret_cast<const float4*>(A0 + g);
                    if (A1) {
                        const float4 d = *reinterpret_cast<const float4*>(A1 + g);
                        v.x += d.x;
                        v.y += d.y;
                        v.z += d.z;
                        v.w += d.w;
                    }
                    return v;
                };
                auto store = [&](int code, const float4& v) {
                    const int b = (code & 0xFFFF) - 1;
                    if (!(code & (1 << 16))) put(b, v.x);
                    put(b + 1, v.y);
                    put(b + 2, v.z);
                    if (!(code & (2 << 16))) put(b + 3, v.w);
                };
                // at most 3 chunks per thread: two in flight, then the third
                {
                    const int t0 = tid, t1 = tid + SG_NT3;
                    long long g0 = 0, g1 = 0;
                    const int c0 = t0 < ntask ? chunk(t0, g0) : -1;
                    const int c1 = t1 < ntask ? chunk(t1, g1) : -1;
                    float4 v0, v1;
                    if (c0 >= 0) v0 = fetch(c0, g0);
                    if (c1 >= 0) v1 = fetch(c1, g1);
                    if (c0 >= 0) store(c0, v0);
                    if (c1 >= 0) store(c1, v1);
                }
                for (int t = tid + 2 * SG_NT3; t < ntask; t += SG_NT3) {
                    long long g;
                    const int c = chunk(t, g);
                    store(c, fetch(c, g));
                }
            }
        }
        constexpr int M0 = (14 * 64 + SG_NT3 - 1) / SG_NT3, M1 = (8 * 6 * 8 + SG_NT3 - 1) / SG_NT3;
        constexpr int MT = M0 + 2 * M1;
        T val[MT];
        int bid[MT];
        if (!vec) {
            const int nv0 = R0 * e[1] * e[2];
#pragma unroll
            for (int j = 0; j < M0; ++j) {
                const int q = tid + j * SG_NT3;
                bid[j] = -1;
                if (q < nv0) {
                    const int r = (int)fR0.div(q), x = q - r * R0;
                    const int z = (int)fe1.div(r), y = r - z * e[1];
                    int gx = org[0] + x - 3;
                    const bool zb = (zm & 1) && (gx < 0 || gx >= n[0]);  // zero boundary value
                    if (gx < 0) gx += n[0];
                    else if (gx >= n[0]) gx -= n[0];
                    bid[j] = x + B0 * ((y + 3) + B1 * (z + 3));
                    val[j] = zb ? T(0) : io.load((gx - org[0]) + n0 * y + n01 * z);
                }
            }
            const int n1 = e[0] * 6 * e[2];
#pragma unroll
            for (int j = 0; j < M1; ++j) {
                const int q = tid + j * SG_NT3;
                bid[M0 + j] = -1;
                if (q < n1) {
                    const int r = (int)fe0.div(q), x = q - r * e[0];
                    const int z = r / 6, h = r - z * 6;
                    const int y = h < 3 ? h - 3 : e[1] + h - 3;
                    int gy = org[1] + y;
                    const bool zb = (zm & 2) && (gy < 0 || gy >= n[1]);
                    if (gy < 0) gy += n[1];
                    else if (gy >= n[1]) gy -= n[1];
                    bid[M0 + j] = (x + 3) + B0 * ((y + 3) + B1 * (z + 3));
                    val[M0 + j] = zb ? T(0) : io.load(x + n0 * (gy - org[1]) + n01 * z);
                }
            }
            const int n2 = e[0] * e[1] * 6;
#pragma unroll
            for (int j = 0; j < M1; ++j) {
                const int q = tid + j * SG_NT3;
                bid[M0 + M1 + j] = -1;
                if (q < n2) {
                    const int r = (int)fe0.div(q), x = q - r * e[0];
                    const int h = (int)fe1.div(r), y = r - h * e[1];
                    const int z = h < 3 ? h - 3 : e[2] + h - 3;
                    int gz = org[2] + z;
                    const bool zb = (zm & 4) && (gz < 0 || gz >= n[2]);
                    if (gz < 0) gz += n[2];
                    else if (gz >= n[2]) gz -= n[2];
                    bid[M0 + M1 + j] = (x + 3) + B0 * ((y + 3) + B1 * (z + 3));
                    val[M0 + M1 + j] = zb ? T(0) : io.load(x + n0 * y + n01 * (gz - org[2]));
                }
            }
#pragma unroll
            for (int j = 0; j < MT; ++j)
                if (bid[j] >= 0) put(bid[j], val[j]);
        }
        __syncthreads();

        // ---- 2) one line per thread: sweep the interfaces, store the flux differences
        const int L0 = e[1] * e[2], L1 = e[0] * e[2], L2 = e[0] * e[1];
        for (int task = tid; task < L0 + L1 + L2; task += SG_NT3) {
            int k, b0, S, line;
            if (task < L0) {
                k = 0;
                const int z = (int)fe1.div(task), y = task - z * e[1];
                b0 = B0 * ((y + 3) + B1 * (z + 3));
                S = 1;
                line = task;
            } else if (task < L0 + L1) {
                k = 1;
                const int q = task - L0;
                const int z = (int)fe0.div(q), x = q - z * e[0];
                b0 = (x + 3) + B0 * B1 * (z + 3);
                S = B0;
                line = q;
            } else {
                k = 2;
                const int q = task - L0 - L1;
                const int y = (int)fe0.div(q), x = q - y * e[0];
                b0 = (x + 3) + B0 * (y + 3);
                S = B0 * B1;
                line = q;
            }
            const int ek = e[k];
            const T rdx = grid_rdx<T>(G, k);
            const T ak = k == 0 ? adv[0] : (k == 1 ? adv[1] : adv[2]);
            const T alpha = burgers ? alpha_b : (ak < T(0) ? -ak : ak);
            // values of f^+ / f^- at box coordinate j along the line
            auto fplus = [&](int j) -> T {
                if (burgers) return bp[b0 + j * S];
                T fp, fm;
                if constexpr (sizeof(T) == 8) Weno<double>::split(bp[b0 + j * S], alpha, ak, 0, fp, fm);
                else {
                    fp = (T)0.5 * (ak + alpha) * bp[b0 + j * S];
                }
                return fp;
            };
            auto fminus = [&](int j) -> T {
                if (burgers) return bm[b0 + j * S];
                T fp, fm;
                if constexpr (sizeof(T) == 8) Weno<double>::split(bp[b0 + j * S], alpha, ak, 0, fp, fm);
                else {
                    fm = (T)0.5 * (ak - alpha) * bp[b0 + j * S];
                }
                return fm;
            };
            SweepSide<T> Pw, Mw;
            // interface 0 (between local points -1 and 0): f^+ at box 0..4, f^- mirrored at box 5..1
            Pw.init(fplus(0), fplus(1), fplus(2), fplus(3), fplus(4), eps4);
            Mw.init(fminus(5), fminus(4), fminus(3), fminus(2), fminus(1), eps4);
            T* D = Dk + k * SG_DK_AXIS + 9 * line;
            T Fprev = sweep_flux(Pw, Mw, ph);
            // ek <= 8: fully unrolled, so the window shifts are register renames, not moves
#pragma unroll
            for (int i = 1; i <= 8; ++i) {
                if (i > ek) break;
                Pw.push_back(fplus(i + 4), eps4);
                Mw.push_front(fminus(i + 5), eps4);
                const T F = sweep_flux(Pw, Mw, ph);
                D[i - 1] = (F - Fprev) * rdx;
                Fprev = F;
            }
        }
        __syncthreads();

        // ---- 3) L = ((0 - D_0) - D_1) - D_2, stage update, alpha of the result
        T mx = T(0);
        bool bad = false;
        bool vec_upd = false;
        if constexpr (sizeof(T) == 4) vec_upd = vec && io.aligned16();
        if constexpr (sizeof(T) == 4) {
            if (vec_upd) {  // four consecutive x points per thread, 16-byte loads and stores
                const int ngrp = 2 * e[1] * e[2];
                for (int t = tid; t < ngrp; t += SG_NT3) {
                    const int c0 = 4 * (t & 1), r = t >> 1;
                    const int c2 = (int)fe1.div(r), c1 = r - c2 * e[1];
                    float L[4];
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        float a = 0.f;
                        a = a - Dk[9 * (c1 + e[1] * c2) + c0 + l];
                        a = a - Dk[SG_DK_AXIS + 9 * (c0 + l + e[0] * c2) + c1];
                        a = a - Dk[2 * SG_DK_AXIS + 9 * (c0 + l + e[0] * c1) + c2];
                        L[l] = a;
                    }
                    const float4 o = io.update4(c0 + n0 * c1 + n01 * c2, L, dt);
                    const float oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        if (!sg_isfinite(oo[l])) bad = true;
                        mx = sg_max(mx, sg_abs(oo[l]));
                    }
                }
            }
        }
        for (int p = vec_upd ? P : tid; p < P; p += SG_NT3) {
            const int r = (int)fe0.div(p), c0 = p - r * e[0];
            const int c2 = (int)fe1.div(r), c1 = r - c2 * e[1];
            T L = T(0);
            L = L - Dk[9 * (c1 + e[1] * c2) + c0];
            L = L - Dk[SG_DK_AXIS + 9 * (c0 + e[0] * c2) + c1];
            L = L - Dk[2 * SG_DK_AXIS + 9 * (c0 + e[0] * c1) + c2];
            const T o = io.update(c0 + n0 * c1 + n01 * c2, L, dt);
            if (!sg_isfinite(o)) bad = true;
            mx = sg_max(mx, sg_abs(o));
        }
        // no barrier here: the next tile writes the box only after this tile's sweep barrier
        // (the box is not read in the update) and Dk only after its own gather barrier
        stage_epilogue_warp(A, w, G, it, mx, bad);
    }
}
