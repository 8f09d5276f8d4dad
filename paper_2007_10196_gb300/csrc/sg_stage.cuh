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
    __device__ __forceinline__ float load(long long g) const {
        if (stage == 0) return U[g];
        if (stage == 1) return U[g] + Ub[g];
        return U[g] + D2[g];
    }
    __device__ __forceinline__ float update(long long g, float L, double dt) const {
        const float d = (float)dt * L;
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
};

template <class T>
__device__ __forceinline__ int stage_parity(const InstState* S) {
    return (int)((S->steps - S->step0) & 1);
}

// Epilogue shared by both kernels: non-finite flag, alpha slot of the next stage, and the
// clearing of the slot two stages ahead (by the grid's first item).
__device__ __forceinline__ void stage_epilogue(const StageArgs& A, const WorkItem& w, const GridDesc* G, int it,
                                               double mx, bool bad, double* red) {
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(A.flags + SG_FLAG_NONFINITE, 1);
    if (A.phys.pde == 1) {
        const double m = block_max(mx, red);
        if (threadIdx.x == 0) atomicMax(A.alpha + w.grid * 3 + (A.stage + 1) % 3, dbits(m));
    }
    if (threadIdx.x == 0 && it == G->first_item) A.alpha[w.grid * 3 + (A.stage + 2) % 3] = 0ull;
}

// ------------------------------------------------------------------------------------
// d <= 3: padded-box kernel.  Per tile: one load of the tile with a 3-point halo on each face
// (periodic wrap), the LF split computed once per loaded value (Burgers: the split is the
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
    __shared__ double red[SG_NT / 32];

    const int tid = threadIdx.x;
    const PhysParams& ph = A.phys;
    const bool burgers = ph.pde == 1;
    const T eps12 = (T)(12.0 * ph.eps);

    for (int it = A.item_begin + blockIdx.x; it < A.item_end; it += gridDim.x) {
        const WorkItem w = A.items[it];
        const GridDesc* G = A.grids + w.grid;
        const InstState* S = A.inst + G->inst;
        if (!S->active) continue;  // uniform: the state is not written during this kernel
        const double dt = S->dt;
        StageIO<T> io;
        io.setup(G, A.stage, stage_parity<T>(S));

        int org[3] = {0, 0, 0}, e[3] = {1, 1, 1}, n[3] = {1, 1, 1};
        long long gs[3] = {1, 0, 0};
        {
            unsigned tt = (unsigned)w.tile;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const unsigned nt = (unsigned)G->nt[k];
                const unsigned tc = tt % nt;
                tt /= nt;
                n[k] = G->n[k];
                org[k] = (int)tc * G->te[k];
                e[k] = min(G->te[k], n[k] - org[k]);
            }
            if (D >= 2) gs[1] = n[0];
            if (D >= 3) gs[2] = (long long)n[0] * n[1];
        }
        const int P = e[0] * e[1] * e[2];
        const int B0 = e[0] + 6, B1 = D >= 2 ? e[1] + 6 : 1;
        const T alpha_b = (T)bitsd(A.alpha[w.grid * 3 + A.stage]);
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
                if (gx < 0) gx += n[0];
                else if (gx >= n[0]) gx -= n[0];
                const long long g = gx + gs[1] * (org[1] + y) + gs[2] * (org[2] + z);
                put(x + B0 * ((y + (D >= 2 ? 3 : 0)) + B1 * (z + (D >= 3 ? 3 : 0))), g);
            }
            if (D >= 2) {
                const int n1 = e[0] * 6 * e[2];  // axis-1 halos
                for (int q = tid; q < n1; q += SG_NT) {
                    const int r = (int)fe0.div((unsigned)q);
                    const int x = q - r * e[0];
                    const int z = r / 6, h = r - z * 6;
                    const int y = h < 3 ? h - 3 : e[1] + h - 3;
                    int gy = org[1] + y;
                    if (gy < 0) gy += n[1];
                    else if (gy >= n[1]) gy -= n[1];
                    const long long g = (org[0] + x) + gs[1] * gy + gs[2] * (org[2] + z);
                    put((x + 3) + B0 * ((y + 3) + B1 * (z + (D >= 3 ? 3 : 0))), g);
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
                    if (gz < 0) gz += n[2];
                    else if (gz >= n[2]) gz -= n[2];
                    const long long g = (org[0] + x) + gs[1] * (org[1] + y) + gs[2] * gz;
                    put((x + 3) + B0 * ((y + 3) + B1 * (z + 3)), g);
                }
            }
        }
        __syncthreads();

        // ---- 2) every interface flux of every axis, once
        const int NF0 = (e[0] + 1) * e[1] * e[2];
        const int NF1 = D >= 2 ? e[0] * (e[1] + 1) * e[2] : 0;
        const int NF2 = D >= 3 ? e[0] * e[1] * (e[2] + 1) : 0;
        const int NF = NF0 + NF1 + NF2;
        for (int q = tid; q < NF; q += SG_NT) {
            int b, Sx;
            double ak;
            if (q < NF0) {
                Sx = 1;
                ak = ph.adv[0];
                const int r = (int)fp0.div((unsigned)q);
                const int i = q - r * (e[0] + 1);
                int y = 0, z = 0;
                if (D >= 2) {
                    z = (int)fe1.div((unsigned)r);
                    y = r - z * e[1];
                }
                b = i + B0 * ((y + (D >= 2 ? 3 : 0)) + B1 * (z + (D >= 3 ? 3 : 0)));
            } else if (D >= 2 && q < NF0 + NF1) {
                Sx = B0;
                ak = ph.adv[1];
                const int qq = q - NF0;
                const int r = (int)fe0.div((unsigned)qq);
                const int x = qq - r * e[0];
                const int z = (int)fp1.div((unsigned)r);
                const int i = r - z * (e[1] + 1);
                b = (x + 3) + B0 * (i + B1 * (z + (D >= 3 ? 3 : 0)));
            } else {
                Sx = B0 * B1;
                ak = ph.adv[2];
                const int qq = q - NF0 - NF1;
                const int r = (int)fe0.div((unsigned)qq);
                const int x = qq - r * e[0];
                const int i = (int)fe1.div((unsigned)r);
                const int y = r - i * e[1];
                b = (x + 3) + B0 * ((y + 3) + B1 * i);
            }
            T F;
            if constexpr (sizeof(T) == 8) {
                if (burgers) {
                    F = Weno<double>::interface_split((const double*)bp + b, (const double*)bm + b, Sx, ph);
                } else {
                    const double a = ak;
                    F = Weno<double>::interface((const double*)bp + b, Sx, a < 0.0 ? -a : a, a, ph);
                }
            } else {
                if (burgers) {
                    F = Weno<float>::interface_split((const float*)bp + b, (const float*)bm + b, Sx, eps12, ph.scheme);
                } else {
                    const float a = (float)ak;
                    F = Weno<float>::interface((const float*)bp + b, Sx, fabsf(a), a, ph, eps12);
                }
            }
            fb[q] = F;
        }
        __syncthreads();

        // ---- 3) flux difference, stage update, alpha of the result
        double mx = 0.0;
        bool bad = false;
        const T r0 = (T)G->rdx[0], r1 = (T)G->rdx[1], r2 = (T)G->rdx[2];
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
            mx = fmax(mx, (double)sg_abs(o));
        }
        stage_epilogue(A, w, G, it, mx, bad, red);
        __syncthreads();  // the next tile overwrites the shared arrays
    }
}

// ------------------------------------------------------------------------------------
// d >= 4 (and any d): line-buffer kernel.  For each axis k the tile's lines along k plus a
// 3-point periodic halo are staged in shared memory, every interface flux of the tile along
// k is computed once, and each thread subtracts (F_{i+1/2} - F_{i-1/2}) / h_k for its points.
// ------------------------------------------------------------------------------------
template <int PPT>
struct LineSmem {
    // worst case over tile shapes with P <= SG_NT*PPT points and extents >= 1:
    // line buffer (ek + 7) * P / ek <= 8 P; flux buffer (ek + 2) * P / ek <= 3 P
    static constexpr int P = SG_NT * PPT;
    static constexpr int LB = 8 * P;
    static constexpr int FB = 3 * P;
};

template <class T, int D, int PPT>
__global__ void __launch_bounds__(SG_NT) sg_stage_line_kernel(const StageArgs A) {
    extern __shared__ __align__(16) unsigned char sg_smem_raw[];
    T* lb = reinterpret_cast<T*>(sg_smem_raw);
    T* fb = lb + LineSmem<PPT>::LB;
    __shared__ double red[SG_NT / 32];

    const int tid = threadIdx.x;
    const PhysParams& ph = A.phys;

    for (int it = A.item_begin + blockIdx.x; it < A.item_end; it += gridDim.x) {
        const WorkItem w = A.items[it];
        const GridDesc* G = A.grids + w.grid;
        const InstState* S = A.inst + G->inst;
        if (!S->active) continue;
        const double dt = S->dt;
        StageIO<T> io;
        io.setup(G, A.stage, stage_parity<T>(S));

        int org[D], ext[D], nn[D];
        long long gstr[D];
        FDiv fd[D];
        int P = 1;
        {
            unsigned tt = (unsigned)w.tile;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const unsigned nt = (unsigned)G->nt[k];
                const unsigned tc = tt % nt;
                tt /= nt;
                nn[k] = G->n[k];
                org[k] = (int)tc * G->te[k];
                ext[k] = min(G->te[k], nn[k] - org[k]);
                gstr[k] = k == 0 ? 1LL : gstr[k - 1] * (long long)nn[k - 1];
                fd[k].init((unsigned)ext[k]);
                P *= ext[k];
            }
        }
        const double alpha_slot = bitsd(A.alpha[w.grid * 3 + A.stage]);

        int cp[PPT][D];
        bool own[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const int p = tid + q * SG_NT;
            own[q] = p < P;
            unsigned r = (unsigned)(own[q] ? p : 0);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const unsigned qq = fd[k].div(r);
                cp[q][k] = (int)(r - qq * (unsigned)ext[k]);
                r = qq;
            }
        }
        T acc[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) acc[q] = T(0);

#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int ek = ext[k];
            const int lines = P / ek;
            const int ls = (ek + 6) | 1;  // odd strides avoid bank conflicts
            const int fs = (ek + 1) | 1;
            const T alpha = ph.pde == 1 ? (T)alpha_slot : (T)sg_abs(ph.adv[k]);
            const T ak = (T)ph.adv[k];
            FDiv fl, fr, ff;
            fl.init((unsigned)lines);
            fr.init((unsigned)(ek + 6));
            ff.init((unsigned)(ek + 1));

            const int NL = lines * (ek + 6);
            for (int e = tid; e < NL; e += SG_NT) {
                int line, i;
                if (k == 0) {
                    line = (int)fr.div((unsigned)e);
                    i = e - line * (ek + 6);
                } else {
                    i = (int)fl.div((unsigned)e);
                    line = e - i * lines;
                }
                long long g = 0;
                unsigned rem = (unsigned)line;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    if (j == k) continue;
                    const unsigned qq = fd[j].div(rem);
                    const int cj = (int)(rem - qq * (unsigned)ext[j]);
                    rem = qq;
                    g += (long long)(org[j] + cj) * gstr[j];
                }
                int ck = org[k] + i - 3;
                if (ck < 0) ck += nn[k];
                else if (ck >= nn[k]) ck -= nn[k];
                g += (long long)ck * gstr[k];
                lb[line * ls + i] = io.load(g);
            }
            __syncthreads();

            const int NF = lines * (ek + 1);
            for (int e = tid; e < NF; e += SG_NT) {
                const int line = (int)ff.div((unsigned)e);
                const int i = e - line * (ek + 1);
                const T* v = lb + line * ls + i;
                if constexpr (sizeof(T) == 8) {
                    fb[line * fs + i] = Weno<double>::interface((const double*)v, 1, (double)alpha, (double)ak, ph);
                } else {
                    fb[line * fs + i] = Weno<float>::interface((const float*)v, 1, (float)alpha, (float)ak, ph,
                                                               (float)(12.0 * ph.eps));
                }
            }
            __syncthreads();

            const T rdx = (T)G->rdx[k];
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                if (!own[q]) continue;
                int line = 0, mul = 1;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    if (j == k) continue;
                    line += cp[q][j] * mul;
                    mul *= ext[j];
                }
                const T* F = fb + line * fs + cp[q][k];
                acc[q] = acc[q] - (F[1] - F[0]) * rdx;
            }
            __syncthreads();
        }

        double mx = 0.0;
        bool bad = false;
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            if (!own[q]) continue;
            long long g = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) g += (long long)(org[k] + cp[q][k]) * gstr[k];
            const T o = io.update(g, acc[q], dt);
            if (!sg_isfinite(o)) bad = true;
            mx = fmax(mx, (double)sg_abs(o));
        }
        stage_epilogue(A, w, G, it, mx, bad, red);
    }
}
