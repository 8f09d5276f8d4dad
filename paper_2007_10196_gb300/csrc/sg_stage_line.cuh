// sg_stage_line.cuh -- the stage kernel for d >= 4 (and d = 2 for the Vlasov-Boltzmann
// model): a sweep over staged lines, built on the stage building blocks of sg_stage.cuh.
#pragma once
#include "sg_stage.cuh"

// ------------------------------------------------------------------------------------
// d >= 4 (and d = 2 for the Vlasov-Boltzmann model): line-sweep kernel over staged lines.
// Per tile and axis k (in the order 0, 1, ...): the tile's lines along k with a 3-point halo at
// each end are staged in shared memory (periodic wrap), four global loads in flight per thread;
// then each thread takes a segment of at most 8 points of one line and slides the five-point
// windows of f^+ and f^- along it (SweepSide, as in the d = 3 sweep kernel), so every interface
// flux is formed once (twice at a segment boundary) from the split values of its stencil, and
// subtracts (F_{i+1/2} - F_{i-1/2}) / h_k from the point's
// accumulator in shared memory: L = ((0 - D_0) - D_1) - ..., the operation order of the FP64
// definition.  Finally each point takes the RK stage update.
// Zero boundary (advection / Burgers, bit k of zmask; every axis of the Vlasov-Boltzmann model):
// halo values beyond the ends of axis k are 0.
// Vlasov-Boltzmann (pde 3, d = 2 d_x): the flux along space axis
// k is v_k u and along velocity axis k is -x_k u, v_k (x_k) the line's node on the partner
// axis; the LF alpha of an axis is the largest |partner node| of the grid; after the flux
// differences each point adds (mu(v) rho(x) - u) / tau (rho from G->ef, mu from G->mu).
// Shared memory: the line buffer (A.box_elems elements: the largest lines x ((e_k + 6) | 1) of
// any axis of any tile), the accumulators (one per tile point) and, per axis, each line's
// offset from the tile origin (one int per tile point at most).  Offsets within a grid are
// 32-bit, relative to the tile origin (grids hold fewer than 2^31 points).
// ------------------------------------------------------------------------------------
template <class T, int D, int PPT>
__global__ void __launch_bounds__(SG_NT, sizeof(T) == 4 ? 4 : 1) sg_stage_line_kernel(const StageArgs A) {
    extern __shared__ __align__(16) unsigned char sg_smem_raw[];
    T* lb = reinterpret_cast<T*>(sg_smem_raw);
    T* accs = lb + A.box_elems;

    const int tid = threadIdx.x;
    const PhysParams& ph = A.phys;
    const T eps4 = sg_eps4<T>(ph.eps);
    const bool burgers = ph.pde == 1;
    const bool vb = ph.pde == 3;
    constexpr int DX = D / 2;  // Vlasov-Boltzmann: space axes 0..DX-1, velocity axes DX..D-1

    for (int it = A.item_begin + blockIdx.x; it < A.item_end; it += gridDim.x) {
        const WorkItem w = A.items[it];
        const GridDesc* G = A.grids + w.grid;
        const InstState* S = A.inst + G->inst;
        if (!S->active) continue;
        const T dt = inst_dt<T>(S);
        StageIO<T> io;
        io.setup(G, A.stage, stage_parity<T>(S));

        int org[D], ext[D], nn[D], tstr[D], gstr[D];
        FDiv fd[D];
        int P = 1;
        {
            int tc[D];
            tile_coords<D>(G, (unsigned)w.tile, tc);
            long long o = 0, st = 1;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                nn[k] = G->n[k];
                org[k] = tc[k] * G->te[k];
                ext[k] = min(G->te[k], nn[k] - org[k]);
                gstr[k] = (int)st;  // < 2^31: the grid holds fewer points
                o += (long long)org[k] * st;
                st *= nn[k];
                tstr[k] = P;
                fd[k].init((unsigned)ext[k]);
                P *= ext[k];
            }
            io.shift(o);  // offsets below are relative to the tile's first point
        }
        int* lbase = reinterpret_cast<int*>(accs + P);  // per-line offsets of the current axis
        const T alpha_slot = alpha_dec<T>(A.alpha[w.grid * 3 + A.stage]);
        const T half_alpha = (T)0.5 * alpha_slot;

#pragma unroll 1
        for (int k = 0; k < D; ++k) {
            // this axis's scalars, selected with compile-time indices (no dynamically indexed arrays)
            int ek = 1, ok = 0, nk = 1, tk = 1, gk = 1;
#pragma unroll
            for (int j = 0; j < D; ++j)
                if (j == k) {
                    ek = ext[j];
                    ok = org[j];
                    nk = nn[j];
                    tk = tstr[j];
                    gk = gstr[j];
                }
            const int lines = P / ek;
            const int ls = (ek + 6) | 1;  // odd stride against bank conflicts
            FDiv fl, fr;
            fl.init((unsigned)lines);
            fr.init((unsigned)(ek + 6));

            // ---- each line's offset from the tile origin (axes j != k), once per line (d >= 4;
            // with one other axis the staging below decomposes the line index itself)
            constexpr bool kLineTable = D >= 4;
            if (kLineTable) {
                for (int line = tid; line < lines; line += SG_NT) {
                    int g = 0;
                    unsigned rem = (unsigned)line;
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        if (j == k) continue;
                        const unsigned qq = fd[j].div(rem);
                        g += (int)(rem - qq * (unsigned)ext[j]) * gstr[j];
                        rem = qq;
                    }
                    lbase[line] = g;
                }
                __syncthreads();
            }

            // ---- stage the lines with their halos: four elements per thread and round,
            // addresses first, then the four loads in flight, then the shared-memory stores
            const int NL = lines * (ek + 6);
            constexpr int RU = 4;
            for (int e0 = tid; e0 < NL; e0 += RU * SG_NT) {
                int dst[RU], src[RU];
                unsigned char kind[RU];  // 0: no element; 1: load; 2: a zero boundary value
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int e = e0 + u * SG_NT;
                    kind[u] = 0;
                    dst[u] = 0;
                    src[u] = 0;
                    if (e >= NL) continue;
                    int line, i;
                    if (k == 0) {
                        line = (int)fr.div((unsigned)e);
                        i = e - line * (ek + 6);
                    } else {
                        i = (int)fl.div((unsigned)e);
                        line = e - i * lines;
                    }
                    dst[u] = line * ls + i;
                    int ck = ok + i - 3;
                    if ((vb || ((ph.zmask >> k) & 1)) && (ck < 0 || ck >= nk)) {  // zero boundary values
                        kind[u] = 2;
                        continue;
                    }
                    if (ck < 0) ck += nk;
                    else if (ck >= nk) ck -= nk;
                    kind[u] = 1;
                    int base = 0;
                    if (kLineTable) {
                        base = lbase[line];
                    } else {
                        unsigned rem = (unsigned)line;
#pragma unroll
                        for (int j = 0; j < D; ++j) {
                            if (j == k) continue;
                            const unsigned qq = fd[j].div(rem);
                            base += (int)(rem - qq * (unsigned)ext[j]) * gstr[j];
                            rem = qq;
                        }
                    }
                    src[u] = base + (ck - ok) * gk;
                }
                T val[RU];
#pragma unroll
                for (int u = 0; u < RU; ++u) val[u] = kind[u] == 1 ? io.load(src[u]) : T(0);
#pragma unroll
                for (int u = 0; u < RU; ++u)
                    if (kind[u]) lb[dst[u]] = val[u];
            }
            __syncthreads();

            // ---- sweep: one line per thread
            const T rdx = grid_rdx<T>(G, k);
            const int pk = k < DX ? k + DX : k - DX;  // Vlasov-Boltzmann partner axis
            T ak = T(0);
#pragma unroll
            for (int j = 0; j < D; ++j)
                if (j == k) ak = (T)ph.adv[j];
            T alpha = burgers ? alpha_slot : sg_abs(ak);
            if (vb) {  // the largest |partner node| of the grid (an end node)
                const T c0 = (T)G->lo[pk], c1 = (T)G->lo[pk] + (T)(G->n[pk] - 1) * (T)G->h[pk];
                alpha = sg_max(sg_abs(c0), sg_abs(c1));
            }
            // segments of at most 8 points, so that long lines (d = 2 tiles) still spread over the
            // block's threads; consecutive threads take consecutive lines.  (Shorter segments to
            // occupy more threads measured slower: each segment sets up its own windows.)
            const int nseg = (ek + 7) >> 3;
            for (int task = tid; task < lines * nseg; task += SG_NT) {
                const int seg = (int)fl.div((unsigned)task), line = task - seg * lines;
                const int i0 = seg << 3, i1 = min(ek, i0 + 8);
                // the line's first point in the tile, and its node on the partner axis
                int pb = 0, cpk = 0;
                unsigned rem = (unsigned)line;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    if (j == k) continue;
                    const unsigned qq = fd[j].div(rem);
                    const int cj = (int)(rem - qq * (unsigned)ext[j]);
                    rem = qq;
                    pb += cj * tstr[j];
                    if (j == pk) cpk = cj + org[j];
                }
                T akl = ak;
                if (vb) {  // v_k along x_k, -x_k along v_k
                    const T c = (T)G->lo[pk] + (T)cpk * (T)G->h[pk];
                    akl = k < DX ? c : -c;
                }
                const T cp = (T)0.5 * (akl + alpha), cm = (T)0.5 * (akl - alpha);
                const T* v = lb + line * ls;
                auto fplus = [&](int j) -> T {
                    if constexpr (sizeof(T) == 8) {
                        double fp, fm;
                        Weno<double>::split(v[j], alpha, akl, ph.pde, fp, fm);
                        return fp;
                    } else {
                        if (burgers) {
                            float fp, fm;
                            Weno<float>::split_burgers(v[j], half_alpha, fp, fm);
                            return fp;
                        }
                        return cp * v[j];
                    }
                };
                auto fminus = [&](int j) -> T {
                    if constexpr (sizeof(T) == 8) {
                        double fp, fm;
                        Weno<double>::split(v[j], alpha, akl, ph.pde, fp, fm);
                        return fm;
                    } else {
                        if (burgers) {
                            float fp, fm;
                            Weno<float>::split_burgers(v[j], half_alpha, fp, fm);
                            return fm;
                        }
                        return cm * v[j];
                    }
                };
                SweepSide<T> Pw, Mw;
                // interface between local points i0-1 and i0 (buffer index = local + 3): f^+ at
                // buffer i0..i0+4, f^- mirrored at i0+5..i0+1
                Pw.init(fplus(i0), fplus(i0 + 1), fplus(i0 + 2), fplus(i0 + 3), fplus(i0 + 4), eps4);
                Mw.init(fminus(i0 + 5), fminus(i0 + 4), fminus(i0 + 3), fminus(i0 + 2), fminus(i0 + 1), eps4);
                T Fprev = sweep_flux(Pw, Mw, ph);
                T* a = accs + pb + i0 * tk;
#pragma unroll 2
                for (int i = i0 + 1; i <= i1; ++i) {
                    Pw.push_back(fplus(i + 4), eps4);
                    Mw.push_front(fminus(i + 5), eps4);
                    const T F = sweep_flux(Pw, Mw, ph);
                    const T Dv = (F - Fprev) * rdx;
                    *a = (k == 0 ? T(0) : *a) - Dv;
                    a += tk;
                    Fprev = F;
                }
            }
            __syncthreads();  // accumulators complete; the line buffer is free for the next axis
        }

        // ---- relaxation (Vlasov-Boltzmann), stage update, alpha of the result
        T mx = T(0);
        bool bad = false;
        const T* rho = (const T*)G->ef;
        const T* mu = (const T*)G->mu;
        const T tau = (T)ph.tau;
        for (int p = tid; p < P; p += SG_NT) {
            unsigned rem = (unsigned)p;
            int g = 0, ix = 0, iv = 0, sv = 1;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const unsigned qq = fd[j].div(rem);
                const int cj = (int)(rem - qq * (unsigned)ext[j]);
                rem = qq;
                g += cj * gstr[j];
                if (vb) {
                    if (j < DX) {
                        ix += (cj + org[j]) * gstr[j];
                    } else {
                        iv += (cj + org[j]) * sv;
                        sv *= nn[j];
                    }
                }
            }
            T L = accs[p];
            if (vb) L = L + (mu[iv] * rho[ix] - io.load(g)) / tau;
            const T o = io.update(g, L, dt);
            if (!sg_isfinite(o)) bad = true;
            mx = sg_max(mx, sg_abs(o));
        }
        // no barrier here: the next tile writes the line buffer (not read in the update) and the
        // accumulators only after its own staging barrier
        stage_epilogue_warp(A, w, G, it, mx, bad);
    }
}
