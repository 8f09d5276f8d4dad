// sg_sweep2.cuh -- the d = 3 FP32 stage kernel with two grid lines per thread.
//
// The same tile, gather, flux differences, stage update and epilogue as sg_stage_sweep3_kernel
// (Section 2.1, Eqs. 2-7, and the Shu-Osher stage), but in the sweep phase each thread carries
// two lines of the same axis of the tile: both have the same length, so they share every
// branch, and each WENO5 / Lax-Friedrichs operation of the sweep is one packed f32x2
// instruction for the two lines.  A block of SG_NT3H = 96 threads holds the 96 line pairs of an
// 8 x 8 x 8 tile (3 axes x 64 lines / 2); the gather and the update loop over the tile with
// that many threads.  The box holds the stencil input u only (one array, 15 x 14 x 14 floats for
// a full tile): the sweep forms the Lax-Friedrichs split of each value it reads (for Burgers the
// same operations as Weno<float>::split_burgers), carrying the last value read into the next
// interface, so that a block needs ~19 KB of shared memory and leaves room for a large L1.
#pragma once
#include "sg_stage.cuh"

#define SG_NT3H 96

// weno_scale3 for two lanes: the scale per lane, the multiplications packed
__device__ __forceinline__ void weno_scale3x2(float2& e0, float2& e1, float2& e2) {
    const float mx = sg_min3(e0.x, e1.x, e2.x), my = sg_min3(e0.y, e1.y, e2.y);
    const float2 sc = make_float2(__uint_as_float(0x7f000000u - (__float_as_uint(mx) & 0x7f800000u)),
                                  __uint_as_float(0x7f000000u - (__float_as_uint(my) & 0x7f800000u)));
    e0 = sg_mul2(e0, sc);
    e1 = sg_mul2(e1, sc);
    e2 = sg_mul2(e2, sc);
    e0 = make_float2(fminf(e0.x, 0x1p20f), fminf(e0.y, 0x1p20f));
    e1 = make_float2(fminf(e1.x, 0x1p20f), fminf(e1.y, 0x1p20f));
    e2 = make_float2(fminf(e2.x, 0x1p20f), fminf(e2.y, 0x1p20f));
}

// SweepSide<float> for two lines: lane x is one line, lane y the other; the same operations
// lane by lane (the rescaling of the smoothness terms per lane).
struct SweepSide2 {
    float2 w0, w1, c, w3, w4;
    float2 d1, d2, d3, d4;
    float2 T0, T1, T2;  // (13/3) t^2 + 4 eps of the three second differences
    __device__ __forceinline__ static float2 tterm(float2 t, float2 ep) {
        return sg_fma2(sg_mul2(sg_f2(13.f / 3.f), t), t, ep);
    }
    __device__ __forceinline__ void init(float2 a, float2 b, float2 cc, float2 d, float2 e, float2 ep) {
        w0 = a; w1 = b; c = cc; w3 = d; w4 = e;
        d1 = sg_sub2(b, a); d2 = sg_sub2(cc, b); d3 = sg_sub2(d, cc); d4 = sg_sub2(e, d);
        T0 = tterm(sg_sub2(d2, d1), ep);
        T1 = tterm(sg_sub2(d3, d2), ep);
        T2 = tterm(sg_sub2(d4, d3), ep);
    }
    __device__ __forceinline__ void push_back(float2 v, float2 ep) {
        w0 = w1; w1 = c; c = w3; w3 = w4;
        d1 = d2; d2 = d3; d3 = d4; d4 = sg_sub2(v, w4);
        w4 = v;
        T0 = T1; T1 = T2;
        T2 = tterm(sg_sub2(d4, d3), ep);
    }
    __device__ __forceinline__ void push_front(float2 v, float2 ep) {
        w4 = w3; w3 = c; c = w1; w1 = w0;
        d4 = d3; d3 = d2; d2 = d1; d1 = sg_sub2(w0, v);
        w0 = v;
        T2 = T1; T1 = T0;
        T0 = tterm(sg_sub2(d2, d1), ep);
    }
    // numerator and denominator of 6 (fhat - c): with s_r as in SweepSide<float>, the candidate
    // differences times 6 are P_0 = 2 s_0 - d_2, P_1 = s_1 + d_3, P_2 = s_2 + d_3, and the linear
    // weights times 10 are (1, 6, 3): num = E_1 (E_2 P_0 + 3 E_0 P_2) + 6 E_0 E_2 P_1,
    // den = E_1 (E_2 + 3 E_0) + 6 E_0 E_2
    __device__ __forceinline__ void value(int linear, float2& num, float2& den) const {
        const float2 k3 = sg_f2(3.f);
        const float2 s0 = sg_fma2(k3, d2, sg_neg2(d1)), s1 = sg_add2(d2, d3);
        const float2 s2 = sg_fma2(k3, d3, sg_neg2(d4));
        const float2 P0 = sg_fma2(sg_f2(2.f), s0, sg_neg2(d2));
        const float2 P1 = sg_add2(s1, d3), P2 = sg_add2(s2, d3);
        float2 E0 = sg_f2(1.f), E1 = sg_f2(1.f), E2 = sg_f2(1.f);
        if (!linear) {
            float2 e0 = sg_fma2(s0, s0, T0);
            float2 e1 = sg_fma2(s1, s1, T1);
            float2 e2 = sg_fma2(s2, s2, T2);
            weno_scale3x2(e0, e1, e2);
            E0 = sg_mul2(e0, e0);
            E1 = sg_mul2(e1, e1);
            E2 = sg_mul2(e2, e2);
        }
        const float2 X6 = sg_mul2(sg_f2(6.f), sg_mul2(E0, E2));
        num = sg_fma2(E1, sg_fma2(E2, P0, sg_mul2(k3, sg_mul2(E0, P2))), sg_mul2(X6, P1));
        den = sg_fma2(E1, sg_fma2(k3, E0, E2), X6);
    }
};

// fhat = fhat^+ + fhat^- of both lines: c^+ + c^- + (1/6) (num^+ / den^+ + num^- / den^-) (each
// den in [10, 10 2^80], normal: the approximate reciprocal is within about an ulp)
__device__ __forceinline__ float2 sweep_flux2(const SweepSide2& P, const SweepSide2& M, int linear) {
    float2 np, dp, nm, dm;
    P.value(linear, np, dp);
    M.value(linear, nm, dm);
    const float2 rp = make_float2(sg_rcp(dp.x), sg_rcp(dp.y));
    const float2 rm = make_float2(sg_rcp(dm.x), sg_rcp(dm.y));
    return sg_fma2(sg_f2(1.f / 6.f), sg_fma2(np, rp, sg_mul2(nm, rm)), sg_add2(P.c, M.c));
}

template <bool ZB, int RUN>
__global__ void __launch_bounds__(SG_NT3H, 6) sg_stage_sweep3x2_kernel(const StageArgs A) {
    extern __shared__ __align__(16) unsigned char sg_smem_raw[];
    float* bp = reinterpret_cast<float*>(sg_smem_raw);  // the stencil input u
    float* Dk = bp + A.box_elems;                        // 3 x SG_DK_AXIS flux differences

    const int tid = threadIdx.x;
    const PhysParams& ph = A.phys;
    const bool burgers = ph.pde == 1;
    const float2 ep = sg_f2(sg_eps4<float>(ph.eps));
    const float adv[3] = {(float)ph.adv[0], (float)ph.adv[1], (float)ph.adv[2]};
    const int zm = ZB ? ph.zmask : 0;  // zero boundary per axis (advection / Burgers)

    // Runs of RUN consecutive work items per block (run c = blockIdx.x, + gridDim.x, ...); the
    // host takes RUN = 2 when the launch has at least two items per block: consecutive tiles of
    // a grid row share half of their x-row chunks, which the second finds in L1.  The next work
    // item is read one item early (its load is in flight during this item).
    auto next_item = [&](int i) {
        return ((i - A.item_begin + 1) % RUN) != 0 ? i + 1 : i + 1 + ((int)gridDim.x - 1) * RUN;
    };
    const int it0 = A.item_begin + (int)blockIdx.x * RUN;
    WorkItem wn;
    if (it0 < A.item_end) wn = A.items[it0];
    for (int it = it0; it < A.item_end; it = next_item(it)) {
        const WorkItem w = wn;
        if (next_item(it) < A.item_end) wn = A.items[next_item(it)];
        const GridDesc* G = A.grids + w.grid;
        const InstState* S = A.inst + G->inst;
        if (!S->active) continue;  // uniform: the state is not written during this kernel
        const float dt = inst_dt<float>(S);
        StageIO<float> io;
        io.setup(G, A.stage, stage_parity<float>(S));

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
        // 32-bit offsets from the tile's first point (a grid holds fewer than 2^31 points)
        const int n0 = n[0], n01 = n[0] * n[1];
        io.shift(org[0] + (long long)n0 * org[1] + (long long)n01 * org[2]);
        const int P = e[0] * e[1] * e[2];
        const int R0 = e[0] + 6;  // valid row length along x
        const int B0 = R0 | 1;    // odd row stride
        const int B1 = e[1] + 6;
        const float alpha_b = alpha_dec<float>(A.alpha[w.grid * 3 + A.stage]);
        FDiv fR0, fe0, fe1;
        fR0.init(R0);
        fe0.init(e[0]);
        fe1.init(e[1]);

        auto put = [&](int bidx, float v) { bp[bidx] = v; };  // the stencil input u
        // ---- 1) gather the padded box (as sg_stage_sweep3_kernel: float4 chunks where the tile
        // is 8 wide at a 4-aligned x origin of a row length divisible by 4 on 16-byte aligned
        // arrays, single values otherwise; zero chunks beyond the ends of zero-boundary axes)
        const float* A0 = nullptr;
        const float* A1 = nullptr;
        io.stencil_src(A0, A1);
        const unsigned long long align = reinterpret_cast<unsigned long long>(A0) | reinterpret_cast<unsigned long long>(A1);
        const bool vec = e[0] == 8 && (org[0] & 3) == 0 && (n[0] & 3) == 0 && (align & 15) == 0;
        if (vec) {
            const int nr0 = e[1] * e[2] * 4, nr1 = 12 * e[2], nr2 = 12 * e[1];
            const int ntask = nr0 + nr1 + nr2;
            auto chunk = [&](int t, int& g) -> int {
                int gx, gy, gz, bx, y, z, flags = 0;
                if (t < nr0) {
                    const int c = t & 3, r = t >> 2;
                    z = (int)fe1.div(r);
                    y = r - z * e[1];
                    bx = 4 * c - 1;
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
                return (bx + 1 + B0 * ((y + 3) + B1 * (z + 3))) | (flags << 16);
            };
            auto fetch = [&](int code, int g) {
                if (code & (4 << 16)) return make_float4(0.f, 0.f, 0.f, 0.f);
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
            // up to five chunks per thread (448 for a full tile), three loads in flight at a time
            constexpr int NU = 3;
            for (int t0 = tid; t0 < ntask; t0 += NU * SG_NT3H) {
                int gg[NU], cc[NU];
                float4 vv[NU];
#pragma unroll
                for (int u = 0; u < NU; ++u) {
                    const int t = t0 + u * SG_NT3H;
                    cc[u] = t < ntask ? chunk(t, gg[u]) : -1;
                }
#pragma unroll
                for (int u = 0; u < NU; ++u)
                    if (cc[u] >= 0) vv[u] = fetch(cc[u], gg[u]);
#pragma unroll
                for (int u = 0; u < NU; ++u)
                    if (cc[u] >= 0) store(cc[u], vv[u]);
            }
        } else {
            constexpr int M0 = (14 * 64 + SG_NT3H - 1) / SG_NT3H, M1 = (8 * 6 * 8 + SG_NT3H - 1) / SG_NT3H;
            const int nv0 = R0 * e[1] * e[2];
#pragma unroll 2
            for (int j = 0; j < M0; ++j) {
                const int q = tid + j * SG_NT3H;
                if (q < nv0) {
                    const int r = (int)fR0.div(q), x = q - r * R0;
                    const int z = (int)fe1.div(r), y = r - z * e[1];
                    int gx = org[0] + x - 3;
                    const bool zb = (zm & 1) && (gx < 0 || gx >= n[0]);
                    if (gx < 0) gx += n[0];
                    else if (gx >= n[0]) gx -= n[0];
                    put(x + B0 * ((y + 3) + B1 * (z + 3)), zb ? 0.f : io.load((gx - org[0]) + n0 * y + n01 * z));
                }
            }
            const int n1 = e[0] * 6 * e[2];
#pragma unroll 2
            for (int j = 0; j < M1; ++j) {
                const int q = tid + j * SG_NT3H;
                if (q < n1) {
                    const int r = (int)fe0.div(q), x = q - r * e[0];
                    const int z = r / 6, h = r - z * 6;
                    const int y = h < 3 ? h - 3 : e[1] + h - 3;
                    int gy = org[1] + y;
                    const bool zb = (zm & 2) && (gy < 0 || gy >= n[1]);
                    if (gy < 0) gy += n[1];
                    else if (gy >= n[1]) gy -= n[1];
                    put((x + 3) + B0 * ((y + 3) + B1 * (z + 3)), zb ? 0.f : io.load(x + n0 * (gy - org[1]) + n01 * z));
                }
            }
            const int n2 = e[0] * e[1] * 6;
#pragma unroll 2
            for (int j = 0; j < M1; ++j) {
                const int q = tid + j * SG_NT3H;
                if (q < n2) {
                    const int r = (int)fe0.div(q), x = q - r * e[0];
                    const int h = (int)fe1.div(r), y = r - h * e[1];
                    const int z = h < 3 ? h - 3 : e[2] + h - 3;
                    int gz = org[2] + z;
                    const bool zb = (zm & 4) && (gz < 0 || gz >= n[2]);
                    if (gz < 0) gz += n[2];
                    else if (gz >= n[2]) gz -= n[2];
                    put((x + 3) + B0 * ((y + 3) + B1 * (z + 3)), zb ? 0.f : io.load(x + n0 * y + n01 * (gz - org[2])));
                }
            }
        }
        __syncthreads();

        // ---- 2) two lines of one axis per thread: lines p and p + H of the axis's L lines
        // (H = ceil(L / 2); with L odd the last thread's second line repeats its first and is
        // not stored)
        {
            const int L0 = e[1] * e[2], L1 = e[0] * e[2], L2 = e[0] * e[1];
            const int H0 = (L0 + 1) >> 1, H1 = (L1 + 1) >> 1, H2 = (L2 + 1) >> 1;
            // box base of line l of axis k
            auto base = [&](int k, int l) -> int {
                if (k == 0) {
                    const int z = (int)fe1.div(l), y = l - z * e[1];
                    return B0 * ((y + 3) + B1 * (z + 3));
                }
                if (k == 1) {
                    const int z = (int)fe0.div(l), x = l - z * e[0];
                    return (x + 3) + B0 * B1 * (z + 3);
                }
                const int y = (int)fe0.div(l), x = l - y * e[0];
                return (x + 3) + B0 * (y + 3);
            };
            for (int task = tid; task < H0 + H1 + H2; task += SG_NT3H) {
                int k, p, L, H, S;
                if (task < H0) {
                    k = 0, p = task, L = L0, H = H0, S = 1;
                } else if (task < H0 + H1) {
                    k = 1, p = task - H0, L = L1, H = H1, S = B0;
                } else {
                    k = 2, p = task - H0 - H1, L = L2, H = H2, S = B0 * B1;
                }
                const int la = p;
                const bool second = p + H < L;
                const int lb = second ? p + H : p;
                const int ba = base(k, la), bb = base(k, lb);
                const int ek = e[k];
                const float rdx = grid_rdx<float>(G, k);
                const float ak = k == 0 ? adv[0] : (k == 1 ? adv[1] : adv[2]);
                const float alpha = burgers ? alpha_b : (ak < 0.f ? -ak : ak);
                const float cp = 0.5f * (ak + alpha), cm = 0.5f * (ak - alpha);
                // u of both lines at box coordinate j along them, and its LF split (Burgers:
                // f^+- = u (u/4 +- alpha/2), Weno<float>::split_burgers lane by lane)
                auto uval = [&](int j) -> float2 { return make_float2(bp[ba + j * S], bp[bb + j * S]); };
                const float2 ha2 = sg_f2(0.5f * alpha);
                auto fplus = [&](float2 v) -> float2 {
                    return burgers ? sg_mul2(v, sg_fma2(sg_f2(0.25f), v, ha2)) : sg_mul2(sg_f2(cp), v);
                };
                auto fminus = [&](float2 v) -> float2 {
                    return burgers ? sg_mul2(v, sg_fma2(sg_f2(0.25f), v, sg_neg2(ha2))) : sg_mul2(sg_f2(cm), v);
                };
                SweepSide2 Pw, Mw;
                // interface 0 (between local points -1 and 0): f^+ at box 0..4, f^- mirrored at box 5..1
                const float2 u0 = uval(0), u1 = uval(1), u2 = uval(2), u3 = uval(3), u4 = uval(4);
                float2 uc = uval(5);  // u at box i + 4 of interface i
                Pw.init(fplus(u0), fplus(u1), fplus(u2), fplus(u3), fplus(u4), ep);
                Mw.init(fminus(uc), fminus(u4), fminus(u3), fminus(u2), fminus(u1), ep);
                float* Da = Dk + k * SG_DK_AXIS + 9 * la;
                float* Db = Dk + k * SG_DK_AXIS + 9 * lb;
                float2 Fprev = sweep_flux2(Pw, Mw, ph.scheme);
                const float2 r2 = sg_f2(rdx);
#pragma unroll
                for (int i = 1; i <= 8; ++i) {
                    if (i > ek) break;
                    const float2 un = uval(i + 5);
                    Pw.push_back(fplus(uc), ep);
                    Mw.push_front(fminus(un), ep);
                    uc = un;
                    const float2 F = sweep_flux2(Pw, Mw, ph.scheme);
                    const float2 D = sg_mul2(sg_sub2(F, Fprev), r2);
                    Da[i - 1] = D.x;
                    if (second) Db[i - 1] = D.y;
                    Fprev = F;
                }
            }
        }
        __syncthreads();

        // ---- 3) L = ((0 - D_0) - D_1) - D_2, stage update, alpha of the result
        float mx = 0.f;
        bool bad = false;
        const bool vec_upd = vec && io.aligned16();
        if (vec_upd) {  // four consecutive x points per thread, 16-byte loads and stores
            const int ngrp = 2 * e[1] * e[2];
            for (int t = tid; t < ngrp; t += SG_NT3H) {
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
                    mx = fmaxf(mx, fabsf(oo[l]));
                }
            }
        } else {
            for (int p = tid; p < P; p += SG_NT3H) {
                const int r = (int)fe0.div(p), c0 = p - r * e[0];
                const int c2 = (int)fe1.div(r), c1 = r - c2 * e[1];
                float L = 0.f;
                L = L - Dk[9 * (c1 + e[1] * c2) + c0];
                L = L - Dk[SG_DK_AXIS + 9 * (c0 + e[0] * c2) + c1];
                L = L - Dk[2 * SG_DK_AXIS + 9 * (c0 + e[0] * c1) + c2];
                const float o = io.update(c0 + n0 * c1 + n01 * c2, L, dt);
                if (!sg_isfinite(o)) bad = true;
                mx = fmaxf(mx, fabsf(o));
            }
        }
        // no barrier here: the next tile writes the box only after this tile's sweep barrier
        // (the box is not read in the update) and Dk only after its own gather barrier
        stage_epilogue_warp(A, w, G, it, mx, bad);
    }
}
