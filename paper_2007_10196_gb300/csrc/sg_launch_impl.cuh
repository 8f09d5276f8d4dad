// sg_launch_impl.cuh -- definitions of sg::Launch<T>; included by exactly one translation
// unit per precision.
#pragma once
#include <algorithm>

#include "sg_kernels.cuh"
#include "sg_launch.h"

namespace sg {

namespace detail {

// d = 3: the line-sweep kernel (SG_NT3 threads; the points-per-thread choice does not apply);
// d <= 2: the padded-box kernel; d >= 4: the line-buffer kernel.
template <class T, int D, int PPT>
struct StageKernel {
    static constexpr int threads = D == 3 ? SG_NT3 : SG_NT;
    static void* fn() {
        if constexpr (D == 3) return (void*)sg_stage_sweep3_kernel<T, false>;
        else if constexpr (D <= 2) return (void*)sg_stage_box_kernel<T, D, PPT>;
        else return (void*)sg_stage_line_kernel<T, D, PPT>;
    }
};

template <class T, int D, int PPT>
cudaError_t stage_one(const StageArgs& a, int nblocks, size_t smem, cudaStream_t s) {
    // the dynamic shared-memory limit was raised by stage_prepare() when the handle was created
    if constexpr (D == 3) {
        if (a.phys.zmask) sg_stage_sweep3_kernel<T, true><<<nblocks, SG_NT3, smem, s>>>(a);
        else sg_stage_sweep3_kernel<T, false><<<nblocks, SG_NT3, smem, s>>>(a);
    }
    else if constexpr (D <= 2) sg_stage_box_kernel<T, D, PPT><<<nblocks, SG_NT, smem, s>>>(a);
    else sg_stage_line_kernel<T, D, PPT><<<nblocks, SG_NT, smem, s>>>(a);
    return cudaGetLastError();
}

template <class T, int D, int PPT>
int prepare_one(size_t smem) {
    const void* kern = StageKernel<T, D, PPT>::fn();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if constexpr (D == 3) {  // the zero-boundary instantiation of the sweep kernel (same resources)
        if (cudaFuncSetAttribute((const void*)sg_stage_sweep3_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, StageKernel<T, D, PPT>::threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

template <class T, int D>
cudaError_t stage_d(int ppt, const StageArgs& a, int nblocks, size_t smem, cudaStream_t s) {
    switch (ppt) {
        case 1: return stage_one<T, D, 1>(a, nblocks, smem, s);
        case 2: return stage_one<T, D, 2>(a, nblocks, smem, s);
        case 4: return stage_one<T, D, 4>(a, nblocks, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class T, int D>
int prepare_d(int ppt, size_t smem) {
    switch (ppt) {
        case 1: return prepare_one<T, D, 1>(smem);
        case 2: return prepare_one<T, D, 2>(smem);
        case 4: return prepare_one<T, D, 4>(smem);
        default: return 0;
    }
}

inline int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 152LL * 32) b = 152LL * 32;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace detail

template <class T>
size_t Launch<T>::stage_smem(int dim, int ppt, long long box, long long flux, int variant) {
    (void)ppt;
    if (dim == 3 && variant == 3) return sizeof(T) * (size_t)(box + flux);  // u only (split in the sweep)
    if (dim <= 3 && variant != 2) return sizeof(T) * (size_t)(2 * box + flux);
    return sizeof(T) * (size_t)(box + flux) + sizeof(int) * (size_t)flux;  // + per-line offsets
}

template <class T>
int Launch<T>::stage_threads(int dim, int variant) {
    return dim == 3 && variant == 0 ? SG_NT3 : (dim == 3 && variant == 3 ? SG_NT3H : SG_NT);
}

namespace detail {
template <class T>
int prepare_box3(int ppt, size_t smem) {
    const void* kern = ppt == 1 ? (const void*)sg_stage_box_kernel<T, 3, 1>
                     : ppt == 2 ? (const void*)sg_stage_box_kernel<T, 3, 2> : (const void*)sg_stage_box_kernel<T, 3, 4>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, SG_NT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}
// d = 2 with the line-buffer kernel (variant 2)
template <class T>
int prepare_line2(int ppt, size_t smem) {
    const void* kern = ppt == 1 ? (const void*)sg_stage_line_kernel<T, 2, 1>
                     : ppt == 2 ? (const void*)sg_stage_line_kernel<T, 2, 2> : (const void*)sg_stage_line_kernel<T, 2, 4>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, SG_NT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}
template <class T>
cudaError_t stage_line2(int ppt, const StageArgs& a, int nblocks, size_t smem, cudaStream_t s) {
    switch (ppt) {
        case 1: sg_stage_line_kernel<T, 2, 1><<<nblocks, SG_NT, smem, s>>>(a); break;
        case 2: sg_stage_line_kernel<T, 2, 2><<<nblocks, SG_NT, smem, s>>>(a); break;
        case 4: sg_stage_line_kernel<T, 2, 4><<<nblocks, SG_NT, smem, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
template <class T>
cudaError_t stage_box3(int ppt, const StageArgs& a, int nblocks, size_t smem, cudaStream_t s) {
    switch (ppt) {
        case 1: sg_stage_box_kernel<T, 3, 1><<<nblocks, SG_NT, smem, s>>>(a); break;
        case 2: sg_stage_box_kernel<T, 3, 2><<<nblocks, SG_NT, smem, s>>>(a); break;
        case 4: sg_stage_box_kernel<T, 3, 4><<<nblocks, SG_NT, smem, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
}  // namespace detail

namespace detail {
// d = 3, FP32, two lines per thread (variant 3); all four instantiations get the same limits
template <class T>
int prepare_sweep2(size_t smem) {
    if constexpr (sizeof(T) != 4) {
        return 0;
    } else {
        const void* kk[4] = {(const void*)sg_stage_sweep3x2_kernel<false, 1>, (const void*)sg_stage_sweep3x2_kernel<true, 1>,
                             (const void*)sg_stage_sweep3x2_kernel<false, 2>, (const void*)sg_stage_sweep3x2_kernel<true, 2>};
        // A small preferred shared-memory carveout: the driver takes the smallest configuration
        // that holds the 6 blocks of ~20 KB the registers allow (ncu: 6 blocks per SM, both
        // limits), and the rest of the unified array (~124 KB) serves as L1, where the update's
        // loads of U and D find the lines the same tile's gather brought in.  Measured: 44% and
        // 58% alike, 72% (~92 KB of L1) 0.6% slower, and the two-array box at 6 blocks with a
        // 28 KB L1 5% slower.
        for (const void* k : kk) {
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
                cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 44) != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
        }
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kk[0], SG_NT3H, smem) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return nb;
    }
}
}  // namespace detail

template <class T>
int Launch<T>::stage_prepare(int dim, int ppt, size_t smem, int variant) {
    if (dim == 3 && variant == 3) return detail::prepare_sweep2<T>(smem);
    if (dim == 3 && variant == 1) return detail::prepare_box3<T>(ppt, smem);
    if (dim == 2 && variant == 2) return detail::prepare_line2<T>(ppt, smem);
    switch (dim) {
        case 1: return detail::prepare_d<T, 1>(ppt, smem);
        case 2: return detail::prepare_d<T, 2>(ppt, smem);
        case 3: return detail::prepare_d<T, 3>(ppt, smem);
        case 4: return detail::prepare_d<T, 4>(ppt, smem);
        case 5: return detail::prepare_d<T, 5>(ppt, smem);
        case 6: return detail::prepare_d<T, 6>(ppt, smem);
        default: return 0;
    }
}

template <class T>
cudaError_t Launch<T>::stage(int dim, int ppt, const StageArgs& a, int nblocks, size_t smem, cudaStream_t s,
                             int variant) {
    if (nblocks < 1) return cudaSuccess;
    if (dim == 3 && variant == 3) {
        if constexpr (sizeof(T) != 4) {
            return cudaErrorInvalidValue;
        } else {
            // pairs of consecutive items per block when there are at least two per block
            const bool pairs = a.item_end - a.item_begin >= 2 * nblocks;
            if (a.phys.zmask) {
                if (pairs) sg_stage_sweep3x2_kernel<true, 2><<<nblocks, SG_NT3H, smem, s>>>(a);
                else sg_stage_sweep3x2_kernel<true, 1><<<nblocks, SG_NT3H, smem, s>>>(a);
            } else {
                if (pairs) sg_stage_sweep3x2_kernel<false, 2><<<nblocks, SG_NT3H, smem, s>>>(a);
                else sg_stage_sweep3x2_kernel<false, 1><<<nblocks, SG_NT3H, smem, s>>>(a);
            }
            return cudaGetLastError();
        }
    }
    if (dim == 3 && variant == 1) return detail::stage_box3<T>(ppt, a, nblocks, smem, s);
    if (dim == 2 && variant == 2) return detail::stage_line2<T>(ppt, a, nblocks, smem, s);
    switch (dim) {
        case 1: return detail::stage_d<T, 1>(ppt, a, nblocks, smem, s);
        case 2: return detail::stage_d<T, 2>(ppt, a, nblocks, smem, s);
        case 3: return detail::stage_d<T, 3>(ppt, a, nblocks, smem, s);
        case 4: return detail::stage_d<T, 4>(ppt, a, nblocks, smem, s);
        case 5: return detail::stage_d<T, 5>(ppt, a, nblocks, smem, s);
        case 6: return detail::stage_d<T, 6>(ppt, a, nblocks, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class T>
cudaError_t Launch<T>::alpha_init(const GridDesc* grids, int ngrids, long long max_pts,
                                  unsigned long long* alpha, int* flags, cudaStream_t s) {
    if (ngrids < 1) return cudaSuccess;
    long long bx = (max_pts + SG_NT - 1) / SG_NT;
    if (bx > 256) bx = 256;
    const int by = ngrids < 65535 ? ngrids : 65535;
    sg_alpha_init_kernel<T><<<dim3((unsigned)bx, (unsigned)by), SG_NT, 0, s>>>(grids, ngrids, alpha, flags);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::restrict_sine(const GridDesc* grids, int ngrids, long long max_npts, int dim, const double* p,
                                     cudaStream_t s) {
    for (int g0 = 0; g0 < ngrids; g0 += 65535) {  // gridDim.y <= 65535 grids per launch
        const int ng = ngrids - g0 < 65535 ? ngrids - g0 : 65535;
        const dim3 grid((unsigned)detail::grid_for(max_npts, 256), (unsigned)ng);
        sg_restrict_sine_kernel<T><<<grid, 256, 0, s>>>(grids + g0, dim, p[0], p[1], p[2], p[3]);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <class T>
cudaError_t Launch<T>::prolong_axis(const T* in, T* out, double* acc, double coeff, long long below,
                                    int min_, int nf, long long above, int r, double eps,
                                    int lagrange, int zero_bc, cudaStream_t s) {
    const long long tot = below * nf * above;
    sg_prolong_axis_kernel<T><<<detail::grid_for(tot, 256), 256, 0, s>>>(in, out, acc, coeff, below, min_,
                                                                          nf, above, r, eps, lagrange, zero_bc);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::efield(const GridDesc* grids, int ngrids, const InstState* inst, unsigned long long* alpha,
                              int stage, int pre_dt, cudaStream_t s) {
    if (ngrids < 1) return cudaSuccess;
    const int nb = ngrids < 65535 ? ngrids : 65535;
    sg_efield_kernel<T><<<nb, 256, 0, s>>>(grids, ngrids, inst, alpha, stage, pre_dt);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::field_energy(const T* u, const T* comp, int n0, int n1, double hx, double hv,
                                    double* scratch, double* out, cudaStream_t s) {
    sg_field_energy_kernel<T><<<1, 256, 0, s>>>(u, comp, n0, n1, hx, hv, scratch, out);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::restrict_landau(const GridDesc& g, double a, double kx, cudaStream_t s) {
    sg_restrict_landau_kernel<T><<<detail::grid_for(g.npts, 256), 256, 0, s>>>(g, a, kx);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::restrict_relax(const GridDesc& g, int dim, double s_norm, cudaStream_t s) {
    sg_restrict_relax_kernel<T><<<detail::grid_for(g.npts, 256), 256, 0, s>>>(g, dim, s_norm);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::density(const GridDesc* grids, int ngrids, long long max_nx, const InstState* inst,
                               int stage, int dim, cudaStream_t s) {
    if (ngrids < 1) return cudaSuccess;
    const long long per = sizeof(T) == 8 ? 32 * SG_DENS_ROWS : 32;  // space nodes per block
    const dim3 grid((unsigned)std::min<long long>((max_nx + per - 1) / per, 1024), (unsigned)std::min(ngrids, 65535));
    sg_density_kernel<T><<<grid, dim3(32, SG_DENS_ROWS), 0, s>>>(grids, ngrids, inst, stage, dim);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::accumulate(const T* u, double* acc, double coeff, long long n, cudaStream_t s) {
    sg_accumulate_kernel<T><<<detail::grid_for(n, 256), 256, 0, s>>>(u, acc, coeff, n);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::gather(const T* u, const long long* idx, T* out, long long n, cudaStream_t s) {
    if (n < 1) return cudaSuccess;
    sg_gather_kernel<T><<<detail::grid_for(n, 256), 256, 0, s>>>(u, idx, out, n);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::prolong_multi(const ProlongTask* tasks, int ntasks, long long nunits, double eps, int lagrange,
                                     cudaStream_t s) {
    if (ntasks < 1 || nunits < 1) return cudaSuccess;
    const unsigned nb = (unsigned)std::min<long long>((nunits + 255) / 256, 1LL << 22);
    sg_prolong_multi_kernel<T, 8><<<nb, 256, 0, s>>>(tasks, ntasks, nunits, eps, lagrange);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::prolong_multi_pairs(const ProlongTask* tasks, int ntasks, long long nunits, double eps,
                                           int lagrange, cudaStream_t s) {
    if constexpr (sizeof(T) != 4) {
        return prolong_multi(tasks, ntasks, nunits, eps, lagrange, s);
    } else {
        if (ntasks < 1 || nunits < 2) return cudaSuccess;
        const unsigned nb = (unsigned)std::min<long long>((nunits / 2 + 255) / 256, 1LL << 22);
        sg_prolong_multi_x2_kernel<8><<<nb, 256, 0, s>>>(tasks, ntasks, nunits, eps, lagrange);
        return cudaGetLastError();
    }
}

template <class T>
cudaError_t Launch<T>::combine_last_axis(const CombineGrid* tab, int G, double* uhat, long long below, int nf,
                                         int exact_coeffs, int zero_last, int pairs_aligned,
                                         double eps, int lagrange, cudaStream_t s) {
    constexpr int J = 8;
    // FP32: two columns per thread, packed f32x2 (sg_combine2.cuh), the grid table in shared
    // memory (16 bytes a grid, at most 48 KB; n below 2^26)
    if constexpr (sizeof(T) == 4) {
        if ((size_t)G * sizeof(CombineEntry) <= 48 * 1024 && nf < (1 << SG_COMBINE_NLR_SHIFT)) {
            constexpr int CY = 8;
            const long long npairs = (below + 1) / 2;
            const dim3 grid2((unsigned)std::min<long long>((nf + J * CY - 1) / (J * CY), 65535),
                             (unsigned)std::min<long long>((npairs + 31) / 32, 65535));
            const dim3 blk(32, CY);
            const size_t sm = (size_t)G * sizeof(CombineEntry);
            const int key = (exact_coeffs ? 4 : 0) | (pairs_aligned ? 2 : 0) | (zero_last ? 1 : 0);
            switch (key) {
#define SG_COMB2(K, E, V, Z)                                                                                   \
    case K:                                                                                                    \
        sg_combine_last_axis_f32x2_kernel<J, CY, E, V, Z><<<grid2, blk, sm, s>>>(tab, G, uhat, below, nf, eps, \
                                                                                 lagrange);                    \
        break;
                SG_COMB2(0, false, false, false)
                SG_COMB2(1, false, false, true)
                SG_COMB2(2, false, true, false)
                SG_COMB2(3, false, true, true)
                SG_COMB2(4, true, false, false)
                SG_COMB2(5, true, false, true)
                SG_COMB2(6, true, true, false)
                SG_COMB2(7, true, true, true)
#undef SG_COMB2
            }
            return cudaGetLastError();
        }
    }
    dim3 grid((unsigned)std::min<long long>((below + 255) / 256, 65535),
              (unsigned)std::min<long long>((nf + J - 1) / J, 65535));
    if (exact_coeffs)
        sg_combine_last_axis_kernel<T, J, true><<<grid, 256, 0, s>>>(tab, G, uhat, below, nf, eps, lagrange, zero_last);
    else
        sg_combine_last_axis_kernel<T, J, false><<<grid, 256, 0, s>>>(tab, G, uhat, below, nf, eps, lagrange, zero_last);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::reduce(const T* u, const T* comp, long long n, int kind, const ExactSpec& X,
                              double* partial, double* out, cudaStream_t s) {
    int nb = (int)((n + 255) / 256);
    if (nb > 1024) nb = 1024;
    if (nb < 1) nb = 1;
    sg_reduce_pass1<T><<<nb, 256, 0, s>>>(u, comp, n, kind, X, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sg_reduce_pass2<<<1, 256, 0, s>>>(partial, nb, kind, out);
    return cudaGetLastError();
}

}  // namespace sg
