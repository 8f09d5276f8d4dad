// sg_launch_impl.cuh -- definitions of sg::Launch<T>; included by exactly one translation
// unit per precision.
#pragma once
#include "sg_kernels.cuh"
#include "sg_launch.h"

namespace sg {

namespace detail {

template <class T, int D, int PPT>
cudaError_t stage_one(const StageArgs& a, int nblocks, cudaStream_t s) {
    auto kern = sg_stage_kernel<T, D, PPT>;
    const size_t smem = sizeof(T) * (size_t)(StageSmem<PPT>::LB + StageSmem<PPT>::FB);
    // the dynamic shared-memory limit was raised by occupancy_one() when the handle was created
    kern<<<nblocks, SG_NT, smem, s>>>(a);
    return cudaGetLastError();
}

template <class T, int D, int PPT>
int occupancy_one() {
    auto kern = sg_stage_kernel<T, D, PPT>;
    const size_t smem = sizeof(T) * (size_t)(StageSmem<PPT>::LB + StageSmem<PPT>::FB);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, SG_NT, smem) != cudaSuccess) return 0;
    return nb;
}

template <class T, int D>
cudaError_t stage_d(int ppt, const StageArgs& a, int nblocks, cudaStream_t s) {
    switch (ppt) {
        case 1: return stage_one<T, D, 1>(a, nblocks, s);
        case 2: return stage_one<T, D, 2>(a, nblocks, s);
        case 4: return stage_one<T, D, 4>(a, nblocks, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class T, int D>
int occ_d(int ppt) {
    switch (ppt) {
        case 1: return occupancy_one<T, D, 1>();
        case 2: return occupancy_one<T, D, 2>();
        case 4: return occupancy_one<T, D, 4>();
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
size_t Launch<T>::stage_smem(int ppt) {
    return sizeof(T) * (size_t)(8 + 3) * SG_NT * (size_t)ppt;
}

template <class T>
int Launch<T>::stage_blocks_per_sm(int dim, int ppt) {
    switch (dim) {
        case 1: return detail::occ_d<T, 1>(ppt);
        case 2: return detail::occ_d<T, 2>(ppt);
        case 3: return detail::occ_d<T, 3>(ppt);
        case 4: return detail::occ_d<T, 4>(ppt);
        case 5: return detail::occ_d<T, 5>(ppt);
        case 6: return detail::occ_d<T, 6>(ppt);
        default: return 0;
    }
}

template <class T>
cudaError_t Launch<T>::stage(int dim, int ppt, const StageArgs& a, int nblocks, cudaStream_t s) {
    if (nblocks < 1) return cudaSuccess;
    switch (dim) {
        case 1: return detail::stage_d<T, 1>(ppt, a, nblocks, s);
        case 2: return detail::stage_d<T, 2>(ppt, a, nblocks, s);
        case 3: return detail::stage_d<T, 3>(ppt, a, nblocks, s);
        case 4: return detail::stage_d<T, 4>(ppt, a, nblocks, s);
        case 5: return detail::stage_d<T, 5>(ppt, a, nblocks, s);
        case 6: return detail::stage_d<T, 6>(ppt, a, nblocks, s);
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
cudaError_t Launch<T>::restrict_sine(const GridDesc& g, int dim, const double* p, cudaStream_t s) {
    sg_restrict_sine_kernel<T><<<detail::grid_for(g.npts, 256), 256, 0, s>>>(g, dim, p[0], p[1], p[2], p[3]);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::prolong_axis(const T* in, T* out, double* acc, double coeff, long long below,
                                    int min_, int nf, long long above, int r, double eps,
                                    int lagrange, cudaStream_t s) {
    const long long tot = below * nf * above;
    sg_prolong_axis_kernel<T><<<detail::grid_for(tot, 256), 256, 0, s>>>(in, out, acc, coeff, below, min_,
                                                                          nf, above, r, eps, lagrange);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::accumulate(const T* u, double* acc, double coeff, long long n, cudaStream_t s) {
    sg_accumulate_kernel<T><<<detail::grid_for(n, 256), 256, 0, s>>>(u, acc, coeff, n);
    return cudaGetLastError();
}

template <class T>
cudaError_t Launch<T>::reduce(const T* u, long long n, int kind, const ExactSpec& X, double* partial,
                              double* out, cudaStream_t s) {
    int nb = (int)((n + 255) / 256);
    if (nb > 1024) nb = 1024;
    if (nb < 1) nb = 1;
    sg_reduce_pass1<T><<<nb, 256, 0, s>>>(u, n, kind, X, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sg_reduce_pass2<<<1, 256, 0, s>>>(partial, nb, kind, out);
    return cudaGetLastError();
}

}  // namespace sg
