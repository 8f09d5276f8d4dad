// FP64 instantiation of the kernels.  Compiled with --fmad=false so that every double
// expression is evaluated as written (no fused multiply-add): the FP64 path then performs
// the same IEEE-754 operations, in the same order, as a plain sequential evaluation of the
// paper's formulas.  Also holds the precision-independent launchers.
#include <algorithm>
#include "sg_launch_impl.cuh"

namespace sg {

template struct Launch<double>;

cudaError_t launch_dt(InstState* inst, int ninst, const GridDesc* grids, const unsigned long long* alpha,
                      const PhysParams& ph, int commit_only, int* flags, cudaStream_t s) {
    if (ninst < 1) return cudaSuccess;
    sg_dt_kernel<<<(ninst + 3) / 4, 128, 0, s>>>(inst, ninst, grids, alpha, ph, commit_only, flags);  // a warp per instance
    return cudaGetLastError();
}

void box_footprint(int d, const int* te, long long* box, long long* flux) {
    long long b = 1, p = 1;
    for (int k = 0; k < d; ++k) {
        b *= te[k] + 6;
        p *= te[k];
    }
    long long f = 0;
    for (int k = 0; k < d; ++k) f += p / te[k] * (te[k] + 1);
    *box = b;
    *flux = f;
}

void line_footprint(int d, const int* te, long long* box, long long* acc) {
    long long p = 1;
    for (int k = 0; k < d; ++k) p *= te[k];
    long long b = 1;
    for (int k = 0; k < d; ++k) b = std::max(b, p / te[k] * (long long)((te[k] + 6) | 1));
    *box = b;
    *acc = p;
}

void sweep_footprint(const int* te, long long* box, long long* flux) {
    *box = (long long)((te[0] + 6) | 1) * (te[1] + 6) * (te[2] + 6);
    *flux = 3 * SG_DK_AXIS;
}

void sweep_tile(const int* n, int* te) {
    for (int k = 0; k < 3; ++k) {
        int t = 0;
        for (int c = 8; c >= 4 && !t; --c)
            if (n[k] % c == 0) t = c;
        te[k] = t ? t : (n[k] < 8 ? n[k] : 8);
    }
}

}  // namespace sg
