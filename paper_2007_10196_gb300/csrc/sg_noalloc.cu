// sg_noalloc.cu -- sg_step_grid_noalloc: one TVD-RK3 step of one periodic FP64 grid held in
// caller memory, with every piece of scratch in a static device array, so that the call
// allocates nothing.
//
// Who needs it: callers that must not call cudaMalloc -- code running under a framework that
// owns all device memory and forbids side allocations, or a real-time loop in which an
// allocation (and the implicit synchronisation cudaMalloc/cudaFree can bring) is not
// allowed.  They pass the grid in and get the stepped grid back; the two intermediate RK
// stages, the grid descriptor, the work queue, the alpha slots and the status flags live in
// `sg_noalloc_scratch` below.
//
// Compiled with --fmad=false, like the FP64 kernels, so that the result equals sg_step's bit
// for bit: the same stage kernel runs, on the same tiles.
#include <cstdint>
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "sg_kernels.cuh"
#include "sg_launch.h"
#include "sgweno.h"

namespace {

constexpr int kMaxTiles = 65536;       // work items (tiles of <= 512 points) of one grid
constexpr int kMaxDevices = 64;
constexpr size_t kHeaderBytes = 4096;  // GridDesc, InstState, alpha slots, flags
constexpr size_t kItemBytes = sizeof(WorkItem) * (size_t)kMaxTiles;
constexpr size_t kScratchDoubles =
    2 * (size_t)SG_NOALLOC_MAX_POINTS + (kHeaderBytes + kItemBytes) / sizeof(double);
// byte offsets inside the scratch array
constexpr size_t kOffU1 = 0;
constexpr size_t kOffU2 = sizeof(double) * (size_t)SG_NOALLOC_MAX_POINTS;
constexpr size_t kOffGrid = 2 * sizeof(double) * (size_t)SG_NOALLOC_MAX_POINTS;
constexpr size_t kOffInst = kOffGrid + 512;
constexpr size_t kOffAlpha = kOffInst + 512;
constexpr size_t kOffFlags = kOffAlpha + 64;
constexpr size_t kOffItems = kOffGrid + kHeaderBytes;
static_assert(sizeof(GridDesc) <= 512 && sizeof(InstState) <= 512, "header layout");
static_assert(kOffFlags + 16 <= kOffItems, "header layout");

}  // namespace

// The scratch: about 16.5 MB, held by every GPU that loads this library until the process
// exits.  Host code must not use this name as an address (it is a host-side stand-in);
// it uses the device address looked up by cudaGetSymbolAddress in na_setup().
static __device__ __align__(256) double sg_noalloc_scratch[kScratchDoubles];

namespace {

std::mutex g_na_mutex;
char* g_na_ptr[kMaxDevices];  // device address of sg_noalloc_scratch, per device

sg_status na_fail(sg_status s, const char* msg) {
    sg::set_last_error(msg);
    return s;
}

sg_status na_cuda(cudaError_t e, const char* what) {
    cudaGetLastError();
    char buf[256];
    snprintf(buf, sizeof buf, "%s failed: %s", what, cudaGetErrorString(e));
    sg::set_last_error(buf);
    return SG_ERR_CUDA;
}

// Once per device, with that device current: the device address of the scratch array.
sg_status na_setup(char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return na_fail(SG_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, sg_noalloc_scratch);
        if (e != cudaSuccess || !p) return na_cuda(e, "cudaGetSymbolAddress(sg_noalloc_scratch)");
        g_na_ptr[dev] = (char*)p;
    }
    *out = g_na_ptr[dev];
    return SG_OK;
}

// Writes the grid descriptor, the instance state and the work queue into the scratch and
// clears the alpha slots and the flags: every call starts from zero there.
__global__ void sg_noalloc_setup_kernel(char* base, GridDesc gd, InstState st, int ntiles) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx == 0) {
        *(GridDesc*)(base + kOffGrid) = gd;
        *(InstState*)(base + kOffInst) = st;
        unsigned long long* a = (unsigned long long*)(base + kOffAlpha);
        a[0] = a[1] = a[2] = 0ull;
        int* f = (int*)(base + kOffFlags);
        f[0] = f[1] = f[2] = f[3] = 0;
    }
    WorkItem* items = (WorkItem*)(base + kOffItems);
    for (int t = idx; t < ntiles; t += gridDim.x * blockDim.x) items[t] = WorkItem{0, t};
}

// Tile extents, as sg_create chooses them (512-point tiles): halve the longest extent, the
// highest axis on ties, until the tile has at most 512 points.
void na_tile(const int* n, int dim, int* te) {
    for (int k = 0; k < dim; ++k) te[k] = n[k];
    for (;;) {
        long long p = 1;
        for (int k = 0; k < dim; ++k) p *= te[k];
        if (p <= 512) break;
        int best = 0;
        for (int k = 1; k < dim; ++k)
            if (te[k] >= te[best]) best = k;
        te[best] = (te[best] + 1) / 2;
    }
}

template <int D>
cudaError_t na_stages(char* base, const PhysParams& ph, int ntiles, int box_elems, size_t smem,
                      cudaStream_t s) {
    auto kern = sg_stage_box_kernel<double, D, 2>;
    // raised on every call: sg_create may since have set a smaller limit for its own tiles
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, nsm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SG_NT, smem)) != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int nblocks = std::max(1, std::min(ntiles, std::max(per_sm, 1) * nsm));
    for (int stage = 0; stage < 3; ++stage) {
        StageArgs a{};
        a.grids = (const GridDesc*)(base + kOffGrid);
        a.items = (const WorkItem*)(base + kOffItems);
        a.inst = (InstState*)(base + kOffInst);
        a.alpha = (unsigned long long*)(base + kOffAlpha);
        a.flags = (int*)(base + kOffFlags);
        a.item_begin = 0;
        a.item_end = ntiles;
        a.stage = stage;
        a.box_elems = box_elems;
        a.phys = ph;
        kern<<<nblocks, SG_NT, smem, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" sg_status sg_step_grid_noalloc(int dim, const long* shape, const double* lo, const double* hi,
                                          int pde, const double* adv_speed, int scheme, double eps,
                                          const double* u_in, double* u_out, double dt, void* cuda_stream) {
    if (dim < 1 || dim > 3) return na_fail(SG_ERR_UNSUPPORTED, "sg_step_grid_noalloc handles dim 1..3");
    if (!shape || !lo || !hi || !u_in || !u_out) return na_fail(SG_ERR_ARG, "NULL argument");
    if (pde != SG_PDE_ADVECTION && pde != SG_PDE_BURGERS) return na_fail(SG_ERR_ARG, "pde");
    if (scheme != SG_WENO5 && scheme != SG_LINEAR5) return na_fail(SG_ERR_ARG, "scheme");
    if (!(eps > 0.0) || !(dt >= 0.0) || dt != dt || dt > 1e300) return na_fail(SG_ERR_ARG, "eps must be > 0 and dt finite, >= 0");
    long long npts = 1;
    int n[SG_MAXD] = {1, 1, 1, 1, 1, 1};
    for (int k = 0; k < dim; ++k) {
        if (shape[k] < 5) return na_fail(SG_ERR_ARG, "every axis needs >= 5 points (the stencil spans 5 distinct nodes)");
        if (!(hi[k] > lo[k])) return na_fail(SG_ERR_ARG, "need lo < hi on every axis");
        if (shape[k] > SG_NOALLOC_MAX_POINTS) return na_fail(SG_ERR_ARG, "grid exceeds SG_NOALLOC_MAX_POINTS points");
        n[k] = (int)shape[k];
        npts *= shape[k];
        if (npts > SG_NOALLOC_MAX_POINTS) return na_fail(SG_ERR_ARG, "grid exceeds SG_NOALLOC_MAX_POINTS points");
    }
    {  // u_in and u_out: the same array, or two that do not overlap
        const uintptr_t a = reinterpret_cast<uintptr_t>(u_in), b = reinterpret_cast<uintptr_t>(u_out);
        const uintptr_t len = sizeof(double) * (uintptr_t)npts;
        if (a != b && a < b + len && b < a + len)
            return na_fail(SG_ERR_ARG, "u_in and u_out overlap without being the same array");
    }
    char* base = nullptr;
    sg_status st = na_setup(&base);
    if (st != SG_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    GridDesc gd{};
    na_tile(n, dim, gd.te);
    int ntiles = 1;
    for (int k = 0; k < SG_MAXD; ++k) {
        if (k < dim) {
            gd.n[k] = n[k];
            gd.nt[k] = (n[k] + gd.te[k] - 1) / gd.te[k];
            gd.ntmag[k] = sg_div_magic64((unsigned)gd.nt[k]);
            gd.h[k] = (hi[k] - lo[k]) / (double)n[k];
            gd.rdx[k] = 1.0 / gd.h[k];
            gd.rdxf[k] = (float)gd.rdx[k];
            gd.lo[k] = lo[k];
            ntiles *= gd.nt[k];
        } else {
            gd.n[k] = gd.te[k] = gd.nt[k] = 1;
            gd.ntmag[k] = 0;
            gd.h[k] = gd.rdx[k] = 1.0;
            gd.rdxf[k] = 1.0f;
        }
    }
    if (ntiles > kMaxTiles) return na_fail(SG_ERR_ARG, "grid needs more work items than the scratch holds");
    gd.u0 = u_out;  // u^n, and u^{n+1} written in place by the last stage
    gd.u1 = base + kOffU1;
    gd.u2 = base + kOffU2;
    gd.u3 = nullptr;
    gd.npts = npts;
    gd.coeff = 1.0;
    gd.inst = 0;
    gd.first_item = 0;
    gd.n_items = ntiles;

    InstState is{};
    is.dt = dt;
    is.dtf = (float)dt;
    is.t_end = dt;
    is.active = 1;
    is.ngrids = 1;

    PhysParams ph{};
    ph.dim = dim;
    ph.pde = pde;
    ph.scheme = scheme;
    ph.eps = eps;
    for (int k = 0; k < SG_MAXD; ++k) ph.adv[k] = (adv_speed && k < dim) ? adv_speed[k] : 1.0;

    long long box = 0, flux = 0;
    sg::box_footprint(dim, gd.te, &box, &flux);
    const size_t smem = sizeof(double) * (size_t)(2 * box + flux);

    cudaError_t e;
    if (u_in != u_out) {
        e = cudaMemcpyAsync(u_out, u_in, sizeof(double) * (size_t)npts, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return na_cuda(e, "cudaMemcpyAsync");
    }
    const int setup_blocks = std::max(1, std::min(256, (ntiles + 255) / 256));
    sg_noalloc_setup_kernel<<<setup_blocks, 256, 0, s>>>(base, gd, is, ntiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return na_cuda(e, "setup kernel");
    // alpha slot 0: max |u| of the stage-0 input
    e = sg::Launch<double>::alpha_init((const GridDesc*)(base + kOffGrid), 1, npts,
                                       (unsigned long long*)(base + kOffAlpha), (int*)(base + kOffFlags), s);
    if (e != cudaSuccess) return na_cuda(e, "alpha kernel");
    switch (dim) {
        case 1: e = na_stages<1>(base, ph, ntiles, (int)box, smem, s); break;
        case 2: e = na_stages<2>(base, ph, ntiles, (int)box, smem, s); break;
        default: e = na_stages<3>(base, ph, ntiles, (int)box, smem, s); break;
    }
    if (e != cudaSuccess) return na_cuda(e, "stage kernel");
    return SG_OK;
}
