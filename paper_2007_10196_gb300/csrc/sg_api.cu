// sg_api.cu -- the C ABI of include/sgweno.h: handle lifecycle, the grid table and work
// queue, device-side time-step control replayed through CUDA graphs, prolongation and
// combination, reductions.  All numerical work runs in the kernels of sg_kernels.cuh.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "sg_device.h"
#include "sg_launch.h"
#include "sgweno.h"

namespace {

thread_local std::string g_err;

sg_alloc_fn g_alloc = nullptr;
sg_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;
long g_live_handles = 0;

sg_status fail(sg_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define SG_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            return fail(SG_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
        }                                                                                  \
    } while (0)

#define SG_TRY(expr)                    \
    do {                                \
        sg_status s_ = (expr);          \
        if (s_ != SG_OK) return s_;     \
    } while (0)

// Device buffer through the allocator hook (or cudaMalloc).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    sg_status alloc(size_t b) {
        release();
        if (b == 0) b = 256;
        void* q = nullptr;
        if (g_alloc) {
            q = g_alloc(b, g_alloc_ctx);
        } else if (cudaMalloc(&q, b) != cudaSuccess) {
            cudaGetLastError();
            q = nullptr;
        }
        if (!q) return fail(SG_ERR_NOMEM, "device allocation of %zu bytes failed", b);
        p = q;
        bytes = b;
        return SG_OK;
    }
    void release() {
        if (!p) return;
        if (g_free) g_free(p, bytes, g_alloc_ctx);
        else cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// Intermediates of the fused prolongation + combination.
struct CombineBuffers {
    DevBuf pool, pa, tab;  // phase-1 pool, phase-1 intermediates, grid and task tables
};

struct PinnedInst {
    InstState* p = nullptr;
    int n = 0;
    ~PinnedInst() {
        if (p) cudaFreeHost(p);
    }
    sg_status alloc(int count) {
        if (cudaMallocHost((void**)&p, sizeof(InstState) * (size_t)count) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(SG_ERR_NOMEM, "pinned host allocation failed");
        }
        n = count;
        std::memset(p, 0, sizeof(InstState) * (size_t)count);
        return SG_OK;
    }
};

long long binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// Levels with |l| = target, l_k in [0, nl], lexicographic with l_0 most significant.
void compositions(int dim, int nl, int k, int remaining, std::array<int, SG_MAXD>& cur,
                  std::vector<std::array<int, SG_MAXD>>& out) {
    if (k == dim - 1) {
        if (remaining <= nl) {
            cur[k] = remaining;
            out.push_back(cur);
        }
        return;
    }
    for (int l = 0; l <= std::min(nl, remaining); ++l) {
        cur[k] = l;
        compositions(dim, nl, k + 1, remaining - l, cur, out);
    }
}

}  // namespace

struct sg_ctx {
    bool is_batch = false;
    int dim = 0, nr = 0, nl = 0, pde = 0;
    sg_params prm{};
    int esize = 8;
    int ppt = 2;       // points per thread of the stage kernel (tile = 256 ppt points)
    int variant = 0;   // stage kernel: 0 = default of the dimension, 1 = padded box (d = 3)
    bool tuned = false;
    double tune_ms = 0.0;  // time of one stage launch of the chosen configuration
    // grids (single handle)
    int G = 0;
    std::vector<std::array<int, SG_MAXD>> levels;
    std::vector<double> coeff;
    std::vector<long long> npts;
    std::vector<long long> offset;  // element offset of each grid inside a state region
    long long total_pts = 0;
    DevBuf arena;  // state regions u0, u1, u2 (and u3 = C for FP32), each all grids concatenated
    DevBuf efield; // Vlasov-Poisson: E of every grid (n_0 values each); Vlasov-Boltzmann: rho
                   // (n_0 ... n_{d/2-1} values each); grids concatenated
    std::vector<long long> ef_offset;
    DevBuf mutab;  // Vlasov-Boltzmann: mu_inf at the velocity nodes of every grid, concatenated
    std::vector<long long> mu_offset;
    long long max_nx = 0;  // Vlasov-Boltzmann: largest space-node count of a grid
    double relax_s = 0.0;  // Vlasov-Boltzmann: normalisation of the Example 5 initial condition (0: not yet formed)
    long long box_elems = 0;  // stage kernel: elements of one padded box (d <= 3) or of the line buffer
    size_t smem = 0;          // stage kernel: dynamic shared memory per block
    // device tables (single handle or batch)
    std::vector<GridDesc> hgrids;
    std::vector<WorkItem> hitems;
    DevBuf dgrids, ditems, alpha, flags, dinst, partial;
    PinnedInst hinst;
    int ninst = 1;
    int blocks_total = 1;
    long long max_grid_pts = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph = nullptr;
    int graph_nsteps = 0;
    long long graph_kernels = 0;
    bool graph_profiled = false;
    // profiling: event pairs around each stage launch (group) of one graph replay
    bool profile = false;
    std::vector<cudaEvent_t> ev;
    int ev_pairs_used = 0;
    double prof_ms = 0.0;
    long long prof_launches = 0;
    // state
    bool initialized = false;
    bool combined = false;
    bool ic_sine = false;
    double ic[4] = {0, 0, 0, 0};
    double t = 0.0;
    long long steps = 0;
    long long launches = 0;
    // combination
    DevBuf uhat, pro_a, pro_b;
    CombineBuffers comb;  // fused form's intermediates (a batch's are shared by its members)
    long long fine_pts = 0;
    // batch
    std::vector<sg_ctx*> members;

    ~sg_ctx() {
        if (graph) cudaGraphExecDestroy(graph);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

PhysParams phys_of(const sg_ctx* h) {
    PhysParams ph{};
    ph.dim = h->dim;
    ph.pde = h->pde;
    ph.scheme = h->prm.scheme;
    ph.prolong = h->prm.prolong;
    ph.eps = h->prm.eps;
    for (int k = 0; k < SG_MAXD; ++k) ph.adv[k] = k < h->dim ? h->prm.adv_speed[k] : 0.0;
    ph.alpha_f32 = h->esize == 4;
    ph.tau = h->prm.tau;
    ph.zmask = 0;
    if (h->pde == SG_PDE_ADVECTION || h->pde == SG_PDE_BURGERS)
        for (int k = 0; k < h->dim; ++k)
            if (h->prm.bc[k] == SG_BC_ZERO) ph.zmask |= 1 << k;
    return ph;
}

double fine_spacing(const sg_ctx* h, int k) {
    return (h->prm.hi[k] - h->prm.lo[k]) / (double)((long long)h->nr << h->nl);
}

// Nominal step of the h^{5/3} rule: coef * (min_k h_k)^{5/3} on the finest grid.
double dt_pow53(const sg_ctx* h) {
    double hm = fine_spacing(h, 0);
    for (int k = 1; k < h->dim; ++k) hm = std::min(hm, fine_spacing(h, k));
    return h->prm.dt_coef * std::pow(hm, 5.0 / 3.0);
}

void fill_inst(const sg_ctx* h, InstState& s, int grid0, double t_end, long long max_steps) {
    s.t = h->t;
    s.dt = 0.0;
    s.dtf = 0.0f;
    s.t_end = t_end;
    s.dt_nom = dt_pow53(h);
    s.cfl = h->prm.cfl;
    for (int k = 0; k < SG_MAXD; ++k) s.hf[k] = k < h->dim ? fine_spacing(h, k) : 1.0;
    s.steps = h->steps;
    s.step0 = h->steps;
    s.step_limit = max_steps > (1LL << 62) - h->steps ? (1LL << 62) : h->steps + max_steps;
    s.active = 0;
    s.pending = 0;
    s.last = 0;
    s.grid0 = grid0;
    s.ngrids = h->G;
    s.dt_rule = h->prm.dt_rule;
    // Vlasov-Boltzmann: the LF alpha of each axis is static, the largest |node| of the partner
    // axis over the grids, evaluated as the stage and dt arithmetic of the handle's precision
    for (int k = 0; k < SG_MAXD; ++k) {
        double a = 0.0;
        if (h->pde == SG_PDE_VLASOV_BOLTZMANN && k < h->dim) {
            const int pk = k < h->dim / 2 ? k + h->dim / 2 : k - h->dim / 2;
            for (const GridDesc& G : h->hgrids) {
                if (h->esize == 4) {
                    const float c0 = (float)G.lo[pk], c1 = (float)G.lo[pk] + (float)(G.n[pk] - 1) * (float)G.h[pk];
                    a = std::max(a, (double)std::max(std::fabs(c0), std::fabs(c1)));
                } else {
                    const double c0 = G.lo[pk], c1 = G.lo[pk] + (double)(G.n[pk] - 1) * G.h[pk];
                    a = std::max(a, std::max(std::fabs(c0), std::fabs(c1)));
                }
            }
        }
        s.alpha_vb[k] = a;
    }
}

// Tile extents: start from the whole grid and halve the longest extent (the highest axis on
// ties, keeping axis 0 long for coalescing) until the tile has at most pmax points.
void choose_tile(const int* n, int dim, int pmax, int* te) {
    for (int k = 0; k < dim; ++k) te[k] = n[k];
    for (;;) {
        long long p = 1;
        for (int k = 0; k < dim; ++k) p *= te[k];
        if (p <= pmax) break;
        int best = 0;
        for (int k = 1; k < dim; ++k)
            if (te[k] >= te[best]) best = k;
        te[best] = (te[best] + 1) / 2;
    }
}

int num_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n;
}

// Shared memory of the stage kernel for the largest tile among the given grids.
void stage_footprint(sg_ctx* h) {
    long long box = 1, flux = 1;
    for (const GridDesc& d : h->hgrids) {
        long long b, f;
        if (h->dim == 3 && (h->variant == 0 || h->variant == 3)) sg::sweep_footprint(d.te, &b, &f);
        else if (h->dim >= 4 || h->variant == 2) sg::line_footprint(h->dim, d.te, &b, &f);
        else sg::box_footprint(h->dim, d.te, &b, &f);
        box = std::max(box, b);
        flux = std::max(flux, f);
    }
    h->box_elems = box;
    h->smem = h->esize == 8 ? sg::Launch<double>::stage_smem(h->dim, h->ppt, box, flux, h->variant)
                            : sg::Launch<float>::stage_smem(h->dim, h->ppt, box, flux, h->variant);
}

int stage_blocks_per_sm(const sg_ctx* h) {
    return h->esize == 8 ? sg::Launch<double>::stage_prepare(h->dim, h->ppt, h->smem, h->variant)
                         : sg::Launch<float>::stage_prepare(h->dim, h->ppt, h->smem, h->variant);
}

cudaError_t launch_stage(const sg_ctx* h, const StageArgs& a, int nblocks) {
    return h->esize == 8 ? sg::Launch<double>::stage(h->dim, h->ppt, a, nblocks, h->smem, h->stream, h->variant)
                         : sg::Launch<float>::stage(h->dim, h->ppt, a, nblocks, h->smem, h->stream, h->variant);
}

// FP32 state: after a call in which instance i took an odd number of steps, U sits in the
// second buffer of the ping-pong pair; swap the pair in the grid tables so that u0 holds U
// again between calls.  `grids` are the instance's entries (a member's own table, or a slice
// of a batch table).
void swap_pair(GridDesc* grids, int n) {
    for (int g = 0; g < n; ++g) std::swap(grids[g].u0, grids[g].u1);
}

// Vlasov-Boltzmann: the density buffers and the table of mu_inf at every grid's velocity
// nodes, mu_inf(v) = exp(-(|v|^2 / (2 theta))) / (2 pi theta)^{d/2}, |v|^2 summed in axis order,
// v_k = lo_k + j h_k (evaluated on the host in FP64; the FP32 table holds the rounded values).
sg_status relax_tables(sg_ctx* h) {
    const int dx = h->dim / 2;
    long long ef_total = 0, mu_total = 0;
    for (int g = 0; g < h->G; ++g) {
        long long nx = 1, nv = 1;
        for (int k = 0; k < dx; ++k) nx *= (long long)h->nr << h->levels[g][k];
        for (int k = dx; k < h->dim; ++k) nv *= (long long)h->nr << h->levels[g][k];
        h->ef_offset.push_back(ef_total);
        h->mu_offset.push_back(mu_total);
        ef_total += nx;
        mu_total += nv;
        h->max_nx = std::max(h->max_nx, nx);
    }
    SG_TRY(h->efield.alloc((size_t)ef_total * h->esize));
    SG_TRY(h->mutab.alloc((size_t)mu_total * h->esize));
    std::vector<double> mu((size_t)mu_total);
    const double theta = h->prm.theta;
    const double norm = std::pow(2.0 * 3.14159265358979323846 * theta, 0.5 * (double)dx);
    for (int g = 0; g < h->G; ++g) {
        long long nv = 1;
        int n[SG_MAXD];
        double hk[SG_MAXD];
        for (int k = dx; k < h->dim; ++k) {
            n[k] = h->nr << h->levels[g][k];
            hk[k] = (h->prm.hi[k] - h->prm.lo[k]) / (double)n[k];
            nv *= n[k];
        }
        for (long long jv = 0; jv < nv; ++jv) {
            long long r = jv;
            double s2 = 0.0;
            for (int k = dx; k < h->dim; ++k) {
                const double v = h->prm.lo[k] + (double)(r % n[k]) * hk[k];
                r /= n[k];
                s2 = s2 + v * v;
            }
            mu[(size_t)(h->mu_offset[g] + jv)] = std::exp(-(s2 / (2.0 * theta))) / norm;
        }
    }
    if (h->esize == 8) {
        SG_CUDA(cudaMemcpy(h->mutab.p, mu.data(), sizeof(double) * mu.size(), cudaMemcpyHostToDevice));
    } else {
        std::vector<float> muf(mu.begin(), mu.end());
        SG_CUDA(cudaMemcpy(h->mutab.p, muf.data(), sizeof(float) * muf.size(), cudaMemcpyHostToDevice));
    }
    return SG_OK;
}

// Normalisation s of the Example 5 initial condition: the integral over the domain of
// prod_k factor_k, a product of one-axis integrals, each by the composite Simpson rule on
// 2 * 10^5 intervals.
double relax_norm(const sg_ctx* h) {
    const int dx = h->dim / 2;
    const long m = 200000;
    double s = 1.0;
    for (int k = 0; k < h->dim; ++k) {
        const double a = h->prm.lo[k], b = h->prm.hi[k], step = (b - a) / (double)m;
        auto f = [&](double x) {
            const double e = std::exp(-0.5 * x * x);
            if (k >= dx) return e;
            const double t = k == 0 ? std::sin(0.5 * x * x) : std::cos(0.5 * x * x);
            return t * t * e;
        };
        double acc = f(a) + f(b);
        for (long i = 1; i < m; ++i) acc += (i & 1 ? 4.0 : 2.0) * f(a + (double)i * step);
        s *= acc * step / 3.0;
    }
    return s;
}

sg_status validate_params(const sg_params* p, int dim) {
    if (p->struct_size != sizeof(sg_params)) return fail(SG_ERR_ARG, "sg_params.struct_size mismatch (use sg_params_init)");
    for (int k = 0; k < dim; ++k) {
        if (!(std::isfinite(p->lo[k]) && std::isfinite(p->hi[k]) && p->hi[k] > p->lo[k]))
            return fail(SG_ERR_ARG, "domain axis %d: need finite lo < hi", k);
        if (p->bc[k] != SG_BC_PERIODIC && p->bc[k] != SG_BC_ZERO)
            return fail(SG_ERR_ARG, "bc[%d] must be SG_BC_PERIODIC or SG_BC_ZERO", k);
        if (!std::isfinite(p->adv_speed[k])) return fail(SG_ERR_ARG, "adv_speed[%d] not finite", k);
    }
    if (p->precision != SG_F64 && p->precision != SG_F32) return fail(SG_ERR_ARG, "precision");
    if (p->exec != SG_PLAIN && p->exec != SG_BATCHED) return fail(SG_ERR_ARG, "exec");
    if (p->scheme != SG_WENO5 && p->scheme != SG_LINEAR5) return fail(SG_ERR_ARG, "scheme");
    if (p->prolong != SG_PROLONG_WENO5 && p->prolong != SG_PROLONG_LAGRANGE5) return fail(SG_ERR_ARG, "prolong");
    if (!(p->eps > 0.0) || !std::isfinite(p->eps)) return fail(SG_ERR_ARG, "eps must be > 0");
    if (p->dt_rule != SG_DT_POW53 && p->dt_rule != SG_DT_CFL) return fail(SG_ERR_ARG, "dt_rule");
    if (!(p->dt_coef > 0.0) || !(p->cfl > 0.0)) return fail(SG_ERR_ARG, "dt_coef and cfl must be > 0");
    if (p->tile_points != 0 && p->tile_points != 256 && p->tile_points != 512 && p->tile_points != 1024)
        return fail(SG_ERR_ARG, "tile_points must be 0, 256, 512 or 1024");
    if (p->stage_kernel != SG_STAGE_AUTO && p->stage_kernel != SG_STAGE_TILED && p->stage_kernel != SG_STAGE_SWEEP &&
        p->stage_kernel != SG_STAGE_SWEEP2)
        return fail(SG_ERR_ARG, "stage_kernel");
    if ((p->stage_kernel == SG_STAGE_SWEEP || p->stage_kernel == SG_STAGE_SWEEP2) && dim != 3)
        return fail(SG_ERR_UNSUPPORTED, "the sweep stage kernels are implemented for d = 3 only");
    if (p->stage_kernel == SG_STAGE_SWEEP2 && p->precision != SG_F32)
        return fail(SG_ERR_UNSUPPORTED, "the two-line sweep kernel is FP32 only");
    if (!(p->theta > 0.0) || !std::isfinite(p->theta) || !(p->tau > 0.0) || std::isnan(p->tau))
        return fail(SG_ERR_ARG, "theta must be finite and > 0, tau > 0");
    return SG_OK;
}

// Builds the device grid table and work queue of a single handle.
sg_status build_tables(sg_ctx* h) {
    const int pmax = 256 * h->ppt;
    char* base = h->arena.as<char>();
    const size_t region = (size_t)h->total_pts * h->esize;
    // a rebuild (reconfiguration) keeps the state buffers where they are: an FP32 handle's
    // ping-pong pair may be swapped
    std::vector<std::pair<void*, void*>> keep;
    if ((int)h->hgrids.size() == h->G)
        for (const GridDesc& d : h->hgrids) keep.emplace_back(d.u0, d.u1);
    h->hgrids.assign(h->G, GridDesc{});
    h->hitems.clear();
    for (int g = 0; g < h->G; ++g) {
        GridDesc& d = h->hgrids[g];
        d.u0 = keep.empty() ? base + (size_t)h->offset[g] * h->esize : keep[g].first;
        d.u1 = keep.empty() ? base + region + (size_t)h->offset[g] * h->esize : keep[g].second;
        d.u2 = base + 2 * region + (size_t)h->offset[g] * h->esize;
        d.u3 = h->esize == 4 ? base + 3 * region + (size_t)h->offset[g] * h->esize : nullptr;
        d.ef = h->pde == SG_PDE_VLASOV || h->pde == SG_PDE_VLASOV_BOLTZMANN
                   ? h->efield.as<char>() + (size_t)h->ef_offset[g] * h->esize : nullptr;
        d.mu = h->pde == SG_PDE_VLASOV_BOLTZMANN ? h->mutab.as<char>() + (size_t)h->mu_offset[g] * h->esize : nullptr;
        d.npts = h->npts[g];
        int n[SG_MAXD] = {1, 1, 1, 1, 1, 1};
        for (int k = 0; k < h->dim; ++k) n[k] = h->nr << h->levels[g][k];
        if (h->dim == 3 && (h->variant == 0 || h->variant == 3)) sg::sweep_tile(n, d.te);
        else choose_tile(n, h->dim, pmax, d.te);
        int ntiles = 1;
        for (int k = 0; k < SG_MAXD; ++k) {
            if (k < h->dim) {
                d.n[k] = n[k];
                d.nt[k] = (n[k] + d.te[k] - 1) / d.te[k];
                d.ntmag[k] = sg_div_magic64((unsigned)d.nt[k]);
                d.h[k] = (h->prm.hi[k] - h->prm.lo[k]) / (double)n[k];
                d.rdx[k] = 1.0 / d.h[k];
                d.rdxf[k] = (float)d.rdx[k];
                d.lo[k] = h->prm.lo[k];
                d.lev[k] = h->levels[g][k];
                ntiles *= d.nt[k];
            } else {
                d.n[k] = 1;
                d.te[k] = 1;
                d.nt[k] = 1;
                d.ntmag[k] = 0;
                d.h[k] = 1.0;
                d.rdx[k] = 1.0;
                d.rdxf[k] = 1.0f;
                d.lo[k] = 0.0;
                d.lev[k] = 0;
            }
        }
        d.coeff = h->coeff[g];
        d.inst = 0;
        d.first_item = (int)h->hitems.size();
        d.n_items = ntiles;
        for (int t = 0; t < ntiles; ++t) h->hitems.push_back(WorkItem{g, t});
    }
    SG_TRY(h->dgrids.alloc(sizeof(GridDesc) * h->hgrids.size()));
    SG_TRY(h->ditems.alloc(sizeof(WorkItem) * h->hitems.size()));
    SG_CUDA(cudaMemcpy(h->dgrids.p, h->hgrids.data(), sizeof(GridDesc) * h->hgrids.size(), cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(h->ditems.p, h->hitems.data(), sizeof(WorkItem) * h->hitems.size(), cudaMemcpyHostToDevice));
    return SG_OK;
}

sg_status alloc_step_buffers(sg_ctx* h, int ngrids_total, int ninst) {
    SG_TRY(h->alpha.alloc(sizeof(unsigned long long) * 3 * (size_t)ngrids_total));
    SG_TRY(h->flags.alloc(sizeof(int) * 4));
    SG_TRY(h->dinst.alloc(sizeof(InstState) * (size_t)ninst));
    SG_TRY(h->partial.alloc(sizeof(double) * 1032));
    SG_TRY(h->hinst.alloc(ninst));
    h->ninst = ninst;
    SG_CUDA(cudaMemset(h->alpha.p, 0, h->alpha.bytes));
    SG_CUDA(cudaMemset(h->flags.p, 0, h->flags.bytes));
    stage_footprint(h);
    const int bps = stage_blocks_per_sm(h);
    if (bps < 1) return fail(SG_ERR_CUDA, "stage kernel cannot be resident (dim %d, %d points/thread)", h->dim, h->ppt);
    h->blocks_total = bps * num_sms();
    return SG_OK;
}

sg_status ensure_events(sg_ctx* h, int pairs) {
    while ((int)h->ev.size() < 2 * pairs) {
        cudaEvent_t e;
        SG_CUDA(cudaEventCreate(&e));
        h->ev.push_back(e);
    }
    return SG_OK;
}

// Vlasov-Poisson: the field of every grid of the handle (or batch) from the stage input.
cudaError_t launch_efield(const sg_ctx* h, int stage, int pre_dt) {
    const int ng = (int)h->hgrids.size();
    return h->esize == 8
               ? sg::Launch<double>::efield(h->dgrids.as<GridDesc>(), ng, h->dinst.as<InstState>(),
                                            h->alpha.as<unsigned long long>(), stage, pre_dt, h->stream)
               : sg::Launch<float>::efield(h->dgrids.as<GridDesc>(), ng, h->dinst.as<InstState>(),
                                           h->alpha.as<unsigned long long>(), stage, pre_dt, h->stream);
}

// Vlasov-Boltzmann: the density of every grid of the handle (or batch) from the stage input.
cudaError_t launch_density(const sg_ctx* h, int stage) {
    const int ng = (int)h->hgrids.size();
    return h->esize == 8 ? sg::Launch<double>::density(h->dgrids.as<GridDesc>(), ng, h->max_nx, h->dinst.as<InstState>(),
                                                       stage, h->dim, h->stream)
                         : sg::Launch<float>::density(h->dgrids.as<GridDesc>(), ng, h->max_nx, h->dinst.as<InstState>(),
                                                      stage, h->dim, h->stream);
}

// Enqueues `nsteps` time steps (dt control + three RK stages each) on the handle's stream.
// With profiling on, each stage launch (or per-grid launch group) is bracketed by an event pair.
sg_status enqueue_steps(sg_ctx* h, int nsteps, long long* kernels) {
    const PhysParams ph = phys_of(h);
    long long nk = 0;
    if (h->profile) SG_TRY(ensure_events(h, 3 * nsteps));
    h->ev_pairs_used = h->profile ? 3 * nsteps : 0;
    for (int s = 0; s < nsteps; ++s) {
        if (h->pde == SG_PDE_VLASOV) {  // E of the step's input first: the CFL step needs max|E|
            SG_CUDA(launch_efield(h, 0, 1));
            ++nk;
        }
        SG_CUDA(sg::launch_dt(h->dinst.as<InstState>(), h->ninst, h->dgrids.as<GridDesc>(),
                              h->alpha.as<unsigned long long>(), ph, 0, h->flags.as<int>(), h->stream));
        ++nk;
        for (int stage = 0; stage < 3; ++stage) {
            StageArgs a{};
            a.grids = h->dgrids.as<GridDesc>();
            a.items = h->ditems.as<WorkItem>();
            a.inst = h->dinst.as<InstState>();
            a.alpha = h->alpha.as<unsigned long long>();
            a.flags = h->flags.as<int>();
            a.stage = stage;
            a.phys = ph;
            a.box_elems = (int)h->box_elems;
            const int pair = 3 * s + stage;
            if (h->pde == SG_PDE_VLASOV && stage > 0) {
                SG_CUDA(launch_efield(h, stage, 0));
                ++nk;
            }
            if (h->pde == SG_PDE_VLASOV_BOLTZMANN) {  // rho of the stage input
                SG_CUDA(launch_density(h, stage));
                ++nk;
            }
            if (h->profile) SG_CUDA(cudaEventRecordWithFlags(h->ev[2 * pair], h->stream, cudaEventRecordExternal));
            const bool batched = h->is_batch || h->prm.exec == SG_BATCHED;
            if (batched) {
                a.item_begin = 0;
                a.item_end = (int)h->hitems.size();
                SG_CUDA(launch_stage(h, a, std::min<int>(a.item_end, h->blocks_total)));
                ++nk;
            } else {
                for (const GridDesc& d : h->hgrids) {
                    a.item_begin = d.first_item;
                    a.item_end = d.first_item + d.n_items;
                    SG_CUDA(launch_stage(h, a, std::min<int>(d.n_items, h->blocks_total)));
                    ++nk;
                }
            }
            if (h->profile) SG_CUDA(cudaEventRecordWithFlags(h->ev[2 * pair + 1], h->stream, cudaEventRecordExternal));
        }
    }
    *kernels = nk;
    return SG_OK;
}

// After the enqueued steps completed: add the stage-launch times to the profile.
sg_status collect_profile(sg_ctx* h) {
    if (!h->profile) return SG_OK;
    const bool batched = h->is_batch || h->prm.exec == SG_BATCHED;
    for (int j = 0; j < h->ev_pairs_used; ++j) {
        float ms = 0.f;
        SG_CUDA(cudaEventElapsedTime(&ms, h->ev[2 * j], h->ev[2 * j + 1]));
        h->prof_ms += ms;
        h->prof_launches += batched ? 1 : (long long)h->hgrids.size();
    }
    return SG_OK;
}

sg_status ensure_graph(sg_ctx* h, int nsteps) {
    if (h->graph && h->graph_nsteps == nsteps && h->graph_profiled == h->profile) {
        h->ev_pairs_used = h->profile ? 3 * nsteps : 0;
        return SG_OK;
    }
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    SG_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    long long nk = 0;
    sg_status st = enqueue_steps(h, nsteps, &nk);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (st != SG_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SG_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->graph = nullptr;
        return fail(SG_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    h->graph_nsteps = nsteps;
    h->graph_kernels = nk;
    h->graph_profiled = h->profile;
    return SG_OK;
}

// A batch's grid table and work queue: its members' tables concatenated, grid g of member i
// owned by instance i.  Uploaded to the device.
sg_status build_batch_tables(sg_ctx* h) {
    h->hgrids.clear();
    h->hitems.clear();
    h->max_grid_pts = 0;
    for (size_t i = 0; i < h->members.size(); ++i) {
        const sg_ctx* m = h->members[i];
        for (const GridDesc& d0 : m->hgrids) {
            GridDesc d = d0;
            d.inst = (int)i;
            d.first_item = (int)h->hitems.size();
            const int g = (int)h->hgrids.size();
            for (int t = 0; t < d.n_items; ++t) h->hitems.push_back(WorkItem{g, t});
            h->hgrids.push_back(d);
        }
        h->max_grid_pts = std::max(h->max_grid_pts, m->max_grid_pts);
        h->max_nx = std::max(h->max_nx, m->max_nx);
    }
    if (h->dgrids.bytes < sizeof(GridDesc) * h->hgrids.size()) SG_TRY(h->dgrids.alloc(sizeof(GridDesc) * h->hgrids.size()));
    if (h->ditems.bytes < sizeof(WorkItem) * h->hitems.size()) SG_TRY(h->ditems.alloc(sizeof(WorkItem) * h->hitems.size()));
    SG_CUDA(cudaMemcpy(h->dgrids.p, h->hgrids.data(), sizeof(GridDesc) * h->hgrids.size(), cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(h->ditems.p, h->hitems.data(), sizeof(WorkItem) * h->hitems.size(), cudaMemcpyHostToDevice));
    return SG_OK;
}

void drop_graph(sg_ctx* h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_nsteps = 0;
}

// Stage-kernel configuration: kernel variant and points per thread (tile size); rebuilds the
// tiles and work queues (of every member, for a batch) and drops the captured graph.
sg_status configure(sg_ctx* h, int variant, int ppt) {
    if (h->is_batch) {
        for (sg_ctx* m : h->members) {
            m->variant = variant;
            m->ppt = ppt;
            SG_TRY(build_tables(m));
            stage_footprint(m);
            m->tuned = true;
            drop_graph(m);
        }
        SG_TRY(build_batch_tables(h));
    }
    h->variant = variant;
    h->ppt = ppt;
    if (!h->is_batch) SG_TRY(build_tables(h));
    if (h->is_batch) {
        for (sg_ctx* m : h->members) {  // members keep a runnable configuration of their own
            const int b = stage_blocks_per_sm(m);
            if (b < 1) return fail(SG_ERR_CUDA, "stage kernel cannot be resident");
            m->blocks_total = b * num_sms();
        }
    }
    stage_footprint(h);
    const int bps = stage_blocks_per_sm(h);
    if (bps < 1) return fail(SG_ERR_CUDA, "stage kernel cannot be resident (dim %d, variant %d, %d points/thread)",
                             h->dim, variant, ppt);
    h->blocks_total = bps * num_sms();
    drop_graph(h);
    return SG_OK;
}

// Autotuner (SG_STAGE_AUTO with tile_points = 0): the first sg_step of a handle or batch
// times one RK-stage launch of each candidate configuration (stage 0 with dt = 0: it writes
// only the first-stage buffer and an alpha slot, both of which the step itself rewrites) and
// keeps the fastest.  Candidates: the tiled kernel with 256-, 512- and 1024-point tiles, and
// for d = 3 the sweep kernel in place of the 256-point tile (FP32: also the two-line sweep).  Choices are cached per
// (dimension, precision, pde, scheme, batch or not, size class) for the life of the process.
struct TuneKey {
    int dim, esize, pde, scheme, batched, size_class;
    bool operator<(const TuneKey& o) const {
        return std::tie(dim, esize, pde, scheme, batched, size_class) <
               std::tie(o.dim, o.esize, o.pde, o.scheme, o.batched, o.size_class);
    }
};
std::map<TuneKey, std::tuple<int, int, double>> g_tuned;  // variant, ppt, ms
std::mutex g_tune_mutex;

sg_status time_stage0(sg_ctx* h, double* ms) {
    for (int i = 0; i < h->ninst; ++i) {
        InstState& s = h->hinst.p[i];
        s.active = 1;
        s.dt = 0.0;
        s.dtf = 0.0f;
        s.steps = s.step0 = 0;
    }
    SG_CUDA(cudaMemcpyAsync(h->dinst.p, h->hinst.p, sizeof(InstState) * h->ninst, cudaMemcpyHostToDevice, h->stream));
    SG_CUDA(cudaMemsetAsync(h->alpha.p, 0, h->alpha.bytes, h->stream));
    if (h->pde == SG_PDE_VLASOV) SG_CUDA(launch_efield(h, 0, 0));
    if (h->pde == SG_PDE_VLASOV_BOLTZMANN) SG_CUDA(launch_density(h, 0));
    cudaEvent_t e0, e1;
    SG_CUDA(cudaEventCreate(&e0));
    SG_CUDA(cudaEventCreate(&e1));
    StageArgs a{};
    a.grids = h->dgrids.as<GridDesc>();
    a.items = h->ditems.as<WorkItem>();
    a.inst = h->dinst.as<InstState>();
    a.alpha = h->alpha.as<unsigned long long>();
    a.flags = h->flags.as<int>();
    a.stage = 0;
    a.phys = phys_of(h);
    a.box_elems = (int)h->box_elems;
    const bool batched = h->is_batch || h->prm.exec == SG_BATCHED;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {  // one warm-up, three timed
        if (rep == 1) err = cudaEventRecord(e0, h->stream);
        if (batched) {
            a.item_begin = 0;
            a.item_end = (int)h->hitems.size();
            if (err == cudaSuccess) err = launch_stage(h, a, std::min<int>(a.item_end, h->blocks_total));
        } else {
            for (const GridDesc& d : h->hgrids) {
                a.item_begin = d.first_item;
                a.item_end = d.first_item + d.n_items;
                if (err == cudaSuccess) err = launch_stage(h, a, std::min<int>(d.n_items, h->blocks_total));
            }
        }
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, h->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SG_CUDA(err);
    SG_CUDA(cudaMemsetAsync(h->flags.p, 0, h->flags.bytes, h->stream));
    *ms = t / 3.0;
    return SG_OK;
}

sg_status autotune(sg_ctx* h) {
    if (h->tuned) return SG_OK;
    long long pts = 0;
    for (const GridDesc& d : h->hgrids) pts += d.npts;
    int size_class = 0;
    while ((1LL << size_class) < pts) ++size_class;
    const TuneKey key{h->dim, h->esize, h->pde, h->prm.scheme, (int)(h->is_batch || h->prm.exec == SG_BATCHED),
                      size_class};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto f = g_tuned.find(key);
        if (f != g_tuned.end()) {
            SG_TRY(configure(h, std::get<0>(f->second), std::get<1>(f->second)));
            h->tuned = true;
            h->tune_ms = std::get<2>(f->second);
            return SG_OK;
        }
    }
    std::vector<std::pair<int, int>> cand;
    if (h->pde == SG_PDE_VLASOV_BOLTZMANN) cand = {{2, 1}, {2, 2}, {2, 4}};
    else if (h->dim == 3 && h->esize == 4) cand = {{3, 2}, {0, 2}, {1, 2}, {1, 4}};
    else if (h->dim == 3) cand = {{0, 2}, {1, 2}, {1, 4}};
    else cand = {{0, 1}, {0, 2}, {0, 4}};
    double best = INFINITY;
    std::pair<int, int> pick = cand[0];
    for (const auto& c : cand) {
        sg_status st = configure(h, c.first, c.second);
        if (st != SG_OK) continue;  // a candidate that cannot run is skipped
        double ms = INFINITY;
        if (time_stage0(h, &ms) != SG_OK) continue;
        if (ms < best) {
            best = ms;
            pick = c;
        }
    }
    SG_TRY(configure(h, pick.first, pick.second));
    h->tuned = true;
    h->tune_ms = std::isfinite(best) ? best : 0.0;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[key] = std::make_tuple(pick.first, pick.second, h->tune_ms);
    return SG_OK;
}

// Would the next dt-control pass mark this instance inactive?  Mirrors sg_dt_kernel.
bool finished(const InstState& s) {
    if (!s.active) return true;
    const double t = s.last ? s.t_end : s.t + s.dt;
    const long long n = s.steps + 1;
    return !(t < s.t_end && n < s.step_limit);
}

// Step loop shared by single handles and batches; h->hinst holds the members' states.
sg_status run_steps(sg_ctx* h) {
    SG_CUDA(cudaMemcpyAsync(h->dinst.p, h->hinst.p, sizeof(InstState) * h->ninst, cudaMemcpyHostToDevice, h->stream));
    SG_CUDA(cudaMemsetAsync(h->alpha.p, 0, h->alpha.bytes, h->stream));
    SG_CUDA(cudaMemsetAsync(h->flags.p, 0, h->flags.bytes, h->stream));
    const int ng = (int)h->hgrids.size();
    if (h->esize == 8)
        SG_CUDA(sg::Launch<double>::alpha_init(h->dgrids.as<GridDesc>(), ng, h->max_grid_pts, h->alpha.as<unsigned long long>(), h->flags.as<int>(), h->stream));
    else
        SG_CUDA(sg::Launch<float>::alpha_init(h->dgrids.as<GridDesc>(), ng, h->max_grid_pts, h->alpha.as<unsigned long long>(), h->flags.as<int>(), h->stream));
    h->launches += 1;
    const int K = h->prm.graph_steps == 0 ? 16 : (h->prm.graph_steps < 0 ? 8 : h->prm.graph_steps);
    const bool use_graph = h->prm.graph_steps >= 0;
    if (use_graph) SG_TRY(ensure_graph(h, K));
    for (;;) {
        if (use_graph) {
            SG_CUDA(cudaGraphLaunch(h->graph, h->stream));
            h->launches += h->graph_kernels;
        } else {
            long long nk = 0;
            SG_TRY(enqueue_steps(h, K, &nk));
            h->launches += nk;
        }
        int lflags[4] = {0, 0, 0, 0};
        SG_CUDA(cudaMemcpyAsync(h->hinst.p, h->dinst.p, sizeof(InstState) * h->ninst, cudaMemcpyDeviceToHost, h->stream));
        SG_CUDA(cudaMemcpyAsync(lflags, h->flags.p, sizeof lflags, cudaMemcpyDeviceToHost, h->stream));
        SG_CUDA(cudaStreamSynchronize(h->stream));
        SG_TRY(collect_profile(h));
        bool all = true;
        for (int i = 0; i < h->ninst; ++i) all = all && finished(h->hinst.p[i]);
        if (all || lflags[SG_FLAG_NONFINITE] || lflags[SG_FLAG_BADDT]) break;  // done, or failed: stop early
    }
    SG_CUDA(sg::launch_dt(h->dinst.as<InstState>(), h->ninst, h->dgrids.as<GridDesc>(),
                          h->alpha.as<unsigned long long>(), phys_of(h), 1, h->flags.as<int>(), h->stream));
    h->launches += 1;
    int hflags[4] = {0, 0, 0, 0};
    SG_CUDA(cudaMemcpyAsync(h->hinst.p, h->dinst.p, sizeof(InstState) * h->ninst, cudaMemcpyDeviceToHost, h->stream));
    SG_CUDA(cudaMemcpyAsync(hflags, h->flags.p, sizeof hflags, cudaMemcpyDeviceToHost, h->stream));
    SG_CUDA(cudaStreamSynchronize(h->stream));
    if (hflags[SG_FLAG_NONFINITE]) return fail(SG_ERR_NONFINITE, "a non-finite value appeared in the solution");
    if (hflags[SG_FLAG_BADDT]) return fail(SG_ERR_NONFINITE, "the time step came out non-positive or non-finite");
    return SG_OK;
}

// Axes with zero values beyond the ends: v of the Vlasov-Poisson system, every axis of the
// Vlasov-Boltzmann model, the SG_BC_ZERO axes of advection and Burgers; the others are periodic.
bool zero_axis(const sg_ctx* h, int k) {
    return (h->pde == SG_PDE_VLASOV && k == 1) || h->pde == SG_PDE_VLASOV_BOLTZMANN ||
           ((h->pde == SG_PDE_ADVECTION || h->pde == SG_PDE_BURGERS) && h->prm.bc[k] == SG_BC_ZERO);
}

// Prolongation of every grid onto the finest grid and the combination sum, one grid at a time:
// the last prolonged axis of each grid adds c_g times its values into uhat (a read-modify-write
// of uhat per grid).  Used when the fused form's intermediates exceed the memory budget.
template <class T>
sg_status prolong_combine_rmw_t(sg_ctx* h, cudaStream_t st, bool sync) {
    const int d = h->dim;
    const long long Nf = (long long)h->nr << h->nl;
    // intermediate buffers: largest array produced by a non-final prolonged axis
    long long need = 1;
    for (int g = 0; g < h->G; ++g) {
        long long m[SG_MAXD];
        std::vector<int> axes;
        for (int k = 0; k < d; ++k) {
            m[k] = (long long)h->nr << h->levels[g][k];
            if (h->levels[g][k] < h->nl) axes.push_back(k);
        }
        for (size_t a = 0; a + 1 < axes.size(); ++a) {
            m[axes[a]] = Nf;
            long long tot = 1;
            for (int k = 0; k < d; ++k) tot *= m[k];
            need = std::max(need, tot);
        }
    }
    if (!h->uhat.p) SG_TRY(h->uhat.alloc(sizeof(double) * (size_t)h->fine_pts));
    if (h->pro_a.bytes < sizeof(T) * (size_t)need) {
        SG_TRY(h->pro_a.alloc(sizeof(T) * (size_t)need));
        SG_TRY(h->pro_b.alloc(sizeof(T) * (size_t)need));
    }
    double* acc = h->uhat.as<double>();
    SG_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)h->fine_pts, st));
    for (int g = 0; g < h->G; ++g) {
        const GridDesc& gd = h->hgrids[g];
        long long m[SG_MAXD];
        std::vector<int> axes;
        for (int k = 0; k < d; ++k) {
            m[k] = gd.n[k];
            if (gd.lev[k] < h->nl) axes.push_back(k);
        }
        const T* src = (const T*)gd.u0;
        if (axes.empty()) {
            SG_CUDA(sg::Launch<T>::accumulate(src, acc, gd.coeff, gd.npts, st));
            h->launches += 1;
            continue;
        }
        T* bufs[2] = {h->pro_a.as<T>(), h->pro_b.as<T>()};
        for (size_t a = 0; a < axes.size(); ++a) {
            const int k = axes[a];
            long long below = 1, above = 1;
            for (int j = 0; j < k; ++j) below *= m[j];
            for (int j = k + 1; j < d; ++j) above *= m[j];
            const int r = 1 << (h->nl - gd.lev[k]);
            const bool last = a + 1 == axes.size();
            T* dst = last ? nullptr : bufs[a & 1];
            SG_CUDA(sg::Launch<T>::prolong_axis(src, dst, last ? acc : nullptr, gd.coeff, below, (int)m[k],
                                                (int)Nf, above, r, h->prm.eps, h->prm.prolong,
                                                zero_axis(h, k) ? 1 : 0, st));
            h->launches += 1;
            m[k] = Nf;
            src = dst;
        }
    }
    if (sync) SG_CUDA(cudaStreamSynchronize(st));
    h->combined = true;
    return SG_OK;
}

// Fused form (Step 3): phase 1 prolongs every grid over axes 0..d-2 into a pool slot (the
// grid itself if none of those axes is coarse), one launch per axis for all grids (a pass over
// a task table; a grid's intermediate arrays get slots of their own); phase 2 prolongs the last
// axis of all grids and forms sum_g c_g P U_g in one pass that writes uhat once.  Buffers come
// from `cb` (the handle's own, or a batch's, shared by its members).  Returns
// SG_ERR_UNSUPPORTED (without touching anything) when the intermediates would exceed the
// budget.
template <class T>
sg_status prolong_combine_fused_t(sg_ctx* h, CombineBuffers& cb, cudaStream_t st, bool sync) {
    constexpr int J = 8;  // fine nodes per unit of a prolongation pass (sg_prolong_multi_kernel)
    const int d = h->dim;
    const long long Nf = (long long)h->nr << h->nl;
    const long long nch = (Nf + J - 1) / J;
    long long below = 1;
    for (int k = 0; k + 1 < d; ++k) below *= Nf;
    // plan: per pass (axis k < d-1) the tasks of the grids coarse on axis k; slots in the pool
    // (each grid's last prolonged axis) and in the intermediate buffer (the others).  Grids are
    // taken in groups whose intermediates fit beside the pool in the budget; each group runs
    // its passes in axis order and reuses the intermediate buffer of the previous group.
    struct Plan {
        int g;
        long long in_off, out_off;  // element offsets: in: -1 = the grid itself, else intermediate;
        bool out_pool;              // out: pool slot or intermediate
        long long below, above;
        int n, r, zero;
    };
    const double budget = h->prm.combine_budget_gb == 0.0 ? 8.0e9 : h->prm.combine_budget_gb * 1e9;
    if (budget < 0.0) return SG_ERR_UNSUPPORTED;
    long long pool = 0;
    std::vector<long long> slot(h->G, -1), gint(h->G, 0);  // pool slot, intermediate elements
    for (int g = 0; g < h->G; ++g) {
        const GridDesc& gd = h->hgrids[g];
        long long m[SG_MAXD];
        int last = -1;
        for (int k = 0; k < d; ++k) {
            m[k] = gd.n[k];
            if (k + 1 < d && gd.lev[k] < h->nl) last = k;
        }
        if (last < 0) continue;
        slot[g] = pool;
        pool += below * m[d - 1];
        for (int k = 0; k < last; ++k) {  // every coarse axis before the last one leaves an array
            if (gd.lev[k] >= h->nl) continue;
            m[k] = Nf;
            long long tot = 1;
            for (int j = 0; j < d; ++j) tot *= m[j];
            gint[g] += tot;
        }
    }
    const double room = budget / sizeof(T) - (double)pool;  // elements left for intermediates
    long long gmax = 0;
    for (long long v : gint) gmax = std::max(gmax, v);
    if (room < (double)gmax) return SG_ERR_UNSUPPORTED;
    std::vector<std::vector<int>> groups(1);
    long long interm = 0, cur = 0;
    for (int g = 0; g < h->G; ++g) {
        if (slot[g] < 0) continue;
        if ((double)(cur + gint[g]) > room) {
            groups.emplace_back();
            cur = 0;
        }
        groups.back().push_back(g);
        cur += gint[g];
        interm = std::max(interm, cur);
    }
    // passes[group][k]
    std::vector<std::vector<std::vector<Plan>>> passes(groups.size(), std::vector<std::vector<Plan>>(d > 1 ? d - 1 : 1));
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        long long ioff = 0;
        for (int g : groups[gi]) {
            const GridDesc& gd = h->hgrids[g];
            long long m[SG_MAXD];
            std::vector<int> axes;
            for (int k = 0; k < d; ++k) {
                m[k] = gd.n[k];
                if (k + 1 < d && gd.lev[k] < h->nl) axes.push_back(k);
            }
            long long in_off = -1;
            for (size_t a = 0; a < axes.size(); ++a) {
                const int k = axes[a];
                Plan pl{};
                pl.g = g;
                pl.in_off = in_off;
                pl.below = 1;
                pl.above = 1;
                for (int j = 0; j < k; ++j) pl.below *= m[j];
                for (int j = k + 1; j < d; ++j) pl.above *= m[j];
                pl.n = (int)m[k];
                pl.r = 1 << (h->nl - gd.lev[k]);
                pl.zero = zero_axis(h, k) ? 1 : 0;
                m[k] = Nf;
                pl.out_pool = a + 1 == axes.size();
                if (pl.out_pool) {
                    pl.out_off = slot[g];
                } else {
                    long long tot = 1;
                    for (int j = 0; j < d; ++j) tot *= m[j];
                    pl.out_off = ioff;
                    ioff += tot;
                }
                in_off = pl.out_off;
                passes[gi][k].push_back(pl);
            }
        }
    }
    // the pass kernel indexes a task's units and columns with 32 bits
    size_t ntask = 0;
    for (const auto& gp : passes)
        for (const auto& ps : gp) {
            ntask += ps.size();
            for (const Plan& pl : ps)
                if ((double)pl.below * (double)nch * (double)pl.above >= 2147483648.0 || pl.below >= (1LL << 31))
                    return SG_ERR_UNSUPPORTED;
        }
    if (!h->uhat.p) SG_TRY(h->uhat.alloc(sizeof(double) * (size_t)h->fine_pts));
    if (cb.pool.bytes < sizeof(T) * (size_t)std::max(pool, 1LL)) SG_TRY(cb.pool.alloc(sizeof(T) * (size_t)std::max(pool, 1LL)));
    if (cb.pa.bytes < sizeof(T) * (size_t)std::max(interm, 1LL)) SG_TRY(cb.pa.alloc(sizeof(T) * (size_t)std::max(interm, 1LL)));
    const size_t tab_bytes = sizeof(CombineGrid) * (size_t)h->G, ptab_off = (tab_bytes + 255) & ~(size_t)255;
    const size_t all_bytes = ptab_off + sizeof(ProlongTask) * std::max<size_t>(ntask, 1);
    if (cb.tab.bytes < all_bytes) SG_TRY(cb.tab.alloc(all_bytes));
    // host copy of both tables, uploaded with one copy
    std::vector<unsigned char> host(all_bytes, 0);
    CombineGrid* tab = reinterpret_cast<CombineGrid*>(host.data());
    ProlongTask* ptab = reinterpret_cast<ProlongTask*>(host.data() + ptab_off);
    T* poolp = cb.pool.as<T>();
    T* intp = cb.pa.as<T>();
    struct Launch1 {
        size_t first;
        int ntasks;
        long long units;
        bool pairs;  // FP32 tasks whose adjacent columns pair up (sg_prolong_multi_x2_kernel)
    };
    std::vector<Launch1> launches;  // per group, per pass, in order
    size_t ti = 0;
    for (const auto& gp : passes)
        for (const auto& ps : gp) {  // passes in axis order: a grid's axes run 0, 1, ..., d-2
            // the pass's tasks in two launches: those whose columns pair up, then the others
            for (int kind = 0; kind < 2; ++kind) {
                long long unit0 = 0;
                const size_t first = ti;
                for (const Plan& pl : ps) {
                    const GridDesc& gd = h->hgrids[pl.g];
                    const void* in = pl.in_off < 0 ? (const void*)gd.u0 : (const void*)(intp + pl.in_off);
                    void* out = pl.out_pool ? (void*)(poolp + pl.out_off) : (void*)(intp + pl.out_off);
                    const bool pairs = sizeof(T) == 4 && pl.below % 2 == 0 &&
                                       ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 7) == 0;
                    if (pairs != (kind == 0)) continue;
                    ProlongTask& t = ptab[ti++];
                    t.in = in;
                    t.out = out;
                    t.unit0 = unit0;
                    t.below = (int)pl.below;
                    t.above = (int)pl.above;
                    t.n = pl.n;
                    t.nf = (int)Nf;
                    t.r = pl.r;
                    t.zero_bc = pl.zero;
                    t.below_mag = sg_div_magic64((unsigned)pl.below);
                    t.nch_mag = sg_div_magic64((unsigned)nch);
                    unit0 += pl.below * nch * pl.above;
                }
                if (ti > first) launches.push_back({first, (int)(ti - first), unit0, kind == 0});
            }
        }
    for (int g = 0; g < h->G; ++g) {
        const GridDesc& gd = h->hgrids[g];
        tab[g].src = slot[g] < 0 ? (const void*)gd.u0 : (const void*)(poolp + slot[g]);
        tab[g].n = gd.n[d - 1];
        tab[g].r = 1 << (h->nl - gd.lev[d - 1]);
        tab[g].coeff = gd.coeff;
        tab[g].coeff_f = (float)gd.coeff;
    }
    SG_CUDA(cudaMemcpyAsync(cb.tab.p, host.data(), all_bytes, cudaMemcpyHostToDevice, st));
    const ProlongTask* dptab = reinterpret_cast<const ProlongTask*>(cb.tab.as<unsigned char>() + ptab_off);
    for (const Launch1& L : launches) {
        if (L.pairs)
            SG_CUDA(sg::Launch<T>::prolong_multi_pairs(dptab + L.first, L.ntasks, L.units, h->prm.eps, h->prm.prolong, st));
        else
            SG_CUDA(sg::Launch<T>::prolong_multi(dptab + L.first, L.ntasks, L.units, h->prm.eps, h->prm.prolong, st));
        h->launches += 1;
    }
    bool exact = true;  // |c| = C(d-1, q) a power of two for every grid (d <= 3)
    for (int g = 0; g < h->G; ++g) {
        const double a = std::fabs(h->coeff[g]);
        exact = exact && a >= 1.0 && std::ldexp(1.0, std::ilogb(a)) == a;
    }
    bool aligned = (below & 1) == 0;  // both columns of every pair with one 8-byte load
    for (int g = 0; g < h->G; ++g) aligned = aligned && (reinterpret_cast<uintptr_t>(tab[g].src) & 7) == 0;
    SG_CUDA(sg::Launch<T>::combine_last_axis(cb.tab.as<CombineGrid>(), h->G, h->uhat.as<double>(), below, (int)Nf,
                                             exact ? 1 : 0, zero_axis(h, d - 1) ? 1 : 0, aligned ? 1 : 0,
                                             h->prm.eps, h->prm.prolong, st));
    h->launches += 1;
    if (sync) SG_CUDA(cudaStreamSynchronize(st));
    h->combined = true;
    return SG_OK;
}

template <class T>
sg_status prolong_combine_t(sg_ctx* h, CombineBuffers& cb, cudaStream_t st, bool sync) {
    const sg_status r = prolong_combine_fused_t<T>(h, cb, st, sync);
    if (r != SG_ERR_UNSUPPORTED) return r;
    return prolong_combine_rmw_t<T>(h, st, sync);
}

sg_status check_handle(sg_handle h) {
    if (!h) return fail(SG_ERR_ARG, "NULL handle");
    return SG_OK;
}

// Vlasov-Poisson field energy (1/2) sum_i E_i^2 h_x of grid `which` or of the combined solution.
sg_status field_energy(sg_ctx* h, int which, double* out) {
    if (h->pde != SG_PDE_VLASOV) return fail(SG_ERR_ARG, "the field energy needs the Vlasov-Poisson PDE");
    int n0, n1;
    double hx, hv;
    const void* u;
    const void* comp = nullptr;
    bool dbl = true;
    if (which == SG_WHICH_COMBINED) {
        if (!h->combined) return fail(SG_ERR_STATE, "no combined solution: call sg_prolong_combine first");
        n0 = n1 = (int)((long long)h->nr << h->nl);
        hx = fine_spacing(h, 0);
        hv = fine_spacing(h, 1);
        u = h->uhat.p;
    } else if (which >= 0 && which < h->G) {
        const GridDesc& d = h->hgrids[which];
        n0 = d.n[0];
        n1 = d.n[1];
        hx = d.h[0];
        hv = d.h[1];
        u = d.u0;
        comp = d.u3;
        dbl = h->esize == 8;
    } else {
        return fail(SG_ERR_ARG, "which = %d out of range", which);
    }
    DevBuf scratch;
    SG_TRY(scratch.alloc(sizeof(double) * (size_t)n0));
    double* dres = h->partial.as<double>() + 1024;
    if (dbl)
        SG_CUDA(sg::Launch<double>::field_energy((const double*)u, nullptr, n0, n1, hx, hv, scratch.as<double>(), dres, h->stream));
    else
        SG_CUDA(sg::Launch<float>::field_energy((const float*)u, (const float*)comp, n0, n1, hx, hv, scratch.as<double>(), dres, h->stream));
    h->launches += 1;
    double r = 0.0;
    SG_CUDA(cudaMemcpyAsync(&r, dres, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    SG_CUDA(cudaStreamSynchronize(h->stream));
    *out = r;
    return SG_OK;
}

}  // namespace

extern "C" {

sg_status sg_params_init(sg_params* p) {
    if (!p) return fail(SG_ERR_ARG, "NULL params");
    std::memset(p, 0, sizeof *p);
    p->struct_size = sizeof(sg_params);
    for (int k = 0; k < SG_MAX_DIM; ++k) {
        p->lo[k] = 0.0;
        p->hi[k] = 4.0;
        p->bc[k] = SG_BC_PERIODIC;
        p->adv_speed[k] = 1.0;
    }
    p->precision = SG_F64;
    p->exec = SG_PLAIN;
    p->scheme = SG_WENO5;
    p->prolong = SG_PROLONG_WENO5;
    p->eps = 1e-3;
    p->dt_rule = SG_DT_POW53;
    p->dt_coef = 1.0;
    p->cfl = 0.4;
    p->cuda_stream = nullptr;
    p->graph_steps = 0;
    p->tile_points = 0;
    p->combine_budget_gb = 0.0;
    p->stage_kernel = SG_STAGE_AUTO;
    p->theta = 1.0;
    p->tau = 1.0;
    return SG_OK;
}

sg_status sg_create(int dim, int root_cells, int level, int pde, const sg_params* params, sg_handle* out) {
    if (!out) return fail(SG_ERR_ARG, "NULL output handle");
    *out = nullptr;
    if (dim < 1 || dim > SG_MAX_DIM) return fail(SG_ERR_ARG, "dim must be in [1, 6]");
    if (root_cells < 5) return fail(SG_ERR_ARG, "root_cells must be >= 5 (five distinct stencil points)");
    if (level < 0 || level > 16 || ((long long)root_cells << level) > (1LL << 20))
        return fail(SG_ERR_ARG, "level must be in [0, 16] with root_cells * 2^level <= 2^20");
    if (pde != SG_PDE_ADVECTION && pde != SG_PDE_BURGERS && pde != SG_PDE_VLASOV && pde != SG_PDE_VLASOV_BOLTZMANN)
        return fail(SG_ERR_ARG, "pde");
    if (pde == SG_PDE_VLASOV && dim != 2) return fail(SG_ERR_ARG, "the Vlasov-Poisson system is 1D1V: dim must be 2");
    if (pde == SG_PDE_VLASOV_BOLTZMANN && dim != 2 && dim != 4 && dim != 6)
        return fail(SG_ERR_ARG, "the Vlasov-Boltzmann model has d space and d velocity axes: dim must be 2, 4 or 6");
    sg_params prm;
    if (params) prm = *params;
    else sg_params_init(&prm);
    SG_TRY(validate_params(&prm, dim));
    try {
        sg_ctx* h = new sg_ctx();
        h->dim = dim;
        h->nr = root_cells;
        h->nl = level;
        h->pde = pde;
        h->prm = prm;
        h->esize = prm.precision == SG_F64 ? 8 : 4;
        h->ppt = prm.tile_points ? prm.tile_points / 256 : 2;
        // d = 3: variant 0 is the sweep kernel, 1 the padded box; other dimensions have one
        const bool autotuned = prm.stage_kernel == SG_STAGE_AUTO && prm.tile_points == 0;
        h->variant = dim == 3 && (autotuned || prm.stage_kernel == SG_STAGE_SWEEP) ? 0 : (dim == 3 ? 1 : 0);
        if (dim == 3 && prm.stage_kernel == SG_STAGE_SWEEP2) h->variant = 3;
        if (pde == SG_PDE_VLASOV_BOLTZMANN) {  // the line-buffer kernel carries the kinetic terms
            if (prm.stage_kernel == SG_STAGE_SWEEP || prm.stage_kernel == SG_STAGE_SWEEP2) {
                delete h;
                return fail(SG_ERR_UNSUPPORTED, "the Vlasov-Boltzmann model runs on the tiled kernel");
            }
            h->variant = 2;
        }
        h->tuned = !autotuned;
        // grid set: |l| = N_L - q, q = 0..d-1, coefficient (-1)^q C(d-1, q)
        for (int q = 0; q < dim && level - q >= 0; ++q) {
            std::vector<std::array<int, SG_MAXD>> ls;
            std::array<int, SG_MAXD> cur{};
            compositions(dim, level, 0, level - q, cur, ls);
            for (auto& l : ls) {
                h->levels.push_back(l);
                h->coeff.push_back((q % 2 ? -1.0 : 1.0) * (double)binom(dim - 1, q));
            }
        }
        h->G = (int)h->levels.size();
        h->total_pts = 0;
        for (int g = 0; g < h->G; ++g) {
            long long n = 1;
            for (int k = 0; k < dim; ++k) {
                n *= (long long)root_cells << h->levels[g][k];  // < 2^31 * 2^20: no overflow
                if (n >= (1LL << 31)) {  // the stage kernels index within a grid with 32-bit offsets
                    delete h;
                    return fail(SG_ERR_UNSUPPORTED, "component grid %d has 2^31 or more points", g);
                }
            }
            h->npts.push_back(n);
            h->offset.push_back(h->total_pts);
            h->total_pts += n;
            h->max_grid_pts = std::max(h->max_grid_pts, n);
        }
        h->fine_pts = 1;
        for (int k = 0; k < dim; ++k) h->fine_pts *= (long long)root_cells << level;
        if (prm.cuda_stream) {
            h->stream = (cudaStream_t)prm.cuda_stream;
        } else {
            cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                cudaGetLastError();
                delete h;
                return fail(SG_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
            }
            h->own_stream = true;
        }
        sg_status st = h->arena.alloc((size_t)h->total_pts * h->esize * (h->esize == 4 ? 4 : 3));
        if (st == SG_OK && pde == SG_PDE_VLASOV) {
            long long ef_total = 0;
            for (int g = 0; g < h->G; ++g) {
                h->ef_offset.push_back(ef_total);
                ef_total += (long long)root_cells << h->levels[g][0];
            }
            st = h->efield.alloc((size_t)ef_total * h->esize);
        }
        if (st == SG_OK && pde == SG_PDE_VLASOV_BOLTZMANN) st = relax_tables(h);
        if (st == SG_OK) st = build_tables(h);
        if (st == SG_OK) st = alloc_step_buffers(h, h->G, 1);
        if (st != SG_OK) {
            delete h;
            return st;
        }
        ++g_live_handles;
        *out = h;
        return SG_OK;
    } catch (const std::bad_alloc&) {
        return fail(SG_ERR_NOMEM, "host allocation failed");
    } catch (...) {
        return fail(SG_ERR_CUDA, "unexpected exception in sg_create");
    }
}

sg_status sg_init(sg_handle h, int ic_kind, const double* p, int n_params) {
    SG_TRY(check_handle(h));
    if (h->is_batch) return fail(SG_ERR_ARG, "sg_init applies to batch members, not to the batch");
    if (ic_kind == SG_IC_LANDAU) {
        if (h->pde != SG_PDE_VLASOV) return fail(SG_ERR_ARG, "SG_IC_LANDAU needs the Vlasov-Poisson PDE");
        if (n_params != 2 || !p || !std::isfinite(p[0]) || !std::isfinite(p[1]))
            return fail(SG_ERR_ARG, "SG_IC_LANDAU takes 2 finite parameters (a, k)");
        for (int g = 0; g < h->G; ++g) {
            if (h->esize == 8) SG_CUDA(sg::Launch<double>::restrict_landau(h->hgrids[g], p[0], p[1], h->stream));
            else SG_CUDA(sg::Launch<float>::restrict_landau(h->hgrids[g], p[0], p[1], h->stream));
            h->launches += 1;
        }
        SG_CUDA(cudaStreamSynchronize(h->stream));
        h->ic_sine = false;
        h->initialized = true;
        h->combined = false;
        h->t = 0.0;
        h->steps = 0;
        return SG_OK;
    }
    if (ic_kind == SG_IC_RELAX) {
        if (h->pde != SG_PDE_VLASOV_BOLTZMANN || (h->dim != 2 && h->dim != 4))
            return fail(SG_ERR_ARG, "SG_IC_RELAX needs the Vlasov-Boltzmann model with dim 2 or 4");
        if (n_params != 0) return fail(SG_ERR_ARG, "SG_IC_RELAX takes no parameters");
        if (h->relax_s == 0.0) h->relax_s = relax_norm(h);  // depends on the domain only
        const double s_norm = h->relax_s;
        for (int g = 0; g < h->G; ++g) {
            if (h->esize == 8) SG_CUDA(sg::Launch<double>::restrict_relax(h->hgrids[g], h->dim, s_norm, h->stream));
            else SG_CUDA(sg::Launch<float>::restrict_relax(h->hgrids[g], h->dim, s_norm, h->stream));
            h->launches += 1;
        }
        SG_CUDA(cudaStreamSynchronize(h->stream));
        h->ic_sine = false;
        h->initialized = true;
        h->combined = false;
        h->t = 0.0;
        h->steps = 0;
        return SG_OK;
    }
    if (ic_kind != SG_IC_SINE || n_params != 4 || !p) return fail(SG_ERR_ARG, "SG_IC_SINE takes 4 parameters");
    for (int i = 0; i < 4; ++i)
        if (!std::isfinite(p[i])) return fail(SG_ERR_ARG, "initial-condition parameter %d not finite", i);
    {
        long long maxp = 1;
        for (int g = 0; g < h->G; ++g) maxp = std::max(maxp, h->hgrids[g].npts);
        if (h->esize == 8) SG_CUDA(sg::Launch<double>::restrict_sine(h->dgrids.as<GridDesc>(), h->G, maxp, h->dim, p, h->stream));
        else SG_CUDA(sg::Launch<float>::restrict_sine(h->dgrids.as<GridDesc>(), h->G, maxp, h->dim, p, h->stream));
        h->launches += 1;
    }
    SG_CUDA(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < 4; ++i) h->ic[i] = p[i];
    h->ic_sine = true;
    h->initialized = true;
    h->combined = false;
    h->t = 0.0;
    h->steps = 0;
    return SG_OK;
}

sg_status sg_init_grid(sg_handle h, int grid, const void* host_values, size_t bytes) {
    SG_TRY(check_handle(h));
    if (h->is_batch) return fail(SG_ERR_ARG, "sg_init_grid applies to batch members");
    if (grid < 0 || grid >= h->G) return fail(SG_ERR_ARG, "grid index %d out of range [0, %d)", grid, h->G);
    if (!host_values) return fail(SG_ERR_ARG, "NULL host buffer");
    const size_t need = (size_t)h->npts[grid] * h->esize;
    if (bytes != need) return fail(SG_ERR_ARG, "grid %d needs %zu bytes, got %zu", grid, need, bytes);
    SG_CUDA(cudaMemcpyAsync(h->hgrids[grid].u0, host_values, need, cudaMemcpyHostToDevice, h->stream));
    if (h->hgrids[grid].u3) SG_CUDA(cudaMemsetAsync(h->hgrids[grid].u3, 0, need, h->stream));
    SG_CUDA(cudaStreamSynchronize(h->stream));
    h->ic_sine = false;
    h->initialized = true;
    h->combined = false;
    h->t = 0.0;
    h->steps = 0;
    return SG_OK;
}

sg_status sg_init_grids(sg_handle h, const void* host_values, size_t bytes) {
    SG_TRY(check_handle(h));
    if (h->is_batch) return fail(SG_ERR_ARG, "sg_init_grids applies to batch members");
    if (!host_values) return fail(SG_ERR_ARG, "NULL host buffer");
    const size_t need = (size_t)h->total_pts * h->esize;
    if (bytes != need) return fail(SG_ERR_ARG, "all grids need %zu bytes, got %zu", need, bytes);
    SG_CUDA(cudaMemcpyAsync(h->hgrids[0].u0, host_values, need, cudaMemcpyHostToDevice, h->stream));
    if (h->hgrids[0].u3) SG_CUDA(cudaMemsetAsync(h->hgrids[0].u3, 0, need, h->stream));
    SG_CUDA(cudaStreamSynchronize(h->stream));
    h->ic_sine = false;
    h->initialized = true;
    h->combined = false;
    h->t = 0.0;
    h->steps = 0;
    return SG_OK;
}

sg_status sg_step(sg_handle h, double t_end, long max_steps, double* t_reached) {
    SG_TRY(check_handle(h));
    if (!std::isfinite(t_end)) return fail(SG_ERR_ARG, "t_end must be finite");
    if (max_steps < 0) return fail(SG_ERR_ARG, "max_steps must be >= 0");
    try {
        if (!h->is_batch) {
            if (!h->initialized) return fail(SG_ERR_STATE, "sg_step before sg_init");
            SG_TRY(autotune(h));
            fill_inst(h, h->hinst.p[0], 0, t_end, max_steps);
            sg_status st = run_steps(h);
            const InstState& s = h->hinst.p[0];
            if (h->esize == 4 && ((s.steps - s.step0) & 1)) {
                swap_pair(h->hgrids.data(), h->G);
                SG_CUDA(cudaMemcpy(h->dgrids.p, h->hgrids.data(), sizeof(GridDesc) * h->hgrids.size(), cudaMemcpyHostToDevice));
            }
            h->t = s.t;
            h->steps = s.steps;
            h->combined = false;
            if (t_reached) *t_reached = h->t;
            return st;
        }
        for (size_t i = 0; i < h->members.size(); ++i) {
            if (!h->members[i]->initialized) return fail(SG_ERR_STATE, "batch member %zu not initialised", i);
            SG_CUDA(cudaStreamSynchronize(h->members[i]->stream));
        }
        SG_TRY(autotune(h));
        int gbase = 0;
        for (size_t i = 0; i < h->members.size(); ++i) {
            sg_ctx* m = h->members[i];
            fill_inst(m, h->hinst.p[i], gbase, t_end, max_steps);
            for (int g = 0; g < m->G; ++g) {  // members may have been stepped on their own
                h->hgrids[gbase + g].u0 = m->hgrids[g].u0;
                h->hgrids[gbase + g].u1 = m->hgrids[g].u1;
            }
            gbase += m->G;
        }
        SG_CUDA(cudaMemcpy(h->dgrids.p, h->hgrids.data(), sizeof(GridDesc) * h->hgrids.size(), cudaMemcpyHostToDevice));
        sg_status st = run_steps(h);
        double tmin = INFINITY;
        bool swapped = false;
        for (size_t i = 0; i < h->members.size(); ++i) {
            sg_ctx* m = h->members[i];
            const InstState& s = h->hinst.p[i];
            if (m->esize == 4 && ((s.steps - s.step0) & 1)) {
                swap_pair(m->hgrids.data(), m->G);
                swap_pair(h->hgrids.data() + s.grid0, m->G);
                SG_CUDA(cudaMemcpy(m->dgrids.p, m->hgrids.data(), sizeof(GridDesc) * m->hgrids.size(), cudaMemcpyHostToDevice));
                swapped = true;
            }
            m->t = s.t;
            m->steps = s.steps;
            m->combined = false;
            tmin = std::min(tmin, m->t);
        }
        if (swapped)
            SG_CUDA(cudaMemcpy(h->dgrids.p, h->hgrids.data(), sizeof(GridDesc) * h->hgrids.size(), cudaMemcpyHostToDevice));
        if (t_reached) *t_reached = tmin;
        return st;
    } catch (const std::bad_alloc&) {
        return fail(SG_ERR_NOMEM, "host allocation failed");
    }
}

sg_status sg_prolong_combine(sg_handle h) {
    SG_TRY(check_handle(h));
    try {
        if (h->is_batch) {
            // members one after another on the batch's stream, sharing its intermediates (stream
            // order keeps them apart); each member's own stream is drained first, once at the end
            // the batch's
            for (sg_ctx* m : h->members) {
                if (!m->initialized) return fail(SG_ERR_STATE, "sg_prolong_combine before sg_init");
                if (m->stream != h->stream) SG_CUDA(cudaStreamSynchronize(m->stream));
            }
            for (sg_ctx* m : h->members)
                SG_TRY(m->esize == 8 ? prolong_combine_t<double>(m, h->comb, h->stream, false)
                                     : prolong_combine_t<float>(m, h->comb, h->stream, false));
            SG_CUDA(cudaStreamSynchronize(h->stream));
            return SG_OK;
        }
        if (!h->initialized) return fail(SG_ERR_STATE, "sg_prolong_combine before sg_init");
        return h->esize == 8 ? prolong_combine_t<double>(h, h->comb, h->stream, true)
                             : prolong_combine_t<float>(h, h->comb, h->stream, true);
    } catch (const std::bad_alloc&) {
        return fail(SG_ERR_NOMEM, "host allocation failed");
    }
}

sg_status sg_read(sg_handle h, int which, void* host_dst, size_t dst_bytes) {
    SG_TRY(check_handle(h));
    if (h->is_batch) return fail(SG_ERR_ARG, "sg_read applies to batch members");
    if (!host_dst) return fail(SG_ERR_ARG, "NULL destination");
    const void* src;
    size_t bytes;
    if (which == SG_WHICH_COMBINED) {
        if (!h->combined) return fail(SG_ERR_STATE, "no combined solution: call sg_prolong_combine first");
        src = h->uhat.p;
        bytes = sizeof(double) * (size_t)h->fine_pts;
    } else if (which >= 0 && which < h->G) {
        src = h->hgrids[which].u0;
        bytes = (size_t)h->npts[which] * h->esize;
    } else if (which == SG_WHICH_ALL_GRIDS) {
        src = h->hgrids[0].u0;
        bytes = (size_t)h->total_pts * h->esize;
    } else {
        return fail(SG_ERR_ARG, "which = %d out of range", which);
    }
    if (dst_bytes < bytes) return fail(SG_ERR_ARG, "destination holds %zu bytes, need %zu", dst_bytes, bytes);
    SG_CUDA(cudaMemcpyAsync(host_dst, src, bytes, cudaMemcpyDeviceToHost, h->stream));
    SG_CUDA(cudaStreamSynchronize(h->stream));
    return SG_OK;
}

sg_status sg_read_points(sg_handle h, int which, const long long* host_idx, size_t n, void* host_dst,
                         size_t dst_bytes) {
    SG_TRY(check_handle(h));
    if (h->is_batch) return fail(SG_ERR_ARG, "sg_read_points applies to batch members");
    if (n == 0) return SG_OK;
    if (!host_idx || !host_dst) return fail(SG_ERR_ARG, "NULL index or destination array");
    const void* src;
    long long count;
    size_t esz;
    if (which == SG_WHICH_COMBINED) {
        if (!h->combined) return fail(SG_ERR_STATE, "no combined solution: call sg_prolong_combine first");
        src = h->uhat.p;
        count = h->fine_pts;
        esz = sizeof(double);
    } else if (which >= 0 && which < h->G) {
        src = h->hgrids[which].u0;
        count = h->npts[which];
        esz = h->esize;
    } else if (which == SG_WHICH_ALL_GRIDS) {
        src = h->hgrids[0].u0;
        count = h->total_pts;
        esz = h->esize;
    } else {
        return fail(SG_ERR_ARG, "which = %d out of range", which);
    }
    if (dst_bytes < n * esz) return fail(SG_ERR_ARG, "destination holds %zu bytes, need %zu", dst_bytes, n * esz);
    for (size_t j = 0; j < n; ++j)
        if (host_idx[j] < 0 || host_idx[j] >= count)
            return fail(SG_ERR_ARG, "index %lld at position %zu outside [0, %lld)", host_idx[j], j, count);
    DevBuf didx, dout;
    SG_TRY(didx.alloc(n * sizeof(long long)));
    SG_TRY(dout.alloc(n * esz));
    SG_CUDA(cudaMemcpyAsync(didx.p, host_idx, n * sizeof(long long), cudaMemcpyHostToDevice, h->stream));
    if (esz == 8)
        SG_CUDA(sg::Launch<double>::gather((const double*)src, didx.as<long long>(), dout.as<double>(), (long long)n, h->stream));
    else
        SG_CUDA(sg::Launch<float>::gather((const float*)src, didx.as<long long>(), dout.as<float>(), (long long)n, h->stream));
    h->launches += 1;
    SG_CUDA(cudaMemcpyAsync(host_dst, dout.p, n * esz, cudaMemcpyDeviceToHost, h->stream));
    SG_CUDA(cudaStreamSynchronize(h->stream));
    return SG_OK;
}

sg_status sg_reduce(sg_handle h, int which, int kind, double* out) {
    SG_TRY(check_handle(h));
    if (h->is_batch) return fail(SG_ERR_ARG, "sg_reduce applies to batch members");
    if (!out) return fail(SG_ERR_ARG, "NULL output");
    if (kind == SG_REDUCE_FIELD_ENERGY) return field_energy(h, which, out);
    const bool entropy = kind == SG_REDUCE_ENTROPY_H2 || kind == SG_REDUCE_ENTROPY_LOG;
    if ((kind < SG_REDUCE_MASS || kind > SG_REDUCE_LINF_EXACT) && !entropy)
        return fail(SG_ERR_ARG, "unknown reduction %d", kind);
    if (entropy && h->pde != SG_PDE_VLASOV_BOLTZMANN)
        return fail(SG_ERR_ARG, "the entropy functionals need the Vlasov-Boltzmann model");
    ExactSpec X{};
    X.dim = h->dim;
    X.pde = h->pde;
    X.nf = (int)((long long)h->nr << h->nl);
    for (int k = 0; k < SG_MAXD; ++k) {
        X.lo[k] = k < h->dim ? h->prm.lo[k] : 0.0;
        X.h[k] = k < h->dim ? fine_spacing(h, k) : 1.0;
        X.adv[k] = k < h->dim ? h->prm.adv_speed[k] : 0.0;
    }
    X.b = h->ic[0];
    X.a = h->ic[1];
    X.w = h->ic[2];
    X.phi = h->ic[3];
    X.t = h->t;
    if (entropy) {  // M = exp(-(|x|^2 + |v|^2)/(2 theta)) / ((2 pi theta)^{d/2} Z), Z over the space domain
        const double th = h->prm.theta, rt = std::sqrt(2.0 * th);
        double Z = 1.0;
        for (int k = 0; k < h->dim / 2; ++k)
            Z *= std::sqrt(3.14159265358979323846 * th / 2.0) * (std::erf(h->prm.hi[k] / rt) - std::erf(h->prm.lo[k] / rt));
        X.theta = th;
        X.mnorm = std::pow(2.0 * 3.14159265358979323846 * th, 0.5 * (double)(h->dim / 2)) * Z;
        for (int k = 0; k < SG_MAXD; ++k) {
            const bool in = k < h->dim;
            X.n[k] = !in ? 1 : (which == SG_WHICH_COMBINED ? X.nf : (which >= 0 && which < h->G ? h->hgrids[which].n[k] : 1));
            if (in && which >= 0 && which < h->G) X.h[k] = h->hgrids[which].h[k];
        }
    }
    const bool exact = kind == SG_REDUCE_L1_EXACT || kind == SG_REDUCE_LINF_EXACT;
    double* dres = h->partial.as<double>() + 1024;
    long long n;
    double vol = 1.0;
    if (which == SG_WHICH_COMBINED) {
        if (!h->combined) return fail(SG_ERR_STATE, "no combined solution: call sg_prolong_combine first");
        if (exact && !h->ic_sine) return fail(SG_ERR_STATE, "exact-solution norms need an SG_IC_SINE initial condition");
        if (exact && phys_of(h).zmask)
            return fail(SG_ERR_STATE, "exact-solution norms assume periodic boundaries (an axis has SG_BC_ZERO)");
        n = h->fine_pts;
        for (int k = 0; k < h->dim; ++k) vol = vol * fine_spacing(h, k);
        SG_CUDA(sg::Launch<double>::reduce(h->uhat.as<double>(), nullptr, n, kind, X, h->partial.as<double>(), dres, h->stream));
    } else if (which >= 0 && which < h->G) {
        if (exact) return fail(SG_ERR_ARG, "exact-solution norms apply to the combined solution (which = -1)");
        n = h->npts[which];
        for (int k = 0; k < h->dim; ++k) vol = vol * h->hgrids[which].h[k];
        if (h->esize == 8)
            SG_CUDA(sg::Launch<double>::reduce((const double*)h->hgrids[which].u0, nullptr, n, kind, X, h->partial.as<double>(), dres, h->stream));
        else  // FP32 state is the float pair U + C
            SG_CUDA(sg::Launch<float>::reduce((const float*)h->hgrids[which].u0, (const float*)h->hgrids[which].u3, n, kind, X, h->partial.as<double>(), dres, h->stream));
    } else {
        return fail(SG_ERR_ARG, "which = %d out of range", which);
    }
    h->launches += 2;
    double r = 0.0;
    SG_CUDA(cudaMemcpyAsync(&r, dres, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    SG_CUDA(cudaStreamSynchronize(h->stream));
    switch (kind) {
        case SG_REDUCE_MASS:
        case SG_REDUCE_ENERGY:
        case SG_REDUCE_ENTROPY_H2:
        case SG_REDUCE_ENTROPY_LOG: r = r * vol; break;
        case SG_REDUCE_L1_EXACT: r = r / (double)n; break;
        default: break;
    }
    *out = r;
    return SG_OK;
}

sg_status sg_num_grids(sg_handle h, int* n) {
    SG_TRY(check_handle(h));
    if (!n) return fail(SG_ERR_ARG, "NULL output");
    *n = h->is_batch ? (int)h->hgrids.size() : h->G;
    return SG_OK;
}

sg_status sg_grid_info(sg_handle h, int g, int* levels, long* shape, double* coeff) {
    SG_TRY(check_handle(h));
    if (h->is_batch) return fail(SG_ERR_ARG, "sg_grid_info applies to batch members");
    if (g < 0 || g >= h->G) return fail(SG_ERR_ARG, "grid index %d out of range", g);
    for (int k = 0; k < h->dim; ++k) {
        if (levels) levels[k] = h->levels[g][k];
        if (shape) shape[k] = (long)h->nr << h->levels[g][k];
    }
    if (coeff) *coeff = h->coeff[g];
    return SG_OK;
}

sg_status sg_time(sg_handle h, double* t, long* steps) {
    SG_TRY(check_handle(h));
    if (t) *t = h->t;
    if (steps) *steps = (long)h->steps;
    return SG_OK;
}

sg_status sg_batch_create(const sg_handle* hs, int n, sg_handle* out) {
    if (!out) return fail(SG_ERR_ARG, "NULL output handle");
    *out = nullptr;
    if (!hs || n < 1) return fail(SG_ERR_ARG, "need at least one member");
    for (int i = 0; i < n; ++i) {
        if (!hs[i] || hs[i]->is_batch) return fail(SG_ERR_ARG, "member %d is NULL or a batch", i);
        const sg_ctx* a = hs[0];
        const sg_ctx* b = hs[i];
        if (b->dim != a->dim || b->pde != a->pde || b->esize != a->esize || b->prm.scheme != a->prm.scheme ||
            b->prm.eps != a->prm.eps || b->prm.tile_points != a->prm.tile_points ||
            b->prm.stage_kernel != a->prm.stage_kernel || b->prm.tau != a->prm.tau)
            return fail(SG_ERR_ARG, "member %d differs in dim, pde, precision, scheme, eps, tau or stage kernel", i);
        for (int k = 0; k < a->dim; ++k) {
            if (b->prm.adv_speed[k] != a->prm.adv_speed[k]) return fail(SG_ERR_ARG, "member %d differs in adv_speed", i);
            if (b->prm.bc[k] != a->prm.bc[k]) return fail(SG_ERR_ARG, "member %d differs in bc", i);
        }
    }
    try {
        sg_ctx* h = new sg_ctx();
        h->is_batch = true;
        h->dim = hs[0]->dim;
        h->pde = hs[0]->pde;
        h->prm = hs[0]->prm;
        h->prm.cuda_stream = nullptr;
        h->esize = hs[0]->esize;
        h->ppt = hs[0]->ppt;
        h->variant = hs[0]->variant;
        h->nr = hs[0]->nr;
        h->nl = hs[0]->nl;
        for (int i = 0; i < n; ++i) h->members.push_back(hs[i]);
        // members that all run on one caller-provided stream: the batch uses it too, so that
        // the caller's stream orders every operation; otherwise the batch owns a stream
        bool shared = !hs[0]->own_stream;
        for (int i = 1; i < n && shared; ++i) shared = !hs[i]->own_stream && hs[i]->stream == hs[0]->stream;
        if (shared) {
            h->stream = hs[0]->stream;
            h->own_stream = false;
        } else {
            cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                cudaGetLastError();
                delete h;
                return fail(SG_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
            }
            h->own_stream = true;
        }
        // every member on the first member's configuration, so one kernel fits every tile
        sg_status st = build_batch_tables(h);
        if (st == SG_OK) st = alloc_step_buffers(h, (int)h->hgrids.size(), n);
        if (st == SG_OK) st = configure(h, h->variant, h->ppt);
        // a batch of autotuned members tunes itself (the batched launch is another workload)
        if (st == SG_OK) h->tuned = !(h->prm.stage_kernel == SG_STAGE_AUTO && h->prm.tile_points == 0);
        if (st != SG_OK) {
            delete h;
            return st;
        }
        ++g_live_handles;
        *out = h;
        return SG_OK;
    } catch (const std::bad_alloc&) {
        return fail(SG_ERR_NOMEM, "host allocation failed");
    }
}

sg_status sg_destroy(sg_handle h) {
    if (!h) return SG_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    delete h;
    --g_live_handles;
    return SG_OK;
}

const char* sg_last_error(void) { return g_err.c_str(); }

sg_status sg_stage_config(sg_handle h, int* kernel, int* tile_points, double* tune_ms) {
    SG_TRY(check_handle(h));
    const bool sweep = h->dim == 3 && (h->variant == 0 || h->variant == 3);
    if (kernel) *kernel = !sweep ? SG_STAGE_TILED : (h->variant == 3 ? SG_STAGE_SWEEP2 : SG_STAGE_SWEEP);
    if (tile_points) *tile_points = sweep ? 512 : 256 * h->ppt;
    if (tune_ms) *tune_ms = h->tune_ms;
    return SG_OK;
}

}  // extern "C"

void sg::set_last_error(const char* msg) { g_err = msg; }

extern "C" {

sg_status sg_set_allocator(sg_alloc_fn alloc, sg_free_fn release, void* ctx) {
    if ((alloc == nullptr) != (release == nullptr)) return fail(SG_ERR_ARG, "alloc and release must both be set or both NULL");
    if (g_live_handles != 0) return fail(SG_ERR_STATE, "cannot change the allocator while handles exist");
    g_alloc = alloc;
    g_free = release;
    g_alloc_ctx = ctx;
    return SG_OK;
}

sg_status sg_launch_count(sg_handle h, long* n) {
    SG_TRY(check_handle(h));
    if (!n) return fail(SG_ERR_ARG, "NULL output");
    *n = (long)h->launches;
    return SG_OK;
}

sg_status sg_set_profiling(sg_handle h, int on) {
    SG_TRY(check_handle(h));
    h->profile = on != 0;
    h->prof_ms = 0.0;
    h->prof_launches = 0;
    return SG_OK;
}

sg_status sg_profile(sg_handle h, int kind, double* ms, long* launches) {
    SG_TRY(check_handle(h));
    if (kind != SG_PROF_STAGE) return fail(SG_ERR_ARG, "unknown profile kind %d", kind);
    if (ms) *ms = h->prof_ms;
    if (launches) *launches = (long)h->prof_launches;
    return SG_OK;
}

}  // extern "C"
