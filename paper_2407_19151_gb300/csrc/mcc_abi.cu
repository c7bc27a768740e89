// C ABI of the collision step (declarations and contracts in include/mcc.h).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mcc.h"
#include "mcc_kernels.h"
#include "mcc_pic.h"

static_assert(mcc::kGroupClasses == MCC_GROUP_CLASSES, "size classes of the ABI and the kernels");

// NVTX range over one entry point (header-only NVTX v3: a no-op unless a profiler injects itself), so that a timeline
// shows each library call on the host thread that issued it.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct mcc_ctx {
    int device;
    int32_t* dbuf;  // [0] status word, [1] work-queue counter, then the N97 tables
    int64_t launches;
    int num_sms;
    size_t smem_optin;
    size_t smem_per_sm;
    int32_t tile_cap;  // particles staged on chip per cell by the one-CTA kernel; 0 = automatic
    int32_t group_cap; // particles per warp of the group kernels' size classes; 0 = automatic
    int32_t group_top; // upper bound of the largest class; 0 = what one CTA's shared memory holds
    size_t smem_reserved;  // shared memory the system reserves per CTA
};

namespace mcc {

// Bytes per particle of the pairing mode's tile (defined with its kernel, mcc_cell.cu).
size_t pair_tile_bytes_per_particle();

// N97 table on the host, in double: A(s) solves G(A) = 1 - coth A + 1/A = 1 - e^-s (bisection to the last bit);
// stored as f = ln(A s) and h df/dx at x = ln s, where df/dx = 1 + s e^-s / (A G'(A)) by implicit
// differentiation, G'(A) = -(1/A^2 - 1/sinh^2 A).
namespace {

void laurent(double A, double& L, double& dL)
{
    // coth A - 1/A = sum_n 2^{2n} B_{2n} A^{2n-1} / (2n)!, for A < 1/2
    static const double c[12] = {1.0 / 3.0,       -1.0 / 45.0,        2.0 / 945.0,        -1.0 / 4725.0,
                                 2.0 / 93555.0,   -1382.0 / 638512875.0, 4.0 / 18243225.0, -3617.0 / 162820783125.0,
                                 87734.0 / 38979295480125.0, -349222.0 / 1531329465290625.0,
                                 310732.0 / 13447856940643125.0, -472728182.0 / 201919571963756521875.0};
    L = 0.0;
    dL = 0.0;
    double p = A;
    for (int n = 0; n < 12; ++n) {
        L += c[n] * p;
        dL += (2 * n + 1) * c[n] * (p / A);
        p *= A * A;
    }
}
double G_of(double A)
{
    if (A < 0.5) {
        double L, dL;
        laurent(A, L, dL);
        return 1.0 - L;
    }
    return 1.0 / A - 2.0 / std::expm1(2.0 * A);
}
double dG_of(double A)
{
    if (A < 0.5) {
        double L, dL;
        laurent(A, L, dL);
        return -dL;
    }
    const double sh = std::sinh(A);
    return -(1.0 / (A * A) - (A < 350.0 ? 1.0 / (sh * sh) : 0.0));
}
}  // namespace

void n97_table(double* f, double* dh)
{
    for (int k = 0; k <= kN97Nodes; ++k) {
        const double x = kN97X0 + kN97H * k;
        const double s = std::exp(x);
        const double z = -std::expm1(-s);
        double lo = 0.0, hi = 1.0 / z + 1.0;
        for (int it = 0; it < 2000; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (G_of(mid) > z) lo = mid;
            else hi = mid;
        }
        const double A = 0.5 * (lo + hi);
        f[k] = std::log(A * s);
        dh[k] = kN97H * (1.0 + s * std::exp(-s) / (A * dG_of(A)));
    }
}

}  // namespace mcc

namespace {

using mcc::StepArgs;

constexpr size_t kTabOffset = 64;  // bytes into the context buffer where the N97 tables start
constexpr size_t kTabDoubles = 2 * (mcc::kN97Nodes + 1);
constexpr size_t kClkOffset = (kTabOffset + kTabDoubles * sizeof(double) + kTabDoubles * sizeof(float) + 63) & ~63;
constexpr size_t kClkWords = 8 * mcc::kGroupClasses;  // phase cycles of the group kernels (phase-timing builds)
constexpr size_t kCtxBytes = kClkOffset + kClkWords * sizeof(unsigned long long);

constexpr size_t kStaticSmemReserve = 1024;  // margin above the cell kernel's static shared memory
#ifndef MCC_AUTO_CTAS
#define MCC_AUTO_CTAS 6
#endif
constexpr int kAutoCtasPerSm = MCC_AUTO_CTAS;  // automatic tile: this many CTAs share one SM's shared memory
constexpr int kMaxCtasPerSm = 2048 / mcc::kThreads;

cudaStream_t S(mcc_stream s) { return reinterpret_cast<cudaStream_t>(s); }

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int cuda_status(cudaError_t e) { return e == cudaSuccess ? MCC_OK : MCC_ERR_CUDA; }

bool valid_params(const mcc_params* p)
{
    if (!p) return false;
    if (p->method != MCC_TA77 && p->method != MCC_N97) return false;
    if (!(p->dt > 0) || !(p->dV > 0) || !(p->eps0 > 0) || !(p->fE > 0) || !(p->fE < 1)) return false;
    if (p->relativistic && !(p->c > 0)) return false;
    if (p->max_corr_passes < 0 || p->fail_policy < 0 || p->fail_policy > 2) return false;
    if (p->weighting != 0 && p->weighting != 1) return false;
    if (p->pairing != 0 && p->pairing != 1) return false;
    return true;
}

// Fill the species / interaction constants of a launch (host FP64; one rounding to float for the mixed path).
int fill_args(StepArgs& a, const mcc_ctx* ctx, const mcc_particles* P, const int64_t* offsets, int32_t n_cells,
              int32_t n_species, const mcc_species* sp, const double* lnL, const int32_t* inter, int32_t n_inter,
              int32_t inter_base, const mcc_params* p)
{
    std::memset(&a, 0, sizeof a);
    if (n_species < 1 || n_species > mcc::kMaxSpecies || n_cells < 0 || n_inter < 1 || n_inter > mcc::kMaxInter)
        return MCC_ERR_INVALID_ARG;
    a.offsets = offsets;
    a.n_cells = n_cells;
    a.S = n_species;
    if (P) {
        a.vx = P->vx;
        a.vy = P->vy;
        a.vz = P->vz;
        a.w = P->w;
        a.n_total = P->n;
    }
    if (sp) {
        for (int s = 0; s < n_species; ++s) {
            if (!(sp[s].m > 0)) return MCC_ERR_INVALID_ARG;
            a.m[s] = sp[s].m;
            a.m_f[s] = (float)sp[s].m;
            a.m_lo[s] = (float)(sp[s].m - (double)a.m_f[s]);
            a.ma[s] = sp[s].m;
            a.ma_f[s] = (float)sp[s].m;
        }
    }
    for (int k = 0; k < n_inter; ++k) {
        const int ia = inter[2 * k], ib = inter[2 * k + 1];
        if (ia < 0 || ib < ia || ib >= n_species) return MCC_ERR_INVALID_ARG;
        mcc::InterConst& ic = a.ic[k];
        ic.a = ia;
        ic.b = ib;
        if (sp && lnL && p) {
            const double qa = sp[ia].q, qb = sp[ib].q, ma = sp[ia].m, mb = sp[ib].m;
            const double mu = ma * mb / (ma + mb);
            const double L = lnL[ia * n_species + ib];
            const double kappa = qa * qa * qb * qb * L * p->dt / (4.0 * M_PI * p->eps0 * p->eps0 * p->dV);
            ic.kappa = kappa;
            ic.kappa_mu2 = kappa / (mu * mu);
            ic.mu_ma = mu / ma;
            ic.mu_mb = mu / mb;
            ic.kappa_f = (float)ic.kappa;
            ic.kappa_mu2_f = (float)ic.kappa_mu2;
            ic.mu_ma_f = (float)ic.mu_ma;
            ic.mu_mb_f = (float)ic.mu_mb;
        }
    }
    a.n_inter = n_inter;
    a.inter_base = inter_base;
    if (p) {
        a.method = p->method;
        a.fail_policy = p->fail_policy;
        a.sort_by_weight = p->sort_by_weight;
        a.max_corr_passes = p->max_corr_passes;
        a.correct = p->correct;
        a.c = p->c;
        a.fE = p->fE;
        a.c_f = (float)p->c;
        a.fE_f = (float)p->fE;
        auto split = [](double x, float& hi, float& lo) {
            hi = (float)x;
            lo = (float)(x - (double)hi);
        };
        split(p->fE, a.fE_f, a.fE_lo);
        split(-p->fE / (1.0 + std::sqrt(1.0 - p->fE)), a.gm1p_f, a.gm1p_lo);
        split(p->fE / (1.0 + std::sqrt(1.0 + p->fE)), a.gm1n_f, a.gm1n_lo);
        split(p->c > 0 ? 1.0 / (p->c * p->c) : 0.0, a.c2inv_f, a.c2inv_lo);
        a.rng.k0 = (uint32_t)p->seed;
        a.rng.k1 = (uint32_t)(p->seed >> 32);
        a.rng.step = (uint32_t)p->step;
        a.rng.cell_base = p->cell_base;
        a.weighting = p->weighting;
        a.pairing = p->pairing;
    }
    a.status = ctx->dbuf;
    a.queue = ctx->dbuf + 1;
    const char* base = reinterpret_cast<const char*>(ctx->dbuf) + kTabOffset;
    a.n97_f = reinterpret_cast<const double*>(base);
    a.n97_dh = a.n97_f + (mcc::kN97Nodes + 1);
    a.n97_f32 = reinterpret_cast<const float*>(base + kTabDoubles * sizeof(double));
    a.n97_dh32 = a.n97_f32 + (mcc::kN97Nodes + 1);
    a.phase_clk = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ctx->dbuf) + kClkOffset);
    return MCC_OK;
}

// Largest on-chip tile (particles) one CTA can stage: the opt-in shared memory minus the kernel's static part.
size_t max_tile_particles(const mcc_ctx* ctx, bool f32)
{
    const size_t fixed = mcc::cell_kernel_static_smem(f32, true, mcc::kFused) + kStaticSmemReserve;
    const size_t avail = ctx->smem_optin > fixed ? ctx->smem_optin - fixed : 0;
    return avail / mcc::tile_bytes_per_particle(f32);
}

// Largest cell of the pairing mode (its compact tile in one CTA's shared memory; the tile layout and its bytes per
// particle are defined with the kernel, in mcc_cell.cu).
size_t max_pair_tile_particles(const mcc_ctx* ctx)
{
    const size_t fixed = mcc::cell_kernel_static_smem(false, false, mcc::kPair) + kStaticSmemReserve;
    const size_t avail = ctx->smem_optin > fixed ? ctx->smem_optin - fixed : 0;
    return avail / mcc::pair_tile_bytes_per_particle();
}

// Automatic tile: the largest that still lets kAutoCtasPerSm CTAs share an SM's shared memory.
int auto_tile(const mcc_ctx* ctx, bool f32)
{
    const size_t fixed = mcc::cell_kernel_static_smem(f32, true, mcc::kFused) + 1024;
    const size_t per_cta = ctx->smem_per_sm / kAutoCtasPerSm;
    const size_t t = per_cta > fixed ? (per_cta - fixed) / mcc::tile_bytes_per_particle(f32) : 64;
    const size_t capmax = max_tile_particles(ctx, f32);
    return (int)(t < capmax ? t : capmax);
}

// Launch one cell-kernel pass over every cell (queue reset, persistent grid of at most max_grid CTAs).
int run_cells(mcc_ctx* ctx, StepArgs& a, bool f32, bool rel, int mode, int cap, cudaStream_t st,
              int max_grid = 1 << 30)
{
    const size_t per = mode == mcc::kPair ? mcc::pair_tile_bytes_per_particle() : mcc::tile_bytes_per_particle(f32);
    const size_t smem = (size_t)cap * per;
    if (mcc::set_cell_smem_limit(f32, rel, mode, smem) != cudaSuccess) return MCC_ERR_CUDA;
    int bps = mcc::cell_kernel_blocks_per_sm(f32, rel, mode, smem);
    if (bps < 1) return MCC_ERR_CUDA;
    int grid = ctx->num_sms * bps;
    if (grid > max_grid) grid = max_grid;
    if (a.n_cells < grid) grid = a.n_cells > 0 ? a.n_cells : 1;
    a.cap = cap;
    cudaError_t e = cudaMemsetAsync(ctx->dbuf + 1, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return MCC_ERR_CUDA;
    e = mcc::launch_cell(f32, rel, mode, a, grid, smem, st);
    ctx->launches += 1;
    return cuda_status(e);
}

// Grid of the adjoint kernel: one CTA per cell, at most two per SM (each holds a slab of the workspace).
int adjoint_grid(const mcc_ctx* ctx, int32_t n_cells)
{
    const int g = ctx->num_sms * 2;
    return n_cells < g ? (n_cells > 0 ? n_cells : 1) : g;
}

}  // namespace

extern "C" {

int mcc_create(mcc_ctx** out, int device)
{
    if (!out) return MCC_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MCC_ERR_INVALID_ARG;
    DeviceGuard g(device);
    mcc_ctx* c = new (std::nothrow) mcc_ctx();
    if (!c) return MCC_ERR_CUDA;
    c->device = device;
    c->launches = 0;
    c->tile_cap = 0;
    c->group_cap = 0;
    c->group_top = 0;
    int optin = 0, sms = 0, per_sm = 0, reserved = 0;
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device);
    c->smem_reserved = (size_t)reserved;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    c->smem_per_sm = (size_t)per_sm;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    c->smem_optin = (size_t)optin;
    c->num_sms = sms;
    // status word, queue counter and the N97 tables (double, then float), computed here once
    double tab[kTabDoubles];
    float tab32[kTabDoubles];
    mcc::n97_table(tab, tab + (mcc::kN97Nodes + 1));
    // float copy: g = A s = exp(f) and h dg/dx = exp(f) (h df/dx)
    for (int k = 0; k <= mcc::kN97Nodes; ++k) {
        const double g = std::exp(tab[k]);
        tab32[k] = (float)g;
        tab32[mcc::kN97Nodes + 1 + k] = (float)(g * tab[mcc::kN97Nodes + 1 + k]);
    }
    if (cudaMalloc(&c->dbuf, kCtxBytes) != cudaSuccess || cudaMemset(c->dbuf, 0, kCtxBytes) != cudaSuccess ||
        cudaMemcpy(reinterpret_cast<char*>(c->dbuf) + kTabOffset, tab, sizeof tab, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(reinterpret_cast<char*>(c->dbuf) + kTabOffset + sizeof tab, tab32, sizeof tab32,
                   cudaMemcpyHostToDevice) != cudaSuccess) {
        if (c->dbuf) cudaFree(c->dbuf);
        delete c;
        return MCC_ERR_CUDA;
    }
    *out = c;
    return MCC_OK;
}

void mcc_destroy(mcc_ctx* ctx)
{
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaFree(ctx->dbuf);
    delete ctx;
}

int mcc_bin_workspace_size(int64_t n, int32_t n_cells, int32_t n_species, size_t* bytes)
{
    if (!bytes || n < 0 || n_cells <= 0 || n_species <= 0) return MCC_ERR_INVALID_ARG;
    *bytes = mcc::bin_workspace_bytes(n, (int64_t)n_cells * n_species);
    return MCC_OK;
}

int mcc_bin(mcc_ctx* ctx, const int32_t* cell, const int32_t* species, int64_t n, int32_t n_cells,
            int32_t n_species, int32_t* perm_out, int64_t* offsets_out, void* ws, size_t ws_bytes, mcc_stream stream)
{
    NvtxRange nvtx_("mcc_bin");
    if (!ctx || n < 0 || n_cells <= 0 || n_species <= 0 || !offsets_out) return MCC_ERR_INVALID_ARG;
    if (n > 0 && (!cell || !species || !perm_out)) return MCC_ERR_INVALID_ARG;
    if (n > INT32_MAX) return MCC_ERR_TOO_LARGE;
    if (!ws || ws_bytes < mcc::bin_workspace_bytes(n, (int64_t)n_cells * n_species)) return MCC_ERR_WORKSPACE;
    DeviceGuard g(ctx->device);
    return cuda_status(mcc::launch_bin(cell, species, n, n_cells, n_species, perm_out, offsets_out, ws, ctx->dbuf,
                                       S(stream), &ctx->launches));
}

int mcc_bin_weighted_workspace_size(int64_t n, int32_t n_cells, int32_t n_species, size_t* bytes)
{
    if (!bytes || n < 0 || n_cells <= 0 || n_species <= 0) return MCC_ERR_INVALID_ARG;
    *bytes = mcc::bin_weighted_workspace_bytes(n, (int64_t)n_cells * n_species);
    return MCC_OK;
}

int mcc_bin_weighted(mcc_ctx* ctx, const int32_t* cell, const int32_t* species, const double* w, int64_t n,
                     int32_t n_cells, int32_t n_species, int32_t* perm_out, int64_t* offsets_out, void* ws,
                     size_t ws_bytes, mcc_stream stream)
{
    NvtxRange nvtx_("mcc_bin_weighted");
    if (!ctx || n < 0 || n_cells <= 0 || n_species <= 0 || !offsets_out) return MCC_ERR_INVALID_ARG;
    if (n > 0 && (!cell || !species || !w || !perm_out)) return MCC_ERR_INVALID_ARG;
    if (n > INT32_MAX) return MCC_ERR_TOO_LARGE;
    if (!ws || ws_bytes < mcc::bin_weighted_workspace_bytes(n, (int64_t)n_cells * n_species))
        return MCC_ERR_WORKSPACE;
    DeviceGuard g(ctx->device);
    return cuda_status(mcc::launch_bin_weighted(cell, species, w, n, n_cells, n_species, perm_out, offsets_out, ws,
                                                ctx->dbuf, S(stream), &ctx->launches));
}

int mcc_bin_static(const int32_t* cell, const int32_t* species, int64_t n, int32_t n_cells, int32_t n_species,
                   int32_t* perm_out, int64_t* offsets_out, mcc_stream stream)
{
    if (n < 0 || n_cells <= 0 || n_species <= 0 || !offsets_out) return MCC_ERR_INVALID_ARG;
    if (n > 0 && (!cell || !species || !perm_out)) return MCC_ERR_INVALID_ARG;
    if (n > INT32_MAX || (int64_t)n_cells * n_species > mcc::static_bin_max_keys()) return MCC_ERR_TOO_LARGE;
    if (stream) {  // the counters' address is the current device's: the stream must run there
        int sdev = -1, cur = -1;
        if (cudaStreamGetDevice(S(stream), &sdev) != cudaSuccess || cudaGetDevice(&cur) != cudaSuccess)
            return MCC_ERR_CUDA;
        if (sdev != cur) return MCC_ERR_INVALID_ARG;
    }
    return cuda_status(mcc::launch_bin_static(cell, species, n, n_cells, n_species, perm_out, offsets_out,
                                              S(stream)));
}

int mcc_species_moments(mcc_ctx* ctx, const mcc_particles* P, const int64_t* offsets, int32_t n_cells,
                        int32_t n_species, const mcc_species* sp, int32_t relativistic, double c,
                        const int32_t* fail_count, double* out, mcc_stream stream)
{
    NvtxRange nvtx_("mcc_species_moments");
    if (!ctx || !P || !offsets || !sp || !out || n_cells < 0 || n_species < 1 || n_species > MCC_MAX_SPECIES)
        return MCC_ERR_INVALID_ARG;
    if (P->prec != MCC_F64 && P->prec != MCC_F32_MIXED) return MCC_ERR_INVALID_ARG;
    if (P->n > 0 && (!P->vx || !P->vy || !P->vz || !P->w)) return MCC_ERR_INVALID_ARG;
    if (relativistic && !(c > 0.0 && std::isfinite(c))) return MCC_ERR_INVALID_ARG;
    mcc::SpeciesConst sc;
    for (int s = 0; s < MCC_MAX_SPECIES; ++s) sc.m[s] = 0.0;
    for (int s = 0; s < n_species; ++s) {
        if (!(sp[s].m > 0.0) || !std::isfinite(sp[s].m)) return MCC_ERR_INVALID_ARG;
        sc.m[s] = sp[s].m;
    }
    DeviceGuard g(ctx->device);
    const cudaError_t e = mcc::launch_species_moments(P->prec == MCC_F32_MIXED, P->vx, P->vy, P->vz, P->w, offsets,
                                                      n_cells, n_species, sc, relativistic != 0, c, fail_count, out,
                                                      ctx->num_sms, S(stream));
    ctx->launches += 1;
    return cuda_status(e);
}

int mcc_gather(const void* in, const int32_t* perm, int64_t n, int32_t elem_bytes, void* out, mcc_stream stream)
{
    if (n < 0 || (elem_bytes != 4 && elem_bytes != 8) || (n > 0 && (!in || !perm || !out))) return MCC_ERR_INVALID_ARG;
    return cuda_status(mcc::launch_gather(in, perm, n, elem_bytes, out, S(stream)));
}

int mcc_gather_n(const void* const* in, void* const* out, const int32_t* elem_bytes, int32_t n_arrays,
                 const int32_t* perm, int64_t n, mcc_stream stream)
{
    NvtxRange nvtx_("mcc_gather_n");
    if (n < 0 || n_arrays < 1 || n_arrays > MCC_MAX_GATHER || !in || !out || !elem_bytes) return MCC_ERR_INVALID_ARG;
    for (int j = 0; j < n_arrays; ++j) {
        if (elem_bytes[j] != 4 && elem_bytes[j] != 8) return MCC_ERR_INVALID_ARG;
        if (n > 0 && (!in[j] || !out[j])) return MCC_ERR_INVALID_ARG;
    }
    if (n > 0 && !perm) return MCC_ERR_INVALID_ARG;
    return cuda_status(mcc::launch_gather_n(in, out, elem_bytes, n_arrays, perm, n, S(stream)));
}

int mcc_push(const mcc_particles* P, void* x, void* y, void* z, const mcc_grid* grid, double dt,
             int32_t relativistic, double c, int32_t* cell_out, mcc_stream stream)
{
    NvtxRange nvtx_("mcc_push");
    if (!P || !grid || P->n < 0 || (P->prec != MCC_F64 && P->prec != MCC_F32_MIXED)) return MCC_ERR_INVALID_ARG;
    if (relativistic != 0 && relativistic != 1) return MCC_ERR_INVALID_ARG;
    const int32_t nc[3] = {grid->nx, grid->ny, grid->nz};
    const double l[3] = {grid->lx, grid->ly, grid->lz};
    int64_t cells = 1;
    for (int d = 0; d < 3; ++d) {
        if (nc[d] < 1 || !(l[d] > 0.0) || !std::isfinite(l[d])) return MCC_ERR_INVALID_ARG;
        cells *= nc[d];
        if (cells > INT32_MAX) return MCC_ERR_INVALID_ARG;
    }
    if (!std::isfinite(dt) || (relativistic && !(c > 0.0 && std::isfinite(c)))) return MCC_ERR_INVALID_ARG;
    if (P->n == 0) return MCC_OK;
    if (!P->vx || !P->vy || !P->vz || !x || !y || !z || !cell_out) return MCC_ERR_INVALID_ARG;
    mcc::PushGrid g;
    for (int d = 0; d < 3; ++d) {
        g.n[d] = nc[d];
        g.l[d] = l[d];
    }
    return cuda_status(mcc::launch_push(P->prec == MCC_F32_MIXED, relativistic != 0, x, y, z, P->vx, P->vy, P->vz,
                                        P->n, g, dt, c, cell_out, S(stream)));
}

int mcc_pair(mcc_ctx* ctx, const int64_t* offsets, int32_t n_cells, int32_t n_species, int32_t sa, int32_t sb,
             int32_t inter, uint64_t seed, uint64_t step, int32_t* pair_i, int32_t* pair_j, uint8_t* pair_flags,
             mcc_stream stream)
{
    NvtxRange nvtx_("mcc_pair");
    if (!ctx || !offsets || !pair_i || !pair_j || !pair_flags || inter < 0 || inter > 0xFFFFFF)
        return MCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    StepArgs a;
    const int32_t ab[2] = {sa, sb};
    mcc_params p;
    std::memset(&p, 0, sizeof p);
    p.seed = seed;
    p.step = step;
    int rc = fill_args(a, ctx, nullptr, offsets, n_cells, n_species, nullptr, nullptr, ab, 1, inter, &p);
    if (rc != MCC_OK) return rc;
    if (n_cells == 0) return MCC_OK;
    a.pair_i = pair_i;
    a.pair_j = pair_j;
    a.pair_flags = pair_flags;
    const int cap = (int)max_pair_tile_particles(ctx);
    return run_cells(ctx, a, false, false, mcc::kPair, cap, S(stream));
}

int mcc_scatter(mcc_ctx* ctx, const mcc_particles* P, const int64_t* offsets, int32_t n_cells, int32_t n_species,
                const mcc_species* sp, const double* lnL, int32_t sa, int32_t sb, int32_t inter, const int32_t* pair_i,
                const int32_t* pair_j, const uint8_t* pair_flags, const mcc_params* p, void* backup,
                mcc_stream stream)
{
    NvtxRange nvtx_("mcc_scatter");
    if (!ctx || !P || !offsets || !sp || !lnL || !pair_i || !pair_j || !pair_flags || !backup || !valid_params(p) ||
        inter < 0 || inter > 0xFFFFFF || p->pairing != 0)
        return MCC_ERR_INVALID_ARG;
    if (P->prec != MCC_F64 && P->prec != MCC_F32_MIXED) return MCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    StepArgs a;
    const int32_t ab[2] = {sa, sb};
    int rc = fill_args(a, ctx, P, offsets, n_cells, n_species, sp, lnL, ab, 1, inter, p);
    if (rc != MCC_OK) return rc;
    if (n_cells == 0) return MCC_OK;
    a.pair_i = const_cast<int32_t*>(pair_i);
    a.pair_j = const_cast<int32_t*>(pair_j);
    a.pair_flags = const_cast<uint8_t*>(pair_flags);
    a.backup = backup;
    const bool f32 = P->prec == MCC_F32_MIXED;
    const int cap = (int)max_tile_particles(ctx, f32);
    return run_cells(ctx, a, f32, p->relativistic != 0, mcc::kScatter, cap, S(stream));
}

int mcc_correct(mcc_ctx* ctx, const mcc_particles* P, const int64_t* offsets, int32_t n_cells, int32_t n_species,
                const mcc_species* sp, int32_t sa, int32_t sb, int32_t inter, const mcc_params* p,
                const void* backup, int32_t* corr_pairs_out, int32_t* fail_flags_out, mcc_stream stream)
{
    NvtxRange nvtx_("mcc_correct");
    if (!ctx || !P || !offsets || !sp || !backup || !valid_params(p) || inter < 0 || inter > 0xFFFFFF)
        return MCC_ERR_INVALID_ARG;
    if (P->prec != MCC_F64 && P->prec != MCC_F32_MIXED) return MCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    StepArgs a;
    const int32_t ab[2] = {sa, sb};
    int rc = fill_args(a, ctx, P, offsets, n_cells, n_species, sp, nullptr, ab, 1, inter, p);
    if (rc != MCC_OK) return rc;
    if (n_cells == 0) return MCC_OK;
    a.backup = const_cast<void*>(backup);
    a.corr_pairs = corr_pairs_out;
    a.fail_count = fail_flags_out;
    const bool f32 = P->prec == MCC_F32_MIXED;
    const int cap = (int)max_tile_particles(ctx, f32);
    return run_cells(ctx, a, f32, p->relativistic != 0, mcc::kCorrect, cap, S(stream));
}

namespace {
// Workspace of mcc_step_fused: the cell order (n_cells int32), the class bounds and queue counters of the group
// kernels, then, when some cell exceeds the largest group class, one slab per resident CTA of the one-CTA kernel.
size_t order_bytes(int32_t n_cells) { return ((size_t)n_cells * sizeof(int32_t) + 255) & ~(size_t)255; }
constexpr size_t kCtrlBytes = 256;  // class_off [2 (kGroupClasses + 1)] and queues [kGroupClasses + 1], int32

int tile_of(const mcc_ctx* ctx, bool f32)
{
    const size_t capmax = max_tile_particles(ctx, f32);
    return ctx->tile_cap > 0 ? (int)((size_t)ctx->tile_cap < capmax ? (size_t)ctx->tile_cap : capmax)
                             : auto_tile(ctx, f32);
}

size_t slab_stride_of(int32_t max_cell, bool f32)
{
    return ((size_t)max_cell * mcc::tile_bytes_per_particle(f32) + 255) & ~(size_t)255;
}

size_t group_static_smem(bool f32, bool rel, int cls)
{
    if (!f32) return 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, mcc::group_kernel(f32, rel, cls)) != cudaSuccess) return 8192;
    return fa.sharedSizeBytes;
}

// Capacity (particles) of each group size class. Class k runs 32 << k threads and holds cells of up to
// per_warp << k particles, so that the shared memory per thread is the same in every class; the largest class
// takes up to what one CTA's shared memory holds, unless the capacity is set explicitly.
void group_caps(const mcc_ctx* ctx, bool f32, bool rel, int32_t caps[mcc::kGroupClasses])
{
    if (!f32) {  // FP64: every cell on the one-CTA kernel
        for (int k = 0; k < mcc::kGroupClasses; ++k) caps[k] = 0;
        return;
    }
    size_t per_warp;
    if (ctx->group_cap > 0) {
        per_warp = (size_t)ctx->group_cap;
    } else {
        const size_t per_cta = ctx->smem_per_sm / mcc::kGroupWarpsPerSm;
        const size_t fixed = ctx->smem_reserved + group_static_smem(f32, rel, 0);  // per one-warp CTA
        per_warp = per_cta > fixed ? (per_cta - fixed) / mcc::kGroupBytesPerParticle : 32;
    }
    for (int k = 0; k < mcc::kGroupClasses; ++k) {
        const size_t st = group_static_smem(f32, rel, k);
        const size_t maxp = ctx->smem_optin > st ? (ctx->smem_optin - st) / mcc::kGroupBytesPerParticle : 0;
        size_t cap = per_warp << k;
        if (k == mcc::kGroupClasses - 1) cap = ctx->group_top > 0 ? (size_t)ctx->group_top : maxp;
        if (cap > maxp) cap = maxp;
        if (cap > 65535) cap = 65535;  // cell-local indices are 16-bit
        caps[k] = (int32_t)cap;
    }
}
}  // namespace

int mcc_step_workspace_size(mcc_ctx* ctx, int32_t prec, int32_t n_cells, int32_t max_cell, size_t* bytes)
{
    if (!ctx || !bytes || max_cell < 0 || n_cells < 0 || (prec != MCC_F64 && prec != MCC_F32_MIXED))
        return MCC_ERR_INVALID_ARG;
    if (max_cell > MCC_MAX_SEGMENT) return MCC_ERR_TOO_LARGE;
    const bool f32 = prec == MCC_F32_MIXED;
    int32_t caps[mcc::kGroupClasses];
    group_caps(ctx, f32, false, caps);
    int32_t caps_rel[mcc::kGroupClasses];
    group_caps(ctx, f32, true, caps_rel);
    const int32_t top = caps[mcc::kGroupClasses - 1] < caps_rel[mcc::kGroupClasses - 1]
                            ? caps[mcc::kGroupClasses - 1]
                            : caps_rel[mcc::kGroupClasses - 1];
    size_t total = order_bytes(n_cells) + kCtrlBytes;
    if (max_cell > top && max_cell > tile_of(ctx, f32))
        total += slab_stride_of(max_cell, f32) * (size_t)ctx->num_sms * kMaxCtasPerSm;
    *bytes = total;
    return MCC_OK;
}

int mcc_set_group_capacity(mcc_ctx* ctx, int32_t particles_per_warp, int32_t largest)
{
    if (!ctx || particles_per_warp < 0 || largest < 0) return MCC_ERR_INVALID_ARG;
    ctx->group_cap = particles_per_warp;
    ctx->group_top = largest;
    return MCC_OK;
}

int mcc_group_capacities(mcc_ctx* ctx, int32_t prec, int32_t relativistic, int32_t* caps_out)
{
    if (!ctx || !caps_out || (prec != MCC_F64 && prec != MCC_F32_MIXED)) return MCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    group_caps(ctx, prec == MCC_F32_MIXED, relativistic != 0, caps_out);
    return MCC_OK;
}

int mcc_step_fused(mcc_ctx* ctx, const mcc_particles* P, const int64_t* offsets, int32_t n_cells, int32_t n_species,
                   const mcc_species* sp, const double* lnL, const int32_t* interactions, int32_t n_inter,
                   const mcc_params* p, int32_t n_steps, int32_t max_cell, int32_t* corr_pairs, int32_t* fail_count,
                   void* ws, size_t ws_bytes, mcc_stream stream)
{
    NvtxRange nvtx_("mcc_step_fused");
    if (!ctx || !P || !offsets || !sp || !lnL || !interactions || !valid_params(p) || n_steps < 0 || max_cell < 0)
        return MCC_ERR_INVALID_ARG;
    if (P->prec != MCC_F64 && P->prec != MCC_F32_MIXED) return MCC_ERR_INVALID_ARG;
    if (max_cell > MCC_MAX_SEGMENT) return MCC_ERR_TOO_LARGE;  // in-cell indices are 20-bit key fields
    DeviceGuard g(ctx->device);
    StepArgs a;
    int rc = fill_args(a, ctx, P, offsets, n_cells, n_species, sp, lnL, interactions, n_inter, 0, p);
    if (rc != MCC_OK) return rc;
    if (n_cells == 0 || n_steps == 0) return MCC_OK;
    a.corr_pairs = corr_pairs;
    a.fail_count = fail_count;
    a.resid = p->residual;
    a.max_cell = max_cell;
    const bool f32 = P->prec == MCC_F32_MIXED;
    const bool rel = p->relativistic != 0;
    size_t need = 0;
    mcc_step_workspace_size(ctx, P->prec, n_cells, max_cell, &need);
    if (!ws || ws_bytes < need) return MCC_ERR_WORKSPACE;
    int32_t caps[mcc::kGroupClasses];
    group_caps(ctx, f32, rel, caps);
    // the group kernels serve the mixed path; the FP64 path runs every cell on the one-CTA kernel
    const bool fallback = !f32 || max_cell > caps[mcc::kGroupClasses - 1];
    int32_t* order = reinterpret_cast<int32_t*>(ws);
    int32_t* class_off = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(ws) + order_bytes(n_cells));
    int32_t* queues = class_off + 2 * (mcc::kGroupClasses + 1);
    // cells by size class, largest first (the order is the same for every step of the call)
    if (mcc::launch_group_order(offsets, n_cells, n_species, caps, order, class_off, S(stream)) != cudaSuccess)
        return MCC_ERR_CUDA;
    ctx->launches += 1;
    a.order = order;
    a.class_off = class_off;
    a.queues = queues;
    a.step_dev = p->step_device;
    // the one-CTA kernel takes the cells above every class from the order's first range
    const int tile = tile_of(ctx, f32);
    int max_grid = 1 << 30;
    StepArgs big = a;
    if (fallback) {
        big.order_range = class_off + 2 * mcc::kGroupClasses;
        if (max_cell > tile) {
            big.slab = reinterpret_cast<char*>(ws) + order_bytes(n_cells) + kCtrlBytes;
            big.slab_stride = (int64_t)slab_stride_of(max_cell, f32);
            big.slab_cap = max_cell;
            max_grid = (int)((ws_bytes - order_bytes(n_cells) - kCtrlBytes) / (size_t)big.slab_stride);
        }
    }
    // under stream capture the marks become event-record nodes of the graph, so that a replay records them too
    unsigned rec_flags = cudaEventRecordDefault;
    if (p->launch_events) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(S(stream), &cs) != cudaSuccess) return MCC_ERR_CUDA;
        if (cs == cudaStreamCaptureStatusActive) rec_flags = cudaEventRecordExternal;
    }
    for (int32_t t = 0; t < n_steps; ++t) {
        a.rng.step = (uint32_t)(p->step + (uint64_t)t);
        a.step_add = (uint32_t)t;
        if (cudaMemsetAsync(queues, 0, sizeof(int32_t) * (mcc::kGroupClasses + 1), S(stream)) != cudaSuccess)
            return MCC_ERR_CUDA;
        cudaEvent_t* ev = (p->launch_events && t == n_steps - 1) ? reinterpret_cast<cudaEvent_t*>(p->launch_events)
                                                                   : nullptr;
        auto mark = [&](int k, int end) {
            if (ev) cudaEventRecordWithFlags(ev[2 * k + end], S(stream), rec_flags);
        };
        mark(mcc::kGroupClasses, 0);
        if (fallback) {
            big.rng.step = a.rng.step;
            big.step_add = a.step_add;
            const int cap = max_cell <= tile ? max_cell : tile;
            rc = run_cells(ctx, big, f32, rel, mcc::kFused, cap, S(stream), max_grid);
            if (rc != MCC_OK) return rc;
        }
        mark(mcc::kGroupClasses, 1);
        for (int cls = mcc::kGroupClasses - 1; cls >= 0; --cls) {
            mark(cls, 0);
            if (!f32 || (cls > 0 && caps[cls - 1] >= max_cell)) {  // no cell can be in this class
                mark(cls, 1);
                continue;
            }
            const size_t smem = (size_t)caps[cls] * mcc::kGroupBytesPerParticle;
            const void* fn = mcc::group_kernel(f32, rel, cls);
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return MCC_ERR_CUDA;
            int bps = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, 32 << cls, smem) != cudaSuccess || bps < 1)
                return MCC_ERR_CUDA;
            int grid = bps * ctx->num_sms;
            if (grid > n_cells) grid = n_cells;
            a.gcls = cls;
            a.gcap = caps[cls];
            const cudaError_t e = mcc::launch_group(f32, rel, cls, a, grid, smem, S(stream));
            ctx->launches += 1;
            if (e != cudaSuccess) return MCC_ERR_CUDA;
            mark(cls, 1);
        }
    }
    if (p->step_device) {
        if (mcc::launch_step_advance(p->step_device, (uint64_t)n_steps, S(stream)) != cudaSuccess) return MCC_ERR_CUDA;
        ctx->launches += 1;
    }
    return MCC_OK;
}

int mcc_adjoint_workspace_size(mcc_ctx* ctx, int32_t n_cells, int32_t max_cell, int32_t max_corr_passes,
                               size_t* bytes)
{
    if (!ctx || !bytes || n_cells < 0 || max_cell < 0 || max_corr_passes < 0) return MCC_ERR_INVALID_ARG;
    if (max_cell > MCC_MAX_SEGMENT) return MCC_ERR_TOO_LARGE;
    const int32_t mc = max_cell > 0 ? max_cell : 1;
    const int32_t ep = max_corr_passes * (mc / 2 + 1) + 1;
    const int grid = adjoint_grid(ctx, n_cells);
    *bytes = mcc::adjoint_slab_bytes(mc, ep) * (size_t)grid;
    return MCC_OK;
}

int mcc_adjoint_tape_size(mcc_ctx* ctx, int32_t n_cells, int32_t max_cell, int32_t max_corr_passes, size_t* bytes)
{
    if (!ctx || !bytes || n_cells < 0 || max_cell < 0 || max_corr_passes < 0) return MCC_ERR_INVALID_ARG;
    if (max_cell > MCC_MAX_SEGMENT) return MCC_ERR_TOO_LARGE;
    const int32_t mc = max_cell > 0 ? max_cell : 1;
    const int32_t ep = max_corr_passes * (mc / 2 + 1) + 1;
    *bytes = mcc::adjoint_slab_bytes(mc, ep) * (size_t)(n_cells > 0 ? n_cells : 1);
    return MCC_OK;
}

int mcc_adjoint(mcc_ctx* ctx, const mcc_particles* P, const int64_t* offsets, int32_t n_cells, int32_t n_species,
                const mcc_species* sp, const double* lnL, int32_t sa, int32_t sb, int32_t inter, const mcc_params* p,
                int32_t max_cell, double* vx_out, double* vy_out, double* vz_out, double* gvx, double* gvy,
                double* gvz, double* gw, double* glnL, int32_t tape, void* ws, size_t ws_bytes, mcc_stream stream)
{
    NvtxRange nvtx_("mcc_adjoint");
    if (!ctx || !P || !offsets || !sp || !lnL || !valid_params(p) || inter < 0 || inter > 0xFFFFFF || max_cell < 0)
        return MCC_ERR_INVALID_ARG;
    if (max_cell > MCC_MAX_SEGMENT) return MCC_ERR_TOO_LARGE;
    if (P->prec != MCC_F64 || p->relativistic || p->weighting != 0 || p->pairing != 0) return MCC_ERR_INVALID_ARG;
    const bool fwd = vx_out || vy_out || vz_out, rev = gvx || gvy || gvz;
    if (fwd && !(vx_out && vy_out && vz_out)) return MCC_ERR_INVALID_ARG;
    if (rev && !(gvx && gvy && gvz && gw && glnL)) return MCC_ERR_INVALID_ARG;
    if (tape < MCC_ADJOINT_RECOMPUTE || tape > MCC_ADJOINT_REPLAY || (tape == MCC_ADJOINT_REPLAY && fwd))
        return MCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    StepArgs a;
    const int32_t ab[2] = {sa, sb};
    int rc = fill_args(a, ctx, P, offsets, n_cells, n_species, sp, lnL, ab, 1, inter, p);
    if (rc != MCC_OK) return rc;
    if (n_cells == 0 || (!fwd && !rev)) return MCC_OK;
    size_t need = 0;
    if (tape == MCC_ADJOINT_RECOMPUTE) mcc_adjoint_workspace_size(ctx, n_cells, max_cell, p->max_corr_passes, &need);
    else mcc_adjoint_tape_size(ctx, n_cells, max_cell, p->max_corr_passes, &need);
    if (!ws || ws_bytes < need) return MCC_ERR_WORKSPACE;
    const int32_t mc = max_cell > 0 ? max_cell : 1;
    const int32_t ep = p->max_corr_passes * (mc / 2 + 1) + 1;
    const cudaError_t e = mcc::launch_adjoint(a, lnL[sa * n_species + sb], vx_out, vy_out, vz_out, gvx, gvy, gvz, gw,
                                              glnL, reinterpret_cast<char*>(ws), mc, ep, tape,
                                              adjoint_grid(ctx, n_cells), S(stream));
    ctx->launches += 1;
    return cuda_status(e);
}

int mcc_sync_status(mcc_ctx* ctx, mcc_stream stream)
{
    if (!ctx) return MCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return MCC_ERR_CUDA;
    int32_t st = 0;
    if (cudaMemcpy(&st, ctx->dbuf, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess) return MCC_ERR_CUDA;
    if (cudaMemset(ctx->dbuf, 0, sizeof(int32_t)) != cudaSuccess) return MCC_ERR_CUDA;
    return st;
}

int64_t mcc_launch_count(mcc_ctx* ctx) { return ctx ? ctx->launches : -1; }

int mcc_debug_record(mcc_ctx* ctx, mcc_stream stream, int32_t* out)
{
    if (!ctx || !out) return MCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return MCC_ERR_CUDA;
    if (cudaMemcpy(out, ctx->dbuf + 4, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return MCC_ERR_CUDA;
    if (cudaMemset(ctx->dbuf + 4, 0, 4 * sizeof(int32_t)) != cudaSuccess) return MCC_ERR_CUDA;
    return MCC_OK;
}

int mcc_phase_clocks(mcc_ctx* ctx, mcc_stream stream, uint64_t* out)
{
    if (!ctx || !out) return MCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return MCC_ERR_CUDA;
    char* p = reinterpret_cast<char*>(ctx->dbuf) + kClkOffset;
    if (cudaMemcpy(out, p, kClkWords * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess) return MCC_ERR_CUDA;
    if (cudaMemset(p, 0, kClkWords * sizeof(uint64_t)) != cudaSuccess) return MCC_ERR_CUDA;
    return MCC_OK;
}

int mcc_phase_clocks_build(void)
{
#ifdef MCC_PHASE_CLOCKS
    return 1;
#else
    return 0;
#endif
}

int mcc_debug_bounds_build(void)
{
#ifdef MCC_DEBUG_BOUNDS
    return 1;
#else
    return 0;
#endif
}

int mcc_set_tile_cap(mcc_ctx* ctx, int32_t cap)
{
    if (!ctx || cap < 0) return MCC_ERR_INVALID_ARG;
    ctx->tile_cap = cap;
    return MCC_OK;
}

const char* mcc_status_string(int status)
{
    switch (status) {
    case MCC_OK: return "ok";
    case MCC_ERR_INVALID_ARG: return "invalid argument";
    case MCC_ERR_CUDA: return "CUDA error";
    case MCC_ERR_WORKSPACE: return "workspace missing or too small";
    case MCC_ERR_TIMEOUT: return "bounded wait timed out";
    case MCC_ERR_CORRECTION_FAILED: return "energy correction could not absorb the violation";
    case MCC_ERR_BOUNDS: return "index or cell size out of bounds";
    case MCC_ERR_TOO_LARGE: return "segment larger than supported";
    default: return "unknown status";
    }
}

}  // extern "C"
