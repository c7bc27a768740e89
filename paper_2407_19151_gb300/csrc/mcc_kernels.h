// Launch interface between the C ABI (mcc_abi.cu) and the kernel translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mcc_device.cuh"

namespace mcc {

enum Mode { kFused = 0, kPair = 1, kScatter = 2, kCorrect = 3 };

// Per-interaction constants, precomputed on the host in FP64 (and rounded once for the mixed path).
struct InterConst {
    int32_t a, b;
    double kappa_mu2;  // q_a^2 q_b^2 lnL_ab dt / (4 pi eps0^2 dV) / mu^2: s = kappa_mu2 w_max N_min / u^3
    double kappa;      // same without 1/mu^2 (relativistic: s = kappa w_max N_min / (|p*|^2 v_rel*))
    double mu_ma, mu_mb;
    float kappa_mu2_f, kappa_f, mu_ma_f, mu_mb_f;
};

struct StepArgs {
    const int64_t* offsets;
    int32_t n_cells, S;
    int64_t n_total;
    void* vx;
    void* vy;
    void* vz;
    const double* w;
    double m[kMaxSpecies];
    float m_f[kMaxSpecies];
    float m_lo[kMaxSpecies];  // m - m_f rounded to float: (m_f, m_lo) is m as float-float
    double ma[kMaxSpecies];  // species masses for the relativistic kinematics
    float ma_f[kMaxSpecies];
    InterConst ic[kMaxInter];
    int32_t n_inter;
    int32_t inter_base;  // counter index of ic[0] (unfused calls: the interaction's index in the step)
    int32_t method, fail_policy, sort_by_weight, max_corr_passes, correct;
    int32_t weighting;  // 0: w_max N_min in s; 1: duplicity weighting (w_max / D_ij) N_max for inter-species pairs
    int32_t pairing;    // 0: order-N pairs; 1: all N x N pairs (fused step only)
    double c, fE;
    float c_f, fE_f;
    float fE_lo;              // fE - fE_f: (fE_f, fE_lo) is fE as float-float
    float gm1p_f, gm1p_lo;    // sqrt(1 - fE) - 1 as float-float (a capped energy pair that loses energy)
    float gm1n_f, gm1n_lo;    // sqrt(1 + fE) - 1 as float-float (a capped energy pair that gains energy)
    float c2inv_f, c2inv_lo;  // 1 / c^2 as float-float
    RngKey rng;
    const uint64_t* step_dev;  // step index in device memory (null: rng.step); step = *step_dev + step_add
    uint32_t step_add;
    const double* n97_f;   // N97 table (see mcc_device.cuh), double and float copies
    const double* n97_dh;
    const float* n97_f32;
    const float* n97_dh32;
    // unfused input / output
    int32_t* pair_i;
    int32_t* pair_j;
    uint8_t* pair_flags;
    void* backup;
    int32_t* corr_pairs;
    int32_t* fail_count;
    int32_t accumulate;
    // control
    int32_t* status;
    int32_t* queue;
    const int32_t* order;  // processing order of the cells (null: index order)
    int32_t cap;        // particles per cell staged in shared memory
    char* slab;         // per-CTA global slabs for larger cells (may be null)
    int64_t slab_stride;
    int32_t slab_cap;
    const int32_t* order_range;  // one-CTA kernel: [begin, end) of `order` to take cells from (null: every cell)
    // group kernels (mcc_group.cuh)
    const int32_t* class_off;  // [2 * kGroupClasses + 2]: begin / end of each size class in `order` (last: the rest)
    int32_t* queues;           // [kGroupClasses + 1] work-queue counters, one per class
    int32_t gcls;              // size class of the launch
    int32_t gcap;              // particles one group stages on chip in this class
    int32_t max_cell;          // the caller's bound on particles per cell (larger cells latch kErrBounds)
    double* resid;             // [2 * n_cells] or null: per-cell |dP| / sum m w |v| and |dE| / E of the exact state
    unsigned long long* phase_clk;  // [8 * kGroupClasses] cycles per phase and class (phase-timing builds)
};

constexpr int kGroupClasses = 5;  // group sizes 32, 64, 128, 256, 512 threads
#ifndef MCC_GROUP_WARPS_PER_SM
#define MCC_GROUP_WARPS_PER_SM 16
#endif
// Warps of the group kernels resident per SM: their register budget (launch bounds) and the automatic capacity
// (shared memory per warp) are both set for this many.
constexpr int kGroupWarpsPerSm = MCC_GROUP_WARPS_PER_SM;

// Bytes per particle of the cell tile (keys, weights, velocities, pre-scatter copy, permutation, weight order).
__host__ __device__ inline size_t tile_bytes_per_particle(bool f32) { return 8 + 8 + (f32 ? 6 * 4 : 6 * 8) + 4 + 4; }

// Shared-memory bytes per particle of the group kernels' cell tile (state, weight, scratch, two orders).
constexpr size_t kGroupBytesPerParticle = 44;

// N97 table: (f, h df/dx) at kN97Nodes + 1 nodes, computed on the host in double.
void n97_table(double* f, double* dh);

// Kernel launches (defined in mcc_cell.cu / mcc_bin.cu).
cudaError_t launch_cell(bool f32, bool rel, int mode, const StepArgs& a, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_step_advance(uint64_t* step, uint64_t by, cudaStream_t st);
cudaError_t launch_cell_order(const int64_t* offsets, int32_t n_cells, int32_t S, int32_t* order, cudaStream_t st);
// Cells ordered by group size class (largest class first; class kGroupClasses = cells above every class), largest
// first within a class; class_off receives each class's [begin, end) in `order`.
cudaError_t launch_group_order(const int64_t* offsets, int32_t n_cells, int32_t S, const int32_t* caps,
                               int32_t* order, int32_t* class_off, cudaStream_t st);
// Group kernels (mcc_group_*.cu): class cls runs groups of 32 << cls threads.
const void* group_kernel(bool f32, bool rel, int cls);
cudaError_t launch_group(bool f32, bool rel, int cls, const StepArgs& a, int grid, size_t smem, cudaStream_t st);
int cell_kernel_blocks_per_sm(bool f32, bool rel, int mode, size_t smem);
cudaError_t set_cell_smem_limit(bool f32, bool rel, int mode, size_t smem);
size_t cell_kernel_static_smem(bool f32, bool rel, int mode);

cudaError_t launch_bin(const int32_t* cell, const int32_t* species, int64_t n, int32_t n_cells, int32_t n_species,
                       int32_t* perm, int64_t* offsets, void* ws, int32_t* status, cudaStream_t st, int64_t* launches);
size_t bin_workspace_bytes(int64_t n, int64_t n_keys);
cudaError_t launch_bin_weighted(const int32_t* cell, const int32_t* species, const double* w, int64_t n,
                                int32_t n_cells, int32_t n_species, int32_t* perm, int64_t* offsets, void* ws,
                                int32_t* status, cudaStream_t st, int64_t* launches);
size_t bin_weighted_workspace_bytes(int64_t n, int64_t n_keys);
cudaError_t launch_bin_static(const int32_t* cell, const int32_t* species, int64_t n, int32_t n_cells,
                              int32_t n_species, int32_t* perm, int64_t* offsets, cudaStream_t st);
int64_t static_bin_max_keys();
// Adjoint of one interaction (mcc_adjoint.cu).
size_t adjoint_slab_bytes(int32_t max_cell, int32_t max_epairs);
cudaError_t launch_adjoint(const StepArgs& a, double lnL, double* ox, double* oy, double* oz, double* gx, double* gy,
                           double* gz, double* gw, double* glnL, char* slab, int32_t max_cell, int32_t max_epairs,
                           int32_t tape,
                           int grid, cudaStream_t st);
cudaError_t launch_gather(const void* in, const int32_t* perm, int64_t n, int elem_bytes, void* out, cudaStream_t st);

// Species masses for the per-species moments (mcc_species_moments).
struct SpeciesConst {
    double m[kMaxSpecies];
};
cudaError_t launch_species_moments(bool f32, const void* vx, const void* vy, const void* vz, const double* w,
                                   const int64_t* offsets, int32_t n_cells, int32_t S, const SpeciesConst& sc,
                                   int rel, double c, const int32_t* fail_count, double* out, int num_sms,
                                   cudaStream_t st);

}  // namespace mcc
