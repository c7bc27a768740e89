/*
 * mcc.h: C ABI of the GB300 (sm_103a) Monte-Carlo Coulomb collision step for weighted particles with exact
 * momentum and energy conservation (Angus et al., "Moment-preserving Monte-Carlo Coulomb collision method for
 * particle codes").
 *
 * The calls follow the paper's statement of the problem: weighted macro-particles in cells of volume dV
 * (Sec. 2, Eq. Klimintovich), a binary interaction between two species (Sec. 3, Sec. 4), and the steps of
 * Algorithm 1.
 *
 * Conventions (every entry point):
 *  - Device arrays are owned by the caller; the library never allocates per call. Host arrays are read before the
 *    call returns.
 *  - Every call is asynchronous on the stream it is given (0 = the legacy default stream) and returns MCC_OK once
 *    its work is enqueued. Argument errors detectable on the host are returned immediately and nothing is enqueued.
 *    Errors found on the device (a cell larger than the declared maximum, a failed energy correction under
 *    MCC_FAIL_ERROR, an invalid segment) are latched in the context's device status word and returned by
 *    mcc_sync_status.
 *  - Particles are stored binned (see mcc_bin): all particles of cell c and species s are contiguous in
 *    [offsets[c*S + s], offsets[c*S + s + 1]), cells in order, species in order within a cell.
 *  - Velocities are structure-of-arrays vx, vy, vz of doubles (MCC_F64) or floats (MCC_F32_MIXED); weights are
 *    always doubles and must be positive and finite. In relativistic mode the stored quantity is the proper
 *    velocity u = gamma v (Appendix A).
 *  - No call traps or spins without a bound; no exception crosses the ABI.
 */
#ifndef MCC_H
#define MCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcc_ctx mcc_ctx;
typedef struct CUstream_st* mcc_stream; /* a cudaStream_t */

typedef enum {
    MCC_OK = 0,
    MCC_ERR_INVALID_ARG = -1,
    MCC_ERR_CUDA = -2,
    MCC_ERR_WORKSPACE = -3,
    MCC_ERR_TIMEOUT = -4,
    MCC_ERR_CORRECTION_FAILED = -5,
    MCC_ERR_BOUNDS = -6,
    MCC_ERR_TOO_LARGE = -7
} mcc_status;

typedef enum { MCC_TA77 = 0, MCC_N97 = 1 } mcc_method;
typedef enum { MCC_F64 = 0, MCC_F32_MIXED = 1 } mcc_precision;
typedef enum { MCC_FAIL_ROLLBACK = 0, MCC_FAIL_MOMENTUM_ONLY = 1, MCC_FAIL_ERROR = 2 } mcc_fail_policy;

/* Maximum species per call and maximum particles per (cell, species) segment. Cell-local particle indices are packed
 * into 20 bits of the pairing keys; the entry points that take max_cell (mcc_step_fused, mcc_adjoint and their
 * workspace sizes) return MCC_ERR_TOO_LARGE for max_cell above MCC_MAX_SEGMENT, and cells above max_cell latch
 * MCC_ERR_BOUNDS and are skipped, so no segment above the limit is ever processed. */
#define MCC_MAX_SPECIES 8
#define MCC_MAX_SEGMENT (1 << 20)

/* Charge and (unweighted) mass of one species. */
typedef struct {
    double q;
    double m;
} mcc_species;

/* Binned particle arrays on the device (caller-owned). prec selects float or double for vx, vy, vz. */
typedef struct {
    void* vx;
    void* vy;
    void* vz;
    const double* w;
    int64_t n;
    int32_t prec; /* mcc_precision */
} mcc_particles;

/* Step parameters. dt, dV, eps0 enter the scattering length of Eq. sab_TA77; c is used in relativistic mode;
 * fE is the energy-correction factor of Eq. U_inelastic; sort_by_weight is the optional sort of Algorithm 1;
 * max_corr_passes bounds the energy-pair passes; correct = 0 runs the scatter alone. seed keys the random stream;
 * step is the time-step index that enters every random counter (taken modulo 2^32); cell_base offsets the cell
 * counter for sharded runs (0 for a whole problem). */
typedef struct {
    int32_t method;       /* mcc_method */
    int32_t relativistic; /* 0 or 1 */
    double dt, dV, eps0, c, fE;
    int32_t sort_by_weight;
    int32_t max_corr_passes;
    int32_t fail_policy; /* mcc_fail_policy */
    int32_t correct;
    uint64_t seed;
    uint64_t step;
    uint32_t cell_base; /* global id of the first cell (the random counters use global cell ids, so a shard of
                           cells [cell_base, cell_base + n_cells) draws exactly what the unsharded run draws) */
    int32_t weighting;  /* 0: s with w_max N_min (Eq. sab_TA77); 1: duplicity weighting, the alternative the paper
                           describes in Sec. 3.2 (Higginson et al.): (w_max / D_ij) N_max for inter-species pairs,
                           D_ij the number of times the smaller population's particle is paired. mcc_adjoint
                           requires 0. */
    int32_t pairing;    /* 0: order-N pairs (Eq. sab_TA77); 1: order N x N (Sec. 3.1, Eq. sab_weighted): every pair
                           of the interaction once per step, in rounds of disjoint pairs over the interaction's random
                           permutations (inter: round r pairs the smaller population's m with the larger one's
                           (m + r) mod N_max; intra: a round-robin tournament), the draw keyed by the slot, s with
                           w_max alone. Fused step only: mcc_pair, mcc_scatter and mcc_adjoint require 0. */
    uint64_t* step_device; /* mcc_step_fused only (null: use step): the step index lives in device memory; step t of
                              a call draws with *step_device + t, and the call adds n_steps to it on its stream after
                              the last step, so that a CUDA graph captured from one call serves every later step */
    double* residual;      /* mcc_step_fused only, nullable: [2 * n_cells] device doubles receiving, per cell of the
                              last step, the conservation of the state held on chip before it is stored (float-float
                              on the mixed path): max_d |P_d - P0_d| / sum m w |v| and |E - E0| / E0, P0 and E0 the
                              cell's momentum and kinetic energy when the step loaded it (Sec. 4: the correction
                              conserves both exactly). Written for every cell of at most the largest group capacity
                              (mcc_group_capacities); other cells are left as they are. */
    void** launch_events;  /* mcc_step_fused only, nullable: 2 * (MCC_GROUP_CLASSES + 1) cudaEvent_t created by the
                              caller; in the last step of the call, events [2k] and [2k + 1] are recorded on the
                              stream just before and after the kernel of size class k (k = MCC_GROUP_CLASSES: the
                              one-CTA kernel of the cells above every class), back to back for a class that is not
                              launched, so that each class kernel can be timed with cudaEventElapsedTime; under
                              stream capture they are recorded as event-record nodes of the graph */
} mcc_params;

#define MCC_GROUP_CLASSES 5

/* Create / destroy a context on `device`. The context owns only a small device buffer (status word, work-queue
 * counter) allocated here, once. */
int mcc_create(mcc_ctx** ctx, int device);
void mcc_destroy(mcc_ctx* ctx);

/* Bytes of device workspace mcc_adjoint needs for n_cells cells of at most max_cell particles when it recomputes
 * (tape = MCC_ADJOINT_RECOMPUTE: one working slab per resident CTA). */
int mcc_adjoint_workspace_size(mcc_ctx* ctx, int32_t n_cells, int32_t max_cell, int32_t max_corr_passes,
                               size_t* bytes);

/* Bytes of one recorded tape of one interaction (tape = MCC_ADJOINT_RECORD / MCC_ADJOINT_REPLAY: one slab per cell,
 * about 250 bytes per particle of max_cell plus 80 bytes per possible energy pair). */
int mcc_adjoint_tape_size(mcc_ctx* ctx, int32_t n_cells, int32_t max_cell, int32_t max_corr_passes, size_t* bytes);

#define MCC_ADJOINT_RECOMPUTE 0
#define MCC_ADJOINT_RECORD 1
#define MCC_ADJOINT_REPLAY 2

/*
 * mcc_adjoint: one interaction (sa, sb) of a step, recomputed from its input state, and optionally its pathwise
 * adjoint. Every random draw and discrete decision is held fixed (Philox draws, permutations and TA77 pairs, the
 * heavier particle's accept test, the weight order, the energy-correction passes and the crossing pair); through the
 * smooth rest of the interaction (Sec. 3.2 s and angle, Eq. vp_pm, Eq. Econs, Eq. DeltaEs, Eqs. vp1/vp2_inelastic,
 * U_inelastic; the Sec. 5.2 rollback) it maps dL/dv after the interaction to dL/dv before it and adds dL/dw and
 * dL/dlnL_ab. Non-relativistic, FP64 (P->prec == MCC_F64) only.
 *   P               state BEFORE the interaction (device, binned; read only)
 *   inter, p        the interaction's index in the step and the step's parameters, as for mcc_scatter
 *   max_cell        largest cell (particles); larger cells latch MCC_ERR_BOUNDS
 *   v*_out          [n] device: the state after the interaction (all three or none; untouched particles copied)
 *   gv*             [n] device, in place: in dL/dv after, out dL/dv before (all of gv*, gw, glnL or none)
 *   gw              [n] device: dL/dw accumulated (+=)
 *   glnL            device, one double: dL/dlnL_ab accumulated (+=, atomically over cells)
 *   tape            MCC_ADJOINT_RECOMPUTE: the call runs the forward (and the reverse sweep if asked) in working
 *                   slabs of ws, nothing kept. MCC_ADJOINT_RECORD: the same, and ws (mcc_adjoint_tape_size bytes)
 *                   keeps every cell's tape afterwards. MCC_ADJOINT_REPLAY: the reverse sweep alone, from the tape a
 *                   recording call on this interaction left in ws (same state, weights, lnL and parameters; the
 *                   caller keeps them unchanged in between); P's velocities are not read, v*_out must be NULL.
 *   ws, ws_bytes    at least mcc_adjoint_workspace_size bytes (recompute) or mcc_adjoint_tape_size bytes (record,
 *                   replay)
 * The recomputed forward equals mcc_scatter followed by mcc_correct for the same inputs (energy passes run in order);
 * a replayed reverse sweep equals the recomputing one bit for bit. Tape overflow latches MCC_ERR_TOO_LARGE.
 */
int mcc_adjoint(mcc_ctx* ctx, const mcc_particles* P, const int64_t* offsets, int32_t n_cells, int32_t n_species,
                const mcc_species* sp, const double* lnL, int32_t sa, int32_t sb, int32_t inter, const mcc_params* p,
                int32_t max_cell, double* vx_out, double* vy_out, double* vz_out, double* gvx, double* gvy,
                double* gvz, double* gw, double* glnL, int32_t tape, void* ws, size_t ws_bytes, mcc_stream stream);

/* Bytes of device workspace mcc_bin needs for n particles and n_keys = n_cells * n_species segments. */
int mcc_bin_workspace_size(int64_t n, int32_t n_cells, int32_t n_species, size_t* bytes);

/*
 * mcc_bin: cell sort (Sec. 2: particles are collided per cell of volume dV).
 * Stable counting sort of particle indices by key = cell[i] * n_species + species[i].
 *   cell, species   [n] device int32, cell in [0, n_cells), species in [0, n_species)
 *   perm_out        [n] device int32: perm_out[k] = index of the k-th particle in binned order; stable, so equal
 *                   keys keep increasing index
 *   offsets_out     [n_cells * n_species + 1] device int64: segment starts, offsets_out[last] = n
 *   ws, ws_bytes    device workspace of at least mcc_bin_workspace_size bytes
 * Out-of-range keys latch MCC_ERR_BOUNDS (those particles are dropped from the output).
 * A segment larger than MCC_MAX_SEGMENT latches MCC_ERR_TOO_LARGE.
 */
int mcc_bin(mcc_ctx* ctx, const int32_t* cell, const int32_t* species, int64_t n, int32_t n_cells,
            int32_t n_species, int32_t* perm_out, int64_t* offsets_out, void* ws, size_t ws_bytes,
            mcc_stream stream);

/* Bytes of device workspace mcc_bin_weighted needs (mcc_bin's counters plus 8 bytes per particle). */
int mcc_bin_weighted_workspace_size(int64_t n, int32_t n_cells, int32_t n_species, size_t* bytes);

/*
 * mcc_bin_weighted: the cell sort of mcc_bin with every (cell, species) segment stored in the order of the optional
 * weight sort of Algorithm 1 (the energy-correction pairs run from the heaviest particle down): descending weight,
 * the weights compared by their IEEE bits truncated to sign, exponent and 32 fraction bits (weights that agree to
 * 2^-32 relative tie), ties in increasing particle index. In this layout the fused step finds each segment with
 * distinct truncated weights already in weight order and skips its per-visit sort; any other layout gives the same
 * results per layout, only with that sort.
 *   w               [n] device double, the particle weights (positive, finite), in the caller's (unbinned) order
 *   other arguments as mcc_bin; ws, ws_bytes at least mcc_bin_weighted_workspace_size bytes
 * Errors as mcc_bin.
 */
int mcc_bin_weighted(mcc_ctx* ctx, const int32_t* cell, const int32_t* species, const double* w, int64_t n,
                     int32_t n_cells, int32_t n_species, int32_t* perm_out, int64_t* offsets_out, void* ws,
                     size_t ws_bytes, mcc_stream stream);

/*
 * mcc_bin_static: the same cell sort as mcc_bin for callers that cannot allocate device memory at all, such as
 * code running under an allocator that must not grow, inside a host callback or driver-level integration where
 * cudaMalloc is unavailable, or a caller without a context to own a workspace. It takes no context and no
 * workspace: its counters live in one file-scope device array of MCC_BIN_STATIC_MAX_KEYS segment counters (three
 * int32 arrays, about 24 MiB) that every GPU loading this library holds until the process exits. The paper has no
 * counterpart; this is an allocation-free variant of mcc_bin.
 *   Arguments and outputs as mcc_bin; n_cells * n_species above MCC_BIN_STATIC_MAX_KEYS returns MCC_ERR_TOO_LARGE
 *   before any work is enqueued. It calls no cudaMalloc, cudaFree or allocating library routine.
 *   The first call on a device looks up that device's address of the array (cudaGetSymbolAddress, with the device
 *   current), so make the first call on each device before any stream capture.
 *   Every call clears the counters it uses on its stream before use, but all calls share the one array: calls that
 *   overlap on the GPU (different streams, or a second call before the first finished) race.
 *   There is no status word: particles with out-of-range cell or species are dropped, which shows as
 *   offsets_out[last] < n, and a (cell, species) segment above MCC_MAX_SEGMENT particles is not reported here (the
 *   context-owning mcc_bin latches MCC_ERR_TOO_LARGE for it). The step entry points catch it downstream: their
 *   max_cell is at most MCC_MAX_SEGMENT, so such a cell latches MCC_ERR_BOUNDS and is skipped.
 *   stream must belong to the current device (MCC_ERR_INVALID_ARG otherwise): the counters' address is the
 *   current device's.
 */
#define MCC_BIN_STATIC_MAX_KEYS (1 << 21)
int mcc_bin_static(const int32_t* cell, const int32_t* species, int64_t n, int32_t n_cells, int32_t n_species,
                   int32_t* perm_out, int64_t* offsets_out, mcc_stream stream);

/*
 * Per-species moments of a binned state, the diagnostics a sharded run sums over its ranks once per step (cells are
 * independent within a step, Sec. 2, so the ranks exchange nothing else). For each species s, out[6 s + k]:
 *   k = 0  sum w_p                 k = 1..3  sum m_s w_p v_p (component k - 1)
 *   k = 4  sum of the kinetic energy, m_s w_p |v_p|^2 / 2 (relativistic: m_s w_p c^2 (gamma_p - 1), v_p the proper
 *          velocity, gamma_p = sqrt(1 + |v_p|^2 / c^2))
 *   k = 5  the number of particles
 * and out[6 n_species] = sum over cells of fail_count (0 when fail_count is NULL).
 *   offsets       [n_cells * n_species + 1] device int64 segment offsets (cell-major)
 *   fail_count    [n_cells] device int32 or NULL (as accumulated by mcc_step_fused)
 *   out           [6 n_species + 1] device doubles, overwritten (cleared on the stream first)
 * Sums in FP64; partial sums are combined with double atomics, so the rounding of the result may differ between
 * runs. Errors: MCC_ERR_INVALID_ARG for a bad argument or species mass, MCC_ERR_CUDA for a launch failure.
 */
int mcc_species_moments(mcc_ctx* ctx, const mcc_particles* particles, const int64_t* offsets, int32_t n_cells,
                        int32_t n_species, const mcc_species* sp, int32_t relativistic, double c,
                        const int32_t* fail_count, double* out, mcc_stream stream);

/* Gather a double or float array through perm: out[k] = in[perm[k]] (elem_bytes 4 or 8). */
int mcc_gather(const void* in, const int32_t* perm, int64_t n, int32_t elem_bytes, void* out, mcc_stream stream);

/* mcc_gather for up to MCC_MAX_GATHER arrays in one pass over perm: out[a][k] = in[a][perm[k]].
 *   in, out, elem_bytes   host arrays of n_arrays entries (device pointers; elem_bytes 4 or 8 each); in[a] and
 *                         out[a] must not overlap
 *   n_arrays              1 .. MCC_MAX_GATHER */
#define MCC_MAX_GATHER 8
int mcc_gather_n(const void* const* in, void* const* out, const int32_t* elem_bytes, int32_t n_arrays,
                 const int32_t* perm, int64_t n, mcc_stream stream);

/*
 * Particle push for PIC coupling. The collision operator is the right-hand side of the Boltzmann equation
 * (Sec. 2, Eq. Boltzmann); a particle-in-cell code advances positions by the left-hand side between collision
 * steps, and the particles then have to be re-binned (mcc_bin) before the next step. mcc_push is the free-streaming
 * part of that advance (the acceleration a = 0): x <- x + v dt per axis, v = u / gamma with
 * gamma = sqrt(1 + |u|^2 / c^2) in relativistic mode (u the stored proper velocity), in a periodic box, and it writes
 * each particle's new cell id for mcc_bin.
 *
 * The grid: nx x ny x nz cells over the box [0, lx) x [0, ly) x [0, lz); cell id = ix + nx * (iy + ny * iz).
 * Arithmetic, in the precision T of the positions (double for MCC_F64, float for MCC_F32_MIXED), every operation
 * rounded to nearest with no fused multiply-add, constants rounded once from double to T: dt, L = l, c2 = c * c
 * (product in double) and sx = nx / lx (quotient in double):
 *   gamma_inv = 1 / sqrt(1 + ((ux*ux + uy*uy) + uz*uz) / c2)   (relativistic; 1 otherwise)
 *   x' = x + (u * gamma_inv) * dt                               (non-relativistic: x + u * dt)
 *   if x' is outside [0, L): r = x' - floor(x' / L) * L; if r < 0, r = r + L; if r >= L, r = r - L; a result
 *   still outside [0, L) (a non-finite x') becomes 0
 *   ix = (int)(x' * sx), at most nx - 1
 * so a host program doing the same operations in T gets the same positions and cell ids bit for bit.
 *   P            velocities (P->prec selects T) and n; P->w is not read
 *   x, y, z      [n] device T: positions in the box, updated in place
 *   cell_out     [n] device int32: the new cell ids
 *   nx, ny, nz   >= 1, nx * ny * nz <= INT32_MAX; lx, ly, lz > 0 and finite; dt finite; c > 0 if relativistic
 */
typedef struct {
    int32_t nx, ny, nz;
    double lx, ly, lz;
} mcc_grid;
int mcc_push(const mcc_particles* P, void* x, void* y, void* z, const mcc_grid* grid, double dt,
             int32_t relativistic, double c, int32_t* cell_out, mcc_stream stream);

/*
 * mcc_pair: random binary pairs of Takizuka-Abe for interaction `inter` between species sa <= sb
 * (Sec. 3.2, Fig. TApairing; Algorithm 1, second step).
 *  intra (sa == sb, n particles): n < 2 none; n even (p0,p1),(p2,p3),...; n odd: (p0,p1),(p1,p2),(p2,p0) with
 *    half the scattering length (flag bit 0) then (p3,p4),...
 *  inter: N_max pairs; pair k = (k-th of the larger population, (k mod N_min)-th of the smaller), each population
 *    in its own random order. p is the random permutation: local indices sorted by a 64-bit key made of 44
 *    Philox-4x32-10 bits (counter = {i/2, cell, step, inter<<8 | 1 + side}, key = seed) and the index (20 bits).
 * Output slots: cell c's pairs start at offsets[c * n_species] (its first particle); a cell never has more pairs
 * than particles, so pair_i / pair_j / pair_flags of length n suffice. Entries beyond a cell's pair count are not
 * written. pair_i holds species-sa particles, pair_j species-sb particles, both as global binned indices.
 * A cell is paired in one CTA's shared memory (20 B per particle: about 11,000 particles on GB300); a larger cell
 * is skipped and latches the bounds error (MCC_ERR_BOUNDS from mcc_sync_status).
 */
int mcc_pair(mcc_ctx* ctx, const int64_t* offsets, int32_t n_cells, int32_t n_species, int32_t sa, int32_t sb,
             int32_t inter, uint64_t seed, uint64_t step, int32_t* pair_i, int32_t* pair_j, uint8_t* pair_flags,
             mcc_stream stream);

/*
 * mcc_scatter: the pair loop of Algorithm 1 for interaction (sa, sb).
 * For each pair in list order: s = q_a^2 q_b^2 lnL_ab w_max N_min dt / (4 pi eps0^2 mu^2 u^3 dV) (Eq. sab_TA77;
 * N_min = N - 1 intra, halved for triplet pairs), TA77 or N97 angle, rotation of u about itself, the lighter particle
 * updated, the heavier with probability w_min / w_max (Sec. 3.2). Pairs sharing a particle run in list order.
 * Relativistic mode rotates the centre-of-momentum momentum instead.
 *   sp[n_species], lnL[n_species * n_species]: host arrays (species constants, Coulomb logarithm per pair)
 *   pair_*: output of mcc_pair for the same (sa, sb, inter, seed, step)
 *   backup: device, 3 * n values of the particle precision ([x | y | z] planes, binned index): receives the
 *           pre-scatter velocities of every particle of species sa and sb (used by mcc_correct)
 * mcc_scatter and mcc_correct hold a cell in one CTA's shared memory (72 B per particle in FP64, about 3,100
 * particles on GB300; 48 B on the mixed path, about 4,700); a larger cell is skipped and latches MCC_ERR_BOUNDS.
 * mcc_step_fused has no such limit (its workspace holds the cells above the on-chip tile).
 */
int mcc_scatter(mcc_ctx* ctx, const mcc_particles* particles, const int64_t* offsets, int32_t n_cells,
                int32_t n_species, const mcc_species* sp, const double* lnL, int32_t sa, int32_t sb, int32_t inter,
                const int32_t* pair_i, const int32_t* pair_j, const uint8_t* pair_flags, const mcc_params* params,
                void* backup, mcc_stream stream);

/*
 * mcc_correct: the moment correction of Algorithm 1 for interaction (sa, sb) (Sec. 4; Appendix A).
 * Momentum shift v -= B w_p with B = sum m_p (v_ps - v_bs) / sum m_p w_p (Eq. vp_pm); energy violation (Eq. Econs)
 * split between species (Eq. DeltaEs); per species, particles in descending weight order (ties in random order;
 * optional) paired (r0,r1),(r2,r3),... then offset by one on the next pass, each pair's centre-of-mass energy lowered
 * by U = sign(D) min(|D|, fE KE_cm) (Eqs. vp1_inelastic, vp2_inelastic, vrel_inelastic, U_inelastic) until D = 0.
 * If D != 0 after max_corr_passes passes the fail policy applies (Sec. 5.2).
 *   backup            the pre-scatter velocities written by mcc_scatter
 *   corr_pairs_out    [n_cells] device int32 or NULL: energy pairs used per cell (written)
 *   fail_flags_out    [n_cells] device int32 or NULL: 1 where the correction failed (written)
 */
int mcc_correct(mcc_ctx* ctx, const mcc_particles* particles, const int64_t* offsets, int32_t n_cells,
                int32_t n_species, const mcc_species* sp, int32_t sa, int32_t sb, int32_t inter,
                const mcc_params* params, const void* backup, int32_t* corr_pairs_out, int32_t* fail_flags_out,
                mcc_stream stream);

/* Bytes of device workspace mcc_step_fused needs for n_cells cells of at most max_cell particles: the cells'
 * processing order, plus per-CTA slabs when some cells exceed the on-chip tile. */
int mcc_step_workspace_size(mcc_ctx* ctx, int32_t prec, int32_t n_cells, int32_t max_cell, size_t* bytes);

/*
 * mcc_step_fused: n_steps whole collision steps (Algorithm 1 for every interaction in list order, each step with
 * index params->step + t). A small kernel orders the cells once per call by size class (mcc_group_capacities),
 * largest first; each step then launches one persistent kernel per non-empty class, in which a group of 32 << k
 * threads takes cells from the class's work queue, stages the cell in shared memory, runs pairing, scatter and
 * correction for every interaction and writes the cell back. Cells above every class run on a one-CTA kernel (from
 * its workspace slab when larger than its on-chip tile). For MCC_F64 the result equals the sequence
 * mcc_pair / mcc_scatter / mcc_correct over the interactions (up to rounding). For MCC_F32_MIXED the velocities of
 * a cell are held as float-float on chip for the whole step, the pair kinematics run in float and every sum,
 * coefficient and energy pair in float-float; they are rounded to float once, when stored.
 *   interactions   host int32 [2 * n_inter], pairs (a, b) with a <= b; interaction k uses index k in the counters
 *   max_cell       an upper bound on particles per cell, at most MCC_MAX_SEGMENT (else MCC_ERR_TOO_LARGE); cells
 *                  above it latch MCC_ERR_BOUNDS and are skipped
 *   corr_pairs     [n_cells] device int32 or NULL: accumulated energy pairs
 *   fail_count     [n_cells] device int32 or NULL: accumulated failed corrections
 *   ws, ws_bytes   workspace of mcc_step_workspace_size bytes
 */
int mcc_step_fused(mcc_ctx* ctx, const mcc_particles* particles, const int64_t* offsets, int32_t n_cells,
                   int32_t n_species, const mcc_species* sp, const double* lnL, const int32_t* interactions,
                   int32_t n_inter, const mcc_params* params, int32_t n_steps, int32_t max_cell,
                   int32_t* corr_pairs, int32_t* fail_count, void* ws, size_t ws_bytes, mcc_stream stream);

/* Particles staged on chip per cell by the one-CTA kernel of mcc_step_fused, which takes the cells above the
 * largest group class (0 = automatic: the largest tile with which six CTAs share an SM's shared memory, or the
 * largest cell if smaller). Cells above it run from the workspace slabs. */
int mcc_set_tile_cap(mcc_ctx* ctx, int32_t cap);

/* Size classes of mcc_step_fused's group kernels: class k (k = 0..4) runs groups of 32 << k threads and takes the
 * cells of at most caps[k] particles (the smallest such k); cells above caps[4] run on the one-CTA kernel.
 * particles_per_warp sets caps[k] = particles_per_warp << k for k < 4 (0 = automatic: the capacity with which
 * sixteen warps share an SM's shared memory); largest sets caps[4] (0 = as large as one CTA's shared memory
 * allows). Every capacity is capped by what one CTA's shared memory holds (44 bytes per particle). Both 0 is the
 * default. Used by the autotuner; the step's results do not depend on it. */
int mcc_set_group_capacity(mcc_ctx* ctx, int32_t particles_per_warp, int32_t largest);

/* The five class capacities mcc_step_fused uses for this precision and mode (caps_out: host int32[5]). */
int mcc_group_capacities(mcc_ctx* ctx, int32_t prec, int32_t relativistic, int32_t* caps_out);

/* Synchronise `stream`, read and clear the device status word; returns MCC_OK or the first latched error. */
int mcc_sync_status(mcc_ctx* ctx, mcc_stream stream);

/* Number of kernel launches enqueued through this context since creation (for launch accounting). */
int64_t mcc_launch_count(mcc_ctx* ctx);

/* Bounds-checked builds (compiled with -DMCC_DEBUG_BOUNDS; mcc_debug_bounds_build() returns 1 there, 0 otherwise):
 * the group kernels of mcc_step_fused check every index into the on-chip tile and every computed global index
 * against its bound; the first violation latches MCC_ERR_BOUNDS and is recorded, and the access uses index 0
 * instead. mcc_debug_record synchronises `stream` and returns (source line, index, bound, count of violations) in
 * out[0..3] (all zero if none), then clears the record. In other builds the record stays zero. */
int mcc_debug_record(mcc_ctx* ctx, mcc_stream stream, int32_t* out);
int mcc_debug_bounds_build(void);

/* Phase-timing builds (compiled with -DMCC_PHASE_CLOCKS; mcc_phase_clocks_build() returns 1 there, 0 otherwise):
 * the group kernels of mcc_step_fused add, per cell visit, the SM clock cycles of each phase, as thread 0 of the
 * group sees them (barrier waits included), to per-class counters. mcc_phase_clocks synchronises `stream`, returns
 * out[8 * k + q] for class k (0..4) and phase q (0 load and weight order, 1 permutations, 2 pair loop, 3 momentum
 * sums and B, 4 shift and energy sums, 5 energy pairs, 6 write-back; q = 7: cell visits) and clears the counters.
 * out: host uint64[40]. In other builds the counters stay zero. */
int mcc_phase_clocks(mcc_ctx* ctx, mcc_stream stream, uint64_t* out);
int mcc_phase_clocks_build(void);

const char* mcc_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif
