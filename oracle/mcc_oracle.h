/*
 * FP64 CPU oracle for the weighted, moment-preserving Monte-Carlo Coulomb collision step
 * (Angus et al., "Moment-preserving Monte-Carlo Coulomb collision method for particle codes").
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow, obviously-correct reference that the CUDA path is
 * checked against. Only the test suite, the smoke check and the benchmark's CPU-baseline leg load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Parity status per function (pins live in tests/test_oracle_*.py):
 *   orc_philox4x32_10      pinned: published Philox-4x32-10 known-answer values.
 *   orc_bin                pinned: equals a stable library sort by (cell, species).
 *   orc_bin_weighted       pinned: equals a library lexicographic sort by (cell, species, truncated weight, index).
 *   orc_nxn_slot           pinned: brute force, every pair of the cell exactly once, rounds disjoint.
 *   orc_pairs              pinned: brute-force structure checks and pairing-uniformity chi-square.
 *   orc_n97_A / angles     pinned: E[cos chi] = exp(-s) by quadrature, asymptotic limits, TA77 variance.
 *   orc_scatter            pinned: expected drag of Eqs. sb_TA_weighted / sa_TA77_weighted, isotropisation and
 *                          equilibration expectations computed by brute force over the N x N pairs.
 *   orc_correct            pinned: exact momentum/energy invariants, first-order limit Eqs. vp1_inelastic_2 /
 *                          vp2_inelastic_2, Test-1 closed-form equilibrium.
 *   orc_push               pinned: exact dyadic displacements and wraps, cell ids against exact rational floors,
 *                          relativistic displacements against 50-digit decimal arithmetic.
 *   relativistic pieces    pinned by invariants (4-momentum conservation, Eq. alpha_Eq0 residual, gamma->1 limit);
 *                          the relativistic scatter kinematics (no printed formula) against their definition by an
 *                          independent route: 50-digit Lorentz boosts into the CM frame show an elastic rotation by
 *                          exactly Theta, mirrored azimuths, and v_rel* as the CM velocity difference. The use of
 *                          |p*|^2 v_rel* in s is a reading, pinned only by its classical limit.
 */
#ifndef MCC_ORACLE_H
#define MCC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_TA77 = 0, ORC_N97 = 1 };
enum { ORC_FAIL_ROLLBACK = 0, ORC_FAIL_MOMENTUM_ONLY = 1, ORC_FAIL_ERROR = 2 };

typedef struct {
    int32_t method;          /* ORC_TA77 or ORC_N97 */
    int32_t relativistic;    /* 0: state is v; 1: state is proper velocity u = gamma v */
    double dt, dV, eps0, c, fE;
    int32_t sort_by_weight;  /* Algorithm 1 optional sort step */
    int32_t max_corr_passes;
    int32_t fail_policy;
    int32_t correct;         /* 0: scatter only, 1: scatter + moment correction */
    uint64_t seed;
    uint64_t step;
    int32_t weighting;       /* 0: the paper's s (w_max, N_min); 1: duplicity weighting (w_max / D_ij, N_max) */
    int32_t pairing;         /* 0: order-N pairs (Eq. sab_TA77); 1: all N x N pairs (Eq. sab_weighted) */
} orc_params;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

int orc_bin(const int32_t* cell, const int32_t* species, int64_t n, int32_t n_cells, int32_t n_species,
            int32_t* perm_out, int64_t* offsets_out);

int orc_bin_weighted(const int32_t* cell, const int32_t* species, const double* w, int64_t n, int32_t n_cells,
                     int32_t n_species, int32_t* perm_out, int64_t* offsets_out);

/* k-th pair slot of the order N x N schedule of a cell (local indices before the random permutations are applied):
 * inter: round r = k / N_min pairs the smaller population's m = k mod N_min with the larger one's (m + r) mod N_max;
 * intra: a round-robin tournament over N players (plus an idle player when N is odd), N/2 (rounded up) slots a round.
 * Returns 0 for a slot that pairs a particle with the idle player (no pair). */
int orc_nxn_slot(int64_t na, int64_t nb, int32_t intra, int64_t k, int64_t* ia, int64_t* jb);
int64_t orc_nxn_slots(int64_t na, int64_t nb, int32_t intra, int64_t* per_round);

int orc_permutation(int64_t n, uint64_t seed, uint64_t step, uint32_t cell, uint32_t inter, uint32_t side,
                    int32_t* perm_out);

int orc_pairs(const int64_t* offsets, int32_t n_cells, int32_t n_species, int32_t sa, int32_t sb, int32_t inter,
              uint64_t seed, uint64_t step, int32_t* pair_i, int32_t* pair_j, uint8_t* pair_flags);

double orc_n97_A(double s);
double orc_n97_L(double A);
void orc_angle(int32_t method, double s, double U1, double U4, double* sin_theta, double* one_minus_cos);
void orc_rotate(const double u[3], double sin_theta, double one_minus_cos, double phi, double du[3]);

void orc_energy_pair(int32_t relativistic, double c, double m1, double m2, double v1[3], double v2[3], double U);
double orc_pair_kecm(int32_t relativistic, double c, double m1, double m2, const double v1[3], const double v2[3]);
void orc_rel_scatter_dp(double c, double ma, double mb, const double ui[3], const double uj[3], double sin_theta,
                        double one_minus_cos, double phi, double dp[3], double* pstar, double* vrel);

int orc_scatter(double* vx, double* vy, double* vz, const double* w, const int64_t* offsets, int32_t n_cells,
                int32_t n_species, const double* q, const double* m, const double* lnL, int32_t sa, int32_t sb,
                int32_t inter, const orc_params* p, double* backup);

int orc_correct(double* vx, double* vy, double* vz, const double* w, const int64_t* offsets, int32_t n_cells,
                int32_t n_species, const double* m, int32_t sa, int32_t sb, int32_t inter, const orc_params* p,
                const double* backup, int32_t* corr_pairs, int32_t* fail_flags);

void orc_set_threads(int32_t n);

/* Free-streaming push of PIC coupling (Sec. 2, Eq. Boltzmann: the left-hand side advances positions, here with
 * a = 0) in a periodic box of nc[0] x nc[1] x nc[2] cells over [0, l[d]). prec 0: double positions and velocities,
 * prec 1: float. Every operation in that precision, rounded, no fused multiply-add; constants rounded once from
 * double (dt, l, c * c, nc / l). Positions updated in place; cell = ix + nx (iy + ny iz). */
int orc_push(int32_t prec, void* x, void* y, void* z, const void* vx, const void* vy, const void* vz, int64_t n,
             const int32_t nc[3], const double l[3], double dt, int32_t relativistic, double c, int32_t* cell);

int orc_step(double* vx, double* vy, double* vz, const double* w, const int64_t* offsets, int32_t n_cells,
             int32_t n_species, const double* q, const double* m, const double* lnL, const int32_t* interactions,
             int32_t n_inter, const orc_params* p, int32_t n_steps, int32_t cell_begin, int32_t cell_end,
             int32_t* corr_pairs, int32_t* fail_count);

#ifdef __cplusplus
}
#endif
#endif
