/*
 * FP64 CPU oracle for the weighted, moment-preserving Monte-Carlo Coulomb collision step.
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow, obviously-correct restatement of the paper's method, used to check
 * the CUDA path. Only the tests, the smoke check and the benchmark's CPU-baseline leg load it. It shares no
 * code with the CUDA library. Everything is IEEE double, built with -ffp-contract=off, round-to-nearest.
 *
 * Method (paper sections in brackets):
 *   - weighted macro-particles f = sum_i w_i delta(v - v_i) / dV per cell                      [Sec. 2, Eq. Klimintovich]
 *   - order-N random pairing of Takizuka-Abe, intra- and inter-species                           [Sec. 3.2, Fig. TApairing]
 *   - pair scattering length s = q_a^2 q_b^2 lnL w_max N_min dt / (4 pi eps0^2 mu^2 u^3 dV)    [Eq. sab_TA77]
 *   - TA77 / N97 centre-of-mass angle from s, lighter particle always updated, heavier one with
 *     probability w_min / w_max                                                                  [Sec. 3.2, Algorithm 1]
 *   - momentum restored by a weight-biased shift                                                 [Eq. vp_pm]
 *   - energy violation, partitioned between species, re-absorbed by zero-angle inelastic pairs   [Eqs. Econs, DeltaEs,
 *                                                                                                  vp1/vp2/vrel/U_inelastic]
 *   - relativistic variant on proper velocity with the quadratic for alpha                        [Appendix A]
 *   - failure fallback (roll the cell back to its pre-scatter velocities)                         [Sec. 5.2]
 *
 * Random numbers: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), keyed by the 64-bit seed; the counter is
 * (index, cell, step, tag). Every draw the method makes is a pure function of that counter, so a GPU
 * implementation can reproduce it draw for draw.
 */
#include "mcc_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------------------------
 * Philox-4x32-10, from its published description: ten rounds of two 32x32->64 multiplications whose high halves
 * are xored with the other two words and the round key; the key is bumped by two Weyl constants between rounds.
 * ---------------------------------------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter tags: which draw a Philox block serves. */
enum { TAG_PERM_A = 1, TAG_PERM_B = 2, TAG_SCAT = 3 };

static void draw(uint64_t seed, uint32_t index, uint32_t cell, uint64_t step, uint32_t inter, uint32_t purpose,
                 uint32_t out[4])
{
    uint32_t ctr[4] = {index, cell, (uint32_t)step, (inter << 8) | purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Uniform on (0,1) from the top 23 bits of a word: ((r >> 9) + 1/2) * 2^-23, exact in binary32 and binary64. */
static double u23(uint32_t r) { return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0); }

/* ------------------------------------------------------------------------------------------------------------
 * Binning: stable sort of particle indices by key = cell * S + species, plus segment offsets.
 * Done the plain way: count, exclusive prefix sum, then place particles in index order.
 * ---------------------------------------------------------------------------------------------------------- */
int orc_bin(const int32_t* cell, const int32_t* species, int64_t n, int32_t n_cells, int32_t n_species,
            int32_t* perm_out, int64_t* offsets_out)
{
    if (n < 0 || n_cells <= 0 || n_species <= 0) return -1;
    int64_t nk = (int64_t)n_cells * n_species;
    for (int64_t k = 0; k <= nk; ++k) offsets_out[k] = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (cell[i] < 0 || cell[i] >= n_cells || species[i] < 0 || species[i] >= n_species) return -1;
        offsets_out[(int64_t)cell[i] * n_species + species[i] + 1] += 1;
    }
    for (int64_t k = 0; k < nk; ++k) offsets_out[k + 1] += offsets_out[k];
    int64_t* cursor = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nk > 0 ? nk : 1));
    if (!cursor) return -2;
    for (int64_t k = 0; k < nk; ++k) cursor[k] = offsets_out[k];
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = (int64_t)cell[i] * n_species + species[i];
        perm_out[cursor[k]++] = (int32_t)i;
    }
    free(cursor);
    return 0;
}

/* ------------------------------------------------------------------------------------------------------------
 * Random permutation of a segment of n particles: sort local indices by a 64-bit key made of 44 Philox bits
 * with the local index in the low 20 bits (keys are therefore distinct). One Philox block serves two indices.
 * ---------------------------------------------------------------------------------------------------------- */
#define PERM_INDEX_BITS 20
#define PERM_MAX_N (1 << PERM_INDEX_BITS)

static uint64_t perm_key(uint64_t seed, uint64_t step, uint32_t cell, uint32_t inter, uint32_t side, uint32_t i)
{
    uint32_t r[4];
    draw(seed, i >> 1, cell, step, inter, side == 0 ? TAG_PERM_A : TAG_PERM_B, r);
    uint32_t hi = (i & 1) ? r[2] : r[0];
    uint32_t lo = (i & 1) ? r[3] : r[1];
    uint64_t k = ((uint64_t)hi << 32) | (uint64_t)lo;
    return (k & ~(uint64_t)(PERM_MAX_N - 1)) | (uint64_t)i;
}

static int cmp_u64(const void* a, const void* b)
{
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

int orc_permutation(int64_t n, uint64_t seed, uint64_t step, uint32_t cell, uint32_t inter, uint32_t side,
                    int32_t* perm_out)
{
    if (n < 0 || n > PERM_MAX_N) return -1;
    if (n == 0) return 0;
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    if (!keys) return -2;
    for (int64_t i = 0; i < n; ++i) keys[i] = perm_key(seed, step, cell, inter, side, (uint32_t)i);
    qsort(keys, (size_t)n, sizeof(uint64_t), cmp_u64);
    for (int64_t i = 0; i < n; ++i) perm_out[i] = (int32_t)(keys[i] & (PERM_MAX_N - 1));
    free(keys);
    return 0;
}

/* ------------------------------------------------------------------------------------------------------------
 * Order-N pairing of Takizuka and Abe [Sec. 3.2, Fig. TApairing].
 *  intra (n particles): n < 2 none. n even: (p0,p1),(p2,p3),... n odd: the first three particles are paired
 *    N x N as (p0,p1),(p1,p2),(p2,p0) with half the scattering length, then (p3,p4),(p5,p6),...
 *  inter: N_max pairs; pair k joins the k-th particle of the larger population with the (k mod N_min)-th of the
 *    smaller one, both populations in their own random order (cyclic reading of the stripped figure).
 * Output: local indices into segment a (li) and segment b (lj); flag bit 0 = triplet pair (s halved).
 * ---------------------------------------------------------------------------------------------------------- */
#define PAIR_TRIPLET 1u

/* Order N x N schedule (Sec. 3.1: every particle of alpha meets every particle of beta once per step). */
int64_t orc_nxn_slots(int64_t na, int64_t nb, int32_t intra, int64_t* per_round)
{
    if (intra) {
        if (na < 2) { *per_round = 0; return 0; }
        int64_t M = na + (na & 1);
        *per_round = M / 2;
        return (M - 1) * (M / 2);
    }
    if (na == 0 || nb == 0) { *per_round = 0; return 0; }
    int64_t lo = na < nb ? na : nb, hi = na < nb ? nb : na;
    *per_round = lo;
    return lo * hi;
}

int orc_nxn_slot(int64_t na, int64_t nb, int32_t intra, int64_t k, int64_t* ia, int64_t* jb)
{
    if (intra) {
        int64_t M = na + (na & 1), half = M / 2;
        int64_t r = k / half, t = k % half;
        int64_t a, b;
        if (t == 0) { a = r; b = M - 1; }
        else { a = (r + t) % (M - 1); b = (r - t + (M - 1)) % (M - 1); }
        if (a >= na || b >= na) return 0; /* the idle player of an odd count */
        *ia = a;
        *jb = b;
        return 1;
    }
    int64_t lo = na < nb ? na : nb, hi = na < nb ? nb : na;
    int64_t r = k / lo, m = k % lo;
    int64_t big = (m + r) % hi;
    if (na >= nb) { *ia = big; *jb = m; }
    else { *ia = m; *jb = big; }
    return 1;
}

static int64_t cell_pair_list(int64_t na, int64_t nb, int intra, uint64_t seed, uint64_t step, uint32_t cell,
                              uint32_t inter, int32_t* li, int32_t* lj, uint8_t* fl, int* err)
{
    *err = 0;
    if (intra) {
        int64_t n = na;
        if (n < 2) return 0;
        int32_t* pa = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        if (!pa || orc_permutation(n, seed, step, cell, inter, 0, pa)) { free(pa); *err = -1; return 0; }
        int64_t np = 0;
        int64_t start = 0;
        if (n % 2 == 1) {
            li[0] = pa[0]; lj[0] = pa[1]; fl[0] = PAIR_TRIPLET;
            li[1] = pa[1]; lj[1] = pa[2]; fl[1] = PAIR_TRIPLET;
            li[2] = pa[2]; lj[2] = pa[0]; fl[2] = PAIR_TRIPLET;
            np = 3;
            start = 3;
        }
        for (int64_t t = start; t + 1 < n; t += 2) {
            li[np] = pa[t]; lj[np] = pa[t + 1]; fl[np] = 0;
            ++np;
        }
        free(pa);
        return np;
    }
    if (na == 0 || nb == 0) return 0;
    int32_t* pa = (int32_t*)malloc(sizeof(int32_t) * (size_t)na);
    int32_t* pb = (int32_t*)malloc(sizeof(int32_t) * (size_t)nb);
    if (!pa || !pb || orc_permutation(na, seed, step, cell, inter, 0, pa) ||
        orc_permutation(nb, seed, step, cell, inter, 1, pb)) {
        free(pa); free(pb); *err = -1; return 0;
    }
    int64_t nmax = na > nb ? na : nb;
    for (int64_t k = 0; k < nmax; ++k) {
        if (na >= nb) { li[k] = pa[k]; lj[k] = pb[k % nb]; }
        else          { li[k] = pa[k % na]; lj[k] = pb[k]; }
        fl[k] = 0;
    }
    free(pa); free(pb);
    return nmax;
}

static int seg(const int64_t* offsets, int32_t S, int32_t c, int32_t s, int64_t* start, int64_t* n)
{
    int64_t k = (int64_t)c * S + s;
    *start = offsets[k];
    *n = offsets[k + 1] - offsets[k];
    return 0;
}

/* Pair lists for one interaction, every cell. Cell c's pairs are written from slot offsets[c*S] (the cell's first
 * particle); a cell never has more pairs than particles, so arrays of length N suffice. Indices are global
 * (binned) particle indices. */
int orc_pairs(const int64_t* offsets, int32_t n_cells, int32_t n_species, int32_t sa, int32_t sb, int32_t inter,
              uint64_t seed, uint64_t step, int32_t* pair_i, int32_t* pair_j, uint8_t* pair_flags)
{
    if (sa < 0 || sb < sa || sb >= n_species) return -1;
    for (int32_t c = 0; c < n_cells; ++c) {
        int64_t a0, na, b0, nb;
        seg(offsets, n_species, c, sa, &a0, &na);
        seg(offsets, n_species, c, sb, &b0, &nb);
        int64_t slot = offsets[(int64_t)c * n_species];
        int64_t cap = na + (sa == sb ? 0 : nb) + 3;
        int32_t* li = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
        int32_t* lj = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
        uint8_t* fl = (uint8_t*)malloc((size_t)cap);
        int err = 0;
        int64_t np = cell_pair_list(na, nb, sa == sb, seed, step, (uint32_t)c, (uint32_t)inter, li, lj, fl, &err);
        for (int64_t k = 0; k < np; ++k) {
            pair_i[slot + k] = (int32_t)(a0 + li[k]);
            pair_j[slot + k] = (int32_t)(b0 + lj[k]);
            pair_flags[slot + k] = fl[k];
        }
        free(li); free(lj); free(fl);
        if (err) return err;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------------------------
 * N97 angle parameter A(s): the root of L(A) = coth(A) - 1/A = exp(-s) (the mean of cos(chi) for the
 * distribution proportional to exp(A cos chi) equals exp(-s)). Solved in the equivalent form
 * G(A) = 1 - L(A) = -expm1(-s), which keeps full relative precision when s is small and A large. L is evaluated
 * from the Laurent series of coth (Bernoulli numbers) below A = 1/2; above it G = 1/A - 2/expm1(2A). The root is
 * found by bisection to the last bit.
 * ---------------------------------------------------------------------------------------------------------- */
double orc_n97_L(double A)
{
    if (A < 0.5) {
        /* coth x - 1/x = sum_{n>=1} 2^{2n} B_{2n} x^{2n-1} / (2n)! */
        static const double B[12] = {1.0 / 6.0,      -1.0 / 30.0,     1.0 / 42.0,     -1.0 / 30.0,
                                     5.0 / 66.0,     -691.0 / 2730.0, 7.0 / 6.0,      -3617.0 / 510.0,
                                     43867.0 / 798.0, -174611.0 / 330.0, 854513.0 / 138.0, -236364091.0 / 2730.0};
        double sum = 0.0, xp = A, fact = 1.0, pow4 = 1.0;
        for (int n = 1; n <= 12; ++n) {
            fact *= (double)(2 * n - 1) * (double)(2 * n);
            pow4 *= 4.0;
            sum += pow4 * B[n - 1] * xp / fact;
            xp *= A * A;
        }
        return sum;
    }
    return 1.0 / tanh(A) - 1.0 / A;
}

/* G(A) = 1 - L(A); coth(A) - 1 = 2 / expm1(2A) */
static double n97_G(double A)
{
    if (A < 0.5) return 1.0 - orc_n97_L(A);
    return 1.0 / A - 2.0 / expm1(2.0 * A);
}

double orc_n97_A(double s)
{
    double z = -expm1(-s); /* 1 - exp(-s) */
    if (!(z < 1.0)) return 0.0;       /* exp(-s) underflows: isotropic limit A -> 0 */
    if (!(z > 0.0)) return INFINITY;  /* s == 0: no scattering */
    /* G is decreasing from 1 to 0; G(A) < 1/A, so G(hi) < z for hi = 1/z + 1. */
    double lo = 0.0, hi = 1.0 / z + 1.0;
    for (int it = 0; it < 4000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (n97_G(mid) > z) lo = mid; else hi = mid;
    }
    /* the bracket has collapsed to adjacent doubles: return the one with the smaller residual */
    return fabs(n97_G(lo) - z) <= fabs(n97_G(hi) - z) ? lo : hi;
}

/* Centre-of-mass polar angle from the scattering length s (returns sin(Theta) and 1 - cos(Theta)).
 *  TA77: tan(Theta/2) = delta ~ N(0, s/2) (variance fixed by s = <Theta^2>/2 of Eq. sij_sji), drawn by
 *        Box-Muller from U1 (radius) and U4 (angle); sin = 2 delta/(1+delta^2), 1-cos = 2 delta^2/(1+delta^2).
 *  N97:  cos chi drawn from the density proportional to exp(A cos chi) by inverting its CDF with V = U1:
 *        1 - cos chi = -log1p(V expm1(-2A)) / A, and 1 + cos chi = log1p((1 - V) expm1(2A)) / A for sin chi. */
void orc_angle(int32_t method, double s, double U1, double U4, double* sin_theta, double* one_minus_cos)
{
    if (method == ORC_TA77) {
        double g = sqrt(-2.0 * log(U1)) * cos(2.0 * M_PI * U4);
        double d = sqrt(0.5 * s) * g;
        if (fabs(d) <= 1.0) {
            double den = 1.0 + d * d;
            *sin_theta = 2.0 * d / den;
            *one_minus_cos = 2.0 * d * d / den;
        } else {
            double t = 1.0 / d;
            double den = 1.0 + t * t;
            *sin_theta = 2.0 * t / den;
            *one_minus_cos = 2.0 / den;
        }
        return;
    }
    double A = orc_n97_A(s);
    double omc, opc;
    if (A == 0.0) { omc = 2.0 * U1; opc = 2.0 * (1.0 - U1); }
    else if (isinf(A)) { omc = 0.0; opc = 2.0; }
    else {
        /* 1 - cos chi = -ln(1 + x) / A with 1 + x = (1 - V) + V exp(-2A), x = -V (1 - exp(-2A)): log1p(x) while x is
         * small, the sum of the two positive terms once it is not (no cancellation either way) */
        double x = -U1 * -expm1(-2.0 * A);
        omc = x > -0.5 ? -log1p(x) / A : -log((1.0 - U1) + U1 * exp(-2.0 * A)) / A;
        /* 1 + cos chi = log1p((1 - V) expm1(2A)) / A from the same inversion, so sin chi stays accurate near
         * back-scatter where 2 - (1 - cos chi) would cancel */
        opc = omc <= 1.0 ? 2.0 - omc : log1p((1.0 - U1) * expm1(2.0 * A)) / A;
    }
    if (omc < 0.0) omc = 0.0;
    if (omc > 2.0) omc = 2.0;
    if (opc < 0.0) opc = 0.0;
    if (opc > 2.0) opc = 2.0;
    *one_minus_cos = omc;
    *sin_theta = sqrt(omc * opc);
}

/* Rotation of the relative velocity u through polar angle Theta and azimuth phi about its own direction
 * (Takizuka-Abe form). Returns du = u' - u. */
void orc_rotate(const double u[3], double sin_theta, double one_minus_cos, double phi, double du[3])
{
    double ux = u[0], uy = u[1], uz = u[2];
    double uperp = sqrt(ux * ux + uy * uy);
    double umag = sqrt(ux * ux + uy * uy + uz * uz);
    double cp = cos(phi), sp = sin(phi);
    if (uperp > 0.0) {
        du[0] = (ux / uperp) * uz * sin_theta * cp - (uy / uperp) * umag * sin_theta * sp - ux * one_minus_cos;
        du[1] = (uy / uperp) * uz * sin_theta * cp + (ux / uperp) * umag * sin_theta * sp - uy * one_minus_cos;
        du[2] = -uperp * sin_theta * cp - uz * one_minus_cos;
    } else {
        du[0] = umag * sin_theta * cp;
        du[1] = umag * sin_theta * sp;
        du[2] = -uz * one_minus_cos;
    }
}

/* gamma - 1 and gamma for proper velocity u: gamma - 1 = |u|^2/c^2 / (gamma + 1), free of cancellation. */
static double gam(double c, const double u[3])
{
    return sqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / (c * c));
}

/* Relativistic pair scatter (the paper gives only the non-relativistic kinematics; this is the standard reading:
 * boost both momenta to the pair's centre-of-momentum frame, rotate p* through (Theta, phi) with the same rotation
 * as above, boost back). Returns dp = p_i' - p_i (and p_j' - p_j = -dp), |p*| and the CM relative speed
 * v_rel* = |p*| (1/(m_a gamma_a*) + 1/(m_b gamma_b*)), which replace mu u and u in Eq. sab_TA77. */
static void rel_cm(double c, double ma, double mb, const double ui[3], const double uj[3], double V[3],
                   double* gC, double pstar[3], double* pmag, double* vrel)
{
    double c2 = c * c;
    double gi = gam(c, ui), gj = gam(c, uj);
    double M = ma * gi + mb * gj; /* E_tot / c^2 */
    double P[3];
    for (int d = 0; d < 3; ++d) { P[d] = ma * ui[d] + mb * uj[d]; V[d] = P[d] / M; }
    /* invariant mass from gamma_rel - 1 = (|u_i - u_j|^2/c^2 - (gamma_i - gamma_j)^2)/2 */
    double du2 = 0.0, ss = 0.0;
    for (int d = 0; d < 3; ++d) { double t = ui[d] - uj[d]; du2 += t * t; ss += (ui[d] - uj[d]) * (ui[d] + uj[d]); }
    double dg = ss / (c2 * (gi + gj));
    double grm1 = 0.5 * (du2 / c2 - dg * dg);
    if (grm1 < 0.0) grm1 = 0.0;
    double Minv = sqrt((ma + mb) * (ma + mb) + 2.0 * ma * mb * grm1);
    *gC = M / Minv;
    double coef_b = (*gC) * (*gC) / (c2 * ((*gC) + 1.0)); /* (gamma_C - 1)/|V|^2 */
    /* p* = q + (gamma_C - 1)(Vhat.q) Vhat with q = (E_j p_i - E_i p_j) / E_tot: the boost of p_i to the CM frame
     * written through the pair's difference, m_a m_b (gamma_j (u_i - u_j) - (gamma_i - gamma_j) u_j) / M, so that
     * co-moving pairs do not cancel */
    double q[3], Vq = 0.0;
    for (int d = 0; d < 3; ++d) {
        q[d] = ma * mb * (gj * (ui[d] - uj[d]) - dg * uj[d]) / M;
        Vq += V[d] * q[d];
    }
    for (int d = 0; d < 3; ++d) pstar[d] = q[d] + coef_b * Vq * V[d];
    double p2 = pstar[0] * pstar[0] + pstar[1] * pstar[1] + pstar[2] * pstar[2];
    *pmag = sqrt(p2);
    double gsa = sqrt(1.0 + p2 / (ma * ma * c2)), gsb = sqrt(1.0 + p2 / (mb * mb * c2));
    *vrel = (*pmag) * (1.0 / (ma * gsa) + 1.0 / (mb * gsb));
}

void orc_rel_scatter_dp(double c, double ma, double mb, const double ui[3], const double uj[3], double sin_theta,
                        double one_minus_cos, double phi, double dp[3], double* pstar_mag, double* vrel)
{
    double V[3], gC, pstar[3];
    rel_cm(c, ma, mb, ui, uj, V, &gC, pstar, pstar_mag, vrel);
    double dps[3];
    orc_rotate(pstar, sin_theta, one_minus_cos, phi, dps);
    /* boost back: the energy term is unchanged (|p*'| = |p*|), so only the linear part acts on dp* */
    double coef_b = gC * gC / (c * c * (gC + 1.0));
    double Vd = V[0] * dps[0] + V[1] * dps[1] + V[2] * dps[2];
    for (int d = 0; d < 3; ++d) dp[d] = dps[d] + coef_b * Vd * V[d];
}

/* ------------------------------------------------------------------------------------------------------------
 * Scatter of one interaction (sa, sb) in one cell [Algorithm 1, pair loop].
 * ---------------------------------------------------------------------------------------------------------- */
typedef struct {
    double* vx; double* vy; double* vz; const double* w;
    const int64_t* offsets; int32_t S;
} state_t;

/* Pre-scatter copy: component d of particle t is at p[(t - base) + d * stride]. */
typedef struct { double* p; int64_t base; int64_t stride; } backup_t;
#define BK(bk, t, d) ((bk).p[((t) - (bk).base) + (int64_t)(d) * (bk).stride])

/* w_max N_min of Eq. sab_TA77, or, with duplicity weighting (Sec. 3.2, the alternative of Higginson et al. that
 * the paper describes), (w_max / D_ij) N_max for inter-species pairs: D_ij is the number of times the particle of
 * the smaller population in pair k is paired during the interaction. Pair k takes that population's (k mod N_min)-th
 * particle, which is paired for every k' = k mod N_min in [0, N_max), i.e. D = floor((N_max - 1 - m) / N_min) + 1
 * with m = k mod N_min. Intra-species pairs keep w_max N_min. */
static double pair_weight_factor(const orc_params* p, int intra, int64_t na, int64_t nb, int64_t k, double wmax,
                                 double nmin)
{
    if (p->weighting != 1 || intra || p->pairing == 1) return wmax * nmin;
    int64_t nlo = na < nb ? na : nb, nhi = na < nb ? nb : na;
    int64_t m = k % nlo;
    double D = (double)((nhi - 1 - m) / nlo + 1);
    return wmax / D * (double)nhi;
}

static void scatter_cell(const state_t* st, int32_t c, const double* q, const double* m, const double* lnL,
                         int32_t sa, int32_t sb, int32_t inter, const orc_params* p, backup_t bk, int* err)
{
    int64_t a0, na, b0, nb;
    seg(st->offsets, st->S, c, sa, &a0, &na);
    seg(st->offsets, st->S, c, sb, &b0, &nb);
    int intra = (sa == sb);
    /* pre-scatter copy of every participant (for Eq. vp_pm, Eq. Econs and the fallback) */
    for (int side = 0; side < (intra ? 1 : 2); ++side) {
        int64_t s0 = side ? b0 : a0, ns = side ? nb : na;
        for (int64_t t = s0; t < s0 + ns; ++t) {
            BK(bk, t, 0) = st->vx[t]; BK(bk, t, 1) = st->vy[t]; BK(bk, t, 2) = st->vz[t];
        }
    }
    int64_t per = 0;
    int64_t nxn = p->pairing == 1 ? orc_nxn_slots(na, nb, intra, &per) : 0;
    int64_t cap = (p->pairing == 1 ? nxn : na + (intra ? 0 : nb)) + 3;
    int32_t* li = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t* lj = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    uint8_t* fl = (uint8_t*)malloc((size_t)cap);
    int64_t* lk = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    int64_t np = 0;
    if (p->pairing == 1) {
        /* Eq. sab_weighted: every pair once, slot k of the schedule over the interaction's random permutations,
         * the draw keyed by the slot */
        int32_t* pa = (int32_t*)malloc(sizeof(int32_t) * (size_t)(na > 0 ? na : 1));
        int32_t* pb = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nb > 0 ? nb : 1));
        if (na > 0) orc_permutation(na, p->seed, p->step, (uint32_t)c, (uint32_t)inter, 0, pa);
        if (!intra && nb > 0) orc_permutation(nb, p->seed, p->step, (uint32_t)c, (uint32_t)inter, 1, pb);
        for (int64_t k = 0; k < nxn; ++k) {
            int64_t a, b;
            if (!orc_nxn_slot(na, nb, intra, k, &a, &b)) continue;
            li[np] = pa[a];
            lj[np] = intra ? pa[b] : pb[b];
            fl[np] = 0;
            lk[np] = k;
            ++np;
        }
        free(pa);
        free(pb);
    } else {
        np = cell_pair_list(na, nb, intra, p->seed, p->step, (uint32_t)c, (uint32_t)inter, li, lj, fl, err);
        for (int64_t k = 0; k < np; ++k) lk[k] = k;
    }
    double nmin = p->pairing == 1 ? 1.0 : (intra ? (double)(na - 1) : (double)(na < nb ? na : nb));
    double ma = m[sa], mb = m[sb];
    double mu = ma * mb / (ma + mb);
    double kappa = q[sa] * q[sa] * q[sb] * q[sb] * lnL[sa * st->S + sb] * p->dt /
                   (4.0 * M_PI * p->eps0 * p->eps0 * p->dV);
    for (int64_t k = 0; k < np; ++k) {
        int64_t i = a0 + li[k], j = b0 + lj[k];
        double vi[3] = {st->vx[i], st->vy[i], st->vz[i]};
        double vj[3] = {st->vx[j], st->vy[j], st->vz[j]};
        double wi = st->w[i], wj = st->w[j];
        double wmax = wi > wj ? wi : wj, wmin = wi > wj ? wj : wi;
        uint32_t r[4];
        draw(p->seed, (uint32_t)lk[k], (uint32_t)c, p->step, (uint32_t)inter, TAG_SCAT, r);
        double U1 = u23(r[0]), U2 = u23(r[1]), U3 = u23(r[2]), U4 = u23(r[3]);
        double dvi[3], dvj[3];
        if (!p->relativistic) {
            double u[3] = {vi[0] - vj[0], vi[1] - vj[1], vi[2] - vj[2]};
            double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            if (u2 == 0.0) continue;
            double umag = sqrt(u2);
            double s = kappa / (mu * mu) * pair_weight_factor(p, intra, na, nb, k, wmax, nmin) / (u2 * umag);
            if (fl[k] & PAIR_TRIPLET) s *= 0.5;
            double st_, omc, du[3];
            orc_angle(p->method, s, U1, U4, &st_, &omc);
            orc_rotate(u, st_, omc, 2.0 * M_PI * U2, du);
            for (int d = 0; d < 3; ++d) { dvi[d] = (mu / ma) * du[d]; dvj[d] = -(mu / mb) * du[d]; }
        } else {
            double du2 = 0.0;
            for (int d = 0; d < 3; ++d) du2 += (vi[d] - vj[d]) * (vi[d] - vj[d]);
            if (du2 == 0.0) continue;
            double V[3], gC, pstar[3], pm, vrel;
            rel_cm(p->c, ma, mb, vi, vj, V, &gC, pstar, &pm, &vrel);
            if (!(pm > 0.0)) continue;
            double s = kappa * pair_weight_factor(p, intra, na, nb, k, wmax, nmin) / (pm * pm * vrel);
            if (fl[k] & PAIR_TRIPLET) s *= 0.5;
            double st_, omc, dp[3];
            orc_angle(p->method, s, U1, U4, &st_, &omc);
            orc_rel_scatter_dp(p->c, ma, mb, vi, vj, st_, omc, 2.0 * M_PI * U2, dp, &pm, &vrel);
            for (int d = 0; d < 3; ++d) { dvi[d] = dp[d] / ma; dvj[d] = -dp[d] / mb; }
        }
        /* lighter particle always updated; heavier with probability w_min/w_max; equal weights: both */
        int upd_i = 1, upd_j = 1;
        if (wi != wj) {
            int heavy_moves = (U3 * wmax < wmin);
            if (wi > wj) upd_i = heavy_moves; else upd_j = heavy_moves;
        }
        if (upd_i) { st->vx[i] += dvi[0]; st->vy[i] += dvi[1]; st->vz[i] += dvi[2]; }
        if (upd_j) { st->vx[j] += dvj[0]; st->vy[j] += dvj[1]; st->vz[j] += dvj[2]; }
    }
    free(li); free(lj); free(fl); free(lk);
}

static int64_t total_n(const int64_t* offsets, int32_t n_cells, int32_t n_species)
{
    return offsets[(int64_t)n_cells * n_species];
}

int orc_scatter(double* vx, double* vy, double* vz, const double* w, const int64_t* offsets, int32_t n_cells,
                int32_t n_species, const double* q, const double* m, const double* lnL, int32_t sa, int32_t sb,
                int32_t inter, const orc_params* p, double* backup)
{
    if (sa < 0 || sb < sa || sb >= n_species) return -1;
    state_t st = {vx, vy, vz, w, offsets, n_species};
    int64_t N = total_n(offsets, n_cells, n_species);
    for (int32_t c = 0; c < n_cells; ++c) {
        int err = 0;
        backup_t bk = {backup, 0, N};
        scatter_cell(&st, c, q, m, lnL, sa, sb, inter, p, bk, &err);
        if (err) return err;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------------------------
 * Energy-correction pair [Eqs. vp1_inelastic, vp2_inelastic, vrel_inelastic; Appendix A for relativistic].
 * Weighted masses m1 = m_s w1, m2 = m_s w2. The pair's centre-of-mass kinetic energy loses U.
 * ---------------------------------------------------------------------------------------------------------- */
double orc_pair_kecm(int32_t relativistic, double c, double m1, double m2, const double v1[3], const double v2[3])
{
    if (!relativistic) {
        double vr2 = 0.0;
        for (int d = 0; d < 3; ++d) vr2 += (v1[d] - v2[d]) * (v1[d] - v2[d]);
        return 0.5 * (m1 * m2 / (m1 + m2)) * vr2;
    }
    /* KE_cm = E_cm - (m1+m2)c^2 with E_cm^2 = (m1+m2)^2 c^4 + 2 m1 m2 c^4 (gamma_rel - 1) */
    double c2 = c * c;
    double g1 = gam(c, v1), g2 = gam(c, v2);
    double du2 = 0.0, ss = 0.0;
    for (int d = 0; d < 3; ++d) { du2 += (v1[d] - v2[d]) * (v1[d] - v2[d]); ss += (v1[d] - v2[d]) * (v1[d] + v2[d]); }
    double dg = ss / (c2 * (g1 + g2));
    double grm1 = 0.5 * (du2 / c2 - dg * dg);
    if (grm1 < 0.0) grm1 = 0.0;
    double Minv = sqrt((m1 + m2) * (m1 + m2) + 2.0 * m1 * m2 * grm1);
    return 2.0 * m1 * m2 * c2 * grm1 / (Minv + m1 + m2);
}

void orc_energy_pair(int32_t relativistic, double c, double m1, double m2, double v1[3], double v2[3], double U)
{
    if (!relativistic) {
        double vr[3], vr2 = 0.0;
        for (int d = 0; d < 3; ++d) { vr[d] = v1[d] - v2[d]; vr2 += vr[d] * vr[d]; }
        double K = 0.5 * (m1 * m2 / (m1 + m2)) * vr2;
        /* v'_R = g v_R, g = sqrt(1 - U/K); g - 1 written as -(U/K)/(1 + g) to avoid cancellation */
        double x = U / K;
        double g = sqrt(1.0 - x);
        double gm1 = -x / (1.0 + g);
        for (int d = 0; d < 3; ++d) {
            v1[d] += (m2 / (m1 + m2)) * gm1 * vr[d];
            v2[d] -= (m1 / (m1 + m2)) * gm1 * vr[d];
        }
        return;
    }
    /* Appendix A: p1' = p1 + alpha du, p2' = p2 - alpha du, sum of sqrt(m_k^2 + |p_k'|^2/c^2) = A = (E_tot - U)/c^2.
     * Quadratic a alpha^2 + b alpha + c0 = 0 of Eq. alpha_Eq1, with its coefficients rewritten free of
     * cancellation (in mass units E~ = E/c^2, U~ = U/c^2):
     *   c0 = U~ (2E~1 - U~)(2E~2 - U~)(2E~1 + 2E~2 - U~)           (= 4 A^2 E~2^2 - D^2)
     *   b  = (4/c^2) du . [2A (E~2 p1 - E~1 p2 + U~ p2) - U~ (2E~1 - U~) p_tot]   (= (4/c^2) du.[D p_tot - 2A^2 p2])
     *   a  = 4 [A^2 |du|^2 / c^2 - (p_tot . du)^2 / c^4]
     * with E~2 p1 - E~1 p2 = m1 m2 (gamma2 du - (gamma1 - gamma2) u2). The root taken is the one of smaller
     * magnitude, which tends to zero with U and to mu_R (sqrt(1 - U/K) - 1) as c -> infinity. */
    double c2 = c * c;
    double g1 = gam(c, v1), g2 = gam(c, v2);
    double E1 = m1 * g1, E2 = m2 * g2, Ut = U / c2;
    double A = E1 + E2 - Ut;
    double du[3], pt[3], u2sq = 0.0, du2 = 0.0, ss = 0.0;
    for (int d = 0; d < 3; ++d) {
        du[d] = v1[d] - v2[d];
        pt[d] = m1 * v1[d] + m2 * v2[d];
        du2 += du[d] * du[d];
        ss += du[d] * (v1[d] + v2[d]);
        u2sq += v2[d] * v2[d];
    }
    (void)u2sq;
    double dg = ss / (c2 * (g1 + g2)); /* gamma1 - gamma2 */
    double bvec_dot = 0.0, ptdu = 0.0;
    for (int d = 0; d < 3; ++d) {
        double x12 = m1 * m2 * (g2 * du[d] - dg * v2[d]); /* E~2 p1 - E~1 p2 */
        double p2d = m2 * v2[d];
        double bv = 2.0 * A * (x12 + Ut * p2d) - Ut * (2.0 * E1 - Ut) * pt[d];
        bvec_dot += du[d] * bv;
        ptdu += pt[d] * du[d];
    }
    double a = 4.0 * (A * A * du2 / c2 - ptdu * ptdu / (c2 * c2));
    double b = 4.0 / c2 * bvec_dot;
    double c0 = Ut * (2.0 * E1 - Ut) * (2.0 * E2 - Ut) * (2.0 * E1 + 2.0 * E2 - Ut);
    double disc = b * b - 4.0 * a * c0;
    if (disc < 0.0) disc = 0.0;
    double qq = -0.5 * (b + (b >= 0.0 ? sqrt(disc) : -sqrt(disc)));
    double r1 = (a != 0.0) ? qq / a : INFINITY;
    double r2 = (qq != 0.0) ? c0 / qq : 0.0;
    double alpha = fabs(r1) < fabs(r2) ? r1 : r2;
    for (int d = 0; d < 3; ++d) {
        v1[d] += alpha * du[d] / m1;
        v2[d] -= alpha * du[d] / m2;
    }
}

/* ------------------------------------------------------------------------------------------------------------
 * Moment correction of one interaction in one cell [Algorithm 1 after the pair loop; Sec. 4; Appendix A].
 * ---------------------------------------------------------------------------------------------------------- */
/* Sort key of the optional weight-descending order: the weight's IEEE bits (weights are positive, so the bits
 * order like the values) inverted for descending order, truncated to sign, exponent and 32 mantissa bits, with the
 * particle's rank in the random permutation in the low 20 bits. Weights that agree to 2^-32 relative therefore tie
 * and keep the random order. */
static uint64_t weight_key(double w, uint32_t rank)
{
    uint64_t b;
    memcpy(&b, &w, sizeof b);
    return (~b & ~(uint64_t)(PERM_MAX_N - 1)) | (uint64_t)rank;
}

/* Cell sort with each segment stored in the order of the optional weight sort of Algorithm 1: orc_bin, then
 * within every (cell, species) segment the stable order by the weight key above (descending weight; weights that
 * agree to 2^-32 relative keep increasing particle index). In this layout the weight order of a segment whose keys
 * are all distinct is the identity. */
int orc_bin_weighted(const int32_t* cell, const int32_t* species, const double* w, int64_t n, int32_t n_cells,
                     int32_t n_species, int32_t* perm_out, int64_t* offsets_out)
{
    int rc = orc_bin(cell, species, n, n_cells, n_species, perm_out, offsets_out);
    if (rc != 0) return rc;
    int64_t nk = (int64_t)n_cells * n_species;
    for (int64_t k = 0; k < nk; ++k) {
        int64_t b = offsets_out[k], len = offsets_out[k + 1] - b;
        if (len < 2) continue;
        if (len > PERM_MAX_N) return -1;
        uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)len);
        int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)len);
        if (!keys || !idx) {
            free(keys);
            free(idx);
            return -2;
        }
        for (int64_t r = 0; r < len; ++r) {
            idx[r] = perm_out[b + r];
            keys[r] = weight_key(w[idx[r]], (uint32_t)r);
        }
        qsort(keys, (size_t)len, sizeof(uint64_t), cmp_u64);
        for (int64_t r = 0; r < len; ++r) perm_out[b + r] = idx[keys[r] & (PERM_MAX_N - 1)];
        free(keys);
        free(idx);
    }
    return 0;
}

/* Kinetic energy of one particle of mass mp (weighted) with state v (velocity or proper velocity). */
static double ke(int rel, double c, double mp, const double v[3])
{
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    if (!rel) return 0.5 * mp * v2;
    double g = sqrt(1.0 + v2 / (c * c));
    return mp * v2 / (g + 1.0); /* m c^2 (gamma - 1) */
}

/* Kinetic-energy difference ke(a) - ke(b) written per particle: for non-relativistic 1/2 m (a-b).(a+b); for
 * relativistic m c^2 (gamma_a - gamma_b) = m (a-b).(a+b) / (gamma_a + gamma_b). */
static double dke(int rel, double c, double mp, const double a[3], const double b[3])
{
    double dd = 0.0;
    for (int d = 0; d < 3; ++d) dd += (a[d] - b[d]) * (a[d] + b[d]);
    if (!rel) return 0.5 * mp * dd;
    double ga = gam(c, a), gb = gam(c, b);
    return mp * dd / (ga + gb);
}

/* Energy-correction loop of one species [Algorithm 1, final loop]: pairs adjacent particles of the order rho,
 * pass p starting at offset p mod 2, U = sign(D) min(|D|, fE KE_cm), D -= U until D == 0. Returns the number of
 * pairs that absorbed energy; *D_io is the remaining violation. */
static int32_t energy_loop(const state_t* st, int rel, double c, double fE, int max_passes, double ms,
                           const int64_t* rho_global, int64_t n, double* D_io)
{
    double D = *D_io;
    int32_t used = 0;
    for (int pass = 0; pass < max_passes && D != 0.0; ++pass) {
        for (int64_t t = pass % 2; t + 1 < n && D != 0.0; t += 2) {
            int64_t i = rho_global[t], j = rho_global[t + 1];
            double v1[3] = {st->vx[i], st->vy[i], st->vz[i]};
            double v2[3] = {st->vx[j], st->vy[j], st->vz[j]};
            double m1 = ms * st->w[i], m2 = ms * st->w[j];
            double K = orc_pair_kecm(rel, c, m1, m2, v1, v2);
            if (!(K > 0.0)) continue;
            double capE = fE * K;
            double U = (D > 0.0 ? 1.0 : -1.0) * (fabs(D) < capE ? fabs(D) : capE);
            orc_energy_pair(rel, c, m1, m2, v1, v2, U);
            st->vx[i] = v1[0]; st->vy[i] = v1[1]; st->vz[i] = v1[2];
            st->vx[j] = v2[0]; st->vy[j] = v2[1]; st->vz[j] = v2[2];
            D -= U;
            ++used;
        }
    }
    *D_io = D;
    return used;
}

static void correct_cell(const state_t* st, int32_t c, const double* m, int32_t sa, int32_t sb, int32_t inter,
                         const orc_params* p, backup_t bk, int32_t* corr_pairs, int32_t* failed)
{
    int64_t a0, na, b0, nb;
    seg(st->offsets, st->S, c, sa, &a0, &na);
    seg(st->offsets, st->S, c, sb, &b0, &nb);
    int intra = (sa == sb);
    *corr_pairs = 0;
    *failed = 0;
    /* nothing was scattered in this cell for this interaction */
    if (intra ? (na < 2) : (na == 0 || nb == 0)) return;
    int rel = p->relativistic;
    int nside = intra ? 1 : 2;
    int64_t s0[2] = {a0, b0}, ns[2] = {na, nb};
    double msp[2] = {m[sa], m[sb]};

    /* Eq. vp_pm: B = sum_p m_p (v_ps - v_bs) / sum_p m_p w_p, m_p = m_s w_p; v_pm = v_ps - B w_p */
    double S[3] = {0.0, 0.0, 0.0}, Sw = 0.0;
    for (int side = 0; side < nside; ++side)
        for (int64_t t = s0[side]; t < s0[side] + ns[side]; ++t) {
            double mp = msp[side] * st->w[t];
            S[0] += mp * (st->vx[t] - BK(bk, t, 0));
            S[1] += mp * (st->vy[t] - BK(bk, t, 1));
            S[2] += mp * (st->vz[t] - BK(bk, t, 2));
            Sw += mp * st->w[t];
        }
    double B[3] = {S[0] / Sw, S[1] / Sw, S[2] / Sw};
    for (int side = 0; side < nside; ++side)
        for (int64_t t = s0[side]; t < s0[side] + ns[side]; ++t) {
            st->vx[t] -= B[0] * st->w[t];
            st->vy[t] -= B[1] * st->w[t];
            st->vz[t] -= B[2] * st->w[t];
        }

    /* Eq. Econs, summed as per-particle kinetic-energy differences from the pre-scatter state */
    double dE = 0.0, Es[2] = {0.0, 0.0}, wsum[2] = {0.0, 0.0};
    for (int side = 0; side < nside; ++side)
        for (int64_t t = s0[side]; t < s0[side] + ns[side]; ++t) {
            double mp = msp[side] * st->w[t];
            double a[3] = {st->vx[t], st->vy[t], st->vz[t]};
            double b[3] = {BK(bk, t, 0), BK(bk, t, 1), BK(bk, t, 2)};
            dE += dke(rel, p->c, mp, a, b);
            Es[side] += ke(rel, p->c, mp, a);
            wsum[side] += st->w[t];
        }

    /* Eq. DeltaEs: partition by mean weight times post-shift energy; a species with fewer than two particles cannot
     * form a pair, so its share goes to the other one. */
    double D[2] = {dE, 0.0};
    int can[2] = {ns[0] >= 2, intra ? 0 : ns[1] >= 2};
    int fail = 0;
    if (!intra) {
        if (can[0] && can[1]) {
            double wa = wsum[0] / (double)na * Es[0], wb = wsum[1] / (double)nb * Es[1];
            double den = wa + wb;
            if (den > 0.0) { D[0] = wa / den * dE; D[1] = dE - D[0]; }
            else if (dE != 0.0) fail = 1;
        } else if (can[0]) { D[0] = dE; D[1] = 0.0; }
        else if (can[1]) { D[0] = 0.0; D[1] = dE; }
        else if (dE != 0.0) fail = 1;
    }

    /* "Delta E_s = 0" (Algorithm 1, loop exit) is read as: no larger than 64 ulps of species s's post-shift kinetic
     * energy. Below that the violation is rounding noise of the sums (it is what equal weights leave). */
    for (int side = 0; side < 2; ++side)
        if (fabs(D[side]) <= 0x1p-47 * Es[side]) D[side] = 0.0;

    /* energy-correction loops, species a then b */
    for (int side = 0; side < nside && !fail; ++side) {
        if (D[side] == 0.0) continue;
        int64_t n = ns[side];
        int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        int64_t* rho = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        orc_permutation(n, p->seed, p->step, (uint32_t)c, (uint32_t)inter, (uint32_t)side, perm);
        if (p->sort_by_weight) {
            /* optional step of Algorithm 1: descending weight; ties keep the random order */
            uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
            for (int64_t r = 0; r < n; ++r) keys[r] = weight_key(st->w[s0[side] + perm[r]], (uint32_t)r);
            qsort(keys, (size_t)n, sizeof(uint64_t), cmp_u64);
            for (int64_t r = 0; r < n; ++r) rho[r] = s0[side] + perm[keys[r] & (PERM_MAX_N - 1)];
            free(keys);
        } else {
            for (int64_t r = 0; r < n; ++r) rho[r] = s0[side] + perm[r];
        }
        double Dside = D[side];
        *corr_pairs += energy_loop(st, rel, p->c, p->fE, p->max_corr_passes, msp[side], rho, n, &Dside);
        if (Dside != 0.0) fail = 1;
        free(perm);
        free(rho);
    }

    if (fail) {
        *failed = 1;
        if (p->fail_policy == ORC_FAIL_ROLLBACK) {
            /* Sec. 5.2 fallback: reset this interaction's particles to their pre-scatter velocities */
            for (int side = 0; side < nside; ++side)
                for (int64_t t = s0[side]; t < s0[side] + ns[side]; ++t) {
                    st->vx[t] = BK(bk, t, 0); st->vy[t] = BK(bk, t, 1); st->vz[t] = BK(bk, t, 2);
                }
        }
    }
}

int orc_correct(double* vx, double* vy, double* vz, const double* w, const int64_t* offsets, int32_t n_cells,
                int32_t n_species, const double* m, int32_t sa, int32_t sb, int32_t inter, const orc_params* p,
                const double* backup, int32_t* corr_pairs, int32_t* fail_flags)
{
    if (sa < 0 || sb < sa || sb >= n_species) return -1;
    state_t st = {vx, vy, vz, w, offsets, n_species};
    int64_t N = total_n(offsets, n_cells, n_species);
    for (int32_t c = 0; c < n_cells; ++c) {
        int32_t cp = 0, f = 0;
        backup_t bk = {(double*)backup, 0, N};
        correct_cell(&st, c, m, sa, sb, inter, p, bk, &cp, &f);
        if (corr_pairs) corr_pairs[c] = cp;
        if (fail_flags) fail_flags[c] = f;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------------------------
 * Full step(s) on cells [cell_begin, cell_end): for each step, for each interaction in list order, scatter then
 * (if enabled) correct. corr_pairs and fail_count (per cell) are accumulated.
 * ---------------------------------------------------------------------------------------------------------- */
int orc_step(double* vx, double* vy, double* vz, const double* w, const int64_t* offsets, int32_t n_cells,
             int32_t n_species, const double* q, const double* m, const double* lnL, const int32_t* interactions,
             int32_t n_inter, const orc_params* p, int32_t n_steps, int32_t cell_begin, int32_t cell_end,
             int32_t* corr_pairs, int32_t* fail_count)
{
    if (cell_begin < 0 || cell_end > n_cells || cell_begin > cell_end) return -1;
    for (int32_t k = 0; k < n_inter; ++k) {
        int32_t a = interactions[2 * k], b = interactions[2 * k + 1];
        if (a < 0 || b < a || b >= n_species) return -1;
    }
    state_t st = {vx, vy, vz, w, offsets, n_species};
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int32_t c = cell_begin; c < cell_end; ++c) {
        /* cell-local pre-scatter copy covering the cell's own particle range */
        int64_t base = offsets[(int64_t)c * n_species], nc = offsets[(int64_t)(c + 1) * n_species] - base;
        double* backup = (double*)malloc(sizeof(double) * 3 * (size_t)(nc > 0 ? nc : 1));
        if (!backup) {
#pragma omp atomic write
            rc = -2;
            continue;
        }
        backup_t bk = {backup, base, nc};
        orc_params ps = *p;
        for (int32_t t = 0; t < n_steps; ++t) {
            ps.step = p->step + (uint64_t)t;
            for (int32_t k = 0; k < n_inter; ++k) {
                int32_t a = interactions[2 * k], b = interactions[2 * k + 1];
                int err = 0;
                scatter_cell(&st, c, q, m, lnL, a, b, k, &ps, bk, &err);
                if (err) {
#pragma omp atomic write
                    rc = err;
                }
                if (ps.correct) {
                    int32_t cp = 0, f = 0;
                    correct_cell(&st, c, m, a, b, k, &ps, bk, &cp, &f);
                    if (corr_pairs) corr_pairs[c] += cp;
                    if (fail_count) fail_count[c] += f;
                }
            }
        }
        free(backup);
    }
    return rc;
}

/* Host threads of the cell loop of orc_step (timing only; the results do not depend on it). */
void orc_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------------------------------------- PIC coupling */

/* Free-streaming push (Sec. 2, Eq. Boltzmann, left-hand side with a = 0): per axis x <- x + v dt, with
 * v = u / gamma, gamma = sqrt(1 + |u|^2 / c^2) in relativistic mode; then the periodic image in [0, L) and the
 * cell index floor(x nx / L). Written once per precision so that each operation rounds in that precision. */
#define ORC_DEFINE_PUSH(T, SUF, SQRT, FLOOR)                                                                        \
    static T orc_wrap_##SUF(T x, T L)                                                                            \
    {                                                                                                            \
        if (x >= (T)0 && x < L) return x;                                                                        \
        T q = FLOOR(x / L);                                                                                      \
        T r = x - q * L;                                                                                         \
        if (r < (T)0) r = r + L;                                                                                 \
        if (r >= L) r = r - L;                                                                                   \
        if (!(r >= (T)0 && r < L)) r = (T)0; /* a non-finite position */                                         \
        return r;                                                                                                \
    }                                                                                                            \
    static void orc_push_##SUF(T* x, T* y, T* z, const T* vx, const T* vy, const T* vz, int64_t n,              \
                               const int32_t nc[3], const double l[3], double dt, int32_t rel, double c,         \
                               int32_t* cell)                                                                    \
    {                                                                                                            \
        const T tdt = (T)dt, c2 = (T)(c * c);                                                                    \
        T L[3], sx[3];                                                                                           \
        for (int d = 0; d < 3; ++d) {                                                                            \
            L[d] = (T)l[d];                                                                                      \
            sx[d] = (T)((double)nc[d] / l[d]);                                                                   \
        }                                                                                                        \
        T* pos[3] = {x, y, z};                                                                                   \
        for (int64_t i = 0; i < n; ++i) {                                                                        \
            const T u[3] = {vx[i], vy[i], vz[i]};                                                                \
            T ginv = (T)1;                                                                                       \
            if (rel) {                                                                                           \
                T s = u[0] * u[0];                                                                               \
                s = s + u[1] * u[1];                                                                             \
                s = s + u[2] * u[2];                                                                             \
                ginv = (T)1 / SQRT((T)1 + s / c2);                                                               \
            }                                                                                                    \
            int32_t id[3];                                                                                       \
            for (int d = 0; d < 3; ++d) {                                                                        \
                const T v = rel ? u[d] * ginv : u[d];                                                            \
                const T step = v * tdt;                                                                          \
                const T p = orc_wrap_##SUF(pos[d][i] + step, L[d]);                                              \
                pos[d][i] = p;                                                                                   \
                const T t = p * sx[d];                                                                           \
                int32_t k = (int32_t)FLOOR(t);                                                                   \
                id[d] = k < nc[d] ? k : nc[d] - 1;                                                               \
            }                                                                                                    \
            cell[i] = id[0] + nc[0] * (id[1] + nc[1] * id[2]);                                                   \
        }                                                                                                        \
    }

ORC_DEFINE_PUSH(double, f64, sqrt, floor)
ORC_DEFINE_PUSH(float, f32, sqrtf, floorf)

int orc_push(int32_t prec, void* x, void* y, void* z, const void* vx, const void* vy, const void* vz, int64_t n,
             const int32_t nc[3], const double l[3], double dt, int32_t relativistic, double c, int32_t* cell)
{
    if (n < 0 || (prec != 0 && prec != 1)) return -1;
    for (int d = 0; d < 3; ++d)
        if (nc[d] < 1 || !(l[d] > 0.0)) return -1;
    if (prec == 0)
        orc_push_f64((double*)x, (double*)y, (double*)z, (const double*)vx, (const double*)vy, (const double*)vz, n,
                     nc, l, dt, relativistic, c, cell);
    else
        orc_push_f32((float*)x, (float*)y, (float*)z, (const float*)vx, (const float*)vy, (const float*)vz, n, nc, l,
                     dt, relativistic, c, cell);
    return 0;
}
