// Cell kernel of the weighted, moment-preserving Monte-Carlo Coulomb collision step.
//
// One CTA owns one cell at a time (persistent CTAs pull cells from an atomic work queue). The cell's particles are
// staged in shared memory as a tile: velocities, their pre-interaction copy, weights, sort keys and the random
// permutation. For every interaction (a, b) of the step it then runs Algorithm 1 of the paper:
//   random permutation(s) (Philox keys, counting sort on the top key bits, insertion sort within a bucket)
//     -> Takizuka-Abe pairs (Sec. 3.2, Fig. TApairing)
//   pair loop: weighted scattering length (Eq. sab_TA77), TA77 / N97 angle, rotation, rejection of the heavier
//              particle with probability 1 - w_min/w_max (Sec. 3.2); inter-species pairs in rounds of N_min
//              disjoint pairs, rounds in order
//   momentum shift (Eq. vp_pm), energy violation (Eq. Econs), split (Eq. DeltaEs), optional weight sort,
//   energy-correction pairs (Eqs. vp1_inelastic, vp2_inelastic, vrel_inelastic, U_inelastic; Appendix A) as a
//   block-wide prefix sum over the pair caps fE * KE_cm, failure fallback (Sec. 5.2).
// The unfused C-ABI calls run single phases of the same code: PAIR writes the pair list, SCATTER the pair loop
// (reading the list, writing the pre-scatter copy), CORRECT the moment correction (reading that copy).
//
// FP64 path: everything in double. Mixed path: float velocities and kinematics, float-float accumulation of the
// per-cell sums, FP64 only for the per-cell coefficients (B, Delta E, its split) computed by one thread.
#include "mcc_kernels.h"

#ifndef MCC_MIN_BLOCKS
#define MCC_MIN_BLOCKS 6
#endif

namespace mcc {
namespace {

template <class V>
struct WStore;
template <>
struct WStore<double> {
    using T = double;
};
template <>
struct WStore<float> {
    using T = float2;  // (hi, lo) split of the double weight
};

template <class V>
struct Tile {
    uint64_t* keys;  // sort keys of segments too large for one warp's registers
    typename WStore<V>::T* w;
    V* v;            // [3][vs]
    V* vb;           // [3][bs] pre-interaction copy
    int32_t* perm;   // random permutation of each species segment (cell-local indices)
    int32_t* rho;    // weight-descending order of each species segment (cell-local indices)
    uint32_t* cnt;   // bucket counters of the permutation sort (cnt_cap entries)
    int cap;         // particles the arrays hold
    int vs, bs;      // plane strides of v and vb
    int cnt_cap;
};

template <class V>
__device__ __forceinline__ Tile<V> make_tile(unsigned char* base, int cap)
{
    Tile<V> t;
    t.cap = cap;
    t.vs = t.bs = cap;
    t.keys = reinterpret_cast<uint64_t*>(base);
    t.w = reinterpret_cast<typename WStore<V>::T*>(base + 8 * (size_t)cap);
    t.v = reinterpret_cast<V*>(base + 16 * (size_t)cap);
    t.vb = t.v + 3 * (size_t)cap;
    t.perm = reinterpret_cast<int32_t*>(base + (16 + 6 * sizeof(V)) * (size_t)cap);
    t.rho = t.perm + cap;
    t.cnt = reinterpret_cast<uint32_t*>(t.vb);  // vb is free while the permutations are built
    t.cnt_cap = (int)(3 * sizeof(V) / 4) * cap;
    return t;
}

// Tile of the pairing mode: keys | permutation | bucket counters (2 per particle: both sides' next powers of two of
// their counts add up to less than twice the cell's count); no velocities, weights or weight order. A tile of these
// holds cells about three times larger than the step's tile.
constexpr size_t kPairTileBytesPerParticle = 8 + 4 + 2 * 4;

template <class V>
__device__ __forceinline__ Tile<V> make_pair_tile(unsigned char* base, int cap)
{
    Tile<V> t;
    t.cap = cap;
    t.vs = t.bs = cap;
    t.keys = reinterpret_cast<uint64_t*>(base);
    t.w = nullptr;
    t.v = nullptr;
    t.vb = nullptr;
    t.perm = reinterpret_cast<int32_t*>(base + 8 * (size_t)cap);
    t.rho = t.perm;
    t.cnt = reinterpret_cast<uint32_t*>(base + 12 * (size_t)cap);
    t.cnt_cap = 2 * cap;
    return t;
}

// A cell above the on-chip tile runs from its CTA's global slab; the shared-memory tile (smem bytes) is then idle,
// so the arrays that fit move there, in order of how much they gain: the bucket counters (shared-memory atomics),
// velocities and weights (random access by pair), sort keys, permutation, weight order, pre-interaction copy.
// ms = the cell's largest species count (the counters of two sides need at most 2 next_pow2(ms) entries).
template <class V>
__device__ __forceinline__ void place_on_chip(Tile<V>& t, unsigned char* smem, size_t bytes, int n, int ms)
{
    size_t used = 0;
    auto take = [&](size_t b) -> unsigned char* {
        b = (b + 15) & ~(size_t)15;
        if (used + b > bytes) return nullptr;
        unsigned char* p = smem + used;
        used += b;
        return p;
    };
    int bm = 1;
    while (bm < ms) bm <<= 1;
    const int ns = (n + 3) & ~3;
    if (unsigned char* p = take(8 * (size_t)bm)) {
        t.cnt = reinterpret_cast<uint32_t*>(p);
        t.cnt_cap = 2 * bm;
    }
    if (unsigned char* p = take(3 * sizeof(V) * (size_t)ns)) {
        t.v = reinterpret_cast<V*>(p);
        t.vs = ns;
    }
    if (unsigned char* p = take(8 * (size_t)ns)) t.w = reinterpret_cast<typename WStore<V>::T*>(p);
    if (unsigned char* p = take(8 * (size_t)ns)) t.keys = reinterpret_cast<uint64_t*>(p);
    if (unsigned char* p = take(4 * (size_t)ns)) t.perm = reinterpret_cast<int32_t*>(p);
    if (unsigned char* p = take(4 * (size_t)ns)) t.rho = reinterpret_cast<int32_t*>(p);
    if (unsigned char* p = take(3 * sizeof(V) * (size_t)ns)) {
        t.vb = reinterpret_cast<V*>(p);
        t.bs = ns;
    }
}

__device__ __forceinline__ double wv(const Tile<double>& t, int i) { return t.w[i]; }
__device__ __forceinline__ float wv(const Tile<float>& t, int i) { return t.w[i].x; }
__device__ __forceinline__ bool w_equal(const Tile<double>& t, int i, int j) { return t.w[i] == t.w[j]; }
__device__ __forceinline__ bool w_equal(const Tile<float>& t, int i, int j)
{
    return t.w[i].x == t.w[j].x && t.w[i].y == t.w[j].y;
}
__device__ __forceinline__ double w_exact(const Tile<double>& t, const StepArgs&, int64_t, int i) { return t.w[i]; }
__device__ __forceinline__ double w_exact(const Tile<float>&, const StepArgs& A, int64_t cs, int i)
{
    return A.w[cs + i];
}
__device__ __forceinline__ void w_store(Tile<double>& t, int i, double w) { t.w[i] = w; }
__device__ __forceinline__ void w_store(Tile<float>& t, int i, double w) { t.w[i] = split_weight(w); }

template <class V>
__device__ __forceinline__ V pick(double d, float f);
template <>
__device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float pick<float>(double, float f) { return f; }

__device__ __forceinline__ void n97_tab(const StepArgs& A, N97Tab<double>& t) { t = {A.n97_f, A.n97_dh}; }
__device__ __forceinline__ void n97_tab(const StepArgs& A, N97Tab<float>& t) { t = {A.n97_f32, A.n97_dh32}; }

struct Shared {
    int off[kMaxSpecies + 1];
    int wmode[kMaxSpecies];  // weight order: 0 distinct (rho fixed for the visit), 1 all equal (rho = perm), 2 ties
                             // (sorted per interaction), 3 stored in strictly descending order (rho = identity)
    int cell;
    uint32_t step;  // the step index of the random counters (from device memory when the caller keeps it there)
    int fail;
    int fast;  // energy pairs of a side finished by the first warp
    alignas(16) unsigned char red_raw[8 * kThreads * 8];  // block_sum partials (8 quantities x 8 bytes)
    alignas(8) unsigned char red[8 * 8];                  // block_sum results (Acc<V>, 8 bytes each)
    double scan_d[kWarps + 1];
    float scan_f[kWarps + 1];
    int iscan[kWarps + 1];
    int iscr[kWarps];
    double B[3];
    float Bf[3];
    double D[2];
    float Df[2];
    alignas(8) unsigned char W1[8 * kMaxSpecies];  // per species sum of w over the cell (Acc<V>, fixed for the visit)
    alignas(8) unsigned char W2[8 * kMaxSpecies];  // per species sum of w^2
};

template <class V>
__device__ __forceinline__ Acc<V>* acc_at(unsigned char* p)
{
    return reinterpret_cast<Acc<V>*>(p);
}

// Per-interaction coefficients, computed by one thread from the block sums. FP64 path: in double. Mixed path: in
// float-float (the float pipe; the FP64 pipe of this part is a small fraction of the float rate).
// Eq. vp_pm: B = sum_s m_s sum w (v_ps - v_bs) / sum_s m_s sum w^2 over the interaction's species (one side intra).
__device__ __forceinline__ void shift_coef(const StepArgs& A, const InterConst& ic, bool intra,
                                           const Acc<double>* r, const Acc<double>* W2, Shared& sh)
{
    const double ma = A.m[ic.a], mb = A.m[ic.b];
    const double Sw = ma * W2[ic.a].x + (intra ? 0.0 : mb * W2[ic.b].x);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double S = ma * r[d].x + (intra ? 0.0 : mb * r[3 + d].x);
        sh.B[d] = S / Sw;
        sh.Bf[d] = (float)sh.B[d];
    }
}
__device__ __forceinline__ void shift_coef(const StepArgs& A, const InterConst& ic, bool intra,
                                           const Acc<float>* r, const Acc<float>* W2, Shared& sh)
{
    const ff ma = {A.m_f[ic.a], A.m_lo[ic.a]}, mb = {A.m_f[ic.b], A.m_lo[ic.b]};
    ff Sw = ff_mul(ma, W2[ic.a].x);
    if (!intra) Sw = ff_add(Sw, ff_mul(mb, W2[ic.b].x));
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        ff S = ff_mul(ma, r[d].x);
        if (!intra) S = ff_add(S, ff_mul(mb, r[3 + d].x));
        sh.Bf[d] = ff_div(S, Sw).hi;
    }
}

// Eq. Econs / Eq. DeltaEs: Delta E of the interaction and its split between the species in proportion to mean
// weight times post-shift energy; r = {dE_a, E_a, dE_b, E_b} (halves and masses applied here), W1 = sums of w.
// A species with fewer than two particles cannot take a share; no eligible species with Delta E != 0 fails.
// |Delta E_s| at or below 2^-47 of species s's post-shift kinetic energy counts as zero (rounding noise).
__device__ __forceinline__ void partition_coef(const StepArgs& A, const InterConst& ic, bool intra, int na, int nb,
                                               const Acc<double>* r, const Acc<double>* W1, Shared& sh)
{
    const double ma = A.m[ic.a], mb = A.m[ic.b];
    const double dE = ma * r[0].x + (intra ? 0.0 : mb * r[2].x);
    double D0 = dE, D1 = 0.0;
    int fail = 0;
    if (!intra) {
        const bool can0 = na >= 2, can1 = nb >= 2;
        if (can0 && can1) {
            const double wa = W1[ic.a].x / (double)na * (ma * r[1].x);
            const double wb = W1[ic.b].x / (double)nb * (mb * r[3].x);
            const double den = wa + wb;
            if (den > 0.0) {
                D0 = wa / den * dE;
                D1 = dE - D0;
            } else if (dE != 0.0) {
                fail = 1;
            }
        } else if (can0) {
            D0 = dE;
        } else if (can1) {
            D0 = 0.0;
            D1 = dE;
        } else if (dE != 0.0) {
            fail = 1;
        }
    }
    sh.D[0] = fabs(D0) <= 0x1p-47 * (ma * r[1].x) ? 0.0 : D0;
    sh.D[1] = fabs(D1) <= 0x1p-47 * (intra ? 0.0 : mb * r[3].x) ? 0.0 : D1;
    sh.fail = fail;
}
__device__ __forceinline__ void partition_coef(const StepArgs& A, const InterConst& ic, bool intra, int na, int nb,
                                               const Acc<float>* r, const Acc<float>* W1, Shared& sh)
{
    const ff ma = {A.m_f[ic.a], A.m_lo[ic.a]}, mb = {A.m_f[ic.b], A.m_lo[ic.b]};
    const ff Ea = ff_mul(ma, r[1].x), Eb = ff_mul(mb, r[3].x);
    ff dE = ff_mul(ma, r[0].x);
    if (!intra) dE = ff_add(dE, ff_mul(mb, r[2].x));
    ff D0 = dE, D1 = {0.f, 0.f};
    int fail = 0;
    if (!intra) {
        const bool can0 = na >= 2, can1 = nb >= 2;
        if (can0 && can1) {
            const ff wa = ff_mul(ff_div(W1[ic.a].x, {(float)na, 0.f}), Ea);
            const ff wb = ff_mul(ff_div(W1[ic.b].x, {(float)nb, 0.f}), Eb);
            const ff den = ff_add(wa, wb);
            if (den.hi > 0.f) {
                D0 = ff_mul(ff_div(wa, den), dE);
                D1 = ff_sub(dE, D0);
            } else if (dE.hi != 0.f) {
                fail = 1;
            }
        } else if (can0) {
            D0 = dE;
        } else if (can1) {
            D0 = {0.f, 0.f};
            D1 = dE;
        } else if (dE.hi != 0.f) {
            fail = 1;
        }
    }
    sh.Df[0] = fabsf(D0.hi) <= 0x1p-47f * Ea.hi ? 0.f : D0.hi;
    sh.Df[1] = fabsf(D1.hi) <= 0x1p-47f * (intra ? 0.f : Eb.hi) ? 0.f : D1.hi;
    sh.fail = fail;
}

// Random permutations of the interaction's one or two species segments: local indices ordered by their 64-bit
// Philox keys (44 random bits above the index). The random bits are uniform, so a counting sort on their top
// log2(B) bits (B = next power of two >= n buckets) already places almost every key; each bucket holding several
// keys is finished by an insertion sort on the full key. The result is the sort by full key (keys are distinct).
// One Philox block gives the keys of two consecutive indices, so each thread draws for a pair. The permutation is
// stored as cell-local particle indices (segment start included).
// Scratch: the pre-interaction copy vb (unused until after the permutations) holds the bucket counters.
template <class V>
__device__ void permutations(const StepArgs& A, const Tile<V>& t, Shared& sh, int c, uint32_t ictr, int nside,
                             int a0, int na, int b0, int nb)
{
    uint32_t* cnt = t.cnt;
    const int s0v[2] = {a0, b0}, nv[2] = {na, nb};
    int lgB[2] = {0, 0}, Bv[2] = {0, 0};
    for (int side = 0; side < nside; ++side) {
        while ((1 << lgB[side]) < nv[side]) ++lgB[side];
        Bv[side] = 1 << lgB[side];
    }
    const int base1 = Bv[0];
    const int L = Bv[0] + (nside > 1 ? Bv[1] : 0);
    for (int side = 0; side < nside; ++side) {
        const int s0 = s0v[side], n = nv[side];
        const uint32_t tag = side ? kTagPermB : kTagPermA;
        for (int h = threadIdx.x; 2 * h < n; h += kThreads) {
            const uint4 r = draw_at(A.rng, sh.step, (uint32_t)h, (uint32_t)c, ictr, tag);
            t.keys[s0 + 2 * h] = ((((uint64_t)r.x << 32) | r.y) & ~kPermMask) | (uint64_t)(2 * h);
            if (2 * h + 1 < n) t.keys[s0 + 2 * h + 1] = ((((uint64_t)r.z << 32) | r.w) & ~kPermMask) | (uint64_t)(2 * h + 1);
        }
    }
    for (int b = threadIdx.x; b < L; b += kThreads) cnt[b] = 0;
    __syncthreads();
    for (int side = 0; side < nside; ++side) {
        const int base = side ? base1 : 0;
        for (int q = threadIdx.x; q < nv[side]; q += kThreads) {
            const uint64_t k = t.keys[s0v[side] + q];
            const int b = lgB[side] ? (int)(k >> (64 - lgB[side])) : 0;
            atomicAdd(&cnt[base + b], 1u);
        }
    }
    __syncthreads();
    // exclusive scan over both sides' buckets (side 1's positions are offset by na)
    {
        const int chunk = (L + kThreads - 1) / kThreads;
        const int lo = threadIdx.x * chunk, hi = min(L, lo + chunk);
        int local = 0;
        for (int b = lo; b < hi; ++b) local += (int)cnt[b];
        int total;
        int run = block_exclusive_scan<int>(local, sh.iscan, total);
        for (int b = lo; b < hi; ++b) {
            const int x = (int)cnt[b];
            cnt[b] = (uint32_t)run;
            run += x;
        }
    }
    __syncthreads();
    for (int side = 0; side < nside; ++side) {
        const int base = side ? base1 : 0, off = side ? na : 0, s0 = s0v[side];
        for (int q = threadIdx.x; q < nv[side]; q += kThreads) {
            const uint64_t k = t.keys[s0 + q];
            const int b = lgB[side] ? (int)(k >> (64 - lgB[side])) : 0;
            const int pos = (int)atomicAdd(&cnt[base + b], 1u) - off;
            t.perm[s0 + pos] = s0 + q;
        }
    }
    __syncthreads();
    // cnt[b] now holds the end of bucket b: finish buckets with several keys
    for (int side = 0; side < nside; ++side) {
        const int base = side ? base1 : 0, off = side ? na : 0, s0 = s0v[side];
        for (int b = threadIdx.x; b < Bv[side]; b += kThreads) {
            const int end = (int)cnt[base + b] - off;
            const int start = b ? (int)cnt[base + b - 1] - off : 0;
            for (int x = start + 1; x < end; ++x) {
                const int v = t.perm[s0 + x];
                const uint64_t kv = t.keys[v];
                int y = x - 1;
                while (y >= start && t.keys[t.perm[s0 + y]] > kv) {
                    t.perm[s0 + y + 1] = t.perm[s0 + y];
                    --y;
                }
                t.perm[s0 + y + 1] = v;
            }
        }
    }
    __syncthreads();
}

template <class V>
__device__ __forceinline__ V* scan_scratch(Shared& sh);
template <>
__device__ __forceinline__ double* scan_scratch<double>(Shared& sh) { return sh.scan_d; }
template <>
__device__ __forceinline__ float* scan_scratch<float>(Shared& sh) { return sh.scan_f; }

// k-th Takizuka-Abe pair of the interaction (cell-local indices). See mcc_pair in mcc.h for the rule.
// pm = p mod N_min (inter only; the callers know it without a division).
template <class V>
__device__ __forceinline__ void pair_at(const Tile<V>& t, bool intra, int na, int nb, int a0, int b0, int p, int pm,
                                        int& i, int& j, uint8_t& f)
{
    f = 0;
    if (intra) {
        if (na & 1) {
            if (p < 3) {
                i = t.perm[a0 + p];
                j = t.perm[a0 + (p + 1) % 3];
                f = kPairTriplet;
                return;
            }
            i = t.perm[a0 + 2 * p - 3];
            j = t.perm[a0 + 2 * p - 2];
            return;
        }
        i = t.perm[a0 + 2 * p];
        j = t.perm[a0 + 2 * p + 1];
        return;
    }
    if (na >= nb) {
        i = t.perm[a0 + p];
        j = t.perm[b0 + pm];
    } else {
        i = t.perm[a0 + pm];
        j = t.perm[b0 + p];
    }
}

// Slot k of the order N x N schedule (local indices into the interaction's permutations). Inter: round k / N_min
// pairs the smaller population's m = k mod N_min with the larger one's (m + round) mod N_max. Intra: round-robin
// tournament (circle method) over N players plus an idle one when N is odd; false for a slot with the idle player.
__device__ __forceinline__ bool nxn_slot(int na, int nb, bool intra, int k, int& a, int& b)
{
    if (intra) {
        const int M = na + (na & 1), half = M / 2;
        const int r = k / half, q = k - r * half;
        if (q == 0) {
            a = r;
            b = M - 1;
        } else {
            a = (r + q) % (M - 1);
            b = (r - q + (M - 1)) % (M - 1);
        }
        return a < na && b < na;
    }
    const int lo = na < nb ? na : nb, hi = na < nb ? nb : na;
    const int r = k / lo, m = k - r * lo;
    const int big = (m + r) % hi;
    if (na >= nb) {
        a = big;
        b = m;
    } else {
        a = m;
        b = big;
    }
    return true;
}

// Heavier particle of an unequal-weight pair moves iff U3 w_max < w_min, decided in FP64 exactly as the
// definition states. The mixed path first decides in float with a bound on the float error and falls back to the
// FP64 test only within that bound of the boundary.
__device__ __forceinline__ bool heavy_moves(const Tile<double>& t, const StepArgs&, int64_t, int i, int j,
                                            uint32_t r)
{
    const double U3 = u23<double>(r);
    const double wi = t.w[i], wj = t.w[j];
    return U3 * fmax(wi, wj) < fmin(wi, wj);
}

__device__ __forceinline__ bool heavy_moves(const Tile<float>& t, const StepArgs& A, int64_t cs, int i, int j,
                                            uint32_t r)
{
    const float U3 = u23<float>(r);
    const float hi_i = t.w[i].x, hi_j = t.w[j].x;
    const float p = U3 * fmaxf(hi_i, hi_j);
    const float wmin = fminf(hi_i, hi_j);
    const float x = p - wmin;
    const float tol = 10.0f * 5.9604645e-8f * fmaxf(p, wmin);
    if (x > tol) return false;
    if (x < -tol) return true;
    const double wi = A.w[cs + i], wj = A.w[cs + j];
    return u23<double>(r) * fmax(wi, wj) < fmin(wi, wj);
}

// acc += w_i (x_new - x_old): on the mixed path the difference as float-float (two_sum, exact) times the weight's
// hi/lo split
__device__ __forceinline__ void add_weighted_change(Acc<double>& acc, const Tile<double>& t, int i, double xn,
                                                    double xo)
{
    acc.add(t.w[i] * (xn - xo));
}
__device__ __forceinline__ void add_weighted_change(Acc<float>& acc, const Tile<float>& t, int i, float xn, float xo)
{
    const float2 w = t.w[i];
    acc.add(ff_mul({w.x, w.y}, ff_two_sum(xn, -xo)));
}

__device__ __forceinline__ void add_weight_sums(Acc<double>& a1, Acc<double>& a2, const Tile<double>& t, int i)
{
    a1.add(t.w[i]);
    a2.add(t.w[i] * t.w[i]);
}
__device__ __forceinline__ void add_weight_sums(Acc<float>& a1, Acc<float>& a2, const Tile<float>& t, int i)
{
    const ff w = {t.w[i].x, t.w[i].y};
    a1.add(w);
    a2.add(ff_mul(w, w));
}

// Relativistic pair, given its CM frame: scattering length with |p*|^2 v_rel* in place of mu^2 u^3, rotation of p*
// through (Theta, phi), boost of the change back to the lab frame. Returns dp = p_i' - p_i.
template <class V>
__device__ __forceinline__ void rel_pair_dp_cm(const StepArgs& A, const InterConst& ic, const RelCM<V>& cm, V cc,
                                               V wf, uint8_t f, V U1, V U2, V U4, V dp[3])
{
    V s = pick<V>(ic.kappa, ic.kappa_f) * wf / (cm.pmag * cm.pmag * cm.vrel);
    if (f & kPairTriplet) s *= (V)0.5;
    V st, omc, sp, cp, dx, dy, dz;
    N97Tab<V> tab;
    n97_tab(A, tab);
    sample_angle<V>(A.method, s, U1, U4, st, omc, tab);
    sincospi_v((V)2 * U2, &sp, &cp);
    rotate<V>(cm.px, cm.py, cm.pz, st, omc, cp, sp, dx, dy, dz);
    const V coef_b = cm.gC * cm.gC / (cc * cc * (cm.gC + (V)1));
    const V Vd = cm.Vx * dx + cm.Vy * dy + cm.Vz * dz;
    dp[0] = dx + coef_b * Vd * cm.Vx;
    dp[1] = dy + coef_b * Vd * cm.Vy;
    dp[2] = dz + coef_b * Vd * cm.Vz;
}

template <class V>
__device__ __noinline__ void rel_pair_dp(const StepArgs& A, const InterConst& ic, const V vi[3], const V vj[3],
                                         V wf, uint8_t f, V U1, V U2, V U4, V dp[3])
{
    const V cc = pick<V>(A.c, A.c_f);
    const V ma = pick<V>(A.ma[ic.a], A.ma_f[ic.a]), mb = pick<V>(A.ma[ic.b], A.ma_f[ic.b]);
    const RelCM<V> cm = rel_cm<V>(cc, ma, mb, vi, vj);
    if (!(cm.pmag > (V)0)) {
        dp[0] = dp[1] = dp[2] = (V)0;
        return;
    }
    rel_pair_dp_cm<V>(A, ic, cm, cc, wf, f, U1, U2, U4, dp);
}

// One scattering pair (Algorithm 1 pair loop).
template <class V, bool REL>
__device__ __forceinline__ void scatter_pair(const StepArgs& A, const Tile<V>& t, int c, int64_t cs, uint32_t ictr,
                                             const InterConst& ic, int p, int i, int j, uint8_t f, int nmin,
                                             int nmax, int pm, uint32_t step)
{
    V vi[3] = {t.v[i], t.v[t.vs + i], t.v[2 * t.vs + i]};
    V vj[3] = {t.v[j], t.v[t.vs + j], t.v[2 * t.vs + j]};
    const V wi = wv(t, i), wj = wv(t, j);
    const V wmax = wi > wj ? wi : wj;
    // w_max N_min of Eq. sab_TA77, or with duplicity weighting (w_max / D_ij) N_max for an inter-species pair: the
    // smaller population's particle of pair p (index pm = p mod N_min) is paired D = (N_max - 1 - pm) / N_min + 1 times
    V wf = wmax * (V)nmin;
    if (A.weighting == 1 && nmax > 0) wf = wmax / (V)((nmax - 1 - pm) / nmin + 1) * (V)nmax;
    const uint4 r = draw_at(A.rng, step, (uint32_t)p, (uint32_t)c, ictr, kTagScat);
    const V U1 = u23<V>(r.x), U2 = u23<V>(r.y), U4 = u23<V>(r.w);
    V dvi[3], dvj[3];
    if (!REL) {
        const V ux = vi[0] - vj[0], uy = vi[1] - vj[1], uz = vi[2] - vj[2];
        const V u2 = ux * ux + uy * uy + uz * uz;
        if (u2 == (V)0) return;
        const V um = sqrt(u2);
        V s = pick<V>(ic.kappa_mu2, ic.kappa_mu2_f) * wf / (u2 * um);
        if (f & kPairTriplet) s *= (V)0.5;
        V st, omc, sp, cp, dx, dy, dz;
        N97Tab<V> tab;
        n97_tab(A, tab);
        sample_angle<V>(A.method, s, U1, U4, st, omc, tab);
        sincospi_v((V)2 * U2, &sp, &cp);
        rotate<V>(ux, uy, uz, st, omc, cp, sp, dx, dy, dz);
        const V fa = pick<V>(ic.mu_ma, ic.mu_ma_f), fb = pick<V>(ic.mu_mb, ic.mu_mb_f);
        dvi[0] = fa * dx; dvi[1] = fa * dy; dvi[2] = fa * dz;
        dvj[0] = -fb * dx; dvj[1] = -fb * dy; dvj[2] = -fb * dz;
    } else {
        V du2 = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) du2 += (vi[d] - vj[d]) * (vi[d] - vj[d]);
        if (du2 == (V)0) return;
        const V cc = pick<V>(A.c, A.c_f);
        const V ma = pick<V>(A.ma[ic.a], A.ma_f[ic.a]), mb = pick<V>(A.ma[ic.b], A.ma_f[ic.b]);
        const RelCM<V> cm = rel_cm<V>(cc, ma, mb, vi, vj);
        if (sizeof(V) == 4 && cm.gC > (V)2) {
            // a fast-moving CM frame amplifies float rounding by ~gamma_C^2: this pair's kinematics run in double
            const double vid[3] = {vi[0], vi[1], vi[2]}, vjd[3] = {vj[0], vj[1], vj[2]};
            double dd[3];
            rel_pair_dp<double>(A, ic, vid, vjd, (double)wf, f, u23<double>(r.x), u23<double>(r.y),
                                u23<double>(r.w), dd);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                dvi[d] = (V)(dd[d] / A.ma[ic.a]);
                dvj[d] = (V)(-dd[d] / A.ma[ic.b]);
            }
        } else {
            if (!(cm.pmag > (V)0)) return;
            V dp[3];
            rel_pair_dp_cm<V>(A, ic, cm, cc, wf, f, U1, U2, U4, dp);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                dvi[d] = dp[d] / ma;
                dvj[d] = -dp[d] / mb;
            }
        }
    }
    bool upd_i = true, upd_j = true;
    if (!w_equal(t, i, j)) {
        const bool moves = heavy_moves(t, A, cs, i, j, r.z);
        if (wi > wj || (wi == wj && w_exact(t, A, cs, i) > w_exact(t, A, cs, j))) upd_i = moves;
        else upd_j = moves;
    }
    if (upd_i) {
#pragma unroll
        for (int d = 0; d < 3; ++d) t.v[d * t.vs + i] = vi[d] + dvi[d];
    }
    if (upd_j) {
#pragma unroll
        for (int d = 0; d < 3; ++d) t.v[d * t.vs + j] = vj[d] + dvj[d];
    }
}

// Energy-pair order of a species segment with partially tied weights: the interaction's random permutation, stably
// sorted by descending weight (keys: weight, rank in the permutation). Out of line: rare.
template <class V>
__device__ __noinline__ void tie_order(const StepArgs& A, const Tile<V>& t, int64_t cs, int s0, int ns)
{
    if (ns <= kWarpSortMax) {
        if (threadIdx.x < 32) {
            for (int r = threadIdx.x; r < ns; r += 32)
                t.keys[s0 + r] = weight_key(w_exact(t, A, cs, t.perm[s0 + r]), (uint32_t)r);
            warp_sort_buf(t.keys + s0, ns);
            for (int m = threadIdx.x; m < ns; m += 32) t.rho[s0 + m] = t.perm[s0 + (int)(t.keys[s0 + m] & kPermMask)];
        }
        __syncthreads();
    } else {
        for (int q = threadIdx.x; q < ns; q += kThreads)
            t.keys[s0 + q] = weight_key(w_exact(t, A, cs, t.perm[s0 + q]), (uint32_t)q);
        __syncthreads();
        block_sort_u64(t.keys + s0, ns);
        for (int q = threadIdx.x; q < ns; q += kThreads) t.rho[s0 + q] = t.perm[s0 + (int)(t.keys[s0 + q] & kPermMask)];
        __syncthreads();
    }
}

// Moment correction of one interaction (Sec. 4, Appendix A, Sec. 5.2).
template <class V, bool REL, int MODE>
__device__ void correct_interaction(const StepArgs& A, const Tile<V>& t, Shared& sh, int c, int64_t cs,
                                    const InterConst& ic, bool intra, int a0, int na, int b0, int nb)
{
    const int nside = intra ? 1 : 2;
    const V cc = pick<V>(A.c, A.c_f);

    // Eq. vp_pm: per species sums of w (v_ps - v_bs), times m_s in FP64; the sums of w^2 are fixed for the visit
    {
        Acc<V> mom[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) mom[m] = Acc<V>::zero();
        for (int side = 0; side < nside; ++side) {
            const int s0 = side ? b0 : a0, ns = side ? nb : na;
            for (int q = threadIdx.x; q < ns; q += kThreads) {
                const int i = s0 + q;
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    add_weighted_change(mom[side * 3 + d], t, i, t.v[d * t.vs + i], t.vb[d * t.bs + i]);
            }
        }
        block_sum<V, 6>(mom, acc_at<V>(sh.red_raw), acc_at<V>(sh.red));
        if (threadIdx.x == 0) shift_coef(A, ic, intra, acc_at<V>(sh.red), acc_at<V>(sh.W2), sh);
        __syncthreads();
    }

    // Momentum shift (Eq. vp_pm) fused with the sums of Eq. Econs as per-particle energy differences and the
    // post-shift species energies (Eq. DeltaEs; its weight sums are fixed for the visit)
    {
        Acc<V> acc[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[m] = Acc<V>::zero();
        for (int side = 0; side < nside; ++side) {
            const int s0 = side ? b0 : a0, ns = side ? nb : na;
            for (int q = threadIdx.x; q < ns; q += kThreads) {
                const int i = s0 + q;
                const V w = wv(t, i);
                V dd = 0, v2 = 0, b2 = 0;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const V x = t.v[d * t.vs + i] - pick<V>(sh.B[d], sh.Bf[d]) * w;  // v_pm = v_ps - B w_p
                    t.v[d * t.vs + i] = x;
                    const V y = t.vb[d * t.bs + i];
                    dd += (x - y) * (x + y);
                    v2 += x * x;
                    b2 += y * y;
                }
                if (!REL) {
                    acc[side * 2 + 0].add((V)0.5 * w * dd);
                    acc[side * 2 + 1].add((V)0.5 * w * v2);
                } else {
                    const V c2 = cc * cc;
                    const V ga = sqrt((V)1 + v2 / c2), gb = sqrt((V)1 + b2 / c2);
                    acc[side * 2 + 0].add(w * dd / (ga + gb));
                    acc[side * 2 + 1].add(w * v2 / (ga + (V)1));
                }
            }
        }
        block_sum<V, 4>(acc, acc_at<V>(sh.red_raw), acc_at<V>(sh.red));
        if (threadIdx.x == 0) partition_coef(A, ic, intra, na, nb, acc_at<V>(sh.red), acc_at<V>(sh.W1), sh);
        __syncthreads();
    }

    // energy-correction pairs, species a then b
    int used = 0;
    for (int side = 0; side < nside; ++side) {
        if (sh.fail) break;
        const V D = pick<V>(sh.D[side], sh.Df[side]);
        if (D == (V)0) continue;
        const int s0 = side ? b0 : a0, ns = side ? nb : na;
        const int spc = side ? ic.b : ic.a;
        const V ms = pick<V>(A.m[spc], A.m_f[spc]);
        // order of the energy pairs: the random permutation, stably sorted by descending weight (optional step of
        // Algorithm 1). Distinct weights: the order fixed at the cell's load; all equal: the permutation itself;
        // partial ties: sorted here by (weight, rank in the permutation).
        const int mode = A.sort_by_weight ? sh.wmode[spc] : 1;
        if (mode == 2) tie_order<V>(A, t, cs, s0, ns);
        const int32_t* order = (mode == 1) ? t.perm : t.rho;
        auto rho = [&](int m) -> int { return mode == 3 ? s0 + m : order[s0 + m]; };
        V Dabs = D < (V)0 ? -D : D;
        const V sgn = D > (V)0 ? (V)1 : (V)-1;
        const V fE = pick<V>(A.fE, A.fE_f);
        // pair m of a pass starting at offset o: its particles, velocities, weighted masses and CM energy K
        auto load_pair = [&](int o, int m, int& i, int& j, V v1[3], V v2[3], V& m1, V& m2) -> V {
            i = rho(o + 2 * m);
            j = rho(o + 2 * m + 1);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                v1[d] = t.v[d * t.vs + i];
                v2[d] = t.v[d * t.vs + j];
            }
            m1 = ms * wv(t, i);
            m2 = ms * wv(t, j);
            if (REL && sizeof(V) == 4 && fast_pair(cc, v1, v2)) {
                const double d1[3] = {v1[0], v1[1], v1[2]}, d2[3] = {v2[0], v2[1], v2[2]};
                return (V)pair_kecm<double, true>(A.c, A.m[side ? ic.b : ic.a] * w_exact(t, A, cs, i),
                                                  A.m[side ? ic.b : ic.a] * w_exact(t, A, cs, j), d1, d2);
            }
            return pair_kecm<V, REL>(cc, m1, m2, v1, v2);
        };
        // the pair takes its cap, or the remainder if it is the crossing pair (excl = caps of the pairs before it)
        auto apply_pair = [&](int i, int j, V v1[3], V v2[3], V m1, V m2, V K, V capv, V excl) {
            const V rem = Dabs - excl;
            const V U = sgn * (rem < capv ? rem : capv);
            if (REL && sizeof(V) == 4 && fast_pair(cc, v1, v2)) {
                double d1[3] = {v1[0], v1[1], v1[2]}, d2[3] = {v2[0], v2[1], v2[2]};
                const double ms_d = A.m[side ? ic.b : ic.a];
                energy_pair<double, true>(A.c, ms_d * w_exact(t, A, cs, i), ms_d * w_exact(t, A, cs, j), (double)K,
                                          d1, d2, (double)U);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    v1[d] = (V)d1[d];
                    v2[d] = (V)d2[d];
                }
            } else {
                energy_pair<V, REL>(cc, m1, m2, K, v1, v2, U);
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                t.v[d * t.vs + i] = v1[d];
                t.v[d * t.vs + j] = v2[d];
            }
            ++used;
        };
        // The crossing pair is nearly always among the first 32 pairs of the first pass: one warp computes their caps
        // and their prefix sum (the same sums, in the same order, as the block scan below) and finishes the side if
        // they absorb |Delta E_s|; otherwise nothing was applied and the block loop runs from the start.
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            const int np0 = ns / 2;
            const bool valid = lane < np0;
            int i = 0, j = 0;
            V v1[3] = {0, 0, 0}, v2[3] = {0, 0, 0}, K = 0, capv = 0, m1 = 1, m2 = 1;
            if (valid) {
                K = load_pair(0, lane, i, j, v1, v2, m1, m2);
                capv = K > (V)0 ? fE * K : (V)0;
            }
            V inc = capv;
#pragma unroll
            for (int s1 = 1; s1 < 32; s1 <<= 1) {
                const V y = __shfl_up_sync(0xffffffffu, inc, s1);
                if (lane >= s1) inc += y;
            }
            V excl = __shfl_up_sync(0xffffffffu, inc, 1);
            if (lane == 0) excl = (V)0;
            const V tot = __shfl_sync(0xffffffffu, inc, 31);
            const bool fast = tot >= Dabs;
            if (fast && valid && K > (V)0 && excl < Dabs) apply_pair(i, j, v1, v2, m1, m2, K, capv, excl);
            if (lane == 0) sh.fast = fast;
        }
        __syncthreads();
        bool done = sh.fast;
        for (int pass = 0; pass < A.max_corr_passes && !done; ++pass) {
            const int o = pass & 1;
            const int np = (ns - o) / 2;
            V carry = 0;
            for (int base = 0; base < np && !done; base += kThreads) {
                const int m = base + threadIdx.x;
                const bool valid = m < np;
                int i = 0, j = 0;
                V v1[3] = {0, 0, 0}, v2[3] = {0, 0, 0}, K = 0, capv = 0, m1 = 1, m2 = 1;
                if (valid) {
                    K = load_pair(o, m, i, j, v1, v2, m1, m2);
                    capv = K > (V)0 ? fE * K : (V)0;
                }
                V total;
                const V excl = block_exclusive_scan<V>(capv, scan_scratch<V>(sh), total) + carry;
                if (valid && K > (V)0 && excl < Dabs) apply_pair(i, j, v1, v2, m1, m2, K, capv, excl);
                carry += total;
                if (carry >= Dabs) done = true;
            }
            if (!done) Dabs -= carry;
        }
        __syncthreads();
        if (!done && threadIdx.x == 0) sh.fail = 1;
        __syncthreads();
    }
    const int used_all = block_sum_int(used, sh.iscr);
    const int failed = sh.fail;
    if (failed) {
        if (A.fail_policy == 0) {
            for (int side = 0; side < nside; ++side) {
                const int s0 = side ? b0 : a0, ns = side ? nb : na;
                for (int q = threadIdx.x; q < ns; q += kThreads) {
                    const int i = s0 + q;
#pragma unroll
                    for (int d = 0; d < 3; ++d) t.v[d * t.vs + i] = t.vb[d * t.bs + i];
                }
            }
        }
        if (A.fail_policy == 2 && threadIdx.x == 0) latch(A.status, kErrCorrectionFailed);
    }
    if (threadIdx.x == 0) {
        if (MODE == kCorrect) {
            if (A.corr_pairs) A.corr_pairs[c] = used_all;
            if (A.fail_count) A.fail_count[c] = failed;
        } else {
            if (A.corr_pairs) A.corr_pairs[c] += used_all;
            if (A.fail_count) A.fail_count[c] += failed;
        }
    }
    __syncthreads();
}

template <class V, bool REL, int MODE>
__device__ void interaction(const StepArgs& A, const Tile<V>& t, Shared& sh, int c, int64_t cs, int k)
{
    const InterConst& ic = A.ic[k];
    const int a = ic.a, b = ic.b;
    const bool intra = (a == b);
    const int a0 = sh.off[a], na = sh.off[a + 1] - a0;
    const int b0 = sh.off[b], nb = sh.off[b + 1] - b0;
    const uint32_t ictr = (uint32_t)(A.inter_base + k);
    const bool active = intra ? (na >= 2) : (na > 0 && nb > 0);
    if (!active) {
        if (MODE == kCorrect && threadIdx.x == 0) {
            if (A.corr_pairs) A.corr_pairs[c] = 0;
            if (A.fail_count) A.fail_count[c] = 0;
        }
        return;
    }
    // random permutation of each participating species (counter = {i/2, cell, step, inter<<8 | 1 + side})
    if (MODE != kScatter) permutations<V>(A, t, sh, c, ictr, intra ? 1 : 2, a0, na, b0, nb);
    const int npairs = intra ? ((na & 1) ? (na + 3) / 2 : na / 2) : (na > nb ? na : nb);
    const int nmin = intra ? na - 1 : (na < nb ? na : nb);
    if (MODE == kPair) {
        for (int p = threadIdx.x; p < npairs; p += kThreads) {
            int i, j;
            uint8_t f;
            pair_at(t, intra, na, nb, a0, b0, p, intra ? 0 : p % nmin, i, j, f);
            A.pair_i[cs + p] = (int32_t)(cs + i);
            A.pair_j[cs + p] = (int32_t)(cs + j);
            A.pair_flags[cs + p] = f;
        }
        __syncthreads();
        return;
    }
    // pre-interaction copy of every participant
    V* gb = reinterpret_cast<V*>(A.backup);
    for (int side = 0; side < (intra ? 1 : 2); ++side) {
        const int s0 = side ? b0 : a0, ns = side ? nb : na;
        for (int q = threadIdx.x; q < ns; q += kThreads) {
            const int i = s0 + q;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (MODE == kCorrect) {
                    t.vb[d * t.bs + i] = gb[d * A.n_total + cs + i];
                } else {
                    const V x = t.v[d * t.vs + i];
                    t.vb[d * t.bs + i] = x;
                    if (MODE == kScatter) gb[d * A.n_total + cs + i] = x;
                }
            }
        }
    }
    __syncthreads();
    if (MODE == kFused || MODE == kScatter) {
        auto get = [&](int p, int pm, int& i, int& j, uint8_t& f) {
            if (MODE == kScatter) {
                i = (int)(A.pair_i[cs + p] - cs);
                j = (int)(A.pair_j[cs + p] - cs);
                f = A.pair_flags[cs + p];
            } else {
                pair_at(t, intra, na, nb, a0, b0, p, pm, i, j, f);
            }
        };
        if (MODE == kFused && A.pairing == 1) {
            // order N x N (Eq. sab_weighted): every pair once, in rounds of disjoint pairs, s with w_max alone
            const int per = intra ? (na + (na & 1)) / 2 : (na < nb ? na : nb);
            const int nslots = intra ? (2 * per - 1) * per : na * nb;
            for (int r0 = 0; r0 < nslots; r0 += per) {
                for (int q = threadIdx.x; q < per; q += kThreads) {
                    int a, b;
                    if (!nxn_slot(na, nb, intra, r0 + q, a, b)) continue;
                    const int i = t.perm[a0 + a], j = intra ? t.perm[a0 + b] : t.perm[b0 + b];
                    scatter_pair<V, REL>(A, t, c, cs, ictr, ic, r0 + q, i, j, 0, 1, 0, 0, sh.step);
                }
                __syncthreads();
            }
        } else {
        // Intra: one round; an odd count starts with the triplet (pairs 0..2 share particles), run in order by thread
        // 0 while the other threads start on pair 3. Inter: rounds of N_min disjoint pairs, in order. One call site
        // keeps a single inlined copy of the pair code.
        const int lead = (intra && (na & 1)) ? 3 : 0;
        const int round = intra ? npairs : nmin;
        for (int r0 = 0; r0 < npairs; r0 += round) {
            const int r1 = r0 + round < npairs ? r0 + round : npairs;
            int p = (lead && threadIdx.x == 0) ? 0 : r0 + lead + (int)threadIdx.x;
            while (p < r1) {
                int i, j;
                uint8_t f;
                get(p, p - r0, i, j, f);
                scatter_pair<V, REL>(A, t, c, cs, ictr, ic, p, i, j, f, nmin, intra ? 0 : npairs, p - r0, sh.step);
                p = (p + 1 < lead) ? p + 1 : (p < lead ? lead + (int)threadIdx.x : p + kThreads);
            }
            __syncthreads();
        }
        }
    }
    if (MODE == kCorrect || (MODE == kFused && A.correct))
        correct_interaction<V, REL, MODE>(A, t, sh, c, cs, ic, intra, a0, na, b0, nb);
}

// Weight-descending order of each species of the cell, fixed for this visit when the weight keys are distinct (one
// warp per species). A segment stored with strictly increasing keys (strictly descending weights, no two within the
// key's tie width) needs no sort (wmode 3). Out of line: it runs once per visit and keeps the per-interaction code
// compact.
template <class V>
__device__ __noinline__ void weight_order(const StepArgs& A, const Tile<V>& t, Shared& sh, int64_t cs, int S)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int sp = 0; sp < S; ++sp) {
        const int s0 = sh.off[sp], ns = sh.off[sp + 1] - s0;
        if (warp != sp % kWarps) continue;
        bool unsorted = false;
        for (int q0 = 0; q0 + 1 < ns && !unsorted; q0 += 32) {
            const int q = q0 + lane;
            const bool bad = q + 1 < ns &&
                             weight_key(w_exact(t, A, cs, s0 + q), 0) >= weight_key(w_exact(t, A, cs, s0 + q + 1), 0);
            unsorted = __any_sync(0xffffffffu, bad);
        }
        if (!unsorted) {
            if (lane == 0) sh.wmode[sp] = 3;
            continue;
        }
        if (ns > kWarpSortMax) {
            if (lane == 0) sh.wmode[sp] = 2;
            continue;
        }
        int tie = 0;
        for (int q = lane; q < ns; q += 32) t.keys[s0 + q] = weight_key(w_exact(t, A, cs, s0 + q), (uint32_t)q);
        warp_sort_buf(t.keys + s0, ns);
        for (int q = lane; q < ns; q += 32) t.rho[s0 + q] = s0 + (int)(t.keys[s0 + q] & kPermMask);
        for (int q = lane; q + 1 < ns; q += 32) tie |= (t.keys[s0 + q] >> kPermBits) == (t.keys[s0 + q + 1] >> kPermBits);
        tie = __any_sync(0xffffffffu, tie);
        const bool all_equal = (t.keys[s0] >> kPermBits) == (t.keys[s0 + ns - 1] >> kPermBits);
        if (lane == 0) sh.wmode[sp] = all_equal ? 1 : (tie ? 2 : 0);
    }
    __syncthreads();
}

template <class V, bool REL, int MODE>
__device__ void process_cell(const StepArgs& A, int c, unsigned char* dyn, Shared& sh)
{
    const int S = A.S;
    const int64_t cs = A.offsets[(int64_t)c * S];
    const int n = (int)(A.offsets[(int64_t)(c + 1) * S] - cs);
    Tile<V> t;
    if (MODE == kPair) {
        if (n > A.cap) {
            if (threadIdx.x == 0) latch(A.status, kErrBounds);
            return;
        }
        t = make_pair_tile<V>(dyn, A.cap);
    } else if (n <= A.cap) {
        t = make_tile<V>(dyn, A.cap);
    } else if (A.slab != nullptr && n <= A.slab_cap) {
        t = make_tile<V>(reinterpret_cast<unsigned char*>(A.slab) + (size_t)blockIdx.x * (size_t)A.slab_stride,
                         A.slab_cap);
        int ms = 0;
        for (int sp = 0; sp < S; ++sp) {
            const int k = (int)(A.offsets[(int64_t)c * S + sp + 1] - A.offsets[(int64_t)c * S + sp]);
            ms = k > ms ? k : ms;
        }
        place_on_chip<V>(t, dyn, (size_t)A.cap * tile_bytes_per_particle(sizeof(V) == 4), n, ms);
    } else {
        if (threadIdx.x == 0) latch(A.status, kErrBounds);
        return;
    }
    if ((int)threadIdx.x <= S) sh.off[threadIdx.x] = (int)(A.offsets[(int64_t)c * S + threadIdx.x] - cs);
    V* gx = reinterpret_cast<V*>(A.vx);
    V* gy = reinterpret_cast<V*>(A.vy);
    V* gz = reinterpret_cast<V*>(A.vz);
    if (MODE != kPair) {
        for (int i = threadIdx.x; i < n; i += kThreads) {
            t.v[i] = gx[cs + i];
            t.v[t.vs + i] = gy[cs + i];
            t.v[2 * t.vs + i] = gz[cs + i];
            w_store(t, i, A.w[cs + i]);
        }
    }
    __syncthreads();
    // per species sums of w and w^2 (Eq. vp_pm denominator, Eq. DeltaEs mean weights), once per visit
    if (MODE == kFused || MODE == kCorrect) {
        for (int sp0 = 0; sp0 < S; sp0 += 4) {
            Acc<V> acc[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[m] = Acc<V>::zero();
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int sp = sp0 + k;
                if (sp >= S) break;
                const int s0 = sh.off[sp], ns = sh.off[sp + 1] - s0;
                for (int q = threadIdx.x; q < ns; q += kThreads) add_weight_sums(acc[2 * k], acc[2 * k + 1], t, s0 + q);
            }
            block_sum<V, 8>(acc, acc_at<V>(sh.red_raw), acc_at<V>(sh.red));
            if (threadIdx.x < 4 && sp0 + (int)threadIdx.x < S) {
                acc_at<V>(sh.W1)[sp0 + threadIdx.x] = acc_at<V>(sh.red)[2 * threadIdx.x];
                acc_at<V>(sh.W2)[sp0 + threadIdx.x] = acc_at<V>(sh.red)[2 * threadIdx.x + 1];
            }
        }
        __syncthreads();
    }
    if ((MODE == kFused || MODE == kCorrect) && A.sort_by_weight) weight_order<V>(A, t, sh, cs, S);
    for (int k = 0; k < A.n_inter; ++k) interaction<V, REL, MODE>(A, t, sh, c, cs, k);
    if (MODE != kPair) {
        for (int i = threadIdx.x; i < n; i += kThreads) {
            gx[cs + i] = t.v[i];
            gy[cs + i] = t.v[t.vs + i];
            gz[cs + i] = t.v[2 * t.vs + i];
        }
    }
}

template <class V, bool REL, int MODE>
__global__ void __launch_bounds__(kThreads, MCC_MIN_BLOCKS) cell_kernel(const __grid_constant__ StepArgs A)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ Shared sh;
    if (threadIdx.x == 0) sh.step = A.step_dev ? (uint32_t)(*A.step_dev + A.step_add) : A.rng.step;
    for (;;) {
        if (threadIdx.x == 0) {
            const int q = atomicAdd(A.queue, 1);
            if (A.order_range) {
                const int b = A.order_range[0], e = A.order_range[1];
                sh.cell = b + q < e ? A.order[b + q] : A.n_cells;
            } else {
                sh.cell = (q < A.n_cells && A.order) ? A.order[q] : q;
            }
        }
        __syncthreads();
        const int c = sh.cell;
        if (c >= A.n_cells) break;
        process_cell<V, REL, MODE>(A, c, dyn, sh);
        __syncthreads();
    }
}

// Advance a step counter kept in device memory (after the steps of one call, so that a captured graph of the call
// serves every later step).
__global__ void k_step_advance(uint64_t* step, uint64_t by)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *step += by;
}

// Cells ordered by descending size class (floor(log2 n)), so the persistent CTAs take the largest cells first and
// the small ones fill in at the end (longest-processing-time order). Order within a class is arbitrary: cells are
// independent, so the result does not depend on it. One CTA; shared-memory counters.
constexpr int kOrderThreads = 1024;

__global__ void __launch_bounds__(kOrderThreads) k_cell_order(const int64_t* __restrict__ offsets, int32_t n_cells,
                                                             int32_t S, int32_t* __restrict__ order)
{
    __shared__ int hist[33];
    if (threadIdx.x < 33) hist[threadIdx.x] = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < n_cells; c += kOrderThreads) {
        const int64_t n = offsets[(int64_t)(c + 1) * S] - offsets[(int64_t)c * S];
        const int cls = n > 0 ? 63 - __clzll((unsigned long long)n) : 0;
        atomicAdd(&hist[32 - (cls > 32 ? 32 : cls)], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 0; b < 33; ++b) {
            const int x = hist[b];
            hist[b] = run;
            run += x;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n_cells; c += kOrderThreads) {
        const int64_t n = offsets[(int64_t)(c + 1) * S] - offsets[(int64_t)c * S];
        const int cls = n > 0 ? 63 - __clzll((unsigned long long)n) : 0;
        order[atomicAdd(&hist[32 - (cls > 32 ? 32 : cls)], 1)] = c;
    }
}

// Cells by group size class for the group kernels: class k holds cells of at most caps[k] particles (the smallest
// such k), class kGroupClasses the cells above every class. The order lists the largest class first and, within a
// class, cells by descending size in steps of an eighth of an octave (longest-processing-time order); class_off[2k]
// and class_off[2k + 1] bound class k. One CTA; shared-memory counters.
constexpr int kGroupSub = 256;
constexpr int kGroupBins = (kGroupClasses + 1) * kGroupSub;

__device__ __forceinline__ int group_bin(int64_t n, const int32_t* caps)
{
    int cls = kGroupClasses;
    for (int k = kGroupClasses - 1; k >= 0; --k)
        if (n <= caps[k]) cls = k;
    const uint64_t x = n > 0 ? (uint64_t)n : 1ull;
    const int lg = 63 - __clzll((unsigned long long)x);
    const int frac = lg >= 3 ? (int)((x >> (lg - 3)) & 7ull) : (int)((x << (3 - lg)) & 7ull);
    int sub = lg * 8 + frac;
    sub = sub > kGroupSub - 1 ? kGroupSub - 1 : sub;
    return (kGroupClasses - cls) * kGroupSub + (kGroupSub - 1 - sub);
}

struct GroupCaps {
    int32_t cap[kGroupClasses];
};

__global__ void __launch_bounds__(kOrderThreads) k_group_order(const int64_t* __restrict__ offsets, int32_t n_cells,
                                                              int32_t S, GroupCaps caps, int32_t* __restrict__ order,
                                                              int32_t* __restrict__ class_off)
{
    __shared__ int hist[kGroupBins];
    __shared__ int warp_tot[kOrderThreads / 32];
    for (int b = threadIdx.x; b < kGroupBins; b += kOrderThreads) hist[b] = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < n_cells; c += kOrderThreads)
        atomicAdd(&hist[group_bin(offsets[(int64_t)(c + 1) * S] - offsets[(int64_t)c * S], caps.cap)], 1);
    __syncthreads();
    // exclusive scan of the bins: each thread owns a run of consecutive bins
    constexpr int kPer = (kGroupBins + kOrderThreads - 1) / kOrderThreads;
    const int lo = threadIdx.x * kPer;
    int local = 0;
    for (int b = lo; b < lo + kPer && b < kGroupBins; ++b) local += hist[b];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    int run = inc - local;
    for (int w = 0; w < warp; ++w) run += warp_tot[w];
    __syncthreads();
    for (int b = lo; b < lo + kPer && b < kGroupBins; ++b) {
        const int x = hist[b];
        hist[b] = run;
        run += x;
    }
    __syncthreads();
    if (threadIdx.x <= kGroupClasses) {
        const int cls = threadIdx.x;
        const int b0 = (kGroupClasses - cls) * kGroupSub;
        class_off[2 * cls] = hist[b0];
        class_off[2 * cls + 1] = b0 + kGroupSub < kGroupBins ? hist[b0 + kGroupSub] : n_cells;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n_cells; c += kOrderThreads) {
        const int b = group_bin(offsets[(int64_t)(c + 1) * S] - offsets[(int64_t)c * S], caps.cap);
        order[atomicAdd(&hist[b], 1)] = c;
    }
}

template <class V, bool REL, int MODE>
const void* kernel_ptr()
{
    return reinterpret_cast<const void*>(&cell_kernel<V, REL, MODE>);
}

const void* select_kernel(bool f32, bool rel, int mode)
{
#define MCC_SEL(V, R)                                   \
    switch (mode) {                                     \
    case kFused: return kernel_ptr<V, R, kFused>();     \
    case kPair: return kernel_ptr<V, R, kPair>();       \
    case kScatter: return kernel_ptr<V, R, kScatter>(); \
    default: return kernel_ptr<V, R, kCorrect>();       \
    }
    if (f32) {
        if (rel) { MCC_SEL(float, true) }
        MCC_SEL(float, false)
    }
    if (rel) { MCC_SEL(double, true) }
    MCC_SEL(double, false)
#undef MCC_SEL
}

}  // namespace

size_t cell_kernel_static_smem(bool f32, bool rel, int mode)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, select_kernel(f32, rel, mode)) != cudaSuccess) return 16384;
    return fa.sharedSizeBytes;
}

cudaError_t set_cell_smem_limit(bool f32, bool rel, int mode, size_t smem)
{
    return cudaFuncSetAttribute(select_kernel(f32, rel, mode), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

int cell_kernel_blocks_per_sm(bool f32, bool rel, int mode, size_t smem)
{
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, select_kernel(f32, rel, mode), kThreads, smem) !=
        cudaSuccess)
        return 0;
    return blocks;
}

cudaError_t launch_step_advance(uint64_t* step, uint64_t by, cudaStream_t st)
{
    k_step_advance<<<1, 32, 0, st>>>(step, by);
    return cudaGetLastError();
}

cudaError_t launch_cell_order(const int64_t* offsets, int32_t n_cells, int32_t S, int32_t* order, cudaStream_t st)
{
    k_cell_order<<<1, kOrderThreads, 0, st>>>(offsets, n_cells, S, order);
    return cudaGetLastError();
}

cudaError_t launch_group_order(const int64_t* offsets, int32_t n_cells, int32_t S, const int32_t* caps,
                               int32_t* order, int32_t* class_off, cudaStream_t st)
{
    GroupCaps gc;
    for (int k = 0; k < kGroupClasses; ++k) gc.cap[k] = caps[k];
    k_group_order<<<1, kOrderThreads, 0, st>>>(offsets, n_cells, S, gc, order, class_off);
    return cudaGetLastError();
}

const void* group_kernel_f32(int cls);
const void* group_kernel_f32rel(int cls);

const void* group_kernel(bool f32, bool rel, int cls)
{
    if (!f32) return nullptr;  // the FP64 path runs on the one-CTA kernel
    return rel ? group_kernel_f32rel(cls) : group_kernel_f32(cls);
}

cudaError_t launch_group(bool f32, bool rel, int cls, const StepArgs& a, int grid, size_t smem, cudaStream_t st)
{
    void* args[] = {const_cast<StepArgs*>(&a)};
    return cudaLaunchKernel(group_kernel(f32, rel, cls), dim3(grid), dim3(32 << cls), args, smem, st);
}

size_t pair_tile_bytes_per_particle() { return kPairTileBytesPerParticle; }

cudaError_t launch_cell(bool f32, bool rel, int mode, const StepArgs& a, int grid, size_t smem, cudaStream_t st)
{
    void* args[] = {const_cast<StepArgs*>(&a)};
    return cudaLaunchKernel(select_kernel(f32, rel, mode), dim3(grid), dim3(kThreads), args, smem, st);
}

}  // namespace mcc
