// Group kernels of the fused collision step on the mixed-precision path: a group of G threads (one CTA) owns one cell
// at a time.
//
// Cells are dispatched by size class: class k holds cells of at most C * 2^k particles and runs with G = 32 * 2^k
// threads, so every class keeps the same shared memory per thread and the GPU the same number of resident warps.
// The smallest class is one warp per cell and synchronises with warp barriers only. The largest class takes the
// largest cell one CTA's shared memory can hold.
//
// Per cell visit the particles are staged in shared memory and the whole step of Algorithm 1 runs there, every
// interaction (a, b) in list order:
//   random permutation(s) (Philox keys, counting sort on the top key bits, insertion sort within a bucket)
//   Takizuka-Abe pairs (Sec. 3.2, Fig. TApairing); inter-species pairs in chunks of G consecutive pairs while
//     N_min >= G (chunks then touch distinct particles), else in rounds of N_min
//   per pair: weighted scattering length (Eq. sab_TA77), TA77 / N97 angle, rotation, rejection of the heavier
//     particle with probability 1 - w_min / w_max
//   momentum shift (Eq. vp_pm), energy violation (Eq. Econs), its split (Eq. DeltaEs), optional weight order,
//   energy-correction pairs (Eqs. vp1_inelastic, vp2_inelastic, vrel_inelastic, U_inelastic; Appendix A) as a
//     prefix sum over the pair caps fE KE_cm, by the group's first warp; failure fallback (Sec. 5.2).
//
// Precision: the velocity state of the cell visit is float-float (hi + lo, ~48 bits) in shared memory and is rounded
// to float once, at write-back. The pair kinematics (relative velocity, scattering length, angle, rotation) run in
// float on that state; every per-cell sum, the coefficients B, Delta E, Delta E_s, the energy-pair caps and their
// prefix sums and the energy pairs run in float-float. Relativistic scatter pairs whose centre-of-momentum frame moves
// with gamma_C > 2, and the energy caps of pairs with a particle at gamma > 2, form their cancelling differences in
// float-float.
//
// Per-species momentum m_s sum w v and energy m_s sum w KE/m are computed once at the cell load and carried through
// the interactions: the scatter changes them, the momentum shift restores the interaction's total (its change to a
// species is B m_s sum w^2), the energy pairs change a species' energy by exactly the U they absorb. The
// pre-interaction sums of Eq. vp_pm and Eq. Econs are therefore the carried values, and no pre-interaction copy of
// the velocities is kept. The fallback of Sec. 5.2 (reset the failing interaction to its pre-interaction state)
// reloads the cell from global memory (unchanged until the write-back) and replays the interactions before the
// failing one, which gives their results bit for bit (every draw and reduction order is fixed), skipping the failed
// one from then on.
#pragma once

#include "mcc_kernels.h"

namespace mcc {
namespace grp {



// Bounds-checked build (-DMCC_DEBUG_BOUNDS): every tile and global index of the group kernels is checked against
// the bound of what it indexes; the first violation latches kErrBounds in the status word and records (source line,
// index, bound, count) in rec[0..3]; the access then uses index 0 instead (results are garbage, memory is safe).
#ifdef MCC_DEBUG_BOUNDS
__device__ __noinline__ inline long long bounds_fail(int* rec, long long i, long long n, int line)
{
    if (rec) {
        if (atomicCAS(rec, 0, line) == 0) {
            rec[1] = (int)i;
            rec[2] = (int)n;
        }
        atomicAdd(rec + 3, 1);
        atomicCAS(rec - 4, 0, kErrBounds);  // the status word sits four words before the record
    }
    return 0;
}
#define CHK(rec, i, n)                                                                                                \
    (((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n))                                        \
         ? (i)                                                                                                        \
         : (decltype(i))bounds_fail((rec), (long long)(i), (long long)(n), __LINE__))
#else
#define CHK(rec, i, n) (i)
#endif

// Phase-timing build (-DMCC_PHASE_CLOCKS): thread 0 of each group reads clock64 at the boundaries of the phases of
// a cell visit and adds the cycles of each phase to A.phase_clk[class * 8 + phase] once per cell (0 load and weight
// order, 1 permutations, 2 pair loop, 3 momentum sums and B, 4 shift and energy sums, 5 energy pairs, 6 write-back).
// The time includes the waits of thread 0 at the group's barriers, so the phases add up to the visit.
struct PhaseClk {
#ifdef MCC_PHASE_CLOCKS
    long long prev;
    long long acc[8];
#endif
};
#ifdef MCC_PHASE_CLOCKS
#define PHASE_MARK(pc, k)                                                                                             \
    do {                                                                                                              \
        if (threadIdx.x == 0) {                                                                                       \
            const long long now_ = clock64();                                                                         \
            (pc).acc[(k)] += now_ - (pc).prev;                                                                        \
            (pc).prev = now_;                                                                                         \
        }                                                                                                             \
    } while (0)
#else
#define PHASE_MARK(pc, k) \
    do {                  \
    } while (0)
#endif

// Tile layout (kGroupBytesPerParticle = 44 bytes per particle): state 24 (three float2 planes), weight 8 (float2),
// scratch 8, permutation 2, weight order 2.

// ----------------------------------------------------------------------------------------------- float-float
__device__ __forceinline__ ff ff_add_f(ff a, float b)
{
    const ff s = ff_two_sum(a.hi, b);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b)
{
    const ff p = ff_two_prod(a.hi, b);
    return ff_fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
// a / b: a first quotient from the hardware reciprocal (a few ulps), then one correction from the remainder
// a - b q1 formed in float-float; relative error about 2^-44 (the sums and energy pairs need ~1e-13).
__device__ __forceinline__ ff ffq_div(ff a, ff b)
{
    const float r = __fdividef(1.f, b.hi);
    const float q1 = a.hi * r;
    const ff bq = ff_mul_f(b, q1);
    const ff rem = ff_sub(a, bq);
    return ff_fast_two_sum(q1, rem.hi * r);
}
// sqrt(a): a first root from the hardware reciprocal square root, then one correction (a - s^2) / (2 s) from the
// residual formed exactly; relative error about 2^-44.
__device__ __forceinline__ ff ffq_sqrt(ff a)
{
    if (!(a.hi > 0.f)) return {0.f, 0.f};
    const float rs = rsqrtf(a.hi);
    const float s = a.hi * rs;
    const ff r = ff_sub(a, ff_two_prod(s, s));
    return ff_fast_two_sum(s, r.hi * (0.5f * rs));
}
__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ ff ff_abs(ff a) { return a.hi < 0.f ? ff_neg(a) : a; }
__device__ __forceinline__ bool ff_is0(ff a) { return a.hi == 0.f; }
__device__ __forceinline__ ff ffk(float v) { return {v, 0.f}; }
__device__ __forceinline__ float ff_round(ff a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ double ff_dbl(ff a) { return (double)a.hi + (double)a.lo; }
// difference of two float-float values rounded to float (the high and low parts subtracted apart, so that close
// velocities keep their relative precision)
__device__ __forceinline__ float ff_diff(ff a, ff b) { return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo)); }
__device__ __forceinline__ ff ff_ld(float2 s) { return {s.x, s.y}; }
__device__ __forceinline__ float2 ff_st(ff x) { return make_float2(x.hi, x.lo); }
__device__ __forceinline__ ff mass_ff(const StepArgs& A, int s) { return {A.m_f[s], A.m_lo[s]}; }

__device__ __forceinline__ ff shx(ff a, int m)
{
    return {__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
}
__device__ __forceinline__ ff shup(ff a, int m)
{
    return {__shfl_up_sync(0xffffffffu, a.hi, m), __shfl_up_sync(0xffffffffu, a.lo, m)};
}
__device__ __forceinline__ ff shidx(ff a, int l)
{
    return {__shfl_sync(0xffffffffu, a.hi, l), __shfl_sync(0xffffffffu, a.lo, l)};
}

// ----------------------------------------------------------------------------------------------- group primitives
template <int G>
__device__ __forceinline__ void gsync()
{
    if (G == 32) __syncwarp();
    else __syncthreads();
}

template <int G>
__device__ __forceinline__ bool gany(bool p)
{
    if (G == 32) return __any_sync(0xffffffffu, p);
    return __syncthreads_or(p) != 0;
}

template <int P>
struct Lg;
template <>
struct Lg<1> {
    static constexpr int v = 0;
};
template <>
struct Lg<2> {
    static constexpr int v = 1;
};
template <>
struct Lg<4> {
    static constexpr int v = 2;
};
template <>
struct Lg<8> {
    static constexpr int v = 3;
};

// Warp reduce-scatter of P (1, 2, 4 or 8) float-float values per lane: rounds with lane masks 16, 8, ... halve the
// set of quantities each lane keeps (the lane with the mask bit set keeps the upper half and adds its partner's
// values of it), then a butterfly on the one kept quantity. Afterwards every lane holds the warp total of quantity
// lane >> (5 - log2 P); the lanes holding one quantity have the same bits (the butterfly's additions are symmetric),
// and the order of additions is fixed.
template <int P>
__device__ __forceinline__ ff warp_rs(ff (&a)[P])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = P / 2, m = 16; h >= 1; h >>= 1, m >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const ff send = up ? a[k] : a[k + h];
            const ff keep = up ? a[k + h] : a[k];
            a[k] = ff_add(keep, shx(send, m));
        }
    }
    ff s = a[0];
#pragma unroll
    for (int m = 16 / P; m >= 1; m >>= 1) s = ff_add(s, shx(s, m));
    return s;
}

template <int G, int P>
struct GRed {
    ff part[P * (G / 32)];
    ff tot[P];
};

// Group sum of P values; every thread receives all P totals in a[] (the same bits in every thread).
template <int G, int P>
__device__ __forceinline__ void gallreduce(ff (&a)[P], GRed<G, 8>& r)
{
    constexpr int SH = 5 - Lg<P>::v;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const ff s = warp_rs<P>(a);
    if (G == 32) {
#pragma unroll
        for (int q = 0; q < P; ++q) a[q] = shidx(s, q << SH);
        return;
    }
    constexpr int W = G / 32;
    if ((lane & ((1 << SH) - 1)) == 0) r.part[(lane >> SH) * W + warp] = s;
    __syncthreads();
    if (warp == 0 && lane < P) {
        ff t = r.part[lane * W];
        for (int w = 1; w < W; ++w) t = ff_add(t, r.part[lane * W + w]);
        r.tot[lane] = t;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < P; ++q) a[q] = r.tot[q];
}

// Group sum of P values for the first warp only (its lanes receive all P totals in a[]); the caller synchronises
// the group before the scratch is used again.
template <int G, int P>
__device__ __forceinline__ void greduce_warp0(ff (&a)[P], GRed<G, 8>& r)
{
    constexpr int SH = 5 - Lg<P>::v;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const ff s = warp_rs<P>(a);
    if (G == 32) {
#pragma unroll
        for (int q = 0; q < P; ++q) a[q] = shidx(s, q << SH);
    } else {
        constexpr int W = G / 32;
        if ((lane & ((1 << SH) - 1)) == 0) r.part[(lane >> SH) * W + warp] = s;
        __syncthreads();
        if (warp == 0) {
            const int q = lane < P ? lane : 0;
            ff t = r.part[q * W];
            for (int w = 1; w < W; ++w) t = ff_add(t, r.part[q * W + w]);
#pragma unroll
            for (int k = 0; k < P; ++k) a[k] = shidx(t, k);
        }
    }
}

// Exclusive prefix sum of one value per lane in lane order over a segment of W (16 or 32) lanes of the warp (lanes
// given by mask), and the segment total. W = WIDTH, or the runtime width when WIDTH is 0 (one copy of the code serves
// both segment widths).
template <int WIDTH>
__device__ __forceinline__ ff seg_scan_excl(ff x, unsigned mask, int width, ff& total)
{
    const int W = WIDTH ? WIDTH : width;
    const int lane = threadIdx.x & (W - 1);
    ff inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        if (o < W) {
            const ff y = {__shfl_up_sync(mask, inc.hi, o, W), __shfl_up_sync(mask, inc.lo, o, W)};
            if (lane >= o) inc = ff_add(y, inc);
        }
    }
    ff exc = {__shfl_up_sync(mask, inc.hi, 1, W), __shfl_up_sync(mask, inc.lo, 1, W)};
    if (lane == 0) exc = {0.f, 0.f};
    total = {__shfl_sync(mask, inc.hi, W - 1, W), __shfl_sync(mask, inc.lo, W - 1, W)};
    return exc;
}

// Exclusive prefix sum of one int per thread in thread order over the group, and the total.
template <int G>
__device__ __forceinline__ int gscan_int(int x, int* scr, int& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    const int exc = inc - x;
    if (G == 32) {
        total = __shfl_sync(0xffffffffu, inc, 31);
        return exc;
    }
    constexpr int W = G / 32;
    if (lane == 31) scr[warp] = inc;
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < W; ++w) {
        const int y = scr[w];
        off += w < warp ? y : 0;
        tot += y;
    }
    __syncthreads();
    total = tot;
    return off + exc;
}

// ----------------------------------------------------------------------------------------------- cell tile
struct GTile {
    float2* v;       // [3][cap]: velocity state (hi, lo), component planes
    float2* w;       // [cap]: weight split into (hi, lo)
    uint64_t* scr;   // [cap]: permutation keys and bucket counters, or 64-bit weight-order keys
    uint16_t* perm;  // [cap]: random permutation of each species segment (cell-local indices)
    uint16_t* rho;   // [cap]: weight-descending order of each species segment (cell-local indices)
    int cap;
    int n;     // particles of the cell in the tile
    int* dbg;  // bounds-check record (MCC_DEBUG_BOUNDS builds)
};

__device__ __forceinline__ GTile gtile(unsigned char* base, int cap, int n, int* dbg)
{
    GTile t;
    t.cap = cap;
    t.n = n;
    t.dbg = dbg;
    t.v = reinterpret_cast<float2*>(base);
    t.w = reinterpret_cast<float2*>(base + 24 * (size_t)cap);
    t.scr = reinterpret_cast<uint64_t*>(base + 32 * (size_t)cap);
    t.perm = reinterpret_cast<uint16_t*>(base + 40 * (size_t)cap);
    t.rho = t.perm + cap;
    return t;
}

template <int G>
struct GShared {
    int off[kMaxSpecies + 1];
    int wmode[kMaxSpecies];  // 0 distinct (rho fixed for the visit), 1 all equal (rho = perm), 2 ties (rho per
                             // interaction), 3 stored in weight order (rho = identity)
    int cell;
    uint32_t step;
    int used_k[kMaxInter];   // energy pairs of interaction k in this visit
    int fail_k[kMaxInter];   // 1 if interaction k failed
    ff P[kMaxSpecies][3];    // carried m_s sum w v per species
    ff E[kMaxSpecies];       // carried m_s sum w KE/m per species
    ff wbar[kMaxSpecies];    // mean weight sum w / N_s (Eq. DeltaEs)
    ff W2m[kMaxSpecies];     // m_s sum w^2 (Eq. vp_pm)
    ff P0[3];                // cell totals at the load (residual output)
    ff E0;
    GRed<G, 8> red;
    ff eres_E[2];   // energy phase results: carried energy of species a, b after their energy pairs
    int eres_i[4];  // pairs used and failure of species a, then of species b
    int sci[G / 32 + 1];
};

// ----------------------------------------------------------------------------------------------- random permutation
// Key of local index q of a side: the Philox block of q/2; bits (r.x, r.y) for even q, (r.z, r.w) for odd q; the
// 64-bit key is (hi << 32 | lo) with its low 20 bits replaced by q. The counting sort uses the top word hi; two
// keys of equal hi (rare) are ordered by the low word, drawn again here.
static __device__ __noinline__ bool key_lo_less(const StepArgs& A, uint32_t step, int c, uint32_t ictr, uint32_t tag,
                                                int qa, int qb)
{
    const uint4 ra = draw_at(A.rng, step, (uint32_t)(qa >> 1), (uint32_t)c, ictr, tag);
    const uint4 rb = draw_at(A.rng, step, (uint32_t)(qb >> 1), (uint32_t)c, ictr, tag);
    const uint32_t la = ((qa & 1) ? ra.w : ra.y) & ~(uint32_t)kPermMask;
    const uint32_t lb = ((qb & 1) ? rb.w : rb.y) & ~(uint32_t)kPermMask;
    return (la | (uint32_t)qa) < (lb | (uint32_t)qb);
}

template <int G>
__device__ void gpermutations(const StepArgs& A, const GTile& t, GShared<G>& sh, int c, uint32_t ictr, int nside,
                              int a0, int na, int b0, int nb, uint32_t step)
{
    uint32_t* key = reinterpret_cast<uint32_t*>(t.scr);  // [cap] top key words by cell-local index
    uint32_t* cnt = key + t.cap;                          // bucket counters
    int lg0 = 0, lg1 = 0;
    while ((2 << lg0) < na) ++lg0;  // 2^lg buckets: half the next power of two (at least one)
    if (nside > 1)
        while ((2 << lg1) < nb) ++lg1;
    const int B0 = 1 << lg0, B1 = nside > 1 ? 1 << lg1 : 0;
    const int L = B0 + B1;  // <= na + nb <= cap
    for (int b = threadIdx.x; b < L; b += G) cnt[CHK(t.dbg, b, t.cap)] = 0;
    gsync<G>();
    // keys of both sides as one range of half-indices h (one Philox block per two particle indices of a side); two
    // blocks per thread and iteration: independent chains for the issue slots
    const int ha = (na + 1) / 2, htot = ha + (nside > 1 ? (nb + 1) / 2 : 0);
    for (int h = threadIdx.x; h < htot; h += 2 * G) {
        const int h2 = h + G;
        const bool sb = h >= ha, sb2 = h2 >= ha;
        const int hl = sb ? h - ha : h, hl2 = sb2 ? h2 - ha : h2;
        const uint4 r = draw_at(A.rng, step, (uint32_t)hl, (uint32_t)c, ictr, sb ? kTagPermB : kTagPermA);
        const uint4 r2 = draw_at(A.rng, step, (uint32_t)hl2, (uint32_t)c, ictr, sb2 ? kTagPermB : kTagPermA);
        {
            const int s0 = sb ? b0 : a0, n = sb ? nb : na, base = sb ? B0 : 0, l = sb ? lg1 : lg0;
            key[CHK(t.dbg, s0 + 2 * hl, t.n)] = r.x;
            atomicAdd(&cnt[CHK(t.dbg, base + (l ? (int)(r.x >> (32 - l)) : 0), t.cap)], 1u);
            if (2 * hl + 1 < n) {
                key[CHK(t.dbg, s0 + 2 * hl + 1, t.n)] = r.z;
                atomicAdd(&cnt[CHK(t.dbg, base + (l ? (int)(r.z >> (32 - l)) : 0), t.cap)], 1u);
            }
        }
        if (h2 < htot) {
            const int s0 = sb2 ? b0 : a0, n = sb2 ? nb : na, base = sb2 ? B0 : 0, l = sb2 ? lg1 : lg0;
            key[CHK(t.dbg, s0 + 2 * hl2, t.n)] = r2.x;
            atomicAdd(&cnt[CHK(t.dbg, base + (l ? (int)(r2.x >> (32 - l)) : 0), t.cap)], 1u);
            if (2 * hl2 + 1 < n) {
                key[CHK(t.dbg, s0 + 2 * hl2 + 1, t.n)] = r2.z;
                atomicAdd(&cnt[CHK(t.dbg, base + (l ? (int)(r2.z >> (32 - l)) : 0), t.cap)], 1u);
            }
        }
    }
    gsync<G>();
    {
        // exclusive scan over both sides' buckets (side b's positions come after side a's na)
        const int chunk = (L + G - 1) / G;
        const int lo = threadIdx.x * chunk, hi = min(L, lo + chunk);
        int local = 0;
        for (int b = lo; b < hi; ++b) local += (int)cnt[CHK(t.dbg, b, t.cap)];
        int total;
        int run = gscan_int<G>(local, sh.sci, total);
        for (int b = lo; b < hi; ++b) {
            const int x = (int)cnt[CHK(t.dbg, b, t.cap)];
            cnt[CHK(t.dbg, b, t.cap)] = (uint32_t)run;
            run += x;
        }
    }
    gsync<G>();
    {
        const int ntot = na + (nside > 1 ? nb : 0);  // both sides as one index range
        for (int qq = threadIdx.x; qq < ntot; qq += G) {
            const bool sb = qq >= na;
            const int q = sb ? qq - na : qq;
            const int s0 = sb ? b0 : a0, base = sb ? B0 : 0, l = sb ? lg1 : lg0, off = sb ? na : 0;
            const uint32_t k = key[CHK(t.dbg, s0 + q, t.n)];
            const int pos = (int)atomicAdd(&cnt[CHK(t.dbg, base + (l ? (int)(k >> (32 - l)) : 0), t.cap)], 1u) - off;
            t.perm[CHK(t.dbg, s0 + pos, t.n)] = (uint16_t)(s0 + q);
        }
    }
    gsync<G>();
    // cnt[b] is now the end of bucket b: order each bucket by the full key (insertion sort)
    for (int bb = threadIdx.x; bb < L; bb += G) {  // both sides' buckets as one range
        const bool sb = bb >= B0;
        const int b = sb ? bb - B0 : bb;
        const int s0 = sb ? b0 : a0, base = sb ? B0 : 0, off = sb ? na : 0;
        const uint32_t tag = sb ? kTagPermB : kTagPermA;
        const int end = (int)cnt[CHK(t.dbg, base + b, t.cap)] - off;
        const int start = b ? (int)cnt[CHK(t.dbg, base + b - 1, t.cap)] - off : 0;
        for (int x = start + 1; x < end; ++x) {
            const int v = t.perm[CHK(t.dbg, s0 + x, t.n)];
            const uint32_t kv = key[CHK(t.dbg, v, t.n)];
            int y = x - 1;
            while (y >= start) {
                const int u = t.perm[CHK(t.dbg, s0 + y, t.n)];
                const uint32_t ku = key[CHK(t.dbg, u, t.n)];
                const bool after = ku > kv || (ku == kv && key_lo_less(A, step, c, ictr, tag, v - s0, u - s0));
                if (!after) break;
                t.perm[CHK(t.dbg, s0 + y + 1, t.n)] = (uint16_t)u;
                --y;
            }
            t.perm[CHK(t.dbg, s0 + y + 1, t.n)] = (uint16_t)v;
        }
    }
    gsync<G>();
}

// ----------------------------------------------------------------------------------------------- weight order
template <int G>
__device__ __forceinline__ void sort_keys(uint64_t* key, int n)
{
    if (n <= kWarpSortMax) {
        if (threadIdx.x < 32) warp_sort_buf(key, n);
    } else {
        block_sort_u64(key, n);
    }
    gsync<G>();
}

// Weight-descending order of each species, once per visit (optional step of Algorithm 1): a segment stored with
// strictly increasing keys needs no order (mode 3; the cell load finds these and passes the others in `need`);
// distinct keys fix the order for the visit (mode 0); all equal
// make it the random permutation (mode 1); partial ties sort it per interaction (mode 2). The species that need a
// sort are sorted at once, species s by warp s mod (G / 32) (segments above the one-warp sort by the whole group,
// one after another).
template <int G>
__device__ __noinline__ void gweight_order(const StepArgs& A, const GTile& t, GShared<G>& sh, int64_t cs, int S,
                                           unsigned need)
{
    constexpr int kWarps = G / 32;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0)
        for (int sp = 0; sp < S; ++sp)
            if (!(need >> sp & 1u)) sh.wmode[sp] = 3;
    if (!need) return;
    for (int sp = 0; sp < S; ++sp) {
        if (!(need >> sp & 1u)) continue;
        const int s0 = sh.off[sp], ns = sh.off[sp + 1] - s0;
        uint64_t* key = t.scr + s0;
        for (int q = threadIdx.x; q < ns; q += G)
            key[CHK(t.dbg, q, ns)] = weight_key(A.w[cs + CHK(t.dbg, s0 + q, t.n)], (uint32_t)q);
    }
    gsync<G>();
    for (int sp = 0; sp < S; ++sp) {  // one-warp sorts, spread over the warps
        const int ns = sh.off[sp + 1] - sh.off[sp];
        if ((need >> sp & 1u) && ns <= kWarpSortMax && warp == sp % kWarps) warp_sort_buf(t.scr + sh.off[sp], ns);
    }
    for (int sp = 0; sp < S; ++sp) {  // larger segments by the whole group
        const int ns = sh.off[sp + 1] - sh.off[sp];
        if ((need >> sp & 1u) && ns > kWarpSortMax) {
            gsync<G>();
            block_sort_u64(t.scr + sh.off[sp], ns);
        }
    }
    gsync<G>();
    for (int sp = 0; sp < S; ++sp) {
        if (!(need >> sp & 1u)) continue;
        const int s0 = sh.off[sp], ns = sh.off[sp + 1] - s0;
        const uint64_t* key = t.scr + s0;
        bool tie = false;
        for (int q = threadIdx.x; q < ns; q += G) {
            t.rho[CHK(t.dbg, s0 + q, t.n)] = (uint16_t)(s0 + (int)(key[CHK(t.dbg, q, ns)] & kPermMask));
            if (q + 1 < ns) tie |= (key[CHK(t.dbg, q, ns)] >> kPermBits) == (key[CHK(t.dbg, q + 1, ns)] >> kPermBits);
        }
        const bool anytie = gany<G>(tie);
        if (threadIdx.x == 0) {
            const bool all_equal = (key[0] >> kPermBits) == (key[CHK(t.dbg, ns - 1, ns)] >> kPermBits);
            sh.wmode[sp] = all_equal ? 1 : (anytie ? 2 : 0);
        }
    }
    gsync<G>();
}

// Energy-pair order of a segment with partially tied weights: the interaction's permutation stably sorted by
// descending weight (keys: weight, rank in the permutation).
template <int G>
__device__ __noinline__ void gtie_order(const StepArgs& A, const GTile& t, int64_t cs, int s0, int ns)
{
    uint64_t* key = t.scr + s0;
    for (int r = threadIdx.x; r < ns; r += G)
        key[CHK(t.dbg, r, ns)] =
            weight_key(A.w[cs + CHK(t.dbg, (int)t.perm[CHK(t.dbg, s0 + r, t.n)], t.n)], (uint32_t)r);
    gsync<G>();
    sort_keys<G>(key, ns);
    for (int m = threadIdx.x; m < ns; m += G)
        t.rho[CHK(t.dbg, s0 + m, t.n)] = t.perm[CHK(t.dbg, s0 + (int)(key[CHK(t.dbg, m, ns)] & kPermMask), t.n)];
    gsync<G>();
}

// ----------------------------------------------------------------------------------------------- scatter
// The heavier particle of an unequal-weight pair moves iff U3 w_max < w_min, decided as the definition states in
// FP64; decided in float with a bound on the float error, and in FP64 only inside it.
__device__ __forceinline__ bool heavy_moves(float wi, float wj, const StepArgs& A, int64_t cs, int i, int j, uint32_t r)
{
    const float p = u23<float>(r) * fmaxf(wi, wj);
    const float wmin = fminf(wi, wj);
    const float x = p - wmin;
    const float tol = 10.0f * 5.9604645e-8f * fmaxf(p, wmin);
    if (x > tol) return false;
    if (x < -tol) return true;
    const double di = A.w[cs + CHK(A.status + 4, i, A.n_total - cs)];
    const double dj = A.w[cs + CHK(A.status + 4, j, A.n_total - cs)];
    return u23<double>(r) * fmax(di, dj) < fmin(di, dj);
}

// Relativistic centre-of-momentum frame from proper velocities ui, uj and their difference du (formed by the caller
// from the float-float state). Same quantities as rel_cm.
template <class V>
__device__ __forceinline__ RelCM<V> rel_cm_du(V c, V ma, V mb, const V ui[3], const V uj[3], const V du[3])
{
    RelCM<V> r;
    const V c2 = c * c;
    const V gi = sqrt((V)1 + (ui[0] * ui[0] + ui[1] * ui[1] + ui[2] * ui[2]) / c2);
    const V gj = sqrt((V)1 + (uj[0] * uj[0] + uj[1] * uj[1] + uj[2] * uj[2]) / c2);
    const V M = ma * gi + mb * gj;
    r.Vx = (ma * ui[0] + mb * uj[0]) / M;
    r.Vy = (ma * ui[1] + mb * uj[1]) / M;
    r.Vz = (ma * ui[2] + mb * uj[2]) / M;
    V du2 = 0, ss = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        du2 += du[d] * du[d];
        ss += du[d] * (ui[d] + uj[d]);
    }
    const V dg = ss / (c2 * (gi + gj));
    V grm1 = (V)0.5 * (du2 / c2 - dg * dg);
    if (grm1 < (V)0) grm1 = 0;
    const V Minv = sqrt((ma + mb) * (ma + mb) + (V)2 * ma * mb * grm1);
    r.gC = M / Minv;
    const V coef_b = r.gC * r.gC / (c2 * (r.gC + (V)1));
    const V k = ma * mb / M;
    const V qx = k * (gj * du[0] - dg * uj[0]);
    const V qy = k * (gj * du[1] - dg * uj[1]);
    const V qz = k * (gj * du[2] - dg * uj[2]);
    const V Vq = r.Vx * qx + r.Vy * qy + r.Vz * qz;
    r.px = qx + coef_b * Vq * r.Vx;
    r.py = qy + coef_b * Vq * r.Vy;
    r.pz = qz + coef_b * Vq * r.Vz;
    const V p2 = r.px * r.px + r.py * r.py + r.pz * r.pz;
    r.pmag = sqrt(p2);
    const V gsa = sqrt((V)1 + p2 / (ma * ma * c2)), gsb = sqrt((V)1 + p2 / (mb * mb * c2));
    r.vrel = r.pmag * ((V)1 / (ma * gsa) + (V)1 / (mb * gsb));
    return r;
}

template <class V>
__device__ __forceinline__ void n97_tab_of(const StepArgs& A, N97Tab<V>& t);
template <>
__device__ __forceinline__ void n97_tab_of<double>(const StepArgs& A, N97Tab<double>& t)
{
    t = {A.n97_f, A.n97_dh};
}
template <>
__device__ __forceinline__ void n97_tab_of<float>(const StepArgs& A, N97Tab<float>& t)
{
    t = {A.n97_f32, A.n97_dh32};
}

// Momentum change dp of particle i of a relativistic pair in its CM frame (rotation of p* through (Theta, phi) and
// the boost of the change back to the lab frame); kappa = the interaction's q^2 q^2 lnL dt / (4 pi eps0^2 dV).
template <class V>
__device__ __forceinline__ void rel_dp(const StepArgs& A, V kappa, const RelCM<V>& cm, V cc, V wf, uint8_t f, V U1,
                                       V U2, V U4, V dp[3])
{
    V s = kappa * wf / (cm.pmag * cm.pmag * cm.vrel);
    if (f & kPairTriplet) s *= (V)0.5;
    V st, omc, sp, cp, dx, dy, dz;
    N97Tab<V> tab;
    n97_tab_of<V>(A, tab);
    sample_angle<V>(A.method, s, U1, U4, st, omc, tab);
    sincospi_v((V)2 * U2, &sp, &cp);
    rotate<V>(cm.px, cm.py, cm.pz, st, omc, cp, sp, dx, dy, dz);
    const V coef_b = cm.gC * cm.gC / (cc * cc * (cm.gC + (V)1));
    const V Vd = cm.Vx * dx + cm.Vy * dy + cm.Vz * dz;
    dp[0] = dx + coef_b * Vd * cm.Vx;
    dp[1] = dy + coef_b * Vd * cm.Vy;
    dp[2] = dz + coef_b * Vd * cm.Vz;
}

// ----------------------------------------------------------------------------------------------- fast relativistic
// Float-float relativistic kinematics for the pairs whose CM frame (gamma_C > 2) or particles (gamma > 2) move fast.
// In float the cancellations of gamma_j du - (gamma_i - gamma_j) u_j (the CM momentum of co-moving particles) and of
// gamma_rel - 1 = (|du|^2 / c^2 - (gamma_i - gamma_j)^2) / 2 lose ~gamma^2 of the precision; formed in float-float
// (about 2^-44) they keep ~2^-37 at gamma = 10, and the rest of the pair's kinematics has no cancellation left.

__device__ __forceinline__ ff ff_dot3(const ff a[3], const ff b[3])
{
    return ff_add(ff_add(ff_mul(a[0], b[0]), ff_mul(a[1], b[1])), ff_mul(a[2], b[2]));
}

// gamma of each particle, the difference du = u1 - u2, |du|^2 and gamma1 - gamma2 = du . (u1 + u2) / (c^2 (g1 + g2)).
struct RelFF {
    ff g1, g2, du[3], du2, dg;
};
__device__ __forceinline__ void rel_ff(ff c2inv, const ff u1[3], const ff u2[3], RelFF& r)
{
    const ff one = ffk(1.f);
    r.g1 = ffq_sqrt(ff_add(one, ff_mul(ff_dot3(u1, u1), c2inv)));
    r.g2 = ffq_sqrt(ff_add(one, ff_mul(ff_dot3(u2, u2), c2inv)));
    ff su[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        r.du[d] = ff_sub(u1[d], u2[d]);
        su[d] = ff_add(u1[d], u2[d]);
    }
    r.du2 = ff_dot3(r.du, r.du);
    r.dg = ffq_div(ff_mul(ff_dot3(r.du, su), c2inv), ff_add(r.g1, r.g2));
}
// gamma_rel - 1 (clamped at 0)
__device__ __forceinline__ ff rel_ff_grm1(const RelFF& r, ff c2inv)
{
    const ff x = ff_sub(ff_mul(r.du2, c2inv), ff_mul(r.dg, r.dg));
    return x.hi > 0.f ? ff{0.5f * x.hi, 0.5f * x.lo} : ffk(0.f);
}

// The CM frame of a relativistic pair (the quantities of rel_cm_du) with the CM momentum formed in float-float.
__device__ __forceinline__ RelCM<float> rel_cm_ff(float cc, ff c2inv, float ma, float mb, const ff ui[3],
                                                  const ff uj[3])
{
    RelFF r;
    rel_ff(c2inv, ui, uj, r);
    RelCM<float> o;
    const float gi = ff_round(r.g1), gj = ff_round(r.g2);
    const float M = ma * gi + mb * gj;
    const float Mr = 1.f / M;
    o.Vx = (ma * ff_round(ui[0]) + mb * ff_round(uj[0])) * Mr;
    o.Vy = (ma * ff_round(ui[1]) + mb * ff_round(uj[1])) * Mr;
    o.Vz = (ma * ff_round(ui[2]) + mb * ff_round(uj[2])) * Mr;
    const float grm1 = ff_round(rel_ff_grm1(r, c2inv));
    const float Minv = sqrtf((ma + mb) * (ma + mb) + 2.f * ma * mb * grm1);
    o.gC = M / Minv;
    const float coef_b = o.gC * o.gC / (cc * cc * (o.gC + 1.f));
    const float k = ma * mb * Mr;
    float q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) q[d] = k * ff_round(ff_sub(ff_mul(r.g2, r.du[d]), ff_mul(r.dg, uj[d])));
    const float Vq = o.Vx * q[0] + o.Vy * q[1] + o.Vz * q[2];
    o.px = q[0] + coef_b * Vq * o.Vx;
    o.py = q[1] + coef_b * Vq * o.Vy;
    o.pz = q[2] + coef_b * Vq * o.Vz;
    const float p2 = o.px * o.px + o.py * o.py + o.pz * o.pz;
    o.pmag = sqrtf(p2);
    const float gsa = sqrtf(1.f + p2 / (ma * ma * cc * cc)), gsb = sqrtf(1.f + p2 / (mb * mb * cc * cc));
    o.vrel = o.pmag * (1.f / (ma * gsa) + 1.f / (mb * gsb));
    return o;
}

// Centre-of-mass kinetic energy of a weighted relativistic pair (weighted masses m1, m2), float-float inputs:
// KE_cm = 2 m1 m2 c^2 (gamma_rel - 1) / (E_cm / c^2 + m1 + m2).
__device__ __forceinline__ float pair_kecm_ff(float cc, ff c2inv, float m1, float m2, const ff u1[3], const ff u2[3])
{
    RelFF r;
    rel_ff(c2inv, u1, u2, r);
    const float grm1 = ff_round(rel_ff_grm1(r, c2inv));
    const float Minv = sqrtf((m1 + m2) * (m1 + m2) + 2.f * m1 * m2 * grm1);
    return 2.f * m1 * m2 * cc * cc * grm1 / (Minv + m1 + m2);
}

// Appendix A energy pair in float-float: p1' = p1 + alpha du, p2' = p2 - alpha du with the pair's total energy
// lowered by U, alpha the root of smaller magnitude of a alpha^2 + b alpha + c0 = 0 (the coefficients of
// energy_pair<., true>, cancellation-free forms). Masses and U are taken in units of m1 + m2 (the quadratic is
// homogeneous of degree one in them: alpha scales with the masses), which keeps b^2 and c0 inside float's range.
// Updates u1, u2 (float-float) in place. Out of line: it runs once per species and interaction (the crossing pair)
// and its code is large.
static __device__ __noinline__ void energy_pair_rel_ff(ff c2inv, ff m1, ff m2, ff u1[3], ff u2[3], ff U)
{
    const ff M12 = ff_add(m1, m2);
    const ff n1 = ffq_div(m1, M12), n2 = ffq_div(m2, M12);
    RelFF r;
    rel_ff(c2inv, u1, u2, r);
    const ff E1 = ff_mul(n1, r.g1), E2 = ff_mul(n2, r.g2);
    const ff Ut = ff_mul(ffq_div(U, M12), c2inv);
    const ff A = ff_sub(ff_add(E1, E2), Ut);
    const ff twoE1mU = ff_sub(ff_add(E1, E1), Ut), twoE2mU = ff_sub(ff_add(E2, E2), Ut);
    const ff n12 = ff_mul(n1, n2);
    ff bdot = ffk(0.f), ptdu = ffk(0.f);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const ff pt = ff_add(ff_mul(n1, u1[d]), ff_mul(n2, u2[d]));
        const ff x12 = ff_mul(n12, ff_sub(ff_mul(r.g2, r.du[d]), ff_mul(r.dg, u2[d])));
        const ff bv = ff_sub(ff_mul(ff_add(A, A), ff_add(x12, ff_mul(Ut, ff_mul(n2, u2[d])))),
                             ff_mul(ff_mul(Ut, twoE1mU), pt));
        bdot = ff_add(bdot, ff_mul(r.du[d], bv));
        ptdu = ff_add(ptdu, ff_mul(pt, r.du[d]));
    }
    const ff a = ff_mul_f(ff_sub(ff_mul(ff_mul(A, A), ff_mul(r.du2, c2inv)), ff_mul(ff_mul(ptdu, ptdu), ff_mul(c2inv, c2inv))),
                          4.f);
    const ff b = ff_mul_f(ff_mul(c2inv, bdot), 4.f);
    // c0 = Ut (2 E1 - Ut) (2 E2 - Ut) (2 E1 + 2 E2 - Ut)
    const ff c0 = ff_mul(ff_mul(Ut, twoE1mU), ff_mul(twoE2mU, ff_add(ff_add(twoE1mU, twoE2mU), Ut)));
    ff disc = ff_sub(ff_mul(b, b), ff_mul_f(ff_mul(a, c0), 4.f));
    if (!(disc.hi > 0.f)) disc = ffk(0.f);
    const ff sq = ffq_sqrt(disc);
    const ff q = ff_mul_f(b.hi >= 0.f ? ff_add(b, sq) : ff_sub(b, sq), -0.5f);
    ff alpha = ffk(0.f);
    if (q.hi != 0.f) {
        alpha = ffq_div(c0, q);
        if (a.hi != 0.f) {
            const ff r1 = ffq_div(q, a);
            if (ff_lt(ff_abs(r1), ff_abs(alpha))) alpha = r1;
        }
    }
    const ff f1 = ffq_div(alpha, n1), f2 = ffq_div(alpha, n2);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        u1[d] = ff_add(u1[d], ff_mul(f1, r.du[d]));
        u2[d] = ff_sub(u2[d], ff_mul(f2, r.du[d]));
    }
}

// Float kinematics of a non-relativistic pair, written for the float path (the same formulas as n97_A_table,
// sample_angle and rotate): one reciprocal per divisor and the hardware square root and reciprocal (a few ulps
// each), so that the angle carries ~1e-7 relative error, within the float kinematics' budget.
__device__ __forceinline__ float fsqrt_fast(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }

__device__ __forceinline__ float n97_A_fast(float s, const N97Tab<float>& tab)
{
    const float z = -expm1f(-s);  // 1 - exp(-s)
    if (!(z < 1.f)) return 0.f;    // exp(-s) underflows: isotropic limit
    if (!(z > 0.f)) return CUDART_INF_F;
    if (s < 1e-3f) return __fdividef(1.f, z);
    if (s > 12.f) {
        const float y = 1.f - z;
        return 3.f * y * (1.f + 0.6f * y * y);
    }
    const float u = (logf(s) - (float)kN97X0) * (float)(1.0 / kN97H);
    int k = (int)u;
    k = k < 0 ? 0 : (k > kN97Nodes - 1 ? kN97Nodes - 1 : k);
    const float t = u - (float)k;
    const float f0 = tab.f[k], f1 = tab.f[k + 1], d0 = tab.dh[k], d1 = tab.dh[k + 1];
    const float t2 = t * t, t3 = t2 * t;
    const float g = (2.f * t3 - 3.f * t2 + 1.f) * f0 + (t3 - 2.f * t2 + t) * d0 + (-2.f * t3 + 3.f * t2) * f1 +
                    (t3 - t2) * d1;  // A s
    return __fdividef(g, s);
}

__device__ __forceinline__ void sample_angle_fast(int method, float s, float U1, float U4, float& sin_t, float& omc,
                                                  const N97Tab<float>& tab)
{
    if (method == 0) {
        const float g = fsqrt_fast(-2.f * logf(U1)) * cospif(2.f * U4);
        const float d = fsqrt_fast(0.5f * s) * g;
        if (fabsf(d) <= 1.f) {
            const float r = __fdividef(1.f, 1.f + d * d);
            sin_t = 2.f * d * r;
            omc = 2.f * d * d * r;
        } else {
            const float tt = __fdividef(1.f, d);
            const float r = __fdividef(1.f, 1.f + tt * tt);
            sin_t = 2.f * tt * r;
            omc = 2.f * r;
        }
        return;
    }
    const float A = n97_A_fast(s, tab);
    float o, q;
    if (A == 0.f) {
        o = 2.f * U1;
        q = 2.f * (1.f - U1);
    } else if (isinf(A)) {
        o = 0.f;
        q = 2.f;
    } else {
        const float rA = __fdividef(1.f, A);
        const float x = -U1 * -expm1f(-2.f * A);
        o = x > -0.5f ? -log1pf(x) * rA : -logf((1.f - U1) + U1 * expf(-2.f * A)) * rA;
        q = o <= 1.f ? 2.f - o : log1pf((1.f - U1) * expm1f(2.f * A)) * rA;
    }
    o = fminf(fmaxf(o, 0.f), 2.f);
    q = fminf(fmaxf(q, 0.f), 2.f);
    omc = o;
    sin_t = fsqrt_fast(o * q);
}

// Rotation of u (magnitude um) through (Theta, phi) about its own direction; returns du = u' - u.
__device__ __forceinline__ void rotate_fast(float ux, float uy, float uz, float um, float sin_t, float omc, float cp,
                                            float sp, float& dx, float& dy, float& dz)
{
    const float up2 = ux * ux + uy * uy;
    if (up2 > 0.f) {
        const float rp = rsqrtf(up2);
        const float uperp = up2 * rp;
        const float ax = ux * rp, ay = uy * rp;
        dx = ax * uz * sin_t * cp - ay * um * sin_t * sp - ux * omc;
        dy = ay * uz * sin_t * cp + ax * um * sin_t * sp - uy * omc;
        dz = -uperp * sin_t * cp - uz * omc;
    } else {
        dx = um * sin_t * cp;
        dy = um * sin_t * sp;
        dz = -uz * omc;
    }
}

// One scattering pair (Algorithm 1 pair loop) on the tile: p is the pair's index in the interaction (the draw's
// counter); wnum = N_min of Eq. sab_TA77 (1 for the N x N pairing); dup > 0 selects duplicity weighting with
// D_ij = dup (s with (w_max / D_ij) N_max).
template <bool REL>
__device__ __forceinline__ void gscatter_pair(const StepArgs& A, const GTile& t, int c, int64_t cs, uint32_t ictr,
                                              const InterConst& ic, int p, int i, int j, uint8_t f, float wnum,
                                              int dup, float nmax, uint32_t step)
{
    const int cap = t.cap;
    ff vi[3], vj[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        vi[d] = ff_ld(t.v[d * cap + CHK(t.dbg, i, t.n)]);
        vj[d] = ff_ld(t.v[d * cap + CHK(t.dbg, j, t.n)]);
    }
    const float2 wi_s = t.w[CHK(t.dbg, i, t.n)], wj_s = t.w[CHK(t.dbg, j, t.n)];
    const float wi = wi_s.x, wj = wj_s.x;
    // w_max N_min of Eq. sab_TA77 with the weights rounded to float, or (w_max / D_ij) N_max
    const float wmax = fmaxf(__fadd_rn(wi_s.x, wi_s.y), __fadd_rn(wj_s.x, wj_s.y));
    const float wf = dup > 0 ? wmax / (float)dup * nmax : wmax * wnum;
    const uint4 r = draw_at(A.rng, step, (uint32_t)p, (uint32_t)c, ictr, kTagScat);
    const float U1 = u23<float>(r.x), U2 = u23<float>(r.y), U4 = u23<float>(r.w);
    float dvi[3], dvj[3], du[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) du[d] = ff_diff(vi[d], vj[d]);
    const float u2 = du[0] * du[0] + du[1] * du[1] + du[2] * du[2];
    if (u2 == 0.f) return;
    if (!REL) {
        const float um = fsqrt_fast(u2);
        float s = __fdividef(ic.kappa_mu2_f * wf, u2 * um);
        if (f & kPairTriplet) s *= 0.5f;
        float st, omc, sp, cp, dx, dy, dz;
        N97Tab<float> tab;
        n97_tab_of<float>(A, tab);
        sample_angle_fast(A.method, s, U1, U4, st, omc, tab);
        sincospif(2.f * U2, &sp, &cp);
        rotate_fast(du[0], du[1], du[2], um, st, omc, cp, sp, dx, dy, dz);
        const float fa = ic.mu_ma_f, fb = ic.mu_mb_f;
        dvi[0] = fa * dx;
        dvi[1] = fa * dy;
        dvi[2] = fa * dz;
        dvj[0] = -fb * dx;
        dvj[1] = -fb * dy;
        dvj[2] = -fb * dz;
    } else {
        const float cc = A.c_f;
        const float ma = A.ma_f[ic.a], mb = A.ma_f[ic.b];
        const float ki[3] = {ff_round(vi[0]), ff_round(vi[1]), ff_round(vi[2])};
        const float kj[3] = {ff_round(vj[0]), ff_round(vj[1]), ff_round(vj[2])};
        const RelCM<float> cm = rel_cm_du<float>(cc, ma, mb, ki, kj, du);
        // a fast-moving CM frame amplifies float rounding by ~gamma_C^2: its CM momentum is formed in float-float
        const RelCM<float> cmx = cm.gC > 2.f ? rel_cm_ff(cc, ff{A.c2inv_f, A.c2inv_lo}, ma, mb, vi, vj) : cm;
        if (!(cmx.pmag > 0.f)) return;
        float dp[3];
        rel_dp<float>(A, ic.kappa_f, cmx, cc, wf, f, U1, U2, U4, dp);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            dvi[d] = dp[d] / ma;
            dvj[d] = -dp[d] / mb;
        }
    }
    bool upd_i = true, upd_j = true;
    if (wi_s.x != wj_s.x || wi_s.y != wj_s.y) {
        const bool moves = heavy_moves(wi, wj, A, cs, i, j, r.z);
        const bool i_heavier = wi > wj || (wi == wj && A.w[cs + CHK(t.dbg, i, t.n)] > A.w[cs + CHK(t.dbg, j, t.n)]);
        if (i_heavier) upd_i = moves;
        else upd_j = moves;
    }
    if (upd_i) {
#pragma unroll
        for (int d = 0; d < 3; ++d) t.v[d * cap + CHK(t.dbg, i, t.n)] = ff_st(ff_add_f(vi[d], dvi[d]));
    }
    if (upd_j) {
#pragma unroll
        for (int d = 0; d < 3; ++d) t.v[d * cap + CHK(t.dbg, j, t.n)] = ff_st(ff_add_f(vj[d], dvj[d]));
    }
}

// Slot k of the order N x N schedule: inter, round k / N_min pairs the smaller population's m = k mod N_min with
// the larger one's (m + round) mod N_max; intra, a round-robin tournament (circle method) over N players plus an
// idle one when N is odd; false for a slot with the idle player.
__device__ __forceinline__ bool gnxn_slot(int na, int nb, bool intra, int k, int& a, int& b)
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

// The pair loop of one interaction. Pairs are processed in rounds of slots that touch distinct particles, rounds in
// order: intra-species, one round of N/2 pairs (an odd count's triplet, pairs 0..2, share particles and run in order
// on thread 0 while the other threads take the remaining pairs); inter-species, chunks of G consecutive pairs while
// N_min >= G (pair k and pair k + N_min share a particle and fall in different chunks), else rounds of N_min; order
// N x N, rounds of the schedule. One call site of the pair code keeps a single copy of it.
template <bool REL, int G>
__device__ __forceinline__ void gscatter(const StepArgs& A, const GTile& t, int c, int64_t cs, uint32_t ictr,
                                         const InterConst& ic, bool intra, int a0, int na, int b0, int nb,
                                         uint32_t step)
{
    const bool nxn = A.pairing == 1;
    const int npairs = intra ? ((na & 1) ? (na + 3) / 2 : na / 2) : (na > nb ? na : nb);
    const int nmin = intra ? na - 1 : (na < nb ? na : nb);
    int total, len;
    if (nxn) {
        len = intra ? (na + (na & 1)) / 2 : nmin;
        total = intra ? (2 * len - 1) * len : na * nb;
    } else {
        total = npairs;
        len = intra ? npairs : (nmin >= G ? G : nmin);
    }
    const bool lead = !nxn && intra && (na & 1);  // the triplet
    const float wnum = nxn ? 1.f : (float)nmin;
    const bool dup = !nxn && !intra && A.weighting == 1;
    int bm = 0;  // r0 mod N_min (inter, order N)
    for (int r0 = 0; r0 < total; r0 += len) {
        const int r1 = r0 + len < total ? r0 + len : total;
        int p, stride, end;
        if (lead) {
            p = threadIdx.x == 0 ? 0 : 3 + (int)threadIdx.x - 1;
            stride = threadIdx.x == 0 ? 1 : G - 1;
            end = threadIdx.x == 0 ? 3 : r1;
        } else {
            p = r0 + (int)threadIdx.x;
            stride = G;
            end = r1;
        }
        for (; p < end; p += stride) {
            int i, j, pm = 0;
            uint8_t f = 0;
            if (nxn) {
                int ia, jb;
                if (!gnxn_slot(na, nb, intra, p, ia, jb)) continue;
                i = t.perm[CHK(t.dbg, a0 + ia, t.n)];
                j = intra ? t.perm[CHK(t.dbg, a0 + jb, t.n)] : t.perm[CHK(t.dbg, b0 + jb, t.n)];
            } else if (intra) {
                if (lead && p < 3) {
                    i = t.perm[CHK(t.dbg, a0 + p, t.n)];
                    j = t.perm[CHK(t.dbg, a0 + (p == 2 ? 0 : p + 1), t.n)];
                    f = kPairTriplet;
                } else {
                    const int q0 = lead ? 2 * p - 3 : 2 * p;
                    i = t.perm[CHK(t.dbg, a0 + q0, t.n)];
                    j = t.perm[CHK(t.dbg, a0 + q0 + 1, t.n)];
                }
            } else {
                pm = bm + (p - r0);
                if (pm >= nmin) pm -= nmin;
                if (na >= nb) {
                    i = t.perm[CHK(t.dbg, a0 + p, t.n)];
                    j = t.perm[CHK(t.dbg, b0 + pm, t.n)];
                } else {
                    i = t.perm[CHK(t.dbg, a0 + pm, t.n)];
                    j = t.perm[CHK(t.dbg, b0 + p, t.n)];
                }
            }
            gscatter_pair<REL>(A, t, c, cs, ictr, ic, p, i, j, f, wnum, dup ? (npairs - 1 - pm) / nmin + 1 : 0,
                               (float)npairs, step);
        }
        gsync<G>();
        if (!nxn && !intra) {
            bm += len;
            if (bm >= nmin) bm -= nmin;
        }
    }
}

// ----------------------------------------------------------------------------------------------- energies
// Kinetic energy of one particle over its weighted mass m_s w: |v|^2 / 2, or relativistic |u|^2 / (gamma + 1).
template <bool REL>
__device__ __forceinline__ ff ke_per_mass(const ff v[3], ff c2inv)
{
    const ff v2 = ff_add(ff_add(ff_mul(v[0], v[0]), ff_mul(v[1], v[1])), ff_mul(v[2], v[2]));
    if (!REL) return ff_mul_f(v2, 0.5f);
    const ff one = ffk(1.f);
    const ff g = ffq_sqrt(ff_add(one, ff_mul(v2, c2inv)));
    return ffq_div(v2, ff_add(g, one));
}

// ----------------------------------------------------------------------------------------------- correction
// Energy-correction loop of one species (Algorithm 1, final loop) by a segment of W lanes (a warp, or a half warp;
// W = WIDTH, or the runtime width when WIDTH is 0): pairs of adjacent particles of the order rho, pass p from offset
// p mod 2, in chunks of W pairs; each pair takes U = fE KE_cm (its cap) up to
// the crossing pair, which takes the remainder of |Delta E_s| (a prefix sum over the caps gives every pair the sum
// of the caps before it). Non-relativistic pairs in float-float (Eqs. vp1_inelastic, vp2_inelastic, vrel_inelastic:
// a capped pair has U / KE_cm = +-fE, so its g - 1 is a constant); relativistic pairs through the Appendix A
// quadratic in float-float. Returns the absorbed energy (signed as D) and adds the pairs used to `used`; done = D was
// absorbed.
template <bool REL, int WIDTH>
__device__ ff energy_loop(const StepArgs& A, const GTile& t, int64_t cs, int s0, int ns, int spc, int mode, ff D,
                          int width, int& used, bool& done)
{
    const int W = WIDTH ? WIDTH : width;
    const int lane = threadIdx.x & (W - 1);
    const unsigned mask = W == 32 ? 0xffffffffu : (0xffffu << (threadIdx.x & 16));
    const int cap = t.cap;
    const ff ms = mass_ff(A, spc);
    const ff fE = {A.fE_f, A.fE_lo};
    const ff gm1p = {A.gm1p_f, A.gm1p_lo};  // sqrt(1 - fE) - 1: a capped pair that loses energy
    const ff gm1n = {A.gm1n_f, A.gm1n_lo};  // sqrt(1 + fE) - 1: a capped pair that gains energy
    const ff c2inv = {A.c2inv_f, A.c2inv_lo};
    const ff Dinit = ff_abs(D);
    ff Dabs = Dinit;
    const bool neg = D.hi < 0.f;
    done = false;
    for (int pass = 0; pass < A.max_corr_passes && !done; ++pass) {
        const int o = pass & 1;
        const int np = (ns - o) / 2;
        ff carry = {0.f, 0.f};
        for (int base = 0; base < np && !done; base += W) {
            const int m = base + lane;
            const bool valid = m < np;
            int i = 0, j = 0;
            ff v1[3], v2[3], vr[3], K = {0.f, 0.f}, capx = {0.f, 0.f}, rw2 = {0.f, 0.f};
            if (valid) {
                const int r1 = o + 2 * m, r2 = r1 + 1;
                i = mode == 3 ? s0 + r1
                              : (mode == 1 ? t.perm[CHK(t.dbg, s0 + r1, t.n)] : t.rho[CHK(t.dbg, s0 + r1, t.n)]);
                j = mode == 3 ? s0 + r2
                              : (mode == 1 ? t.perm[CHK(t.dbg, s0 + r2, t.n)] : t.rho[CHK(t.dbg, s0 + r2, t.n)]);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    v1[d] = ff_ld(t.v[d * cap + CHK(t.dbg, i, t.n)]);
                    v2[d] = ff_ld(t.v[d * cap + CHK(t.dbg, j, t.n)]);
                    vr[d] = ff_sub(v1[d], v2[d]);
                }
                const float2 wi = t.w[CHK(t.dbg, i, t.n)], wj = t.w[CHK(t.dbg, j, t.n)];
                if (!REL) {
                    // K = (1/2) mu_R |v_R|^2 with mu_R = m_s w_1 r_2, r_2 = w_2 / (w_1 + w_2)
                    const ff w1 = {wi.x, wi.y}, w2 = {wj.x, wj.y};
                    rw2 = ffq_div(w2, ff_add(w1, w2));
                    const ff vr2 = ff_add(ff_add(ff_mul(vr[0], vr[0]), ff_mul(vr[1], vr[1])), ff_mul(vr[2], vr[2]));
                    K = ff_mul(ff_mul(ff_mul(ms, w1), rw2), ff{0.5f * vr2.hi, 0.5f * vr2.lo});
                    capx = ff_mul(fE, K);
                } else {
                    const float cc = A.c_f;
                    float k1[3], k2[3], dk[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        k1[d] = ff_round(v1[d]);
                        k2[d] = ff_round(v2[d]);
                        dk[d] = ff_diff(v1[d], v2[d]);
                    }
                    const float Kf = fast_pair(cc, k1, k2)
                                         ? pair_kecm_ff(cc, c2inv, A.m_f[spc] * wi.x, A.m_f[spc] * wj.x, v1, v2)
                                         : pair_kecm_du<float>(cc, A.m_f[spc] * wi.x, A.m_f[spc] * wj.x, k1, k2, dk);
                    K = ffk(Kf);
                    capx = ffk(Kf > 0.f ? A.fE_f * Kf : 0.f);
                }
                if (!(K.hi > 0.f)) capx = {0.f, 0.f};
            }
            ff total;
            const ff excl = ff_add(seg_scan_excl<WIDTH>(capx, mask, W, total), carry);
            if (valid && K.hi > 0.f && ff_lt(excl, Dabs)) {
                const ff rem = ff_sub(Dabs, excl);
                const bool crossing = ff_lt(rem, capx);
                const ff Uabs = crossing ? rem : capx;
                const ff U = neg ? ff_neg(Uabs) : Uabs;
                if (!REL) {
                    // g - 1 = -x / (1 + sqrt(1 - x)), x = U / KE_cm: +-fE for a capped pair (one constant each way)
                    ff gm1 = neg ? gm1n : gm1p;
                    if (crossing) {
                        const ff x = ffq_div(U, K);
                        const ff one = ffk(1.f);
                        gm1 = ff_neg(ffq_div(x, ff_add(one, ffq_sqrt(ff_sub(one, x)))));
                    }
                    const ff f1 = ff_mul(rw2, gm1);  // (m2 / (m1 + m2)) (g - 1)
                    const ff f2 = ff_sub(gm1, f1);  // (m1 / (m1 + m2)) (g - 1)
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        t.v[d * cap + CHK(t.dbg, i, t.n)] = ff_st(ff_add(v1[d], ff_mul(f1, vr[d])));
                        t.v[d * cap + CHK(t.dbg, j, t.n)] = ff_st(ff_sub(v2[d], ff_mul(f2, vr[d])));
                    }
                } else {
                    const float2 wi = t.w[CHK(t.dbg, i, t.n)], wj = t.w[CHK(t.dbg, j, t.n)];
                    energy_pair_rel_ff(c2inv, ff_mul(ms, ff{wi.x, wi.y}), ff_mul(ms, ff{wj.x, wj.y}), v1, v2, U);
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        t.v[d * cap + CHK(t.dbg, i, t.n)] = ff_st(v1[d]);
                        t.v[d * cap + CHK(t.dbg, j, t.n)] = ff_st(v2[d]);
                    }
                }
                ++used;
            }
            carry = ff_add(carry, total);
            if (!ff_lt(carry, Dabs)) done = true;
            __syncwarp(mask);
        }
        if (!done) Dabs = ff_sub(Dabs, carry);
    }
    const ff absorbed = done ? Dinit : ff_sub(Dinit, Dabs);
    return neg ? ff_neg(absorbed) : absorbed;
}

template <bool REL, int WIDTH>
__device__ __noinline__ ff energy_loop_ool(const StepArgs& A, const GTile& t, int64_t cs, int s0, int ns, int spc,
                                           int mode, ff D, int width, int& used, bool& done)
{
    return energy_loop<REL, WIDTH>(A, t, cs, s0, ns, spc, mode, D, width, used, done);
}

// One out-of-line copy of the energy loop serves every call site (a smaller instruction footprint of the cell visit:
// 8% faster than inlined copies); one-warp groups run it on a whole warp or on half warps, with the width at run
// time.
template <bool REL, int G>
__device__ __forceinline__ ff energy_call(const StepArgs& A, const GTile& t, int64_t cs, int s0, int ns, int spc,
                                          int mode, ff D, int width, int& used, bool& done)
{
    return energy_loop_ool<REL, G == 32 ? 0 : 32>(A, t, cs, s0, ns, spc, mode, D, width, used, done);
}

// Moment correction of one interaction (Sec. 4, Appendix A, Sec. 5.2). Returns 1 if the interaction failed under
// the rollback policy (the caller replays the cell without it).
template <bool REL, int G>
__device__ int gcorrect(const StepArgs& A, const GTile& t, GShared<G>& sh, int c, int64_t cs, int k,
                        const InterConst& ic, bool intra, int a0, int na, int b0, int nb, PhaseClk& pc)
{
    const int cap = t.cap;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nside = intra ? 1 : 2;
    const ff zero = {0.f, 0.f};
    const ff ma = mass_ff(A, ic.a), mb = mass_ff(A, ic.b);
    const ff c2inv = {A.c2inv_f, A.c2inv_lo};
    // energy-pair order of tied species (rare), before the energy pairs read it
    if (A.sort_by_weight) {
        if (sh.wmode[ic.a] == 2) gtie_order<G>(A, t, cs, a0, na);
        if (!intra && sh.wmode[ic.b] == 2) gtie_order<G>(A, t, cs, b0, nb);
    }

    // Eq. vp_pm: B = (sum_p m_p v_ps - sum_p m_p v_bs) / sum_p m_p w_p over the interaction's particles, the
    // pre-scatter sum being the carried per-species momentum
    ff B[3], Pa[3], Pb[3];
    {
        ff acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = zero;
        // both species' particles as one index range (fewer partly filled passes over the group)
        const int ntot = na + (nside > 1 ? nb : 0);
#pragma unroll 1  // rolled: a smaller instruction footprint
        for (int q = threadIdx.x; q < ntot; q += G) {
            const bool sb = q >= na;
            const int i = sb ? b0 + (q - na) : a0 + q;
            const float2 ws = t.w[CHK(t.dbg, i, t.n)];
            const ff w = {ws.x, ws.y};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const ff x = ff_mul(w, ff_ld(t.v[d * cap + CHK(t.dbg, i, t.n)]));
                if (sb) acc[3 + d] = ff_add(acc[3 + d], x);
                else acc[d] = ff_add(acc[d], x);
            }
        }
        // one reduction for intra and inter (the species-b slots are zero for intra): one copy of its code
        gallreduce<G, 8>(acc, sh.red);
        const ff inv = ffq_div(ffk(1.f), intra ? sh.W2m[ic.a] : ff_add(sh.W2m[ic.a], sh.W2m[ic.b]));
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            Pa[d] = ff_mul(ma, acc[d]);
            Pb[d] = intra ? zero : ff_mul(mb, acc[3 + d]);
            ff dP = ff_sub(Pa[d], sh.P[ic.a][d]);
            if (!intra) dP = ff_add(dP, ff_sub(Pb[d], sh.P[ic.b][d]));
            B[d] = ff_mul(dP, inv);
        }
    }

    PHASE_MARK(pc, 3);
    // momentum shift v_pm = v_ps - B w_p (Eq. vp_pm) and the post-shift species energies (Eq. DeltaEs)
    ff e2[2] = {zero, zero};
    {
        const int ntot = na + (nside > 1 ? nb : 0);
#pragma unroll 1  // rolled: a smaller instruction footprint
        for (int q = threadIdx.x; q < ntot; q += G) {
            const bool sb = q >= na;
            const int i = sb ? b0 + (q - na) : a0 + q;
            const float2 ws = t.w[CHK(t.dbg, i, t.n)];
            const ff w = {ws.x, ws.y};
            ff v[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                v[d] = ff_sub(ff_ld(t.v[d * cap + CHK(t.dbg, i, t.n)]), ff_mul(B[d], w));
                t.v[d * cap + CHK(t.dbg, i, t.n)] = ff_st(v[d]);
            }
            const ff kp = ff_mul(w, ke_per_mass<REL>(v, c2inv));
            if (sb) e2[1] = ff_add(e2[1], kp);
            else e2[0] = ff_add(e2[0], kp);
        }
    }
    // Energy pairs: one species (intra, or any interaction under a fail policy other than rollback) on the first
    // warp; the two species of an inter-species interaction under the rollback policy at once, on the two half
    // warps (one-warp groups) or the first two warps. Their pairs are disjoint; the oracle runs species b only if
    // species a did not fail, and a failed interaction is replayed without it, so only the pair count of species b
    // is dropped when species a fails.
    const bool both = !intra && A.fail_policy == 0;
    if (!both || G == 32) greduce_warp0<G, 2>(e2, sh.red);  // intra: e2[1] is zero
    else gallreduce<G, 2>(e2, sh.red);
    PHASE_MARK(pc, 4);
    // unit 0 runs species a (and b when not both), unit 1 species b
    const int unit = both ? (G == 32 ? lane >> 4 : warp) : (warp == 0 ? 0 : 2);
    if (unit < 2) {
        const ff Epm0 = ff_mul(ma, e2[0]), Epm1 = intra ? zero : ff_mul(mb, e2[1]);
        // Eq. Econs: Delta E = E_pm - E_bs, the pre-interaction energies carried; Eq. DeltaEs: its split in proportion
        // to mean weight times post-shift energy. A species with fewer than two particles cannot take a share; no
        // eligible species with Delta E != 0 fails. |Delta E_s| at or below 2^-47 of the species' post-shift energy
        // counts as zero (rounding noise).
        ff dE = ff_sub(Epm0, sh.E[ic.a]);
        if (!intra) dE = ff_add(dE, ff_sub(Epm1, sh.E[ic.b]));
        ff D0 = dE, D1 = zero;
        int fail = 0;
        if (!intra) {
            const bool can0 = na >= 2, can1 = nb >= 2;
            if (can0 && can1) {
                const ff wa = ff_mul(sh.wbar[ic.a], Epm0), wb = ff_mul(sh.wbar[ic.b], Epm1);
                const ff den = ff_add(wa, wb);
                if (den.hi > 0.f) {
                    D0 = ff_mul(ffq_div(wa, den), dE);
                    D1 = ff_sub(dE, D0);
                } else if (!ff_is0(dE)) {
                    fail = 1;
                }
            } else if (can0) {
                D0 = dE;
            } else if (can1) {
                D0 = zero;
                D1 = dE;
            } else if (!ff_is0(dE)) {
                fail = 1;
            }
        }
        if (fabsf(D0.hi) <= 0x1p-47f * Epm0.hi) D0 = zero;
        if (fabsf(D1.hi) <= 0x1p-47f * Epm1.hi) D1 = zero;
        ff Eaft0 = Epm0, Eaft1 = Epm1;
        int used0 = 0, used1 = 0, fail0 = 0, fail1 = 0;
        if (both) {
            // this unit's species
            const int side = unit;
            const ff Ds = side ? D1 : D0;
            if (!fail && !ff_is0(Ds)) {
                bool done;
                const int s0 = side ? b0 : a0, ns = side ? nb : na, spc = side ? ic.b : ic.a;
                const int mode = A.sort_by_weight ? sh.wmode[spc] : 1;
                int u = 0;
                const ff ab = energy_call<REL, G>(A, t, cs, s0, ns, spc, mode, Ds, G == 32 ? 16 : 32, u, done);
                if (side) {
                    Eaft1 = ff_sub(Eaft1, ab);
                    used1 = u;
                    fail1 = !done;
                } else {
                    Eaft0 = ff_sub(Eaft0, ab);
                    used0 = u;
                    fail0 = !done;
                }
            }
        } else {
            // energy-correction pairs, species a then b
            if (!fail && !ff_is0(D0)) {
                bool done;
                const int mode = A.sort_by_weight ? sh.wmode[ic.a] : 1;
                Eaft0 = ff_sub(Eaft0, energy_call<REL, G>(A, t, cs, a0, na, ic.a, mode, D0, 32, used0, done));
                if (!done) fail0 = 1;
            }
            if (!fail && !fail0 && !intra && !ff_is0(D1)) {
                bool done;
                const int mode = A.sort_by_weight ? sh.wmode[ic.b] : 1;
                Eaft1 = ff_sub(Eaft1, energy_call<REL, G>(A, t, cs, b0, nb, ic.b, mode, D1, 32, used1, done));
                if (!done) fail1 = 1;
            }
        }
        // per unit: lane totals of the pair counts, then the unit's first lane publishes its species' results
        const unsigned mask = (both && G == 32) ? (0xffffu << (threadIdx.x & 16)) : 0xffffffffu;
        const int width = (both && G == 32) ? 16 : 32;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            if (o < width) {
                used0 += __shfl_xor_sync(mask, used0, o);
                used1 += __shfl_xor_sync(mask, used1, o);
            }
        }
        __syncwarp(mask);
        if ((lane & (width - 1)) == 0) {
            if (unit == 0) {
                sh.eres_E[0] = Eaft0;
                sh.eres_i[0] = used0;
                sh.eres_i[1] = fail | fail0;
                if (!both) {
                    sh.eres_E[1] = Eaft1;
                    sh.eres_i[2] = used1;
                    sh.eres_i[3] = fail1;
                }
            } else {
                sh.eres_E[1] = Eaft1;
                sh.eres_i[2] = used1;
                sh.eres_i[3] = fail1;
            }
        }
    }
    gsync<G>();
    // every thread reads the outcome; thread 0 updates the carried sums, which are read again only after the next
    // interaction's barriers (so no barrier closes this one)
    const int fa = sh.eres_i[1], fb = sh.eres_i[3];
    const int fail = fa | fb;
    if (threadIdx.x == 0) {
        sh.used_k[k] = sh.eres_i[0] + (fa ? 0 : sh.eres_i[2]);
        sh.fail_k[k] = fail;
        sh.E[ic.a] = sh.eres_E[0];
#pragma unroll
        for (int d = 0; d < 3; ++d) sh.P[ic.a][d] = ff_sub(Pa[d], ff_mul(B[d], sh.W2m[ic.a]));
        if (!intra) {
            sh.E[ic.b] = sh.eres_E[1];
#pragma unroll
            for (int d = 0; d < 3; ++d) sh.P[ic.b][d] = ff_sub(Pb[d], ff_mul(B[d], sh.W2m[ic.b]));
        }
        if (fail && A.fail_policy == 2) latch(A.status, kErrCorrectionFailed);
    }
    PHASE_MARK(pc, 5);
    return (fail && A.fail_policy == 0) ? 1 : 0;
}

// ----------------------------------------------------------------------------------------------- cell visit
// Load the cell into the tile; per-species sums (w, m w^2, momentum, energy) and the weight-order modes.
template <bool REL, int G>
__device__ __forceinline__ void gload(const StepArgs& A, const GTile& t, GShared<G>& sh, int64_t cs, int S)
{
    const int cap = t.cap;
    const float* gv[3] = {reinterpret_cast<const float*>(A.vx), reinterpret_cast<const float*>(A.vy),
                          reinterpret_cast<const float*>(A.vz)};
    const ff zero = {0.f, 0.f};
    const ff c2inv = {A.c2inv_f, A.c2inv_lo};
    ff tot[4] = {zero, zero, zero, zero};
    const bool order = A.correct && A.sort_by_weight;
    unsigned need = 0;  // species whose segment is not stored in strictly descending weight
    for (int sp = 0; sp < S; ++sp) {
        const int s0 = sh.off[sp], ns = sh.off[sp + 1] - s0;
        ff acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = zero;
        float unordered = 0.f;  // neighbours out of the stored weight order (counted in slot 6 of the reduction)
#pragma unroll 1  // rolled: a smaller instruction footprint
        for (int q = threadIdx.x; q < ns; q += G) {
            const int i = s0 + q;
            const double wd = A.w[cs + CHK(t.dbg, i, t.n)];
            if (order && q + 1 < ns && weight_key(wd, 0) >= weight_key(A.w[cs + CHK(t.dbg, i + 1, t.n)], 0))
                unordered += 1.f;
            const float2 ws = split_weight(wd);
            t.w[CHK(t.dbg, i, t.n)] = ws;
            const ff w = {ws.x, ws.y};
            ff v[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                v[d] = ffk(gv[d][cs + CHK(t.dbg, i, t.n)]);
                t.v[d * cap + CHK(t.dbg, i, t.n)] = ff_st(v[d]);
                acc[2 + d] = ff_add(acc[2 + d], ff_mul(w, v[d]));
            }
            acc[0] = ff_add(acc[0], w);
            acc[1] = ff_add(acc[1], ff_mul(w, w));
            acc[5] = ff_add(acc[5], ff_mul(w, ke_per_mass<REL>(v, c2inv)));
        }
        acc[6] = ffk(unordered);
        gallreduce<G, 8>(acc, sh.red);
        if (acc[6].hi > 0.f) need |= 1u << sp;
        const ff m = mass_ff(A, sp);
        const ff Pm[3] = {ff_mul(m, acc[2]), ff_mul(m, acc[3]), ff_mul(m, acc[4])};
        const ff Em = ff_mul(m, acc[5]);
        if (threadIdx.x == 0) {
            sh.wbar[sp] = ns > 0 ? ffq_div(acc[0], ffk((float)ns)) : zero;
            sh.W2m[sp] = ff_mul(m, acc[1]);
            sh.P[sp][0] = Pm[0];
            sh.P[sp][1] = Pm[1];
            sh.P[sp][2] = Pm[2];
            sh.E[sp] = Em;
        }
        tot[0] = ff_add(tot[0], Pm[0]);
        tot[1] = ff_add(tot[1], Pm[1]);
        tot[2] = ff_add(tot[2], Pm[2]);
        tot[3] = ff_add(tot[3], Em);
    }
    if (threadIdx.x == 0) {
        sh.P0[0] = tot[0];
        sh.P0[1] = tot[1];
        sh.P0[2] = tot[2];
        sh.E0 = tot[3];
    }
    gsync<G>();
    if (order) gweight_order<G>(A, t, sh, cs, S, need);
}

template <bool REL, int G>
__device__ void gcell(const StepArgs& A, int c, unsigned char* dyn, GShared<G>& sh)
{
    const int S = A.S;
    const int64_t cs = A.offsets[(int64_t)c * S];
    const int n = (int)(A.offsets[(int64_t)(c + 1) * S] - cs);
    if (n > A.gcap || n > A.max_cell) {
        if (threadIdx.x == 0) latch(A.status, kErrBounds);
        return;
    }
    const GTile t = gtile(dyn, A.gcap, n, A.status ? A.status + 4 : nullptr);
    if ((int)threadIdx.x <= S) sh.off[threadIdx.x] = (int)(A.offsets[(int64_t)c * S + threadIdx.x] - cs);
    for (int k = threadIdx.x; k < kMaxInter; k += G) {
        sh.used_k[k] = 0;
        sh.fail_k[k] = 0;
    }
    gsync<G>();
    PhaseClk pc;
#ifdef MCC_PHASE_CLOCKS
    pc.prev = clock64();
#pragma unroll
    for (int q = 0; q < 8; ++q) pc.acc[q] = 0;
#endif
    const uint32_t step = sh.step;
    // one call site of the cell load: the Sec. 5.2 fallback (an interaction failed) restarts the visit from the stored
    // state, skipping the failed interactions
    uint64_t skip = 0;
    for (bool again = true; again;) {
        again = false;
        gload<REL, G>(A, t, sh, cs, S);
        PHASE_MARK(pc, 0);
        for (int k = 0; k < A.n_inter; ++k) {
            if ((skip >> k) & 1ull) continue;
            const InterConst& ic = A.ic[k];
            const bool intra = ic.a == ic.b;
            const int a0 = sh.off[ic.a], na = sh.off[ic.a + 1] - a0;
            const int b0 = sh.off[ic.b], nb = sh.off[ic.b + 1] - b0;
            const bool active = intra ? (na >= 2) : (na > 0 && nb > 0);
            if (!active) continue;
            const uint32_t ictr = (uint32_t)(A.inter_base + k);
            gpermutations<G>(A, t, sh, c, ictr, intra ? 1 : 2, a0, na, b0, nb, step);
            PHASE_MARK(pc, 1);
            gscatter<REL, G>(A, t, c, cs, ictr, ic, intra, a0, na, b0, nb, step);
            PHASE_MARK(pc, 2);
            if (!A.correct) continue;
            if (gcorrect<REL, G>(A, t, sh, c, cs, k, ic, intra, a0, na, b0, nb, pc)) {
                skip |= 1ull << k;
                again = true;
                break;
            }
        }
    }
    // write back: the float-float state rounded once to float
    const int cap = t.cap;
    float* gv[3] = {reinterpret_cast<float*>(A.vx), reinterpret_cast<float*>(A.vy), reinterpret_cast<float*>(A.vz)};
#pragma unroll 1  // rolled: a smaller instruction footprint
    for (int i = threadIdx.x; i < n; i += G) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
            gv[d][cs + CHK(t.dbg, i, t.n)] = ff_round(ff_ld(t.v[d * cap + CHK(t.dbg, i, t.n)]));
    }
    if (A.resid) {
        // conservation of the exact state before the store: |P - P0| / sum m w |v| and |E - E0| / E0 per cell
        const ff zero = {0.f, 0.f};
        const ff c2inv = {A.c2inv_f, A.c2inv_lo};
        ff tot[4] = {zero, zero, zero, zero};
        ff amag = zero;
        for (int sp = 0; sp < S; ++sp) {
            const int s0 = sh.off[sp], ns = sh.off[sp + 1] - s0;
            ff acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = zero;
            for (int q = threadIdx.x; q < ns; q += G) {
                const int i = s0 + q;
                const float2 ws = t.w[CHK(t.dbg, i, t.n)];
                const ff w = {ws.x, ws.y};
                ff v[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    v[d] = ff_ld(t.v[d * cap + CHK(t.dbg, i, t.n)]);
                    acc[d] = ff_add(acc[d], ff_mul(w, v[d]));
                }
                acc[3] = ff_add(acc[3], ff_mul(w, ke_per_mass<REL>(v, c2inv)));
                const float vx = ff_round(v[0]), vy = ff_round(v[1]), vz = ff_round(v[2]);
                acc[4] = ff_add_f(acc[4], ws.x * sqrtf(vx * vx + vy * vy + vz * vz));
            }
            gallreduce<G, 8>(acc, sh.red);
            const ff m = mass_ff(A, sp);
#pragma unroll
            for (int q = 0; q < 4; ++q) tot[q] = ff_add(tot[q], ff_mul(m, acc[q]));
            amag = ff_add(amag, ff_mul(m, acc[4]));
        }
        if (threadIdx.x == 0) {
            double dp = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) dp = fmax(dp, fabs(ff_dbl(ff_sub(tot[d], sh.P0[d]))));
            const double am = ff_dbl(amag);
            A.resid[2 * (int64_t)c] = am > 0.0 ? dp / am : dp;
            const double e0 = ff_dbl(sh.E0);
            const double de = fabs(ff_dbl(ff_sub(tot[3], sh.E0)));
            A.resid[2 * (int64_t)c + 1] = e0 > 0.0 ? de / e0 : de;
        }
    }
    if (threadIdx.x == 0) {
        int u = 0, f = 0;
        for (int k = 0; k < A.n_inter; ++k) {
            u += sh.used_k[k];
            f += sh.fail_k[k];
        }
        if (A.corr_pairs) A.corr_pairs[c] += u;
        if (A.fail_count) A.fail_count[c] += f;
    }
    PHASE_MARK(pc, 6);
#ifdef MCC_PHASE_CLOCKS
    if (threadIdx.x == 0 && A.phase_clk) {
#pragma unroll
        for (int q = 0; q < 7; ++q)
            atomicAdd(A.phase_clk + 8 * A.gcls + q, (unsigned long long)pc.acc[q]);
        atomicAdd(A.phase_clk + 8 * A.gcls + 7, 1ull);  // cells
    }
#endif
}

template <bool REL, int G>
__global__ void __launch_bounds__(G, kGroupWarpsPerSm / (G / 32) > 0 ? kGroupWarpsPerSm / (G / 32) : 1)
    group_kernel(const __grid_constant__ StepArgs A)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ GShared<G> sh;
    const int cls = A.gcls;
    const int beg = A.class_off[2 * cls], end = A.class_off[2 * cls + 1];
    if (threadIdx.x == 0) sh.step = A.step_dev ? (uint32_t)(*A.step_dev + A.step_add) : A.rng.step;
    for (;;) {
        if (threadIdx.x == 0) {
            const int q = beg + atomicAdd(&A.queues[cls], 1);
            sh.cell = q < end ? A.order[CHK(A.status ? A.status + 4 : nullptr, q, A.n_cells)] : -1;
        }
        gsync<G>();
        const int c = sh.cell;
        if (c < 0) break;
        gcell<REL, G>(A, c, dyn, sh);
        gsync<G>();
    }
}

template <bool REL, int G>
const void* group_kernel_ptr()
{
    return reinterpret_cast<const void*>(&group_kernel<REL, G>);
}

}  // namespace grp
}  // namespace mcc
