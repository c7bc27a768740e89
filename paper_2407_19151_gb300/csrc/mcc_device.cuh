// Device building blocks of the collision step: counter-based random numbers, float-float accumulators,
// block-wide reductions / scans / sorts in shared memory, the TA77 and N97 angle samplers, the rotation of the
// relative velocity, relativistic centre-of-momentum kinematics and the inelastic energy-correction pair.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

namespace mcc {

#ifndef MCC_THREADS
#define MCC_THREADS 128
#endif
constexpr int kThreads = MCC_THREADS;  // threads cooperating on one cell (one CTA)
constexpr int kWarps = kThreads / 32;
constexpr int kMaxSpecies = 8;
constexpr int kMaxInter = kMaxSpecies * (kMaxSpecies + 1) / 2;
constexpr int kPermBits = 20;
constexpr uint64_t kPermMask = (1ull << kPermBits) - 1ull;
constexpr uint32_t kTagPermA = 1u, kTagPermB = 2u, kTagScat = 3u;
constexpr uint8_t kPairTriplet = 1u;

// Device status codes (mirror mcc_status).
constexpr int kErrCorrectionFailed = -5;
constexpr int kErrBounds = -6;
constexpr int kErrTooLarge = -7;

__device__ __forceinline__ void latch(int* status, int code)
{
    if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------------------------------------------
// Philox-4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 -> 64-bit products, the high halves xored with
// the other words and the round key, the key advanced by two Weyl increments between rounds.
// ---------------------------------------------------------------------------------------------------------------
struct RngKey {
    uint32_t k0, k1, step;
    uint32_t cell_base;  // global id of local cell 0
};

__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                               uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// One Philox block for (index, cell, step, interaction, purpose).
__device__ __forceinline__ uint4 draw(const RngKey& k, uint32_t index, uint32_t cell, uint32_t inter,
                                      uint32_t purpose)
{
    return philox4x32_10(index, cell + k.cell_base, k.step, (inter << 8) | purpose, k.k0, k.k1);
}

// The same block with the step index given apart (read from device memory by the caller when it keeps it there).
__device__ __forceinline__ uint4 draw_at(const RngKey& k, uint32_t step, uint32_t index, uint32_t cell, uint32_t inter,
                                         uint32_t purpose)
{
    return philox4x32_10(index, cell + k.cell_base, step, (inter << 8) | purpose, k.k0, k.k1);
}

// Uniform on (0, 1): ((r >> 9) + 1/2) 2^-23, exact in float and double.
template <class V>
__device__ __forceinline__ V u23(uint32_t r)
{
    return ((V)(r >> 9) + (V)0.5) * (V)(1.0 / 8388608.0);
}

// Permutation key of local index i: 44 random bits above the 20-bit index (distinct keys).
__device__ __forceinline__ uint64_t perm_key(const RngKey& k, uint32_t cell, uint32_t inter, uint32_t side,
                                             uint32_t i)
{
    const uint4 b = draw(k, i >> 1, cell, inter, side ? kTagPermB : kTagPermA);
    const uint32_t hi = (i & 1u) ? b.z : b.x;
    const uint32_t lo = (i & 1u) ? b.w : b.y;
    return ((((uint64_t)hi << 32) | (uint64_t)lo) & ~kPermMask) | (uint64_t)i;
}

// Weight-descending order key: inverted IEEE bits of the (positive) weight truncated to 44 bits, then the rank in
// the random permutation, so that weights equal to 2^-32 relative keep the random order.
__device__ __forceinline__ uint64_t weight_key(double w, uint32_t rank)
{
    const uint64_t b = (uint64_t)__double_as_longlong(w);
    return (~b & ~kPermMask) | (uint64_t)rank;
}

// ---------------------------------------------------------------------------------------------------------------
// Float-float ("double-single") accumulation for the mixed-precision path: error-free sum (Knuth) and product
// (FMA) transformations, giving ~48-bit sums of float terms without the FP64 pipe.
// ---------------------------------------------------------------------------------------------------------------
struct __align__(8) ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ ff ff_two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const ff s = ff_two_sum(a.hi, b.hi);
    const float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return ff_fast_two_sum(s.hi, lo);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    ff p = ff_two_prod(a.hi, b.hi);
    const float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return ff_fast_two_sum(p.hi, lo);
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// a / b: float quotient of the high parts, then one correction from the float-float remainder a - q b.
__device__ __forceinline__ ff ff_div(ff a, ff b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const ff r = ff_sub(a, ff_mul(b, {q1, 0.f}));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return ff_fast_two_sum(q1, q2);
}

__device__ __forceinline__ ff ff_from_double(double x)
{
    const float hi = __double2float_rn(x);
    const float lo = __double2float_rn(x - (double)hi);
    return {hi, lo};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Split a positive normal double w into hi + lo floats with integer operations only (no FP64 pipe): hi carries the
// sign, exponent and top 23 mantissa bits (truncated), lo the remaining 29 mantissa bits rounded to 24. The pair
// represents w to about 2^-53 relative. Valid for 2^-75 < |w| < 2^127; outside that range falls back to converts.
__device__ __forceinline__ float2 split_weight(double w)
{
    const uint64_t b = (uint64_t)__double_as_longlong(w);
    const uint32_t top = (uint32_t)(b >> 32);
    const int e = (int)((top >> 20) & 0x7FFu);
    if (e < 949 || e > 1023 + 126) {
        const float hi = __double2float_rz(w);
        return make_float2(hi, __double2float_rn(w - (double)hi));
    }
    const uint32_t sign = top & 0x80000000u;
    const uint64_t mant = b & ((1ull << 52) - 1ull);
    const float hi = __uint_as_float(sign | ((uint32_t)(e - 1023 + 127) << 23) | (uint32_t)(mant >> 29));
    const uint32_t mlo = (uint32_t)(mant & 0x1FFFFFFFull);
    const float scale = __uint_as_float((uint32_t)(e - 1075 + 127) << 23);  // 2^(e - 1075), normal for e > 948
    const float lo = __uint_as_float(sign | __float_as_uint(__uint2float_rn(mlo) * scale));
    return make_float2(hi, lo);
}

// Accumulator type per precision: double for the FP64 path, float-float for the mixed path.
template <class V>
struct Acc;

template <>
struct Acc<double> {
    double x;
    __device__ __forceinline__ static Acc zero() { return {0.0}; }
    __device__ __forceinline__ void add(double t) { x += t; }
    __device__ __forceinline__ void add(Acc o) { x += o.x; }
    __device__ __forceinline__ double value() const { return x; }
    __device__ __forceinline__ Acc shfl_xor(int m) const { return {__shfl_xor_sync(0xffffffffu, x, m)}; }
};

template <>
struct Acc<float> {
    ff x;
    __device__ __forceinline__ static Acc zero() { return {{0.f, 0.f}}; }
    __device__ __forceinline__ void add(float t)
    {
        const ff s = ff_two_sum(x.hi, t);
        x = ff_fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
    }
    __device__ __forceinline__ void add(ff t) { x = ff_add(x, t); }
    __device__ __forceinline__ void add(Acc o) { x = ff_add(x, o.x); }
    __device__ __forceinline__ double value() const { return ff_to_double(x); }
    __device__ __forceinline__ Acc shfl_xor(int m) const
    {
        return {{__shfl_xor_sync(0xffffffffu, x.hi, m), __shfl_xor_sync(0xffffffffu, x.lo, m)}};
    }
};

// Block-wide sum of M accumulators in a fixed order (reproducible). Each thread parks its M partial sums in shared
// memory; warp w then reduces quantities w, w + kWarps, ... (its lanes add kThreads/32 partials each, then a warp
// tree). The M sums are left in out[m] (shared, accumulator type) for the caller to read after the final barrier.
// scratch: shared, M * kThreads * sizeof(Acc<V>) bytes. Must be called by all threads of the block.
template <class V, int M>
__device__ __forceinline__ void block_sum(Acc<V> (&a)[M], Acc<V>* scratch, Acc<V>* out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int m = 0; m < M; ++m) scratch[m * kThreads + threadIdx.x] = a[m];
    __syncthreads();
    for (int m = warp; m < M; m += kWarps) {
        Acc<V> s = scratch[m * kThreads + lane];
#pragma unroll
        for (int k = 1; k < kThreads / 32; ++k) s.add(scratch[m * kThreads + lane + 32 * k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s.add(s.shfl_xor(o));
        if (lane == 0) out[m] = s;
    }
    __syncthreads();
}

// Block-wide exclusive prefix sum of one value per thread (thread order), and the total.
// scratch: shared, kWarps + 1 values of T. Must be called by all threads.
template <class T>
__device__ __forceinline__ T block_exclusive_scan(T x, T* scratch, T& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    T exc = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) exc = T(0);
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T s = lane < kWarps ? scratch[lane] : T(0);
        T si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        T se = __shfl_up_sync(0xffffffffu, si, 1);  // exclusive warp offsets
        if (lane == 0) se = T(0);
        if (lane < kWarps) scratch[lane] = se;
        if (lane == kWarps - 1) scratch[kWarps] = si;
    }
    __syncthreads();
    const T res = scratch[warp] + exc;
    total = scratch[kWarps];
    __syncthreads();
    return res;
}

__device__ __forceinline__ int block_sum_int(int x, int* scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) scratch[warp] = x;
    __syncthreads();
    int s = 0;
    for (int w = 0; w < kWarps; ++w) s += scratch[w];
    __syncthreads();
    return s;
}

// Ascending sort of n 64-bit keys in place (shared or global memory), block-wide. Bitonic network in its "flip"
// form: every comparator puts the minimum at the lower index, so positions >= n act as +infinity and are skipped.
__device__ __forceinline__ void cmpx(uint64_t* a, int lo, int hi)
{
    const uint64_t x = a[lo], y = a[hi];
    if (x > y) {
        a[lo] = y;
        a[hi] = x;
    }
}

__device__ __forceinline__ void block_sort_u64(uint64_t* a, int n)
{
    if (n < 2) return;
    int logP = 0;
    while ((1 << logP) < n) ++logP;
    const int half_work = 1 << (logP - 1);
    for (int lg = 1; lg <= logP; ++lg) {
        const int size = 1 << lg, hmask = (size >> 1) - 1;
        for (int i = threadIdx.x; i < half_work; i += blockDim.x) {
            const int pos = i & hmask;
            const int base = (i >> (lg - 1)) << lg;
            const int lo = base + pos, hi = base + size - 1 - pos;
            if (hi < n) cmpx(a, lo, hi);
        }
        __syncthreads();
        for (int ls = lg - 2; ls >= 0; --ls) {
            const int stride = 1 << ls;
            for (int i = threadIdx.x; i < half_work; i += blockDim.x) {
                const int lo = ((i >> ls) << (ls + 1)) + (i & (stride - 1));
                const int hi = lo + stride;
                if (hi < n) cmpx(a, lo, hi);
            }
            __syncthreads();
        }
    }
}

// Same network over int32 keys (binning: segment entries sorted by particle index).
__device__ __forceinline__ void block_sort_i32(int32_t* a, int n)
{
    if (n < 2) return;
    int logP = 0;
    while ((1 << logP) < n) ++logP;
    const int half_work = 1 << (logP - 1);
    for (int lg = 1; lg <= logP; ++lg) {
        const int size = 1 << lg, hmask = (size >> 1) - 1;
        for (int i = threadIdx.x; i < half_work; i += blockDim.x) {
            const int pos = i & hmask;
            const int base = (i >> (lg - 1)) << lg;
            const int lo = base + pos, hi = base + size - 1 - pos;
            if (hi < n) {
                const int32_t x = a[lo], y = a[hi];
                if (x > y) { a[lo] = y; a[hi] = x; }
            }
        }
        __syncthreads();
        for (int ls = lg - 2; ls >= 0; --ls) {
            const int stride = 1 << ls;
            for (int i = threadIdx.x; i < half_work; i += blockDim.x) {
                const int lo = ((i >> ls) << (ls + 1)) + (i & (stride - 1));
                const int hi = lo + stride;
                if (hi < n) {
                    const int32_t x = a[lo], y = a[hi];
                    if (x > y) { a[lo] = y; a[hi] = x; }
                }
            }
            __syncthreads();
        }
    }
}

constexpr int kWarpSortMax = 512;  // segments up to this size are sorted by one warp

// Ascending sort of n <= 512 keys in place in buf (shared or global) by the calling warp: the bitonic network in
// its "flip" form (positions >= n act as +infinity), one warp barrier per stage. The loops stay rolled: fully
// unrolled register networks (one per size up to 512) took over half of each step kernel's code, and the step ran
// 17% slower on unordered segments through instruction-cache misses.
static __device__ __noinline__ void warp_sort_rolled(uint64_t* a, int n)
{
    const int lane = threadIdx.x & 31;
    int logP = 0;
    while ((1 << logP) < n) ++logP;
    const int half_work = 1 << (logP - 1);
#pragma unroll 1
    for (int lg = 1; lg <= logP; ++lg) {
        const int size = 1 << lg, hmask = (size >> 1) - 1;
#pragma unroll 1
        for (int i = lane; i < half_work; i += 32) {
            const int base = (i >> (lg - 1)) << lg;
            const int lo = base + (i & hmask), hi = base + size - 1 - (i & hmask);
            if (hi < n) cmpx(a, lo, hi);
        }
        __syncwarp();
#pragma unroll 1
        for (int ls = lg - 2; ls >= 0; --ls) {
            const int stride = 1 << ls;
#pragma unroll 1
            for (int i = lane; i < half_work; i += 32) {
                const int lo = ((i >> ls) << (ls + 1)) + (i & (stride - 1)), hi = lo + stride;
                if (hi < n) cmpx(a, lo, hi);
            }
            __syncwarp();
        }
    }
}

__device__ __forceinline__ void warp_sort_buf(uint64_t* buf, int n)
{
    __syncwarp();
    if (n >= 2) warp_sort_rolled(buf, n);
    __syncwarp();
}

// Energy-correction pairs of fast particles (gamma > 2 for either) need more than float on the mixed path: the pair's
// CM kinetic energy and the Appendix-A quadratic lose ~gamma^2 of float precision for co-moving particles (double in
// the one-CTA kernel, float-float in the group kernels).
template <class V>
__device__ __forceinline__ bool fast_pair(V c, const V v1[3], const V v2[3])
{
    const V lim = (V)3 * c * c;  // |u|^2 > 3 c^2  <=>  gamma > 2
    return (v1[0] * v1[0] + v1[1] * v1[1] + v1[2] * v1[2]) > lim || (v2[0] * v2[0] + v2[1] * v2[1] + v2[2] * v2[2]) > lim;
}

// Centre-of-mass kinetic energy of a weighted relativistic pair (as pair_kecm) with the difference of the proper
// velocities du given apart (formed from a more precise state by the caller).
template <class V>
__device__ __forceinline__ V pair_kecm_du(V c, V m1, V m2, const V v1[3], const V v2[3], const V du[3])
{
    const V c2 = c * c;
    const V g1 = sqrt((V)1 + (v1[0] * v1[0] + v1[1] * v1[1] + v1[2] * v1[2]) / c2);
    const V g2 = sqrt((V)1 + (v2[0] * v2[0] + v2[1] * v2[1] + v2[2] * v2[2]) / c2);
    V du2 = 0, ss = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        du2 += du[d] * du[d];
        ss += du[d] * (v1[d] + v2[d]);
    }
    const V dg = ss / (c2 * (g1 + g2));
    V grm1 = (V)0.5 * (du2 / c2 - dg * dg);
    if (grm1 < (V)0) grm1 = 0;
    const V Minv = sqrt((m1 + m2) * (m1 + m2) + (V)2 * m1 * m2 * grm1);
    return (V)2 * m1 * m2 * c2 * grm1 / (Minv + m1 + m2);
}

// ---------------------------------------------------------------------------------------------------------------
// N97: A(s) solves L(A) = coth A - 1/A = exp(-s), taken in the equivalent form G(A) = 1 - L(A) = -expm1(-s) so that
// small s (large A) keeps full relative precision. G is decreasing and convex, so Newton converges from any start
// (one step from the left of the root lands right of it, then monotone). Below A = 1/2, L and L' come from the
// Laurent series of coth (coefficients 2^{2n} B_{2n} / (2n)!); above, G = 1/A - 2/expm1(2A).
// ---------------------------------------------------------------------------------------------------------------
__device__ __forceinline__ void n97_G_dG(double A, double& G, double& dG)
{
    if (A < 0.5) {
        const double c[12] = {3.33333333333333315e-01,  -2.22222222222222231e-02, 2.11640211640211654e-03,
                              -2.11640211640211649e-04, 2.13777991555769346e-05,  -2.16440428080639722e-06,
                              2.19259478518737778e-07,  -2.22146087899796781e-08, 2.25078465168089944e-09,
                              -2.28051512045921834e-10, 2.31064325990026242e-11,  -2.34117068198248822e-12};
        const double x2 = A * A;
        double p = c[11], q = 23.0 * c[11];
#pragma unroll
        for (int k = 10; k >= 0; --k) {
            p = fma(p, x2, c[k]);
            q = fma(q, x2, (double)(2 * k + 1) * c[k]);
        }
        G = 1.0 - p * A;
        dG = -q;
        return;
    }
    G = 1.0 / A - 2.0 / expm1(2.0 * A);
    const double sh = sinh(A);
    dG = -(1.0 / (A * A) - (A < 350.0 ? 1.0 / (sh * sh) : 0.0));
}

__device__ __forceinline__ void n97_G_dG(float A, float& G, float& dG)
{
    if (A < 0.5f) {
        const float x2 = A * A;
        const float p = fmaf(fmaf(fmaf(fmaf(2.13777991555769346e-05f, x2, -2.11640211640211649e-04f), x2,
                                       2.11640211640211654e-03f), x2, -2.22222222222222231e-02f), x2,
                             3.33333333333333315e-01f);
        const float q = fmaf(fmaf(fmaf(fmaf(1.92400192400192391e-04f, x2, -1.48148148148148141e-03f), x2,
                                       1.05820105820105814e-02f), x2, -6.66666666666666657e-02f), x2,
                             3.33333333333333315e-01f);
        G = 1.0f - p * A;
        dG = -q;
        return;
    }
    G = 1.0f / A - 2.0f / expm1f(2.0f * A);
    const float sh = sinhf(A);
    dG = -(1.0f / (A * A) - (A < 40.0f ? 1.0f / (sh * sh) : 0.0f));
}

// Table of f(x) = ln(A s) over x = ln s in [kN97X0, kN97X0 + kN97Nodes * kN97H]: node k holds (f, h df/dx) for
// cubic Hermite interpolation (error ~1e-9). Built on the host when a context is created. The float copy holds
// g = A s = exp(f) and h dg/dx instead: |f| reaches 8.5, where a float entry of f would carry ~5e-7 of A's relative
// error, while a float entry of g carries 6e-8.
constexpr int kN97Nodes = 512;
constexpr double kN97X0 = -6.907755278982137;  // ln 1e-3
constexpr double kN97X1 = 2.4849066497880004;  // ln 12
constexpr double kN97H = (kN97X1 - kN97X0) / kN97Nodes;

template <class V>
struct N97Tab {
    const V* f;   // kN97Nodes + 1 values of ln(A s) (double) or A s (float)
    const V* dh;  // kN97Nodes + 1 values of h times their derivative in ln s
};

// First approximation of A(s): below s = 1e-3, A = 1/(1 - e^-s) (exact to rounding there, since G(A) = 1/A up to
// 2/expm1(2A) < e^-2000); above s = 12, the inversion A = 3y (1 + 3y^2/5) of L(A) = A/3 - A^3/45 with y = e^-s
// (error O(y^5)); in between the table.
template <class V>
__device__ __forceinline__ V n97_A_table(V s, V z, const N97Tab<V>& tab)
{
    if (s < (V)1e-3) return (V)1 / z;
    if (s > (V)12) {
        const V y = (V)1 - z;
        return (V)3 * y * ((V)1 + (V)0.6 * y * y);
    }
    const V u = (log(s) - (V)kN97X0) * (V)(1.0 / kN97H);
    int k = (int)u;
    k = k < 0 ? 0 : (k > kN97Nodes - 1 ? kN97Nodes - 1 : k);
    const V t = u - (V)k;
    const V f0 = tab.f[k], f1 = tab.f[k + 1], d0 = tab.dh[k], d1 = tab.dh[k + 1];
    const V t2 = t * t, t3 = t2 * t;
    const V f = ((V)2 * t3 - (V)3 * t2 + (V)1) * f0 + (t3 - (V)2 * t2 + t) * d0 + ((V)-2 * t3 + (V)3 * t2) * f1 +
                (t3 - t2) * d1;
    if (sizeof(V) == 4) return f / s;  // the float table holds A s
    return exp(f) / s;
}

template <class V>
__device__ __forceinline__ V n97_A(V s, const N97Tab<V>& tab)
{
    const V z = -expm1(-s);                  // 1 - exp(-s)
    if (!(z < (V)1)) return (V)0;            // exp(-s) underflows: isotropic limit
    if (!(z > (V)0)) return (V)CUDART_INF;   // s == 0: no scattering
    V A = n97_A_table<V>(s, z, tab);
    if (sizeof(V) == 4) return A;            // ~1e-9 from the table: below float resolution
    // Newton converges quadratically: once a step is a few ulps the next would only chase rounding noise in G, so
    // stop there (a step of 4 ulps leaves an error far below one ulp).
    const int iters = 6;
    const V tol = (V)1e-15;
    for (int it = 0; it < iters; ++it) {
        V G, dG;
        n97_G_dG(A, G, dG);
        V An = A - (G - z) / dG;
        if (!(An > (V)0)) An = (V)0.5 * A;
        const V d = fabs(An - A);
        A = An;
        if (d <= tol * A) break;
    }
    return A;
}

// Centre-of-mass polar angle from the scattering length: sin(Theta) and 1 - cos(Theta).
//  TA77: tan(Theta/2) = delta ~ N(0, s/2) by Box-Muller from (U1, U4).
//  N97:  1 - cos chi = -log1p(U1 expm1(-2A)) / A (inverse CDF of the density proportional to exp(A cos chi)),
//        1 + cos chi = log1p((1 - U1) expm1(2A)) / A.
template <class V>
__device__ __forceinline__ void sample_angle(int method, V s, V U1, V U4, V& sin_t, V& omc, const N97Tab<V>& tab)
{
    if (method == 0) {
        const V g = sqrt((V)-2 * log(U1)) * cospi((V)2 * U4);
        const V d = sqrt((V)0.5 * s) * g;
        if (fabs(d) <= (V)1) {
            const V den = (V)1 + d * d;
            sin_t = (V)2 * d / den;
            omc = (V)2 * d * d / den;
        } else {
            const V t = (V)1 / d;
            const V den = (V)1 + t * t;
            sin_t = (V)2 * t / den;
            omc = (V)2 / den;
        }
        return;
    }
    const V A = n97_A(s, tab);
    V o, q;
    if (A == (V)0) {
        o = (V)2 * U1;
        q = (V)2 * ((V)1 - U1);
    } else if (isinf(A)) {
        o = (V)0;
        q = (V)2;
    } else {
        // 1 - cos chi = -ln(1 + x)/A, 1 + x = (1 - U1) + U1 exp(-2A): log1p(x) while x is small, else the sum of
        // the two positive terms; 1 + cos chi = log1p((1 - U1) expm1(2A))/A past 90 degrees (no cancellation)
        const V x = -U1 * -expm1((V)-2 * A);
        o = x > (V)-0.5 ? -log1p(x) / A : -log(((V)1 - U1) + U1 * exp((V)-2 * A)) / A;
        q = o <= (V)1 ? (V)2 - o : log1p(((V)1 - U1) * expm1((V)2 * A)) / A;
    }
    o = fmin(fmax(o, (V)0), (V)2);
    q = fmin(fmax(q, (V)0), (V)2);
    omc = o;
    sin_t = sqrt(o * q);
}

// Rotation of u through (Theta, phi) about its own direction; returns du = u' - u.
template <class V>
__device__ __forceinline__ void rotate(V ux, V uy, V uz, V sin_t, V omc, V cp, V sp, V& dx, V& dy, V& dz)
{
    const V uperp = sqrt(ux * ux + uy * uy);
    const V u = sqrt(ux * ux + uy * uy + uz * uz);
    if (uperp > (V)0) {
        const V ax = ux / uperp, ay = uy / uperp;
        dx = ax * uz * sin_t * cp - ay * u * sin_t * sp - ux * omc;
        dy = ay * uz * sin_t * cp + ax * u * sin_t * sp - uy * omc;
        dz = -uperp * sin_t * cp - uz * omc;
    } else {
        dx = u * sin_t * cp;
        dy = u * sin_t * sp;
        dz = -uz * omc;
    }
}

__device__ __forceinline__ void sincospi_v(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void sincospi_v(float x, float* s, float* c) { sincospif(x, s, c); }

// Relativistic centre-of-momentum frame of a pair with proper velocities ui, uj and masses ma, mb: CM velocity V,
// gamma_C, boosted momentum p* of particle i, |p*| and the CM relative speed v_rel*.
template <class V>
struct RelCM {
    V Vx, Vy, Vz, gC, px, py, pz, pmag, vrel;
};

template <class V>
__device__ __forceinline__ RelCM<V> rel_cm(V c, V ma, V mb, const V ui[3], const V uj[3])
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
        const V t = ui[d] - uj[d];
        du2 += t * t;
        ss += t * (ui[d] + uj[d]);
    }
    const V dg = ss / (c2 * (gi + gj));
    V grm1 = (V)0.5 * (du2 / c2 - dg * dg);
    if (grm1 < (V)0) grm1 = 0;
    const V Minv = sqrt((ma + mb) * (ma + mb) + (V)2 * ma * mb * grm1);
    r.gC = M / Minv;
    const V coef_b = r.gC * r.gC / (c2 * (r.gC + (V)1));
    // p* = q + (gamma_C - 1)(Vhat.q) Vhat, q = (E_j p_i - E_i p_j)/E_tot = m_a m_b (gamma_j du - (gamma_i - gamma_j) u_j)/M:
    // the CM momentum through the pair's difference (no cancellation for co-moving pairs)
    const V k = ma * mb / M;
    const V qx = k * (gj * (ui[0] - uj[0]) - dg * uj[0]);
    const V qy = k * (gj * (ui[1] - uj[1]) - dg * uj[1]);
    const V qz = k * (gj * (ui[2] - uj[2]) - dg * uj[2]);
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

// Centre-of-mass kinetic energy of a weighted pair (masses m1, m2 already weighted).
template <class V, bool REL>
__device__ __forceinline__ V pair_kecm(V c, V m1, V m2, const V v1[3], const V v2[3])
{
    if (!REL) {
        V vr2 = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) vr2 += (v1[d] - v2[d]) * (v1[d] - v2[d]);
        return (V)0.5 * (m1 * m2 / (m1 + m2)) * vr2;
    }
    const V c2 = c * c;
    const V g1 = sqrt((V)1 + (v1[0] * v1[0] + v1[1] * v1[1] + v1[2] * v1[2]) / c2);
    const V g2 = sqrt((V)1 + (v2[0] * v2[0] + v2[1] * v2[1] + v2[2] * v2[2]) / c2);
    V du2 = 0, ss = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        du2 += (v1[d] - v2[d]) * (v1[d] - v2[d]);
        ss += (v1[d] - v2[d]) * (v1[d] + v2[d]);
    }
    const V dg = ss / (c2 * (g1 + g2));
    V grm1 = (V)0.5 * (du2 / c2 - dg * dg);
    if (grm1 < (V)0) grm1 = 0;
    const V Minv = sqrt((m1 + m2) * (m1 + m2) + (V)2 * m1 * m2 * grm1);
    return (V)2 * m1 * m2 * c2 * grm1 / (Minv + m1 + m2);
}

// Zero-angle inelastic pair: the pair's CM energy K loses U, momentum unchanged (Eqs. vp1_inelastic,
// vp2_inelastic, vrel_inelastic; Appendix A quadratic in alpha for relativistic particles).
template <class V, bool REL>
__device__ __forceinline__ void energy_pair(V c, V m1, V m2, V K, V v1[3], V v2[3], V U)
{
    if (!REL) {
        const V x = U / K;
        const V gm1 = -x / ((V)1 + sqrt((V)1 - x));
        const V f1 = m2 / (m1 + m2) * gm1, f2 = m1 / (m1 + m2) * gm1;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const V vr = v1[d] - v2[d];
            v1[d] += f1 * vr;
            v2[d] -= f2 * vr;
        }
        return;
    }
    const V c2 = c * c;
    const V g1 = sqrt((V)1 + (v1[0] * v1[0] + v1[1] * v1[1] + v1[2] * v1[2]) / c2);
    const V g2 = sqrt((V)1 + (v2[0] * v2[0] + v2[1] * v2[1] + v2[2] * v2[2]) / c2);
    const V E1 = m1 * g1, E2 = m2 * g2, Ut = U / c2;
    const V A = E1 + E2 - Ut;
    V du[3], pt[3], du2 = 0, ss = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        du[d] = v1[d] - v2[d];
        pt[d] = m1 * v1[d] + m2 * v2[d];
        du2 += du[d] * du[d];
        ss += du[d] * (v1[d] + v2[d]);
    }
    const V dg = ss / (c2 * (g1 + g2));
    V bdot = 0, ptdu = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const V x12 = m1 * m2 * (g2 * du[d] - dg * v2[d]);
        const V bv = (V)2 * A * (x12 + Ut * m2 * v2[d]) - Ut * ((V)2 * E1 - Ut) * pt[d];
        bdot += du[d] * bv;
        ptdu += pt[d] * du[d];
    }
    const V a = (V)4 * (A * A * du2 / c2 - ptdu * ptdu / (c2 * c2));
    const V b = (V)4 / c2 * bdot;
    const V c0 = Ut * ((V)2 * E1 - Ut) * ((V)2 * E2 - Ut) * ((V)2 * E1 + (V)2 * E2 - Ut);
    V disc = b * b - (V)4 * a * c0;
    if (disc < (V)0) disc = 0;
    const V q = (V)-0.5 * (b + (b >= (V)0 ? sqrt(disc) : -sqrt(disc)));
    const V r1 = (a != (V)0) ? q / a : (V)CUDART_INF;
    const V r2 = (q != (V)0) ? c0 / q : (V)0;
    const V alpha = fabs(r1) < fabs(r2) ? r1 : r2;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        v1[d] += alpha * du[d] / m1;
        v2[d] -= alpha * du[d] / m2;
    }
    (void)K;
}

}  // namespace mcc
