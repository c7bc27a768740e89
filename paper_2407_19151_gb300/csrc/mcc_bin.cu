// Cell binning: stable counting sort of particles by key = cell * S + species (particles collide per cell of
// volume dV, Sec. 2), and a gather through the resulting permutation.
//
// histogram (atomic counts) -> exclusive scan -> scatter with atomic cursors (order within a segment arbitrary)
// -> per-segment sort of the particle indices, which restores the stable (index) order. The result does not depend
// on the order in which the atomics were served. The atomics are warp-aggregated (lanes with equal keys add once),
// which matters for nearly binned input such as a re-bin after a particle push; segments of up to 512 entries are
// sorted by one warp in its slice of shared memory (warp barriers only), larger ones by a whole CTA.
#include <mutex>

#include "mcc_kernels.h"

// Counters of mcc_bin_static: every device that loads the library holds this array until the process exits.
// counts | cursors | large-segment list, the layout launch_bin expects for kStaticBinKeys segments.
constexpr int64_t kStaticBinKeys = 1 << 21;
constexpr size_t kStaticBinHalf = ((size_t)kStaticBinKeys * sizeof(int32_t) + 255) & ~(size_t)255;
constexpr size_t kStaticBinList = ((size_t)(kStaticBinKeys + 1) * sizeof(int32_t) + 255) & ~(size_t)255;
static __device__ __align__(256) int32_t g_bin_static_scratch[(2 * kStaticBinHalf + kStaticBinList) / sizeof(int32_t)];

namespace mcc {
namespace {

constexpr int kBinThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kSegCap = 12288;  // indices sorted in shared memory per segment; larger segments sort in place
constexpr int kSegCapW = 4096;  // weight-order keys sorted in shared memory per segment; larger ones in the workspace

constexpr int kWarpSeg = 512;  // segments up to this size are sorted by one warp

// Key of particle i (cell * S + species), or -1 past the end or out of range (latched).
__device__ __forceinline__ long long bin_key(const int32_t* __restrict__ cell, const int32_t* __restrict__ species,
                                             int64_t i, int64_t n, int32_t n_cells, int32_t S, int32_t* status)
{
    if (i >= n) return -1;
    const int32_t c = cell[i], s = species[i];
    if (c < 0 || c >= n_cells || s < 0 || s >= S) {
        if (status) latch(status, kErrBounds);
        return -1;
    }
    return (long long)c * S + s;
}

// All lanes of a warp run the same trips (the loop index is the warp's base), so the match below sees the full warp.
__global__ void k_hist(const int32_t* __restrict__ cell, const int32_t* __restrict__ species, int64_t n,
                       int32_t n_cells, int32_t S, int32_t* __restrict__ counts, int32_t* status)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const long long key = bin_key(cell, species, base + lane, n, n_cells, S, status);
        const unsigned m = __match_any_sync(0xffffffffu, key);
        if (key >= 0 && lane == __ffs(m) - 1) atomicAdd(&counts[key], __popc(m));
    }
}

// Exclusive scan of nk counts into nk + 1 offsets, in three passes over tiles of kScanTile keys: each CTA scans its
// tile (tile-local offsets) and leaves the tile's total in counts[first key of the tile]; one CTA scans the tile
// totals in place (their exclusive prefixes) and writes offsets[nk]; each CTA adds its tile's prefix. The counts are
// not read again after the scan, so their tile-start slots can carry the totals.
constexpr int kScanTile = 4 * kScanThreads;

// Exclusive scan of v over the CTA (kScanThreads threads); returns this thread's exclusive prefix, *total the sum.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* wsum, int64_t* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t t = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    *total = wsum[31];
    return x - v + (wid > 0 ? wsum[wid - 1] : 0);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tile(int32_t* __restrict__ counts, int64_t nk,
                                                            int64_t* __restrict__ offsets, int32_t* status)
{
    __shared__ int64_t wsum[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + 4 * threadIdx.x;
    int32_t c[4];
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c[j] = base + j < nk ? counts[base + j] : 0;
        if (c[j] > (1 << kPermBits)) latch(status, kErrTooLarge);
        s += c[j];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(s, wsum, &total);  // every thread has read its counts before this returns
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (base + j < nk) offsets[base + j] = run;
        run += c[j];
    }
    if (threadIdx.x == 0) counts[(int64_t)blockIdx.x * kScanTile] = (int32_t)total;  // total <= n <= INT32_MAX
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(int32_t* __restrict__ counts, int64_t nk, int64_t tiles,
                                                           int64_t* __restrict__ offsets)
{
    __shared__ int64_t wsum[kScanThreads / 32];
    const int64_t chunk = (tiles + kScanThreads - 1) / kScanThreads;
    const int64_t b = (int64_t)threadIdx.x * chunk;
    const int64_t e = b + chunk < tiles ? b + chunk : tiles;
    int64_t s = 0;
    for (int64_t t = b; t < e; ++t) s += counts[t * kScanTile];
    int64_t total;
    int64_t run = block_exclusive_scan(s, wsum, &total);
    for (int64_t t = b; t < e; ++t) {
        const int32_t x = counts[t * kScanTile];
        counts[t * kScanTile] = (int32_t)run;
        run += x;
    }
    if (threadIdx.x == 0) offsets[nk] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(const int32_t* __restrict__ counts, int64_t nk,
                                                           int64_t* __restrict__ offsets)
{
    if (blockIdx.x == 0) return;
    const int64_t pre = counts[(int64_t)blockIdx.x * kScanTile];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int j = threadIdx.x; j < kScanTile; j += kScanThreads)
        if (base + j < nk) offsets[base + j] += pre;
}

__global__ void k_scatter(const int32_t* __restrict__ cell, const int32_t* __restrict__ species, int64_t n,
                          int32_t n_cells, int32_t S, const int64_t* __restrict__ offsets,
                          int32_t* __restrict__ cursor, int32_t* __restrict__ perm)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const long long key = bin_key(cell, species, base + lane, n, n_cells, S, nullptr);
        const unsigned m = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(m) - 1;
        int32_t at = 0;
        if (key >= 0 && lane == leader) at = atomicAdd(&cursor[key], __popc(m));
        at = __shfl_sync(0xffffffffu, at, leader);
        if (key >= 0) perm[offsets[key] + at + __popc(m & ((1u << lane) - 1u))] = (int32_t)(base + lane);
    }
}

// Ascending sort of n <= kWarpSeg entries in the calling warp's shared-memory slice: the bitonic network in its
// "flip" form (every comparator puts the smaller entry at the lower index, so positions >= n act as +infinity and
// are skipped), one warp barrier per stage. Loops stay rolled: the code is small enough to stay in the instruction
// cache. cmpx(lo, hi) orders the entries at two positions.
template <class Cmpx>
__device__ __forceinline__ void warp_sort_smem(int n, Cmpx cmpx)
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
            if (hi < n) cmpx(lo, hi);
        }
        __syncwarp();
#pragma unroll 1
        for (int ls = lg - 2; ls >= 0; --ls) {
            const int stride = 1 << ls;
#pragma unroll 1
            for (int i = lane; i < half_work; i += 32) {
                const int lo = ((i >> ls) << (ls + 1)) + (i & (stride - 1)), hi = lo + stride;
                if (hi < n) cmpx(lo, hi);
            }
            __syncwarp();
        }
    }
}

// Small segments (2 .. kWarpSeg entries), one warp each, sorted in the warp's shared-memory slice (the loop index is
// warp-uniform, so whole warps take the same branches). w == nullptr: the entries by particle index. Otherwise
// straight into the weight order of mcc_bin_weighted: pairs (weight key with a zero rank field, particle index)
// sorted lexicographically, which is descending truncated weight with ties in increasing index. The ids of the
// larger segments are appended to `large` (large[0] the count, zeroed before) for the CTA-wide sorts.
// WEIGHTED: the weight-order keys need a second slab; the index-only sort keeps 2 KB per warp, so that more warps
// fit an SM (the sorts are latency-bound).
template <bool WEIGHTED>
__global__ void __launch_bounds__(kBinThreads) k_segsort_warp(const int64_t* __restrict__ offsets, int64_t nk,
                                                              const double* __restrict__ w, int32_t* __restrict__ perm,
                                                              int32_t* __restrict__ large)
{
    __shared__ uint64_t kslab[WEIGHTED ? kBinThreads / 32 : 1][WEIGHTED ? kWarpSeg : 1];
    __shared__ int32_t islab[kBinThreads / 32][kWarpSeg];
    const int lane = threadIdx.x & 31;
    uint64_t* kb = kslab[WEIGHTED ? threadIdx.x >> 5 : 0];
    int32_t* ib = islab[threadIdx.x >> 5];
    const int64_t warp = ((int64_t)blockIdx.x * kBinThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kBinThreads) >> 5;
    for (int64_t seg = warp; seg < nk; seg += nwarps) {
        const int64_t b = offsets[seg];
        const int n = (int)(offsets[seg + 1] - b);
        if (n > kWarpSeg && lane == 0) large[1 + atomicAdd(&large[0], 1)] = (int32_t)seg;
        if (n < 2 || n > kWarpSeg) continue;
        int32_t* p = perm + b;
        if (!WEIGHTED) {
            for (int i = lane; i < n; i += 32) ib[i] = p[i];
            __syncwarp();
            warp_sort_smem(n, [ib](int lo, int hi) {
                const int32_t x = ib[lo], y = ib[hi];
                if (x > y) {
                    ib[lo] = y;
                    ib[hi] = x;
                }
            });
        } else {
            for (int i = lane; i < n; i += 32) {
                const int32_t q = p[i];
                ib[i] = q;
                kb[i] = weight_key(w[q], 0u);
            }
            __syncwarp();
            warp_sort_smem(n, [kb, ib](int lo, int hi) {
                const uint64_t x = kb[lo], y = kb[hi];
                const int32_t a = ib[lo], c = ib[hi];
                if (x > y || (x == y && a > c)) {
                    kb[lo] = y;
                    kb[hi] = x;
                    ib[lo] = c;
                    ib[hi] = a;
                }
            });
        }
        for (int i = lane; i < n; i += 32) p[i] = ib[i];
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kBinThreads) k_segsort(const int64_t* __restrict__ offsets,
                                                         const int32_t* __restrict__ large, int32_t* __restrict__ perm)
{
    __shared__ int32_t buf[kSegCap];
    const int32_t n_large = large[0];
    for (int32_t q = blockIdx.x; q < n_large; q += gridDim.x) {
        const int64_t seg = large[1 + q];
        const int64_t b = offsets[seg];
        const int n = (int)(offsets[seg + 1] - b);
        if (n <= kSegCap) {
            for (int i = threadIdx.x; i < n; i += kBinThreads) buf[i] = perm[b + i];
            __syncthreads();
            block_sort_i32(buf, n);
            for (int i = threadIdx.x; i < n; i += kBinThreads) perm[b + i] = buf[i];
        } else {
            block_sort_i32(perm + b, n);
        }
        __syncthreads();
    }
}

// Weight order of every large segment (run after k_segsort, so a segment's entries are in increasing particle index):
// keys = weight_key(w, rank) (descending weight truncated to 32 fraction bits, ties by rank = by index), sorted, then
// each slot takes the index its key's rank points to. keys: [n] workspace, holds the keys of large segments and
// the reordered indices before they are copied back.
__global__ void __launch_bounds__(kBinThreads) k_segsort_w(const int64_t* __restrict__ offsets,
                                                           const int32_t* __restrict__ large,
                                                           const double* __restrict__ w, int32_t* __restrict__ perm,
                                                           uint64_t* __restrict__ keys)
{
    __shared__ uint64_t buf[kSegCapW];
    const int32_t n_large = large[0];
    for (int32_t q = blockIdx.x; q < n_large; q += gridDim.x) {
        const int64_t seg = large[1 + q];
        const int64_t b = offsets[seg];
        const int n = (int)(offsets[seg + 1] - b);
        uint64_t* k = n <= kSegCapW ? buf : keys + b;
        for (int i = threadIdx.x; i < n; i += kBinThreads) k[i] = weight_key(w[perm[b + i]], (uint32_t)i);
        __syncthreads();
        block_sort_u64(k, n);
        // each thread reads only its own slot of k before writing that slot of keys
        for (int i = threadIdx.x; i < n; i += kBinThreads)
            keys[b + i] = (uint64_t)(uint32_t)perm[b + (int)(k[i] & kPermMask)];
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += kBinThreads) perm[b + i] = (int32_t)(uint32_t)keys[b + i];
        __syncthreads();
    }
}

// Four elements per thread and iteration, their permuted reads issued together (more reads in flight).
template <class T>
__global__ void k_gather(const T* __restrict__ in, const int32_t* __restrict__ perm, int64_t n, T* __restrict__ out)
{
    constexpr int U = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n; base += U * stride) {
        int32_t p[U];
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) p[u] = base + u * stride < n ? perm[base + u * stride] : 0;
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = base + u * stride < n ? __ldg(in + p[u]) : T(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (base + u * stride < n) out[base + u * stride] = v[u];
    }
}

int grid_for(int64_t n, int threads)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)sms * 16;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

// Workspace: counts | cursors (one int32 per segment each) | large-segment list (count, then segment ids).
size_t bin_workspace_bytes(int64_t n, int64_t n_keys)
{
    (void)n;
    const size_t one = ((size_t)n_keys * sizeof(int32_t) + 255) & ~(size_t)255;
    const size_t lst = ((size_t)(n_keys + 1) * sizeof(int32_t) + 255) & ~(size_t)255;
    return 2 * one + lst;
}

static int32_t* large_list(void* ws, int64_t nk)
{
    const size_t one = ((size_t)nk * sizeof(int32_t) + 255) & ~(size_t)255;
    return reinterpret_cast<int32_t*>(reinterpret_cast<char*>(ws) + 2 * one);
}

// hist -> scan -> scatter -> small segments by one warp each (index order, or with w the weight order directly)
// -> large segments by index, one CTA each.
static cudaError_t bin_core(const int32_t* cell, const int32_t* species, int64_t n, int32_t n_cells,
                            int32_t n_species, const double* w, int32_t* perm, int64_t* offsets, void* ws,
                            int32_t* status, cudaStream_t st, int64_t* launches)
{
    const int64_t nk = (int64_t)n_cells * n_species;
    const size_t one = ((size_t)nk * sizeof(int32_t) + 255) & ~(size_t)255;
    int32_t* counts = reinterpret_cast<int32_t*>(ws);
    int32_t* cursor = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(ws) + one);
    int32_t* large = large_list(ws, nk);
    cudaError_t e = cudaMemsetAsync(ws, 0, bin_workspace_bytes(n, nk), st);
    if (e != cudaSuccess) return e;
    const int g = grid_for(n, kBinThreads);
    if (n > 0) k_hist<<<g, kBinThreads, 0, st>>>(cell, species, n, n_cells, n_species, counts, status);
    const int64_t tiles = (nk + kScanTile - 1) / kScanTile;
    k_scan_tile<<<(unsigned)tiles, kScanThreads, 0, st>>>(counts, nk, offsets, status);
    k_scan_top<<<1, kScanThreads, 0, st>>>(counts, nk, tiles, offsets);
    k_scan_add<<<(unsigned)tiles, kScanThreads, 0, st>>>(counts, nk, offsets);
    *launches += 3;
    if (n > 0) {
        k_scatter<<<g, kBinThreads, 0, st>>>(cell, species, n, n_cells, n_species, offsets, cursor, perm);
        if (w)
            k_segsort_warp<true><<<grid_for(nk * 32, kBinThreads), kBinThreads, 0, st>>>(offsets, nk, w, perm, large);
        else
            k_segsort_warp<false><<<grid_for(nk * 32, kBinThreads), kBinThreads, 0, st>>>(offsets, nk, w, perm, large);
        k_segsort<<<grid_for(n / (kWarpSeg + 1) * kBinThreads, kBinThreads), kBinThreads, 0, st>>>(offsets, large,
                                                                                                 perm);
        *launches += 4;
    }
    return cudaGetLastError();
}

cudaError_t launch_bin(const int32_t* cell, const int32_t* species, int64_t n, int32_t n_cells, int32_t n_species,
                       int32_t* perm, int64_t* offsets, void* ws, int32_t* status, cudaStream_t st, int64_t* launches)
{
    return bin_core(cell, species, n, n_cells, n_species, nullptr, perm, offsets, ws, status, st, launches);
}

size_t bin_weighted_workspace_bytes(int64_t n, int64_t n_keys)
{
    return bin_workspace_bytes(n, n_keys) + (((size_t)n * sizeof(uint64_t) + 255) & ~(size_t)255);
}

cudaError_t launch_bin_weighted(const int32_t* cell, const int32_t* species, const double* w, int64_t n,
                                int32_t n_cells, int32_t n_species, int32_t* perm, int64_t* offsets, void* ws,
                                int32_t* status, cudaStream_t st, int64_t* launches)
{
    const int64_t nk = (int64_t)n_cells * n_species;
    cudaError_t e = bin_core(cell, species, n, n_cells, n_species, w, perm, offsets, ws, status, st, launches);
    if (e != cudaSuccess || n == 0) return e;
    uint64_t* keys = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(ws) + bin_workspace_bytes(n, nk));
    const int32_t* large = large_list(ws, nk);  // the segments above kWarpSeg, already in index order
    k_segsort_w<<<grid_for(n / (kWarpSeg + 1) * kBinThreads, kBinThreads), kBinThreads, 0, st>>>(offsets, large, w,
                                                                                               perm, keys);
    *launches += 1;
    return cudaGetLastError();
}

// Device address of g_bin_static_scratch on the current device. The host-side name is only a stand-in, so the
// address is looked up once per device (with that device current) and cached.
static void* static_bin_scratch(int* err)
{
    static std::mutex mu;
    static void* addr[256] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        *err = 1;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bin_static_scratch) != cudaSuccess || !p) {
            *err = 1;
            return nullptr;
        }
        addr[dev] = p;
    }
    *err = 0;
    return addr[dev];
}

int64_t static_bin_max_keys() { return kStaticBinKeys; }

cudaError_t launch_bin_static(const int32_t* cell, const int32_t* species, int64_t n, int32_t n_cells,
                              int32_t n_species, int32_t* perm, int64_t* offsets, cudaStream_t st)
{
    int err = 0;
    void* ws = static_bin_scratch(&err);
    if (err) return cudaErrorInvalidSymbol;
    int64_t launches = 0;
    // launch_bin clears both counter arrays on the stream before its kernels; no status word (out-of-range
    // particles are dropped, visible as offsets[last] < n)
    return launch_bin(cell, species, n, n_cells, n_species, perm, offsets, ws, nullptr, st, &launches);
}

cudaError_t launch_gather(const void* in, const int32_t* perm, int64_t n, int elem_bytes, void* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int g = grid_for(n, kBinThreads);
    if (elem_bytes == 8)
        k_gather<uint64_t><<<g, kBinThreads, 0, st>>>(reinterpret_cast<const uint64_t*>(in), perm, n,
                                                      reinterpret_cast<uint64_t*>(out));
    else
        k_gather<uint32_t><<<g, kBinThreads, 0, st>>>(reinterpret_cast<const uint32_t*>(in), perm, n,
                                                      reinterpret_cast<uint32_t*>(out));
    return cudaGetLastError();
}

}  // namespace mcc
