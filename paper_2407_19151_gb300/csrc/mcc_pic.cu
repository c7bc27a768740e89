// PIC coupling: the free-streaming particle push (x <- x + v dt, periodic box, new cell ids) and a gather of several
// particle arrays through one permutation, the two per-step passes that re-binning adds around the collision step
// once positions move. Both are streaming kernels bound by HBM bandwidth: the push reads positions and velocities
// and writes positions and cell ids (40 B per particle for float, 76 B for double); the gather reads the permutation
// once and moves every array's element.
#include <cmath>

#include "mcc_pic.h"

namespace mcc {
namespace {

constexpr int kPushThreads = 256;

// Every operation of the push rounded to nearest with no contraction into a fused multiply-add, so that the
// positions, and the cell ids they decide, are reproducible bit for bit by a host program in the same precision.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rsqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double rsqrt_rn(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float rfloor(float a) { return floorf(a); }
__device__ __forceinline__ double rfloor(double a) { return floor(a); }

template <class T>
struct PushK {
    T dt, c2, L[3], sx[3];
    int32_t n[3];
};

// Periodic wrap into [0, L); a non-finite coordinate becomes 0.
template <class T>
__device__ __forceinline__ T wrap(T x, T L)
{
    if (x >= (T)0 && x < L) return x;
    T r = rsub(x, rmul(rfloor(rdiv(x, L)), L));
    if (r < (T)0) r = radd(r, L);
    if (r >= L) r = rsub(r, L);
    if (!(r >= (T)0 && r < L)) r = (T)0;
    return r;
}

template <class T, bool REL>
__global__ void __launch_bounds__(kPushThreads)
    k_push(T* __restrict__ x, T* __restrict__ y, T* __restrict__ z, const T* __restrict__ vx,
           const T* __restrict__ vy, const T* __restrict__ vz, int64_t n, PushK<T> k, int32_t* __restrict__ cell)
{
    for (int64_t i = (int64_t)blockIdx.x * kPushThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kPushThreads) {
        const T u[3] = {vx[i], vy[i], vz[i]};
        T ginv = (T)1;
        if (REL) {
            const T s = radd(radd(rmul(u[0], u[0]), rmul(u[1], u[1])), rmul(u[2], u[2]));
            ginv = rdiv((T)1, rsqrt_rn(radd((T)1, rdiv(s, k.c2))));
        }
        T p[3] = {x[i], y[i], z[i]};
        int id[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const T v = REL ? rmul(u[d], ginv) : u[d];
            p[d] = wrap(radd(p[d], rmul(v, k.dt)), k.L[d]);
            const int c = (int)rmul(p[d], k.sx[d]);  // p >= 0: truncation is the floor
            id[d] = c < k.n[d] ? c : k.n[d] - 1;
        }
        x[i] = p[0];
        y[i] = p[1];
        z[i] = p[2];
        cell[i] = id[0] + k.n[0] * (id[1] + k.n[1] * id[2]);
    }
}

struct GatherN {
    const void* in[8];
    void* out[8];
    int32_t bytes[8];
    int32_t n_arrays;
};

// Four elements per thread and iteration (their permutation entries loaded first, then every array's four reads
// issued together): more reads in flight per thread for the latency of the permuted loads.
constexpr int kGatherUnroll = 4;

template <class T>
__device__ __forceinline__ void gather4(const void* in, void* out, const int64_t (&p)[kGatherUnroll], int64_t base,
                                        int64_t stride, int64_t n)
{
    T v[kGatherUnroll];
#pragma unroll
    for (int u = 0; u < kGatherUnroll; ++u)
        v[u] = base + u * stride < n ? __ldg(static_cast<const T*>(in) + p[u]) : T(0);
#pragma unroll
    for (int u = 0; u < kGatherUnroll; ++u)
        if (base + u * stride < n) static_cast<T*>(out)[base + u * stride] = v[u];
}

__global__ void __launch_bounds__(kPushThreads) k_gather_n(GatherN a, const int32_t* __restrict__ perm, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * kPushThreads;
    for (int64_t base = (int64_t)blockIdx.x * kPushThreads + threadIdx.x; base < n; base += kGatherUnroll * stride) {
        int64_t p[kGatherUnroll];
#pragma unroll
        for (int u = 0; u < kGatherUnroll; ++u) p[u] = base + u * stride < n ? perm[base + u * stride] : 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j >= a.n_arrays) break;
            if (a.bytes[j] == 8) gather4<uint64_t>(a.in[j], a.out[j], p, base, stride, n);
            else gather4<uint32_t>(a.in[j], a.out[j], p, base, stride, n);
        }
    }
}

int stream_grid(int64_t n)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + kPushThreads - 1) / kPushThreads;
    const int64_t cap = (int64_t)sms * 8;  // eight 256-thread CTAs per SM, grid-stride beyond
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

template <class T>
cudaError_t push_t(bool rel, void* x, void* y, void* z, const void* vx, const void* vy, const void* vz, int64_t n,
                   const PushGrid& g, double dt, double c, int32_t* cell, cudaStream_t st)
{
    PushK<T> k;
    k.dt = (T)dt;
    k.c2 = (T)(c * c);
    for (int d = 0; d < 3; ++d) {
        k.L[d] = (T)g.l[d];
        k.sx[d] = (T)((double)g.n[d] / g.l[d]);
        k.n[d] = g.n[d];
    }
    const int grid = stream_grid(n);
    T* X = static_cast<T*>(x);
    T* Y = static_cast<T*>(y);
    T* Z = static_cast<T*>(z);
    const T* VX = static_cast<const T*>(vx);
    const T* VY = static_cast<const T*>(vy);
    const T* VZ = static_cast<const T*>(vz);
    if (rel)
        k_push<T, true><<<grid, kPushThreads, 0, st>>>(X, Y, Z, VX, VY, VZ, n, k, cell);
    else
        k_push<T, false><<<grid, kPushThreads, 0, st>>>(X, Y, Z, VX, VY, VZ, n, k, cell);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_push(bool f32, bool rel, void* x, void* y, void* z, const void* vx, const void* vy, const void* vz,
                        int64_t n, const PushGrid& g, double dt, double c, int32_t* cell_out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    return f32 ? push_t<float>(rel, x, y, z, vx, vy, vz, n, g, dt, c, cell_out, st)
               : push_t<double>(rel, x, y, z, vx, vy, vz, n, g, dt, c, cell_out, st);
}

cudaError_t launch_gather_n(const void* const* in, void* const* out, const int32_t* elem_bytes, int n_arrays,
                            const int32_t* perm, int64_t n, cudaStream_t st)
{
    if (n <= 0 || n_arrays <= 0) return cudaSuccess;
    GatherN a{};
    for (int j = 0; j < n_arrays; ++j) {
        a.in[j] = in[j];
        a.out[j] = out[j];
        a.bytes[j] = elem_bytes[j];
    }
    a.n_arrays = n_arrays;
    k_gather_n<<<stream_grid(n), kPushThreads, 0, st>>>(a, perm, n);
    return cudaGetLastError();
}

}  // namespace mcc
