// Per-species moments of a binned state, the diagnostics that sharded runs all-reduce once per step: for each
// species s, sum w, sum m w v (three components), sum of the kinetic energy (1/2 m w |v|^2, or m w c^2 (gamma - 1)
// for proper velocities) and the particle count, plus the sum of the per-cell failure counts.
//
// One CTA per group of cells (grid-stride), one species at a time: each thread accumulates its particles'
// contributions in six FP64 registers, the CTA reduces them with warp shuffles and shared memory and adds its partial
// sums to the output with double atomics, so the summation order varies between runs at the rounding level.
#include "mcc_kernels.h"

namespace mcc {
namespace {

constexpr int kMomThreads = 256;
constexpr int kMomFields = 6;  // sum w, sum m w vx, vy, vz, sum KE, count

template <class V>
__global__ void __launch_bounds__(kMomThreads) k_species_moments(const V* __restrict__ vx, const V* __restrict__ vy,
                                                                 const V* __restrict__ vz, const double* __restrict__ w,
                                                                 const int64_t* __restrict__ offsets, int32_t n_cells,
                                                                 int32_t S, SpeciesConst sc, int rel, double c,
                                                                 const int32_t* __restrict__ fail_count, double* out)
{
    __shared__ double red[kMomThreads / 32][kMomFields];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double c2 = c * c;
    for (int s = 0; s < S; ++s) {
        const double m = sc.m[s];
        double acc[kMomFields] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int32_t cell = blockIdx.x; cell < n_cells; cell += gridDim.x) {
            const int64_t b = offsets[(int64_t)cell * S + s], e = offsets[(int64_t)cell * S + s + 1];
            for (int64_t i = b + threadIdx.x; i < e; i += kMomThreads) {
                const double x = (double)vx[i], y = (double)vy[i], z = (double)vz[i], mw = m * w[i];
                const double v2 = x * x + y * y + z * z;
                acc[0] += w[i];
                acc[1] += mw * x;
                acc[2] += mw * y;
                acc[3] += mw * z;
                acc[4] += rel ? mw * v2 / (sqrt(1.0 + v2 / c2) + 1.0) : 0.5 * mw * v2;
                acc[5] += 1.0;
            }
        }
#pragma unroll
        for (int f = 0; f < kMomFields; ++f) {
            double x = acc[f];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) red[wid][f] = x;
        }
        __syncthreads();
        if (threadIdx.x < kMomFields) {
            double x = 0.0;
            for (int k = 0; k < kMomThreads / 32; ++k) x += red[k][threadIdx.x];
            if (x != 0.0) atomicAdd(&out[s * kMomFields + threadIdx.x], x);
        }
        __syncthreads();
    }
    if (fail_count) {
        double f = 0.0;
        for (int32_t cell = blockIdx.x * kMomThreads + threadIdx.x; cell < n_cells; cell += gridDim.x * kMomThreads)
            f += (double)fail_count[cell];
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        if (lane == 0 && f != 0.0) atomicAdd(&out[S * kMomFields], f);
    }
}

}  // namespace

cudaError_t launch_species_moments(bool f32, const void* vx, const void* vy, const void* vz, const double* w,
                                   const int64_t* offsets, int32_t n_cells, int32_t S, const SpeciesConst& sc,
                                   int rel, double c, const int32_t* fail_count, double* out, int num_sms,
                                   cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * (size_t)(S * kMomFields + 1), st);
    if (e != cudaSuccess || n_cells == 0) return e;
    int grid = 4 * num_sms;
    if (grid > n_cells) grid = n_cells;
    if (f32)
        k_species_moments<float><<<grid, kMomThreads, 0, st>>>(
            static_cast<const float*>(vx), static_cast<const float*>(vy), static_cast<const float*>(vz), w, offsets,
            n_cells, S, sc, rel, c, fail_count, out);
    else
        k_species_moments<double><<<grid, kMomThreads, 0, st>>>(
            static_cast<const double*>(vx), static_cast<const double*>(vy), static_cast<const double*>(vz), w,
            offsets, n_cells, S, sc, rel, c, fail_count, out);
    return cudaGetLastError();
}

}  // namespace mcc
