// Launchers of the PIC-coupling kernels (free-streaming push, multi-array gather); contracts in include/mcc.h.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace mcc {

struct PushGrid {
    int32_t n[3];   // cells per axis
    double l[3];    // box lengths
};

// Positions and velocities of precision f32 ? float : double; cell_out int32.
cudaError_t launch_push(bool f32, bool rel, void* x, void* y, void* z, const void* vx, const void* vy, const void* vz,
                        int64_t n, const PushGrid& g, double dt, double c, int32_t* cell_out, cudaStream_t st);

// out[a][k] = in[a][perm[k]] for a < n_arrays (<= 8), elem_bytes 4 or 8 each.
cudaError_t launch_gather_n(const void* const* in, void* const* out, const int32_t* elem_bytes, int n_arrays,
                            const int32_t* perm, int64_t n, cudaStream_t st);

}  // namespace mcc
