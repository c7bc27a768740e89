// Group kernels of the fused step (mixed precision), relativistic = false (one translation unit per variant keeps the
// build parallel).
#include "mcc_group.cuh"

namespace mcc {

const void* group_kernel_f32(int cls)
{
    switch (cls) {
    case 0: return grp::group_kernel_ptr<false, 32>();
    case 1: return grp::group_kernel_ptr<false, 64>();
    case 2: return grp::group_kernel_ptr<false, 128>();
    case 3: return grp::group_kernel_ptr<false, 256>();
    default: return grp::group_kernel_ptr<false, 512>();
    }
}

}  // namespace mcc
