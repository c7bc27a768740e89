// Group kernels of the fused step (mixed precision), relativistic = true (one translation unit per variant keeps the
// build parallel).
#include "mcc_group.cuh"

namespace mcc {

const void* group_kernel_f32rel(int cls)
{
    switch (cls) {
    case 0: return grp::group_kernel_ptr<true, 32>();
    case 1: return grp::group_kernel_ptr<true, 64>();
    case 2: return grp::group_kernel_ptr<true, 128>();
    case 3: return grp::group_kernel_ptr<true, 256>();
    default: return grp::group_kernel_ptr<true, 512>();
    }
}

}  // namespace mcc
