// Instantiations of the 2D direct set kernel (FP32-filtered and plain FP64 forms).
#include "hpmc_launch.h"
#include "hpmc_sweep2d_direct.cuh"

namespace hpmc {

SetKernel set2d_direct_kernel(bool fixed_nv, bool f32)
{
    if (f32) {
        if (fixed_nv) return { (const void*)&k_set2d_direct<5, true>, sizeof(Direct2Warp) };
        return { (const void*)&k_set2d_direct<0, true>, sizeof(Direct2Warp) };
    }
    if (fixed_nv) return { (const void*)&k_set2d_direct<5, false>, sizeof(Direct2Warp) };
    return { (const void*)&k_set2d_direct<0, false>, sizeof(Direct2Warp) };
}

}  // namespace hpmc
