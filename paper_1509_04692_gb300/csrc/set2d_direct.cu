// Instantiations of the 2D direct set kernel (FP32-filtered form).
#include "hpmc_launch.h"
#include "hpmc_sweep2d_direct.cuh"

namespace hpmc {

SetKernel set2d_direct_kernel(bool fixed_nv)
{
    if (fixed_nv) return { (const void*)&k_set2d_direct<5>, sizeof(Direct2Warp) };
    return { (const void*)&k_set2d_direct<0>, sizeof(Direct2Warp) };
}

}  // namespace hpmc
