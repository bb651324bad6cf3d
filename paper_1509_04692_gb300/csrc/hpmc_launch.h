// hpmc_launch.h -- host-side table of the set-kernel instantiations.
#pragma once
#include <cstddef>

namespace hpmc {

struct SetKernel {
    const void* fn;          // __global__ function (Dev, Shape, int nxt, int sigma, const uint32_t*)
    size_t smem_per_warp;    // dynamic shared memory per warp
};

// lanes per cell G in {1, 2, 4, 8, 16, 32}; fixed_nv: shape specialised on
// the vertex count (5 for pentagons in 2D, 8 for cubes in 3D).
SetKernel set2d_f32_kernel(int G, bool fixed_nv);
SetKernel set2d_f64_kernel(int G, bool fixed_nv);
SetKernel set3d_f32_kernel(int G, bool fixed_nv);
SetKernel set3d_f64_kernel(int G, bool fixed_nv);

}  // namespace hpmc
