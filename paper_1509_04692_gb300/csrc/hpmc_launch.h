// hpmc_launch.h -- host-side table of the set-kernel instantiations.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "hpmc_types.h"

namespace hpmc {

struct SetKernel {
    const void* fn;          // __global__ function (Dev, Shape, int nxt, int sigma, const uint32_t*)
    size_t smem_per_warp;    // dynamic shared memory per warp
};

// lanes per cell G in {1, 2, 4, 8, 16, 32}; G = 0 selects the 2D direct kernel.  2D fixed_nv: specialised on 5
// vertices (pentagons).  3D nv: specialised kernels for 8 (cubes) and 20
// (dodecahedra) vertices, the generic one otherwise.
SetKernel set2d_f32_kernel(int G, bool fixed_nv);
SetKernel set2d_f64_kernel(int G, bool fixed_nv);
SetKernel set3d_f32_kernel(int G, int nv);
SetKernel set3d_f64_kernel(int G, int nv);
SetKernel set3d_f32_nv20(int G);
// 2D direct kernel (one lane per cell, no staging), FP32-filtered or plain FP64 form
SetKernel set2d_direct_kernel(bool fixed_nv, bool f32);
SetKernel set3d_f64_nv20(int G);

// select table of the latency-regime set kernels (selects.cu): bytes of one
// record, and the kernel that fills dv.msel for the running sweep
size_t select_record_bytes(int dim);
cudaError_t launch_selects(const Dev& dv, int dim, uint32_t grid, cudaStream_t st);

}  // namespace hpmc
