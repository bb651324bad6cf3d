// Instantiations of the FP32-filtered 2D set kernel.
#include "hpmc_sweep2d.cuh"
#include "hpmc_launch.h"

namespace hpmc {

template <int G, int NV>
static SetKernel make2f()
{
    return { (const void*)&k_set2d<G, true, NV>, sizeof(Warp2<G, true>) };
}

SetKernel set2d_f32_kernel(int G, bool fixed_nv)
{
    switch (G) {
    case 1: return fixed_nv ? make2f<1, 5>() : make2f<1, 0>();
    case 2: return fixed_nv ? make2f<2, 5>() : make2f<2, 0>();
    case 4: return fixed_nv ? make2f<4, 5>() : make2f<4, 0>();
    case 8: return fixed_nv ? make2f<8, 5>() : make2f<8, 0>();
    case 16: return fixed_nv ? make2f<16, 5>() : make2f<16, 0>();
    case 32: return fixed_nv ? make2f<32, 5>() : make2f<32, 0>();
    default: return { nullptr, 0 };
    }
}

}  // namespace hpmc
