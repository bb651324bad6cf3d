// Instantiations of the plain FP64 2D set kernel.
#include "hpmc_sweep2d.cuh"
#include "hpmc_launch.h"

namespace hpmc {

template <int G, int NV>
static SetKernel make2d()
{
    return { (const void*)&k_set2d<G, false, NV>, sizeof(Warp2<G, false>) };
}

SetKernel set2d_f64_kernel(int G, bool fixed_nv)
{
    switch (G) {
    case 1: return fixed_nv ? make2d<1, 5>() : make2d<1, 0>();
    case 2: return fixed_nv ? make2d<2, 5>() : make2d<2, 0>();
    case 4: return fixed_nv ? make2d<4, 5>() : make2d<4, 0>();
    case 8: return fixed_nv ? make2d<8, 5>() : make2d<8, 0>();
    case 16: return fixed_nv ? make2d<16, 5>() : make2d<16, 0>();
    case 32: return fixed_nv ? make2d<32, 5>() : make2d<32, 0>();
    default: return { nullptr, 0 };
    }
}

}  // namespace hpmc
