// Instantiations of the plain FP64 3D set kernel.
#include "hpmc_sweep3d.cuh"
#include "hpmc_launch.h"

namespace hpmc {

template <int G, int NV>
static SetKernel make3d()
{
    return { (const void*)&k_set3d<G, false, NV>, sizeof(Warp3<G, false>) };
}

SetKernel set3d_f64_kernel(int G, int nv)
{
    if (nv == 20) return set3d_f64_nv20(G);
    const bool fixed_nv = nv == 8;
    switch (G) {
    case 1: return fixed_nv ? make3d<1, 8>() : make3d<1, 0>();
    case 2: return fixed_nv ? make3d<2, 8>() : make3d<2, 0>();
    case 4: return fixed_nv ? make3d<4, 8>() : make3d<4, 0>();
    case 8: return fixed_nv ? make3d<8, 8>() : make3d<8, 0>();
    case 16: return fixed_nv ? make3d<16, 8>() : make3d<16, 0>();
    case 32: return fixed_nv ? make3d<32, 8>() : make3d<32, 0>();
    default: return { nullptr, 0 };
    }
}

}  // namespace hpmc
