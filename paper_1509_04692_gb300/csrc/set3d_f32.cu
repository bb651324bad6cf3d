// Instantiations of the FP32-filtered 3D set kernel (certified FP32 GJK).
#include "hpmc_sweep3d.cuh"
#include "hpmc_launch.h"

namespace hpmc {

template <int G, int NV>
static SetKernel make3f()
{
    return { (const void*)&k_set3d<G, true, NV>, sizeof(Warp3<G, true>) };
}

SetKernel set3d_f32_kernel(int G, int nv)
{
    if (nv == 20) return set3d_f32_nv20(G);
    const bool fixed_nv = nv == 8;
    switch (G) {
    case 1: return fixed_nv ? make3f<1, 8>() : make3f<1, 0>();
    case 2: return fixed_nv ? make3f<2, 8>() : make3f<2, 0>();
    case 4: return fixed_nv ? make3f<4, 8>() : make3f<4, 0>();
    case 8: return fixed_nv ? make3f<8, 8>() : make3f<8, 0>();
    case 16: return fixed_nv ? make3f<16, 8>() : make3f<16, 0>();
    case 32: return fixed_nv ? make3f<32, 8>() : make3f<32, 0>();
    default: return { nullptr, 0 };
    }
}

}  // namespace hpmc
