// Instantiations of the FP32-filtered 3D set kernel for 20-vertex polyhedra
// (the regular dodecahedron), in a translation unit of their own so that
// the build compiles them in parallel with the others.
#include "hpmc_sweep3d.cuh"
#include "hpmc_launch.h"

namespace hpmc {

template <int G>
static SetKernel make20()
{
    return { (const void*)&k_set3d<G, true, 20>, sizeof(Warp3<G, true>) };
}

SetKernel set3d_f32_nv20(int G)
{
    switch (G) {
    case 1: return make20<1>();
    case 2: return make20<2>();
    case 4: return make20<4>();
    case 8: return make20<8>();
    case 16: return make20<16>();
    case 32: return make20<32>();
    default: return { nullptr, 0 };
    }
}

}  // namespace hpmc
