// 3D (convex polyhedra): overlap-check kernel.
#include "hpmc_device.cuh"
#include "hpmc_launch.h"

namespace hpmc {

// Count overlapping pairs of the sorted buffer `b` (lower tag counts the pair)
// with the FP64 contract: circumsphere cull, then GJK.
template <int NV>
__global__ void k_check3d(Dev dv, Shape3 sh, int b, int32_t only_r, unsigned long long* out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.ntot) return;
    const uint32_t r = dv.rep_of[i];
    if (only_r >= 0 && (int32_t)r != only_r) return;
    const Rep& rp = dv.reps[r];
    const Bufs& B = dv.buf[b];
    const int ix = cell_axis(B.px[i], dv.shift[3 * r], rp.L[0], rp.inv_w[0], rp.nc[0]);
    const int iy = cell_axis(B.py[i], dv.shift[3 * r + 1], rp.L[1], rp.inv_w[1], rp.nc[1]);
    const int iz = cell_axis(B.pz[i], dv.shift[3 * r + 2], rp.L[2], rp.inv_w[2], rp.nc[2]);
    const uint32_t ti = B.tag[i];
    const double qA[4] = { B.q0[i], B.q1[i], B.q2[i], B.q3[i] };
    unsigned long long n = 0;
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                const int jx = (ix + ox + rp.nc[0]) % rp.nc[0];
                const int jy = (iy + oy + rp.nc[1]) % rp.nc[1];
                const int jz = (iz + oz + rp.nc[2]) % rp.nc[2];
                const uint32_t cc = rp.cbase + (uint32_t)jx +
                                    (uint32_t)rp.nc[0] * ((uint32_t)jy + (uint32_t)rp.nc[1] * (uint32_t)jz);
                for (uint32_t e = dv.start[cc]; e < dv.start[cc + 1]; ++e) {
                    if (B.tag[e] <= ti) continue;
                    double D[3];
                    D[0] = min_image(B.px[e] - B.px[i], rp.L[0], rp.halfL[0]);
                    D[1] = min_image(B.py[e] - B.py[i], rp.L[1], rp.halfL[1]);
                    D[2] = min_image(B.pz[e] - B.pz[i], rp.L[2], rp.halfL[2]);
                    if ((D[0] * D[0] + D[1] * D[1]) + D[2] * D[2] > sh.rc2) continue;
                    const double qB[4] = { B.q0[e], B.q1[e], B.q2[e], B.q3[e] };
                    int it = 0;
                    if (overlap3d64<NV>(sh, D, qA, qB, &it)) n += 1;
                }
            }
    if (n) atomicAdd(out, n);
}

}  // namespace hpmc

int hpmc_check3d_launch(const hpmc::Dev& dv, const hpmc::Shape3& sh, int b, int32_t r,
                        unsigned long long* out, uint32_t ntot)
{
    const int T = 128;
    if (sh.nv == 8) hpmc::k_check3d<8><<<(ntot + T - 1) / T, T>>>(dv, sh, b, r, out);
    else hpmc::k_check3d<0><<<(ntot + T - 1) / T, T>>>(dv, sh, b, r, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -5;
}
