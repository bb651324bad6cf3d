// selects.cu -- the state-independent part of every trial move of a sweep.
//
// Select k of cell c in checkerboard set sigma draws its Philox words from the
// counter (c, sweep, k, sigma) alone (Sec. 2.5.2: counter-based streams, one
// per cell and select), so its particle pick and its move deltas -- the
// translation, and the Cayley rotation (2D) or the normalised quaternion step
// (3D) of the FP64 contract, with their FP32 counterparts -- are known before
// any move of the sweep is made.  They cost FP64 uniforms, divisions and a
// square root.  On this GPU an FP64 warp instruction takes the same pipe time
// however few of its lanes are active, and inside the latency-regime set
// kernels (G >= 8 lanes per cell) only min(nselect, G) of G lanes carry one
// in a cell's first chunk of selects; here one thread computes one select, 32
// per warp instruction, for the whole sweep.  The host runs this kernel on a
// second stream while the cell list is rebuilt (after the shift kernel has
// advanced the sweep counter), and the set kernels load the records of their
// first chunk (later chunks keep all G lanes busy and are computed there).
#include "hpmc_launch.h"
#include "hpmc_sweep2d.cuh"
#include "hpmc_sweep3d.cuh"

namespace hpmc {

// record i = c * msel_stride + k of global cell c, msel_stride = min(largest
// nselect, G); selects k >= nselect of a replica with fewer selects than the
// stride are left unwritten (never read)
template <int DIM>
__global__ void __launch_bounds__(256) k_selects(Dev dv)
{
    const uint32_t stride = dv.msel_stride;
    const uint64_t total = min((uint64_t)dv.ctot * stride, dv.msel_n);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = (uint32_t)(i / stride);
        const uint32_t k = (uint32_t)(i - (uint64_t)c * stride);
        uint32_t lo = 0, hi = dv.R;                   // replica of cell c (cbase ascending)
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (dv.reps[mid].cbase <= c) lo = mid; else hi = mid;
        }
        const Rep& rp = dv.reps[lo];
        if (k >= rp.nselect) continue;
        const uint32_t cl = c - rp.cbase;
        const uint32_t nc0 = (uint32_t)rp.nc[0], nc1 = (uint32_t)rp.nc[1];
        const uint32_t ix = cl % nc0, iy = (cl / nc0) % nc1, iz = cl / (nc0 * nc1);
        const uint32_t sigma = (ix & 1u) | ((iy & 1u) << 1) | (DIM == 3 ? (iz & 1u) << 2 : 0u);
        const uint64_t sweep = dv.sweep[lo] - 1;      // the running sweep
        if constexpr (DIM == 2)
            static_cast<MoveData*>(dv.msel)[i] = precompute_select(rp, rp.seed, sweep, sigma, cl, k);
        else
            static_cast<MoveData3*>(dv.msel)[i] = precompute_select3(rp, rp.seed, sweep, sigma, cl, k);
    }
}

size_t select_record_bytes(int dim)
{
    return dim == 2 ? sizeof(MoveData) : sizeof(MoveData3);
}

cudaError_t launch_selects(const Dev& dv, int dim, uint32_t grid, cudaStream_t st)
{
    if (dim == 2) k_selects<2><<<grid, 256, 0, st>>>(dv);
    else k_selects<3><<<grid, 256, 0, st>>>(dv);
    return cudaGetLastError();
}

}  // namespace hpmc
