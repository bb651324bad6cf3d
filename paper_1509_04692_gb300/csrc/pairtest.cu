// pairtest.cu -- hpmc_pair_test: the overlap test on independent pairs, in
// the FP64 contract and in the FP32 filter, for validation against the oracle.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "../../include/hpmc.h"
#include "hpmc_bounds.h"
#include "hpmc_device.cuh"
#include "hpmc_filter.cuh"
#include "hpmc_gjk32.cuh"
#include "hpmc_mpr32.cuh"
#include "hpmc_gjk64w.cuh"
#include "hpmc_shape.h"

namespace {

using namespace hpmc;

__global__ void k_pairs2d(Shape2 sh, float E, uint32_t n, const double* D, const double* qA, const double* qB,
                          int32_t* o64, int32_t* o32)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dx = D[2 * i], dy = D[2 * i + 1];
    const double ca = qA[2 * i], sa = qA[2 * i + 1], cb = qB[2 * i], sb = qB[2 * i + 1];
    o64[i] = overlap2d64<0>(sh, dx, dy, ca, sa, cb, sb) ? 1 : 0;
    if (sh.round) { o32[i] = 2; return; }            // disks: the set kernels' cull decides
    const int v = sat32<0>(sh, E, (float)dx, (float)dy, (float)ca, (float)sa, (float)cb, (float)sb);
    o32[i] = v == 1 ? 1 : (v == 0 ? 0 : 2);
}

__global__ void k_pairs3d(const __grid_constant__ Shape3 sh, float e_pb, float e_va, float tau, float box_sep,
                          float box_ov, uint32_t n, const double* D, const double* qA, const double* qB, int32_t* o64,
                          int32_t* o32)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double d[3] = { D[3 * i], D[3 * i + 1], D[3 * i + 2] };
    const double a[4] = { qA[4 * i], qA[4 * i + 1], qA[4 * i + 2], qA[4 * i + 3] };
    const double b[4] = { qB[4 * i], qB[4 * i + 1], qB[4 * i + 2], qB[4 * i + 3] };
    int it = 0;
    o64[i] = overlap3d64<0>(sh, d, a, b, &it) ? 1 : 0;
    if (sh.round) { o32[i] = 2; return; }            // spheres: the set kernels' cull decides
    const float4 fa = make_float4((float)a[0], (float)a[1], (float)a[2], (float)a[3]);
    const float4 fb = make_float4((float)b[0], (float)b[1], (float)b[2], (float)b[3]);
    const float dx = (float)d[0], dy = (float)d[1], dz = (float)d[2];
    const int v = sh.box  ? box32_sat(sh, dx, dy, dz, fa, fb, box_sep, box_ov)
                  : sh.mpr ? mpr32_cert<0>(sh, dx, dy, dz, fa, fb, e_pb, e_va, tau)
                           : gjk32_cert<0>(sh, dx, dy, dz, fa, fb, e_pb, e_va, tau);
    o32[i] = v;   // 0, 1, or the reason it is uncertain (>= 2)
}

// one warp per pair: the warp-cooperative FP64 GJK the FP32-filtered 3D
// kernels use for their re-checks
__global__ void k_pairs3d_warp(const __grid_constant__ Shape3 sh, uint32_t n, const double* D, const double* qA,
                               const double* qB, int32_t* o64, int32_t* oit)
{
    const uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;                               // whole warps leave together
    const double d[3] = { D[3 * i], D[3 * i + 1], D[3 * i + 2] };
    const double a[4] = { qA[4 * i], qA[4 * i + 1], qA[4 * i + 2], qA[4 * i + 3] };
    const double b[4] = { qB[4 * i], qB[4 * i + 1], qB[4 * i + 2], qB[4 * i + 3] };
    int it = 0;
    const bool ov = overlap3d64_warp<0>(sh, d, a, b, &it);
    if ((threadIdx.x & 31) == 0) {
        o64[i] = ov ? 1 : 0;
        oit[i] = it;
    }
}

// one warp per pair: the FP64 box certificate of the FP32-filtered sweep's
// re-checks (0 separated, 1 overlap, 2 left to the GJK)
__global__ void k_pairs_box64(const __grid_constant__ Shape3 sh, double sep, double ov, uint32_t n, const double* D,
                              const double* qA, const double* qB, int32_t* out)
{
    const uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;                               // whole warps leave together
    const double d[3] = { D[3 * i], D[3 * i + 1], D[3 * i + 2] };
    const double a[4] = { qA[4 * i], qA[4 * i + 1], qA[4 * i + 2], qA[4 * i + 3] };
    const double b[4] = { qB[4 * i], qB[4 * i + 1], qB[4 * i + 2], qB[4 * i + 3] };
    const int v = box64_sat_warp(sh, d, a, b, sep, ov);
    if ((threadIdx.x & 31) == 0) out[i] = v;
}

float up32(double x)
{
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
}

}  // namespace

extern "C" int hpmc_pair_test(int dim, const double* verts, uint32_t nv, uint32_t n, const double* D,
                              const double* qA, const double* qB, int32_t* out64, int32_t* out32)
{
    if (!D || !qA || !qB || !out64 || !out32) return HPMC_ERR_INVALID_ARG;
    Shape2 s2{};
    Shape3 s3{};
    double Rc = 0.0, rc2 = 0.0;
    int rc = build_shapes(dim, verts, nv, s2, s3, Rc, rc2);
    if (rc) return rc;
    if (n == 0) return 0;
    const int qd = dim == 2 ? 2 : 4;
    // FP32 inputs are plain casts of the FP64 ones: errors of one rounding
    Margins g{};
    g.e_dlt = kU32 * 2.0 * Rc * 1.01;
    g.e_ori = kU32 * 1.01;
    double vm = 0.0, nm = 0.0, am = 0.0;
    if (dim == 2) {
        for (int k = 0; k < s2.nv; ++k) {
            vm = std::fmax(vm, std::fmax(std::fabs(s2.vx[k]), std::fabs(s2.vy[k])));
            nm = std::fmax(nm, std::fmax(std::fabs(s2.nx[k]), std::fabs(s2.ny[k])));
            am = std::fmax(am, std::fmax(std::fabs(s2.alo[k]), std::fabs(s2.ahi[k])));
        }
    } else {
        for (int k = 0; k < s3.nv; ++k)
            for (int a = 0; a < 3; ++a) vm = std::fmax(vm, std::fabs(s3.v[k][a]));
    }
    double *dD = nullptr, *dA = nullptr, *dB = nullptr;
    int32_t *d64 = nullptr, *d32 = nullptr;
    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&dD, sizeof(double) * n * dim);
    if (e == cudaSuccess) e = cudaMalloc(&dA, sizeof(double) * n * qd);
    if (e == cudaSuccess) e = cudaMalloc(&dB, sizeof(double) * n * qd);
    if (e == cudaSuccess) e = cudaMalloc(&d64, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d32, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMemcpy(dD, D, sizeof(double) * n * dim, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dA, qA, sizeof(double) * n * qd, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, qB, sizeof(double) * n * qd, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int T = 128;
        if (dim == 2) {
            const float E = up32(sat2_margin(g, Rc, vm, nm, am));
            k_pairs2d<<<(n + T - 1) / T, T>>>(s2, E, n, dD, dA, dB, d64, d32);
        } else {
            const float epb = up32(gjk3_vertex_margin(g, Rc, vm));
            const float tau = up32(1e-9 * 2.0 * Rc);
            // the box margins assume |D| <= 2R: here R covers the longest D
            // given (the sweeps only test pairs their cull keeps)
            double dm = 0.0;
            for (uint32_t i = 0; i < n; ++i)
                dm = std::fmax(dm, std::sqrt(D[3 * i] * D[3 * i] + D[3 * i + 1] * D[3 * i + 1] + D[3 * i + 2] * D[3 * i + 2]));
            const double Rb = std::fmax(Rc, 0.5 * dm * (1.0 + 1e-6));
            Margins gb = g;
            gb.e_dlt = kU32 * 2.0 * Rb * 1.01;
            const double bh[3] = { std::fabs(s3.v[0][0]), std::fabs(s3.v[0][1]), std::fabs(s3.v[0][2]) };
            const BoxMargins bm = box_sat_margins(gb, Rb, bh, (double)tau);
            k_pairs3d<<<(n + T - 1) / T, T>>>(s3, epb, up32(2.0 * kU32 * vm), tau, up32(bm.sep), up32(bm.ov), n, dD,
                                              dA, dB, d64, d32);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out64, d64, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out32, d32, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    cudaFree(dD);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(d64);
    cudaFree(d32);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? HPMC_ERR_OOM : HPMC_ERR_CUDA;
    }
    return 0;
}

extern "C" int hpmc_pair_test_warp3d(const double* verts, uint32_t nv, uint32_t n, const double* D,
                                     const double* qA, const double* qB, int32_t* out64, int32_t* iters)
{
    if (!D || !qA || !qB || !out64 || !iters) return HPMC_ERR_INVALID_ARG;
    Shape2 s2{};
    Shape3 s3{};
    double Rc = 0.0, rc2 = 0.0;
    int rc = build_shapes(3, verts, nv, s2, s3, Rc, rc2);
    if (rc) return rc;
    if (n == 0) return 0;
    double *dD = nullptr, *dA = nullptr, *dB = nullptr;
    int32_t *d64 = nullptr, *dit = nullptr;
    cudaError_t e = cudaMalloc(&dD, sizeof(double) * n * 3);
    if (e == cudaSuccess) e = cudaMalloc(&dA, sizeof(double) * n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dB, sizeof(double) * n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d64, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dit, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMemcpy(dD, D, sizeof(double) * n * 3, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dA, qA, sizeof(double) * n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, qB, sizeof(double) * n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const uint32_t wpb = 4;
        k_pairs3d_warp<<<(n + wpb - 1) / wpb, 32 * wpb>>>(s3, n, dD, dA, dB, d64, dit);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out64, d64, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(iters, dit, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    cudaFree(dD);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(d64);
    cudaFree(dit);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? HPMC_ERR_OOM : HPMC_ERR_CUDA;
    }
    return 0;
}

extern "C" int hpmc_pair_test_box64(const double* verts, uint32_t nv, uint32_t n, const double* D, const double* qA,
                                    const double* qB, int32_t* out)
{
    if (!D || !qA || !qB || !out) return HPMC_ERR_INVALID_ARG;
    Shape2 s2{};
    Shape3 s3{};
    double Rc = 0.0, rc2 = 0.0;
    int rc = build_shapes(3, verts, nv, s2, s3, Rc, rc2);
    if (rc) return rc;
    if (!s3.box) return HPMC_ERR_INVALID_ARG;
    if (n == 0) return 0;
    // margins for the longest D given (the sweeps only test culled pairs)
    double dm = 0.0;
    for (uint32_t i = 0; i < n; ++i)
        dm = std::fmax(dm, std::sqrt(D[3 * i] * D[3 * i] + D[3 * i + 1] * D[3 * i + 1] + D[3 * i + 2] * D[3 * i + 2]));
    const double Rb = std::fmax(Rc, 0.5 * dm * (1.0 + 1e-6));
    const double bh[3] = { std::fabs(s3.v[0][0]), std::fabs(s3.v[0][1]), std::fabs(s3.v[0][2]) };
    const BoxMargins bm = box_sat_margins64(Rb, bh, (double)up32(1e-9 * 2.0 * Rc));
    double *dD = nullptr, *dA = nullptr, *dB = nullptr;
    int32_t* dO = nullptr;
    cudaError_t e = cudaMalloc(&dD, sizeof(double) * n * 3);
    if (e == cudaSuccess) e = cudaMalloc(&dA, sizeof(double) * n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dB, sizeof(double) * n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dO, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMemcpy(dD, D, sizeof(double) * n * 3, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dA, qA, sizeof(double) * n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, qB, sizeof(double) * n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const uint32_t wpb = 4;
        k_pairs_box64<<<(n + wpb - 1) / wpb, 32 * wpb>>>(s3, bm.sep, bm.ov, n, dD, dA, dB, dO);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dO, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    cudaFree(dD);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dO);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? HPMC_ERR_OOM : HPMC_ERR_CUDA;
    }
    return 0;
}
