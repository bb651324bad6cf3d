// Host-side check of the shape constants the kernels rely on (test helper,
// built by tests/test_shape_host.py).  Reads "dim nv" and nv vertices of dim
// coordinates from stdin, runs build_shapes, and prints one line of
// key=value pairs.  3D: the return code, the box / central-symmetry /
// interior-origin flags, the box half extents, whether the FP32 copies are
// the vertices' casts in some order (and, for symmetric shapes, in pairs k,
// k + nv/2 of opposite sign), and the box test's FP32 and FP64 margins
// relative to the circumdiameter.  2D: the FP32 separating-axis margin for
// inputs that are FP32 casts of the FP64 ones.
#include <vector_types.h>

#include <cstdio>
#include <vector>

#include "hpmc_bounds.h"
#include "hpmc_shape.h"

int main()
{
    int dim = 0;
    unsigned nv = 0;
    if (std::scanf("%d %u", &dim, &nv) != 2 || (dim != 2 && dim != 3)) return 2;
    std::vector<double> v((size_t)dim * nv);
    for (size_t i = 0; i < v.size(); ++i)
        if (std::scanf("%lf", &v[i]) != 1) return 2;
    hpmc::Shape2 s2{};
    hpmc::Shape3 s3{};
    double Rc = 0.0, rc2 = 0.0;
    const int rc = hpmc::build_shapes(dim, v.data(), nv, s2, s3, Rc, rc2);
    std::printf("rc=%d", rc);
    if (rc) {
        std::printf("\n");
        return 0;
    }
    if (dim == 2) {
        hpmc::Margins g{};
        g.e_dlt = hpmc::kU32 * 2.0 * Rc * 1.01;
        g.e_ori = hpmc::kU32 * 1.01;
        double vm = 0.0, nm = 0.0, am = 0.0;
        for (int k = 0; k < s2.nv; ++k) {
            vm = std::fmax(vm, std::fmax(std::fabs(s2.vx[k]), std::fabs(s2.vy[k])));
            nm = std::fmax(nm, std::fmax(std::fabs(s2.nx[k]), std::fabs(s2.ny[k])));
            am = std::fmax(am, std::fmax(std::fabs(s2.alo[k]), std::fabs(s2.ahi[k])));
        }
        std::printf(" Rc=%.17g E=%.9g\n", Rc, hpmc::sat2_margin(g, Rc, vm, nm, am));
        return 0;
    }
    // the FP32 copies: a permutation of the casts
    bool perm = true;
    std::vector<int> used(nv, 0);
    for (unsigned k = 0; k < nv && perm; ++k) {
        bool found = false;
        for (unsigned i = 0; i < nv && !found; ++i)
            if (!used[i] && s3.fv[k][0] == (float)v[3 * i] && s3.fv[k][1] == (float)v[3 * i + 1] &&
                s3.fv[k][2] == (float)v[3 * i + 2]) {
                used[i] = 1;
                found = true;
            }
        perm = found;
    }
    bool pairs = true;
    if (s3.sym)
        for (unsigned k = 0; k < nv / 2; ++k)
            for (int a = 0; a < 3; ++a) pairs = pairs && s3.fv[k + nv / 2][a] == -s3.fv[k][a];
    std::printf(" box=%d sym=%d mpr=%d Rc=%.17g perm=%d pairs=%d bh=%.9g,%.9g,%.9g", s3.box, s3.sym, s3.mpr, Rc,
                perm ? 1 : 0, pairs ? 1 : 0, s3.bh[0], s3.bh[1], s3.bh[2]);
    if (s3.box) {
        hpmc::Margins g{};
        g.e_dlt = hpmc::kU32 * 2.0 * Rc * 1.01;     // an FP32 cast of a separation within 2R
        g.e_ori = hpmc::kU32 * 1.000001 + 2e-15;      // an FP32 cast of a unit quaternion
        const double h[3] = { std::fabs(s3.v[0][0]), std::fabs(s3.v[0][1]), std::fabs(s3.v[0][2]) };
        const double tau = 1e-9 * 2.0 * Rc;
        const hpmc::BoxMargins m32 = hpmc::box_sat_margins(g, Rc, h, tau);
        const hpmc::BoxMargins m64 = hpmc::box_sat_margins64(Rc, h, tau);
        std::printf(" sep32=%.9g ov32=%.9g sep64=%.9g ov64=%.9g", m32.sep / (2 * Rc), m32.ov / (2 * Rc),
                    m64.sep / (2 * Rc), m64.ov / (2 * Rc));
    }
    std::printf("\n");
    return 0;
}
