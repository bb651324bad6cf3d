/*
 * hpmc_oracle.c -- plain, slow CPU oracle for the checkerboard hard-particle
 * Metropolis Monte Carlo sweep (Anderson, Irrgang & Glotzer, "Scalable
 * Metropolis Monte Carlo for simulation of hard shapes").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference against which the
 * CUDA library is checked.  Only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * Everything is FP64 and uses only +, -, *, / and sqrt (plus tan() once, on the
 * host, for the rotation half-width); build with -O2 -ffp-contract=off and no
 * fast-math so that every operation is a single IEEE round-to-nearest step.
 *
 * Paper passages followed:
 *   Sec. 2.1        Metropolis steps: select, trial move r+dr and q*dq, overlap
 *                   check against all others, reject on the first overlap.
 *   Sec. 2.2.1      Cell list: cell width >= d_max, bucket sort, 3^d stencil.
 *   Sec. 2.3, Eq. 2 Overlap test in the frame of particle A; support function
 *                   of B-A; separating-axis test for convex polygons.
 *   Sec. 2.5        Counter/hash based random streams keyed per trial move.
 *   Sec. 2.5.1      Random displacement of the whole system between steps
 *                   (here: a random shift of the cell grid).
 *   Sec. 2.5.2      2^d colour checkerboard; moves that leave the active cell
 *                   are rejected; one set of cells moves at a time.
 * Where the paper is silent the oracle follows the readings listed in the
 * header comments below (philox counter layout, move distributions, ties).
 *
 * The cells of one checkerboard set never touch one another, so or_sweep can
 * share them out over host threads (or_set_threads; serial by default) with
 * a trajectory identical byte for byte to the serial one.
 *
 * Parity status: every function here is pinned by the CPU tests (Philox
 * known-answer vectors, brute-force polygon/polyhedron predicates, SAT-15 for
 * boxes, ideal-gas closed forms in 2D and 3D, move distributions, O(N^2)
 * no-overlap, zero net probability current of one-particle chains in 2D and
 * 3D (detailed balance), the two-pentagon pair-distance law, the exact
 * one-move acceptance probability of a pentagon beside another (Minkowski
 * sum overlap region integrated against the in-cell probability); for
 * disks/spheres the contact definition, lattice closed forms of the
 * scale-distribution histogram and the dilute disk and sphere virial series; for
 * volume moves the ideal-gas Gamma law).
 */
#define _POSIX_C_SOURCE 200809L
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXV 64
#define OR_GJK_MAXIT 32

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), written from the      */
/* published definition: 10 rounds of two 32x32->64 multiplies with key      */
/* bumps by the Weyl constants between rounds.                              */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* u in [0,1) from the top 53 bits of the 64-bit word (a<<32 | b); exact. */
double or_u53(uint32_t a, uint32_t b)
{
    uint64_t m = (((uint64_t)a << 32) | (uint64_t)b) >> 11;
    return (double)m * (1.0 / 9007199254740992.0);
}

/* Stream layouts (reading of Sec. 2.5: one independent stream per trial move,
 * keyed here by seed, sweep, set, cell and select).
 *   key     = (lo32(seed), hi32(seed))
 *   move    : ctr = (cell, lo32(sweep), (hi32(sweep) << 16) | k, (1<<24)|(set<<16)|block)
 *   shift   : ctr = (0,    lo32(sweep), (hi32(sweep) << 16),     (2<<24)|block)      */
static void or_move_block(uint64_t seed, uint64_t sweep, uint32_t set, uint32_t cell,
                          uint32_t k, uint32_t block, uint32_t out[4])
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { cell, (uint32_t)sweep, ((uint32_t)(sweep >> 32) << 16) | k,
                        (1u << 24) | (set << 16) | block };
    or_philox4x32_10(ctr, key, out);
}

static void or_shift_block(uint64_t seed, uint64_t sweep, uint32_t block, uint32_t out[4])
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { 0u, (uint32_t)sweep, ((uint32_t)(sweep >> 32) << 16), (2u << 24) | block };
    or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* System description                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dim;                    /* 2 or 3 */
    double L[3], halfL[3];      /* box lengths (orthorhombic, periodic) */
    int nc[3];                  /* cells per axis (even, >= 4) */
    double w[3], inv_w[3];      /* cell width and nc/L */
    double wcell_min;           /* max(2R, w_min): the narrowest allowed cell */
    int nv;                     /* vertices of the (single) shape; 0: disk/sphere */
    double v[OR_MAXV][3];       /* local-frame vertices */
    double R;                   /* circumradius */
    double rc2;                 /* (2R)^2: circumsphere cull threshold */
    /* 2D separating-axis constants: outward edge normals and A's own
     * projection interval on each of them. */
    double nrm[OR_MAXV][2];
    double alo[OR_MAXV], ahi[OR_MAXV];
    /* trial move parameters */
    double d, a, tau;
    uint32_t nselect;
    uint64_t seed;
    int nthreads;               /* host threads sharing a set's cells (<= 1: serial) */
} or_system;

size_t or_system_size(void) { return sizeof(or_system); }

/* Cell list geometry (Sec. 2.2.1): the shortest cell side must be at least
 * d_max = 2R.  Reading: ncell = floor(L / max(2R, w_min)), made even (for the
 * 2^d colouring) and required >= 4 (unique minimum image inside a stencil). */
/* nv = 0 selects hard disks (2D) or spheres (3D) of radius verts[0] (the
 * paper's validation systems, Sec. 4): the shape is its own circumsphere. */
int or_init(or_system* s, int dim, const double* L, const double* verts, int nv, double w_min)
{
    memset(s, 0, sizeof(*s));
    if (dim != 2 && dim != 3) return -1;
    if (nv != 0 && (nv < 3 || nv > OR_MAXV)) return -1;
    s->dim = dim;
    s->nv = nv;
    for (int i = 0; i < nv; ++i)
        for (int k = 0; k < dim; ++k) s->v[i][k] = verts[i * dim + k];
    double r2 = 0.0;
    for (int i = 0; i < nv; ++i) {
        double q = s->v[i][0] * s->v[i][0] + s->v[i][1] * s->v[i][1];
        if (dim == 3) q = q + s->v[i][2] * s->v[i][2];
        if (q > r2) r2 = q;
    }
    if (nv == 0) {
        if (!(verts[0] > 0.0)) return -1;
        r2 = verts[0] * verts[0];
    }
    s->R = nv == 0 ? verts[0] : sqrt(r2);
    double dcut = s->R + s->R;
    s->rc2 = dcut * dcut;
    double wmin = dcut > w_min ? dcut : w_min;
    s->wcell_min = wmin;
    for (int k = 0; k < dim; ++k) {
        if (!(L[k] > 0.0)) return -1;
        s->L[k] = L[k];
        s->halfL[k] = 0.5 * L[k];
        int n = (int)floor(L[k] / wmin);
        if (n % 2) n -= 1;
        if (n < 4) return -2;
        s->nc[k] = n;
        s->w[k] = L[k] / (double)n;
        s->inv_w[k] = (double)n / L[k];
    }
    if (dim == 2 && nv > 0) {
        /* convex, counter-clockwise polygon: every turn must be strictly left */
        for (int i = 0; i < nv; ++i) {
            const double* p0 = s->v[i];
            const double* p1 = s->v[(i + 1) % nv];
            const double* p2 = s->v[(i + 2) % nv];
            double cr = (p1[0] - p0[0]) * (p2[1] - p1[1]) - (p1[1] - p0[1]) * (p2[0] - p1[0]);
            if (!(cr > 0.0)) return -1;
        }
        for (int k = 0; k < nv; ++k) {
            const double* p = s->v[k];
            const double* q = s->v[(k + 1) % nv];
            s->nrm[k][0] = q[1] - p[1];          /* e_y        */
            s->nrm[k][1] = p[0] - q[0];          /* -e_x       */
            double lo = 0.0, hi = 0.0;
            for (int i = 0; i < nv; ++i) {
                double t = s->nrm[k][0] * s->v[i][0] + s->nrm[k][1] * s->v[i][1];
                if (i == 0 || t < lo) lo = t;
                if (i == 0 || t > hi) hi = t;
            }
            s->alo[k] = lo;
            s->ahi[k] = hi;
        }
    }
    return 0;
}

/* Reading of Sec. 2.1 "small random trial move": translation uniform in
 * [-d, d)^dim; rotation by a Cayley/half-angle tangent t uniform in
 * [-tan(a/2), tan(a/2)) per rotation axis, so a 2D rotation never exceeds a. */
int or_set_moves(or_system* s, double d, double a, uint32_t nselect, uint64_t seed)
{
    if (!(d >= 0.0) || !(a >= 0.0) || nselect == 0 || nselect > 65535) return -1;
    s->d = d;
    s->a = a;
    s->tau = tan(0.5 * a);
    s->nselect = nselect;
    s->seed = seed;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Grid shift and cell assignment                                            */
/* ------------------------------------------------------------------------ */

/* Sec. 2.5.1: one random displacement of the whole system per step.  Reading:
 * shift the cell grid origin by s in [0, w)^dim instead of moving particles. */
void or_grid_shift(const or_system* s, uint64_t sweep, double sh[3])
{
    uint32_t r[4];
    or_shift_block(s->seed, sweep, 0, r);
    sh[0] = s->w[0] * or_u53(r[0], r[1]);
    sh[1] = s->w[1] * or_u53(r[2], r[3]);
    sh[2] = 0.0;
    if (s->dim == 3) {
        or_shift_block(s->seed, sweep, 1, r);
        sh[2] = s->w[2] * or_u53(r[0], r[1]);
    }
}

/* Cell index of one coordinate: truncation of (x - shift) * nc/L after
 * wrapping into [0, L); an index that rounds up to nc is clamped to nc-1. */
static int or_cell_axis(const or_system* s, int k, double x, double shift)
{
    double y = x - shift;
    if (y < 0.0) y = y + s->L[k];
    int i = (int)(y * s->inv_w[k]);
    if (i >= s->nc[k]) i = s->nc[k] - 1;
    return i;
}

int or_cell_of(const or_system* s, const double sh[3], const double* x, int idx[3])
{
    idx[2] = 0;
    for (int k = 0; k < s->dim; ++k) idx[k] = or_cell_axis(s, k, x[k], sh[k]);
    return idx[0] + s->nc[0] * (idx[1] + s->nc[1] * idx[2]);
}

static int or_ncells(const or_system* s)
{
    return s->nc[0] * s->nc[1] * (s->dim == 3 ? s->nc[2] : 1);
}

/* Cell list by bucket sort (Sec. 2.2.1).  Reading: inside a cell the list is
 * in ascending tag order.  Outputs start[C+1] and idx[N]. */
void or_build_cells(const or_system* s, uint32_t N, const double* pos, const double sh[3],
                    uint32_t* start, uint32_t* idx, int* cell_of_tag)
{
    int C = or_ncells(s);
    for (int c = 0; c <= C; ++c) start[c] = 0;
    for (uint32_t t = 0; t < N; ++t) {
        int ci[3];
        int c = or_cell_of(s, sh, pos + (size_t)t * s->dim, ci);
        cell_of_tag[t] = c;
        start[c + 1] += 1;
    }
    for (int c = 0; c < C; ++c) start[c + 1] += start[c];
    uint32_t* fill = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(C > 0 ? C : 1));
    for (int c = 0; c < C; ++c) fill[c] = start[c];
    for (uint32_t t = 0; t < N; ++t) idx[fill[cell_of_tag[t]]++] = t;
    free(fill);
}

/* ------------------------------------------------------------------------ */
/* Overlap test, 2D: separating axes of two convex polygons (Sec. 2.3),      */
/* evaluated in the frame of particle A.                                     */
/* ------------------------------------------------------------------------ */

/* B placed in A's frame by rotation (cr, sr) and offset (lx, ly); tests the
 * edge normals of A.  Returns 1 when one of them separates. */
static int or_sat_half(const or_system* s, double cr, double sr, double lx, double ly)
{
    double px[OR_MAXV], py[OR_MAXV];
    for (int i = 0; i < s->nv; ++i) {
        px[i] = (cr * s->v[i][0] - sr * s->v[i][1]) + lx;
        py[i] = (sr * s->v[i][0] + cr * s->v[i][1]) + ly;
    }
    for (int k = 0; k < s->nv; ++k) {
        double lo = 0.0, hi = 0.0;
        for (int i = 0; i < s->nv; ++i) {
            double t = s->nrm[k][0] * px[i] + s->nrm[k][1] * py[i];
            if (i == 0 || t < lo) lo = t;
            if (i == 0 || t > hi) hi = t;
        }
        if (s->ahi[k] < lo || hi < s->alo[k]) return 1;
    }
    return 0;
}

/* D(Delta, zA, zB): Delta = r_B - r_A (minimum image), z = (cos, sin).
 * Returns 1 for overlap (touching counts as overlap), 0 when separated. */
int or_overlap_2d(const or_system* s, const double D[2], const double zA[2], const double zB[2])
{
    if (s->nv == 0) return (D[0] * D[0] + D[1] * D[1]) <= s->rc2;    /* disks: distance <= 2R */
    double cA = zA[0], sA = zA[1], cB = zB[0], sB = zB[1];
    double cr = cA * cB + sA * sB;
    double sr = cA * sB - sA * cB;
    double lx = cA * D[0] + sA * D[1];
    double ly = cA * D[1] - sA * D[0];
    if (or_sat_half(s, cr, sr, lx, ly)) return 0;
    double mx = cB * D[0] + sB * D[1];
    double my = cB * D[1] - sB * D[0];
    if (or_sat_half(s, cr, -sr, -mx, -my)) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Overlap test, 3D: boolean GJK on the Minkowski difference B - A in A's     */
/* frame, support function of Eq. 2 with B's vertices moved into A's frame    */
/* once per pair.  Quaternions are (w, x, y, z).                              */
/* ------------------------------------------------------------------------ */
static void or_qmul(const double a[4], const double b[4], double o[4])
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

/* rotate v by unit quaternion q:  t = 2 (q_v x v);  v' = v + w t + q_v x t */
static void or_qrot(const double q[4], const double v[3], double o[3])
{
    double tx = 2.0 * (q[2] * v[2] - q[3] * v[1]);
    double ty = 2.0 * (q[3] * v[0] - q[1] * v[2]);
    double tz = 2.0 * (q[1] * v[1] - q[2] * v[0]);
    o[0] = (v[0] + q[0] * tx) + (q[2] * tz - q[3] * ty);
    o[1] = (v[1] + q[0] * ty) + (q[3] * tx - q[1] * tz);
    o[2] = (v[2] + q[0] * tz) + (q[1] * ty - q[2] * tx);
}

static double or_dot3(const double a[3], const double b[3])
{
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

static void or_cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static void or_sub3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}

typedef struct {
    const or_system* s;
    double pb[OR_MAXV][3];      /* B's vertices in A's frame */
} or_gjk_pair;

/* support of B - A in direction d: argmax over B's vertices of p.d minus the
 * argmin over A's local vertices of v.d; ties go to the lowest index. */
static void or_support(const or_gjk_pair* g, const double d[3], double out[3])
{
    const or_system* s = g->s;
    int ib = 0, ia = 0;
    double best = or_dot3(g->pb[0], d);
    for (int i = 1; i < s->nv; ++i) {
        double t = or_dot3(g->pb[i], d);
        if (t > best) { best = t; ib = i; }
    }
    double least = or_dot3(s->v[0], d);
    for (int j = 1; j < s->nv; ++j) {
        double t = or_dot3(s->v[j], d);
        if (t < least) { least = t; ia = j; }
    }
    or_sub3(g->pb[ib], s->v[ia], out);
}

static void or_neg3(const double a[3], double o[3])
{
    o[0] = -a[0]; o[1] = -a[1]; o[2] = -a[2];
}

/* Closest point to the origin of segment [a, b].  Returns the feature as a
 * bit mask over (a=1, b=2). */
static int or_closest_seg(const double a[3], const double b[3], double out[3])
{
    double ab[3], ap[3];
    or_sub3(b, a, ab);
    or_neg3(a, ap);
    double tn = or_dot3(ab, ap);
    if (tn <= 0.0) { memcpy(out, a, 3 * sizeof(double)); return 1; }
    double den = or_dot3(ab, ab);
    if (tn >= den) { memcpy(out, b, 3 * sizeof(double)); return 2; }
    double t = tn / den;
    out[0] = a[0] + t * ab[0];
    out[1] = a[1] + t * ab[1];
    out[2] = a[2] + t * ab[2];
    return 3;
}

/* Closest point to the origin of triangle (a, b, c) by the Voronoi regions
 * of its vertices, edges and face.  Feature mask over (a=1, b=2, c=4);
 * returns 0 for a degenerate face (zero barycentric denominator). */
static int or_closest_tri(const double a[3], const double b[3], const double c[3], double out[3])
{
    double ab[3], ac[3], ap[3], bp[3], cp[3];
    or_sub3(b, a, ab);
    or_sub3(c, a, ac);
    or_neg3(a, ap);
    double d1 = or_dot3(ab, ap);
    double d2 = or_dot3(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) { memcpy(out, a, 3 * sizeof(double)); return 1; }
    or_neg3(b, bp);
    double d3 = or_dot3(ab, bp);
    double d4 = or_dot3(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) { memcpy(out, b, 3 * sizeof(double)); return 2; }
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
        double t = d1 / (d1 - d3);
        out[0] = a[0] + t * ab[0]; out[1] = a[1] + t * ab[1]; out[2] = a[2] + t * ab[2];
        return 3;
    }
    or_neg3(c, cp);
    double d5 = or_dot3(ab, cp);
    double d6 = or_dot3(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) { memcpy(out, c, 3 * sizeof(double)); return 4; }
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
        double t = d2 / (d2 - d6);
        out[0] = a[0] + t * ac[0]; out[1] = a[1] + t * ac[1]; out[2] = a[2] + t * ac[2];
        return 5;
    }
    double va = d3 * d6 - d5 * d4;
    double e43 = d4 - d3, e56 = d5 - d6;
    if (va <= 0.0 && e43 >= 0.0 && e56 >= 0.0) {
        double t = e43 / (e43 + e56);
        double bc[3];
        or_sub3(c, b, bc);
        out[0] = b[0] + t * bc[0]; out[1] = b[1] + t * bc[1]; out[2] = b[2] + t * bc[2];
        return 6;
    }
    double sum = (va + vb) + vc;
    if (!(sum > 0.0)) return 0;
    double den = 1.0 / sum;
    double v = vb * den, w = vc * den;
    out[0] = (a[0] + ab[0] * v) + ac[0] * w;
    out[1] = (a[1] + ab[1] * v) + ac[1] * w;
    out[2] = (a[2] + ab[2] * v) + ac[2] * w;
    return 7;
}

/* Is the origin strictly on the other side of plane (p, q, r) from s? */
static int or_origin_outside(const double p[3], const double q[3], const double r[3], const double s[3])
{
    double pq[3], pr[3], ps[3], po[3], n[3];
    or_sub3(q, p, pq);
    or_sub3(r, p, pr);
    or_cross3(pq, pr, n);
    or_neg3(p, po);
    or_sub3(s, p, ps);
    double sp = or_dot3(po, n);
    double sd = or_dot3(ps, n);
    return (sp > 0.0 && sd < 0.0) || (sp < 0.0 && sd > 0.0);
}

/* Reduce simplex sp[0..n-1] (insertion order) to the feature nearest the
 * origin; v receives the nearest point.  Returns 1 when the origin is inside
 * the tetrahedron or the face is degenerate (both count as overlap). */
static int or_gjk_reduce(double sp[4][3], int* n, double v[3])
{
    int mask = 0;
    if (*n == 2) {
        mask = or_closest_seg(sp[0], sp[1], v);
    } else if (*n == 3) {
        mask = or_closest_tri(sp[0], sp[1], sp[2], v);
        if (mask == 0) return 1;
    } else {
        static const int F[4][4] = { { 0, 1, 2, 3 }, { 0, 1, 3, 2 }, { 0, 2, 3, 1 }, { 1, 2, 3, 0 } };
        int found = 0;
        double best = 0.0;
        for (int f = 0; f < 4; ++f) {
            const int* ix = F[f];
            if (!or_origin_outside(sp[ix[0]], sp[ix[1]], sp[ix[2]], sp[ix[3]])) continue;
            double pt[3];
            int m = or_closest_tri(sp[ix[0]], sp[ix[1]], sp[ix[2]], pt);
            if (m == 0) return 1;
            double dd = or_dot3(pt, pt);
            if (!found || dd < best) {
                found = 1;
                best = dd;
                memcpy(v, pt, sizeof pt);
                mask = 0;
                for (int k = 0; k < 3; ++k) if (m & (1 << k)) mask |= 1 << ix[k];
            }
        }
        if (!found) return 1;
    }
    int m = 0;
    for (int k = 0; k < *n; ++k) {
        if (mask & (1 << k)) {
            if (m != k) memcpy(sp[m], sp[k], sizeof sp[0]);
            m += 1;
        }
    }
    *n = m;
    return 0;
}

/* D(Delta, qA, qB) for convex polyhedra: GJK distance iteration on B - A
 * with the boolean exits of an intersection query.  v is the point of the
 * current simplex nearest the origin; w = S(-v) is a new support point.
 * v.w > 0 gives a separating plane (separated); v = 0 or the origin inside
 * the simplex means overlap; 32 iterations without a verdict count as
 * overlap.  Returns 1 for overlap, 0 when separated; *iters receives the
 * number of support evaluations after the first (33 at the cap). */
int or_overlap_3d(const or_system* s, const double D[3], const double qA[4], const double qB[4],
                  int* iters)
{
    if (s->nv == 0) {                                                 /* spheres */
        *iters = 0;
        return ((D[0] * D[0] + D[1] * D[1]) + D[2] * D[2]) <= s->rc2;
    }
    or_gjk_pair g;
    g.s = s;
    double qAc[4] = { qA[0], -qA[1], -qA[2], -qA[3] };
    double qr[4], l[3];
    or_qmul(qAc, qB, qr);
    or_qrot(qAc, D, l);
    for (int i = 0; i < s->nv; ++i) {
        double r[3];
        or_qrot(qr, s->v[i], r);
        g.pb[i][0] = r[0] + l[0];
        g.pb[i][1] = r[1] + l[1];
        g.pb[i][2] = r[2] + l[2];
    }
    double d[3];
    or_neg3(l, d);
    if (d[0] == 0.0 && d[1] == 0.0 && d[2] == 0.0) d[0] = -1.0;
    double sp[4][3], v[3];
    int n = 1;
    or_support(&g, d, sp[0]);
    memcpy(v, sp[0], sizeof v);
    for (int it = 0; it < OR_GJK_MAXIT; ++it) {
        if (iters) *iters = it + 1;
        double vv = or_dot3(v, v);
        if (vv == 0.0) return 1;
        double nv[3], w[3];
        or_neg3(v, nv);
        or_support(&g, nv, w);
        if (or_dot3(v, w) > 0.0) return 0;
        memcpy(sp[n], w, sizeof w);
        n += 1;
        if (or_gjk_reduce(sp, &n, v)) return 1;
    }
    if (iters) *iters = OR_GJK_MAXIT + 1;    /* cap reached: counted as overlap */
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Trial moves (Sec. 2.1 step 2: r' = r + dr, q' = q . dq)                   */
/* ------------------------------------------------------------------------ */

/* Random words of one select: 2 Philox blocks in 2D, 4 in 3D. */
static void or_move_words(const or_system* s, uint64_t sweep, uint32_t set, uint32_t cell,
                          uint32_t k, uint32_t r[16])
{
    int nb = (s->dim == 2) ? 2 : 4;
    for (int b = 0; b < nb; ++b) or_move_block(s->seed, sweep, set, cell, k, (uint32_t)b, r + 4 * b);
}

static double or_wrap_pos(double x, double L)
{
    if (x < 0.0) x = x + L;
    if (x >= L) x = x - L;
    return x;
}

/* Proposal from the words r[]: translation and rotation of particle (x, q).
 * 2D q = (c, s); 3D q = (w, x, y, z).  Outputs x', q'. */
void or_propose(const or_system* s, const uint32_t* r, const double* x, const double* q,
                double* xn, double* qn)
{
    if (s->dim == 2) {
        double dx = s->d * (2.0 * or_u53(r[1], r[2]) - 1.0);
        double dy = s->d * (2.0 * or_u53(r[3], r[4]) - 1.0);
        double t = s->tau * (2.0 * or_u53(r[5], r[6]) - 1.0);
        xn[0] = or_wrap_pos(x[0] + dx, s->L[0]);
        xn[1] = or_wrap_pos(x[1] + dy, s->L[1]);
        double tt = t * t;
        double inv = 1.0 / (1.0 + tt);
        double cd = (1.0 - tt) * inv;
        double sd = (t + t) * inv;
        double c1 = q[0] * cd - q[1] * sd;
        double s1 = q[0] * sd + q[1] * cd;
        double n2 = c1 * c1 + s1 * s1;
        double f = 1.5 - 0.5 * n2;
        qn[0] = c1 * f;
        qn[1] = s1 * f;
    } else {
        double dx = s->d * (2.0 * or_u53(r[1], r[2]) - 1.0);
        double dy = s->d * (2.0 * or_u53(r[3], r[4]) - 1.0);
        double dz = s->d * (2.0 * or_u53(r[5], r[6]) - 1.0);
        double v0 = s->tau * (2.0 * or_u53(r[7], r[8]) - 1.0);
        double v1 = s->tau * (2.0 * or_u53(r[9], r[10]) - 1.0);
        double v2 = s->tau * (2.0 * or_u53(r[11], r[12]) - 1.0);
        xn[0] = or_wrap_pos(x[0] + dx, s->L[0]);
        xn[1] = or_wrap_pos(x[1] + dy, s->L[1]);
        xn[2] = or_wrap_pos(x[2] + dz, s->L[2]);
        double vv = (v0 * v0 + v1 * v1) + v2 * v2;
        double inv = 1.0 / sqrt(1.0 + vv);
        double dq[4] = { inv, v0 * inv, v1 * inv, v2 * inv };
        double q1[4];
        or_qmul(q, dq, q1);
        double n2 = ((q1[0] * q1[0] + q1[1] * q1[1]) + q1[2] * q1[2]) + q1[3] * q1[3];
        double f = 1.5 - 0.5 * n2;
        qn[0] = q1[0] * f; qn[1] = q1[1] * f; qn[2] = q1[2] * f; qn[3] = q1[3] * f;
    }
}

/* test hook: the proposal of select k in cell `cell` of set `set` */
void or_propose_from_stream(const or_system* s, uint64_t sweep, uint32_t set, uint32_t cell,
                            uint32_t k, uint32_t n_c, const double* x, const double* q,
                            uint32_t* pick, double* xn, double* qn)
{
    uint32_t r[16];
    or_move_words(s, sweep, set, cell, k, r);
    *pick = (uint32_t)(((uint64_t)r[0] * (uint64_t)n_c) >> 32);
    or_propose(s, r, x, q, xn, qn);
}

static double or_min_image(double dlt, double L, double halfL)
{
    if (dlt > halfL) dlt = dlt - L;
    else if (dlt < -halfL) dlt = dlt + L;
    return dlt;
}

/* ------------------------------------------------------------------------ */
/* The sweep (Sec. 2.1 + 2.2.1 + 2.5.1 + 2.5.2)                              */
/* ------------------------------------------------------------------------ */

/* The nselect trial moves of one active cell (ix, iy, iz) of set `set`
 * (Sec. 2.5.2: the moves of one cell run in sequence; a trial that leaves the
 * cell is rejected, so the cell's contents stay fixed during the set).
 * counters[0] accept, [1] reject_overlap, [2] reject_boundary, [3] gjk caps */
static void or_cell_moves(const or_system* s, double* pos, double* orient, const double sh[3],
                          const uint32_t* start, const uint32_t* idx, uint64_t sweep, int set,
                          int ix, int iy, int iz, uint64_t* counters)
{
    const int dim = s->dim;
    const int qd = (dim == 2) ? 2 : 4;
    int cell = ix + s->nc[0] * (iy + s->nc[1] * iz);
    uint32_t n_c = start[cell + 1] - start[cell];
    if (n_c == 0) return;                             /* empty cells propose nothing */
    for (uint32_t k = 0; k < s->nselect; ++k) {
        uint32_t r[16];
        or_move_words(s, sweep, (uint32_t)set, (uint32_t)cell, k, r);
        uint32_t j = (uint32_t)(((uint64_t)r[0] * (uint64_t)n_c) >> 32);
        uint32_t i = idx[start[cell] + j];
        double xn[3] = { 0, 0, 0 }, qn[4] = { 0, 0, 0, 0 };
        or_propose(s, r, pos + (size_t)i * dim, orient + (size_t)i * qd, xn, qn);
        /* checkerboard rule: a trial position outside the
         * active cell is rejected (Sec. 2.5.1 / 2.5.2) */
        int ci[3];
        if (or_cell_of(s, sh, xn, ci) != cell) { counters[2] += 1; continue; }
        int overlap = 0;
        for (int oz = (dim == 3 ? -1 : 0); oz <= (dim == 3 ? 1 : 0) && !overlap; ++oz)
        for (int oy = -1; oy <= 1 && !overlap; ++oy)
        for (int ox = -1; ox <= 1 && !overlap; ++ox) {
            int jx = (ix + ox + s->nc[0]) % s->nc[0];
            int jy = (iy + oy + s->nc[1]) % s->nc[1];
            int jz = (dim == 3) ? (iz + oz + s->nc[2]) % s->nc[2] : 0;
            int nb = jx + s->nc[0] * (jy + s->nc[1] * jz);
            for (uint32_t e = start[nb]; e < start[nb + 1]; ++e) {
                uint32_t b = idx[e];
                if (b == i) continue;
                double D[3] = { 0, 0, 0 };
                double q2 = 0.0;
                for (int kk = 0; kk < dim; ++kk) {
                    D[kk] = or_min_image(pos[(size_t)b * dim + kk] - xn[kk], s->L[kk], s->halfL[kk]);
                }
                q2 = D[0] * D[0] + D[1] * D[1];
                if (dim == 3) q2 = q2 + D[2] * D[2];
                if (q2 > s->rc2) continue;           /* circumsphere cull */
                int ov;
                if (s->nv == 0) {
                    ov = 1;                 /* disks/spheres: q2 <= (2R)^2 */
                } else if (dim == 2) {
                    ov = or_overlap_2d(s, D, qn, orient + (size_t)b * qd);
                } else {
                    int it = 0;
                    ov = or_overlap_3d(s, D, qn, orient + (size_t)b * qd, &it);
                    if (it > OR_GJK_MAXIT) counters[3] += 1;
                }
                if (ov) { overlap = 1; break; }     /* early exit (Sec. 2.1) */
            }
        }
        if (overlap) { counters[1] += 1; continue; }
        for (int kk = 0; kk < dim; ++kk) pos[(size_t)i * dim + kk] = xn[kk];
        for (int kk = 0; kk < qd; ++kk) orient[(size_t)i * qd + kk] = qn[kk];
        counters[0] += 1;
    }
}

/* One set of a sweep: every active cell (parity bits = set) in turn, or,
 * with nthr > 1, the cells whose rank in that order is thr modulo nthr.
 * Active cells of one set never touch one another (a moved particle stays in
 * its cell, and a cell's 3^d stencil holds no other active cell), so the
 * result does not depend on how the cells are shared out. */
static void or_set_cells(const or_system* s, double* pos, double* orient, const double sh[3],
                         const uint32_t* start, const uint32_t* idx, uint64_t sweep, int set,
                         int thr, int nthr, uint64_t* counters)
{
    const int dim = s->dim;
    const int nz = (dim == 3) ? s->nc[2] : 1;
    int px = set & 1, py = (set >> 1) & 1, pz = (set >> 2) & 1;
    long rank = 0;
    for (int iz = 0; iz < nz; ++iz) {
        if (dim == 3 && (iz & 1) != pz) continue;
        for (int iy = 0; iy < s->nc[1]; ++iy) {
            if ((iy & 1) != py) continue;
            for (int ix = 0; ix < s->nc[0]; ++ix) {
                if ((ix & 1) != px) continue;
                if (rank++ % nthr != thr) continue;
                or_cell_moves(s, pos, orient, sh, start, idx, sweep, set, ix, iy, iz, counters);
            }
        }
    }
}

/* One thread's share of a set (threaded sweeps). */
typedef struct {
    const or_system* s;
    double* pos;
    double* orient;
    const double* sh;
    const uint32_t* start;
    const uint32_t* idx;
    uint64_t sweep;
    int set, thr, nthr;
    uint64_t counters[4];
} or_share;

static void* or_share_run(void* p)
{
    or_share* a = (or_share*)p;
    or_set_cells(a->s, a->pos, a->orient, a->sh, a->start, a->idx, a->sweep, a->set, a->thr, a->nthr,
                 a->counters);
    return NULL;
}

/* Host threads for the sets of or_sweep (1 = serial, the default). */
int or_set_threads(or_system* s, int nthreads)
{
    if (nthreads < 1 || nthreads > 1024) return -1;
    s->nthreads = nthreads;
    return 0;
}

/* counters[0] accept, [1] reject_overlap, [2] reject_boundary, [3] gjk caps */
int or_sweep(or_system* s, uint32_t N, double* pos, double* orient, uint64_t sweep0,
             uint32_t nsweeps, uint64_t* counters)
{
    const int dim = s->dim;
    const int C = or_ncells(s);
    uint32_t* start = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(C + 1));
    uint32_t* idx = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(N > 0 ? N : 1));
    int* cell_of = (int*)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    if (!start || !idx || !cell_of) { free(start); free(idx); free(cell_of); return -3; }
    const int nsets = 1 << dim;
    const int nthr = s->nthreads > 1 ? s->nthreads : 1;
    int rc = 0;

    if (nthr == 1) {
        for (uint32_t sw = 0; sw < nsweeps; ++sw) {
            uint64_t sweep = sweep0 + sw;
            double sh[3];
            or_grid_shift(s, sweep, sh);
            or_build_cells(s, N, pos, sh, start, idx, cell_of);
            for (int set = 0; set < nsets; ++set)
                or_set_cells(s, pos, orient, sh, start, idx, sweep, set, 0, 1, counters);
        }
    } else {
        /* each set forks nthr shares and joins them before the next set; a
         * share whose thread cannot be started runs on this thread */
        or_share* sh_args = (or_share*)calloc((size_t)nthr, sizeof(or_share));
        pthread_t* tid = (pthread_t*)calloc((size_t)nthr, sizeof(pthread_t));
        int* started = (int*)calloc((size_t)nthr, sizeof(int));
        if (!sh_args || !tid || !started) rc = -3;
        for (uint32_t sw = 0; sw < nsweeps && rc == 0; ++sw) {
            uint64_t sweep = sweep0 + sw;
            double sh[3];
            or_grid_shift(s, sweep, sh);
            or_build_cells(s, N, pos, sh, start, idx, cell_of);
            for (int set = 0; set < nsets; ++set) {
                for (int t = 0; t < nthr; ++t) {
                    or_share* a = &sh_args[t];
                    a->s = s; a->pos = pos; a->orient = orient; a->sh = sh;
                    a->start = start; a->idx = idx; a->sweep = sweep;
                    a->set = set; a->thr = t; a->nthr = nthr;
                    started[t] = (t > 0) && pthread_create(&tid[t], NULL, or_share_run, a) == 0;
                }
                or_share_run(&sh_args[0]);
                for (int t = 1; t < nthr; ++t) {
                    if (started[t]) pthread_join(tid[t], NULL);
                    else or_share_run(&sh_args[t]);
                }
            }
        }
        if (rc == 0)
            for (int t = 0; t < nthr; ++t)
                for (int k = 0; k < 4; ++k) counters[k] += sh_args[t].counters[k];
        free(sh_args);
        free(tid);
        free(started);
    }
    free(start);
    free(idx);
    free(cell_of);
    return rc;
}

/* Test hook: n independent one-sweep runs of or_sweep, each from the same
 * configuration (pos0, ori0) at sweep index sweep0 + k.  moved[k*N + i] is 1
 * when particle i's position or orientation changed in run k; shifts[3k..]
 * receives that run's grid shift.  Used to measure the one-move acceptance
 * frequency of a fixed configuration (Sec. 2.1). */
int or_sweep_repeats(or_system* s, uint32_t N, const double* pos0, const double* ori0, uint64_t sweep0,
                     uint32_t n, uint8_t* moved, double* shifts)
{
    const int dim = s->dim, qd = (dim == 2) ? 2 : 4;
    double* pos = (double*)malloc(sizeof(double) * (size_t)N * dim);
    double* ori = (double*)malloc(sizeof(double) * (size_t)N * qd);
    if (!pos || !ori) { free(pos); free(ori); return -3; }
    int rc = 0;
    for (uint32_t k = 0; k < n && rc == 0; ++k) {
        uint64_t cnt[4] = { 0, 0, 0, 0 };
        memcpy(pos, pos0, sizeof(double) * (size_t)N * dim);
        memcpy(ori, ori0, sizeof(double) * (size_t)N * qd);
        rc = or_sweep(s, N, pos, ori, sweep0 + k, 1, cnt);
        or_grid_shift(s, sweep0 + k, shifts + 3 * (size_t)k);
        for (uint32_t i = 0; i < N; ++i)
            moved[(size_t)k * N + i] = (uint8_t)(memcmp(pos + (size_t)i * dim, pos0 + (size_t)i * dim,
                                                        sizeof(double) * dim) != 0 ||
                                                 memcmp(ori + (size_t)i * qd, ori0 + (size_t)i * qd,
                                                        sizeof(double) * qd) != 0);
    }
    free(pos);
    free(ori);
    return rc;
}

/* Batch evaluation of the overlap contract on many pairs (for tests); in 3D
 * iters[p] (when iters is not NULL) receives the GJK's support evaluations
 * after the first, the count or_overlap_3d reports. */
void or_overlap_batch_it(const or_system* s, uint32_t n, const double* D, const double* qA,
                         const double* qB, int32_t* out, int32_t* iters)
{
    const int dim = s->dim, qd = (dim == 2) ? 2 : 4;
    for (uint32_t p = 0; p < n; ++p) {
        if (dim == 2) out[p] = or_overlap_2d(s, D + 2 * (size_t)p, qA + 2 * (size_t)p, qB + 2 * (size_t)p);
        else {
            int it = 0;
            out[p] = or_overlap_3d(s, D + 3 * (size_t)p, qA + (size_t)qd * p, qB + (size_t)qd * p, &it);
            if (iters) iters[p] = it;
        }
    }
}

void or_overlap_batch(const or_system* s, uint32_t n, const double* D, const double* qA,
                      const double* qB, int32_t* out)
{
    or_overlap_batch_it(s, n, D, qA, qB, out, 0);
}

/* ------------------------------------------------------------------------ */
/* Pressure by the scale distribution (Sec. 4): for disks/spheres of        */
/* diameter sigma, compressing every position by the factor (1 - x) makes a  */
/* pair at distance r overlap for x >= x* = 1 - sigma / r.  The histogram of  */
/* x* near 0 extrapolated to x = 0 gives beta P / rho = 1 + h(0) / (dim N),  */
/* h the number of pairs per unit x.  Every unordered pair (all pairs,       */
/* minimum image) with 0 <= x* < x_max adds one to bin (int)(x* nbins/x_max). */
/* ------------------------------------------------------------------------ */
/* Shaped particles (volume perturbation for particles with shape, Sec. 4):
 * with positions compressed by (1 - x) and the shapes unchanged, a pair at D
 * overlaps from x* on (overlap(lambda D) is monotone in lambda for convex
 * shapes containing their centres).  Reading: the bin of x* is found with
 * the overlap contract at the bin edges e_k = k h, h = x_max / nbins, by
 * bisection: if the pair overlaps at e_nbins, the smallest overlapping edge
 * index k (lo = 0, hi = nbins; while hi - lo > 1: mid = (lo + hi) / 2,
 * overlap at e_mid ? hi = mid : lo = mid) gives bin hi - 1; the scaled
 * separation is D_a * (1 - e_k) per axis. */
static int or_sdf_shaped_bin(const or_system* s, const double D[3], const double* qi, const double* qj,
                             double h, uint32_t nbins)
{
    const int dim = s->dim;
    #define OR_OVERLAP_AT(k, out)                                                 \
        do {                                                                      \
            const double sc = 1.0 - (double)(k) * h;                              \
            double Ds[3] = { D[0] * sc, D[1] * sc, dim == 3 ? D[2] * sc : 0.0 };  \
            if (dim == 2) out = or_overlap_2d(s, Ds, qi, qj);                     \
            else { int it_ = 0; out = or_overlap_3d(s, Ds, qi, qj, &it_); }       \
        } while (0)
    int top = 0;
    OR_OVERLAP_AT(nbins, top);
    if (!top) return -1;
    uint32_t lo = 0, hi = nbins;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        int ov = 0;
        OR_OVERLAP_AT(mid, ov);
        if (ov) hi = mid; else lo = mid;
    }
    #undef OR_OVERLAP_AT
    return (int)lo;
}

int or_sdf_histogram(const or_system* s, uint32_t N, const double* pos, const double* orient, double x_max,
                     uint32_t nbins, uint64_t* hist)
{
    if (!(x_max > 0.0) || !(x_max < 1.0) || nbins == 0) return -1;
    const int dim = s->dim, qd = (dim == 2) ? 2 : 4;
    if (s->nv != 0) {
        const double h = x_max / (double)nbins;
        for (uint32_t i = 0; i < N; ++i)
            for (uint32_t j = i + 1; j < N; ++j) {
                double D[3] = { 0, 0, 0 };
                for (int k = 0; k < dim; ++k)
                    D[k] = or_min_image(pos[(size_t)j * dim + k] - pos[(size_t)i * dim + k], s->L[k], s->halfL[k]);
                const int b = or_sdf_shaped_bin(s, D, orient + (size_t)i * qd, orient + (size_t)j * qd, h, nbins);
                if (b >= 0) hist[b] += 1;
            }
        return 0;
    }
    const double sigma = s->R + s->R;
    const double scale = (double)nbins / x_max;
    for (uint32_t i = 0; i < N; ++i)
        for (uint32_t j = i + 1; j < N; ++j) {
            double D[3] = { 0, 0, 0 };
            for (int k = 0; k < dim; ++k)
                D[k] = or_min_image(pos[(size_t)j * dim + k] - pos[(size_t)i * dim + k], s->L[k], s->halfL[k]);
            double q2 = D[0] * D[0] + D[1] * D[1];
            if (dim == 3) q2 = q2 + D[2] * D[2];
            const double x = 1.0 - sigma / sqrt(q2);
            if (!(x >= 0.0) || !(x < x_max)) continue;
            const int b = (int)(x * scale);
            if (b < (int)nbins) hist[b] += 1;
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Isotropic volume move (NPT ensemble, which the paper runs following      */
/* Frenkel & Smit).  Readings: one trial V' = V + dV_max (2u - 1); every    */
/* box length and position scaled by f = (V'/V)^(1/dim) (sqrt / cbrt), a    */
/* position that rounds onto L' wraps to 0; the cell grid of the trial box */
/* follows the creation rule (nc = floor(L'/max(2R, w_min)), even, a trial  */
/* with fewer than 4 cells on an axis is rejected); any overlapping pair    */
/* rejects; otherwise accept                                                */
/* when u' < exp(-beta_P (V' - V) + N log(V'/V)).  Stream: key = seed,      */
/* ctr = (lo32(m), hi32(m), 0, 4 << 24) for the m-th move attempt; u from   */
/* words (0, 1), u' from words (2, 3).  Returns 1 when accepted.            */
/* ------------------------------------------------------------------------ */
int or_box_move(or_system* s, uint32_t N, double* pos, const double* orient, double beta_P, double dV_max,
                uint64_t m)
{
    const int dim = s->dim, qd = (dim == 2) ? 2 : 4;
    uint32_t key[2] = { (uint32_t)s->seed, (uint32_t)(s->seed >> 32) };
    uint32_t ctr[4] = { (uint32_t)m, (uint32_t)(m >> 32), 0u, 4u << 24 };
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    const double u1 = or_u53(w[0], w[1]), u2 = or_u53(w[2], w[3]);
    double V = s->L[0] * s->L[1];
    if (dim == 3) V = V * s->L[2];
    const double dV = dV_max * (2.0 * u1 - 1.0);
    const double Vn = V + dV;
    if (!(Vn > 0.0)) return 0;
    const double ratio = Vn / V;
    const double f = (dim == 2) ? sqrt(ratio) : cbrt(ratio);
    or_system t = *s;
    for (int k = 0; k < dim; ++k) {
        t.L[k] = s->L[k] * f;
        t.halfL[k] = 0.5 * t.L[k];
        int n = (int)floor(t.L[k] / s->wcell_min);
        if (n % 2) n -= 1;
        if (n < 4) return 0;
        t.nc[k] = n;
        t.w[k] = t.L[k] / (double)n;
        t.inv_w[k] = (double)n / t.L[k];
    }
    double* np = (double*)malloc(sizeof(double) * (size_t)N * dim + 8);
    if (!np) return -3;
    for (uint32_t i = 0; i < N; ++i)
        for (int k = 0; k < dim; ++k) {
            double x = pos[(size_t)i * dim + k] * f;
            if (x >= t.L[k]) x = x - t.L[k];
            np[(size_t)i * dim + k] = x;
        }
    int overlap = 0;
    for (uint32_t i = 0; i < N && !overlap; ++i)
        for (uint32_t j = i + 1; j < N && !overlap; ++j) {
            double D[3] = { 0, 0, 0 };
            for (int k = 0; k < dim; ++k)
                D[k] = or_min_image(np[(size_t)j * dim + k] - np[(size_t)i * dim + k], t.L[k], t.halfL[k]);
            double q2 = D[0] * D[0] + D[1] * D[1];
            if (dim == 3) q2 = q2 + D[2] * D[2];
            if (q2 > t.rc2) continue;
            if (dim == 2) overlap = or_overlap_2d(&t, D, orient + (size_t)i * qd, orient + (size_t)j * qd);
            else {
                int it = 0;
                overlap = or_overlap_3d(&t, D, orient + (size_t)i * qd, orient + (size_t)j * qd, &it);
            }
        }
    int acc = 0;
    if (!overlap) {
        const double arg = -beta_P * dV + (double)N * log(ratio);
        if (u2 < exp(arg)) acc = 1;
    }
    if (acc) {
        memcpy(pos, np, sizeof(double) * (size_t)N * dim);
        *s = t;
    }
    free(np);
    return acc;
}

void or_get_box(const or_system* s, double* L)
{
    for (int k = 0; k < 3; ++k) L[k] = s->L[k];
}

/* Exported geometry for tests */
void or_get_geometry(const or_system* s, double* R, double* rc2, int* nc, double* w, double* inv_w)
{
    *R = s->R;
    *rc2 = s->rc2;
    for (int k = 0; k < 3; ++k) { nc[k] = s->nc[k]; w[k] = s->w[k]; inv_w[k] = s->inv_w[k]; }
}

double or_get_tau(const or_system* s) { return s->tau; }

/* ------------------------------------------------------------------------ */
/* Random sequential addition (test-input generation only): place N shapes  */
/* one at a time at uniform random positions/orientations, keeping a trial  */
/* only when it overlaps none of the shapes already placed.  Uses the same  */
/* overlap contract as the sweep.  Stream: ctr = (lo32(t), hi32(t), b,      */
/* 3<<24) with key = seed, for attempt t and block b.                        */
/* ------------------------------------------------------------------------ */
int or_rsa_2d(const or_system* s, uint32_t N, uint64_t seed, uint64_t max_attempts,
              double* pos, double* orient, uint64_t* attempts_used)
{
    if (s->dim != 2) return -1;
    int C = s->nc[0] * s->nc[1];
    int* head = (int*)malloc(sizeof(int) * (size_t)C);
    int* next = (int*)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    if (!head || !next) { free(head); free(next); return -3; }
    for (int c = 0; c < C; ++c) head[c] = -1;
    const double zero[3] = { 0.0, 0.0, 0.0 };
    const double two_pi = 6.283185307179586;
    uint32_t placed = 0;
    uint64_t t = 0;
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    while (placed < N && t < max_attempts) {
        uint32_t r0[4], r1[4];
        uint32_t c0[4] = { (uint32_t)t, (uint32_t)(t >> 32), 0u, 3u << 24 };
        uint32_t c1[4] = { (uint32_t)t, (uint32_t)(t >> 32), 1u, 3u << 24 };
        or_philox4x32_10(c0, key, r0);
        or_philox4x32_10(c1, key, r1);
        t += 1;
        double x[2] = { s->L[0] * or_u53(r0[0], r0[1]), s->L[1] * or_u53(r0[2], r0[3]) };
        if (x[0] >= s->L[0]) x[0] = 0.0;
        if (x[1] >= s->L[1]) x[1] = 0.0;
        double th = two_pi * or_u53(r1[0], r1[1]);
        double z[2] = { cos(th), sin(th) };
        int ci[3];
        or_cell_of(s, zero, x, ci);
        int bad = 0;
        for (int oy = -1; oy <= 1 && !bad; ++oy)
        for (int ox = -1; ox <= 1 && !bad; ++ox) {
            int jx = (ci[0] + ox + s->nc[0]) % s->nc[0];
            int jy = (ci[1] + oy + s->nc[1]) % s->nc[1];
            for (int b = head[jx + s->nc[0] * jy]; b >= 0; b = next[b]) {
                double D[2] = { or_min_image(pos[2 * b] - x[0], s->L[0], s->halfL[0]),
                                or_min_image(pos[2 * b + 1] - x[1], s->L[1], s->halfL[1]) };
                if (D[0] * D[0] + D[1] * D[1] > s->rc2) continue;
                if (or_overlap_2d(s, D, z, orient + 2 * (size_t)b)) { bad = 1; break; }
            }
        }
        if (bad) continue;
        pos[2 * placed] = x[0];
        pos[2 * placed + 1] = x[1];
        orient[2 * placed] = z[0];
        orient[2 * placed + 1] = z[1];
        int c = ci[0] + s->nc[0] * ci[1];
        next[placed] = head[c];
        head[c] = (int)placed;
        placed += 1;
    }
    free(head);
    free(next);
    *attempts_used = t;
    return placed == N ? 0 : -4;
}
