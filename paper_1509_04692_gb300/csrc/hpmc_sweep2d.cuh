// hpmc_sweep2d.cuh -- one checkerboard set of the 2D sweep (Sec. 2.5.2).
//
// Work unit: one warp takes a strip of S = 32/G consecutive active cells of
// one row of one replica (G lanes per cell).  The three rows of neighbour
// cells that the strip's 3x3 stencils touch are contiguous ranges of the
// cell-sorted state, so the warp stages them into its shared memory with
// coalesced 16-byte loads (two ranges per row when the row wraps).  Inside a
// cell the nselect trial moves are sequential; across the S cells of the
// warp they run in lockstep.  For every move the G lanes of a cell stride
// over its stencil doing the circumsphere cull; survivors of all cells go to
// a warp-wide shared-memory pair queue (ballot compaction) that the warp
// drains with full overlap tests, skipping pairs of moves already known to
// overlap (early exit on the first overlap, Sec. 2.1; the block queue of
// Sec. 2.5.3 rebuilt at warp granularity with __ballot_sync).
//
// Two regimes, chosen by G:
//  * throughput (G < 8): one lane per queued pair runs the whole
//    separating-axis test with early exit; moves are generated on the fly.
//  * latency (G >= 8): the picks and move deltas (FP32 and the FP64
//    contract's) of the first G selects of a cell come from the table
//    k_selects wrote for the sweep (selects.cu), later chunks are computed
//    here, one select per lane; each queued pair is spread over 2*nv lanes,
//    one separating axis each, reduced with ballots.
//
// F32 = true : every decision is first taken in FP32 with the certified
//              margins of Rep (hpmc_bounds.h); FP64 only for accepted moves
//              and uncertified verdicts.  F32 = false: plain FP64 contract.
#pragma once
#include "hpmc_device.cuh"
#include "hpmc_filter.cuh"

namespace hpmc {

// Precomputed data of one select (latency regime): written for every select
// of the sweep by k_selects, loaded by the set kernel.
struct __align__(16) MoveData {
    double dx, dy, cd, sd;      // FP64 contract: translation and Cayley rotation
    float fdx, fdy, fcd, fsd;   // FP32 versions
    uint32_t r0;                // pick word (entry = cell begin + r0 * n_c / 2^32)
    uint32_t pad[3];
};

// Move deltas and pick word of select k of a cell (state independent).
__device__ __forceinline__ MoveData precompute_select(const Rep& rp, uint64_t seed, uint64_t sweep,
                                                      uint32_t sigma, uint32_t cell, uint32_t k)
{
    const uint4 b0 = move_block(seed, sweep, sigma, cell, k, 0);
    const uint4 b1 = move_block(seed, sweep, sigma, cell, k, 1);
    MoveData m;
    m.r0 = b0.x;
    m.dx = rp.d_s * pm53(b0.y, b0.z);
    m.dy = rp.d_s * pm53(b0.w, b1.x);
    const double t = rp.tau_s * pm53(b1.y, b1.z);
    const double tt = t * t;
    const double inv = 1.0 / (1.0 + tt);
    m.cd = (1.0 - tt) * inv;
    m.sd = (t + t) * inv;
    m.fdx = __fmul_rn(rp.d32, m24(b0.y));
    m.fdy = __fmul_rn(rp.d32, m24(b0.w));
    const float ft = __fmul_rn(rp.tau32, m24(b1.y));
    const float ftt = __fmul_rn(ft, ft);
    const float finv = __frcp_rn(__fadd_rn(1.0f, ftt));
    m.fcd = __fmul_rn(__fsub_rn(1.0f, ftt), finv);
    m.fsd = __fmul_rn(__fadd_rn(ft, ft), finv);
    m.pad[0] = m.pad[1] = m.pad[2] = 0u;
    return m;
}

template <int G, bool F32>
struct Warp2 {
    static constexpr int S = 32 / G;                  // cells per strip
    static constexpr int M = 2 * S + 1;               // staged cells per row
    static constexpr int CAPX = 9 * M;
    static constexpr int CAP = CAPX < 128 ? 128 : (CAPX > 512 ? 512 : CAPX);
    static constexpr int QCAP = 64;
    static constexpr bool LAT = G >= 8;
    static constexpr int KCH = LAT ? G : 1;           // selects precomputed per chunk
    float4 ent[F32 ? CAP : 1];                        // FP32: rel.x, rel.y, c, s
    double2 ep[F32 ? 1 : CAP];                        // FP64: x, y
    double2 eo[F32 ? 1 : CAP];                        // FP64: c, s
    uint32_t gidx[CAP];                               // sorted slot of each entry
    uint16_t sbeg[3][M + 1];                          // staged begin of each cell
    uint16_t beg[S][9];                               // stencil cell begins per cell
    uint16_t pfx[S][10];                              // stencil prefix counts per cell
    float2 qd[QCAP];                                  // queued Delta32 (FP32 form)
    uint16_t qe[QCAP];                                // queued neighbour entry
    uint8_t qg[QCAP];                                 // queued group (cell)
    float4 tr[S];                                     // FP32 trial rel', z'
    double2 tp[S], tz[S];                             // FP64 trial x', z' (FP64 form)
    uint32_t rw[S][6];                                // words r1..r6 of the move
    uint16_t eA[S];                                   // entry of the moving particle
    MoveData mv[LAT ? S : 1][KCH];                    // latency regime: precomputed selects
    unsigned int ovmask;                              // cells whose move overlaps
};

// FP64 trial of a move from its words (rare path in the FP32 form).
__device__ __forceinline__ Trial2 trial_of(const Rep& rp, const Bufs& B, uint32_t gA,
                                           const uint32_t* w)
{
    return propose2d(rp, B.px[gA], B.py[gA], B.q0[gA], B.q1[gA], w[0], w[1], w[2], w[3], w[4], w[5]);
}

// FP64 trial from precomputed contract deltas (identical operations to
// propose2d, split between the precompute and this step).
__device__ __forceinline__ Trial2 apply64(const Rep& rp, double x, double y, double c, double s,
                                          const MoveData& m)
{
    Trial2 o;
    o.x = wrap_pos_bits(x + m.dx, rp.L[0]);
    o.y = wrap_pos_bits(y + m.dy, rp.L[1]);
    const double c1 = c * m.cd - s * m.sd;
    const double s1 = c * m.sd + s * m.cd;
    const double n2 = c1 * c1 + s1 * s1;
    const double f = 1.5 - 0.5 * n2;
    o.c = c1 * f;
    o.s = s1 * f;
    return o;
}

// One axis of the separating-axis test in FP32 (latency regime): the shape
// moved into the frame of the tested normals by (c, s) and (lx, ly),
// projected on normal k.  Returns the larger of the two interval gaps.
template <int NV>
__device__ __forceinline__ float axis_gap32(const Shape2& sh, int k, float c, float s, float lx, float ly)
{
    const int nv = NV ? NV : sh.nv;
    const float nx = sh.fnx[k], ny = sh.fny[k];
    float lo = 0.f, hi = 0.f;
#pragma unroll
    for (int i = 0; i < nv; ++i) {
        const float px = __fmaf_rn(c, sh.fvx[i], __fmaf_rn(-s, sh.fvy[i], lx));
        const float py = __fmaf_rn(s, sh.fvx[i], __fmaf_rn(c, sh.fvy[i], ly));
        const float t = __fmaf_rn(nx, px, __fmul_rn(ny, py));
        lo = i ? fminf(lo, t) : t;
        hi = i ? fmaxf(hi, t) : t;
    }
    return fmaxf(__fsub_rn(lo, sh.fahi[k]), __fsub_rn(sh.falo[k], hi));
}

// Register budget: 128 a thread (two 256-thread blocks per SM) for the
// latency regime; blocks of at most 192 threads and 168 registers for G <= 4,
// whose per-pair SAT spills at 128 (measured: the 512 replicas +4%).
template <int G, bool F32, int NV>
__global__ void __launch_bounds__(G >= 8 ? 256 : 192, 2)
k_set2d(Dev dv, Shape2 sh, int nxt, int sigma, const uint32_t* __restrict__ item_base)
{
    pdl_wait();
    using W = Warp2<G, F32>;
    constexpr int S = W::S;
    constexpr bool LAT = W::LAT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    W& ws = reinterpret_cast<W*>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int grp = lane / G;
    const int sl = lane - grp * G;
    const unsigned FULL = 0xffffffffu;
    const Bufs B = dv.buf[nxt];
    const uint32_t* __restrict__ start = dv.start;
    const uint32_t nitems = item_base[dv.R];
    const uint32_t wpb = blockDim.x >> 5;
    const int nvv = NV ? NV : sh.nv;
    const MoveData* __restrict__ msel = static_cast<const MoveData*>(dv.msel);
    const uint32_t mstride = dv.msel_stride;
    HPMC_STAMP_NS(dv, blockIdx.x * wpb + (threadIdx.x >> 5), lane, 28);

    for (uint32_t item = blockIdx.x * wpb + (threadIdx.x >> 5); item < nitems;
         item += gridDim.x * wpb) {
        const bool first = item == blockIdx.x * wpb + (threadIdx.x >> 5);
        const uint32_t wid = blockIdx.x * wpb + (threadIdx.x >> 5);
        HPMC_STAMP(dv, wid, first, lane, 0);
        // ---- replica and strip of this work item
        uint32_t lo = 0, hi = dv.R;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(item_base + mid) <= item) lo = mid; else hi = mid;
        }
        const uint32_t r = lo;
        const Rep& rp = dv.reps[r];
        const int nc0 = rp.nc[0], nc1 = rp.nc[1];
        const int nax = nc0 >> 1;
        const int spr = (nax + S - 1) / S;
        const uint32_t local = item - __ldg(item_base + r);
        const int row = (int)(local / spr);
        const int strip = (int)(local - (uint32_t)row * spr);
        const int iy = 2 * row + ((sigma >> 1) & 1);
        const int jfirst = strip * S;
        const int Sv = min(S, nax - jfirst);
        const uint64_t sweep = dv.sweep[r] - 1;          // the running sweep
        const double shx = dv.shift[3 * r], shy = dv.shift[3 * r + 1];
        const uint64_t seed = rp.seed;
        const uint32_t nsel = rp.nselect;
        HPMC_STAMP(dv, wid, first, lane, 1);
        unsigned c_moves = 0, c_acc = 0, c_rov = 0, c_rbd = 0, c_cull = 0, c_chk = 0, c_rechk = 0;
        uint32_t rowbase[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) rowbase[q] = rp.cbase + (uint32_t)nc0 * (uint32_t)((iy - 1 + q + nc1) % nc1);

        // ---- cell starts of the whole strip (first pass, first try), issued
        // before the select precompute so that the loads overlap it
        constexpr int NCH = (W::M + 31) / 32;           // 32-column chunks per row
        uint32_t s0[3][NCH], s1[3][NCH];
        {
            const int xa = ((sigma & 1) + 2 * jfirst - 1 + nc0) % nc0;
            const int Mp = 2 * Sv + 1;
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    const int m = ch * 32 + lane;
                    s0[q][ch] = 0u; s1[q][ch] = 0u;
                    if (m < Mp) {
                        const uint32_t c = rowbase[q] + (uint32_t)((xa + m) % nc0);
                        s0[q][ch] = start[c];
                        s1[q][ch] = start[c + 1];
                    }
                }
        }
        if (LAT) {
            // ---- selects of the first chunk of every cell of the strip
            const uint32_t k = (uint32_t)sl;
            if (grp < Sv && k < nsel) {
                const int ixp = (sigma & 1) + 2 * (jfirst + grp);
                const uint32_t cg = rp.cbase + (uint32_t)ixp + (uint32_t)nc0 * (uint32_t)iy;
                ws.mv[grp][sl] = msel[(size_t)cg * mstride + k];
            }
        }
        HPMC_STAMP(dv, wid, first, lane, 2);
        int j0 = 0;
        bool preloaded = true;
        while (j0 < Sv) {
            // ---- choose the sub-strip [j0, j1) whose staged rows fit CAP
            int j1 = Sv;
            bool skip_cell = false;
            int xa = 0, Mp = 0;
            uint32_t (&cnt)[3][NCH] = s1;                  // counts replace the cell ends
            for (;;) {
                xa = ((sigma & 1) + 2 * (jfirst + j0) - 1 + nc0) % nc0;
                Mp = 2 * (j1 - j0) + 1;
                if (!preloaded) {
#pragma unroll
                    for (int q = 0; q < 3; ++q)
#pragma unroll
                        for (int ch = 0; ch < NCH; ++ch) {
                            const int m = ch * 32 + lane;
                            s0[q][ch] = 0u; s1[q][ch] = 0u;
                            if (m < Mp) {
                                const uint32_t c = rowbase[q] + (uint32_t)((xa + m) % nc0);
                                s0[q][ch] = start[c];
                                s1[q][ch] = start[c + 1];
                            }
                        }
                }
                preloaded = false;
                uint32_t mine = 0;
#pragma unroll
                for (int q = 0; q < 3; ++q)
#pragma unroll
                    for (int ch = 0; ch < NCH; ++ch) {
                        cnt[q][ch] = (ch * 32 + lane < Mp) ? s1[q][ch] - s0[q][ch] : 0u;
                        mine += cnt[q][ch];
                    }
                const uint32_t tot = __reduce_add_sync(FULL, mine);
                if (tot <= (uint32_t)W::CAP) break;
                if (j1 == j0 + 1) { skip_cell = true; break; }
                j1 = j0 + (j1 - j0) / 2;
            }
            if (skip_cell) {
                if (lane == 0) atomicOr(dv.error, ERR_CAPACITY);
                j0 += 1;
                continue;
            }
            // ---- staged begin of every cell (per-row scans of the counts)
            uint32_t off_row[4];
            off_row[0] = 0;
            uint32_t gA0[3], gB0[3], lenA[3];
            const int mwrap = (xa + Mp > nc0) ? nc0 - xa : Mp;     // first column wrapped to x = 0
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                uint32_t run = 0;
                uint32_t at_wrap = 0;
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    const int m = ch * 32 + lane;
                    const uint32_t c = cnt[q][ch];
                    uint32_t incl = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t t = __shfl_up_sync(FULL, incl, o);
                        if (lane >= o) incl += t;
                    }
                    const uint32_t excl = run + incl - c;
                    if (m < Mp) ws.sbeg[q][m] = (uint16_t)(off_row[q] + excl);
                    // entries before the wrap column, and its global start
                    if (mwrap < Mp && mwrap >= ch * 32 && mwrap < ch * 32 + 32) {
                        at_wrap = __shfl_sync(FULL, excl, mwrap - ch * 32);
                        gB0[q] = __shfl_sync(FULL, s0[q][ch], mwrap - ch * 32);
                    }
                    run += __shfl_sync(FULL, incl, 31);
                }
                gA0[q] = __shfl_sync(FULL, s0[q][0], 0);
                if (mwrap >= Mp) { at_wrap = run; gB0[q] = 0u; }
                lenA[q] = at_wrap;
                if (lane == 0) ws.sbeg[q][Mp] = (uint16_t)(off_row[q] + run);
                off_row[q + 1] = off_row[q] + run;
            }
            // ---- stage every entry of the three rows (coalesced 16-byte loads)
            {
                const uint32_t total = off_row[3];
                for (uint32_t t = lane; t < total; t += 32) {
                    const bool r1 = t >= off_row[1], r2 = t >= off_row[2];
                    const uint32_t o = r2 ? off_row[2] : (r1 ? off_row[1] : 0u);
                    const uint32_t la = r2 ? lenA[2] : (r1 ? lenA[1] : lenA[0]);
                    const uint32_t ga = r2 ? gA0[2] : (r1 ? gA0[1] : gA0[0]);
                    const uint32_t gb = r2 ? gB0[2] : (r1 ? gB0[1] : gB0[0]);
                    const uint32_t u = t - o;
                    const uint32_t gi = u < la ? ga + u : gb + (u - la);
                    ws.gidx[t] = gi;
                    if (F32) {
                        ws.ent[t] = B.f4a[gi];
                    } else {
                        ws.ep[t] = make_double2(B.px[gi], B.py[gi]);
                        ws.eo[t] = make_double2(B.q0[gi], B.q1[gi]);
                    }
                }
            }
            HPMC_STAMP(dv, wid, first, lane, 3);
            // ---- stencil tables of each cell of the sub-strip
            const bool valid = grp < (j1 - j0);
            const int jc = j0 + grp;                       // strip cell of this group
            const int mc = 1 + 2 * grp;
            const int ix = (sigma & 1) + 2 * (jfirst + jc);
            const uint32_t cell_local = (uint32_t)ix + (uint32_t)nc0 * (uint32_t)iy;
            // cell origins i * w of the relative coordinates (as in k_place)
            const double iwx = (double)ix * rp.w[0];
            const double iwy = (double)iy * rp.w[1];
            __syncwarp();
            if (sl == 0) {
                uint16_t p = 0;
                ws.pfx[grp][0] = 0;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const int qr = q / 3, qc = q % 3;
                    const uint16_t b = valid ? ws.sbeg[qr][mc - 1 + qc] : 0;
                    const uint16_t e = valid ? ws.sbeg[qr][mc + qc] : 0;
                    ws.beg[grp][q] = b;
                    p = (uint16_t)(p + (e - b));
                    ws.pfx[grp][q + 1] = p;
                }
            }
            __syncwarp();
            const uint32_t cb = valid ? ws.sbeg[1][mc] : 0;
            const uint32_t n_c = valid ? (uint32_t)ws.sbeg[1][mc + 1] - cb : 0;
            const int T = ws.pfx[grp][9];
            const bool live_cell = valid && n_c > 0;
            // one cell per warp: each lane's first candidate (stencil cell q,
            // staged entry e) is fixed for the whole set
            int cand_q = 0, cand_e = 0;
            if (S == 1 && lane < T) {
#pragma unroll
                for (int qq = 1; qq < 9; ++qq) cand_q += (lane >= (int)ws.pfx[0][qq]) ? 1 : 0;
                cand_e = ws.beg[0][cand_q] + (lane - ws.pfx[0][cand_q]);
            }
            HPMC_STAMP(dv, wid, first, lane, 4);

#pragma unroll 1
            for (uint32_t k0 = 0; k0 < nsel; k0 += W::KCH) {
                if (LAT && k0 > 0) {
                    // ---- selects of a later chunk, one per lane
                    const uint32_t k = k0 + (uint32_t)sl;
                    if (live_cell && k < nsel)
                        ws.mv[jc][sl] = precompute_select(rp, seed, sweep, (uint32_t)sigma, cell_local, k);
                    __syncwarp();
                }
                HPMC_STAMP(dv, wid, first, lane, 5);
                const uint32_t kend = min(nsel, k0 + (uint32_t)W::KCH);
#pragma unroll 1
                for (uint32_t k = k0; k < kend; ++k) {
                    // ---- propose (one lane per cell)
                    int status = 0;                       // 0 idle, 1 active, 2 left the cell
                    double ax64 = 0.0, ay64 = 0.0, ac64 = 0.0, as64 = 0.0;   // A's FP64 state
                    if (sl == 0 && live_cell) {
                        c_moves += 1;
                        uint32_t eA;
                        float fdx, fdy, fcd, fsd;
                        uint32_t wr[6] = { 0u, 0u, 0u, 0u, 0u, 0u };
                        if (LAT) {
                            const MoveData& m = ws.mv[jc][k - k0];
                            eA = cb + __umulhi(m.r0, n_c);
                            fdx = m.fdx; fdy = m.fdy; fcd = m.fcd; fsd = m.fsd;
                        } else {
                            const uint4 b0 = move_block(seed, sweep, (uint32_t)sigma, cell_local, k, 0);
                            const uint4 b1 = move_block(seed, sweep, (uint32_t)sigma, cell_local, k, 1);
                            wr[0] = b0.y; wr[1] = b0.z; wr[2] = b0.w; wr[3] = b1.x; wr[4] = b1.y; wr[5] = b1.z;
                            eA = cb + __umulhi(b0.x, n_c);
                            fdx = __fmul_rn(rp.d32, m24(wr[0]));
                            fdy = __fmul_rn(rp.d32, m24(wr[2]));
                            const float ft = __fmul_rn(rp.tau32, m24(wr[4]));
                            const float ftt = __fmul_rn(ft, ft);
                            const float finv = __frcp_rn(__fadd_rn(1.0f, ftt));
                            fcd = __fmul_rn(__fsub_rn(1.0f, ftt), finv);
                            fsd = __fmul_rn(__fadd_rn(ft, ft), finv);
                        }
                        if (!LAT) {
#pragma unroll
                            for (int q = 0; q < 6; ++q) ws.rw[grp][q] = wr[q];
                        }
                        ws.eA[grp] = (uint16_t)eA;
                        if (F32) {
                            const uint32_t gA = ws.gidx[eA];
                            if (!LAT) {
                                // prefetch A's FP64 state for the update (used after the tests)
                                ax64 = B.px[gA]; ay64 = B.py[gA]; ac64 = B.q0[gA]; as64 = B.q1[gA];
                            }
                            const float4 f = ws.ent[eA];
                            const float rx = __fadd_rn(f.x, fdx), ry = __fadd_rn(f.y, fdy);
                            const float cz = __fmaf_rn(f.z, fcd, -__fmul_rn(f.w, fsd));
                            const float sz = __fmaf_rn(f.z, fsd, __fmul_rn(f.w, fcd));
                            ws.tr[grp] = make_float4(rx, ry, cz, sz);
                            const bool out = rx < rp.out_lo || ry < rp.out_lo || rx > rp.out_hi[0] ||
                                             ry > rp.out_hi[1];
                            const bool in = rx > rp.in_lo && ry > rp.in_lo && rx < rp.in_hi[0] &&
                                            ry < rp.in_hi[1];
                            if (out) {
                                status = 2;
                            } else if (in) {
                                status = 1;
                            } else {
                                c_rechk += 1;
                                const Trial2 t2 =
                                    LAT ? apply64(rp, B.px[gA], B.py[gA], B.q0[gA], B.q1[gA], ws.mv[jc][k - k0])
                                        : propose2d(rp, B.px[gA], B.py[gA], B.q0[gA], B.q1[gA], wr[0], wr[1],
                                                    wr[2], wr[3], wr[4], wr[5]);
                                const bool ok = cell_axis(t2.x, shx, rp.L[0], rp.inv_w[0], nc0) == ix &&
                                                cell_axis(t2.y, shy, rp.L[1], rp.inv_w[1], nc1) == iy;
                                status = ok ? 1 : 2;
                            }
                        } else {
                            const double2 p = ws.ep[eA], o = ws.eo[eA];
                            Trial2 t2;
                            if (LAT) t2 = apply64(rp, p.x, p.y, o.x, o.y, ws.mv[jc][k - k0]);
                            else t2 = propose2d(rp, p.x, p.y, o.x, o.y, wr[0], wr[1], wr[2], wr[3], wr[4], wr[5]);
                            ws.tp[grp] = make_double2(t2.x, t2.y);
                            ws.tz[grp] = make_double2(t2.c, t2.s);
                            const bool ok = cell_axis(t2.x, shx, rp.L[0], rp.inv_w[0], nc0) == ix &&
                                            cell_axis(t2.y, shy, rp.L[1], rp.inv_w[1], nc1) == iy;
                            status = ok ? 1 : 2;
                        }
                    }
                    if (lane == 0) ws.ovmask = 0u;
                    status = __shfl_sync(FULL, status, grp * G);
                    HPMC_STAMP(dv, wid, first, lane, 6 + 3 * (int)k);
                    __syncwarp();
                    const int myA = (status == 1) ? (int)ws.eA[grp] : -1;
                    // latency regime: lanes 0 and 1 of the cell prefetch the FP64
                    // state the lane-split update needs (own coordinate, c, s)
                    double pf_p = 0.0, pf_c = 0.0, pf_s = 0.0;
                    if (F32 && LAT && status == 1 && sl < 2) {
                        const uint32_t gA = ws.gidx[myA];
                        pf_p = sl ? B.py[gA] : B.px[gA];
                        pf_c = B.q0[gA];
                        pf_s = B.q1[gA];
                    }
                    float4 trA = make_float4(0.f, 0.f, 0.f, 0.f);
                    double2 tpA = make_double2(0.0, 0.0);
                    if (status == 1) {
                        if (F32) trA = ws.tr[grp]; else tpA = ws.tp[grp];
                    }

                    if constexpr (S == 1 && F32) {
                    // ---- one cell per warp: candidates over the lanes, survivors
                    // of the cull taken straight from its ballot (no queue); each
                    // survivor's separating axes spread over 2*nv lanes whose data
                    // arrive by shuffles from the survivor's lane
                    bool ovl = false;
                    if (status == 1) {
                        const int seg = nvv > 0 ? 2 * nvv : 2;
                        const int ppr = 32 / seg;
                        const int p = lane / seg, wi = lane - (lane / seg) * seg;
                        const int hf = wi / nvv, axk = wi - hf * nvv;
#pragma unroll 1
                        for (int t0 = 0; t0 < T && !ovl; t0 += 32) {
                            const int t = t0 + lane;
                            bool keep = false;
                            float dlx = 0.f, dly = 0.f, zbc = 0.f, zbs = 0.f;
                            int e = 0;
                            if (t < T) {
                                int q;
                                if (t0 == 0) {
                                    q = cand_q;
                                    e = cand_e;
                                } else {
                                    q = 0;
#pragma unroll
                                    for (int qq = 1; qq < 9; ++qq) q += (t >= (int)ws.pfx[0][qq]) ? 1 : 0;
                                    e = ws.beg[0][q] + (t - ws.pfx[0][q]);
                                }
                                if (e != myA) {
                                    c_cull += 1;
                                    const int ox = q % 3 - 1, oy = q / 3 - 1;
                                    const float4 f = ws.ent[e];
                                    zbc = f.z;
                                    zbs = f.w;
                                    const float Px = __fadd_rn(f.x, (float)ox * rp.w32[0]);
                                    const float Py = __fadd_rn(f.y, (float)oy * rp.w32[1]);
                                    dlx = __fsub_rn(Px, trA.x);
                                    dly = __fsub_rn(Py, trA.y);
                                    const float q32 = __fmaf_rn(dlx, dlx, __fmul_rn(dly, dly));
                                    if (q32 < rp.cull_keep) {
                                        keep = true;
                                    } else if (q32 > rp.cull_skip) {
                                        keep = false;
                                    } else {
                                        c_rechk += 1;
                                        const uint32_t gA = ws.gidx[myA];
                                        const Trial2 t2 = apply64(rp, B.px[gA], B.py[gA], B.q0[gA], B.q1[gA],
                                                                  ws.mv[jc][k - k0]);
                                        const uint32_t gB = ws.gidx[e];
                                        const double Dx = min_image(B.px[gB] - t2.x, rp.L[0], rp.halfL[0]);
                                        const double Dy = min_image(B.py[gB] - t2.y, rp.L[1], rp.halfL[1]);
                                        keep = (Dx * Dx + Dy * Dy) <= sh.rc2;
                                    }
                                }
                            }
                            // disks: a kept pair (|D|^2 <= (2R)^2) is the overlap
                            const bool rov = NV == 0 && sh.round && keep;
                            if (rov) { keep = false; c_chk += 1; }
                            if (__any_sync(FULL, rov)) ovl = true;
                            unsigned bal = __ballot_sync(FULL, keep);
#pragma unroll 1
                            while (bal != 0u && !ovl) {
                                const int np = min(__popc(bal), ppr);
                                const bool act = p < np;
                                const int src = act ? (int)__fns(bal, 0, p + 1) : lane;
                                const float sDx = __shfl_sync(FULL, dlx, src);
                                const float sDy = __shfl_sync(FULL, dly, src);
                                const float sbc = __shfl_sync(FULL, zbc, src);
                                const float sbs = __shfl_sync(FULL, zbs, src);
                                const int se = __shfl_sync(FULL, e, src);
                                bool sep = false, ovc = false;
                                if (act) {
                                    const float cr = __fmaf_rn(trA.z, sbc, __fmul_rn(trA.w, sbs));
                                    const float sr = __fmaf_rn(trA.z, sbs, -__fmul_rn(trA.w, sbc));
                                    float lx, ly, ss;
                                    if (hf == 0) {
                                        lx = __fmaf_rn(trA.z, sDx, __fmul_rn(trA.w, sDy));
                                        ly = __fmaf_rn(trA.z, sDy, -__fmul_rn(trA.w, sDx));
                                        ss = sr;
                                    } else {
                                        lx = -__fmaf_rn(sbc, sDx, __fmul_rn(sbs, sDy));
                                        ly = -__fmaf_rn(sbc, sDy, -__fmul_rn(sbs, sDx));
                                        ss = -sr;
                                    }
                                    const float g = axis_gap32<NV>(sh, axk, cr, ss, lx, ly);
                                    sep = g > rp.sat_e;
                                    ovc = g < -rp.sat_e;
                                }
                                const unsigned bs = __ballot_sync(FULL, sep);
                                const unsigned bo = __ballot_sync(FULL, ovc);
                                const unsigned segm = (seg == 32 ? FULL : ((1u << seg) - 1u)) << (p * seg);
                                bool pair_sep = false, pair_ov = false, pair_unc = false;
                                if (act) {
                                    pair_sep = (bs & segm) != 0u;
                                    pair_ov = !pair_sep && (bo & segm) == segm;
                                    pair_unc = !pair_sep && !pair_ov;
                                }
                                if (__any_sync(FULL, pair_unc)) {
                                    bool sep64 = false;
                                    if (pair_unc) {
                                        const uint32_t gA = ws.gidx[myA];
                                        const Trial2 t2 = apply64(rp, B.px[gA], B.py[gA], B.q0[gA], B.q1[gA],
                                                                  ws.mv[jc][k - k0]);
                                        const uint32_t gB = ws.gidx[se];
                                        const double Dx = min_image(B.px[gB] - t2.x, rp.L[0], rp.halfL[0]);
                                        const double Dy = min_image(B.py[gB] - t2.y, rp.L[1], rp.halfL[1]);
                                        sep64 = axis_separates64<NV>(sh, hf, axk, Dx, Dy, t2.c, t2.s, B.q0[gB],
                                                                     B.q1[gB]);
                                    }
                                    const unsigned b64 = __ballot_sync(FULL, sep64);
                                    if (pair_unc) {
                                        pair_sep = (b64 & segm) != 0u;
                                        pair_ov = !pair_sep;
                                        if (wi == 0) c_rechk += 1;
                                    }
                                }
                                if (act && wi == 0) c_chk += 1;
                                ovl = __any_sync(FULL, act && pair_ov);
                                for (int i = 0; i < np; ++i) bal &= bal - 1u;
                            }
                        }
                    }
                    if (lane == 0 && ovl) ws.ovmask = 1u;
                    __syncwarp();
                    } else {
                    // ---- cull into the pair queue, drain with overlap tests
                    int qn = 0;
#pragma unroll 1
                    for (int it = 0;; ++it) {
                        const int t = sl + it * G;
                        const bool live = (status == 1) && t < T && !((ws.ovmask >> grp) & 1u);
                        bool keep = false;
                        float2 dl = make_float2(0.f, 0.f);
                        int e = 0;
                        if (live) {
                            int q = 0;
#pragma unroll
                            for (int qq = 1; qq < 9; ++qq) q += (t >= (int)ws.pfx[grp][qq]) ? 1 : 0;
                            e = ws.beg[grp][q] + (t - ws.pfx[grp][q]);
                            if (e != myA) {
                                c_cull += 1;
                                const int ox = q % 3 - 1, oy = q / 3 - 1;
                                if (F32) {
                                    const float4 f = ws.ent[e];
                                    const float Px = __fadd_rn(f.x, (float)ox * rp.w32[0]);
                                    const float Py = __fadd_rn(f.y, (float)oy * rp.w32[1]);
                                    dl.x = __fsub_rn(Px, trA.x);
                                    dl.y = __fsub_rn(Py, trA.y);
                                    const float q32 = __fmaf_rn(dl.x, dl.x, __fmul_rn(dl.y, dl.y));
                                    if (q32 < rp.cull_keep) {
                                        keep = true;
                                    } else if (q32 > rp.cull_skip) {
                                        keep = false;
                                    } else {
                                        c_rechk += 1;
                                        const uint32_t gA = ws.gidx[myA];
                                        const Trial2 t2 = LAT ? apply64(rp, B.px[gA], B.py[gA], B.q0[gA], B.q1[gA],
                                                                        ws.mv[jc][k - k0])
                                                              : trial_of(rp, B, gA, ws.rw[grp]);
                                        const uint32_t gB = ws.gidx[e];
                                        const double Dx = min_image(B.px[gB] - t2.x, rp.L[0], rp.halfL[0]);
                                        const double Dy = min_image(B.py[gB] - t2.y, rp.L[1], rp.halfL[1]);
                                        keep = (Dx * Dx + Dy * Dy) <= sh.rc2;
                                    }
                                } else {
                                    const double2 pb = ws.ep[e];
                                    const double Dx = min_image(pb.x - tpA.x, rp.L[0], rp.halfL[0]);
                                    const double Dy = min_image(pb.y - tpA.y, rp.L[1], rp.halfL[1]);
                                    keep = (Dx * Dx + Dy * Dy) <= sh.rc2;
                                }
                            }
                        }
                        if (NV == 0 && sh.round && keep) {       // disks: kept = overlap
                            keep = false;
                            c_chk += 1;
                            atomicOr(&ws.ovmask, 1u << grp);
                        }
                        const unsigned bal = __ballot_sync(FULL, keep);
                        if (keep) {
                            const int pos = qn + __popc(bal & ((1u << lane) - 1u));
                            ws.qe[pos] = (uint16_t)e;
                            ws.qg[pos] = (uint8_t)grp;
                            ws.qd[pos] = dl;
                        }
                        qn += __popc(bal);
                        const bool any_live = __any_sync(FULL, live) != 0;
                        __syncwarp();
                        const int per_round = (LAT && F32) ? 32 / (nvv > 0 ? 2 * nvv : 2) : 32;
                        while (qn >= 32 || (!any_live && qn > 0)) {
                            const int np = qn < per_round ? qn : per_round;
                            if (LAT && F32) {
                                // one separating axis of one pair per lane
                                const int seg = nvv > 0 ? 2 * nvv : 2;
                                const int p = lane / seg;
                                const int wi = lane - p * seg;
                                const int hf = wi / nvv, axk = wi - hf * nvv;
                                const bool act = p < np && !((ws.ovmask >> ws.qg[p]) & 1u);
                                bool sep = false, ovc = false;
                                int e2 = 0, g2 = 0;
                                if (act) {
                                    e2 = ws.qe[p];
                                    g2 = ws.qg[p];
                                    const float2 d2 = ws.qd[p];
                                    const float4 ta = ws.tr[g2];
                                    const float4 fb = ws.ent[e2];
                                    const float cr = __fmaf_rn(ta.z, fb.z, __fmul_rn(ta.w, fb.w));
                                    const float sr = __fmaf_rn(ta.z, fb.w, -__fmul_rn(ta.w, fb.z));
                                    float lx, ly, cc, ss;
                                    if (hf == 0) {
                                        lx = __fmaf_rn(ta.z, d2.x, __fmul_rn(ta.w, d2.y));
                                        ly = __fmaf_rn(ta.z, d2.y, -__fmul_rn(ta.w, d2.x));
                                        cc = cr; ss = sr;
                                    } else {
                                        lx = -__fmaf_rn(fb.z, d2.x, __fmul_rn(fb.w, d2.y));
                                        ly = -__fmaf_rn(fb.z, d2.y, -__fmul_rn(fb.w, d2.x));
                                        cc = cr; ss = -sr;
                                    }
                                    const float g = axis_gap32<NV>(sh, axk, cc, ss, lx, ly);
                                    sep = g > rp.sat_e;
                                    ovc = g < -rp.sat_e;
                                }
                                const unsigned bs = __ballot_sync(FULL, sep);
                                const unsigned bo = __ballot_sync(FULL, ovc);
                                const unsigned segm = (seg == 32 ? FULL : ((1u << seg) - 1u)) << (p * seg);
                                bool pair_sep = false, pair_ov = false, pair_unc = false;
                                if (act) {
                                    pair_sep = (bs & segm) != 0u;
                                    pair_ov = !pair_sep && (bo & segm) == segm;
                                    pair_unc = !pair_sep && !pair_ov;
                                }
                                if (__any_sync(FULL, pair_unc)) {
                                    // uncertified pairs: the FP64 contract, one axis per
                                    // lane (same operations as sat_half64 for that axis)
                                    bool sep64 = false;
                                    if (pair_unc) {
                                        const uint32_t gA = ws.gidx[ws.eA[g2]];
                                        const Trial2 t2 = apply64(rp, B.px[gA], B.py[gA], B.q0[gA], B.q1[gA],
                                                                  ws.mv[j0 + g2][k - k0]);
                                        const uint32_t gB = ws.gidx[e2];
                                        const double Dx = min_image(B.px[gB] - t2.x, rp.L[0], rp.halfL[0]);
                                        const double Dy = min_image(B.py[gB] - t2.y, rp.L[1], rp.halfL[1]);
                                        sep64 = axis_separates64<NV>(sh, hf, axk, Dx, Dy, t2.c, t2.s, B.q0[gB],
                                                                     B.q1[gB]);
                                    }
                                    const unsigned b64 = __ballot_sync(FULL, sep64);
                                    if (pair_unc) {
                                        pair_sep = (b64 & segm) != 0u;
                                        pair_ov = !pair_sep;
                                        if (wi == 0) c_rechk += 1;
                                    }
                                }
                                if (act && wi == 0) {
                                    c_chk += 1;
                                    if (pair_ov) atomicOr(&ws.ovmask, 1u << g2);
                                }
                            } else if (lane < np) {
                                const int e2 = ws.qe[lane];
                                const int g2 = ws.qg[lane];
                                if (!((ws.ovmask >> g2) & 1u)) {
                                    c_chk += 1;
                                    bool ov;
                                    if (F32) {
                                        const float2 d2 = ws.qd[lane];
                                        const float4 ta = ws.tr[g2];
                                        const float4 fb = ws.ent[e2];
                                        const int v = sat32<NV>(sh, rp.sat_e, d2.x, d2.y, ta.z, ta.w, fb.z, fb.w);
                                        if (v == 2) {
                                            c_rechk += 1;
                                            const uint32_t gA = ws.gidx[ws.eA[g2]];
                                            const Trial2 t2 = trial_of(rp, B, gA, ws.rw[g2]);
                                            const uint32_t gB = ws.gidx[e2];
                                            const double Dx = min_image(B.px[gB] - t2.x, rp.L[0], rp.halfL[0]);
                                            const double Dy = min_image(B.py[gB] - t2.y, rp.L[1], rp.halfL[1]);
                                            ov = overlap2d64<NV>(sh, Dx, Dy, t2.c, t2.s, B.q0[gB], B.q1[gB]);
                                        } else {
                                            ov = (v == 1);
                                        }
                                    } else {
                                        const double2 pa = ws.tp[g2], za = ws.tz[g2];
                                        const double2 pb = ws.ep[e2], zb = ws.eo[e2];
                                        const double Dx = min_image(pb.x - pa.x, rp.L[0], rp.halfL[0]);
                                        const double Dy = min_image(pb.y - pa.y, rp.L[1], rp.halfL[1]);
                                        ov = overlap2d64<NV>(sh, Dx, Dy, za.x, za.y, zb.x, zb.y);
                                    }
                                    if (ov) atomicOr(&ws.ovmask, 1u << g2);
                                }
                            }
                            __syncwarp();
                            // move the unprocessed tail to the front
                            const int rest = qn - np;
                            uint16_t te = 0; uint8_t tg = 0; float2 td = make_float2(0.f, 0.f);
                            if (lane < rest) { te = ws.qe[np + lane]; tg = ws.qg[np + lane]; td = ws.qd[np + lane]; }
                            __syncwarp();
                            if (lane < rest) { ws.qe[lane] = te; ws.qg[lane] = tg; ws.qd[lane] = td; }
                            __syncwarp();
                            qn = rest;
                        }
                        if (!any_live && qn == 0) break;
                    }
                    }   // queue path

                    HPMC_STAMP(dv, wid, first, lane, 7 + 3 * (int)k);
                    // ---- accept or reject (one lane per cell)
                    if constexpr (F32 && LAT) {
                        // contract update split over lanes 0 (x', c') and 1 (y',
                        // s') of the cell: each FP64 instruction then serves both
                        // components (identical operations; s1 = c sd - (-s) cd
                        // rounds as c sd + s cd)
                        const bool acc = status == 1 && !((ws.ovmask >> grp) & 1u);
                        if (sl == 0 && status != 0) {
                            if (status == 2) c_rbd += 1;
                            else if (acc) c_acc += 1;
                            else c_rov += 1;
                        }
                        const bool upd = acc && sl < 2;
                        const unsigned um = __ballot_sync(FULL, upd);
                        if (upd) {
                            const int eA = ws.eA[grp];
                            const uint32_t gA = ws.gidx[eA];
                            const MoveData& m = ws.mv[jc][k - k0];
                            const double pn = wrap_pos_bits(pf_p + (sl ? m.dy : m.dx), rp.L[sl]);
                            const double v = sl ? m.sd : m.cd, z = sl ? m.cd : m.sd;
                            const double wv = sl ? -pf_s : pf_s;
                            const double q1 = pf_c * v - wv * z;
                            const double sq = q1 * q1;
                            const double n2 = sq + __shfl_xor_sync(um, sq, 1);
                            const double f = 1.5 - 0.5 * n2;
                            const double qn = q1 * f;
                            const float rel = (float)(cell_coord_bits(pn, sl ? shy : shx, rp.L[sl]) - (sl ? iwy : iwx));
                            const float fq = (float)qn;
                            const float rel_o = __shfl_xor_sync(um, rel, 1);
                            const float fq_o = __shfl_xor_sync(um, fq, 1);
                            if (sl == 0) {
                                B.px[gA] = pn;
                                B.q0[gA] = qn;
                                const float4 nf = make_float4(rel, rel_o, fq, fq_o);
                                B.f4a[gA] = nf;
                                ws.ent[eA] = nf;
                            } else {
                                B.py[gA] = pn;
                                B.q1[gA] = qn;
                            }
                        }
                    } else if (sl == 0 && status != 0) {
                        if (status == 2) {
                            c_rbd += 1;
                        } else if ((ws.ovmask >> grp) & 1u) {
                            c_rov += 1;
                        } else {
                            c_acc += 1;
                            const int eA = ws.eA[grp];
                            const uint32_t gA = ws.gidx[eA];
                            Trial2 t2;
                            if (F32) {
                                t2 = propose2d(rp, ax64, ay64, ac64, as64, ws.rw[grp][0], ws.rw[grp][1],
                                               ws.rw[grp][2], ws.rw[grp][3], ws.rw[grp][4], ws.rw[grp][5]);
                            } else {
                                t2.x = tpA.x; t2.y = tpA.y;
                                t2.c = ws.tz[grp].x; t2.s = ws.tz[grp].y;
                            }
                            B.px[gA] = t2.x; B.py[gA] = t2.y;
                            B.q0[gA] = t2.c; B.q1[gA] = t2.s;
                            const float4 nf = make_float4(
                                (float)(cell_coord_bits(t2.x, shx, rp.L[0]) - iwx),
                                (float)(cell_coord_bits(t2.y, shy, rp.L[1]) - iwy), (float)t2.c, (float)t2.s);
                            B.f4a[gA] = nf;
                            if (F32) ws.ent[eA] = nf;
                            else { ws.ep[eA] = make_double2(t2.x, t2.y); ws.eo[eA] = make_double2(t2.c, t2.s); }
                        }
                    }
                    __syncwarp();
                    HPMC_STAMP(dv, wid, first, lane, 8 + 3 * (int)k);
                }
            }
            j0 = j1;
            __syncwarp();
        }
        HPMC_STAMP(dv, wid, first, lane, 30);
        // ---- counters of this item
        c_moves = __reduce_add_sync(FULL, c_moves);
        c_acc = __reduce_add_sync(FULL, c_acc);
        c_rov = __reduce_add_sync(FULL, c_rov);
        c_rbd = __reduce_add_sync(FULL, c_rbd);
        c_cull = __reduce_add_sync(FULL, c_cull);
        c_chk = __reduce_add_sync(FULL, c_chk);
        c_rechk = __reduce_add_sync(FULL, c_rechk);
        if (lane == 0) {
            unsigned long long* C = dv.counters + (size_t)r * kNumCounters;
            atomicAdd(C + CNT_MOVES, (unsigned long long)c_moves);
            atomicAdd(C + CNT_ACCEPT, (unsigned long long)c_acc);
            atomicAdd(C + CNT_REJ_OVERLAP, (unsigned long long)c_rov);
            atomicAdd(C + CNT_REJ_BOUNDARY, (unsigned long long)c_rbd);
            atomicAdd(C + CNT_CULL, (unsigned long long)c_cull);
            atomicAdd(C + CNT_CHECKS, (unsigned long long)c_chk);
            if (c_rechk) atomicAdd(C + CNT_RECHECK, (unsigned long long)c_rechk);
        }
    }
    HPMC_STAMP_NS(dv, blockIdx.x * wpb + (threadIdx.x >> 5), lane, 29);
}

}  // namespace hpmc
