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
// a warp-wide shared-memory pair queue (ballot compaction) that all 32 lanes
// drain with full overlap tests, 32 pairs per round, skipping pairs of moves
// already known to overlap (early exit on the first overlap, Sec. 2.1 /
// Sec. 2.5.3 block queue, rebuilt at warp granularity with __ballot_sync).
//
// F32 = true : every decision is first taken in FP32 with the certified
//              margins of Rep (hpmc_bounds.h); FP64 only for accepted moves
//              and uncertified verdicts.  F32 = false: plain FP64 contract.
#pragma once
#include "hpmc_device.cuh"
#include "hpmc_filter.cuh"

namespace hpmc {

template <int G, bool F32>
struct Warp2 {
    static constexpr int S = 32 / G;                  // cells per strip
    static constexpr int M = 2 * S + 1;               // staged cells per row
    static constexpr int CAPX = 9 * M;
    static constexpr int CAP = CAPX < 128 ? 128 : (CAPX > 512 ? 512 : CAPX);
    static constexpr int QCAP = 64;
    float4 ent[F32 ? CAP : 1];                        // FP32: rel.x, rel.y, c, s
    double2 ep[F32 ? 1 : CAP];                        // FP64: x, y
    double2 eo[F32 ? 1 : CAP];                        // FP64: c, s
    uint32_t gidx[CAP];                               // sorted slot of each entry
    uint16_t sbeg[3][M + 1];                          // staged begin of each cell
    float2 qd[QCAP];                                  // queued Delta32 (FP32 form)
    uint16_t qe[QCAP];                                // queued neighbour entry
    uint8_t qg[QCAP];                                 // queued group (cell)
    float4 tr[S];                                     // FP32 trial rel', z'
    double2 tp[S], tz[S];                             // FP64 trial x', z' (FP64 form)
    uint32_t rw[S][6];                                // words r1..r6 of the move
    uint16_t eA[S];                                   // entry of the moving particle
    unsigned int ovmask;                              // cells whose move overlaps
};

// Number of particles in cells x0 .. x0+len-1 (periodic in x) of one row.
__device__ __forceinline__ uint32_t row_count(const uint32_t* start, uint32_t rowbase, int nc0,
                                              int x0, int len)
{
    const int xa = (x0 + nc0) % nc0;
    if (xa + len <= nc0) return start[rowbase + xa + len] - start[rowbase + xa];
    return (start[rowbase + nc0] - start[rowbase + xa]) +
           (start[rowbase + (xa + len - nc0)] - start[rowbase]);
}

// FP64 trial of the move of group gq (recomputed from the words; rare path
// in the FP32 form, every move in the FP64 form).
__device__ __forceinline__ Trial2 trial_of(const Rep& rp, const Bufs& B, uint32_t gA,
                                           const uint32_t* w)
{
    return propose2d(rp, B.px[gA], B.py[gA], B.q0[gA], B.q1[gA], w[0], w[1], w[2], w[3], w[4], w[5]);
}

template <int G, bool F32, int NV>
__global__ void __launch_bounds__(256)
k_set2d(Dev dv, Shape2 sh, int nxt, int sigma, const uint32_t* __restrict__ item_base)
{
    using W = Warp2<G, F32>;
    constexpr int S = W::S;
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

    for (uint32_t item = blockIdx.x * wpb + (threadIdx.x >> 5); item < nitems;
         item += gridDim.x * wpb) {
        // ---- replica and strip of this work item
        uint32_t lo = 0, hi = dv.R;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (item_base[mid] <= item) lo = mid; else hi = mid;
        }
        const uint32_t r = lo;
        const Rep rp = dv.reps[r];
        const int nc0 = rp.nc[0], nc1 = rp.nc[1];
        const int nax = nc0 >> 1;
        const int spr = (nax + S - 1) / S;
        const uint32_t local = item - item_base[r];
        const int row = (int)(local / spr);
        const int strip = (int)(local - (uint32_t)row * spr);
        const int iy = 2 * row + ((sigma >> 1) & 1);
        const int jfirst = strip * S;
        const int Sv = min(S, nax - jfirst);
        const uint64_t sweep = dv.sweep[r] - 1;          // the running sweep
        const double shx = dv.shift[3 * r], shy = dv.shift[3 * r + 1];
        unsigned long long c_moves = 0, c_acc = 0, c_rov = 0, c_rbd = 0, c_cull = 0, c_chk = 0,
                           c_rechk = 0;
        uint32_t rowbase[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) rowbase[q] = rp.cbase + (uint32_t)nc0 * (uint32_t)((iy - 1 + q + nc1) % nc1);

        int j0 = 0;
        while (j0 < Sv) {
            // ---- choose the sub-strip [j0, j1) whose staged rows fit CAP
            int j1 = Sv;
            bool skip_cell = false;
            for (;;) {
                const int x0 = (sigma & 1) + 2 * (jfirst + j0) - 1;
                const int len = 2 * (j1 - j0) + 1;
                uint32_t tot = 0;
#pragma unroll
                for (int q = 0; q < 3; ++q) tot += row_count(start, rowbase[q], nc0, x0, len);
                if (tot <= (uint32_t)W::CAP) break;
                if (j1 == j0 + 1) { skip_cell = true; break; }
                j1 = j0 + (j1 - j0) / 2;
            }
            if (skip_cell) {
                if (lane == 0) atomicOr(dv.error, ERR_CAPACITY);
                j0 += 1;
                continue;
            }
            const int x0 = (sigma & 1) + 2 * (jfirst + j0) - 1;
            const int Mp = 2 * (j1 - j0) + 1;
            // ---- stage the three rows
            uint32_t off = 0;
#pragma unroll 1
            for (int q = 0; q < 3; ++q) {
                const int xa = (x0 + nc0) % nc0;
                uint32_t run = 0;
                int mwrap = Mp;                          // first m that wrapped to x = 0
                for (int mb = 0; mb < Mp; mb += 32) {
                    const int m = mb + lane;
                    uint32_t cnt = 0;
                    if (m < Mp) {
                        const int xm = (xa + m) % nc0;
                        const uint32_t c = rowbase[q] + (uint32_t)xm;
                        cnt = start[c + 1] - start[c];
                    }
                    uint32_t incl = cnt;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t t = __shfl_up_sync(FULL, incl, o);
                        if (lane >= o) incl += t;
                    }
                    if (m < Mp) ws.sbeg[q][m] = (uint16_t)(off + run + incl - cnt);
                    run += __shfl_sync(FULL, incl, 31);
                }
                if (lane == 0) ws.sbeg[q][Mp] = (uint16_t)(off + run);
                if (xa + Mp > nc0) mwrap = nc0 - xa;
                const uint32_t gA0 = start[rowbase[q] + xa];
                const uint32_t gB0 = start[rowbase[q]];
                __syncwarp();
                const uint32_t lenA = (mwrap < Mp) ? (uint32_t)ws.sbeg[q][mwrap] - off : run;
                for (uint32_t t = lane; t < run; t += 32) {
                    const uint32_t gi = t < lenA ? gA0 + t : gB0 + (t - lenA);
                    const uint32_t si = off + t;
                    ws.gidx[si] = gi;
                    if (F32) {
                        ws.ent[si] = B.f4a[gi];
                    } else {
                        ws.ep[si] = make_double2(B.px[gi], B.py[gi]);
                        ws.eo[si] = make_double2(B.q0[gi], B.q1[gi]);
                    }
                }
                off += run;
            }
            __syncwarp();

            // ---- my cell and its 3x3 stencil inside the staged rows
            const int jc = j0 + grp;
            const bool valid = grp < (j1 - j0);
            const int mc = 1 + 2 * grp;
            const int ix = (sigma & 1) + 2 * (jfirst + jc);
            const uint32_t cell_local = (uint32_t)ix + (uint32_t)nc0 * (uint32_t)iy;
            int pfx[10];
            int beg[9];
            uint32_t n_c = 0, cb = 0;
            if (valid) {
                cb = ws.sbeg[1][mc];
                n_c = ws.sbeg[1][mc + 1] - cb;
                pfx[0] = 0;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const int qr = q / 3, qc = q % 3;
                    beg[q] = ws.sbeg[qr][mc - 1 + qc];
                    pfx[q + 1] = pfx[q] + (ws.sbeg[qr][mc + qc] - beg[q]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 9; ++q) { beg[q] = 0; pfx[q + 1] = 0; }
                pfx[0] = 0;
            }
            const int T = pfx[9];
            const bool live_cell = valid && n_c > 0;

#pragma unroll 1
            for (uint32_t k = 0; k < rp.nselect; ++k) {
                // ---- propose (one lane per cell)
                int status = 0;                       // 0 idle, 1 active, 2 left the cell
                if (sl == 0 && live_cell) {
                    const uint4 b0 = move_block(rp.seed, sweep, (uint32_t)sigma, cell_local, k, 0);
                    const uint4 b1 = move_block(rp.seed, sweep, (uint32_t)sigma, cell_local, k, 1);
                    const uint32_t wr[6] = { b0.y, b0.z, b0.w, b1.x, b1.y, b1.z };
                    const uint32_t eA = cb + __umulhi(b0.x, n_c);
#pragma unroll
                    for (int q = 0; q < 6; ++q) ws.rw[grp][q] = wr[q];
                    ws.eA[grp] = (uint16_t)eA;
                    c_moves += 1;
                    if (F32) {
                        const float4 f = ws.ent[eA];
                        const float dx = __fmul_rn(rp.d32, m24(wr[0]));
                        const float dy = __fmul_rn(rp.d32, m24(wr[2]));
                        const float t = __fmul_rn(rp.tau32, m24(wr[4]));
                        const float rx = __fadd_rn(f.x, dx), ry = __fadd_rn(f.y, dy);
                        float cz, sz;
                        rotate32(f.z, f.w, t, cz, sz);
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
                            const Trial2 t2 = trial_of(rp, B, ws.gidx[eA], wr);
                            const bool ok = cell_axis(t2.x, shx, rp.L[0], rp.inv_w[0], nc0) == ix &&
                                            cell_axis(t2.y, shy, rp.L[1], rp.inv_w[1], nc1) == iy;
                            status = ok ? 1 : 2;
                        }
                    } else {
                        const double2 p = ws.ep[eA], o = ws.eo[eA];
                        const Trial2 t2 = propose2d(rp, p.x, p.y, o.x, o.y, wr[0], wr[1], wr[2], wr[3],
                                                    wr[4], wr[5]);
                        ws.tp[grp] = make_double2(t2.x, t2.y);
                        ws.tz[grp] = make_double2(t2.c, t2.s);
                        const bool ok = cell_axis(t2.x, shx, rp.L[0], rp.inv_w[0], nc0) == ix &&
                                        cell_axis(t2.y, shy, rp.L[1], rp.inv_w[1], nc1) == iy;
                        status = ok ? 1 : 2;
                    }
                }
                if (lane == 0) ws.ovmask = 0u;
                status = __shfl_sync(FULL, status, grp * G);
                __syncwarp();
                const int myA = (status == 1) ? (int)ws.eA[grp] : -1;
                float4 trA = make_float4(0.f, 0.f, 0.f, 0.f);
                double2 tpA = make_double2(0.0, 0.0);
                if (status == 1) {
                    if (F32) trA = ws.tr[grp]; else tpA = ws.tp[grp];
                }

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
                        for (int qq = 1; qq < 9; ++qq) q += (t >= pfx[qq]) ? 1 : 0;
                        e = beg[q] + (t - pfx[q]);
                        if (e != myA) {
                            c_cull += 1;
                            const int ox = q % 3 - 1, oy = q / 3 - 1;
                            if (F32) {
                                const float4 f = ws.ent[e];
                                const float Px = __fadd_rn(f.x, (float)ox * rp.w32[0]);
                                const float Py = __fadd_rn(f.y, (float)oy * rp.w32[1]);
                                dl.x = __fsub_rn(Px, trA.x);
                                dl.y = __fsub_rn(Py, trA.y);
                                const float q32 = __fadd_rn(__fmul_rn(dl.x, dl.x), __fmul_rn(dl.y, dl.y));
                                if (q32 < rp.cull_keep) {
                                    keep = true;
                                } else if (q32 > rp.cull_skip) {
                                    keep = false;
                                } else {
                                    c_rechk += 1;
                                    const uint32_t gA = ws.gidx[myA];
                                    const Trial2 t2 = trial_of(rp, B, gA, ws.rw[grp]);
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
                    while (qn >= 32 || (!any_live && qn > 0)) {
                        const int np = qn < 32 ? qn : 32;
                        if (lane < np) {
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

                // ---- accept or reject (one lane per cell)
                if (sl == 0 && status != 0) {
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
                            t2 = trial_of(rp, B, gA, ws.rw[grp]);
                        } else {
                            t2.x = tpA.x; t2.y = tpA.y;
                            t2.c = ws.tz[grp].x; t2.s = ws.tz[grp].y;
                        }
                        B.px[gA] = t2.x; B.py[gA] = t2.y;
                        B.q0[gA] = t2.c; B.q1[gA] = t2.s;
                        const float4 nf = make_float4(
                            (float)rel_in_cell(t2.x, shx, rp.L[0], rp.w[0], ix),
                            (float)rel_in_cell(t2.y, shy, rp.L[1], rp.w[1], iy), (float)t2.c, (float)t2.s);
                        B.f4a[gA] = nf;
                        if (F32) ws.ent[eA] = nf;
                        else { ws.ep[eA] = make_double2(t2.x, t2.y); ws.eo[eA] = make_double2(t2.c, t2.s); }
                    }
                }
                __syncwarp();
            }
            j0 = j1;
            __syncwarp();
        }
        // ---- counters of this item
        c_moves = __reduce_add_sync(FULL, (unsigned)c_moves);
        c_acc = __reduce_add_sync(FULL, (unsigned)c_acc);
        c_rov = __reduce_add_sync(FULL, (unsigned)c_rov);
        c_rbd = __reduce_add_sync(FULL, (unsigned)c_rbd);
        c_cull = __reduce_add_sync(FULL, (unsigned)c_cull);
        c_chk = __reduce_add_sync(FULL, (unsigned)c_chk);
        c_rechk = __reduce_add_sync(FULL, (unsigned)c_rechk);
        if (lane == 0) {
            unsigned long long* C = dv.counters + (size_t)r * kNumCounters;
            atomicAdd(C + CNT_MOVES, c_moves);
            atomicAdd(C + CNT_ACCEPT, c_acc);
            atomicAdd(C + CNT_REJ_OVERLAP, c_rov);
            atomicAdd(C + CNT_REJ_BOUNDARY, c_rbd);
            atomicAdd(C + CNT_CULL, c_cull);
            atomicAdd(C + CNT_CHECKS, c_chk);
            if (c_rechk) atomicAdd(C + CNT_RECHECK, c_rechk);
        }
    }
}

}  // namespace hpmc
