// hpmc_sweep3d.cuh -- one checkerboard set of the 3D sweep (Sec. 2.5.2, 8 sets).
//
// Same organisation as the 2D kernel: one warp takes a strip of S = 32/G
// consecutive active cells along x of one (y, z) row of one replica; the nine
// neighbour rows that the strip's 3x3x3 stencils touch are contiguous ranges
// of the cell-sorted state and are staged into shared memory with coalesced
// 16-byte loads.  The nselect moves of a cell are sequential; the cells of a
// warp run in lockstep; the G lanes of a cell split its circumsphere cull;
// survivors go to a warp-wide shared-memory pair queue drained 32 pairs at a
// time, one pair per lane (GJK is a long sequential iteration, so a pair is
// not split further), skipping pairs of moves already known to overlap.
//
// F32 = true : cull and in-cell decisions certified in FP32; each pair runs
//              the certified FP32 GJK (hpmc_gjk32.cuh); the pairs it cannot
//              certify are then re-decided by the FP64 contract GJK, one pair
//              at a time by the whole warp (hpmc_gjk64w.cuh).
// F32 = false: plain FP64 contract.
#pragma once
#include "hpmc_device.cuh"
#include "hpmc_gjk32.cuh"
#include "hpmc_mpr32.cuh"
#include "hpmc_gjk64w.cuh"

namespace hpmc {

// Random words and orientation step of one select (state independent).  The
// latency-regime kernels (G >= 8) load the first chunk of a cell's selects
// from the table k_selects wrote for the sweep (selects.cu); later chunks,
// and every chunk of the other kernels, are computed here, one (cell,
// select) per lane.
struct __align__(16) MoveData3 {
    double dq[4];        // (1, v) / sqrt(1 + v.v), the contract's orientation step
    uint32_t w[12];      // words r1..r12
    uint32_t r0;         // pick word
    uint32_t pad;
};

__device__ __forceinline__ MoveData3 precompute_select3(const Rep& rp, uint64_t seed, uint64_t sweep,
                                                        uint32_t sigma, uint32_t cell, uint32_t k)
{
    uint32_t w16[16];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint4 bb = move_block(seed, sweep, sigma, cell, k, (uint32_t)b);
        w16[4 * b] = bb.x; w16[4 * b + 1] = bb.y; w16[4 * b + 2] = bb.z; w16[4 * b + 3] = bb.w;
    }
    MoveData3 m;
    m.r0 = w16[0];
#pragma unroll
    for (int q = 0; q < 12; ++q) m.w[q] = w16[q + 1];
    orient_step3(rp, w16, m.dq);
    m.pad = 0;
    return m;
}

template <int G, bool F32>
struct Warp3 {
    static constexpr int S = 32 / G;                  // cells per strip
    static constexpr int M = 2 * S + 1;               // staged cells per row
    static constexpr int CAPX = 9 * M * 4;
    static constexpr int CAP = CAPX < 256 ? 256 : (CAPX > 1024 ? 1024 : CAPX);
    static constexpr int QCAP = 64;
    float4 ea[F32 ? CAP : 1];                         // FP32 rel.x, rel.y, rel.z, qw
    float4 eb[F32 ? CAP : 1];                         // FP32 qx, qy, qz, -
    double ep[F32 ? 1 : CAP][3];                      // FP64 position
    double eq[F32 ? 1 : CAP][4];                      // FP64 quaternion
    uint32_t gidx[CAP];
    uint16_t sbeg[9][M + 1];
    uint32_t rowinfo[10][4];                          // per row: offset, entries before the x wrap, starts

    uint16_t beg[S][27];
    uint16_t pfx[S][28];
    // FP32 form: stencil position t of the strip's cell g -> staged entry e
    // and stencil cell q, as e | q << 10 at tab[tb[g] + t] (e < CAP <= 1024,
    // q < 27).  The cells' stencils overlap in one column, so they hold at
    // most twice the staged entries.
    uint16_t tab[F32 ? 2 * CAP : 1];
    uint16_t tb[S];
    float4 qoff[F32 ? 27 : 1];                        // FP32 offsets (ox w, oy w, oz w) of stencil cell q
    float4 qd[QCAP];                                  // queued Delta32
    uint16_t qe[QCAP];
    uint8_t qg[QCAP];
    float4 tra[S], trb[S];                            // FP32 trial: rel', qw' / qx', qy', qz'
    double tp[S][3], tq[S][4];                        // FP64 trial (position: FP64 form; orientation: both)
    uint32_t rw[S][12];                               // words r1..r12
    uint16_t eA[S];
    MoveData3 mv[S][G];                               // selects of the current chunk
    unsigned int ovmask;
};

__device__ __forceinline__ uint32_t row_count3(const uint32_t* start, uint32_t rowbase, int nc0, int xa, int len)
{
    if (xa + len <= nc0) return start[rowbase + xa + len] - start[rowbase + xa];
    return (start[rowbase + nc0] - start[rowbase + xa]) + (start[rowbase + (xa + len - nc0)] - start[rowbase]);
}

// FP64 trial position of the contract from words r1..r6 (the position part
// of propose3d, same operations); the rare FP64 paths of the FP32 form take
// the trial orientation from the proposal (ws.tq) instead of recomputing it.
__device__ __forceinline__ void trial3_pos(const Rep& rp, const Bufs& B, uint32_t gA, const uint32_t* w12,
                                           double x[3])
{
    x[0] = wrap_pos_bits(B.px[gA] + rp.d_s * pm53(w12[0], w12[1]), rp.L[0]);
    x[1] = wrap_pos_bits(B.py[gA] + rp.d_s * pm53(w12[2], w12[3]), rp.L[1]);
    x[2] = wrap_pos_bits(B.pz[gA] + rp.d_s * pm53(w12[4], w12[5]), rp.L[2]);
}

template <int G, bool F32, int NV>
// One block of up to 256 threads per SM is enough residency for these
// latency-bound kernels; the register budget that buys (up to 255 a thread)
// keeps the inlined FP32 GJK free of spills (measured: cubes +15%,
// dodecahedra +15% against a 128-register cap).
__global__ void __launch_bounds__(256, 1)
k_set3d(Dev dv, const __grid_constant__ Shape3 sh, int nxt, int sigma, const uint32_t* __restrict__ item_base)
{
    pdl_wait();
    using W = Warp3<G, F32>;
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
    const uint32_t wid = blockIdx.x * wpb + (threadIdx.x >> 5);
    const MoveData3* __restrict__ msel = static_cast<const MoveData3*>(dv.msel);
    const uint32_t mstride = dv.msel_stride;
    HPMC_STAMP_NS(dv, wid, lane, 28);

    for (uint32_t item = wid; item < nitems; item += gridDim.x * wpb) {
        const bool first = item == wid;
        (void)first;
        HPMC_STAMP(dv, wid, first, lane, 0);
        uint32_t lo = 0, hi = dv.R;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(item_base + mid) <= item) lo = mid; else hi = mid;
        }
        const uint32_t r = lo;
        const Rep& rp = dv.reps[r];
        const int nc0 = rp.nc[0], nc1 = rp.nc[1], nc2 = rp.nc[2];
        const int nax = nc0 >> 1;
        const int spr = (nax + S - 1) / S;
        const uint32_t local = item - __ldg(item_base + r);
        const int row = (int)(local / spr);
        const int strip = (int)(local - (uint32_t)row * spr);
        const int ny2 = nc1 >> 1;
        const int iy = 2 * (row % ny2) + ((sigma >> 1) & 1);
        const int iz = 2 * (row / ny2) + ((sigma >> 2) & 1);
        const int jfirst = strip * S;
        const int Sv = min(S, nax - jfirst);
        const uint64_t sweep = dv.sweep[r] - 1;
        const double shx = dv.shift[3 * r], shy = dv.shift[3 * r + 1], shz = dv.shift[3 * r + 2];
        const uint64_t seed = rp.seed;
        const uint32_t nsel = rp.nselect;
        unsigned c_moves = 0, c_acc = 0, c_rov = 0, c_rbd = 0, c_cull = 0, c_chk = 0, c_rechk = 0, c_cap = 0;
        uint32_t rowbase[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int jy = (iy + (q % 3) - 1 + nc1) % nc1;
            const int jz = (iz + (q / 3) - 1 + nc2) % nc2;
            rowbase[q] = rp.cbase + (uint32_t)nc0 * ((uint32_t)jy + (uint32_t)nc1 * (uint32_t)jz);
        }
        const double iwy = (double)iy * rp.w[1];
        const double iwz = (double)iz * rp.w[2];
        HPMC_STAMP(dv, wid, first, lane, 1);

        int j0 = 0;
        while (j0 < Sv) {
            // ---- sub-strip [j0, j1) whose nine staged rows fit CAP: every
            // cell start of the nine rows is loaded at once (one round trip)
            constexpr int NCH = (W::M + 31) / 32;       // 32-column chunks per row
            int j1 = Sv;
            bool skip_cell = false;
            int xa = 0, Mp = 0;
            uint32_t s0[9][NCH], cnt[9][NCH];
            for (;;) {
                xa = ((sigma & 1) + 2 * (jfirst + j0) - 1 + nc0) % nc0;
                Mp = 2 * (j1 - j0) + 1;
                uint32_t mine = 0;
#pragma unroll
                for (int q = 0; q < 9; ++q)
#pragma unroll
                    for (int ch = 0; ch < NCH; ++ch) {
                        const int m = ch * 32 + lane;
                        s0[q][ch] = 0u;
                        cnt[q][ch] = 0u;
                        if (m < Mp) {
                            const uint32_t c = rowbase[q] + (uint32_t)((xa + m) % nc0);
                            const uint32_t a0 = start[c];
                            s0[q][ch] = a0;
                            cnt[q][ch] = start[c + 1] - a0;
                            mine += cnt[q][ch];
                        }
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
            const int mwrap = (xa + Mp > nc0) ? nc0 - xa : Mp;   // first column wrapped to x = 0
            // ---- staged begin of every cell (per-row scans of the counts)
            uint32_t off = 0;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                uint32_t run = 0, at_wrap = 0, gb = 0;
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
                    if (m < Mp) ws.sbeg[q][m] = (uint16_t)(off + excl);
                    if (mwrap < Mp && mwrap >= ch * 32 && mwrap < ch * 32 + 32) {
                        at_wrap = __shfl_sync(FULL, excl, mwrap - ch * 32);
                        gb = __shfl_sync(FULL, s0[q][ch], mwrap - ch * 32);
                    }
                    run += __shfl_sync(FULL, incl, 31);
                }
                const uint32_t ga = __shfl_sync(FULL, s0[q][0], 0);
                if (mwrap >= Mp) at_wrap = run;
                if (lane == 0) {
                    ws.sbeg[q][Mp] = (uint16_t)(off + run);
                    ws.rowinfo[q][0] = off;
                    ws.rowinfo[q][1] = at_wrap;
                    ws.rowinfo[q][2] = ga;
                    ws.rowinfo[q][3] = gb;
                }
                off += run;
            }
            if (lane == 0) ws.rowinfo[9][0] = off;
            __syncwarp();
            // ---- stage every entry of the nine rows: four entries a lane in
            // flight (all loads issued before the first store)
            auto entry_of = [&](uint32_t t) {
                int q = 0;
#pragma unroll
                for (int qq = 1; qq < 9; ++qq) q += (t >= ws.rowinfo[qq][0]) ? 1 : 0;
                const uint32_t u = t - ws.rowinfo[q][0];
                const uint32_t la = ws.rowinfo[q][1];
                return u < la ? ws.rowinfo[q][2] + u : ws.rowinfo[q][3] + (u - la);
            };
            if constexpr (F32) {
                for (uint32_t t0 = lane; t0 < off; t0 += 128) {
                    uint32_t gi[4];
                    float4 fa[4], fb[4];
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4) {
                        const uint32_t t = t0 + 32u * k4;
                        if (t < off) {
                            gi[k4] = entry_of(t);
                            fa[k4] = B.f4a[gi[k4]];
                            fb[k4] = B.f4b[gi[k4]];
                        }
                    }
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4) {
                        const uint32_t t = t0 + 32u * k4;
                        if (t < off) {
                            ws.gidx[t] = gi[k4];
                            ws.ea[t] = fa[k4];
                            ws.eb[t] = fb[k4];
                        }
                    }
                }
            } else {
                for (uint32_t t = lane; t < off; t += 32) {
                    const uint32_t gi = entry_of(t);
                    ws.gidx[t] = gi;
                    ws.ep[t][0] = B.px[gi]; ws.ep[t][1] = B.py[gi]; ws.ep[t][2] = B.pz[gi];
                    ws.eq[t][0] = B.q0[gi]; ws.eq[t][1] = B.q1[gi];
                    ws.eq[t][2] = B.q2[gi]; ws.eq[t][3] = B.q3[gi];
                }
            }
            __syncwarp();
            HPMC_STAMP(dv, wid, first, lane, 3);
            // ---- stencil tables
            const bool valid = grp < (j1 - j0);
            const int mc = 1 + 2 * grp;
            const int ix = (sigma & 1) + 2 * (jfirst + j0 + grp);
            const uint32_t cell_local = (uint32_t)ix + (uint32_t)nc0 * ((uint32_t)iy + (uint32_t)nc1 * (uint32_t)iz);
            const double iwx = (double)ix * rp.w[0];
            if (sl == 0) {
                uint16_t p = 0;
                ws.pfx[grp][0] = 0;
#pragma unroll
                for (int q = 0; q < 27; ++q) {
                    const int qr = q / 3, qc = q % 3;            // row (y, z), column x
                    const uint16_t b = valid ? ws.sbeg[qr][mc - 1 + qc] : 0;
                    const uint16_t e = valid ? ws.sbeg[qr][mc + qc] : 0;
                    ws.beg[grp][q] = b;
                    p = (uint16_t)(p + (e - b));
                    ws.pfx[grp][q + 1] = p;
                }
            }
            __syncwarp();
            const uint32_t cb = valid ? ws.sbeg[4][mc] : 0;    // centre row (y, z) = q 4
            const uint32_t n_c = valid ? (uint32_t)ws.sbeg[4][mc + 1] - cb : 0;
            const int T = ws.pfx[grp][27];
            uint32_t tbase = 0;
            if constexpr (F32) {
                // the entry table, once per sub-strip instead of a search of
                // the 27 stencil prefixes for every candidate of every select
                if (lane == 0) {
                    uint32_t acc = 0;
                    for (int g = 0; g < S; ++g) {
                        ws.tb[g] = (uint16_t)acc;
                        acc += ws.pfx[g][27];
                    }
                }
                if (lane < 27)
                    ws.qoff[lane] = make_float4((float)(lane % 3 - 1) * rp.w32[0], (float)((lane / 3) % 3 - 1) * rp.w32[1],
                                                (float)(lane / 9 - 1) * rp.w32[2], 0.f);
                __syncwarp();
                tbase = ws.tb[grp];
                for (int t = sl; t < T; t += G) {
                    int q = 0;
#pragma unroll
                    for (int qq = 1; qq < 27; ++qq) q += (t >= (int)ws.pfx[grp][qq]) ? 1 : 0;
                    ws.tab[tbase + t] = (uint16_t)((ws.beg[grp][q] + (t - ws.pfx[grp][q])) | (q << 10));
                }
                __syncwarp();
            }
            const bool live_cell = valid && n_c > 0;

#pragma unroll 1
            HPMC_STAMP(dv, wid, first, lane, 4);
#pragma unroll 1
            for (uint32_t k0 = 0; k0 < nsel; k0 += G) {
            // ---- Philox words and orientation steps of a chunk of selects, one
            // (cell, select) per lane
            {
                const uint32_t kk = k0 + (uint32_t)sl;
                if (live_cell && kk < nsel) {
                    if (G >= 8 && k0 == 0)
                        ws.mv[grp][sl] = msel[(size_t)(rp.cbase + cell_local) * mstride + kk];
                    else
                        ws.mv[grp][sl] = precompute_select3(rp, seed, sweep, (uint32_t)sigma, cell_local, kk);
                }
                __syncwarp();
            }
            const uint32_t kend = min(nsel, k0 + (uint32_t)G);
#pragma unroll 1
            for (uint32_t k = k0; k < kend; ++k) {
                const MoveData3& m = ws.mv[grp][k - k0];
                int status = 0;
                if (sl == 0 && live_cell) {
                    c_moves += 1;
                    const uint32_t eA = cb + __umulhi(m.r0, n_c);
#pragma unroll
                    for (int q = 0; q < 12; ++q) ws.rw[grp][q] = m.w[q];
                    ws.eA[grp] = (uint16_t)eA;
                    if (F32) {
                        const float4 fa = ws.ea[eA];
                        const float rx = __fadd_rn(fa.x, __fmul_rn(rp.d32, m24(m.w[0])));
                        const float ry = __fadd_rn(fa.y, __fmul_rn(rp.d32, m24(m.w[2])));
                        const float rz = __fadd_rn(fa.z, __fmul_rn(rp.d32, m24(m.w[4])));
                        ws.tra[grp] = make_float4(rx, ry, rz, 0.f);
                        const bool out = rx < rp.out_lo || ry < rp.out_lo || rz < rp.out_lo || rx > rp.out_hi[0] ||
                                         ry > rp.out_hi[1] || rz > rp.out_hi[2];
                        const bool in = rx > rp.in_lo && ry > rp.in_lo && rz > rp.in_lo && rx < rp.in_hi[0] &&
                                        ry < rp.in_hi[1] && rz < rp.in_hi[2];
                        if (out) {
                            status = 2;
                        } else if (in) {
                            status = 1;
                        } else {
                            c_rechk += 1;
                            double x[3];
                            trial3_pos(rp, B, ws.gidx[eA], ws.rw[grp], x);
                            const bool ok = cell_axis(x[0], shx, rp.L[0], rp.inv_w[0], nc0) == ix &&
                                            cell_axis(x[1], shy, rp.L[1], rp.inv_w[1], nc1) == iy &&
                                            cell_axis(x[2], shz, rp.L[2], rp.inv_w[2], nc2) == iz;
                            status = ok ? 1 : 2;
                        }
                    } else {
                        double x[3];
                        x[0] = wrap_pos_bits(ws.ep[eA][0] + rp.d_s * pm53(m.w[0], m.w[1]), rp.L[0]);
                        x[1] = wrap_pos_bits(ws.ep[eA][1] + rp.d_s * pm53(m.w[2], m.w[3]), rp.L[1]);
                        x[2] = wrap_pos_bits(ws.ep[eA][2] + rp.d_s * pm53(m.w[4], m.w[5]), rp.L[2]);
#pragma unroll
                        for (int a = 0; a < 3; ++a) ws.tp[grp][a] = x[a];
                        const bool ok = cell_axis(x[0], shx, rp.L[0], rp.inv_w[0], nc0) == ix &&
                                        cell_axis(x[1], shy, rp.L[1], rp.inv_w[1], nc1) == iy &&
                                        cell_axis(x[2], shz, rp.L[2], rp.inv_w[2], nc2) == iz;
                        status = ok ? 1 : 2;
                    }
                }
                if (lane == 0) ws.ovmask = 0u;
                status = __shfl_sync(FULL, status, grp * G);
                __syncwarp();
                // ---- trial orientation of the contract, only for moves that stay
                // in their cell; with 4+ lanes per cell each of lanes 0..3
                // computes one quaternion component (same operations)
                {
                    constexpr int NQ = G >= 4 ? 4 : 1;
                    const bool on = status == 1 && sl < NQ;
                    const unsigned om = __ballot_sync(FULL, on);
                    if (on) {
                        const int eA = ws.eA[grp];
                        double qa[4];
                        if (F32) {
                            const uint32_t gA = ws.gidx[eA];
                            qa[0] = B.q0[gA]; qa[1] = B.q1[gA]; qa[2] = B.q2[gA]; qa[3] = B.q3[gA];
                        } else {
#pragma unroll
                            for (int a = 0; a < 4; ++a) qa[a] = ws.eq[eA][a];
                        }
                        if constexpr (NQ == 4) {
                            const double c = qmul_component(qa, m.dq, sl);
                            const double sq = c * c;
                            const int base = grp * G;
                            const double s0 = __shfl_sync(om, sq, base), s1 = __shfl_sync(om, sq, base + 1);
                            const double s2 = __shfl_sync(om, sq, base + 2), s3 = __shfl_sync(om, sq, base + 3);
                            const double n2 = ((s0 + s1) + s2) + s3;
                            const double f = 1.5 - 0.5 * n2;
                            const double o = c * f;
                            ws.tq[grp][sl] = o;
                            if (F32) {
                                if (sl == 0) ws.tra[grp].w = (float)o;
                                else if (sl == 1) ws.trb[grp].x = (float)o;
                                else if (sl == 2) ws.trb[grp].y = (float)o;
                                else ws.trb[grp].z = (float)o;
                            }
                        } else {
                            double o[4];
                            orient_apply3(qa, m.dq, o);
#pragma unroll
                            for (int a = 0; a < 4; ++a) ws.tq[grp][a] = o[a];
                            if (F32) {
                                ws.tra[grp].w = (float)o[0];
                                ws.trb[grp] = make_float4((float)o[1], (float)o[2], (float)o[3], 0.f);
                            }
                        }
                    }
                }
                if (k < 7) HPMC_STAMP(dv, wid, first, lane, 6 + 3 * (int)k);
                __syncwarp();
                const int myA = (status == 1) ? (int)ws.eA[grp] : -1;
                float4 ta = make_float4(0.f, 0.f, 0.f, 0.f);
                double tpx = 0.0, tpy = 0.0, tpz = 0.0;
                if (status == 1) {
                    if (F32) ta = ws.tra[grp];
                    else { tpx = ws.tp[grp][0]; tpy = ws.tp[grp][1]; tpz = ws.tp[grp][2]; }
                }
                // ---- cull into the pair queue, drain with GJK
                int qn = 0;
#pragma unroll 1
                for (int it = 0;; ++it) {
                    const int t = sl + it * G;
                    const bool live = (status == 1) && t < T && !((ws.ovmask >> grp) & 1u);
                    bool keep = false, ins = false;
                    float4 dl = make_float4(0.f, 0.f, 0.f, 0.f);
                    int e = 0;
                    if (live) {
                        int q = 0;
                        if constexpr (F32) {
                            const uint32_t te = ws.tab[tbase + t];
                            e = (int)(te & 1023u);
                            q = (int)(te >> 10);
                        } else {
#pragma unroll
                            for (int qq = 1; qq < 27; ++qq) q += (t >= (int)ws.pfx[grp][qq]) ? 1 : 0;
                            e = ws.beg[grp][q] + (t - ws.pfx[grp][q]);
                        }
                        if (e != myA) {
                            c_cull += 1;
                            if (F32) {
                                const float4 f = ws.ea[e];
                                const float4 o = ws.qoff[q];
                                dl.x = __fsub_rn(__fadd_rn(f.x, o.x), ta.x);
                                dl.y = __fsub_rn(__fadd_rn(f.y, o.y), ta.y);
                                dl.z = __fsub_rn(__fadd_rn(f.z, o.z), ta.z);
                                const float q32 = __fmaf_rn(dl.x, dl.x, __fmaf_rn(dl.y, dl.y, __fmul_rn(dl.z, dl.z)));
                                if (q32 < rp.ins32) {
                                    ins = true;                    // inscribed balls meet
                                } else if (q32 < rp.cull_keep) {
                                    keep = true;
                                } else if (q32 > rp.cull_skip) {
                                    keep = false;
                                } else {
                                    c_rechk += 1;
                                    double x[3];
                                    trial3_pos(rp, B, ws.gidx[myA], ws.rw[grp], x);
                                    const uint32_t gB = ws.gidx[e];
                                    const double Dx = min_image(B.px[gB] - x[0], rp.L[0], rp.halfL[0]);
                                    const double Dy = min_image(B.py[gB] - x[1], rp.L[1], rp.halfL[1]);
                                    const double Dz = min_image(B.pz[gB] - x[2], rp.L[2], rp.halfL[2]);
                                    keep = ((Dx * Dx + Dy * Dy) + Dz * Dz) <= sh.rc2;
                                }
                            } else {
                                const double Dx = min_image(ws.ep[e][0] - tpx, rp.L[0], rp.halfL[0]);
                                const double Dy = min_image(ws.ep[e][1] - tpy, rp.L[1], rp.halfL[1]);
                                const double Dz = min_image(ws.ep[e][2] - tpz, rp.L[2], rp.halfL[2]);
                                const double q2 = (Dx * Dx + Dy * Dy) + Dz * Dz;
                                ins = q2 < rp.ins64;
                                keep = !ins && q2 <= sh.rc2;
                            }
                        }
                    }
                    if (NV == 0 && sh.round && keep) {           // spheres: kept = overlap
                        keep = false;
                        ins = true;
                    }
                    if (ins) {
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
                    while (qn >= 32 || (!any_live && qn > 0)) {
                        const int np = qn < 32 ? qn : 32;
                        bool need64 = false;                       // FP32 verdict uncertain
                        if (lane < np) {
                            const int e2 = ws.qe[lane];
                            const int g2 = ws.qg[lane];
                            if (!((ws.ovmask >> g2) & 1u)) {
                                c_chk += 1;
                                bool ov = false;
                                int its = 0;
                                if (F32) {
                                    const float4 d2 = ws.qd[lane];
                                    const float4 a1 = ws.tra[g2], a2 = ws.trb[g2];
                                    const float4 b1 = ws.ea[e2], b2 = ws.eb[e2];
                                    const float4 qa = make_float4(a1.w, a2.x, a2.y, a2.z);
                                    const float4 qb = make_float4(b1.w, b2.x, b2.y, b2.z);
                                    int v;
                                    if ((NV == 8 || NV == 0) && sh.box)
                                        v = box32_sat(sh, d2.x, d2.y, d2.z, qa, qb, rp.box_esep, rp.box_eov);
                                    else if (NV != 8 && sh.mpr)       // (8 vertices: boxes, else GJK)
                                        v = mpr32_cert<NV>(sh, d2.x, d2.y, d2.z, qa, qb, rp.e_pb32, rp.e_va32,
                                                           rp.tau3);
                                    else
                                        v = gjk32_cert<NV>(sh, d2.x, d2.y, d2.z, qa, qb, rp.e_pb32, rp.e_va32,
                                                           rp.tau3);
                                    need64 = v >= GJK32_UNCERTAIN;
                                    ov = (v == GJK32_OVERLAP);
                                } else {
                                    const double D[3] = { min_image(ws.ep[e2][0] - ws.tp[g2][0], rp.L[0], rp.halfL[0]),
                                                          min_image(ws.ep[e2][1] - ws.tp[g2][1], rp.L[1], rp.halfL[1]),
                                                          min_image(ws.ep[e2][2] - ws.tp[g2][2], rp.L[2], rp.halfL[2]) };
                                    const double qa[4] = { ws.tq[g2][0], ws.tq[g2][1], ws.tq[g2][2], ws.tq[g2][3] };
                                    const double qb[4] = { ws.eq[e2][0], ws.eq[e2][1], ws.eq[e2][2], ws.eq[e2][3] };
                                    ov = overlap3d64<NV>(sh, D, qa, qb, &its);
                                }
                                if (its > kGjkMaxIt) c_cap += 1;
                                if (ov) atomicOr(&ws.ovmask, 1u << g2);
                            }
                        }
                        if (F32) {
                            // the uncertain pairs, one at a time by the whole warp
                            // (FP64 contract; a pair whose cell already overlaps
                            // is skipped: its move is rejected either way)
                            unsigned um = __ballot_sync(FULL, need64);
                            __syncwarp();
#pragma unroll 1
                            while (um != 0u) {
                                const int src = __ffs(um) - 1;
                                um &= um - 1u;
                                const int g2 = ws.qg[src];
                                if ((ws.ovmask >> g2) & 1u) continue;
                                const int e2 = ws.qe[src];
                                double x[3];
                                trial3_pos(rp, B, ws.gidx[ws.eA[g2]], ws.rw[g2], x);
                                const uint32_t gB = ws.gidx[e2];
                                const double D[3] = { min_image(B.px[gB] - x[0], rp.L[0], rp.halfL[0]),
                                                      min_image(B.py[gB] - x[1], rp.L[1], rp.halfL[1]),
                                                      min_image(B.pz[gB] - x[2], rp.L[2], rp.halfL[2]) };
                                const double qa[4] = { ws.tq[g2][0], ws.tq[g2][1], ws.tq[g2][2], ws.tq[g2][3] };
                                const double qB[4] = { B.q0[gB], B.q1[gB], B.q2[gB], B.q3[gB] };
                                int its = 0;
                                bool ov;
                                const int bv = ((NV == 8 || NV == 0) && sh.box)
                                                   ? box64_sat_warp(sh, D, qa, qB, rp.box_sep64, rp.box_ov64)
                                                   : 2;
                                if (bv < 2) ov = bv == 1;
                                else ov = overlap3d64_warp<NV>(sh, D, qa, qB, &its);
                                if (lane == src) {
                                    c_rechk += 1;
                                    if (its > kGjkMaxIt) c_cap += 1;
                                }
                                if (ov && lane == 0) ws.ovmask |= 1u << g2;
                                __syncwarp();
                            }
                        }
                        __syncwarp();
                        const int rest = qn - np;
                        uint16_t te = 0; uint8_t tg = 0; float4 td = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (lane < rest) { te = ws.qe[np + lane]; tg = ws.qg[np + lane]; td = ws.qd[np + lane]; }
                        __syncwarp();
                        if (lane < rest) { ws.qe[lane] = te; ws.qg[lane] = tg; ws.qd[lane] = td; }
                        __syncwarp();
                        qn = rest;
                    }
                    if (!any_live && qn == 0) break;
                }
                if (k < 7) HPMC_STAMP(dv, wid, first, lane, 7 + 3 * (int)k);
                // ---- accept or reject
                if (sl == 0 && status != 0) {
                    if (status == 2) {
                        c_rbd += 1;
                    } else if ((ws.ovmask >> grp) & 1u) {
                        c_rov += 1;
                    } else {
                        c_acc += 1;
                        const int eA = ws.eA[grp];
                        const uint32_t gA = ws.gidx[eA];
                        Trial3 t3;
                        if (F32) {
                            // position from the words; orientation as computed at the proposal
                            const uint32_t* w = ws.rw[grp];
                            t3.x[0] = wrap_pos_bits(B.px[gA] + rp.d_s * pm53(w[0], w[1]), rp.L[0]);
                            t3.x[1] = wrap_pos_bits(B.py[gA] + rp.d_s * pm53(w[2], w[3]), rp.L[1]);
                            t3.x[2] = wrap_pos_bits(B.pz[gA] + rp.d_s * pm53(w[4], w[5]), rp.L[2]);
#pragma unroll
                            for (int a = 0; a < 4; ++a) t3.q[a] = ws.tq[grp][a];
                        } else {
#pragma unroll
                            for (int a = 0; a < 3; ++a) t3.x[a] = ws.tp[grp][a];
#pragma unroll
                            for (int a = 0; a < 4; ++a) t3.q[a] = ws.tq[grp][a];
                        }
                        B.px[gA] = t3.x[0]; B.py[gA] = t3.x[1]; B.pz[gA] = t3.x[2];
                        B.q0[gA] = t3.q[0]; B.q1[gA] = t3.q[1]; B.q2[gA] = t3.q[2]; B.q3[gA] = t3.q[3];
                        const float4 na = make_float4((float)(cell_coord_bits(t3.x[0], shx, rp.L[0]) - iwx),
                                                      (float)(cell_coord_bits(t3.x[1], shy, rp.L[1]) - iwy),
                                                      (float)(cell_coord_bits(t3.x[2], shz, rp.L[2]) - iwz),
                                                      (float)t3.q[0]);
                        const float4 nb = make_float4((float)t3.q[1], (float)t3.q[2], (float)t3.q[3], 0.f);
                        B.f4a[gA] = na;
                        B.f4b[gA] = nb;
                        if (F32) { ws.ea[eA] = na; ws.eb[eA] = nb; }
                        else {
#pragma unroll
                            for (int a = 0; a < 3; ++a) ws.ep[eA][a] = t3.x[a];
#pragma unroll
                            for (int a = 0; a < 4; ++a) ws.eq[eA][a] = t3.q[a];
                        }
                    }
                }
                __syncwarp();
                if (k < 7) HPMC_STAMP(dv, wid, first, lane, 8 + 3 * (int)k);
            }
            }   // chunks of selects
            j0 = j1;
            __syncwarp();
        }
        HPMC_STAMP(dv, wid, first, lane, 30);
        c_moves = __reduce_add_sync(FULL, c_moves);
        c_acc = __reduce_add_sync(FULL, c_acc);
        c_rov = __reduce_add_sync(FULL, c_rov);
        c_rbd = __reduce_add_sync(FULL, c_rbd);
        c_cull = __reduce_add_sync(FULL, c_cull);
        c_chk = __reduce_add_sync(FULL, c_chk);
        c_rechk = __reduce_add_sync(FULL, c_rechk);
        c_cap = __reduce_add_sync(FULL, c_cap);
#ifdef HPMC_TRACE
        // point 31 of the traced item: its FP64 re-checks (a count, not a stamp)
        if (first && lane == 0 && dv.trace && wid < dv.trace_warps)
            dv.trace[(size_t)wid * kTracePoints + 31] = c_rechk;
#endif
        if (lane == 0) {
            unsigned long long* C = dv.counters + (size_t)r * kNumCounters;
            atomicAdd(C + CNT_MOVES, (unsigned long long)c_moves);
            atomicAdd(C + CNT_ACCEPT, (unsigned long long)c_acc);
            atomicAdd(C + CNT_REJ_OVERLAP, (unsigned long long)c_rov);
            atomicAdd(C + CNT_REJ_BOUNDARY, (unsigned long long)c_rbd);
            atomicAdd(C + CNT_CULL, (unsigned long long)c_cull);
            atomicAdd(C + CNT_CHECKS, (unsigned long long)c_chk);
            if (c_rechk) atomicAdd(C + CNT_RECHECK, (unsigned long long)c_rechk);
            if (c_cap) atomicAdd(C + CNT_GJKCAP, (unsigned long long)c_cap);
        }
    }
    HPMC_STAMP_NS(dv, wid, lane, 29);
}

}  // namespace hpmc
