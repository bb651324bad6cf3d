// hpmc_sweep2d_direct.cuh -- one checkerboard set of the 2D sweep (Sec. 2.5.2)
// with one lane per active cell and no shared-memory staging (the
// throughput regime of large systems, where every SM has thousands of cells).
//
// Work unit: one warp takes 32 consecutive active cells of one row of one
// replica, one lane per cell.  A lane reads the begins and sizes of its 3 x 3
// stencil cells once per set and then runs its cell's nselect trial moves in
// sequence.  For every move it walks the stencil cell by cell, reading the
// FP32 mirror of each neighbour straight from the cell-sorted buffer (the
// stencils of the 32 cells of a warp overlap, so most reads hit L1), and
// culls by circumsphere.  Survivors of all lanes go to a warp-wide pair queue
// (ballot compaction) that the warp drains once the cull is done, 32 pairs at a time, one
// separating-axis test per lane, skipping pairs of moves already known to
// overlap (the early exit of Sec. 2.1).
//
// Columns and rows of the stencil that a trial cannot reach are not read:
// every particle of the lower neighbour column lies below the cell's lower
// wall, so when the trial sits farther than the circumdiameter above that
// wall (plus the certified FP32 error and the FP64 rounding of the cell
// rule), the FP64 contract culls every pair with that column; likewise for
// the upper column and the two neighbour rows.  With cells of twice the
// circumdiameter (the 2^24-pentagon system) a trial needs 4 of the 9 cells on
// average.  The decisions are the contract's either way.
//
// Each lane draws its select's Philox words itself (every lane has a move, so
// no lane idles through them), keeps the words for the FP64 contract, and
// proposes in FP32.  FP64 arithmetic runs for accepted moves and for the
// rare FP32 verdicts the certified margins cannot decide, exactly as in the
// other set kernels; it needs no select table, so no table kernel competes
// with the cell-list rebuild for the FP64 pipe.
//
// The plain FP64 form (F32 = false) keeps the structure with the contract's
// own arithmetic: the FP64 trial at the proposal (whose cell-relative
// coordinate drives the same skipping, with FP64 rounding bounds), the FP64
// circumsphere cull on positions read through L1 and the FP64
// separating-axis test in the drain.
#pragma once
#include "hpmc_sweep2d.cuh"

namespace hpmc {

struct __align__(16) Direct2Warp {
    static constexpr int QCAP = 192;
    uint32_t wd[6][32];               // Philox words r1..r6 of each lane's select
    double acc[4][32];                // the moving particle's FP64 x, y, c, s (asynchronous copies)
    float2 qd[QCAP];                  // queued Delta32 (B relative to the trial)
    float2 qz[QCAP];                  // queued B orientation (FP32 mirror)
    uint32_t qe[QCAP];                // queued B slot in the sorted buffer
    uint8_t qg[QCAP];                 // queued owner lane
    float2 tz[32];                    // FP32 trial orientation of each lane's move
    uint32_t ea[32];                  // sorted slot of each lane's moving particle
    uint32_t sb[9][32];               // stencil cell q of each lane: sorted begin
    uint32_t sn[9][32];               // and size
    unsigned int ovmask;              // lanes whose move overlaps
};

// asynchronous global -> shared copies of the issuing thread (cp.async);
// the thread's own later wait makes them visible to it
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// The rare FP64 paths stay out of line, so that their registers do not
// weigh on the common path of the kernel.  Each recomputes the contract's
// trial of the moving particle (slot gA) from its select's words w[0..5].

// in-cell test of the FP64 contract trial (FP32 verdict not certified)
__device__ __noinline__ bool direct_in_cell64(const Rep& rp, const Bufs& B, const uint32_t* w, uint32_t gA,
                                              double shx, double shy, int ix, int iy)
{
    const Trial2 t2 = propose2d(rp, B.px[gA], B.py[gA], B.q0[gA], B.q1[gA], w[0], w[1], w[2], w[3], w[4], w[5]);
    return cell_axis(t2.x, shx, rp.L[0], rp.inv_w[0], rp.nc[0]) == ix &&
           cell_axis(t2.y, shy, rp.L[1], rp.inv_w[1], rp.nc[1]) == iy;
}

// circumsphere cull of the FP64 contract (FP32 verdict not certified)
__device__ __noinline__ bool direct_keep64(const Rep& rp, double rc2, const Bufs& B, const uint32_t* w, uint32_t gA,
                                           uint32_t gB)
{
    const Trial2 t2 = propose2d(rp, B.px[gA], B.py[gA], B.q0[gA], B.q1[gA], w[0], w[1], w[2], w[3], w[4], w[5]);
    const double Dx = min_image(B.px[gB] - t2.x, rp.L[0], rp.halfL[0]);
    const double Dy = min_image(B.py[gB] - t2.y, rp.L[1], rp.halfL[1]);
    return (Dx * Dx + Dy * Dy) <= rc2;
}

// separating-axis test of the FP64 contract on a queued pair (FP32 verdict
// not certified)
template <int NV>
__device__ __noinline__ bool direct_overlap64(const Shape2& sh, const Rep& rp, const Bufs& B, const uint32_t* w,
                                              uint32_t gA, uint32_t gB)
{
    const Trial2 t2 = propose2d(rp, B.px[gA], B.py[gA], B.q0[gA], B.q1[gA], w[0], w[1], w[2], w[3], w[4], w[5]);
    const double Dx = min_image(B.px[gB] - t2.x, rp.L[0], rp.halfL[0]);
    const double Dy = min_image(B.py[gB] - t2.y, rp.L[1], rp.halfL[1]);
    return overlap2d64<NV>(sh, Dx, Dy, t2.c, t2.s, B.q0[gB], B.q1[gB]);
}

// One round of the pair queue: the np entries [base, base + np), one per lane,
// each a certified FP32 separating-axis test (the FP64 contract when the
// FP32 verdict is not certified); a pair whose owner already overlaps is
// skipped.  Adds the tests run and the FP64 re-checks to chk, rechk.
template <int NV, bool F32>
__device__ __forceinline__ void direct_drain_round(Direct2Warp& ws, int lane, int base, int np, const Shape2& sh,
                                                   const Rep& rp, const Bufs& B, unsigned& chk, unsigned& rechk)
{
    if (lane < np) {
        const int p = base + lane;
        const int g2 = ws.qg[p];
        if (!((ws.ovmask >> g2) & 1u)) {
            chk += 1;
            bool pov;
            if constexpr (F32) {
                const float2 d2 = ws.qd[p], zb = ws.qz[p], za = ws.tz[g2];
                const int v = sat32<NV>(sh, rp.sat_e, d2.x, d2.y, za.x, za.y, zb.x, zb.y);
                pov = v == 1;
                if (v == 2) {
                    rechk += 1;
                    const uint32_t w[6] = { ws.wd[0][g2], ws.wd[1][g2], ws.wd[2][g2],
                                            ws.wd[3][g2], ws.wd[4][g2], ws.wd[5][g2] };
                    pov = direct_overlap64<NV>(sh, rp, B, w, ws.ea[g2], ws.qe[p]);
                }
            } else {
                // FP64 form: the contract's test on the owner's trial (ws.acc)
                const uint32_t gB = ws.qe[p];
                const double Dx = min_image(B.px[gB] - ws.acc[0][g2], rp.L[0], rp.halfL[0]);
                const double Dy = min_image(B.py[gB] - ws.acc[1][g2], rp.L[1], rp.halfL[1]);
                pov = overlap2d64<NV>(sh, Dx, Dy, ws.acc[2][g2], ws.acc[3][g2], B.q0[gB], B.q1[gB]);
            }
            if (pov) atomicOr(&ws.ovmask, 1u << g2);
        }
    }
    __syncwarp();
}

// the same round out of line, for a queue about to overflow inside the cull
// loop (rare): the loop then carries no separating-axis registers
template <int NV, bool F32>
__device__ __noinline__ uint2 direct_drain_round_out(Direct2Warp& ws, int lane, int base, int np, const Shape2& sh,
                                                     const Rep& rp, const Bufs& B)
{
    unsigned chk = 0, rechk = 0;
    direct_drain_round<NV, F32>(ws, lane, base, np, sh, rp, B, chk, rechk);
    return make_uint2(chk, rechk);
}

template <int NV, bool F32>
__global__ void __launch_bounds__(256, 2)
k_set2d_direct(Dev dv, Shape2 sh, int nxt, int sigma, const uint32_t* __restrict__ item_base)
{
    pdl_wait();
    using W = Direct2Warp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    W& ws = reinterpret_cast<W*>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const unsigned lt_mask = (1u << lane) - 1u;
    const Bufs B = dv.buf[nxt];
    const uint32_t* __restrict__ start = dv.start;
    const uint32_t nitems = item_base[dv.R];
    const uint32_t wpb = blockDim.x >> 5;

    for (uint32_t item = blockIdx.x * wpb + (threadIdx.x >> 5); item < nitems; item += gridDim.x * wpb) {
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
        const int spr = (nax + 31) / 32;
        const uint32_t local = item - __ldg(item_base + r);
        const int row = (int)(local / spr);
        const int strip = (int)(local - (uint32_t)row * spr);
        const int iy = 2 * row + ((sigma >> 1) & 1);
        const int jx = strip * 32 + lane;
        const bool valid = jx < nax;
        const int ix = (sigma & 1) + 2 * jx;
        const uint64_t sweep = dv.sweep[r] - 1;           // the running sweep
        const uint32_t nsel = rp.nselect;
        const uint32_t cell_local = (uint32_t)ix + (uint32_t)nc0 * (uint32_t)iy;
        const float wx = rp.w32[0], wy = rp.w32[1];
        const uint64_t seed = rp.seed;

        // ---- stencil cells, q = 3 (oy + 1) + (ox + 1): sorted begin and size
        uint32_t T = 0, cb = 0, n_c = 0;
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            uint32_t b = 0u, n = 0u;
            if (valid) {
                const int ox = q % 3 - 1, oy = q / 3 - 1;
                int cx = ix + ox, cy = iy + oy;
                cx = cx < 0 ? cx + nc0 : (cx >= nc0 ? cx - nc0 : cx);
                cy = cy < 0 ? cy + nc1 : (cy >= nc1 ? cy - nc1 : cy);
                const uint32_t c = rp.cbase + (uint32_t)cx + (uint32_t)nc0 * (uint32_t)cy;
                b = start[c];
                n = start[c + 1] - b;
            }
            ws.sb[q][lane] = b;
            ws.sn[q][lane] = n;
            T += n;
            if (q == 4) { cb = b; n_c = n; }
        }
        const bool live_cell = valid && n_c > 0;
        unsigned c_moves = 0, c_acc = 0, c_rov = 0, c_rbd = 0, c_cull = 0, c_chk = 0, c_rechk = 0;
        uint32_t eA_prev = 0xffffffffu;                    // slot this lane moved in its last select

#pragma unroll 1
        for (uint32_t k = 0; k < nsel; ++k) {
            // ---- propose: FP32 trial from the select record
            int status = 0;                                // 0 idle, 1 in the cell, 2 left it
            uint32_t eA = 0;
            float4 tr = make_float4(0.f, 0.f, 0.f, 0.f);
            double rx64 = 0.0, ry64 = 0.0;                 // FP64 form: the trial's cell-relative position
            if constexpr (F32) cp_async_wait_all();        // the last accept's operands
            if (!F32 && live_cell) {
                // FP64 form: the contract's trial itself, kept in ws.acc for the
                // cull, the separating-axis tests and the accept
                c_moves += 1;
                const uint4 b0 = move_block(seed, sweep, (uint32_t)sigma, cell_local, k, 0);
                const uint4 b1 = move_block(seed, sweep, (uint32_t)sigma, cell_local, k, 1);
                eA = cb + __umulhi(b0.x, n_c);
                const Trial2 t2 = propose2d(rp, B.px[eA], B.py[eA], B.q0[eA], B.q1[eA], b0.y, b0.z, b0.w, b1.x, b1.y,
                                            b1.z);
                ws.acc[0][lane] = t2.x;
                ws.acc[1][lane] = t2.y;
                ws.acc[2][lane] = t2.c;
                ws.acc[3][lane] = t2.s;
                status = (cell_axis(t2.x, dv.shift[3 * r], rp.L[0], rp.inv_w[0], rp.nc[0]) == ix &&
                          cell_axis(t2.y, dv.shift[3 * r + 1], rp.L[1], rp.inv_w[1], rp.nc[1]) == iy) ? 1 : 2;
                rx64 = cell_coord_bits(t2.x, dv.shift[3 * r], rp.L[0]) - (double)ix * rp.w[0];
                ry64 = cell_coord_bits(t2.y, dv.shift[3 * r + 1], rp.L[1]) - (double)iy * rp.w[1];
                ws.ea[lane] = eA;
            }
            if (F32 && live_cell) {
                c_moves += 1;
                // Philox words of select k of this cell (Sec. 2.5: one stream per trial move)
                const uint4 b0 = move_block(seed, sweep, (uint32_t)sigma, cell_local, k, 0);
                const uint4 b1 = move_block(seed, sweep, (uint32_t)sigma, cell_local, k, 1);
                eA = cb + __umulhi(b0.x, n_c);
                // a plain load: this lane may have written the slot earlier in the set
                const float4 f = B.f4a[eA];
                // the accept's FP64 operands, copied while the move is decided
                // (a slot this lane just moved is already staged, with its new state)
                if (eA != eA_prev) {
                    cp_async8(&ws.acc[0][lane], B.px + eA);
                    cp_async8(&ws.acc[1][lane], B.py + eA);
                    cp_async8(&ws.acc[2][lane], B.q0 + eA);
                    cp_async8(&ws.acc[3][lane], B.q1 + eA);
                }
                cp_async_commit();
                ws.wd[0][lane] = b0.y; ws.wd[1][lane] = b0.z; ws.wd[2][lane] = b0.w;
                ws.wd[3][lane] = b1.x; ws.wd[4][lane] = b1.y; ws.wd[5][lane] = b1.z;
                // FP32 trial (the deltas as the select table computes them)
                const float fdx = __fmul_rn(rp.d32, m24(b0.y));
                const float fdy = __fmul_rn(rp.d32, m24(b0.w));
                const float ft = __fmul_rn(rp.tau32, m24(b1.y));
                const float ftt = __fmul_rn(ft, ft);
                const float finv = __frcp_rn(__fadd_rn(1.0f, ftt));
                const float fcd = __fmul_rn(__fsub_rn(1.0f, ftt), finv);
                const float fsd = __fmul_rn(__fadd_rn(ft, ft), finv);
                const float rx = __fadd_rn(f.x, fdx), ry = __fadd_rn(f.y, fdy);
                const float cz = __fmaf_rn(f.z, fcd, -__fmul_rn(f.w, fsd));
                const float sz = __fmaf_rn(f.z, fsd, __fmul_rn(f.w, fcd));
                tr = make_float4(rx, ry, cz, sz);
                const bool out = rx < rp.out_lo || ry < rp.out_lo || rx > rp.out_hi[0] || ry > rp.out_hi[1];
                const bool in = rx > rp.in_lo && ry > rp.in_lo && rx < rp.in_hi[0] && ry < rp.in_hi[1];
                if (out) {
                    status = 2;
                } else if (in) {
                    status = 1;
                } else {
                    c_rechk += 1;
                    const uint32_t w[6] = { b0.y, b0.z, b0.w, b1.x, b1.y, b1.z };
                    status = direct_in_cell64(rp, B, w, eA, dv.shift[3 * r], dv.shift[3 * r + 1], ix, iy) ? 1 : 2;
                }
                ws.tz[lane] = make_float2(cz, sz);
                ws.ea[lane] = eA;
            }
            if (lane == 0) ws.ovmask = 0u;
            __syncwarp();

            // ---- the stencil cells within reach of the trial, and their candidates
            uint32_t mask = 0u, Tn = 0u;
            if (status == 1) {
                // (the FP64 form tests its FP64 trial coordinate)
                const bool need_l = F32 ? !(tr.x > rp.reach_lo[0]) : !(rx64 > rp.reach64_lo[0]);
                const bool need_r = F32 ? !(tr.x < rp.reach_hi[0]) : !(rx64 < rp.reach64_hi[0]);
                const bool need_b = F32 ? !(tr.y > rp.reach_lo[1]) : !(ry64 > rp.reach64_lo[1]);
                const bool need_t = F32 ? !(tr.y < rp.reach_hi[1]) : !(ry64 < rp.reach64_hi[1]);
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const int ox = q % 3 - 1, oy = q / 3 - 1;
                    const bool need = (ox < 0 ? need_l : (ox > 0 ? need_r : true)) &&
                                      (oy < 0 ? need_b : (oy > 0 ? need_t : true));
                    const uint32_t n = ws.sn[q][lane];
                    if (need && n) {
                        mask |= 1u << q;
                        Tn += n;
                    }
                }
                c_cull += T - 1u;                          // the stencil's candidates (self excluded)
            }
            bool ov = false;                               // this lane's move overlaps
            int qn = 0;


            // ---- cull: a cursor over the lane's candidates, cell by cell of its
            // mask, the next candidate's data loaded one trip ahead
            const uint32_t trips = __reduce_max_sync(FULL, Tn);
            uint32_t m_left = mask;
            uint32_t ec = 0, eend = 0;
            float oxc = 0.f, oyc = 0.f;                    // FP32 offset of the cursor's cell
            float4 fc = make_float4(0.f, 0.f, 0.f, 0.f);
            double xc = 0.0, yc = 0.0;                     // FP64 form: the next candidate's position
            const double tx64 = F32 ? 0.0 : ws.acc[0][lane], ty64 = F32 ? 0.0 : ws.acc[1][lane];
            auto fetch = [&]() {
                if constexpr (F32) {
                    fc = B.f4a[ec];
                } else {
                    xc = B.px[ec];
                    yc = B.py[ec];
                }
            };
            // the cell the cursor enters next: its range and offset
            auto enter = [&]() {
                const int kq = __ffs(m_left) - 1;
                m_left &= m_left - 1u;
                ec = ws.sb[kq][lane];
                eend = ec + ws.sn[kq][lane];
                const int qy = (kq * 11) >> 5;             // kq / 3 for kq < 9
                const int qx = kq - 3 * qy;
                oxc = qx == 0 ? -wx : (qx == 2 ? wx : 0.f);
                oyc = qy == 0 ? -wy : (qy == 2 ? wy : 0.f);
            };
            if (Tn) {
                enter();
                fetch();
            }
#pragma unroll 1
            for (uint32_t i = 0; i < trips; ++i) {
                const bool live = i < Tn && !ov;
                const uint32_t e = ec;
                const float offx = oxc, offy = oyc;
                const float4 f = fc;
                const double xe = xc, ye = yc;
                if (live && i + 1 < Tn) {                  // advance and prefetch
                    ec += 1u;
                    if (ec == eend) enter();
                    fetch();
                }
                bool keep = false;
                float dlx = 0.f, dly = 0.f;
                if (!F32 && live && e != eA) {
                    // FP64 form: the contract's circumsphere cull
                    const double Dx = min_image(xe - tx64, rp.L[0], rp.halfL[0]);
                    const double Dy = min_image(ye - ty64, rp.L[1], rp.halfL[1]);
                    keep = (Dx * Dx + Dy * Dy) <= sh.rc2;
                    if (NV == 0 && sh.round && keep) {     // disks: a kept pair is the overlap
                        keep = false;
                        c_chk += 1;
                        ov = true;
                    }
                }
                if (F32 && live && e != eA) {
                    dlx = __fsub_rn(__fadd_rn(f.x, offx), tr.x);
                    dly = __fsub_rn(__fadd_rn(f.y, offy), tr.y);
                    const float q32 = __fmaf_rn(dlx, dlx, __fmul_rn(dly, dly));
                    if (q32 < rp.cull_keep) {
                        keep = true;
                    } else if (q32 > rp.cull_skip) {
                        keep = false;
                    } else {
                        c_rechk += 1;
                        const uint32_t w[6] = { ws.wd[0][lane], ws.wd[1][lane], ws.wd[2][lane],
                                                ws.wd[3][lane], ws.wd[4][lane], ws.wd[5][lane] };
                        keep = direct_keep64(rp, sh.rc2, B, w, eA, e);
                    }
                    if (NV == 0 && sh.round && keep) {     // disks: a kept pair is the overlap
                        keep = false;
                        c_chk += 1;
                        ov = true;
                    }
                }
                const unsigned bal = __ballot_sync(FULL, keep);
                if (keep) {
                    const int p = qn + __popc(bal & lt_mask);
                    if (F32) {
                        ws.qd[p] = make_float2(dlx, dly);
                        ws.qz[p] = make_float2(f.z, f.w);
                    }
                    ws.qe[p] = e;
                    ws.qg[p] = (uint8_t)lane;
                }
                qn += __popc(bal);
                if (qn > W::QCAP - 32) {                   // room for one more trip's survivors
                    __syncwarp();
                    const uint2 cr = direct_drain_round_out<NV, F32>(ws, lane, qn - 32, 32, sh, rp, B);
                    c_chk += cr.x;
                    c_rechk += cr.y;
                    qn -= 32;
                    ov = ov || ((ws.ovmask >> lane) & 1u);
                }
            }
            // ---- separating-axis tests of the queued pairs, 32 at a time
            __syncwarp();
            while (qn > 0) {
                const int np = min(qn, 32);
                direct_drain_round<NV, F32>(ws, lane, qn - np, np, sh, rp, B, c_chk, c_rechk);
                qn -= np;
            }
            ov = ov || ((ws.ovmask >> lane) & 1u);
            __syncwarp();

            // ---- accept or reject
            eA_prev = 0xffffffffu;
            if (status == 2) {
                c_rbd += 1;
            } else if (status == 1) {
                if (ov) {
                    c_rov += 1;
                } else {
                    c_acc += 1;
                    Trial2 t2;
                    if constexpr (F32) {
                        cp_async_wait_all();
                        t2 = propose2d(rp, ws.acc[0][lane], ws.acc[1][lane], ws.acc[2][lane], ws.acc[3][lane],
                                       ws.wd[0][lane], ws.wd[1][lane], ws.wd[2][lane], ws.wd[3][lane],
                                       ws.wd[4][lane], ws.wd[5][lane]);
                    } else {
                        t2.x = ws.acc[0][lane];                // the trial computed at the proposal
                        t2.y = ws.acc[1][lane];
                        t2.c = ws.acc[2][lane];
                        t2.s = ws.acc[3][lane];
                    }
                    B.px[eA] = t2.x;
                    B.py[eA] = t2.y;
                    B.q0[eA] = t2.c;
                    B.q1[eA] = t2.s;
                    // keep the new state staged for a next select of the same particle
                    ws.acc[0][lane] = t2.x;
                    ws.acc[1][lane] = t2.y;
                    ws.acc[2][lane] = t2.c;
                    ws.acc[3][lane] = t2.s;
                    eA_prev = eA;
                    // cell origins i * w of the relative coordinates (as in k_place)
                    const double shx = dv.shift[3 * r], shy = dv.shift[3 * r + 1];
                    const double iwx = (double)ix * rp.w[0];
                    const double iwy = (double)iy * rp.w[1];
                    B.f4a[eA] = make_float4((float)(cell_coord_bits(t2.x, shx, rp.L[0]) - iwx),
                                            (float)(cell_coord_bits(t2.y, shy, rp.L[1]) - iwy), (float)t2.c,
                                            (float)t2.s);
                }
            }
            __syncwarp();
        }
        cp_async_wait_all();
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
}

}  // namespace hpmc
