// The list-mode MLEM hot path (Eq. iter with Eq. kernel over 3-sigma windows).
//
// One persistent block per SM pulls work items (an image tile and a run of the
// events whose window centre lies in it) from an atomic queue.  For each item it
// stages rho' = s*rho of the tile plus a halo that holds every window of those
// events in shared memory and zeroes an accumulator of the same shape.  Warps
// are grouped (G warps per group); a group takes one event at a time and each of
// its lanes takes one image row of the event's window (or one segment of it):
//   pass 1: walk the lane's chord of the ellipse, evaluate P (Eq. kernel) in the
//           log2 domain (one rsqrt and one ex2 per pixel), keep P in registers
//           and accumulate D_j = sum P rho' (the denominator of Eq. iter);
//           warp shuffles and one named barrier reduce D_j over the group;
//   pass 2: add P / D_j into the shared accumulator (shared-memory atomics; two
//           groups may touch the same pixel).
// At the end of the item the accumulator is flushed to the global
// back-projection A with one atomic add per touched pixel; the finalize kernel
// then forms rho <- rho * A.  This replaces the paper's warp-per-event kernel
// with texture reads (Sec. 4.2) by row-per-lane evaluation, a register cache of
// P between the passes (the paper caches in shared memory and registers too),
// and shared-memory accumulation of the scatter.
#pragma once

#include "tsp_device.cuh"

namespace tsp {

// Per-lane row constants.  For m = 0 .. len-1 the lane's pixel m has
//   u = u0 + m dz,  Q = aCa + 2 oCb = Q0 + m dQ,
//   A = sqrt(log2e/2) aCb = A0 + m dA,  s = sqrt(log2e iz) u = su0 + m dsu,
// and Eq. kernel becomes
//   P = Q^(-1/2) 2^(C0 - s^2 + A^2/Q),  C0 = log2 K - (log2e/2) 4 il Dy^2 c2i,
// K = det^(1/2)(C^-1) / (2 pi^2) (reading R4).
struct RowK {
    int len, sbase;
    float Q0, dQ, A0, dA, su0, dsu, C0;
};

// Extra row constants of the sigma-gradient (adjoint) pass:
//   u = u0 + m du, aCb = b0 + m db (unscaled), Qz/2 = qz0 + m dqz,
//   Cz = cz0 + m dcz, and the row constants kz = 1/iz, kl = 1/(2 il) - Bl/2,
//   Cl, Ql/2 (see the derivative formulas in the gradient pass).
struct RowG {
    float u0, du, b0, db, qz0, dqz, cz0, dcz, kz, kl, cl, qlh;
};

// An idle lane: no pixels, and constants that keep its (discarded) pass-1
// arithmetic finite.
template <bool GRAD>
__device__ __forceinline__ void row_idle(RowK& r, RowG& rg)
{
    r.len = 0;
    r.sbase = 0;
    r.Q0 = 1.0f; r.dQ = 0.0f; r.A0 = 0.0f; r.dA = 0.0f; r.su0 = 0.0f; r.dsu = 0.0f;
    r.C0 = -126.0f;
    if (GRAD) {
        rg.u0 = rg.du = rg.b0 = rg.db = rg.qz0 = rg.dqz = rg.cz0 = rg.dcz = 0.0f;
        rg.kz = rg.kl = rg.cl = rg.qlh = 0.0f;
    }
}

// Row constants of lane row iy (segment seg) for a buffer whose element 0 is
// pixel (oy, oz), with row stride `stride` and extent rh x rw.  The event
// preparation guarantees that every chord lies inside that extent; the clamp
// below keeps every access in bounds regardless (clipped pixels are counted).
template <int LMAX, bool GRAD>
__device__ __forceinline__ void make_row(const Geo& g, const float4& ev, const double4* ev64,
                                         int iy, int seg, int oy, int oz, int stride, int rh,
                                         int rw, RowK& r, RowG& rg, unsigned& qclip,
                                         unsigned& lclip)
{
    row_idle<GRAD>(r, rg);
    Chord c = row_chord(g, ev, ev64, iy);
    int lo = c.lo + seg * LMAX;
    int hi = c.lo + c.count - 1;                     // last chord pixel
    if (iy < oy || iy >= oy + rh) {
        lclip += (unsigned)max(c.count, 0);
        return;
    }
    if (lo < oz || hi >= oz + rw) {
        const int lo2 = max(lo, oz), hi2 = min(hi, oz + rw - 1);
        lclip += (unsigned)(max(hi - lo + 1, 0) - max(hi2 - lo2 + 1, 0));
        lo = lo2;
        hi = hi2;
    }
    int len = min(hi - lo + 1, LMAX);
    if (len <= 0) return;
    const float t = ev.z, c2i = ev.w, y = c.y, Dy = c.Dy;
    float u0 = fmaf((float)lo, g.dz, g.z0) - c.zc;
    float y2 = y * y;
    float aCa = 2.0f * g.iz * (g.R * g.R + y2) * c2i * c2i + 4.0f * g.il * y2 * t * t * c2i;
    float two_dlt = 4.0f * g.il * y * fmaf(2.0f * t, t, 1.0f) * Dy * c2i;    // 2 * delta
    float alpha = -2.0f * g.iz * y * c2i;                                     // aCb slope in u
    float beta = 4.0f * g.il * y * t * Dy * c2i;                              // aCb at u = 0
    float gam2 = -4.0f * g.iz * y * t * c2i;                                  // 2 oCb slope in u
    float Qu0 = aCa + two_dlt + gam2 * u0;
    float dQ = gam2 * g.dz;
    // Reading R5: P = 0 where Q <= 0.  Q is linear along the chord, so the
    // pixels with Q > 0 form a sub-range; keep only that.
    float Qlast = fmaf((float)(len - 1), dQ, Qu0);
    if (!(Qu0 > 0.0f && Qlast > 0.0f)) {
        int mlo = 0, mhi = len - 1;
        if (dQ > 0.0f && !(Qu0 > 0.0f))
            mlo = (int)fminf(floorf(-Qu0 / dQ) + 1.0f, (float)len);
        if (dQ < 0.0f && !(Qlast > 0.0f))
            mhi = (int)fmaxf(fminf(ceilf(-Qu0 / dQ) - 1.0f, (float)len), -1.0f);
        if (dQ == 0.0f) mhi = -1;
        mlo = max(mlo, 0);
        mhi = min(mhi, len - 1);
        int keep = max(mhi - mlo + 1, 0);
        qclip += (unsigned)(len - keep);
        if (keep == 0) return;
        lo += mlo;
        len = keep;
        u0 = fmaf((float)mlo, g.dz, u0);
        Qu0 = fmaf((float)mlo, dQ, Qu0);
    }
    r.len = len;
    r.sbase = (iy - oy) * stride + (lo - oz);
    r.Q0 = Qu0;
    r.dQ = dQ;
    r.A0 = g.kA * fmaf(alpha, u0, beta);
    r.dA = g.kA * alpha * g.dz;
    r.su0 = g.ksu * u0;
    r.dsu = g.ksu * g.dz;
    r.C0 = g.log2K - g.half_log2e * c.B0;
    if (GRAD) {
        rg.u0 = u0;
        rg.du = g.dz;
        rg.b0 = fmaf(alpha, u0, beta);
        rg.db = alpha * g.dz;
        // Q = iz Qz + il Ql with Qz = 2 (R^2 + y^2) c2i^2 - 4 y t c2i u and
        // Ql = 4 y^2 t^2 c2i + 4 y (1 + 2 t^2) Dy c2i; aCb = iz Cz + il Cl with
        // Cz = -2 y c2i u, Cl = 4 y t Dy c2i; bCb = iz 2u^2 + il Bl, Bl = 4 Dy^2 c2i.
        float qzc = (g.R * g.R + y2) * c2i * c2i;                     // Qz/2 at u = 0
        float qzs = -2.0f * y * t * c2i;                               // (Qz/2) slope
        rg.qz0 = fmaf(qzs, u0, qzc);
        rg.dqz = qzs * g.dz;
        rg.cz0 = -2.0f * y * c2i * u0;
        rg.dcz = -2.0f * y * c2i * g.dz;
        float Bl = 4.0f * Dy * Dy * c2i;
        rg.kz = 1.0f / g.iz;
        rg.kl = 0.5f / g.il - 0.5f * Bl;
        rg.cl = 4.0f * y * t * Dy * c2i;
        rg.qlh = 2.0f * y2 * t * t * c2i + 2.0f * y * fmaf(2.0f * t, t, 1.0f) * Dy * c2i;
    }
}

// Pass 1 over the lane's chord: P[m] for m < len (values beyond len are
// unspecified), the partial denominator sum P rho', and in GRAD mode the
// partial sums of rho' P dlogP/d(iz) and rho' P dlogP/d(il).  rp points at the
// lane's first pixel (reads up to LMAX-1 floats past the chord end must stay
// inside the buffer; callers pad it).
template <int LMAX, bool GRAD>
__device__ __forceinline__ void pass1(const RowK& r, const RowG& rg, const float* rp, int maxlen,
                                      float (&P)[LMAX], float& Dp, float& Ez, float& El)
{
#pragma unroll
    for (int m = 0; m < LMAX; ++m) {
        if ((m & 3) == 0 && m >= maxlen) break;
        const float fm = (float)m;
        float Q = fmaf(fm, r.dQ, r.Q0);
        float rq = rsqrt_approx(Q);
        float su = fmaf(fm, r.dsu, r.su0);
        float Aw = fmaf(fm, r.dA, r.A0);
        float w = Aw * rq;
        float arg = fmaf(w, w, fmaf(-su, su, r.C0));
        float p = rq * ex2_approx(arg);
        P[m] = p;
        float rhop = rp[m];
        bool on = m < r.len;
        if (on) Dp = fmaf(p, rhop, Dp);
        if (GRAD) {
            // d log P / d iz = 1/iz - u^2 + X Cz - (Qz/2)(1/Q + X^2)
            // d log P / d il = 1/(2 il) - Bl/2 + X Cl - (Ql/2)(1/Q + X^2)
            // with X = aCb / Q.
            float u = fmaf(fm, rg.du, rg.u0);
            float aCb = fmaf(fm, rg.db, rg.b0);
            float iq = rq * rq;
            float X = aCb * iq;
            float S = fmaf(X, X, iq);
            float qzh = fmaf(fm, rg.dqz, rg.qz0);
            float cz = fmaf(fm, rg.dcz, rg.cz0);
            float dz_ = fmaf(-qzh, S, fmaf(X, cz, fmaf(-u, u, rg.kz)));
            float dl_ = fmaf(-rg.qlh, S, fmaf(X, rg.cl, rg.kl));
            if (on) {
                const float wgt = p * rhop;
                Ez = fmaf(wgt, dz_, Ez);
                El = fmaf(wgt, dl_, El);
            }
        }
    }
}

// Pass 2: acc[m] += P[m] * invD for m < len.
template <int LMAX>
__device__ __forceinline__ void pass2(const RowK& r, float* acc, int maxlen, const float (&P)[LMAX],
                                      float invD)
{
#pragma unroll
    for (int m = 0; m < LMAX; ++m) {
        if ((m & 3) == 0 && m >= maxlen) break;
        if (m < r.len) atomicAdd(acc + m, P[m] * invD);
    }
}

struct LeaderSums {
    double logD, giz, gil;
    unsigned long long used;
};

// One event processed by a group of G warps.  Lane-row q = wig*32 + lane
// covers image row rows.x + q / nseg, segment q % nseg.  part: 2*G floats of
// shared scratch for the group's cross-warp reduction (double-buffered by
// parity).  Returns nothing; leader lanes accumulate their sums.
template <int LMAX, int MODE>
__device__ __forceinline__ void process_event(const Geo& g, const EventsView& evs, int e, int G,
                                              int nseg, int wig, int lane, int bar_id,
                                              float* part, int& parity, const float* rp_base,
                                              float* acc_base, int oy, int oz, int stride, int rh,
                                              int rw, LeaderSums& ls, unsigned& qclip,
                                              unsigned& lclip)
{
    constexpr bool GRAD = (MODE == kGrad);
    const float4 ev = evs.geo[e];
    const int2 rws = evs.rows[e];
    const int q = wig * 32 + lane;
    const int rowi = q / nseg;
    const int seg = q - rowi * nseg;
    RowK r;
    RowG rg;
    if (rowi < rws.y)
        make_row<LMAX, GRAD>(g, ev, evs.geo64 + e, rws.x + rowi, seg, oy, oz, stride, rh, rw, r,
                             rg, qclip, lclip);
    else
        row_idle<GRAD>(r, rg);
    const int maxlen = __reduce_max_sync(0xffffffffu, (unsigned)r.len);
    float P[LMAX];
    float Dp = 0.0f, Ez = 0.0f, El = 0.0f;
    pass1<LMAX, GRAD>(r, rg, rp_base + r.sbase, maxlen, P, Dp, Ez, El);
    float D = warp_sum(Dp);
    if (GRAD) {
        Ez = warp_sum(Ez);
        El = warp_sum(El);
    }
    if (G > 1) {
        const int nv = GRAD ? 3 : 1;
        float* slot = part + parity * (3 * G);
        if (lane == 0) {
            slot[wig] = D;
            if (GRAD) {
                slot[G + wig] = Ez;
                slot[2 * G + wig] = El;
            }
        }
        named_barrier(bar_id, G * 32);
        D = 0.0f;
        Ez = 0.0f;
        El = 0.0f;
        for (int w = 0; w < G; ++w) {
            D += slot[w];
            if (nv > 1) {
                Ez += slot[G + w];
                El += slot[2 * G + w];
            }
        }
        parity ^= 1;
    }
    if (D > 0.0f) {
        if (wig == 0 && lane == 0) {
            ls.used += 1;
            if (MODE != kMlem) ls.logD += (double)logf(D);
            if (GRAD) {
                ls.giz += (double)(Ez / D);
                ls.gil += (double)(El / D);
            }
        }
        if (MODE != kLoglik) {
            const float invD = 1.0f / D;
            pass2<LMAX>(r, acc_base + r.sbase, maxlen, P, invD);
        }
    }
}

__device__ __forceinline__ void flush_leader_sums(const LeaderSums& ls, unsigned qclip,
                                                  unsigned lclip, Accum* accum, int mode)
{
    if (ls.used) atomicAdd(&accum->n_used, ls.used);
    if (lclip) atomicAdd(&accum->n_lclip, (unsigned long long)lclip);
    if (mode != kMlem && ls.logD != 0.0) atomicAdd(&accum->sum_logD, ls.logD);
    if (mode == kGrad) {
        if (ls.giz != 0.0) atomicAdd(&accum->g_iz, ls.giz);
        if (ls.gil != 0.0) atomicAdd(&accum->g_il, ls.gil);
    }
    if (qclip) atomicAdd(&accum->n_qclip, (unsigned long long)qclip);
}

// Persistent tile kernel.  Shared memory: rho' region, accumulator region
// (each RH*RS floats), then kPadFloats of slack, then the groups' reduction
// slots (kWarps/G groups x 2 parities x 3G floats).
template <int LMAX, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_tiles(Geo g, Tiling tl, EventsView evs, const int4* __restrict__ items, int n_items,
        const float* __restrict__ rhop, float* __restrict__ A, Accum* accum, int G, int nseg)
{
    extern __shared__ float4 smem_f4[];
    float* s_rp = reinterpret_cast<float*>(smem_f4);
    const int region = tl.RH * tl.RS;
    float* s_acc = s_rp + region;
    float* s_part = s_acc + region + kPadFloats;
    __shared__ int s_item;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ngroups = kWarps / G;
    const int grp = warp / G, wig = warp - grp * G;
    float* part = s_part + grp * (2 * 3 * G);
    int parity = 0;
    LeaderSums ls = {0.0, 0.0, 0.0, 0ull};
    unsigned qclip = 0, lclip = 0;

    // slack after the accumulator: finite values for reads past chord ends
    for (int k = tid; k < kPadFloats; k += kThreads) s_acc[region + k] = 0.0f;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(&accum->queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int4 item = items[it];                // (tile, first event, count, 0)
        const int ty = item.x / tl.tiles_z, tz = item.x - (item.x / tl.tiles_z) * tl.tiles_z;
        const int oy = ty * tl.TY - tl.HY, oz = tz * tl.TZ - tl.HZ;
        for (int rr = warp; rr < tl.RH; rr += kWarps) {
            const int iy = oy + rr;
            const bool row_in = iy >= 0 && iy < g.ny;
            for (int cc = lane; cc < tl.RS; cc += 32) {
                const int iz = oz + cc;
                float v = 0.0f;
                if (row_in && cc < tl.RW && iz >= 0 && iz < g.nz) v = rhop[(size_t)iy * g.nz + iz];
                s_rp[rr * tl.RS + cc] = v;
                if (MODE != kLoglik) s_acc[rr * tl.RS + cc] = 0.0f;
            }
        }
        __syncthreads();
        if (grp < ngroups) {
            for (int e = item.y + grp; e < item.y + item.z; e += ngroups)
                process_event<LMAX, MODE>(g, evs, e, G, nseg, wig, lane, 1 + grp, part, parity,
                                          s_rp, s_acc, oy, oz, tl.RS, tl.RH, tl.RW, ls, qclip,
                                          lclip);
        }
        __syncthreads();
        if (MODE != kLoglik) {
            for (int rr = warp; rr < tl.RH; rr += kWarps) {
                const int iy = oy + rr;
                if (iy < 0 || iy >= g.ny) continue;
                for (int cc = lane; cc < tl.RW; cc += 32) {
                    const int iz = oz + cc;
                    const float v = s_acc[rr * tl.RS + cc];
                    if (iz >= 0 && iz < g.nz && v != 0.0f) atomicAdd(A + (size_t)iy * g.nz + iz, v);
                }
            }
            __syncthreads();
        }
    }
    flush_leader_sums(ls, qclip, lclip, accum, MODE);
}

// Events whose window does not fit their tile's halo: same evaluation, with
// rho' read from global memory and the scatter done by global atomics.
template <int LMAX, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_outliers(Geo g, EventsView evs, int first, int count, const float* __restrict__ rhop,
           float* __restrict__ A, Accum* accum, int G, int nseg)
{
    __shared__ float s_part[kWarps * 2 * 3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ngroups = kWarps / G;
    const int grp = warp / G, wig = warp - grp * G;
    float* part = s_part + grp * (2 * 3 * G);
    int parity = 0;
    LeaderSums ls = {0.0, 0.0, 0.0, 0ull};
    unsigned qclip = 0, lclip = 0;
    if (grp < ngroups) {
        for (int k = blockIdx.x * ngroups + grp; k < count; k += gridDim.x * ngroups)
            process_event<LMAX, MODE>(g, evs, first + k, G, nseg, wig, lane, 1 + grp, part,
                                      parity, rhop, A, 0, 0, g.nz, g.ny, g.nz, ls, qclip, lclip);
    }
    flush_leader_sums(ls, qclip, lclip, accum, MODE);
}

}  // namespace tsp
