// The list-mode MLEM hot path (Eq. iter with Eq. kernel over 3-sigma windows).
//
// One persistent block per SM pulls work items (an angle bin, an image tile of
// that bin's sheared frame, and a run of the events whose window-centre pixel
// lies in the tile) from an atomic queue.  For each item it stages rho' = s*rho
// of the tile's region in shared memory, row by row in the bin's sheared frame
// (so that the chords of all its events are centred on nearly the same stored
// column), and zeroes an accumulator of the same shape.  Warps are grouped (G
// warps per group); a group takes one event at a time and each lane takes one
// image row of the event's window (or one side of it):
//   pass 1: walk the lane's chord of the ellipse outward from its centre,
//           evaluate P (Eq. kernel) in the log2 domain (one rsqrt and one ex2
//           per pixel, two pixels per packed f32x2 instruction), keep P rho'
//           (P in the adjoint pass and in the accumulator-only tiles) in the
//           lane's tensor memory and accumulate
//           D_j = sum P rho' (the denominator of Eq. iter); warp shuffles and a
//           named barrier reduce D_j over the group;
//   pass 2: add the terms P rho' / D_j in [0, 1] into the item's two-word
//           fixed-point accumulator with native integer shared-memory atomics
//           (two groups may touch the same pixel; the layout constants in
//           tsp_device.cuh state the split and its bounds).  The adjoint pass
//           and the accumulator-only tiles add P / D_j as floats.
// A warp's lanes hold 32 distinct rows (paired around the window's middle);
// with the sheared frame and a row stride of 1 mod 32 words their accesses at
// each step fall in distinct banks.
// At the end of the item the accumulator is flushed to the global
// back-projection A with one atomic add per touched pixel (the fixed-point sum
// divided by the pixel's rho'); the finalize kernel then forms rho <- rho * A.
//
// Relative to the paper's GPU design (one warp per event over its bounding
// box, rho read through the texture cache, Sec. 4.2): lanes own chords of the
// ellipse instead of bounding-box pixels (no ellipse-test waste), P is cached
// between the two passes as in the paper but in tensor memory rather than
// registers (so that 1024-thread blocks fit), and the scatter goes to shared
// memory first.
#pragma once

#include <type_traits>

#include "tsp_device.cuh"

namespace tsp {

// Pixel order of a lane's chord, relative to its centre column c:
//   kAlt: 0, +1, -1, +2, -2, ...  (whole chord, one lane per row)
//   kPos: 0, +1, +2, ...          (right half, when a row is split over two lanes)
//   kNeg: -1, -2, ...             (left half)
enum Trav : int { kAlt = 0, kPos = 1, kNeg = 2 };

template <int TRAV>
__host__ __device__ constexpr int trav_delta(int m)
{
    return TRAV == kAlt ? ((m & 1) ? (m + 1) / 2 : -(m / 2)) : (TRAV == kPos ? m : -(m + 1));
}

// Storage frame of a lane's buffer: row iy of the image is stored at
// (iy - oy) * stride; its image column iz at column iz - (zbase + shift(iy)),
// shift(iy) = rint(shear * (iy - Y0)).  Extent rh x rw.
struct Frame {
    int oy, zbase, Y0, stride, rh, rw;
    float shear;
};

// Per-lane row constants, relative to the lane's traversal origin c.  Step m
// (d = trav_delta(m)) is inside the lane's chord iff m < lim_odd (m odd) or
// m < lim_even (m even).  For step m with d = trav_delta(m):
//   u = u0 + d dz,  Q = aCa + 2 oCb = Q0 + d dQ,
//   A = sqrt(log2e/2) aCb = A0 + d dA,  s = sqrt(log2e iz) u = su0 + d dsu,
// and Eq. kernel becomes
//   P = Q^(-1/2) 2^(C0 - s^2 + A^2/Q),  C0 = log2 K - (log2e/2) 4 il Dy^2 c2i,
// K = det^(1/2)(C^-1) / (2 pi^2) (reading R4).  base is the byte address of
// pixel c in the shared window (32-bit) or in the global image.
template <bool SMEM>
struct RowK {
    int lim_odd, lim_even;
    typename std::conditional<SMEM, unsigned, unsigned long long>::type base;
    unsigned long long gbase;   // rho' in global memory (tiles that stage only A)
    float Q0, dQ, A0, dA, su0, dsu, C0;
};

// Per-block counters kept in shared memory (registers are the scarce resource
// of the hot loop): events used, sum of log D, the sigma-gradient sums, and the
// pixels dropped by reading R5 (Q <= 0) or by the region clamp.
struct BlockSums {
    unsigned long long used, qclip, lclip, pad;
    double logD, giz, gil, pad2;
};

// Extra row constants of the sigma-gradient (adjoint) pass:
//   u = u0 + d du, aCb = b0 + d db (unscaled), Qz/2 = qz0 + d dqz,
//   Cz = cz0 + d dcz, and the row constants kz = 1/iz, kl = 1/(2 il) - Bl/2,
//   Cl, Ql/2 (see the derivative formulas in the gradient pass).
struct RowG {
    float u0, du, b0, db, qz0, dqz, cz0, dcz, kz, kl, cl, qlh;
};

// An idle lane: no pixels, and constants that keep its (discarded) pass-1
// arithmetic finite.
template <bool GRAD, bool SMEM>
__device__ __forceinline__ void row_idle(RowK<SMEM>& r, RowG& rg)
{
    r.lim_odd = 0;
    r.lim_even = 0;
    r.base = 0;
    r.Q0 = 1.0f; r.dQ = 0.0f; r.A0 = 0.0f; r.dA = 0.0f; r.su0 = 0.0f; r.dsu = 0.0f;
    r.C0 = -126.0f;
    if (GRAD) {
        rg.u0 = rg.du = rg.b0 = rg.db = rg.qz0 = rg.dqz = rg.cz0 = rg.dcz = 0.0f;
        rg.kz = rg.kl = rg.cl = rg.qlh = 0.0f;
    }
}

// Row constants of lane row iy (valid_row = false for a lane without a row)
// for the traversal TRAV.  All 32 lanes of the warp must call it together: the
// lanes agree on one stored column (the middle of their chord centres) as
// their common traversal origin, so that at every step neighbouring lanes
// (neighbouring rows, row stride = 1 mod 32 words) address distinct banks.  A
// lane whose chord does not contain that column starts at its own centre.
// The event preparation guarantees that every chord lies inside the frame;
// the clamp keeps every access in bounds regardless (clipped pixels are
// counted).
template <int TRAV, int LMAX, bool GRAD, bool SMEM, bool GLD>
__device__ __forceinline__ void make_row(const Geo& g, const EvSig& es, const float4& ev,
                                         const Ev64* ev64, int iy, bool valid_row, int evflags,
                                         const Frame* fp,
                                         const float* base, const float* gimg, RowK<SMEM>& r,
                                         RowG& rg, BlockSums* bs)
{
    row_idle<GRAD, SMEM>(r, rg);
    Chord c;
    c.y = c.Dy = c.B0 = c.zc = 0.0f;
    int lo = 0, hi = -1, z0row = 0;
    const Frame f = *fp;
    float Qc = 0.0f, gam2 = 0.0f;
    if (valid_row) {
        c = row_chord(g, es, ev, ev64, iy, !(evflags & kEvExact));
        lo = c.lo;
        hi = c.lo + c.count - 1;
        if (c.count > 0 && (iy < f.oy || iy >= f.oy + f.rh)) {
            atomicAdd(&bs->lclip, (unsigned long long)c.count);
            hi = lo - 1;
        }
        z0row = f.zbase + (int)rintf(__fmul_rn(f.shear, (float)(iy - f.Y0)));
        if (hi >= lo && (lo < z0row || hi >= z0row + f.rw)) {
            const int lo2 = max(lo, z0row), hi2 = min(hi, z0row + f.rw - 1);
            atomicAdd(&bs->lclip, (unsigned long long)(c.count - max(hi2 - lo2 + 1, 0)));
            lo = lo2;
            hi = hi2;
        }
        if (hi >= lo) {
            row_q(g, es, ev, c, Qc, gam2);
        }
        // Reading R5: P = 0 where Q <= 0.  Q is linear along the chord, so the
        // pixels with Q > 0 form a sub-range; keep only that (unless the event
        // preparation bounded Q > 0 over the whole window).
        if (hi >= lo && !(evflags & kEvQPos)) {
            const float ulo = fmaf((float)lo, g.dz, g.z0) - c.zc;
            const float uhi = fmaf((float)hi, g.dz, g.z0) - c.zc;
            const float Qlo = fmaf(gam2, ulo, Qc), Qhi = fmaf(gam2, uhi, Qc);
            if (!(Qlo > 0.0f && Qhi > 0.0f)) {
                const int n0 = hi - lo + 1;
                const float dQ = gam2 * g.dz;
                int mlo = 0, mhi = n0 - 1;
                if (dQ > 0.0f && !(Qlo > 0.0f))
                    mlo = (int)fminf(floorf(-Qlo / dQ) + 1.0f, (float)n0);
                if (dQ < 0.0f && !(Qhi > 0.0f))
                    mhi = (int)fmaxf(fminf(ceilf(-Qlo / dQ) - 1.0f, (float)n0), -1.0f);
                if (dQ == 0.0f) mhi = -1;
                mlo = max(mlo, 0);
                mhi = min(mhi, n0 - 1);
                const int keep = max(mhi - mlo + 1, 0);
                atomicAdd(&bs->qclip, (unsigned long long)(n0 - keep));
                hi = lo + mhi;
                lo = lo + mlo;
            }
        }
    }
    const bool has = hi >= lo;
    const int sc = ((lo + hi) >> 1) - z0row;               // stored column of the centre
    const int smin = __reduce_min_sync(0xffffffffu, has ? sc : 0x7fffffff);
    const int smax = __reduce_max_sync(0xffffffffu, has ? sc : (int)0x80000000);
    if (!has) {
        // A lane without pixels still gets an in-bounds address, in its own
        // (virtual) row at the warp's common column: the packed passes run it
        // through their unpredicated pairs with P = 0, and its own row keeps
        // its accesses in a bank of their own (one dummy address shared by the
        // idle lanes would make the warp's atomics collide).  Rows and columns
        // are clamped to the frame; on a whole-image frame the flat index is
        // clamped into the padded image, as is the global rho' address.
        const int vr = min(max(iy - f.oy, 0), f.rh - 1);
        const int col = min(max(smin <= smax ? (smin + (smax - smin) / 2) : (f.rw >> 1), 0),
                            f.rw - 1);
        const long long lo_i = LMAX / 2;
        const long long hi_i = (long long)g.ny * g.nz + kPadFloats - LMAX / 2 - 1;
        long long sidx = (long long)vr * f.stride + col;
        if constexpr (SMEM) {
            r.base = (unsigned)__cvta_generic_to_shared(base) + 4u * (unsigned)sidx;
        } else {
            sidx = min(max(sidx, lo_i), hi_i);
            r.base = (unsigned long long)(base + sidx);
        }
        if constexpr (GLD) {
            const int iyv = min(max(f.oy + vr, 0), g.ny - 1);
            const int zv = f.zbase + (int)rintf(__fmul_rn(f.shear, (float)(f.oy + vr - f.Y0)));
            const long long gi = min(max((long long)iyv * g.nz + min(max(zv + col, 0), g.nz - 1),
                                         lo_i), hi_i);
            r.gbase = (unsigned long long)(gimg + gi);
        }
        return;
    }
    // The common origin is used only when it lies within 2 columns of the
    // lane's own chord centre cc and keeps the lane's walk within LMAX steps;
    // otherwise the lane starts at cc (then kAlt needs exactly hi - lo + 1 <=
    // LMAX steps and each half of kPos / kNeg at most LMAX).
    const int k0 = (int)(((long long)smin + (long long)smax) >> 1);
    const int cc = (lo + hi) >> 1;
    int o = k0 + z0row;
    if (o < cc - 2 || o > cc + 2 || o < lo || o > hi) o = cc;
    if (TRAV == kAlt && max(2 * (hi - o), 2 * (o - lo) + 1) > LMAX) o = cc;
    if (TRAV == kPos && hi - o + 1 > LMAX) o = cc;
    if (TRAV == kNeg && o - lo > LMAX) o = cc;
    const int L = o - lo, R = hi - o;
    if (TRAV == kAlt) {
        r.lim_odd = 2 * R;          // odd m reach d = (m+1)/2 <= R
        r.lim_even = 2 * L + 1;     // even m reach d = -m/2 >= -L
    } else if (TRAV == kPos) {
        r.lim_odd = r.lim_even = R + 1;
    } else {
        r.lim_odd = r.lim_even = L;
    }
    const float t = ev.z, c2i = ev.w, y = c.y, Dy = c.Dy;
    float alpha, beta;
    row_acb(g, es, ev, c, alpha, beta);
    const float u0 = fmaf((float)o, g.dz, g.z0) - c.zc;
    const int sidx = (iy - f.oy) * f.stride + (o - z0row);
    if constexpr (SMEM)
        r.base = (unsigned)__cvta_generic_to_shared(base) + 4u * (unsigned)sidx;
    else
        r.base = (unsigned long long)(base + sidx);
    if constexpr (GLD) r.gbase = (unsigned long long)(gimg + (size_t)iy * g.nz + o);
    r.Q0 = fmaf(gam2, u0, Qc);
    r.dQ = gam2 * g.dz;
    r.A0 = g.kA * fmaf(alpha, u0, beta);
    r.dA = g.kA * alpha * g.dz;
    r.su0 = es.ksu * u0;
    r.dsu = es.ksu * g.dz;
    r.C0 = es.log2K - g.half_log2e * c.B0;
    if (GRAD) {
        const float y2 = y * y;
        rg.u0 = u0;
        rg.du = g.dz;
        rg.b0 = fmaf(alpha, u0, beta);
        rg.db = alpha * g.dz;
        // Q = iz Qz + il Ql with Qz = 2 (R^2 + y^2) c2i^2 - 4 y t c2i u and
        // Ql = 4 y^2 t^2 c2i + 4 y (1 + 2 t^2) Dy c2i; aCb = iz Cz + il Cl with
        // Cz = -2 y c2i u, Cl = 4 y t Dy c2i; bCb = iz 2u^2 + il Bl, Bl = 4 Dy^2 c2i.
        const float qzc = (g.R * g.R + y2) * c2i * c2i;                 // Qz/2 at u = 0
        const float qzs = -2.0f * y * t * c2i;                           // (Qz/2) slope
        rg.qz0 = fmaf(qzs, u0, qzc);
        rg.dqz = qzs * g.dz;
        rg.cz0 = -2.0f * y * c2i * u0;
        rg.dcz = -2.0f * y * c2i * g.dz;
        const float Bl = 4.0f * Dy * Dy * c2i;
        rg.kz = es.ldz;
        rg.kl = es.ldl - 0.5f * Bl;
        rg.cl = 4.0f * y * t * Dy * c2i;
        rg.qlh = 2.0f * y2 * t * t * c2i + 2.0f * y * fmaf(2.0f * t, t, 1.0f) * Dy * c2i;
        // the sum Ez is wanted with respect to the base iz: d/d iz = (1/f^2) d/d iz_event,
        // so every term of the z derivative carries 1/f^2 (u through 1/f, as it
        // enters squared); with a constant sigma_z these factors are 1
        rg.u0 *= es.inv_f;
        rg.du *= es.inv_f;
        rg.qz0 *= es.inv_f2;
        rg.dqz *= es.inv_f2;
        rg.cz0 *= es.inv_f2;
        rg.dcz *= es.inv_f2;
        rg.kz *= es.inv_f2;
    }
}

// Predicated load of rho' and accumulation of the denominator: if (m < len)
// { v = mem[base + OFF]; D += p * v; } else v = 0.  Inactive lanes touch no
// memory.
template <bool SMEM, int OFF>
__device__ __forceinline__ float load_acc(const RowK<SMEM>& r, int lim, int m, float p, float& D)
{
    float v;
    if constexpr (SMEM) {
#ifdef TSP_DEBUG_CHECKS
        if (m < lim && !tsp_sh_ok(r.base + OFF, 4, 4)) return 0.0f;
#endif
        asm(
            "{\n\t.reg .pred q;\n\t"
            "setp.lt.s32 q, %2, %3;\n\t"
            "mov.b32 %0, 0;\n\t"
            "@q ld.shared.f32 %0, [%4+%5];\n\t"
            "@q fma.rn.f32 %1, %6, %0, %1;\n\t}"
            : "=&f"(v), "+f"(D)
            : "r"(m), "r"(lim), "r"(r.base), "n"(OFF), "f"(p));
    } else {
        asm(
            "{\n\t.reg .pred q;\n\t"
            "setp.lt.s32 q, %2, %3;\n\t"
            "mov.b32 %0, 0;\n\t"
            "@q ld.global.f32 %0, [%4+%5];\n\t"
            "@q fma.rn.f32 %1, %6, %0, %1;\n\t}"
            : "=&f"(v), "+f"(D)
            : "r"(m), "r"(lim), "l"(r.base), "n"(OFF), "f"(p));
    }
    return v;
}

// As load_acc, from global memory through the read-only path.
template <int OFF>
__device__ __forceinline__ float load_acc_g(unsigned long long base, int lim, int m, float p,
                                            float& D)
{
    float v;
    asm(
        "{\n\t.reg .pred q;\n\t"
        "setp.lt.s32 q, %2, %3;\n\t"
        "mov.b32 %0, 0;\n\t"
        "@q ld.global.nc.f32 %0, [%4+%5];\n\t"
        "@q fma.rn.f32 %1, %6, %0, %1;\n\t}"
        : "=&f"(v), "+f"(D)
        : "r"(m), "r"(lim), "l"(base), "n"(OFF), "f"(p));
    return v;
}

// Predicated reduction: if (m < len) mem[base + OFF] += v.
template <bool SMEM, int OFF>
__device__ __forceinline__ void red_add(const RowK<SMEM>& r, int lim, int m, float v)
{
    if constexpr (SMEM) {
#ifdef TSP_DEBUG_CHECKS
        if (m < lim && !tsp_sh_ok(r.base + OFF, 4, 5)) return;
#endif
        asm volatile(
            "{\n\t.reg .pred q;\n\t"
            "setp.lt.s32 q, %0, %1;\n\t"
            "@q red.shared.add.f32 [%2+%3], %4;\n\t}" ::"r"(m),
            "r"(lim), "r"(r.base), "n"(OFF), "f"(v)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred q;\n\t"
            "setp.lt.s32 q, %0, %1;\n\t"
            "@q red.global.add.f32 [%2+%3], %4;\n\t}" ::"r"(m),
            "r"(lim), "l"(r.base), "n"(OFF), "f"(v)
            : "memory");
    }
}

// P cache in tensor memory.  Each thread keeps the kernel values of its row
// segment (P rho' in the fixed-point MLEM pass) in its own TMEM lane instead of
// registers: warp w uses lanes 32 (w mod 4) .. +31 (the lane quarter a warp may
// access) and a slice of tm_slice(LMAX) columns starting at column
// tm_slice(LMAX) * (w / 4).  Pass 1 stores 16, 8 or 4 values at a time (4 in
// the scalar pass), pass 2 loads them back; the registers this frees go to
// more resident warps.  (The paper's kernel keeps P in registers or
// recomputes it.)
__host__ __device__ constexpr int pow2_at_least(int x, int p = 1)
{
    return p >= x ? p : pow2_at_least(x, 2 * p);
}
__host__ __device__ constexpr int tm_slice(int lmax) { return pow2_at_least(lmax); }
// Columns a block of `warps` warps allocates (a power of two, 32 .. 512).
__host__ __device__ constexpr int tm_block_cols(int lmax, int warps)
{
    return pow2_at_least(tm_slice(lmax) * ((warps + 3) / 4) < 32 ? 32
                                                                 : tm_slice(lmax) * ((warps + 3) / 4));
}

// Executed by one whole warp; the base address goes to *s_addr.
template <int NCOLS>
__device__ __forceinline__ void tm_alloc(unsigned* s_addr)
{
    static_assert(NCOLS >= 32 && NCOLS <= 512 && (NCOLS & (NCOLS - 1)) == 0, "TMEM columns");
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(s_addr)),
                 "n"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Executed by the warp that allocated.
template <int NCOLS>
__device__ __forceinline__ void tm_dealloc(unsigned base)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "n"(NCOLS)
                 : "memory");
}

// Block-wide ordering of tensor-memory operations around a barrier.
__device__ __forceinline__ void tm_sync_threads()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// TMEM address of this warp's first P column (lane field: its lane quarter).
template <int LMAX>
__device__ __forceinline__ unsigned tm_thread_addr(unsigned base, int warp)
{
    return base + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(tm_slice(LMAX) * (warp >> 2));
}

__device__ __forceinline__ void tm_st4(unsigned a, float x0, float x1, float x2, float x3)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a),
                 "f"(x0), "f"(x1), "f"(x2), "f"(x3)
                 : "memory");
}

__device__ __forceinline__ void tm_ld4(unsigned a, float& x0, float& x1, float& x2, float& x3)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(x0), "=f"(x1), "=f"(x2), "=f"(x3)
                 : "r"(a)
                 : "memory");
}

__device__ __forceinline__ void tm_st8(unsigned a, float x0, float x1, float x2, float x3, float x4,
                                       float x5, float x6, float x7)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(a),
                 "f"(x0), "f"(x1), "f"(x2), "f"(x3), "f"(x4), "f"(x5), "f"(x6), "f"(x7)
                 : "memory");
}

__device__ __forceinline__ void tm_ld8(unsigned a, float (&x)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]), "=f"(x[4]), "=f"(x[5]),
                   "=f"(x[6]), "=f"(x[7])
                 : "r"(a)
                 : "memory");
}

__device__ __forceinline__ void tm_st16(unsigned a, const float (&x)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, "
                 "%9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(a),
                 "f"(x[0]), "f"(x[1]), "f"(x[2]), "f"(x[3]), "f"(x[4]), "f"(x[5]), "f"(x[6]),
                 "f"(x[7]), "f"(x[8]), "f"(x[9]), "f"(x[10]), "f"(x[11]), "f"(x[12]), "f"(x[13]),
                 "f"(x[14]), "f"(x[15])
                 : "memory");
}

__device__ __forceinline__ void tm_ld16(unsigned a, float (&x)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
                 "%10, %11, %12, %13, %14, %15}, [%16];"
                 : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3]), "=f"(x[4]), "=f"(x[5]),
                   "=f"(x[6]), "=f"(x[7]), "=f"(x[8]), "=f"(x[9]), "=f"(x[10]), "=f"(x[11]),
                   "=f"(x[12]), "=f"(x[13]), "=f"(x[14]), "=f"(x[15])
                 : "r"(a)
                 : "memory");
}

__device__ __forceinline__ void tm_wait_st()
{
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tm_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Pass 1, step M (template recursion so that each step's address offset is a
// compile-time immediate).  The kernel value of step M goes to TMEM column
// tma + M (values beyond the lane's length are unspecified), four steps at a
// time through P (ST: pass 2 follows); Dp the partial denominator; in GRAD mode Ez, El the partial
// sums of rho' P dlogP/d(iz) and rho' P dlogP/d(il).
template <int TRAV, int LMAX, bool GRAD, bool SMEM, bool GLD, bool ST, int M>
__device__ __forceinline__ void pass1_step(const RowK<SMEM>& r, const RowG& rg, int maxlen,
                                           unsigned tma, float (&P)[4], float& Dp, float& Ez,
                                           float& El)
{
    if constexpr (M < LMAX) {
        if constexpr ((M & 3) == 0) {
            if (M >= maxlen) return;
        }
        constexpr int d = trav_delta<TRAV>(M);
        const float fd = (float)d;
        const float Q = fmaf(fd, r.dQ, r.Q0);
        const float rq = rsqrt_approx(Q);
        const float su = fmaf(fd, r.dsu, r.su0);
        const float Aw = fmaf(fd, r.dA, r.A0);
        const float w = Aw * rq;
        const float arg = fmaf(w, w, fmaf(-su, su, r.C0));
        const float p = rq * ex2_approx(arg);
        P[M & 3] = p;
        if constexpr (ST && (M & 3) == 3) tm_st4(tma + (M - 3), P[0], P[1], P[2], P[3]);
        const int lim = (M & 1) ? r.lim_odd : r.lim_even;
        float rhop;
        if constexpr (GLD)
            rhop = load_acc_g<4 * d>(r.gbase, lim, M, p, Dp);
        else
            rhop = load_acc<SMEM, 4 * d>(r, lim, M, p, Dp);
        if constexpr (GRAD) {
            // d log P / d iz = 1/iz - u^2 + X Cz - (Qz/2)(1/Q + X^2)
            // d log P / d il = 1/(2 il) - Bl/2 + X Cl - (Ql/2)(1/Q + X^2)
            // with X = aCb / Q.
            const float u = fmaf(fd, rg.du, rg.u0);
            const float aCb = fmaf(fd, rg.db, rg.b0);
            const float iq = rq * rq;
            const float X = aCb * iq;
            const float S = fmaf(X, X, iq);
            const float qzh = fmaf(fd, rg.dqz, rg.qz0);
            const float cz = fmaf(fd, rg.dcz, rg.cz0);
            const float dz_ = fmaf(-qzh, S, fmaf(X, cz, fmaf(-u, u, rg.kz)));
            const float dl_ = fmaf(-rg.qlh, S, fmaf(X, rg.cl, rg.kl));
            if (M < lim) {
                const float wgt = p * rhop;
                Ez = fmaf(wgt, dz_, Ez);
                El = fmaf(wgt, dl_, El);
            }
        }
        pass1_step<TRAV, LMAX, GRAD, SMEM, GLD, ST, M + 1>(r, rg, maxlen, tma, P, Dp, Ez, El);
    }
}

// Pass 2, step M: acc[d(M)] += P(M) * invD for M < len, P(M) loaded back from
// TMEM four steps at a time.
template <int TRAV, int LMAX, bool SMEM, int M>
__device__ __forceinline__ void pass2_step(const RowK<SMEM>& r, int maxlen, unsigned tma,
                                           float (&P)[4], float invD)
{
    if constexpr (M < LMAX) {
        if constexpr ((M & 3) == 0) {
            if (M >= maxlen) return;
            tm_ld4(tma + M, P[0], P[1], P[2], P[3]);
            tm_wait_ld();
        }
        red_add<SMEM, 4 * trav_delta<TRAV>(M)>(r, (M & 1) ? r.lim_odd : r.lim_even, M,
                                               P[M & 3] * invD);
        pass2_step<TRAV, LMAX, SMEM, M + 1>(r, maxlen, tma, P, invD);
    }
}

// ---------------------------------------------------------------------------
// Pair-packed MLEM and log-likelihood passes.
//
// A lane walks its chord two pixels at a time.  The arithmetic of the two
// pixels of a pair is done by packed f32x2 instructions (one issue for both);
// the SFU operations and the memory accesses stay per pixel.  Pair k (1-based)
// holds the pixels at column offsets d0(k), d1(k) from the lane's origin:
//   kAlt: (+k, -(k-1));  kPos: (2k-2, 2k-1);  kNeg: (-(2k-1), -2k)
// so every traversal covers its pixels in LMAX/2 pairs.  The first pixel of
// pair k lies on the lane's chord iff k <= la, the second iff k <= lb.  The
// pairs up to the smallest limit of the warp's active lanes (kfast) run
// without any test; the others, up to the largest limit (kmax), test each
// pixel.  A lane without pixels evaluates P = 0 exactly (its exponent is
// -1000, which ex2.approx.ftz flushes to zero) at an in-bounds address of its
// own row (make_row), and constrains neither kfast nor kmax.  Along a row, with d the column offset:
//   Q = Q0 + d dQ,  A = A0 + d dA,  E = C0 - s^2 = e0 + d (e1 + d e2),
//   P = Q^(-1/2) 2^(E + A^2/Q)       (Eq. kernel in the log2 domain).
template <int TRAV>
__host__ __device__ constexpr int pair_d0(int k)
{
    return TRAV == kAlt ? k : (TRAV == kPos ? 2 * k - 2 : -(2 * k - 1));
}
template <int TRAV>
__host__ __device__ constexpr int pair_d1(int k)
{
    return TRAV == kAlt ? -(k - 1) : (TRAV == kPos ? 2 * k - 1 : -2 * k);
}

template <bool SMEM>
struct RowP {
    typename std::conditional<SMEM, unsigned, unsigned long long>::type base;
    unsigned long long gbase;   // rho' in global memory (tiles that stage only A)
    int la, lb;
};

// The row constants as pairs (the same value twice) for the packed operations,
// and the step of the pair offsets.
struct PairC {
    float2 Q0, dQ, A0, dA, e0, e1, e2, inc;
};

// Packed row of a lane from its scalar row constants.  active: the lane has
// pixels.
template <int TRAV, int LMAX, bool SMEM, bool GLD>
__device__ __forceinline__ void pair_row(const RowK<SMEM>& r, bool active, RowP<SMEM>& q, PairC& c)
{
    float Q0 = r.Q0, dQ = r.dQ, A0 = r.A0, dA = r.dA;
    float e0 = fmaf(-r.su0, r.su0, r.C0), e1 = -2.0f * r.su0 * r.dsu, e2 = -(r.dsu * r.dsu);
    if (active) {
        q.base = r.base;
        q.gbase = r.gbase;
        if (TRAV == kAlt) {
            q.la = r.lim_odd >> 1;
            q.lb = (r.lim_even + 1) >> 1;
        } else {
            q.la = (r.lim_odd + 1) >> 1;
            q.lb = r.lim_odd >> 1;
        }
    } else {
        // no pixels: P = 0 at the lane's in-bounds idle address (make_row); no
        // pixel is inside, so the predicated pairs skip the lane
        q.base = r.base;
        q.gbase = r.gbase;
        q.la = q.lb = 0;
        Q0 = 1.0f;
        dQ = A0 = dA = e1 = e2 = 0.0f;
        e0 = -1000.0f;
    }
    c.Q0 = make_float2(Q0, Q0);
    c.dQ = make_float2(dQ, dQ);
    c.A0 = make_float2(A0, A0);
    c.dA = make_float2(dA, dA);
    c.e0 = make_float2(e0, e0);
    c.e1 = make_float2(e1, e1);
    c.e2 = make_float2(e2, e2);
    c.inc = make_float2((float)(pair_d0<TRAV>(2) - pair_d0<TRAV>(1)),
                        (float)(pair_d1<TRAV>(2) - pair_d1<TRAV>(1)));
}

// Running addresses of a lane's two pixel streams: the first pixels of the
// pairs (byte address a0 of pair k) and the second ones (a1); a pair step moves
// them by the traversal's pixel step times 4 bytes.  The chunk loops below
// advance them two pairs at a time, so every access uses a register address
// plus a small immediate and the loops need no unrolled copies per chunk.
template <int TRAV>
__host__ __device__ constexpr int pair_step0() { return pair_d0<TRAV>(2) - pair_d0<TRAV>(1); }
template <int TRAV>
__host__ __device__ constexpr int pair_step1() { return pair_d1<TRAV>(2) - pair_d1<TRAV>(1); }

// rho' at address A + OFF: unpredicated, or (PRED) only when k <= lim, else 0.
template <bool SMEM, bool GLD, bool PRED, int OFF>
__device__ __forceinline__ float ld_rhop(typename std::conditional<SMEM && !GLD, unsigned,
                                                                   unsigned long long>::type a,
                                         int k, int lim)
{
    float v;
    if constexpr (GLD) {
        if constexpr (PRED)
            asm("{\n\t.reg .pred q;\n\tsetp.le.s32 q, %1, %2;\n\tmov.b32 %0, 0;\n\t"
                "@q ld.global.nc.f32 %0, [%3+%4];\n\t}"
                : "=&f"(v) : "r"(k), "r"(lim), "l"(a), "n"(OFF));
        else
            asm("ld.global.nc.f32 %0, [%1+%2];" : "=f"(v) : "l"(a), "n"(OFF));
    } else if constexpr (SMEM) {
#ifdef TSP_DEBUG_CHECKS
        if ((!PRED || k <= lim) && !tsp_sh_ok(a + (unsigned)OFF, 4, 1)) return 0.0f;
#endif
        if constexpr (PRED)
            asm volatile("{\n\t.reg .pred q;\n\tsetp.le.s32 q, %1, %2;\n\tmov.b32 %0, 0;\n\t"
                         "@q ld.shared.f32 %0, [%3+%4];\n\t}"
                         : "=&f"(v) : "r"(k), "r"(lim), "r"(a), "n"(OFF) : "memory");
        else
            asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF) : "memory");
    } else {
        if constexpr (PRED)
            asm volatile("{\n\t.reg .pred q;\n\tsetp.le.s32 q, %1, %2;\n\tmov.b32 %0, 0;\n\t"
                         "@q ld.global.f32 %0, [%3+%4];\n\t}"
                         : "=&f"(v) : "r"(k), "r"(lim), "l"(a), "n"(OFF) : "memory");
        else
            asm volatile("ld.global.f32 %0, [%1+%2];" : "=f"(v) : "l"(a), "n"(OFF) : "memory");
    }
    return v;
}

// Pass 1 for one pair: kernel values of its two pixels, or (PV) their
// products P rho' (returned), the denominator partial sums D2 += P rho'; kk
// holds the pair's offsets and is advanced.  a0 / a1: addresses of the pair's
// two pixels (plus OFF0 / OFF1).
template <bool SMEM, bool GLD, bool PRED, bool PV, int OFF0, int OFF1, class Addr>
__device__ __forceinline__ float2 p1_pair(Addr a0, Addr a1, int k, int la, int lb, const PairC& c,
                                          float2& kk, float2& D2)
{
    const float2 q = __ffma2_rn(kk, c.dQ, c.Q0);
    float2 rq;
    rq.x = rsqrt_approx(q.x);
    rq.y = rsqrt_approx(q.y);
    const float2 a = __ffma2_rn(kk, c.dA, c.A0);
    const float2 e = __ffma2_rn(kk, __ffma2_rn(kk, c.e2, c.e1), c.e0);
    const float2 w = __fmul2_rn(a, rq);
    const float2 g = __ffma2_rn(w, w, e);
    float2 x;
    x.x = ex2_approx(g.x);
    x.y = ex2_approx(g.y);
    float2 p = __fmul2_rn(rq, x);
    if constexpr (PRED) {
        // beyond the lane's chord P is 0 exactly: the denominator ignores the
        // pixel and pass 2 may add the (zero) value without a predicate
        p.x = k <= la ? p.x : 0.0f;
        p.y = k <= lb ? p.y : 0.0f;
    }
    // A staged region has slack around it, so its loads need no predicate
    // (the values of pixels outside the chord meet P = 0); loads from a global
    // image keep theirs, as the chord's offsets may run past the image's start.
    constexpr bool kLdPred = PRED && !(SMEM && !GLD);
    float2 v;
    v.x = ld_rhop<SMEM, GLD, kLdPred, OFF0>(a0, k, la);
    v.y = ld_rhop<SMEM, GLD, kLdPred, OFF1>(a1, k, lb);
    kk = __fadd2_rn(kk, c.inc);
    if constexpr (PV) {
        const float2 pv = __fmul2_rn(p, v);
        D2 = __fadd2_rn(D2, pv);
        return pv;
    } else {
        D2 = __ffma2_rn(p, v, D2);
        return p;
    }
}

// Pass 1 over pairs 1 .. kmax, eight, four or two pairs (one tensor-memory
// store when ST) per loop step: unpredicated while the pairs are <= kfast, then
// two at a time predicated.
// Returns with D2 the two partial denominators; PV stores P rho' instead of P.
template <int TRAV, int LMAX, bool SMEM, bool GLD, bool ST, bool PV>
__device__ __forceinline__ void pass1_pairs(const RowP<SMEM>& r, const PairC& c, int kfast,
                                            int kmax, float2& D2, unsigned tma)
{
    using Addr = typename std::conditional<SMEM && !GLD, unsigned, unsigned long long>::type;
    constexpr int s0 = 4 * pair_step0<TRAV>(), s1 = 4 * pair_step1<TRAV>();
    Addr a0, a1;
    if constexpr (GLD) {
        a0 = (Addr)(r.gbase + (unsigned long long)(4ll * pair_d0<TRAV>(1)));
        a1 = (Addr)(r.gbase + (unsigned long long)(4ll * pair_d1<TRAV>(1)));
    } else {
        a0 = (Addr)(r.base + (Addr)(4ll * pair_d0<TRAV>(1)));
        a1 = (Addr)(r.base + (Addr)(4ll * pair_d1<TRAV>(1)));
    }
    float2 kk = make_float2((float)pair_d0<TRAV>(1), (float)pair_d1<TRAV>(1));
    unsigned col = tma;
    int k = 1;
    // eight pairs per step (one 16-column store: fewer tensor-memory
    // operations, each of which the warp must reach together), then four, then
    // two; the eight-pair steps only over a staged rho' region (with rho' from
    // global memory they held more loads in flight than the registers allow)
    for (; (SMEM && !GLD) && k + 7 <= kfast; k += 8) {
        float x[16];
        float2 t;
        t = p1_pair<SMEM, GLD, false, PV, 0, 0>(a0, a1, k, r.la, r.lb, c, kk, D2);
        x[0] = t.x, x[1] = t.y;
        t = p1_pair<SMEM, GLD, false, PV, s0, s1>(a0, a1, k, r.la, r.lb, c, kk, D2);
        x[2] = t.x, x[3] = t.y;
        t = p1_pair<SMEM, GLD, false, PV, 2 * s0, 2 * s1>(a0, a1, k, r.la, r.lb, c, kk, D2);
        x[4] = t.x, x[5] = t.y;
        t = p1_pair<SMEM, GLD, false, PV, 3 * s0, 3 * s1>(a0, a1, k, r.la, r.lb, c, kk, D2);
        x[6] = t.x, x[7] = t.y;
        t = p1_pair<SMEM, GLD, false, PV, 4 * s0, 4 * s1>(a0, a1, k, r.la, r.lb, c, kk, D2);
        x[8] = t.x, x[9] = t.y;
        t = p1_pair<SMEM, GLD, false, PV, 5 * s0, 5 * s1>(a0, a1, k, r.la, r.lb, c, kk, D2);
        x[10] = t.x, x[11] = t.y;
        t = p1_pair<SMEM, GLD, false, PV, 6 * s0, 6 * s1>(a0, a1, k, r.la, r.lb, c, kk, D2);
        x[12] = t.x, x[13] = t.y;
        t = p1_pair<SMEM, GLD, false, PV, 7 * s0, 7 * s1>(a0, a1, k, r.la, r.lb, c, kk, D2);
        x[14] = t.x, x[15] = t.y;
        if constexpr (ST) tm_st16(col, x);
        a0 += (Addr)(8 * s0);
        a1 += (Addr)(8 * s1);
        col += 16;
    }
    for (; k + 3 <= kfast; k += 4) {
        const float2 pa = p1_pair<SMEM, GLD, false, PV, 0, 0>(a0, a1, k, r.la, r.lb, c, kk, D2);
        const float2 pb = p1_pair<SMEM, GLD, false, PV, s0, s1>(a0, a1, k + 1, r.la, r.lb, c, kk,
                                                                D2);
        const float2 pc = p1_pair<SMEM, GLD, false, PV, 2 * s0, 2 * s1>(a0, a1, k + 2, r.la, r.lb,
                                                                        c, kk, D2);
        const float2 pd = p1_pair<SMEM, GLD, false, PV, 3 * s0, 3 * s1>(a0, a1, k + 3, r.la, r.lb,
                                                                        c, kk, D2);
        if constexpr (ST) tm_st8(col, pa.x, pa.y, pb.x, pb.y, pc.x, pc.y, pd.x, pd.y);
        a0 += (Addr)(4 * s0);
        a1 += (Addr)(4 * s1);
        col += 8;
    }
    for (; k + 1 <= kfast; k += 2) {
        const float2 pa = p1_pair<SMEM, GLD, false, PV, 0, 0>(a0, a1, k, r.la, r.lb, c, kk, D2);
        const float2 pb = p1_pair<SMEM, GLD, false, PV, s0, s1>(a0, a1, k + 1, r.la, r.lb, c, kk,
                                                                D2);
        if constexpr (ST) tm_st4(col, pa.x, pa.y, pb.x, pb.y);
        a0 += (Addr)(2 * s0);
        a1 += (Addr)(2 * s1);
        col += 4;
    }
    for (; k <= kmax; k += 2) {
        const float2 pa = p1_pair<SMEM, GLD, true, PV, 0, 0>(a0, a1, k, r.la, r.lb, c, kk, D2);
        const float2 pb = p1_pair<SMEM, GLD, true, PV, s0, s1>(a0, a1, k + 1, r.la, r.lb, c, kk,
                                                               D2);
        if constexpr (ST) tm_st4(col, pa.x, pa.y, pb.x, pb.y);
        a0 += (Addr)(2 * s0);
        a1 += (Addr)(2 * s1);
        col += 4;
    }
    (void)LMAX;
}

// acc += v at the four pixels of pairs k, k + 1 (addresses a0, a0 + S0 for the
// first pixels, a1, a1 + S1 for the second ones), in one asm block.  In shared
// memory unconditionally: outside a lane's chord its values are 0 (pass 1
// zeroes P there) and its addresses stay inside the region's slack, and a lane
// without pixels adds zeros in its own row; predicated atomics would cost a
// branch and a reconvergence barrier each.  In global memory (the whole-image
// frame, where the offsets may run past the image's start) with predicates:
// PRED, each pixel only when its pair lies inside (k <= la, k <= lb,
// k + 1 <= la, k + 1 <= lb); else every pixel of a lane with pixels (act).
template <bool SMEM, bool PRED, int S0, int S1, class Addr>
__device__ __forceinline__ void red4(Addr a0, Addr a1, int k, int la, int lb, int act, float a,
                                     float b, float c, float d)
{
    if constexpr (SMEM) {
        (void)k, (void)la, (void)lb, (void)act;
#ifdef TSP_DEBUG_CHECKS
        if (!(tsp_sh_ok(a0, 4, 3) && tsp_sh_ok(a1, 4, 3) && tsp_sh_ok(a0 + (unsigned)S0, 4, 3) &&
              tsp_sh_ok(a1 + (unsigned)S1, 4, 3)))
            return;
#endif
        asm volatile(
            "red.shared.add.f32 [%0], %4;\n\tred.shared.add.f32 [%1], %5;\n\t"
            "red.shared.add.f32 [%0+%2], %6;\n\tred.shared.add.f32 [%1+%3], %7;"
            ::"r"(a0), "r"(a1), "n"(S0), "n"(S1), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
    } else {
        if constexpr (PRED)
            asm volatile(
                "{\n\t.reg .pred p0, p1, p2, p3;\n\t.reg .s32 k1;\n\tadd.s32 k1, %0, 1;\n\t"
                "setp.le.s32 p0, %0, %1;\n\tsetp.le.s32 p1, %0, %2;\n\t"
                "setp.le.s32 p2, k1, %1;\n\tsetp.le.s32 p3, k1, %2;\n\t"
                "@p0 red.global.add.f32 [%3], %7;\n\t@p1 red.global.add.f32 [%4], %8;\n\t"
                "@p2 red.global.add.f32 [%3+%5], %9;\n\t@p3 red.global.add.f32 [%4+%6], %10;\n\t}"
                ::"r"(k), "r"(la), "r"(lb), "l"(a0), "l"(a1), "n"(S0), "n"(S1), "f"(a), "f"(b),
                "f"(c), "f"(d) : "memory");
        else
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.s32 p, %0, 0;\n\t"
                "@p red.global.add.f32 [%1], %5;\n\t@p red.global.add.f32 [%2], %6;\n\t"
                "@p red.global.add.f32 [%1+%3], %7;\n\t@p red.global.add.f32 [%2+%4], %8;\n\t}"
                ::"r"(act), "l"(a0), "l"(a1), "n"(S0), "n"(S1), "f"(a), "f"(b), "f"(c), "f"(d)
                : "memory");
    }
}

// Pass 2 over pairs 1 .. kmax: acc += P / D, P loaded back from tensor memory
// eight or four values at a time (P is 0 outside each lane's chord); the
// shared-memory forms add every pixel, the global ones only the chord's.
// r.base addresses the accumulator.
template <int TRAV, bool SMEM>
__device__ __forceinline__ void pass2_pairs(const RowP<SMEM>& r, int act, int kfast, int kmax,
                                            unsigned tma, float2 invD)
{
    using Addr = typename std::conditional<SMEM, unsigned, unsigned long long>::type;
    constexpr int s0 = 4 * pair_step0<TRAV>(), s1 = 4 * pair_step1<TRAV>();
    Addr a0 = (Addr)(r.base + (Addr)(4ll * pair_d0<TRAV>(1)));
    Addr a1 = (Addr)(r.base + (Addr)(4ll * pair_d1<TRAV>(1)));
    unsigned col = tma;
    int k = 1;
    for (; k + 3 <= kfast; k += 4) {
        float x[8];
        tm_ld8(col, x);
        tm_wait_ld();
        const float2 pa = __fmul2_rn(make_float2(x[0], x[1]), invD);
        const float2 pb = __fmul2_rn(make_float2(x[2], x[3]), invD);
        const float2 pc = __fmul2_rn(make_float2(x[4], x[5]), invD);
        const float2 pd = __fmul2_rn(make_float2(x[6], x[7]), invD);
        red4<SMEM, false, s0, s1>(a0, a1, k, r.la, r.lb, act, pa.x, pa.y, pb.x, pb.y);
        red4<SMEM, false, s0, s1>(a0 + (Addr)(2 * s0), a1 + (Addr)(2 * s1), k + 2, r.la, r.lb, act,
                                  pc.x, pc.y, pd.x, pd.y);
        a0 += (Addr)(4 * s0);
        a1 += (Addr)(4 * s1);
        col += 8;
    }
    for (; k + 1 <= kfast; k += 2) {
        float x0, x1, x2, x3;
        tm_ld4(col, x0, x1, x2, x3);
        tm_wait_ld();
        const float2 pa = __fmul2_rn(make_float2(x0, x1), invD);
        const float2 pb = __fmul2_rn(make_float2(x2, x3), invD);
        red4<SMEM, false, s0, s1>(a0, a1, k, r.la, r.lb, act, pa.x, pa.y, pb.x, pb.y);
        a0 += (Addr)(2 * s0);
        a1 += (Addr)(2 * s1);
        col += 4;
    }
    for (; k <= kmax; k += 2) {
        float x0, x1, x2, x3;
        tm_ld4(col, x0, x1, x2, x3);
        tm_wait_ld();
        const float2 pa = __fmul2_rn(make_float2(x0, x1), invD);
        const float2 pb = __fmul2_rn(make_float2(x2, x3), invD);
        red4<SMEM, true, s0, s1>(a0, a1, k, r.la, r.lb, act, pa.x, pa.y, pb.x, pb.y);
        a0 += (Addr)(2 * s0);
        a1 += (Addr)(2 * s1);
        col += 4;
    }
}

// The fixed-point terms of two pairs (four pixels; pa = pair k, pb = pair k + 1,
// .x the first pixels, .y the second ones) added into the H words at a0, a1,
// a0 + S0, a1 + S1 and the L words kAccWords words further on.  v holds
// P rho', s2 = 2^12 / D and sl = 2^32 / D, so x 2^12 = v s2:
//   t1 = 2^23 + v s2 rounded toward zero   (bits: magic + H, H = floor(x 2^12)),
//   c  = (2^43 + 2^23) - t1 2^20 = 2^23 - H 2^20        (exact),
//   t2 = v sl + c rounded to nearest = 2^23 + (x 2^12 - H) 2^20 rounded
//                                                       (bits: magic + L),
// the remainder taken from the FMA's exact product v sl.
template <int S0, int S1>
__device__ __forceinline__ void fx4(unsigned a0, unsigned a1, float2 pa, float2 pb, float2 s2,
                                    float2 sl)
{
    const float2 M = make_float2(kFxMagic, kFxMagic);
    const float2 m20 = make_float2(-1048576.0f, -1048576.0f);        // -2^20
    const float2 K = make_float2(0x1p43f + 0x1p23f, 0x1p43f + 0x1p23f);
    const float2 ha = __ffma2_rz(pa, s2, M), hb = __ffma2_rz(pb, s2, M);
    const float2 la = __ffma2_rn(pa, sl, __ffma2_rn(ha, m20, K));
    const float2 lb = __ffma2_rn(pb, sl, __ffma2_rn(hb, m20, K));
#ifdef TSP_DEBUG_CHECKS
    {
        constexpr unsigned C = 4u * kAccWords;
        if (!(tsp_sh_ok(a0, 4, 2) && tsp_sh_ok(a1, 4, 2) && tsp_sh_ok(a0 + (unsigned)S0, 4, 2) &&
              tsp_sh_ok(a1 + (unsigned)S1, 4, 2) && tsp_sh_ok(a0 + C, 4, 2) &&
              tsp_sh_ok(a1 + C, 4, 2) && tsp_sh_ok(a0 + C + (unsigned)S0, 4, 2) &&
              tsp_sh_ok(a1 + C + (unsigned)S1, 4, 2)))
            return;
    }
#endif
    asm volatile(
        "red.shared.add.u32 [%0], %4;\n\tred.shared.add.u32 [%1], %5;\n\t"
        "red.shared.add.u32 [%0+%2], %6;\n\tred.shared.add.u32 [%1+%3], %7;\n\t"
        "red.shared.add.u32 [%0+%12], %8;\n\tred.shared.add.u32 [%1+%12], %9;\n\t"
        "red.shared.add.u32 [%0+%13], %10;\n\tred.shared.add.u32 [%1+%14], %11;"
        ::"r"(a0), "r"(a1), "n"(S0), "n"(S1),
        "r"(__float_as_uint(ha.x)), "r"(__float_as_uint(ha.y)), "r"(__float_as_uint(hb.x)),
        "r"(__float_as_uint(hb.y)), "r"(__float_as_uint(la.x)), "r"(__float_as_uint(la.y)),
        "r"(__float_as_uint(lb.x)), "r"(__float_as_uint(lb.y)), "n"(4 * kAccWords),
        "n"(4 * kAccWords + S0), "n"(4 * kAccWords + S1)
        : "memory");
}

// Pass 2 of the MLEM tile pass in fixed point: the terms x = P rho' / D of
// pairs 1 .. kmax (P rho' loaded back from tensor memory 16, 8 or 4 values at
// a time, 0 outside each lane's chord) added to the item's two-word
// accumulator at r.base (H words).
template <int TRAV>
__device__ __forceinline__ void pass2_fx(const RowP<true>& r, int kfast, int kmax, unsigned tma,
                                         float2 s2, float2 sl)
{
    constexpr int s0 = 4 * pair_step0<TRAV>(), s1 = 4 * pair_step1<TRAV>();
    unsigned a0 = r.base + (unsigned)(4 * pair_d0<TRAV>(1));
    unsigned a1 = r.base + (unsigned)(4 * pair_d1<TRAV>(1));
    unsigned col = tma;
    int k = 1;
    for (; k + 7 <= kfast; k += 8) {
        float x[16];
        tm_ld16(col, x);
        tm_wait_ld();
        fx4<s0, s1>(a0, a1, make_float2(x[0], x[1]), make_float2(x[2], x[3]), s2, sl);
        fx4<s0, s1>(a0 + (unsigned)(2 * s0), a1 + (unsigned)(2 * s1), make_float2(x[4], x[5]),
                    make_float2(x[6], x[7]), s2, sl);
        fx4<s0, s1>(a0 + (unsigned)(4 * s0), a1 + (unsigned)(4 * s1), make_float2(x[8], x[9]),
                    make_float2(x[10], x[11]), s2, sl);
        fx4<s0, s1>(a0 + (unsigned)(6 * s0), a1 + (unsigned)(6 * s1), make_float2(x[12], x[13]),
                    make_float2(x[14], x[15]), s2, sl);
        a0 += (unsigned)(8 * s0);
        a1 += (unsigned)(8 * s1);
        col += 16;
    }
    for (; k + 3 <= kfast; k += 4) {
        float x[8];
        tm_ld8(col, x);
        tm_wait_ld();
        fx4<s0, s1>(a0, a1, make_float2(x[0], x[1]), make_float2(x[2], x[3]), s2, sl);
        fx4<s0, s1>(a0 + (unsigned)(2 * s0), a1 + (unsigned)(2 * s1), make_float2(x[4], x[5]),
                    make_float2(x[6], x[7]), s2, sl);
        a0 += (unsigned)(4 * s0);
        a1 += (unsigned)(4 * s1);
        col += 8;
    }
    for (; k <= kmax; k += 2) {
        float x0, x1, x2, x3;
        tm_ld4(col, x0, x1, x2, x3);
        tm_wait_ld();
        fx4<s0, s1>(a0, a1, make_float2(x0, x1), make_float2(x2, x3), s2, sl);
        a0 += (unsigned)(2 * s0);
        a1 += (unsigned)(2 * s1);
        col += 4;
    }
}

// One event processed by a group of G warps; the lane holds row rows.x + rowi
// with traversal TRAV.  part: 6*G floats of shared scratch for the group's
// cross-warp reduction (double-buffered by parity).
// GLD (tiles that stage only A): rho' is read from the global image rp_base
// and the frame addresses the staged accumulator acc_base.
template <int TRAV, int LMAX, int MODE, bool SMEM, bool GLD, bool KZ>
__device__ __forceinline__ void event_rows(const Geo& g, const EventsView& evs, int e, int rowi,
                                           const Frame* f, const float* rp_base, float* acc_base,
                                           int G, int wig, int lane, int bar_id, float* part,
                                           int& parity, BlockSums* bs, unsigned tma)
{
    constexpr bool GRAD = (MODE == kGrad);
    // the MLEM pass over a staged region accumulates in fixed point (fx4)
    constexpr bool kFx = (MODE == kMlem) && SMEM && !GLD;
    const float4 ev = evs.geo[e];
    int2 rws = evs.rows[e];
    const int evflags = rws.y & ~kEvRowsMask;
    rws.y &= kEvRowsMask;
    RowK<SMEM> r;
    RowG rg;
    // Rows are paired around the middle of the window (lane-row 2k -> mid - k,
    // 2k + 1 -> mid + k + 1), so that each warp holds rows of similar chord
    // length: its lanes run out of pixels at nearly the same step, which
    // lengthens the unpredicated pairs of the packed passes and shortens the
    // idle tail.  Rows 2k and 2k + 1 sit on opposite sides of the middle, an
    // odd distance apart, so a warp's 32 rows still fall in 32 distinct banks
    // at a common column.
    const int mid = (rws.y - 1) >> 1, k = rowi >> 1;
    const int ri = (rowi & 1) ? mid + k + 1 : mid - k;
    // KZ: the event's own sigma_z (z profile); else the context's constants
    make_row<TRAV, LMAX, GRAD, SMEM, GLD>(g, KZ ? ev_sig(g, ev) : geo_sig(g), ev, evs.geo64 + e,
                                          rws.x + ri, ri >= 0 && ri < rws.y, evflags, f,
                                          GLD ? acc_base : rp_base, rp_base, r, rg, bs);
    float D = 0.0f, Ez = 0.0f, El = 0.0f;
    float P[4];
    int maxlen = 0, kfast = 0, kmax = 0;
    RowP<SMEM> q;
    const bool active = max(r.lim_odd, r.lim_even) > 0;
    if constexpr (!GRAD) {
        PairC c;
        pair_row<TRAV, LMAX, SMEM, GLD>(r, active, q, c);
        kmax = __reduce_max_sync(0xffffffffu, active ? max(q.la, q.lb) : 0);
        // (a warp without active lanes has kmax = 0 and does no pair at all)
        kfast = min(kmax, __reduce_min_sync(0xffffffffu, active ? min(q.la, q.lb) : LMAX / 2));
        float2 D2 = make_float2(0.0f, 0.0f);
        pass1_pairs<TRAV, LMAX, SMEM, GLD, MODE != kLoglik, kFx>(q, c, kfast, kmax, D2, tma);
        D = D2.x + D2.y;
    } else {
        maxlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)max(r.lim_odd, r.lim_even));
        float Dp = 0.0f;
        pass1_step<TRAV, LMAX, GRAD, SMEM, GLD, true, 0>(r, rg, maxlen, tma, P, Dp, Ez, El);
        D = Dp;
    }
    if (MODE != kLoglik) tm_wait_st();
    D = warp_sum(D);
    if (GRAD) {
        Ez = warp_sum(Ez);
        El = warp_sum(El);
    }
    if (G > 1) {
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
            if (GRAD) {
                Ez += slot[G + w];
                El += slot[2 * G + w];
            }
        }
        parity ^= 1;
    }
    if (D > 0.0f) {
        if (wig == 0 && lane == 0) {
            atomicAdd(&bs->used, 1ull);
            if (MODE != kMlem) atomicAdd(&bs->logD, (double)logf(D));
            if (GRAD) {
                atomicAdd(&bs->giz, (double)(Ez / D));
                atomicAdd(&bs->gil, (double)(El / D));
            }
        }
        if (MODE != kLoglik) {
            // the accumulator has the rho' buffer's layout at a fixed byte offset
            // (GLD: the frame already addresses the accumulator)
            const auto off = (decltype(r.base))((const char*)acc_base - (const char*)rp_base);
            const float invD = 1.0f / D;
            if constexpr (kFx) {
                q.base += off;
                const float s = invD * 4096.0f, sl = invD * 0x1p32f;
                pass2_fx<TRAV>(q, kfast, kmax, tma, make_float2(s, s), make_float2(sl, sl));
            } else if constexpr (!GRAD) {
                if (!GLD) q.base += off;
                const float2 invD2 = make_float2(invD, invD);
                pass2_pairs<TRAV, SMEM>(q, (int)active, kfast, kmax, tma, invD2);
            } else {
                RowK<SMEM> ra = r;
                if (!GLD) ra.base += off;
                pass2_step<TRAV, LMAX, SMEM, 0>(ra, maxlen, tma, P, invD);
            }
        }
    }
}

// NSEG = 1: lane-row q = blk*32 + lane covers its row whole (kAlt).  NSEG = 2:
// even warps cover the right halves and odd warps the left halves of rows
// rb*32 + lane (a warp-uniform choice, no divergence).  The row block of warp
// wig is rotated by the group's index (rot = grp mod the number of blocks):
// a block's warps sit on the SM's schedulers by warp index mod 4, and without
// the rotation warp wig of every group, with the same rows of the window (the
// middle rows, with the longest chords, for wig = 0), would land on the same
// scheduler, which would then carry the most work.
template <int LMAX, int MODE, int NSEG, bool SMEM, bool GLD, bool KZ>
__device__ __forceinline__ void process_event(const Geo& g, const EventsView& evs, int e, int G,
                                              int wig, int lane, int bar_id, float* part,
                                              int& parity, const Frame* f, const float* rp_base,
                                              float* acc_base, BlockSums* bs, unsigned tma,
                                              int rot)
{
    if constexpr (NSEG == 1) {
        int blk = wig + rot;
        blk -= blk >= G ? G : 0;
        event_rows<kAlt, LMAX, MODE, SMEM, GLD, KZ>(g, evs, e, blk * 32 + lane, f, rp_base, acc_base,
                                               G, wig, lane, bar_id, part, parity, bs, tma);
    } else {
        const int nb = G >> 1;
        int rb = (wig >> 1) + rot;
        rb -= rb >= nb ? nb : 0;
        if ((wig & 1) == 0)
            event_rows<kPos, LMAX, MODE, SMEM, GLD, KZ>(g, evs, e, rb * 32 + lane, f,
                                                   rp_base, acc_base, G, wig, lane, bar_id, part,
                                                   parity, bs, tma);
        else
            event_rows<kNeg, LMAX, MODE, SMEM, GLD, KZ>(g, evs, e, rb * 32 + lane, f,
                                                   rp_base, acc_base, G, wig, lane, bar_id, part,
                                                   parity, bs, tma);
    }
}

__device__ __forceinline__ void init_block_sums(BlockSums* bs)
{
    if (threadIdx.x == 0) {
        bs->used = bs->qclip = bs->lclip = 0ull;
        bs->logD = bs->giz = bs->gil = 0.0;
    }
}

__device__ __forceinline__ void flush_block_sums(const BlockSums* bs, Accum* accum, int mode)
{
    if (threadIdx.x != 0) return;
    if (bs->used) atomicAdd(&accum->n_used, bs->used);
    if (bs->lclip) atomicAdd(&accum->n_lclip, bs->lclip);
    if (bs->qclip) atomicAdd(&accum->n_qclip, bs->qclip);
    if (mode != kMlem && bs->logD != 0.0) atomicAdd(&accum->sum_logD, bs->logD);
    if (mode == kGrad) {
        if (bs->giz != 0.0) atomicAdd(&accum->g_iz, bs->giz);
        if (bs->gil != 0.0) atomicAdd(&accum->g_il, bs->gil);
    }
}

// Frame of tile bin `bin` (the staged region of Tiling), or the whole image
// for bin < 0 (the outlier path).
__device__ __forceinline__ Frame tile_frame(const Geo& g, const Tiling& tl, int bin)
{
    Frame f;
    if (bin < 0) {
        f.oy = 0;
        f.zbase = 0;
        f.Y0 = 0;
        f.stride = g.nz;
        f.rh = g.ny;
        f.rw = g.nz;
        f.shear = 0.0f;
        return f;
    }
    const int tiles_per_bin = tl.tiles_y * tl.tiles_z;
    const int b = bin / tiles_per_bin;
    const int rest = bin - b * tiles_per_bin;
    const int ty = rest / tl.tiles_z, tz = rest - ty * tl.tiles_z;
    f.oy = ty * tl.TY - tl.HY;
    f.zbase = tz * tl.TZ - tl.HZ - tl.zs_off;
    f.Y0 = tl.Y0;
    f.stride = tl.RS;
    f.rh = tl.RH;
    f.rw = tl.RW;
    f.shear = bin_shear(tl, b);
    return f;
}

// Persistent tile kernel.  Work items are int4 (tile bin, first event, count,
// reconstruction).  Plain form (BATCH = false): one reconstruction, passed as
// `p`.  Batched form: item.w indexes `table`, whose record is copied to shared
// memory when it changes.  `queue` is the work counter (zero at launch).
// GLD: only the accumulator is staged (windows too large for both regions);
// rho' is read from the global image through the read-only cache.  KZ: the
// form for a z-dependent sigma_z (each event's own resolution constants; a
// batch takes it when any of its reconstructions has one); the form without
// it reads the context's constants.  (The two are separate kernels because
// the gradient pass is at the register limit: holding both row setups in one
// kernel spilled there.)
template <int LMAX, int MODE, int NSEG, bool BATCH, bool GLD = false, bool KZ = false>
__global__ void __launch_bounds__(pass_threads(LMAX, MODE, NSEG, BATCH), 1)
k_tiles(Inst p, const Inst* __restrict__ table, const int4* __restrict__ items, int n_items,
        int* queue)
{
    constexpr int kThreads = pass_threads(LMAX, MODE, NSEG, BATCH);
    constexpr int kWarps = kThreads / 32;
    extern __shared__ float4 smem_f4[];
    float* const smem = reinterpret_cast<float*>(smem_f4);
    __shared__ int s_item;
    __shared__ Frame s_frame;
    __shared__ BlockSums s_sums;
    __shared__ Inst s_inst;
    __shared__ unsigned s_tmem;
    const Inst& I = BATCH ? s_inst : p;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kCols = tm_block_cols(LMAX, kWarps);
    if (warp == 0) tm_alloc<kCols>(&s_tmem);
    init_block_sums(&s_sums);
#ifdef TSP_DEBUG_CHECKS
    if (tid == 0) tsp_dbg_word = 0ull;
#endif
    // the slack around the rho' region is read (times P = 0) by the
    // unpredicated pass-1 loads, so it must hold finite values
    if (!BATCH) {
        const int region = p.tl.RH * p.tl.RS;
        float* s_rp = smem + kPadFloats;
        float* s_acc = GLD ? s_rp : s_rp + region + 2 * kPadFloats;
        for (int k = tid; k < kPadFloats; k += kThreads) {
            s_rp[-kPadFloats + k] = 0.0f;
            s_rp[region + k] = 0.0f;
            s_acc[-kPadFloats + k] = 0.0f;
            s_acc[region + k] = 0.0f;
        }
    }
    int cur = -1;                                 // reconstruction held in s_inst
    tm_sync_threads();
    const unsigned tma = tm_thread_addr<LMAX>(s_tmem, warp);

    for (;;) {
        if (tid == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int4 item = items[it];
        if (BATCH && item.w != cur) {
            if (cur >= 0 && tid == 0) {
                flush_block_sums(&s_sums, s_inst.accum, MODE);
                init_block_sums(&s_sums);
#ifdef TSP_DEBUG_CHECKS
                if (tsp_dbg_word) atomicCAS(&s_inst.accum->dbg, 0ull, tsp_dbg_word);
                tsp_dbg_word = 0ull;
#endif
            }
            __syncthreads();
            const unsigned long long* src = reinterpret_cast<const unsigned long long*>(table + item.w);
            unsigned long long* dst = reinterpret_cast<unsigned long long*>(&s_inst);
            for (int k = tid; k < (int)(sizeof(Inst) / 8); k += kThreads) dst[k] = src[k];
            cur = item.w;
            __syncthreads();
            const int region = s_inst.tl.RH * s_inst.tl.RS;
            float* s_rp = smem + kPadFloats;
            float* s_acc = s_rp + region + 2 * kPadFloats;
            for (int k = tid; k < kPadFloats; k += kThreads) {
                s_rp[-kPadFloats + k] = 0.0f;
                s_rp[region + k] = 0.0f;
                s_acc[-kPadFloats + k] = 0.0f;
                s_acc[region + k] = 0.0f;
            }
        }
        const Geo& g = I.g;
        const Tiling& tl = I.tl;
        const int G = I.G;
        const int ngroups = group_count(kWarps, G);
        const int grp = warp / G, wig = warp - grp * G;
        const int region = tl.RH * tl.RS;
        float* s_rp = smem + kPadFloats;
        float* s_acc = GLD ? s_rp : s_rp + region + 2 * kPadFloats;
        // the L words of the fixed-point accumulator (MLEM over a staged region)
        unsigned* s_accL = GLD ? nullptr : reinterpret_cast<unsigned*>(s_acc) + kAccWords;
        float* part = (GLD ? s_acc : s_acc + kAccWords) + region + kPadFloats + grp * (2 * 3 * G);
        int parity = 0;
        const Frame f = tile_frame(g, tl, item.x);
        if (tid == 0) s_frame = f;
        if (GLD) {
            if (MODE != kLoglik)
                for (int k = tid; k < region; k += kThreads) s_acc[k] = 0.0f;
        } else {
            for (int rr = warp; rr < tl.RH; rr += kWarps) {
                const int iy = f.oy + rr;
                const bool row_in = iy >= 0 && iy < g.ny;
                const int z0row = f.zbase + (int)rintf(__fmul_rn(f.shear, (float)(iy - f.Y0)));
                for (int cc = lane; cc < tl.RS; cc += 32) {
                    const int iz = z0row + cc;
                    float v = 0.0f;
                    if (row_in && cc < tl.RW && iz >= 0 && iz < g.nz)
                        v = I.rhop[(size_t)iy * g.nz + iz];
                    s_rp[rr * tl.RS + cc] = v;
                    if (MODE != kLoglik) s_acc[rr * tl.RS + cc] = 0.0f;
                    if (MODE == kMlem) s_accL[rr * tl.RS + cc] = 0u;
                }
            }
        }
        __syncthreads();
        if (grp < ngroups) {
            const int rot = grp % (NSEG == 1 ? G : (G >> 1));
            for (int e = item.y + grp; e < item.y + item.z; e += ngroups)
                process_event<LMAX, MODE, NSEG, true, GLD, KZ>(
                    g, I.evs, e, G, wig, lane, 1 + grp, part, parity, &s_frame,
                    GLD ? I.rhop : s_rp, s_acc, &s_sums, tma, rot);
        }
        __syncthreads();
        if (MODE != kLoglik) {
            for (int rr = warp; rr < tl.RH; rr += kWarps) {
                const int iy = f.oy + rr;
                if (iy < 0 || iy >= g.ny) continue;
                const int z0row = f.zbase + (int)rintf(__fmul_rn(f.shear, (float)(iy - f.Y0)));
                for (int cc = lane; cc < tl.RW; cc += 32) {
                    const int iz = z0row + cc;
                    const int k = rr * tl.RS + cc;
                    float v;
                    if (MODE == kMlem && !GLD) {
                        // A += X / rho' (the fixed-point sums, see kAccWords)
                        const unsigned wh = __float_as_uint(s_acc[k]), wl = s_accL[k];
                        const unsigned sh = wh & 0xFFFFFFu, sl = wl - (wh & 0xFF000000u);
                        const float X = fmaf((float)sl, 0x1p-32f, (float)sh * 0x1p-12f);
                        const float rp = s_rp[k];
                        v = rp > 0.0f ? X / rp : 0.0f;
                    } else {
                        v = s_acc[k];
                    }
                    if (iz >= 0 && iz < g.nz && v != 0.0f)
                        atomicAdd(I.A + (size_t)iy * g.nz + iz, v);
                }
            }
            __syncthreads();
        }
    }
    tm_sync_threads();
    if (!BATCH || cur >= 0) flush_block_sums(&s_sums, I.accum, MODE);
#ifdef TSP_DEBUG_CHECKS
    if (tid == 0 && tsp_dbg_word && (!BATCH || cur >= 0))
        atomicCAS(&I.accum->dbg, 0ull, tsp_dbg_word);
#endif
    if (warp == 0) tm_dealloc<kCols>(s_tmem);
}

// Events whose window does not fit their tile's region: same evaluation, with
// rho' read from global memory and the scatter done by global atomics.
template <int LMAX, int MODE, int NSEG>
__global__ void __launch_bounds__(pass_threads(LMAX, MODE, NSEG, false), 1)
k_outliers(Geo g, EventsView evs, int first, int count, const float* __restrict__ rhop,
           float* __restrict__ A, Accum* accum, int G)
{
    constexpr int kWarps = pass_threads(LMAX, MODE, NSEG, false) / 32;
    __shared__ float s_part[kWarps * 2 * 3];
    __shared__ Frame s_frame;
    __shared__ BlockSums s_sums;
    __shared__ unsigned s_tmem;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kCols = tm_block_cols(LMAX, kWarps);
    if (warp == 0) tm_alloc<kCols>(&s_tmem);
    const int ngroups = group_count(kWarps, G);
    const int grp = warp / G, wig = warp - grp * G;
    float* part = s_part + grp * (2 * 3 * G);
    int parity = 0;
    init_block_sums(&s_sums);
    if (tid == 0) {
        s_frame.oy = 0;
        s_frame.zbase = 0;
        s_frame.Y0 = 0;
        s_frame.stride = g.nz;
        s_frame.rh = g.ny;
        s_frame.rw = g.nz;
        s_frame.shear = 0.0f;
    }
    tm_sync_threads();
    const unsigned tma = tm_thread_addr<LMAX>(s_tmem, warp);
    if (grp < ngroups) {
        const int rot = grp % (NSEG == 1 ? G : (G >> 1));
        for (int k = blockIdx.x * ngroups + grp; k < count; k += gridDim.x * ngroups)
            process_event<LMAX, MODE, NSEG, false, false, true>(g, evs, first + k, G, wig, lane,
                                                                1 + grp, part, parity, &s_frame,
                                                                rhop, A, &s_sums, tma, rot);
    }
    tm_sync_threads();
    flush_block_sums(&s_sums, accum, MODE);
    if (warp == 0) tm_dealloc<kCols>(s_tmem);
}

// Batched outlier kernel: items (-1, first, count, reconstruction), one block
// per item at a time.
template <int LMAX, int MODE, int NSEG>
__global__ void __launch_bounds__(pass_threads(LMAX, MODE, NSEG, true), 1)
k_outliers_batch(const Inst* __restrict__ table, const int4* __restrict__ items, int n_items)
{
    constexpr int kThreads = pass_threads(LMAX, MODE, NSEG, true);
    constexpr int kWarps = kThreads / 32;
    __shared__ float s_part[kWarps * 2 * 3];
    __shared__ Frame s_frame;
    __shared__ BlockSums s_sums;
    __shared__ Inst s_inst;
    __shared__ unsigned s_tmem;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kCols = tm_block_cols(LMAX, kWarps);
    if (warp == 0) tm_alloc<kCols>(&s_tmem);
    tm_sync_threads();
    const unsigned tma = tm_thread_addr<LMAX>(s_tmem, warp);
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 item = items[it];
        __syncthreads();
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(table + item.w);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(&s_inst);
        for (int k = tid; k < (int)(sizeof(Inst) / 8); k += kThreads) dst[k] = src[k];
        init_block_sums(&s_sums);
        __syncthreads();
        if (tid == 0) s_frame = tile_frame(s_inst.g, s_inst.tl, -1);
        __syncthreads();
        const int G = s_inst.G;
        const int ngroups = group_count(kWarps, G);
        const int grp = warp / G, wig = warp - grp * G;
        float* part = s_part + grp * (2 * 3 * G);
        int parity = 0;
        if (grp < ngroups) {
            const int rot = grp % (NSEG == 1 ? G : (G >> 1));
            for (int k = grp; k < item.z; k += ngroups)
                process_event<LMAX, MODE, NSEG, false, false, true>(
                    s_inst.g, s_inst.evs, item.y + k, G, wig, lane, 1 + grp, part, parity,
                    &s_frame, s_inst.rhop, s_inst.A, &s_sums, tma, rot);
        }
        __syncthreads();
        flush_block_sums(&s_sums, s_inst.accum, MODE);
    }
    tm_sync_threads();
    if (warp == 0) tm_dealloc<kCols>(s_tmem);
}

}  // namespace tsp
