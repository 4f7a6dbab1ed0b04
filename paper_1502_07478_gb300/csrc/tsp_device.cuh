// Device-side data structures and helpers shared by the libtsp kernels.
//
// Notation (Sec. 2-3 of the paper): an event is reconstructed by Eq. 2 at
// (yt, zt) with tan(theta~) = t; c2i = 1 + t^2 = 1/cos^2(theta~).  For a pixel
// centred at (y, z): Dy = y - yt, u = (z - zt) - t*Dy (the first two entries of
// the vector b).  With the diagonal C^-1 = diag(iz, iz, il), iz = 1/sigma_z^2,
// il = 1/sigma_dl^2, the quadratic forms of Eq. kernel reduce to
//   bCb = 2 iz u^2 + 4 il Dy^2 c2i                               (App. B)
//   aCa = 2 iz (R^2 + y^2) c2i^2 + 4 il y^2 t^2 c2i
//   aCb = -2 iz y c2i u + 4 il y t Dy c2i
//   oCb = -2 iz y t c2i u + 2 il y (1 + 2 t^2) Dy c2i
// using a_3 = -2 y tan sec (the derivative of e_3 = -2 y sec).  Within one image
// row (fixed y) every term is a polynomial of degree <= 2 in u, so each lane
// computes row constants once and walks its chord of the 3-sigma ellipse.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tsp {

constexpr int kPadFloats = 128;        // slack after image-sized buffers (>= max LMAX)

enum Mode : int { kMlem = 0, kLoglik = 1, kGrad = 2 };

// Threads per persistent block of the passes: 1024 for every pass.  The P
// cache lives in tensor memory, not registers, so the one-lane-per-row passes
// fit 64 registers a thread (a few spilled in some forms, off the pixel loop)
// and the two-lanes-per-row passes hold both half-row traversals without
// spilling; at 0.5 mm an event takes 16 warps, so a block of 32 runs two events
// at a time.  A group of G <= kMinWarps warps always fits, and a block runs at
// most 15 groups of two or more warps (one named barrier each, ids 1..15).
__host__ __device__ constexpr int pass_threads(int lmax, int mode, int nseg, bool batch)
{
    return (void)lmax, (void)mode, (void)nseg, (void)batch, 1024;
}
constexpr int kMinWarps = 16;
constexpr int kMaxWarps = 32;

// Event groups of G warps in a block of `warps` warps.  Groups of more than one
// warp synchronise on named barriers 1..15, so there are at most 15 of them.
__host__ __device__ constexpr int group_count(int warps, int G)
{
    return G > 1 && warps / G > 15 ? 15 : warps / G;
}

// Per-reconstruction constants, passed by value to the kernels.
struct Geo {
    int ny, nz;
    float y0, z0;           // centre of pixel (0, 0)
    float dy, dz, inv_dy, inv_dz;
    float R;
    float iz, il;           // 1/sigma_z^2, 1/sigma_dl^2
    float cut2;             // cut^2: window is bCb <= cut2
    float hy_coef;          // bounding-box half-height = hy_coef / sqrt(c2i)
    float hz_a, hz_b;       // bounding-box half-width = sqrt(hz_a + hz_b * t^2/c2i)
    float log2K;            // log2 of det^(1/2)(C^-1) / (2 pi^2)
    float ksu;              // sqrt(log2(e) iz)
    float kA;               // sqrt(log2(e) / 2)
    float half_log2e;       // log2(e) / 2
    float inv_sqrt_2iz;     // 1 / sqrt(2 iz)
    // the cross term gamma of C^-1 (Sec. 3) enters only row constants:
    //   Q += -gR8 t c2i sec (y + Dy),  aCb += -gR4 c2i sec Dy  (bCb unchanged)
    float gR8, gR4;         // 8 gamma R, 4 gamma R
    float g2;               // 2 gamma^2
    float ldz, ldl;         // (1/2) d log det(C^-1) / d iz, / d il
    // z-dependent resolution (Sec. 3): an event at z~ has sigma_z f,
    // f = 1 + kz min(1, zs2 z~^2); kz = 0 keeps sigma_z constant
    float kz, zs2;          // kappa_z, (2/L)^2
    // double-precision copies for the exact window decision near its boundary
    double y0d, z0d, dyd, dzd, Rd, izd, ild, cut2d;
    double Ld;              // strip length
    double kzd, zs2d;
};

// Resolution constants of one event.  With kz = 0 they are the Geo's; else the
// event's sigma_z is sigma_z f (f = 1 + kz min(1, (2 z~/L)^2)), so that
// iz -> iz/f^2, 1/sqrt(2 iz) -> f/sqrt(2 iz), sqrt(log2(e) iz) -> /f, the box
// term hz_a -> hz_a f^2, log2 K moves by half the log2 of the ratio of
// det(C^-1) = iz (iz il - 2 gamma^2), and so do the log-determinant
// derivatives.  inv_f2 = 1/f^2 = d iz_event / d iz turns the event's d/d iz
// into one with respect to the base value.  The quantities that decide window
// membership are formed with explicitly rounded operations, so that the event
// preparation and the passes derive the same chords.
struct EvSig {
    float iz, inv_sqrt_2iz, ksu, log2K, hz_a, ldz, ldl, inv_f, inv_f2;
};

// The context's constants (kz = 0).
__device__ __forceinline__ EvSig geo_sig(const Geo& g)
{
    EvSig s;
    s.iz = g.iz;
    s.inv_sqrt_2iz = g.inv_sqrt_2iz;
    s.ksu = g.ksu;
    s.log2K = g.log2K;
    s.hz_a = g.hz_a;
    s.ldz = g.ldz;
    s.ldl = g.ldl;
    s.inv_f = 1.0f;
    s.inv_f2 = 1.0f;
    return s;
}

__device__ __forceinline__ EvSig ev_sig(const Geo& g, const float4& ev)
{
    if (g.kz == 0.0f) return geo_sig(g);
    EvSig s;
    const float f = __fmaf_rn(g.kz, fminf(__fmul_rn(__fmul_rn(ev.y, ev.y), g.zs2), 1.0f), 1.0f);
    const float f2 = __fmul_rn(f, f);
    s.inv_f = __fdiv_rn(1.0f, f);
    s.inv_f2 = __fdiv_rn(1.0f, f2);
    s.iz = __fmul_rn(g.iz, s.inv_f2);
    s.inv_sqrt_2iz = __fmul_rn(g.inv_sqrt_2iz, f);
    s.ksu = __fdiv_rn(g.ksu, f);
    s.hz_a = __fmul_rn(g.hz_a, f2);
    // det(C^-1) = iz (iz il - 2 gamma^2), base (e0) and event (e1) factors
    const float e0 = g.iz * g.il - g.g2, e1 = s.iz * g.il - g.g2;
    s.log2K = g.log2K + 0.5f * log2f(s.inv_f2 * (e1 / e0));
    s.ldz = (s.iz * g.il - 0.5f * g.g2) / (s.iz * e1);
    s.ldl = 0.5f * s.iz / e1;
    return s;
}

// Image tiling used by the shared-memory accumulation.
//
// Events are binned by the angle bin b of tan(theta~) (width dtb, starting at
// t0) and by a tile of a sheared image frame: column iz of row iy has sheared
// coordinate z' = iz - shift_b(iy) + zs_off with
//   shift_b(iy) = rint(s_b * (iy - Y0)),  s_b = (t0 + (b + 1/2) dtb) dy/dz,
// the shift that lines up the chord centres of events with tan(theta~) near
// the bin centre.  Tile (b, ty, tz) holds the events whose window-centre pixel
// has row in [ty TY, +TY) and sheared column in [tz TZ, +TZ).  Its staged
// region has RH = TY + 2 HY rows starting at row ty TY - HY; region row iy
// starts at image column  tz TZ - HZ - zs_off + shift_b(iy)  and is RW columns
// wide, stored with row stride RS floats.  Bin index = (b*tiles_y + ty)*tiles_z
// + tz; one more bin collects the outliers.
struct Tiling {
    int TY, TZ, HY, HZ;
    int RH, RW, RS;
    int tiles_y, tiles_z, nb;
    float t0, dtb, inv_dtb;
    float rho_yz;              // dy / dz
    int Y0, zs_off;
};

__device__ __forceinline__ float bin_shear(const Tiling& tl, int b)
{
    return __fmul_rn(__fmaf_rn((float)b + 0.5f, tl.dtb, tl.t0), tl.rho_yz);
}

__device__ __forceinline__ int row_shift(const Tiling& tl, float shear, int iy)
{
    return (int)rintf(__fmul_rn(shear, (float)(iy - tl.Y0)));
}

// The MLEM tile pass accumulates, per pixel and work item, the responsibility
// sum X = sum_j P_jl rho'_l / D_j (each term in [0, 1], since D_j >= P_jl rho'_l)
// in fixed point over two 32-bit words, with native integer shared-memory adds
// (a float add to shared memory is a compare-and-swap loop on this GPU).  Term
// x is split as x 2^12 = H + L 2^-20 with H = floor(x 2^12) <= 4096 and
// L = round((x 2^12 - H) 2^20) <= 2^20, both formed by adding the magic 2^23
// in float and taking the bits (bits = 0x4B000000 + integer; L from the
// exact product inside an FMA); the words are added unreduced.  With at most kItemMaxEvents events an item (each event
// adds a nonzero term to a pixel at most once), the H word's low 24 bits hold
// sum H exactly (<= 4000 * 4097 < 2^24) and its top byte the magic's total,
// which the L word received the same number of times:
//   sum H = wh & 0xFFFFFF,   sum L = wl - (wh & 0xFF000000)   (mod 2^32, exact
// as sum L <= 4000 * 2^20 < 2^32), X = (sum H + sum L 2^-20) 2^-12, quantum
// 2^-32 per term.  The flush adds X / rho'_l to A.  (At a pixel with rho' = 0
// the terms are 0 and the item adds nothing to A there; the update rho A is 0
// at such a pixel either way.)
constexpr int kItemMaxEvents = 4000;
constexpr float kFxMagic = 8388608.0f;            // 2^23
constexpr unsigned kFxMagicBits = 0x4B000000u;

// Distance, in 32-bit words, from a pixel's H word to its L word: a
// compile-time constant, so that the scatter reaches both words from one
// register address.  A region of RH*RS <= kAccWords - 2*kPadFloats words
// keeps the L region and both regions' slack apart.
constexpr int kAccWords = 18432;

// Shared-memory layout of the tile kernel, in 32-bit words: kPadFloats slack,
// the rho' region (RH*RS), 2*kPadFloats slack, the accumulator's H region
// (RH*RS; the float accumulator of the other passes), its L region at
// kAccWords words from the H region, kPadFloats slack, then the groups'
// reduction slots (warps/G groups x 2 parities x 3G floats <= 6*kMaxWarps).
__host__ __device__ constexpr size_t tiles_smem_floats(int RH, int RS)
{
    return (size_t)kPadFloats + (size_t)RH * RS + 2 * kPadFloats + (size_t)kAccWords +
           (size_t)RH * RS + kPadFloats + 6 * kMaxWarps;
}

// A staged region fits the two-word accumulator layout.
__host__ __device__ constexpr bool tiles_region_fits(int RH, int RS)
{
    return (long long)RH * RS <= (long long)kAccWords - 2 * kPadFloats;
}

// The same with only the accumulator staged (rho' read from global memory).
__host__ __device__ constexpr size_t tiles_acc_smem_floats(int RH, int RS)
{
    return (size_t)kPadFloats + (size_t)RH * RS + kPadFloats + 6 * kMaxWarps;
}

// Device-side accumulators of one pass.
struct Accum {
    unsigned long long n_used;   // events with D > 0
    unsigned long long n_qclip;  // in-window pixels dropped because Q <= 0
    unsigned long long n_lclip;  // chord pixels beyond the lane capacity (must stay 0)
    unsigned long long dbg;      // TSP_DEBUG_CHECKS builds: the first shared-memory access
                                 // outside a block's dynamic window since the context was
                                 // created (not cleared per pass), as
                                 // (site << 32) | (byte offset from the window + 1); else 0
    double sum_logD;             // sum_j log D_j
    double g_iz;                 // sum_j (1/D_j) sum_i rho'_i P_ji dlogP/d(iz)
    double g_il;                 // sum_j (1/D_j) sum_i rho'_i P_ji dlogP/d(il)
    double sum_rhop;             // sum_i s_i rho_i
    int queue;                   // persistent-kernel work counter
    int pad1[3];
};

// Bounds checks of a TSP_DEBUG_CHECKS build (a substitute for a memory checker):
// every shared-memory access of the tile passes' pixel loops is tested against
// the block's dynamic shared-memory window; an access outside it is skipped and
// the first one is recorded in tsp_dbg_word (per block), which the kernel
// copies to Accum::dbg at its end.  Sites: 1 pass-1 rho' load, 2 pass-2
// fixed-point add, 3 pass-2 float add, 4 scalar pass load, 5 scalar pass add.
// Release builds compile the checks away (tsp_sh_ok is the literal true).
#ifdef TSP_DEBUG_CHECKS
extern __shared__ float4 tsp_dyn_smem[];
__shared__ unsigned long long tsp_dbg_word;

__device__ __forceinline__ bool tsp_sh_ok(unsigned a, unsigned bytes, int site)
{
    const unsigned lo = (unsigned)__cvta_generic_to_shared(tsp_dyn_smem);
    unsigned n;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(n));
    if (a >= lo && a - lo + bytes <= n) return true;
    atomicCAS(&tsp_dbg_word, 0ull, ((unsigned long long)site << 32) | (unsigned)(a - lo + 1u));
    return false;
}
#else
__device__ __forceinline__ constexpr bool tsp_sh_ok(unsigned, unsigned, int) { return true; }
#endif

// Double-precision event geometry (y~, z~, tan theta~, 1 + tan^2), 32-byte
// aligned so that one event is one 32-byte load.
struct __align__(32) Ev64 {
    double x, y, z, w;
};

__host__ __device__ __forceinline__ Ev64 make_ev64(double x, double y, double z, double w)
{
    Ev64 e;
    e.x = x;
    e.y = y;
    e.z = z;
    e.w = w;
    return e;
}

// Prepared events in binned order.
struct EventsView {
    const float4* __restrict__ geo;    // (yt, zt, t, c2i) per event, rounded from geo64
    const Ev64* __restrict__ geo64; // (yt, zt, t, c2i) in double precision
    const int2* __restrict__ rows;     // (first row, row count) of the non-empty chords
};

// One reconstruction as the tile kernel reads it: its constants, tiling,
// prepared events, rho' and back-projection buffers, pass accumulators and
// group size (warps per event).  The plain kernel takes it as a launch
// parameter; the batched kernel reads the record of each work item's
// reconstruction from a device table into shared memory.
struct Inst {
    Geo g;
    Tiling tl;
    EventsView evs;
    const float* rhop;
    float* A;
    Accum* accum;
    int G;
    int pad;
};
static_assert(sizeof(Inst) % 8 == 0, "Inst is copied in 8-byte words");

// Key of an event in the binning: its tile index, the outlier bin (the last
// bin), or kKeyEmpty for events whose window holds no pixel centre.
constexpr int kKeyEmpty = -1;

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void named_barrier(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Eq. 2 (first forms) for one event, in double precision; returns false for
// non-finite input.  ev = (y~, z~, tan theta~, 1 + tan^2).
__device__ __forceinline__ bool direct_reconstruction(const Geo& g, float zu, float zd, float dl,
                                                      Ev64& ev)
{
    if (!(isfinite(zu) && isfinite(zd) && isfinite(dl))) return false;
    const double t = ((double)zu - (double)zd) / (2.0 * g.Rd);
    const double c2i = 1.0 + t * t;
    const double yt = -0.5 * (double)dl / sqrt(c2i);
    const double zt = 0.5 * ((double)zu + (double)zd + 2.0 * yt * t);
    ev = make_ev64(yt, zt, t, c2i);
    return true;
}

// Clamp a float index range [lo, hi] to [0, n-1] without overflow in the
// float -> int conversion.  Returns the number of indices (>= 0).
__device__ __forceinline__ int clamp_range(float flo, float fhi, int n, int& lo)
{
    flo = fminf(fmaxf(flo, 0.0f), (float)n);
    fhi = fmaxf(fminf(fhi, (float)(n - 1)), -1.0f);
    lo = (int)flo;
    int hi = (int)fhi;
    return hi >= lo ? hi - lo + 1 : 0;
}

// The chord of row iy inside the event's cut ellipse: pixel columns
// [lo, lo + count) with bCb <= cut2 at their centres, clipped to the grid.
// Also returns Dy, y and B0 = 4 il Dy^2 c2i, zc = zt + t Dy (single precision).
struct Chord {
    int lo, count;
    float y, Dy, B0, zc;
};

// The single-precision window decision is checked in double precision when a
// chord end lies within a bound on its rounding error of a pixel centre, or
// when rem = cut2 - B0 is within its own error bound of 0, so that membership
// agrees with a double-precision evaluation of bCb <= cut^2 at every pixel.
// The bounds are a few times the worst-case error of the single-precision
// expressions (below 4e-4 pixel on the workloads' grids), including the
// relative error of the approximate reciprocal square root that gives
// sqrt(rem) (2^-22.9 for rsqrt.approx):
//   end:  kEndRel * (|x| + (|zc| + umax + |z0|)/dz)            (coordinates)
//       + kEndRel * cut2 / sqrt(rem) / sqrt(2 iz) / dz           (from umax)
//   rem:  kRemRel * cut2
// The check evaluates bCb in double precision at the pixels next to the
// uncertain end (the error is far below one pixel, so an end moves by at most
// one column) -- only multiplications and additions, no division or root.
constexpr float kEndRel = 1e-6f;
constexpr float kRemRel = 1e-5f;

// bCb of column iz in the row with offset Dy (B0 = 4 il Dy^2 c2i), double
// precision: the window quantity of Sec. 3 for a diagonal C^-1.
// The event's iz in double precision (see EvSig).
__device__ __forceinline__ double ev_izd(const Geo& g, const Ev64& e)
{
    if (g.kzd == 0.0) return g.izd;
    const double f = 1.0 + g.kzd * fmin(e.y * e.y * g.zs2d, 1.0);
    return g.izd / (f * f);
}

__device__ __forceinline__ double bq_fp64(const Geo& g, const Ev64& e, double izd, double Dy,
                                          double B0, int iz)
{
    const double u = (g.z0d + (double)iz * g.dzd) - (e.y + e.z * Dy);
    return 2.0 * izd * u * u + B0;
}

__device__ __forceinline__ int float_to_index(float x)
{
    return (int)fminf(fmaxf(x, -1.0e9f), 1.0e9f);
}

// Explicitly rounded operations (never contracted into FMAs), so that the
// event preparation and the MLEM passes derive bit-identical chords whatever
// the surrounding code lets the compiler fuse.  check = false skips the
// uncertainty tests (exact for an event whose preparation found no row that
// needed the double-precision decision: the same single-precision values
// decide the same way); *unsure (when given) records that a row needed it.
__device__ __forceinline__ Chord row_chord(const Geo& g, const EvSig& es, const float4& ev,
                                           const Ev64* __restrict__ ev64, int iy,
                                           bool check = true, bool* unsure = nullptr)
{
    Chord c;
    c.y = __fmaf_rn((float)iy, g.dy, g.y0);
    c.Dy = __fsub_rn(c.y, ev.x);
    c.B0 = __fmul_rn(__fmul_rn(__fmul_rn(4.0f * g.il, c.Dy), c.Dy), ev.w);
    c.zc = __fmaf_rn(ev.z, c.Dy, ev.y);
    c.lo = 0;
    c.count = 0;
    const float rem = __fsub_rn(g.cut2, c.B0);
    const bool unsure_rem = check && fabsf(rem) < kRemRel * g.cut2;
    bool unsure_lo = false, unsure_hi = false;
    int a = 0, b = -1;                                // candidate columns [a, b]
    if (rem >= 0.0f) {
        const float rs = rsqrt_approx(fmaxf(rem, 1e-30f));   // 1/sqrt(rem)
        const float sr = __fmul_rn(rem, rs);                  // sqrt(rem)
        const float umax = __fmul_rn(sr, es.inv_sqrt_2iz);
        const float xlo = __fmul_rn(__fsub_rn(__fsub_rn(c.zc, umax), g.z0), g.inv_dz);
        const float xhi = __fmul_rn(__fsub_rn(__fadd_rn(c.zc, umax), g.z0), g.inv_dz);
        if (check) {
            const float coord = (fabsf(c.zc) + umax + fabsf(g.z0)) * g.inv_dz;
            const float m = kEndRel * (fabsf(xhi) + coord) +
                            kEndRel * g.cut2 * es.inv_sqrt_2iz * g.inv_dz * rs;
            unsure_lo = fabsf(xlo - rintf(xlo)) < m;
            unsure_hi = fabsf(xhi - rintf(xhi)) < m;
        }
        a = float_to_index(ceilf(xlo));
        b = float_to_index(floorf(xhi));
    }
    if (unsure && (unsure_rem || unsure_lo || unsure_hi)) *unsure = true;
    if (unsure_rem || unsure_lo || unsure_hi) {
        const Ev64 e = *ev64;
        // (with the context's constants inv_f2 is the literal 1: no z profile)
        const double izd = es.inv_f2 == 1.0f ? g.izd : ev_izd(g, e);
        const double Dy = (g.y0d + (double)iy * g.dyd) - e.x;
        const double B0 = 4.0 * g.ild * Dy * Dy * e.w;
        if (unsure_rem) {
            // at most a few pixels around the chord centre can be inside
            const int k = float_to_index(rintf(__fmul_rn(__fsub_rn(c.zc, g.z0), g.inv_dz)));
            a = 0;
            b = -1;
            for (int iz = k - 2; iz <= k + 2; ++iz) {
                if (bq_fp64(g, e, izd, Dy, B0, iz) <= g.cut2d) {
                    if (b < a) a = iz;
                    b = iz;
                }
            }
        } else {
            if (unsure_lo) {
                if (bq_fp64(g, e, izd, Dy, B0, a - 1) <= g.cut2d) --a;
                else if (bq_fp64(g, e, izd, Dy, B0, a) > g.cut2d) ++a;
            }
            if (unsure_hi) {
                if (bq_fp64(g, e, izd, Dy, B0, b + 1) <= g.cut2d) ++b;
                else if (bq_fp64(g, e, izd, Dy, B0, b) > g.cut2d) --b;
            }
        }
    }
    if (b >= a) {
        c.lo = max(a, 0);
        const int hi = min(b, g.nz - 1);
        c.count = hi >= c.lo ? hi - c.lo + 1 : 0;
        if (c.count == 0) c.lo = 0;
    }
    return c;
}

// Row polynomials of Eq. kernel along the chord of row c (u = z - zc):
//   Q(u) = aCa + 2 oCb = Qc + gam2 u,    aCb(u) = alpha u + beta.
__device__ __forceinline__ void row_q(const Geo& g, const EvSig& es, const float4& ev,
                                      const Chord& c, float& Qc, float& gam2)
{
    const float t = ev.z, c2i = ev.w, y = c.y, Dy = c.Dy, y2 = y * y;
    const float aCa = 2.0f * es.iz * (g.R * g.R + y2) * c2i * c2i + 4.0f * g.il * y2 * t * t * c2i;
    Qc = aCa + 4.0f * g.il * y * fmaf(2.0f * t, t, 1.0f) * Dy * c2i;   // Q at u = 0
    if (g.gR8 != 0.0f) Qc -= g.gR8 * t * c2i * sqrtf(c2i) * (y + Dy);
    gam2 = -4.0f * es.iz * y * t * c2i;                                // 2 oCb slope
}

__device__ __forceinline__ void row_acb(const Geo& g, const EvSig& es, const float4& ev,
                                        const Chord& c, float& alpha, float& beta)
{
    const float t = ev.z, c2i = ev.w, y = c.y, Dy = c.Dy;
    alpha = -2.0f * es.iz * y * c2i;           // aCb slope in u
    beta = 4.0f * g.il * y * t * Dy * c2i;     // aCb at u = 0
    if (g.gR4 != 0.0f) beta -= g.gR4 * c2i * sqrtf(c2i) * Dy;
}

// Flags kept in the high bits of an event's row count (int2 (first row, rows)):
// kEvExact, no row of the event's window needed the double-precision window
// decision (row_chord may skip its uncertainty tests); kEvQPos, Q > 0 over the
// whole window (reading R5's clip cannot apply).  The event preparation sets
// them; forms that do not leave them clear, and every reader masks the count.
constexpr int kEvRowsMask = 0xFFFF;
constexpr int kEvExact = 1 << 29;
constexpr int kEvQPos = 1 << 30;

// A lower bound of Q = aCa + 2 oCb over every point of the event's window:
// with y = y~ + Dy, |Dy| <= hy (window half-height) and |u| <= umax (largest
// chord half-width), each term of row_q's Q is bounded below (the terms in
// y^2 t^2 and the y^2 part of aCa are >= 0).  The event is flagged when the
// bound exceeds 1e-3 of its leading term 2 iz R^2 c2i^2: that margin is three
// orders above the single-precision rounding of this bound and of the row
// polynomials, so single precision suffices here.
__device__ __forceinline__ bool q_positive_over_window(const Geo& g, const EvSig& es,
                                                       const float4& ev)
{
    const float t = fabsf(ev.z), c2i = ev.w;
    const float hy = g.hy_coef * rsqrtf(c2i) * 1.001f + g.dy;
    const float umax = sqrtf(g.cut2) * es.inv_sqrt_2iz + g.dz;
    const float ymax = fabsf(ev.x) + hy;
    const float lead = 2.0f * es.iz * g.R * g.R * c2i * c2i;
    float q = lead - 4.0f * g.il * ymax * (2.0f * t * t + 1.0f) * hy * c2i -
              4.0f * es.iz * ymax * t * c2i * umax;
    if (g.gR8 != 0.0f) q -= fabsf(g.gR8) * t * c2i * sqrtf(c2i) * (ymax + hy);
    return q > 1e-3f * lead;
}

// Bounding box of the event's window in pixel rows and columns, clipped to the
// grid (App. B half-extents, widened by 1e-5 relative so that FP32 rounding
// never drops a row whose chord is non-empty).
__device__ __forceinline__ void event_bbox(const Geo& g, const EvSig& es, const float4& ev,
                                           int& iy_lo, int& nrows,
                                           int& iz_lo, int& ncols)
{
    float hy = g.hy_coef * rsqrtf(ev.w) * 1.00001f;
    float s2 = ev.z * ev.z / ev.w;
    float hz = sqrtf(fmaf(g.hz_b, s2, es.hz_a)) * 1.00001f;
    nrows = clamp_range(ceilf((ev.x - hy - g.y0) * g.inv_dy), floorf((ev.x + hy - g.y0) * g.inv_dy),
                        g.ny, iy_lo);
    ncols = clamp_range(ceilf((ev.y - hz - g.z0) * g.inv_dz), floorf((ev.y + hz - g.z0) * g.inv_dz),
                        g.nz, iz_lo);
}

}  // namespace tsp
