// Auxiliary kernels of libtsp: sensitivity (Eq. s-yz), per-event preparation
// (Eq. 2 and the App. B window), binning of events by image tile, the image
// update that closes one iteration of Eq. iter, and small reductions.
#include <cstdlib>
#include <cstring>
#include <climits>
#include <cmath>

#include "tsp_launch.h"

namespace tsp {

namespace {

constexpr int kAuxThreads = 256;

inline int blocks_for(long long n, int per_block, int cap = 65535 * 8)
{
    long long b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

__device__ __forceinline__ double block_sum(double v, double* sh)
{
    // blockDim.x == kAuxThreads
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kAuxThreads / 32; ++w) t += sh[w];
    __syncthreads();
    return t;
}

// Eq. s-yz at pixel centres, in double precision, clamped at 0.
__global__ void k_sensitivity(double R, double L, int ny, int nz, double dy, double dz, float* s)
{
    const long long npix = (long long)ny * nz;
    const double hl = 0.5 * L;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix;
         i += (long long)gridDim.x * blockDim.x) {
        const int iy = (int)(i / nz), iz = (int)(i - (long long)iy * nz);
        const double y = -R + (iy + 0.5) * dy;
        const double z = -hl + (iz + 0.5) * dz;
        double v = 0.0;
        if (fabs(y) < R) {
            const double tmax = fmin((hl - z) / (R - y), (hl + z) / (R + y));
            const double tmin = fmax(-(hl + z) / (R - y), (z - hl) / (R + y));
            v = (atan(tmax) - atan(tmin)) / 3.14159265358979323846;
        }
        s[i] = (float)fmax(v, 0.0);
    }
}

// Per-event preparation.  counters: [0] non-finite events, [1] events with an
// empty window, [2] outliers, [3] in-window pixels (pixel evaluations).
// bin_count has nbins entries; the last bin collects the outliers.
__global__ void k_setup(Geo g, Tiling tl, long long n, const float* __restrict__ zu,
                        const float* __restrict__ zd, const float* __restrict__ dl,
                        float4* __restrict__ geo, Ev64* __restrict__ geo64,
                        int2* __restrict__ rows, int* __restrict__ key,
                        unsigned long long* counters, int* bin_count, int nbins)
{
    extern __shared__ int s_hist[];
    const bool use_smem = nbins <= 8192;
    if (use_smem) {
        for (int b = threadIdx.x; b < nbins; b += blockDim.x) s_hist[b] = 0;
        __syncthreads();
    }
    unsigned long long bad = 0, empty = 0, outl = 0, pix = 0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        Ev64 e64 = make_ev64(0.0, 0.0, 0.0, 1.0);
        float4 ev = make_float4(0.f, 0.f, 0.f, 1.f);
        int k = kKeyEmpty;
        int2 rw = make_int2(0, 0);
        if (!direct_reconstruction(g, zu[j], zd[j], dl[j], e64)) {
            ++bad;
        } else {
            ev = make_float4((float)e64.x, (float)e64.y, (float)e64.z, (float)e64.w);
            const EvSig es = ev_sig(g, ev);
            int iy_lo, nrows, iz_lo, ncols;
            event_bbox(g, es, ev, iy_lo, nrows, iz_lo, ncols);
            // angle bin and sheared tile of the pixel holding the window centre
            const float fb = floorf((ev.z - tl.t0) * tl.inv_dtb);
            const bool bin_ok = fb >= 0.0f && fb < (float)tl.nb;
            const int b = bin_ok ? (int)fb : 0;
            const float shear = bin_shear(tl, b);
            const int iyc = (int)fminf(fmaxf(floorf((ev.x - g.y0) * g.inv_dy + 0.5f), 0.f),
                                       (float)(g.ny - 1));
            const int izc = (int)fminf(fmaxf(floorf((ev.y - g.z0) * g.inv_dz + 0.5f), 0.f),
                                       (float)(g.nz - 1));
            const int zp = min(max(izc - row_shift(tl, shear, iyc) + tl.zs_off, 0),
                               tl.tiles_z * tl.TZ - 1);
            const int ty = iyc / tl.TY, tz = zp / tl.TZ;
            const int oy = ty * tl.TY - tl.HY, zbase = tz * tl.TZ - tl.HZ - tl.zs_off;
            bool fits = bin_ok, unsure = false;
            int first = -1, last = -1;
            unsigned long long cnt = 0;
            for (int r = 0; r < nrows; ++r) {
                const int iy = iy_lo + r;
                const Chord c = row_chord(g, es, ev, &e64, iy, true, &unsure);
                if (c.count > 0) {
                    if (first < 0) first = iy;
                    last = iy;
                    cnt += (unsigned long long)c.count;
                    const int z0row = zbase + row_shift(tl, shear, iy);
                    fits = fits && iy >= oy && iy < oy + tl.RH && c.lo >= z0row &&
                           c.lo + c.count <= z0row + tl.RW;
                }
            }
            if (cnt == 0) {
                ++empty;
            } else {
                pix += cnt;
                rw = make_int2(first, (last - first + 1) | (unsure ? 0 : kEvExact) |
                                          (q_positive_over_window(g, es, ev) ? kEvQPos : 0));
                k = fits ? (b * tl.tiles_y + ty) * tl.tiles_z + tz : nbins - 1;
                if (!fits) ++outl;
            }
        }
        geo[j] = ev;
        geo64[j] = e64;
        rows[j] = rw;
        key[j] = k;
        if (k >= 0) {
            if (use_smem) atomicAdd(&s_hist[k], 1);
            else atomicAdd(&bin_count[k], 1);
        }
    }
    // warp-aggregate the counters
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
        empty += __shfl_xor_sync(0xffffffffu, empty, o);
        outl += __shfl_xor_sync(0xffffffffu, outl, o);
        pix += __shfl_xor_sync(0xffffffffu, pix, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicAdd(&counters[0], bad);
        if (empty) atomicAdd(&counters[1], empty);
        if (outl) atomicAdd(&counters[2], outl);
        if (pix) atomicAdd(&counters[3], pix);
    }
    if (use_smem) {
        __syncthreads();
        for (int b = threadIdx.x; b < nbins; b += blockDim.x)
            if (s_hist[b]) atomicAdd(&bin_count[b], s_hist[b]);
    }
}

// Counting-sort scatter of the prepared events into binned order.  Within a
// block the rank of an event in its bin comes from a shared-memory counter and
// one global reservation is made per (block, bin).
__global__ void k_scatter(long long n, int nbins, const int* __restrict__ key,
                          const float4* __restrict__ geo_in, const Ev64* __restrict__ g64_in,
                          const int2* __restrict__ rows_in, const long long* __restrict__ offsets,
                          int* cursor, float4* __restrict__ geo_out, Ev64* __restrict__ g64_out,
                          int2* __restrict__ rows_out)
{
    extern __shared__ int s_cnt[];   // [nbins] local counts, then [nbins] reserved bases
    int* s_base = s_cnt + nbins;
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    int k = kKeyEmpty, rank = 0;
    if (j < n) {
        k = key[j];
        if (k >= 0) rank = atomicAdd(&s_cnt[k], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (s_cnt[b]) s_base[b] = atomicAdd(&cursor[b], s_cnt[b]);
    __syncthreads();
    if (k >= 0) {
        const long long pos = offsets[k] + s_base[k] + rank;
        geo_out[pos] = geo_in[j];
        g64_out[pos] = g64_in[j];
        rows_out[pos] = rows_in[j];
    }
}

__global__ void k_scatter_global(long long n, const int* __restrict__ key,
                                 const float4* __restrict__ geo_in,
                                 const Ev64* __restrict__ g64_in,
                                 const int2* __restrict__ rows_in,
                                 const long long* __restrict__ offsets, int* cursor,
                                 float4* __restrict__ geo_out, Ev64* __restrict__ g64_out,
                                 int2* __restrict__ rows_out)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        const int k = key[j];
        if (k < 0) continue;
        const long long pos = offsets[k] + atomicAdd(&cursor[k], 1);
        geo_out[pos] = geo_in[j];
        g64_out[pos] = g64_in[j];
        rows_out[pos] = rows_in[j];
    }
}

// Start of a pass: clear the accumulators and the work counter.
__global__ void k_begin(Accum* a)
{
    if (threadIdx.x == 0) {
        a->n_used = 0ull;
        a->n_qclip = 0ull;
        a->n_lclip = 0ull;
        a->sum_logD = 0.0;
        a->g_iz = 0.0;
        a->g_il = 0.0;
        a->sum_rhop = 0.0;
        a->queue = 0;
    }
}

// End of one iteration of Eq. iter: rho <- rho * A (A = sum_j P_j / D_j), then
// rho' = s rho for the next pass, A <- 0, and sum_i s_i rho_i.
__global__ void k_finalize(int npix, float* __restrict__ rho, float* __restrict__ rhop,
                           float* __restrict__ A, const float* __restrict__ s, Accum* a)
{
    __shared__ double sh[kAuxThreads / 32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
        const float r = rho[i] * A[i];
        const float p = s[i] * r;
        rho[i] = r;
        rhop[i] = p;
        A[i] = 0.0f;
        acc += (double)p;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) atomicAdd(&a->sum_rhop, acc);
}

// g_rho = s (A - 1); A <- 0.
__global__ void k_grad_finalize(int npix, float* __restrict__ g, float* __restrict__ A,
                                const float* __restrict__ s)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
        g[i] = s[i] * (A[i] - 1.0f);
        A[i] = 0.0f;
    }
}

// rho' = s rho and sum_i rho'_i.
__global__ void k_set_rhop(int npix, const float* __restrict__ rho, const float* __restrict__ s,
                           float* __restrict__ rhop, Accum* a)
{
    __shared__ double sh[kAuxThreads / 32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
        const float p = s[i] * rho[i];
        rhop[i] = p;
        acc += (double)p;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) atomicAdd(&a->sum_rhop, acc);
}

// Batched forms of k_begin and of the per-pixel kernels: blockIdx.y selects
// the reconstruction.  op 0 = end of an MLEM iteration (k_finalize), 1 = rho'
// refresh (k_set_rhop), 2 = gradient (k_grad_finalize), 3 = A <- 0.
__global__ void k_batch_begin(const BatchImg* __restrict__ im, int k, int* queue, int nq)
{
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        Accum* a = im[i].accum;
        a->n_used = 0ull;
        a->n_qclip = 0ull;
        a->n_lclip = 0ull;
        a->sum_logD = 0.0;
        a->g_iz = 0.0;
        a->g_il = 0.0;
        a->sum_rhop = 0.0;
        a->queue = 0;
    }
    for (int q = threadIdx.x; q < nq; q += blockDim.x) queue[q] = 0;
}

__global__ void k_batch_pixels(const BatchImg* __restrict__ im, int op)
{
    __shared__ double sh[kAuxThreads / 32];
    const BatchImg b = im[blockIdx.y];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.npix; i += gridDim.x * blockDim.x) {
        if (op == 0) {
            const float r = b.rho[i] * b.A[i];
            const float p = b.s[i] * r;
            b.rho[i] = r;
            b.rhop[i] = p;
            b.A[i] = 0.0f;
            acc += (double)p;
        } else if (op == 1) {
            const float p = b.s[i] * b.rho[i];
            b.rhop[i] = p;
            acc += (double)p;
        } else if (op == 2) {
            b.g[i] = b.s[i] * (b.A[i] - 1.0f);
            b.A[i] = 0.0f;
        } else {
            b.A[i] = 0.0f;
        }
    }
    if (op >= 2) return;
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) atomicAdd(&b.accum->sum_rhop, acc);
}

// Direct-reconstruction image (Eq. 2, Sec. 2): count the events whose point
// (y~, z~) falls in each pixel.  Evaluated in double precision with every
// operation explicitly rounded (no contraction), in the order of Eq. 2's first
// forms: t = (zu - zd) / 2R, y~ = -dl / 2 / sqrt(1 + t^2),
// z~ = (zu + zd + 2 y~ t) / 2; pixel (iy, iz) covers [-R + iy dy, +dy) x
// [-L/2 + iz dz, +dz).
__global__ void k_direct_hist(Geo g, long long n, const float* __restrict__ zu,
                              const float* __restrict__ zd, const float* __restrict__ dl,
                              unsigned* __restrict__ h)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        const double u = zu[j], d = zd[j], l = dl[j];
        if (!(isfinite(u) && isfinite(d) && isfinite(l))) continue;
        const double t = __ddiv_rn(__dsub_rn(u, d), __dmul_rn(2.0, g.Rd));
        const double y = __ddiv_rn(__dmul_rn(-0.5, l), __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(t, t))));
        const double z =
            __dmul_rn(0.5, __dadd_rn(__dadd_rn(u, d), __dmul_rn(__dmul_rn(2.0, y), t)));
        const double fy = __ddiv_rn(__dadd_rn(y, g.Rd), g.dyd);
        const double fz = __ddiv_rn(__dadd_rn(z, __dmul_rn(0.5, g.Ld)), g.dzd);
        if (!(fy >= 0.0 && fy < (double)g.ny && fz >= 0.0 && fz < (double)g.nz)) continue;
        atomicAdd(&h[(size_t)(int)floor(fy) * g.nz + (int)floor(fz)], 1u);
    }
}

__global__ void k_counts_to_float(int n, const unsigned* __restrict__ h, float* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (float)h[i];
}

__global__ void k_fill(float* p, long long n, float v)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_check_image(int n, const float* __restrict__ rho, int* bad)
{
    int b = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float v = rho[i];
        if (!(isfinite(v) && v >= 0.0f)) b = 1;
    }
    if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

}  // namespace

bool cinv_valid(const tsp_params& p)
{
    // kappa_z in [0, 1]; C^-1 positive definite for every event's sigma_z,
    // the largest being sigma_z (1 + kappa_z)
    if (!(std::isfinite(p.kappa_z) && p.kappa_z >= 0.0 && p.kappa_z <= 1.0)) return false;
    const double szmax = p.sigma_z * (1.0 + p.kappa_z);
    const double iz = 1.0 / (szmax * szmax), il = 1.0 / (p.sigma_dl * p.sigma_dl);
    return std::isfinite(p.gamma) && 2.0 * p.gamma * p.gamma < iz * il;
}

Geo make_geo(const tsp_params& p)
{
    const double dy = p.dy > 0 ? p.dy : 2.0 * p.R / p.ny;
    const double dz = p.dz > 0 ? p.dz : p.L / p.nz;
    const double cut = p.cut > 0 ? p.cut : 3.0;
    const double iz = 1.0 / (p.sigma_z * p.sigma_z), il = 1.0 / (p.sigma_dl * p.sigma_dl);
    const double gm = p.gamma;
    const double log2e = 1.4426950408889634, pi = 3.14159265358979323846;
    Geo g{};
    g.ny = p.ny;
    g.nz = p.nz;
    g.dy = (float)dy;
    g.dz = (float)dz;
    g.inv_dy = (float)(1.0 / dy);
    g.inv_dz = (float)(1.0 / dz);
    g.y0 = (float)(-p.R + 0.5 * dy);
    g.z0 = (float)(-0.5 * p.L + 0.5 * dz);
    g.R = (float)p.R;
    g.iz = (float)iz;
    g.il = (float)il;
    g.cut2 = (float)(cut * cut);
    g.hy_coef = (float)(cut * p.sigma_dl / 2.0);
    g.hz_a = (float)(cut * cut * p.sigma_z * p.sigma_z / 2.0);
    g.hz_b = (float)(cut * cut * p.sigma_dl * p.sigma_dl / 4.0);
    // reading R4: K = det^(1/2)(C^-1) / (2 pi^2), det(C^-1) = iz^2 il - 2 iz gamma^2
    const double det = iz * iz * il - 2.0 * iz * gm * gm;
    g.log2K = (float)std::log2(std::sqrt(det) / (2.0 * pi * pi));
    g.ksu = (float)std::sqrt(log2e * iz);
    g.kA = (float)std::sqrt(log2e / 2.0);
    g.half_log2e = (float)(log2e / 2.0);
    g.inv_sqrt_2iz = (float)(1.0 / std::sqrt(2.0 * iz));
    g.gR8 = (float)(8.0 * gm * p.R);
    g.gR4 = (float)(4.0 * gm * p.R);
    g.g2 = (float)(2.0 * gm * gm);
    g.kz = (float)p.kappa_z;
    g.zs2 = (float)(4.0 / (p.L * p.L));
    g.kzd = p.kappa_z;
    g.zs2d = 4.0 / (p.L * p.L);
    g.ldz = (float)((iz * il - gm * gm) / (iz * (iz * il - 2.0 * gm * gm)));
    g.ldl = (float)(0.5 * iz / (iz * il - 2.0 * gm * gm));
    g.y0d = -p.R + 0.5 * dy;
    g.z0d = -0.5 * p.L + 0.5 * dz;
    g.dyd = dy;
    g.dzd = dz;
    g.Rd = p.R;
    g.izd = iz;
    g.ild = il;
    g.cut2d = cut * cut;
    g.Ld = p.L;
    return g;
}

int sim_fault()
{
    const char* v = std::getenv("TSP_SIM_FAULT");
    if (!v) return kSimNone;
    if (!std::strcmp(v, "oom")) return kSimOom;
    if (!std::strcmp(v, "launch")) return kSimLaunch;
    if (!std::strcmp(v, "nan_event")) return kSimNan;
    if (!std::strcmp(v, "timeout")) return kSimTimeout;
    return kSimNone;
}

cudaError_t launch_sensitivity(double R, double L, int ny, int nz, double dy, double dz, float* s,
                               cudaStream_t st)
{
    k_sensitivity<<<blocks_for((long long)ny * nz, kAuxThreads, 4096), kAuxThreads, 0, st>>>(
        R, L, ny, nz, dy, dz, s);
    return cudaGetLastError();
}

cudaError_t launch_setup(const Geo& g, const Tiling& tl, long long n, const float* zu,
                         const float* zd, const float* dl, float4* geo, Ev64* geo64, int2* rows,
                         int* key, unsigned long long* counters, int* bin_count, int nbins,
                         cudaStream_t st)
{
    if (cudaError_t f = sim_launch()) return f;
    if (n <= 0) return cudaSuccess;
    const size_t smem = nbins <= 8192 ? (size_t)nbins * sizeof(int) : 0;
    k_setup<<<blocks_for(n, kAuxThreads * 8, 4096), kAuxThreads, smem, st>>>(
        g, tl, n, zu, zd, dl, geo, geo64, rows, key, counters, bin_count, nbins);
    return cudaGetLastError();
}

cudaError_t launch_scatter(long long n, int nbins, const int* key, const float4* geo_in,
                           const Ev64* g64_in, const int2* rows_in, const long long* offsets,
                           int* cursor, float4* geo_out, Ev64* g64_out, int2* rows_out,
                           cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (nbins <= 4096) {
        k_scatter<<<blocks_for(n, kAuxThreads * 4, INT_MAX), kAuxThreads * 4,
                    2 * (size_t)nbins * sizeof(int), st>>>(n, nbins, key, geo_in, g64_in, rows_in,
                                                           offsets, cursor, geo_out, g64_out,
                                                           rows_out);
    } else {
        k_scatter_global<<<blocks_for(n, kAuxThreads, 4096), kAuxThreads, 0, st>>>(
            n, key, geo_in, g64_in, rows_in, offsets, cursor, geo_out, g64_out, rows_out);
    }
    return cudaGetLastError();
}

cudaError_t launch_begin(Accum* accum, cudaStream_t st)
{
    if (cudaError_t f = sim_launch()) return f;
    k_begin<<<1, 32, 0, st>>>(accum);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int npix, float* rho, float* rhop, float* A, const float* s,
                            Accum* accum, cudaStream_t st)
{
    if (cudaError_t f = sim_launch()) return f;
    k_finalize<<<blocks_for(npix, kAuxThreads * 4, 1024), kAuxThreads, 0, st>>>(npix, rho, rhop, A,
                                                                               s, accum);
    return cudaGetLastError();
}

cudaError_t launch_grad_finalize(int npix, float* g, float* A, const float* s, cudaStream_t st)
{
    if (cudaError_t f = sim_launch()) return f;
    k_grad_finalize<<<blocks_for(npix, kAuxThreads * 4, 1024), kAuxThreads, 0, st>>>(npix, g, A, s);
    return cudaGetLastError();
}

cudaError_t launch_set_rhop(int npix, const float* rho, const float* s, float* rhop, Accum* accum,
                            cudaStream_t st)
{
    if (cudaError_t f = sim_launch()) return f;
    k_set_rhop<<<blocks_for(npix, kAuxThreads * 4, 1024), kAuxThreads, 0, st>>>(npix, rho, s, rhop,
                                                                               accum);
    return cudaGetLastError();
}

cudaError_t launch_direct_image(const Geo& g, long long n, const float* zu, const float* zd,
                                const float* dl, unsigned* h, float* out, cudaStream_t st)
{
    const int npix = g.ny * g.nz;
    cudaError_t e = cudaMemsetAsync(h, 0, sizeof(unsigned) * (size_t)npix, st);
    if (e != cudaSuccess) return e;
    if (n > 0)
        k_direct_hist<<<blocks_for(n, kAuxThreads * 8, 4096), kAuxThreads, 0, st>>>(g, n, zu, zd,
                                                                                  dl, h);
    k_counts_to_float<<<blocks_for(npix, kAuxThreads * 4, 1024), kAuxThreads, 0, st>>>(npix, h,
                                                                                      out);
    return cudaGetLastError();
}

cudaError_t launch_fill(float* p, long long n, float v, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_fill<<<blocks_for(n, kAuxThreads * 4, 4096), kAuxThreads, 0, st>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_check_image(int n, const float* rho, int* bad, cudaStream_t st)
{
    k_check_image<<<blocks_for(n, kAuxThreads * 4, 1024), kAuxThreads, 0, st>>>(n, rho, bad);
    return cudaGetLastError();
}

cudaError_t launch_batch_begin(const BatchImg* im, int k, int* queue, int nq, cudaStream_t st)
{
    if (cudaError_t f = sim_launch()) return f;
    k_batch_begin<<<1, kAuxThreads, 0, st>>>(im, k, queue, nq);
    return cudaGetLastError();
}

cudaError_t launch_batch_pixels(const BatchImg* im, int k, int max_npix, int op, cudaStream_t st)
{
    if (cudaError_t f = sim_launch()) return f;
    if (k <= 0) return cudaSuccess;
    const dim3 grid(blocks_for(max_npix, kAuxThreads * 4, 256), k);
    k_batch_pixels<<<grid, kAuxThreads, 0, st>>>(im, op);
    return cudaGetLastError();
}

cudaError_t launch_batch_pass(int lmax, int mode, const BatchArgs& a, cudaStream_t st)
{
    if (cudaError_t f = sim_launch()) return f;
    switch (lmax) {
    case 12: return launch_batch_pass_l<12>(mode, a, st);
    case 24: return launch_batch_pass_l<24>(mode, a, st);
    case 48: return launch_batch_pass_l<48>(mode, a, st);
    case 64: return launch_batch_pass_l<64>(mode, a, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_batch_pass(int lmax, size_t smem)
{
    switch (lmax) {
    case 12: return prepare_batch_pass_l<12>(smem);
    case 24: return prepare_batch_pass_l<24>(smem);
    case 48: return prepare_batch_pass_l<48>(smem);
    case 64: return prepare_batch_pass_l<64>(smem);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pass(int lmax, int mode, const PassArgs& a, cudaStream_t st)
{
    if (cudaError_t f = sim_launch()) return f;
    switch (lmax) {
    case 12: return launch_pass_l<12>(mode, a, st);
    case 24: return launch_pass_l<24>(mode, a, st);
    case 48: return launch_pass_l<48>(mode, a, st);
    case 64: return launch_pass_l<64>(mode, a, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_pass(int lmax, int mode, size_t smem)
{
    switch (lmax) {
    case 12: return prepare_pass_l<12>(mode, smem);
    case 24: return prepare_pass_l<24>(mode, smem);
    case 48: return prepare_pass_l<48>(mode, smem);
    case 64: return prepare_pass_l<64>(mode, smem);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tsp
