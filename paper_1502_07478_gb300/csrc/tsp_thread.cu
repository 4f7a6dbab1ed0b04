// Thread-granularity MLEM pass: one event per thread, the shape of the
// paper's thread-granularity kernel (Sec. 4.2, compared there with one warp
// per event).  Kept as an ablation of the tile kernel, selectable per context
// (tsp_set_variant): the thread walks its event's window row by row (chords of
// the cut ellipse, the same membership decision as the tile kernel), reads
// rho' from global memory, and evaluates P twice -- for the denominator, then
// for the scatter by global atomics -- since one thread cannot cache a window
// of kernel values.
#include "tsp_launch.h"

namespace tsp {

namespace {

constexpr int kThreadBlock = 256;

__global__ void __launch_bounds__(kThreadBlock)
k_thread_events(Geo g, EventsView evs, int n, const float* __restrict__ rhop,
                float* __restrict__ A, Accum* accum)
{
    unsigned long long used = 0, qclip = 0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const float4 ev = evs.geo[j];
        int2 rws = evs.rows[j];
        rws.y &= kEvRowsMask;
        const EvSig es = ev_sig(g, ev);
        float D = 0.0f, invD = 0.0f;
        for (int pass = 0; pass < 2; ++pass) {
            for (int r = 0; r < rws.y; ++r) {
                const int iy = rws.x + r;
                const Chord c = row_chord(g, es, ev, evs.geo64 + j, iy);
                if (c.count == 0) continue;
                float Qc, gam2, alpha, beta;
                row_q(g, es, ev, c, Qc, gam2);
                row_acb(g, es, ev, c, alpha, beta);
                const float u0 = fmaf((float)c.lo, g.dz, g.z0) - c.zc;
                const float Q0 = fmaf(gam2, u0, Qc), dQ = gam2 * g.dz;
                const float A0 = g.kA * fmaf(alpha, u0, beta), dA = g.kA * alpha * g.dz;
                const float su0 = es.ksu * u0, dsu = es.ksu * g.dz;
                const float C0 = es.log2K - g.half_log2e * c.B0;
                const size_t base = (size_t)iy * g.nz + c.lo;
                for (int k = 0; k < c.count; ++k) {
                    const float fd = (float)k;
                    const float Q = fmaf(fd, dQ, Q0);
                    if (!(Q > 0.0f)) {           // reading R5: P = 0
                        if (pass == 0) ++qclip;
                        continue;
                    }
                    const float rq = rsqrt_approx(Q);
                    const float su = fmaf(fd, dsu, su0);
                    const float w = fmaf(fd, dA, A0) * rq;
                    const float p = rq * ex2_approx(fmaf(w, w, fmaf(-su, su, C0)));
                    if (pass == 0)
                        D = fmaf(p, __ldg(rhop + base + k), D);
                    else
                        atomicAdd(A + base + k, p * invD);
                }
            }
            if (pass == 0) {
                if (!(D > 0.0f)) break;
                invD = 1.0f / D;
                ++used;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        used += __shfl_xor_sync(0xffffffffu, used, o);
        qclip += __shfl_xor_sync(0xffffffffu, qclip, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (used) atomicAdd(&accum->n_used, used);
        if (qclip) atomicAdd(&accum->n_qclip, qclip);
    }
}

}  // namespace

cudaError_t launch_thread_pass(const Geo& g, const EventsView& evs, int n, const float* rhop,
                               float* A, Accum* accum, int sms, cudaStream_t st)
{
    if (cudaError_t f = sim_launch()) return f;
    if (n <= 0) return cudaSuccess;
    int blocks = (n + kThreadBlock - 1) / kThreadBlock;
    if (blocks > 8 * sms) blocks = 8 * sms;
    k_thread_events<<<blocks, kThreadBlock, 0, st>>>(g, evs, n, rhop, A, accum);
    return cudaGetLastError();
}

}  // namespace tsp
