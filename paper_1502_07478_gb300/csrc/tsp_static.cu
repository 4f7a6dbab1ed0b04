// tsp_mlem_update_noalloc: one MLEM update that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs under a fixed device
// memory budget handed out by a host framework, real-time acquisition loops
// where an allocation (and the implicit synchronisation it may bring) is not
// allowed, or plug-ins that must not touch the allocator of the process that
// hosts them.  For them this entry point runs the same MLEM pass as
// tsp_iterate, but keeps all its scratch (the staged rho', the back-projection
// accumulator, the prepared events of one chunk, the pass counters) in one
// file-scope static device array of fixed size.  The caller passes inputs and
// the output; nothing is allocated on the device or on the host.
//
// The pass is the global-memory variant of the MLEM kernel (the one that
// serves events whose window does not fit a tile): rho' is read from the
// scratch copy and the scatter goes to the scratch accumulator with global
// atomics, chunk by chunk.  Results equal tsp_iterate's up to the order of
// floating-point summation.
#include <atomic>
#include <cmath>
#include <cstdio>

#include "tsp.h"
#include "tsp_launch.h"

using namespace tsp;

namespace {

// Layout of the static scratch (bytes, each part 256-byte aligned).
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kImgBytes = align_up(sizeof(float) * ((size_t)TSP_NOALLOC_MAX_PIXELS + kPadFloats));
constexpr size_t kOffRhop = 0;
constexpr size_t kOffA = kOffRhop + kImgBytes;
constexpr size_t kOffGeo = kOffA + kImgBytes;
constexpr size_t kOffGeo64 = kOffGeo + align_up(sizeof(float4) * (size_t)TSP_NOALLOC_CHUNK);
constexpr size_t kOffRows = kOffGeo64 + align_up(sizeof(Ev64) * (size_t)TSP_NOALLOC_CHUNK);
constexpr size_t kOffAccum = kOffRows + align_up(sizeof(int2) * (size_t)TSP_NOALLOC_CHUNK);
constexpr size_t kScratchBytes = kOffAccum + align_up(sizeof(Accum));
static_assert(kScratchBytes <= (size_t)TSP_NOALLOC_SCRATCH_BYTES, "scratch size in tsp.h too small");

// The scratch array.  Every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_tsp_noalloc_scratch[TSP_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch, looked up once per device.
constexpr int kMaxDevices = 64;
std::atomic<unsigned char*> g_scratch_addr[kMaxDevices];

int report(char* errbuf, size_t errlen, int code, const char* fmt, long long a = 0, long long b = 0)
{
    if (errbuf && errlen) snprintf(errbuf, errlen, fmt, a, b);
    return code;
}

// Eq. 2 in double precision, the App. B box and the first and last rows with a
// non-empty chord, for events [0, n) of a chunk.  Non-finite events get no rows.
__global__ void k_prepare_chunk(Geo g, long long n, const float* __restrict__ zu,
                                const float* __restrict__ zd, const float* __restrict__ dl,
                                float4* __restrict__ geo, Ev64* __restrict__ geo64,
                                int2* __restrict__ rows)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        Ev64 e64 = make_ev64(0.0, 0.0, 0.0, 1.0);
        float4 ev = make_float4(0.f, 0.f, 0.f, 1.f);
        int2 rw = make_int2(0, 0);
        if (direct_reconstruction(g, zu[j], zd[j], dl[j], e64)) {
            ev = make_float4((float)e64.x, (float)e64.y, (float)e64.z, (float)e64.w);
            const EvSig es = ev_sig(g, ev);
            int iy_lo, nrows, iz_lo, ncols;
            event_bbox(g, es, ev, iy_lo, nrows, iz_lo, ncols);
            int first = -1, last = -1;
            for (int r = 0; r < nrows; ++r) {
                const Chord c = row_chord(g, es, ev, &e64, iy_lo + r);
                if (c.count > 0) {
                    if (first < 0) first = iy_lo + r;
                    last = iy_lo + r;
                }
            }
            if (first >= 0) rw = make_int2(first, last - first + 1);
        }
        geo[j] = ev;
        geo64[j] = e64;
        rows[j] = rw;
    }
}

// rho_out = rho_in * A: the end of one update of Eq. iter.
__global__ void k_update_out(int npix, const float* __restrict__ rho_in,
                             const float* __restrict__ A, float* __restrict__ rho_out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x)
        rho_out[i] = rho_in[i] * A[i];
}

// Kernel constants and lane layout for params: the lane layout comes from
// lane_plan(), the helper the context planner uses, so this pass launches the
// kernel form whose lane capacity the chords of k_prepare_chunk were sized
// for.  Returns TSP_OK or TSP_EINVAL.
int geometry(const tsp_params& p, Geo& g, int& lmax, int& nseg, int& G, char* errbuf,
             size_t errlen)
{
    auto pos = [](double v) { return std::isfinite(v) && v > 0.0; };
    if (!pos(p.R) || !pos(p.L) || p.ny <= 0 || p.nz <= 0 || !pos(p.sigma_z) ||
        !pos(p.sigma_dl) || !(p.dy == 0.0 || pos(p.dy)) || !(p.dz == 0.0 || pos(p.dz)) ||
        !(p.cut == 0.0 || pos(p.cut)) || p.flags != 0 || !cinv_valid(p))
        return report(errbuf, errlen, TSP_EINVAL, "invalid tsp_params");
    g = make_geo(p);
    LanePlan lp;
    if (const char* why = lane_plan(p, lp)) return report(errbuf, errlen, TSP_EINVAL, why);
    lmax = lp.lmax;
    nseg = lp.nseg;
    G = lp.G;
    return TSP_OK;
}

}  // namespace

extern "C" int tsp_mlem_update_noalloc(const tsp_params* params, const float* zu, const float* zd,
                                       const float* dl, int64_t n, const float* s,
                                       const float* rho_in, float* rho_out, void* stream,
                                       char* errbuf, size_t errlen)
{
    if (errbuf && errlen) errbuf[0] = '\0';
    if (!params) return report(errbuf, errlen, TSP_EINVAL, "params is NULL");
    if (n < 0) return report(errbuf, errlen, TSP_EINVAL, "n < 0");
    if (n > 0 && (!zu || !zd || !dl)) return report(errbuf, errlen, TSP_EINVAL, "event pointer is NULL");
    if (!s || !rho_in || !rho_out) return report(errbuf, errlen, TSP_EINVAL, "image pointer is NULL");
    if (rho_in == rho_out) return report(errbuf, errlen, TSP_EINVAL, "rho_out must not alias rho_in");
    const long long npix = (long long)params->ny * (long long)params->nz;
    if (npix > TSP_NOALLOC_MAX_PIXELS)
        return report(errbuf, errlen, TSP_EINVAL,
                      "ny*nz = %lld exceeds the static scratch limit of %lld pixels", npix,
                      (long long)TSP_NOALLOC_MAX_PIXELS);
    Geo g;
    int lmax = 0, nseg = 1, G = 1;
    int rc = geometry(*params, g, lmax, nseg, G, errbuf, errlen);
    if (rc) return rc;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return report(errbuf, errlen, TSP_ECUDA, "cudaGetDevice failed");
    unsigned char* base = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!base) {
        // set-up, once per device, with that device current
        e = cudaGetSymbolAddress((void**)&base, g_tsp_noalloc_scratch);
        if (e != cudaSuccess || !base)
            return report(errbuf, errlen, TSP_ECUDA, "cudaGetSymbolAddress of the scratch failed");
        g_scratch_addr[dev].store(base, std::memory_order_release);
    }
    float* rhop = reinterpret_cast<float*>(base + kOffRhop);
    float* A = reinterpret_cast<float*>(base + kOffA);
    float4* geo = reinterpret_cast<float4*>(base + kOffGeo);
    Ev64* geo64 = reinterpret_cast<Ev64*>(base + kOffGeo64);
    int2* rows = reinterpret_cast<int2*>(base + kOffRows);
    Accum* accum = reinterpret_cast<Accum*>(base + kOffAccum);
    cudaStream_t st = (cudaStream_t)stream;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        sms <= 0) {
        cudaGetLastError();   // leave no pending error for a later launch check
        return report(errbuf, errlen, TSP_ECUDA, "cudaDeviceGetAttribute(MultiProcessorCount) failed");
    }

    // the scratch keeps the previous call's contents: clear what must start at 0
    if ((e = launch_begin(accum, st)) != cudaSuccess ||
        (e = launch_fill(A, npix + kPadFloats, 0.0f, st)) != cudaSuccess ||
        (e = launch_fill(rhop + npix, kPadFloats, 0.0f, st)) != cudaSuccess ||
        (e = launch_set_rhop((int)npix, rho_in, s, rhop, accum, st)) != cudaSuccess)
        return report(errbuf, errlen, TSP_ECUDA, "launch failed");
    PassArgs a;
    a.g = g;
    a.tl = Tiling{};
    a.evs.geo = geo;
    a.evs.geo64 = geo64;
    a.evs.rows = rows;
    a.items = nullptr;
    a.n_items = 0;
    a.outlier_first = 0;
    a.rhop = rhop;
    a.A = A;
    a.accum = accum;
    a.G = G;
    a.nseg = nseg;
    a.gld = 0;
    a.grid = sms;
    a.smem = 0;
    for (long long c0 = 0; c0 < n; c0 += TSP_NOALLOC_CHUNK) {
        const long long nc = (n - c0 < TSP_NOALLOC_CHUNK) ? n - c0 : TSP_NOALLOC_CHUNK;
        const int blocks = (int)((nc + 255) / 256);
        k_prepare_chunk<<<blocks, 256, 0, st>>>(g, nc, zu + c0, zd + c0, dl + c0, geo, geo64, rows);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return report(errbuf, errlen, TSP_ECUDA, "launch failed");
        a.outlier_count = (int)nc;
        if ((e = launch_pass(lmax, kMlem, a, st)) != cudaSuccess)
            return report(errbuf, errlen, TSP_ECUDA, "launch failed");
    }
    k_update_out<<<(int)((npix + 1023) / 1024), 256, 0, st>>>((int)npix, rho_in, A, rho_out);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return report(errbuf, errlen, TSP_ECUDA, "launch failed");
    return TSP_OK;
}
