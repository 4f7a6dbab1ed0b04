// Host-side launch interface of the libtsp kernels (internal to the library).
#pragma once

#include <cmath>

#include <cuda_runtime.h>

#include "tsp.h"
#include "tsp_device.cuh"

namespace tsp {

// Kernel constants of a (validated) parameter set (tsp_kernels.cu).
Geo make_geo(const tsp_params& p);
// Whether the parameters give a positive-definite C^-1 (2 gamma^2 < iz il).
bool cinv_valid(const tsp_params& p);

// Host-side fault injection, for tests of the error paths without a device
// fault.  The environment variable TSP_SIM_FAULT names one failure that the
// library then simulates at every site it reaches, for as long as the
// variable holds that value:
//   oom        device allocations fail as cudaMalloc does when memory is
//              exhausted (the entry point returns TSP_ENOMEM and unwinds)
//   launch     the kernel-launch helpers fail before enqueuing anything, with
//              cudaErrorLaunchOutOfResources (TSP_ECUDA)
//   nan_event  every uploaded chunk gets a NaN in its first z_u after the copy
//              (the event preparation rejects the upload: TSP_EINVAL)
//   timeout    the bounded wait (tsp_wait) gives up at once, as when the
//              enqueued work outlasts the limit (TSP_ETIMEOUT)
// Unset or any other value: no fault.
enum SimFault : int { kSimNone = 0, kSimOom = 1, kSimLaunch = 2, kSimNan = 3, kSimTimeout = 4 };
int sim_fault();

// The error a launch helper returns under TSP_SIM_FAULT=launch, else success.
inline cudaError_t sim_launch() { return sim_fault() == kSimLaunch ? cudaErrorLaunchOutOfResources : cudaSuccess; }

// cudaMalloc, or a simulated exhaustion under TSP_SIM_FAULT=oom.
template <class T>
cudaError_t dmalloc(T** p, size_t bytes)
{
    if (sim_fault() == kSimOom) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

// Lane capacities (pixels of one row segment a lane walks) compiled in.
constexpr int kLmaxList[] = {12, 24, 48, 64};
constexpr int kLmaxCount = 4;

// Lane layout of a parameter set's windows, shared by the context planner and
// the allocation-free entry point so that both launch the kernel form that
// the event preparation's chords were sized for:
//   need     longest chord of a window row in pixels, plus 2: the chord of the
//            cut ellipse is at most 2 cut sigma_z / sqrt(2) wide, with the
//            largest sigma_z of any event, sigma_z (1 + kappa_z)
//   lmax     smallest compiled capacity holding a whole chord (nseg = 1), else
//            one holding half a chord plus 2 (nseg = 2: two lanes per row)
//   maxrows  most rows of one window (|Dy| <= cut sigma_dl cos / 2), plus 2
//   G        warps per event: nseg lanes for each of maxrows rows
// Returns nullptr, or the reason the windows fit no compiled kernel.
struct LanePlan {
    int need, lmax, nseg, maxrows, G;
};

inline const char* lane_plan(const tsp_params& p, LanePlan& lp)
{
    const double dy = p.dy > 0 ? p.dy : 2.0 * p.R / p.ny;
    const double dz = p.dz > 0 ? p.dz : p.L / p.nz;
    const double cut = p.cut > 0 ? p.cut : 3.0;
    const double umax = cut * p.sigma_z * (1.0 + p.kappa_z) / std::sqrt(2.0);
    lp.need = (int)std::floor(2.0 * umax / dz) + 2;
    lp.lmax = 0;
    lp.nseg = 1;
    for (int k = 0; k < kLmaxCount && !lp.lmax; ++k)
        if (kLmaxList[k] >= lp.need) lp.lmax = kLmaxList[k];
    for (int k = 0; k < kLmaxCount && !lp.lmax; ++k)
        if (kLmaxList[k] >= lp.need / 2 + 2) {
            lp.lmax = kLmaxList[k];
            lp.nseg = 2;
        }
    if (!lp.lmax) return "window chords too long for the compiled lane capacities";
    const double hy = cut * p.sigma_dl / 2.0 * 1.00001;
    lp.maxrows = (int)std::floor(2.0 * hy / dy) + 2;
    lp.G = lp.nseg * ((lp.maxrows + 31) / 32);
    if (lp.G > kMinWarps) return "window has more rows than one block can hold";
    return nullptr;
}

// Lane capacity for two lanes per row (the accumulator-only tiles), or 0.
inline int lane_lmax_split(int need)
{
    for (int k = 0; k < kLmaxCount; ++k)
        if (kLmaxList[k] >= need / 2 + 2) return kLmaxList[k];
    return 0;
}

struct PassArgs {
    Geo g;
    Tiling tl;
    EventsView evs;
    const int4* items;
    int n_items;
    int outlier_first, outlier_count;
    const float* rhop;
    float* A;
    Accum* accum;
    int G, nseg;
    int gld;           // tiles stage only A; rho' read from global (nseg = 2)
    int grid;          // persistent blocks
    size_t smem;       // dynamic shared memory of the tile kernel
};

// A batched pass: the tile items (bin, first, count, reconstruction) of every
// reconstruction in `table`, in one persistent launch, and the outlier items
// (-1, first, count, reconstruction) in a second launch when there are any.
struct BatchArgs {
    const Inst* table;
    const int4* items;
    int n_items;
    const int4* outlier_items;
    int n_outlier_items;
    int* queue;        // work counter, zeroed before the launch
    int nseg;
    int kz;            // some reconstruction has a z-dependent sigma_z
    int grid;
    size_t smem;
};

// Image buffers of one reconstruction of a batch, for the batched per-pixel
// kernels.
struct BatchImg {
    float* rho;
    float* rhop;
    float* A;
    const float* s;
    float* g;          // gradient output (op 2)
    Accum* accum;
    int npix;
    int pad;
};

// Tile kernel + outlier kernel of one pass (MODE = kMlem, kLoglik or kGrad).
cudaError_t launch_pass(int lmax, int mode, const PassArgs& a, cudaStream_t st);
// Raise the dynamic shared-memory limit of the tile kernel for (lmax, mode).
cudaError_t prepare_pass(int lmax, int mode, size_t smem);

// Batched pass (MODE = kMlem or kGrad) and its shared-memory limit.
cudaError_t launch_batch_pass(int lmax, int mode, const BatchArgs& a, cudaStream_t st);
cudaError_t prepare_batch_pass(int lmax, size_t smem);

// Per-LMAX entry points (one translation unit each).
template <int LMAX>
cudaError_t launch_pass_l(int mode, const PassArgs& a, cudaStream_t st);
template <int LMAX>
cudaError_t prepare_pass_l(int mode, size_t smem);
template <int LMAX>
cudaError_t launch_batch_pass_l(int mode, const BatchArgs& a, cudaStream_t st);
template <int LMAX>
cudaError_t prepare_batch_pass_l(size_t smem);

// Auxiliary kernels (tsp_kernels.cu).
cudaError_t launch_sensitivity(double R, double L, int ny, int nz, double dy, double dz, float* s,
                               cudaStream_t st);
cudaError_t launch_setup(const Geo& g, const Tiling& tl, long long n, const float* zu,
                         const float* zd, const float* dl, float4* geo, Ev64* geo64, int2* rows,
                         int* key, unsigned long long* counters, int* bin_count, int nbins,
                         cudaStream_t st);
cudaError_t launch_scatter(long long n, int nbins, const int* key, const float4* geo_in,
                           const Ev64* g64_in, const int2* rows_in, const long long* offsets,
                           int* cursor, float4* geo_out, Ev64* g64_out, int2* rows_out,
                           cudaStream_t st);
cudaError_t launch_begin(Accum* accum, cudaStream_t st);
cudaError_t launch_finalize(int npix, float* rho, float* rhop, float* A, const float* s,
                            Accum* accum, cudaStream_t st);
cudaError_t launch_grad_finalize(int npix, float* g, float* A, const float* s, cudaStream_t st);
cudaError_t launch_set_rhop(int npix, const float* rho, const float* s, float* rhop, Accum* accum,
                            cudaStream_t st);
cudaError_t launch_batch_begin(const BatchImg* im, int k, int* queue, int nq, cudaStream_t st);
cudaError_t launch_batch_pixels(const BatchImg* im, int k, int max_npix, int op, cudaStream_t st);
// Thread-granularity MLEM pass over the n binned events (tsp_thread.cu).
cudaError_t launch_thread_pass(const Geo& g, const EventsView& evs, int n, const float* rhop,
                               float* A, Accum* accum, int sms, cudaStream_t st);
cudaError_t launch_direct_image(const Geo& g, long long n, const float* zu, const float* zd,
                                const float* dl, unsigned* h, float* out, cudaStream_t st);
cudaError_t launch_fill(float* p, long long n, float v, cudaStream_t st);
cudaError_t launch_check_image(int npix, const float* rho, int* bad, cudaStream_t st);

}  // namespace tsp
