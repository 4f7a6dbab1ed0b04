// Host-side state of a libtsp context and the internal helpers shared by the
// plain (tsp_api.cu) and batched (tsp_batch.cu) entry points.
#pragma once

#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "tsp.h"
#include "tsp_launch.h"

// Schedule knobs of the tile pass (what the autotuner chooses):
//   ty_cap       upper bound on the tile height TY (rows of window centres per
//                tile; the shared-memory budget may force a smaller TY)
//   items_per_sm target number of work items per SM; a tile's events are cut
//                into items of E = placed / (items_per_sm * SMs) events,
//                clamped to [32, 4096]
//   order        batched item order: 0 = longest estimated item first,
//                1 = round robin over the reconstructions
struct Schedule {
    int ty_cap = 128;
    int items_per_sm = 8;
    int order = 0;
};

// The ranges tsp.h documents for the schedule knobs.
inline bool schedule_valid(const tsp_schedule& s)
{
    return s.ty_cap >= 4 && s.ty_cap <= 128 && s.items_per_sm >= 1 && s.items_per_sm <= 64 &&
           (s.order == 0 || s.order == 1) && s.reserved == 0;
}
#define TSP_SCHEDULE_RANGES "schedule: ty_cap in [4,128], items_per_sm in [1,64], order 0 or 1, reserved 0"

struct tsp_ctx {
    tsp_params p{};
    tsp::Geo g{};
    tsp::Tiling tl{};
    int lmax = 0, nseg = 1, G = 1;
    int gld = 0;             // tiles stage only A, rho' read from global memory
    int variant = 0;         // MLEM pass: 0 tiles, 1 one thread per event
    int need = 0;            // longest chord of a window row, in pixels (+2)
    int maxrows = 0;         // most rows of one window
    int dev = 0, num_sms = 0;
    size_t smem = 0;
    int npix = 0;
    int nbins = 0;
    Schedule sched;
    float* rho = nullptr;
    float* rhop = nullptr;   // s * rho, padded by kPadFloats zeros
    float* A = nullptr;
    float* s = nullptr;
    float* gbuf = nullptr;
    tsp::Accum* accum = nullptr;
    long long n = 0, cap = 0;
    float *zu = nullptr, *zd = nullptr, *dl = nullptr;
    float4 *geo_u = nullptr, *geo = nullptr;
    tsp::Ev64 *geo64_u = nullptr, *geo64 = nullptr;
    int2 *rows_u = nullptr, *rows = nullptr;
    int* key = nullptr;
    int4* items = nullptr;
    int n_items = 0, items_cap = 0;
    std::vector<int> bin_cnt;          // events per bin (host copy; last = outliers)
    std::vector<long long> bin_off;    // first event of each bin in binned order
    long long outlier_first = 0, n_outliers = 0;
    unsigned long long counters_h[4] = {0, 0, 0, 0};
    unsigned long long* counters = nullptr;
    int* bin_count = nullptr;
    long long* offsets = nullptr;
    int* cursor = nullptr;
    int* flag = nullptr;
    bool uploaded = false, sens_ready = false;
    bool appending = false;           // between tsp_begin_events and tsp_end_events
    long long n_total = 0;            // events declared by tsp_begin_events
    cudaStream_t copy_stream = nullptr;   // host-to-device event copies
    cudaEvent_t copy_ev = nullptr;
    cudaEvent_t wait_ev = nullptr;        // tsp_wait's completion marker
    long long iterations = 0;
    cudaStream_t cap_stream = nullptr;
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        long long launches = 0;               // kernel nodes per replay
        std::vector<cudaEvent_t> ev;          // start/stop pairs around each MLEM pass
    };
    std::map<int, Graph> graphs;
    int last_graph = -1;                      // n_iter of the last replayed graph
    bool profiling = false;
    long long launches = 0;
    std::string err;
};

namespace tsp_host {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// An NVTX range around one entry point (upload, binning, iteration, readout),
// for timelines taken with a profiler; free when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Record msg as the context's last error (or the creation error when c is
// NULL) and return code.
int fail(tsp_ctx* c, int code, const std::string& msg);

template <class T>
void dfree(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

// Largest dynamic shared memory a tile kernel may request on device dev (the
// limit every tile kernel function is raised to).
size_t dyn_smem_limit(int dev);
// Check a parameter set (TSP_EINVAL with a message on c, or on the creation
// error when c is NULL).
int validate(const tsp_params* p, tsp_ctx* c);
// Kernel constants, lane capacity, group size and tiling from c->p and
// c->sched.ty_cap.
int plan(tsp_ctx* c);
// Eq. 2, windows and binning of the uploaded events; builds the plain items.
int prepare_events(tsp_ctx* c, cudaStream_t st);
// Tile items (bin, first, count, w) of runs of at most E events, the tiles of
// each run index interleaved.
std::vector<int4> tile_items(const tsp_ctx* c, long long E, int w);
// Events per item for `placed` binned events spread over `sms` SMs.
long long item_events(long long placed, int items_per_sm, int sms);
int ensure_sensitivity(tsp_ctx* c, cudaStream_t st);
int refresh_rhop(tsp_ctx* c, cudaStream_t st);
void clear_graphs(tsp_ctx* c);

}  // namespace tsp_host

#define TSP_CUDA(ctx, call)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return tsp_host::fail((ctx),                                                      \
                                  e_ == cudaErrorMemoryAllocation ? TSP_ENOMEM : TSP_ECUDA,   \
                                  std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)
