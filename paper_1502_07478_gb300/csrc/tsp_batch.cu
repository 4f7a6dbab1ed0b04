// libtsp batched entry points: many independent reconstructions advanced
// together.  Each reconstruction keeps its own context (geometry, resolution,
// grid, events, images); the batch adds a device table of their Inst records,
// merged lists of work items, and CUDA graphs in which an iteration of Eq. iter
// is a reset of the pass accumulators, persistent tile passes over the items of
// all reconstructions, and the per-pixel update of all images -- whatever the
// batch size.  The reconstructions are grouped by the tile kernel their
// windows need (lane capacity and row split, which also fix its block size):
// one persistent launch per group present (plus the batched outlier kernel when
// some events need it).  The tile schedule (tile height, items per SM, item
// order) is chosen by a measuring autotuner.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "tsp_ctx.h"

using namespace tsp;
using namespace tsp_host;

// The reconstructions of a batch that share one tile kernel (lane capacity
// lmax, row split nseg): their merged work items and outlier items.
struct BatchClass {
    int lmax = 0, nseg = 1;
    bool kz = false;           // some member has a z-dependent sigma_z
    size_t smem = 0;
    double work = 0.0;         // estimated pass work (events x window pixels)
    int4* items = nullptr;
    int4* oitems = nullptr;
    int n_items = 0, n_oitems = 0, items_cap = 0, oitems_cap = 0;
};

constexpr int kMaxClasses = 2 * kLmaxCount;

struct tsp_batch {
    std::vector<tsp_ctx*> inst;
    int dev = 0, num_sms = 0;
    Schedule sched;
    bool dirty = true;
    int max_npix = 0;
    Inst* table = nullptr;
    BatchImg* imgs = nullptr;
    BatchClass cls[kMaxClasses];
    int n_cls = 0;
    int* queue = nullptr;       // one work counter per class
    cudaStream_t cap_stream = nullptr;
    // The classes' tile launches run as parallel branches (one stream each,
    // forked from and joined back into the pass's stream), the class with
    // the most work launched first: blocks of a later class take the SMs that
    // an earlier class's blocks leave at the end of their queue, instead of
    // each launch ending in its own tail.
    cudaStream_t cls_stream[kMaxClasses] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kMaxClasses] = {};
    int cls_order[kMaxClasses] = {};
    std::map<int, tsp_ctx::Graph> graphs;
    int last_graph = -1;
    bool profiling = false;
    long long launches = 0;
    std::string err;
};

namespace {

thread_local std::string g_batch_create_error;

int bfail(tsp_batch* b, int code, const std::string& msg)
{
    if (b) b->err = msg;
    else g_batch_create_error = msg;
    return code;
}

// A failed call on reconstruction i: carry its message over.
int bfail_inst(tsp_batch* b, int i, int code)
{
    return bfail(b, code, "reconstruction " + std::to_string(i) + ": " + b->inst[i]->err);
}

#define BATCH_CUDA(b, call)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? TSP_ENOMEM : TSP_ECUDA,       \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

void clear_batch_graphs(tsp_batch* b)
{
    for (auto& kv : b->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        for (cudaEvent_t e : kv.second.ev) cudaEventDestroy(e);
    }
    b->graphs.clear();
    b->last_graph = -1;
}

int check_index(tsp_batch* b, int i)
{
    if (!b) return bfail(nullptr, TSP_EINVAL, "batch is NULL");
    if (i < 0 || i >= (int)b->inst.size())
        return bfail(b, TSP_EINVAL, "reconstruction index out of range");
    return TSP_OK;
}

int validate_schedule(tsp_batch* b, const tsp_schedule* s)
{
    if (!s) return bfail(b, TSP_EINVAL, "schedule is NULL");
    if (!schedule_valid(*s)) return bfail(b, TSP_EINVAL, TSP_SCHEDULE_RANGES);
    return TSP_OK;
}

// Mean in-window pixels per event of reconstruction c: the cut ellipse has
// area pi cut^2 sigma_z sigma_dl cos / sqrt(8) (mean cos about 0.9).
double window_pixels(const tsp_ctx* c)
{
    const double cut = c->p.cut > 0 ? c->p.cut : 3.0;
    return 3.14159265358979 * cut * cut * c->p.sigma_z * c->p.sigma_dl * 0.9 /
           (std::sqrt(8.0) * c->g.dy * c->g.dz);
}

// Lane capacity, rows per lane and shared memory of the batched kernel, the
// Inst table, and the merged, ordered item lists.
int rebuild(tsp_batch* b, cudaStream_t st)
{
    const int k = (int)b->inst.size();
    for (int i = 0; i < k; ++i)
        if (!b->inst[i]->uploaded)
            return bfail(b, TSP_ESTATE,
                         "reconstruction " + std::to_string(i) + " has no uploaded events");
    std::vector<Inst> table(k);
    std::vector<BatchImg> imgs(k);
    int max_npix = 0;
    long long placed = 0;
    // kernel class of every reconstruction: its own lane capacity and row split
    int n_cls = 0;
    int cls_lmax[kMaxClasses], cls_nseg[kMaxClasses];
    std::vector<int> cls_of(k);
    for (int i = 0; i < k; ++i) {
        tsp_ctx* c = b->inst[i];
        int q = 0;
        while (q < n_cls && !(cls_lmax[q] == c->lmax && cls_nseg[q] == c->nseg)) ++q;
        if (q == n_cls) {
            cls_lmax[q] = c->lmax;
            cls_nseg[q] = c->nseg;
            ++n_cls;
        }
        cls_of[i] = q;
        Inst& t = table[i];
        std::memset(&t, 0, sizeof(Inst));
        t.g = c->g;
        t.tl = c->tl;
        t.evs.geo = c->geo;
        t.evs.geo64 = c->geo64;
        t.evs.rows = c->rows;
        t.rhop = c->rhop;
        t.A = c->A;
        t.accum = c->accum;
        t.G = c->G;
        BatchImg& m = imgs[i];
        m.rho = c->rho;
        m.rhop = c->rhop;
        m.A = c->A;
        m.s = c->s;
        m.g = c->gbuf;
        m.accum = c->accum;
        m.npix = c->npix;
        m.pad = 0;
        max_npix = std::max(max_npix, c->npix);
        if (!c->bin_cnt.empty())
            placed += std::accumulate(c->bin_cnt.begin(), c->bin_cnt.end() - 1, 0ll);
    }
    // items: tile runs of at most E events, E from the whole batch's load
    const long long E = item_events(placed, b->sched.items_per_sm, b->num_sms);
    const size_t limit = dyn_smem_limit(b->dev);
    for (int q = 0; q < n_cls; ++q) {
        BatchClass& bc = b->cls[q];
        bc.lmax = cls_lmax[q];
        bc.nseg = cls_nseg[q];
        bc.kz = false;
        bc.smem = 0;
        bc.work = 0.0;
        std::vector<std::vector<int4>> lists;
        std::vector<int> members;
        std::vector<int4> outl;
        for (int i = 0; i < k; ++i) {
            if (cls_of[i] != q) continue;
            const tsp_ctx* c = b->inst[i];
            bc.smem = std::max(bc.smem, c->smem);
            if (c->p.kappa_z != 0.0) bc.kz = true;
            members.push_back(i);
            // a reconstruction whose tiles stage only the accumulator is not
            // supported by the batched tile kernel: all its events take the
            // batched global-memory path
            long long first = c->outlier_first, count = c->n_outliers;
            if (c->gld) {
                first = 0;
                count = c->outlier_first + c->n_outliers;
                lists.emplace_back();
            } else {
                lists.push_back(tile_items(c, E, i));
            }
            for (long long j = 0; j < count; j += 64)
                outl.push_back(make_int4(-1, (int)(first + j),
                                         (int)std::min<long long>(64, count - j), i));
        }
        std::vector<int4> items;
        if (b->sched.order == 0) {
            // longest estimated item first: events x window pixels, plus the
            // staging of the item's region
            std::vector<std::pair<double, int4>> cost;
            for (size_t m = 0; m < members.size(); ++m) {
                const tsp_ctx* c = b->inst[members[m]];
                const double w = window_pixels(c);
                const double stage = 0.25 * c->tl.RH * c->tl.RS;
                for (const int4& it : lists[m]) cost.emplace_back(it.z * w + stage, it);
            }
            for (const auto& x : cost) bc.work += x.first;
            std::stable_sort(cost.begin(), cost.end(),
                             [](const auto& x, const auto& y) { return x.first > y.first; });
            items.reserve(cost.size());
            for (const auto& x : cost) items.push_back(x.second);
        } else {
            for (size_t j = 0;; ++j) {
                bool any = false;
                for (const auto& l : lists)
                    if (j < l.size()) {
                        items.push_back(l[j]);
                        any = true;
                    }
                if (!any) break;
            }
            for (size_t m = 0; m < members.size(); ++m) {
                const tsp_ctx* c = b->inst[members[m]];
                for (const int4& it : lists[m]) bc.work += it.z * window_pixels(c);
            }
        }
        for (const int4& it : outl) bc.work += it.z * window_pixels(b->inst[it.w]);
        if (bc.smem > limit) return bfail(b, TSP_EINVAL, "tile region exceeds the shared memory");
        BATCH_CUDA(b, prepare_batch_pass(bc.lmax, limit));
        if ((int)items.size() > bc.items_cap) {
            dfree(bc.items);
            BATCH_CUDA(b, dmalloc(&bc.items, sizeof(int4) * items.size()));
            bc.items_cap = (int)items.size();
        }
        if ((int)outl.size() > bc.oitems_cap) {
            dfree(bc.oitems);
            BATCH_CUDA(b, dmalloc(&bc.oitems, sizeof(int4) * outl.size()));
            bc.oitems_cap = (int)outl.size();
        }
        if (!items.empty())
            BATCH_CUDA(b, cudaMemcpyAsync(bc.items, items.data(), sizeof(int4) * items.size(),
                                          cudaMemcpyHostToDevice, st));
        if (!outl.empty())
            BATCH_CUDA(b, cudaMemcpyAsync(bc.oitems, outl.data(), sizeof(int4) * outl.size(),
                                          cudaMemcpyHostToDevice, st));
        bc.n_items = (int)items.size();
        bc.n_oitems = (int)outl.size();
        BATCH_CUDA(b, cudaStreamSynchronize(st));   // the host vectors go out of scope
    }
    BATCH_CUDA(b, cudaMemcpyAsync(b->table, table.data(), sizeof(Inst) * k,
                                  cudaMemcpyHostToDevice, st));
    BATCH_CUDA(b, cudaMemcpyAsync(b->imgs, imgs.data(), sizeof(BatchImg) * k,
                                  cudaMemcpyHostToDevice, st));
    BATCH_CUDA(b, cudaStreamSynchronize(st));
    b->n_cls = n_cls;
    for (int q = 0; q < n_cls; ++q) b->cls_order[q] = q;
    std::stable_sort(b->cls_order, b->cls_order + n_cls,
                     [b](int x, int y) { return b->cls[x].work > b->cls[y].work; });
    b->max_npix = max_npix;
    clear_batch_graphs(b);
    b->dirty = false;
    return TSP_OK;
}

BatchArgs batch_args(const tsp_batch* b, int q)
{
    const BatchClass& bc = b->cls[q];
    BatchArgs a;
    a.table = b->table;
    a.items = bc.items;
    a.n_items = bc.n_items;
    a.outlier_items = bc.oitems;
    a.n_outlier_items = bc.n_oitems;
    a.queue = b->queue + q;
    a.nseg = bc.nseg;
    a.kz = bc.kz ? 1 : 0;
    a.grid = b->num_sms;
    a.smem = bc.smem;
    return a;
}

long long batch_pass_launches(const tsp_batch* b)
{
    long long n = 0;
    for (int q = 0; q < b->n_cls; ++q)
        n += (b->cls[q].n_items > 0 ? 1 : 0) + (b->cls[q].n_oitems > 0 ? 1 : 0);
    return n;
}

// One batched pass (MODE kMlem or kGrad): the tile passes of every class, as
// parallel branches forked from and joined back into st (also inside a
// stream capture), largest estimated work first.
cudaError_t launch_batch_passes(const tsp_batch* b, int mode, cudaStream_t st)
{
    if (b->n_cls == 1) return launch_batch_pass(b->cls[0].lmax, mode, batch_args(b, 0), st);
    cudaError_t e = cudaEventRecord(b->fork_ev, st);
    for (int j = 0; j < b->n_cls && e == cudaSuccess; ++j) {
        const int q = b->cls_order[j];
        cudaStream_t cs = b->cls_stream[j];
        e = cudaStreamWaitEvent(cs, b->fork_ev, 0);
        if (e == cudaSuccess) e = launch_batch_pass(b->cls[q].lmax, mode, batch_args(b, q), cs);
        if (e == cudaSuccess) e = cudaEventRecord(b->join_ev[j], cs);
    }
    for (int j = 0; j < b->n_cls && e == cudaSuccess; ++j)
        e = cudaStreamWaitEvent(st, b->join_ev[j], 0);
    return e;
}

int capture_batch(tsp_batch* b, int n_iter, tsp_ctx::Graph* out)
{
    cudaStream_t cs = b->cap_stream;
    const int k = (int)b->inst.size();
    std::vector<cudaEvent_t> ev;
    if (b->profiling) {
        ev.resize(2 * (size_t)n_iter, nullptr);
        for (auto& x : ev) BATCH_CUDA(b, cudaEventCreate(&x));
    }
    cudaGraph_t graph = nullptr;
    BATCH_CUDA(b, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < n_iter && e == cudaSuccess; ++it) {
        e = launch_batch_begin(b->imgs, k, b->queue, b->n_cls, cs);
        if (e == cudaSuccess && b->profiling)
            e = cudaEventRecordWithFlags(ev[2 * it], cs, cudaEventRecordExternal);
        if (e == cudaSuccess) e = launch_batch_passes(b, kMlem, cs);
        if (e == cudaSuccess && b->profiling)
            e = cudaEventRecordWithFlags(ev[2 * it + 1], cs, cudaEventRecordExternal);
        if (e == cudaSuccess) e = launch_batch_pixels(b->imgs, k, b->max_npix, 0, cs);
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        for (cudaEvent_t x : ev) cudaEventDestroy(x);
        return bfail(b, TSP_ECUDA, std::string("graph capture: ") +
                                       cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        for (cudaEvent_t x : ev) cudaEventDestroy(x);
        return bfail(b, TSP_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    out->exec = exec;
    out->launches = (long long)n_iter * (2 + batch_pass_launches(b));
    out->ev = std::move(ev);
    return TSP_OK;
}

// Apply a schedule to every reconstruction: a new tile height re-plans and
// re-bins the events; the item split and order only change the merged items.
int apply_schedule(tsp_batch* b, const tsp_schedule* s, cudaStream_t st)
{
    const bool replan = s->ty_cap != b->sched.ty_cap;
    b->sched.ty_cap = s->ty_cap;
    b->sched.items_per_sm = s->items_per_sm;
    b->sched.order = s->order;
    for (int i = 0; i < (int)b->inst.size(); ++i) {
        tsp_ctx* c = b->inst[i];
        c->sched = b->sched;
        if (replan) {
            int rc = plan(c);
            if (rc) return bfail_inst(b, i, rc);
            if (c->uploaded && (rc = prepare_events(c, st))) return bfail_inst(b, i, rc);
        }
    }
    b->dirty = true;
    return TSP_OK;
}

// Time of one batched MLEM pass (best of `reps`), leaving the images as they
// were: the back-projections are cleared and rho' re-summed afterwards.
int time_batch_pass(tsp_batch* b, int reps, float* ms, cudaStream_t st)
{
    if (b->dirty) {
        int rc = rebuild(b, st);
        if (rc) return rc;
    }
    const int k = (int)b->inst.size();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BATCH_CUDA(b, cudaEventCreate(&e0));
    BATCH_CUDA(b, cudaEventCreate(&e1));
    float best = 1e30f;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = launch_batch_begin(b->imgs, k, b->queue, b->n_cls, st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = launch_batch_passes(b, kMlem, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = launch_batch_pixels(b->imgs, k, b->max_npix, 3, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        best = std::min(best, t);
        b->launches += 3 + batch_pass_launches(b);
    }
    if (e == cudaSuccess) e = launch_batch_pixels(b->imgs, k, b->max_npix, 1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BATCH_CUDA(b, e);
    *ms = best;
    return TSP_OK;
}

}  // namespace

extern "C" {

const char* tsp_batch_last_error(const tsp_batch* b)
{
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

int tsp_batch_create(const tsp_params* params, int k, tsp_batch** out)
{
    if (!out) return bfail(nullptr, TSP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || k <= 0) return bfail(nullptr, TSP_EINVAL, "need k >= 1 parameter sets");
    if (k > (1 << 20)) return bfail(nullptr, TSP_EINVAL, "k > 2^20");
    for (int i = 0; i < k; ++i)
        if (int rc = validate(&params[i], nullptr))
            return bfail(nullptr, rc,
                         "reconstruction " + std::to_string(i) + ": " + tsp_last_error(nullptr));
    tsp_batch* b = new tsp_batch();
    auto bail = [&](int code) {
        g_batch_create_error = b->err;
        tsp_batch_destroy(b);
        return code;
    };
    if (cudaGetDevice(&b->dev) != cudaSuccess) {
        b->err = "no CUDA device";
        return bail(TSP_ECUDA);
    }
    if (cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->dev) !=
            cudaSuccess ||
        b->num_sms <= 0) {
        cudaGetLastError();
        b->err = "cudaDeviceGetAttribute(MultiProcessorCount) failed";
        return bail(TSP_ECUDA);
    }
    b->inst.reserve(k);
    for (int i = 0; i < k; ++i) {
        tsp_ctx* c = nullptr;
        int rc = tsp_create(&params[i], &c);
        if (rc) {
            b->err = "reconstruction " + std::to_string(i) + ": " + tsp_last_error(nullptr);
            return bail(rc);
        }
        b->inst.push_back(c);
        c->sched = b->sched;
    }
    cudaError_t e = dmalloc(&b->table, sizeof(Inst) * k);
    if (e == cudaSuccess) e = dmalloc(&b->imgs, sizeof(BatchImg) * k);
    if (e == cudaSuccess) e = dmalloc(&b->queue, sizeof(int) * kMaxClasses);
    if (e == cudaSuccess) e = cudaMemset(b->queue, 0, sizeof(int) * kMaxClasses);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
    for (int q = 0; q < kMaxClasses && e == cudaSuccess; ++q) {
        e = cudaStreamCreateWithFlags(&b->cls_stream[q], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[q], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        b->err = std::string("tsp_batch_create: ") + cudaGetErrorString(e);
        return bail(e == cudaErrorMemoryAllocation ? TSP_ENOMEM : TSP_ECUDA);
    }
    *out = b;
    return TSP_OK;
}

void tsp_batch_destroy(tsp_batch* b)
{
    if (!b) return;
    DeviceGuard dg(b->dev);
    cudaDeviceSynchronize();
    clear_batch_graphs(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    for (int q = 0; q < kMaxClasses; ++q) {
        if (b->cls_stream[q]) cudaStreamDestroy(b->cls_stream[q]);
        if (b->join_ev[q]) cudaEventDestroy(b->join_ev[q]);
    }
    dfree(b->table);
    dfree(b->imgs);
    for (BatchClass& bc : b->cls) {
        dfree(bc.items);
        dfree(bc.oitems);
    }
    dfree(b->queue);
    for (tsp_ctx* c : b->inst) tsp_destroy(c);
    delete b;
}

int tsp_batch_size(const tsp_batch* b) { return b ? (int)b->inst.size() : 0; }

int tsp_batch_upload_events(tsp_batch* b, int i, const float* zu, const float* zd,
                            const float* dl, int64_t n, int on_device, void* stream)
{
    NvtxRange nvtx_("tsp_batch_upload_events");
    int rc = check_index(b, i);
    if (rc) return rc;
    b->dirty = true;
    if ((rc = tsp_upload_events(b->inst[i], zu, zd, dl, n, on_device, stream)))
        return bfail_inst(b, i, rc);
    return TSP_OK;
}

int tsp_batch_set_image(tsp_batch* b, int i, const float* rho, int on_device, void* stream)
{
    int rc = check_index(b, i);
    if (rc) return rc;
    if ((rc = tsp_set_image(b->inst[i], rho, on_device, stream))) return bfail_inst(b, i, rc);
    return TSP_OK;
}

int tsp_batch_set_sigma(tsp_batch* b, int i, double sigma_z, double sigma_dl, void* stream)
{
    int rc = check_index(b, i);
    if (rc) return rc;
    b->dirty = true;
    if ((rc = tsp_set_sigma(b->inst[i], sigma_z, sigma_dl, stream))) return bfail_inst(b, i, rc);
    return TSP_OK;
}

int tsp_batch_iterate(tsp_batch* b, int n_iter, void* stream)
{
    NvtxRange nvtx_("tsp_batch_iterate");
    if (!b) return bfail(nullptr, TSP_EINVAL, "batch is NULL");
    if (n_iter < 0) return bfail(b, TSP_EINVAL, "n_iter < 0");
    DeviceGuard dg(b->dev);
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if (b->dirty && (rc = rebuild(b, st))) return rc;
    if (n_iter == 0) return TSP_OK;
    auto it = b->graphs.find(n_iter);
    if (it == b->graphs.end()) {
        tsp_ctx::Graph gr;
        if ((rc = capture_batch(b, n_iter, &gr))) return rc;
        it = b->graphs.emplace(n_iter, std::move(gr)).first;
    }
    BATCH_CUDA(b, cudaGraphLaunch(it->second.exec, st));
    b->launches += it->second.launches;
    b->last_graph = n_iter;
    for (tsp_ctx* c : b->inst) c->iterations += n_iter;
    return TSP_OK;
}

int tsp_batch_read_image(tsp_batch* b, int i, float* out, int which, int on_device, void* stream)
{
    NvtxRange nvtx_("tsp_batch_read_image");
    int rc = check_index(b, i);
    if (rc) return rc;
    if (which == 2) {
        if (!out) return bfail(b, TSP_EINVAL, "out is NULL");
        tsp_ctx* c = b->inst[i];
        DeviceGuard dg(b->dev);
        cudaStream_t st = (cudaStream_t)stream;
        BATCH_CUDA(b, cudaMemcpyAsync(out, c->gbuf, sizeof(float) * c->npix,
                                      on_device ? cudaMemcpyDeviceToDevice
                                                : cudaMemcpyDeviceToHost,
                                      st));
        if (!on_device) BATCH_CUDA(b, cudaStreamSynchronize(st));
        return TSP_OK;
    }
    if ((rc = tsp_read_image(b->inst[i], out, which, on_device, stream)))
        return bfail_inst(b, i, rc);
    return TSP_OK;
}

int tsp_batch_loglik_grad(tsp_batch* b, double* L_out, double* g_sigma, void* stream)
{
    NvtxRange nvtx_("tsp_batch_loglik_grad");
    if (!b) return bfail(nullptr, TSP_EINVAL, "batch is NULL");
    DeviceGuard dg(b->dev);
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if (b->dirty && (rc = rebuild(b, st))) return rc;
    const int k = (int)b->inst.size();
    BATCH_CUDA(b, launch_batch_begin(b->imgs, k, b->queue, b->n_cls, st));
    BATCH_CUDA(b, launch_batch_pixels(b->imgs, k, b->max_npix, 1, st));
    BATCH_CUDA(b, launch_batch_passes(b, kGrad, st));
    BATCH_CUDA(b, launch_batch_pixels(b->imgs, k, b->max_npix, 2, st));
    b->launches += 3 + batch_pass_launches(b);
    std::vector<Accum> h(k);
    for (int i = 0; i < k; ++i)
        BATCH_CUDA(b, cudaMemcpyAsync(&h[i], b->inst[i]->accum, sizeof(Accum),
                                      cudaMemcpyDeviceToHost, st));
    BATCH_CUDA(b, cudaStreamSynchronize(st));
    for (int i = 0; i < k; ++i) {
        if (L_out) L_out[i] = h[i].sum_logD - h[i].sum_rhop;
        if (g_sigma) {
            const double sz = b->inst[i]->p.sigma_z, sl = b->inst[i]->p.sigma_dl;
            g_sigma[2 * i] = h[i].g_iz * (-2.0 / (sz * sz * sz));
            g_sigma[2 * i + 1] = h[i].g_il * (-2.0 / (sl * sl * sl));
        }
    }
    return TSP_OK;
}

int tsp_batch_stats(tsp_batch* b, int i, tsp_stats_t* out, void* stream)
{
    int rc = check_index(b, i);
    if (rc) return rc;
    if ((rc = tsp_stats(b->inst[i], out, stream))) return bfail_inst(b, i, rc);
    out->launches = b->launches;
    return TSP_OK;
}

int tsp_batch_get_schedule(tsp_batch* b, tsp_schedule* out)
{
    if (!b) return bfail(nullptr, TSP_EINVAL, "batch is NULL");
    if (!out) return bfail(b, TSP_EINVAL, "out is NULL");
    out->ty_cap = b->sched.ty_cap;
    out->items_per_sm = b->sched.items_per_sm;
    out->order = b->sched.order;
    out->reserved = 0;
    return TSP_OK;
}

int tsp_batch_set_schedule(tsp_batch* b, const tsp_schedule* s, void* stream)
{
    if (!b) return bfail(nullptr, TSP_EINVAL, "batch is NULL");
    int rc = validate_schedule(b, s);
    if (rc) return rc;
    DeviceGuard dg(b->dev);
    return apply_schedule(b, s, (cudaStream_t)stream);
}

int tsp_batch_autotune(tsp_batch* b, tsp_schedule* chosen, float* best_ms, void* stream)
{
    if (!b) return bfail(nullptr, TSP_EINVAL, "batch is NULL");
    DeviceGuard dg(b->dev);
    cudaStream_t st = (cudaStream_t)stream;
    tsp_schedule best{b->sched.ty_cap, b->sched.items_per_sm, b->sched.order, 0};
    float best_t = 0.0f;
    int rc = time_batch_pass(b, 2, &best_t, st);
    if (rc) return rc;
    auto trial = [&](tsp_schedule s) -> int {
        int r = apply_schedule(b, &s, st);
        float t = 0.0f;
        if (!r) r = time_batch_pass(b, 2, &t, st);
        if (r) return r;
        if (t < best_t) {
            best_t = t;
            best = s;
        }
        return TSP_OK;
    };
    // coordinate descent: item order, then items per SM, then tile height
    for (int order : {0, 1}) {
        tsp_schedule s = best;
        s.order = order;
        if (s.order != best.order && (rc = trial(s))) return rc;
    }
    for (int ips : {2, 4, 8, 16, 32}) {
        tsp_schedule s = best;
        s.items_per_sm = ips;
        if (s.items_per_sm != best.items_per_sm && (rc = trial(s))) return rc;
    }
    for (int ty : {16, 32, 64, 128}) {
        tsp_schedule s = best;
        s.ty_cap = ty;
        if (s.ty_cap != best.ty_cap && (rc = trial(s))) return rc;
    }
    if ((rc = apply_schedule(b, &best, st))) return rc;
    if ((rc = rebuild(b, st))) return rc;
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = best_t;
    return TSP_OK;
}

int tsp_batch_set_profiling(tsp_batch* b, int on)
{
    if (!b) return bfail(nullptr, TSP_EINVAL, "batch is NULL");
    DeviceGuard dg(b->dev);
    if ((bool)on != b->profiling) {
        BATCH_CUDA(b, cudaDeviceSynchronize());
        clear_batch_graphs(b);
        b->profiling = on != 0;
    }
    return TSP_OK;
}

int tsp_batch_pass_times(tsp_batch* b, float* ms, int max, int* count, void* stream)
{
    if (!b) return bfail(nullptr, TSP_EINVAL, "batch is NULL");
    if (!count || (max > 0 && !ms)) return bfail(b, TSP_EINVAL, "NULL output");
    *count = 0;
    DeviceGuard dg(b->dev);
    auto it = b->graphs.find(b->last_graph);
    if (it == b->graphs.end() || it->second.ev.empty()) return TSP_OK;
    BATCH_CUDA(b, cudaStreamSynchronize((cudaStream_t)stream));
    const auto& ev = it->second.ev;
    const int n = std::min<int>(max, (int)(ev.size() / 2));
    for (int q = 0; q < n; ++q)
        BATCH_CUDA(b, cudaEventElapsedTime(&ms[q], ev[2 * q], ev[2 * q + 1]));
    *count = n;
    return TSP_OK;
}

}  // extern "C"
