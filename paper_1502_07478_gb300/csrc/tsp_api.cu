// libtsp host side: the C ABI declared in include/tsp.h.
//
// A context owns the image buffers (rho, rho' = s rho, the back-projection
// accumulator A, the sensitivity s), the uploaded events and their prepared,
// binned form, and a cache of CUDA graphs that replay n iterations of
// Eq. iter.  Every entry point validates its arguments, runs on the context's
// device, and reports failures through return codes and tsp_last_error().
#include <algorithm>
#include <chrono>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "tsp_ctx.h"

using namespace tsp;

namespace tsp_host {

thread_local std::string g_create_error;

int fail(tsp_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    else g_create_error = msg;
    return code;
}

void clear_graphs(tsp_ctx* c)
{
    for (auto& kv : c->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        for (cudaEvent_t e : kv.second.ev) cudaEventDestroy(e);
    }
    c->graphs.clear();
    c->last_graph = -1;
}

// Kernel launches made by one MLEM/loglik/gradient pass.
long long pass_launches(const tsp_ctx* c)
{
    return (c->n_items > 0 ? 1 : 0) + (c->n_outliers > 0 ? 1 : 0);
}

// One MLEM pass of the context's variant.
cudaError_t launch_mlem_pass(tsp_ctx* c, const PassArgs& a, cudaStream_t st)
{
    if (c->variant == 1)
        return launch_thread_pass(c->g, a.evs, (int)(c->outlier_first + c->n_outliers), c->rhop,
                                  c->A, c->accum, c->num_sms, st);
    return launch_pass(c->lmax, kMlem, a, st);
}

long long mlem_pass_launches(const tsp_ctx* c)
{
    if (c->variant == 1) return c->outlier_first + c->n_outliers > 0 ? 1 : 0;
    return pass_launches(c);
}

size_t dyn_smem_limit(int dev)
{
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess ||
        optin <= 0)
        optin = 227 * 1024;
    return (size_t)optin - 2048;    // room for the kernels' static shared memory
}

// Derive the kernel constants, lane capacity, group size and tiling from the
// parameters.  Returns TSP_OK or TSP_EINVAL.
int plan(tsp_ctx* c)
{
    const tsp_params& p = c->p;
    const double dy = p.dy > 0 ? p.dy : 2.0 * p.R / p.ny;
    const double dz = p.dz > 0 ? p.dz : p.L / p.nz;
    const double cut = p.cut > 0 ? p.cut : 3.0;
    c->g = make_geo(p);

    // lane capacity, row split, rows per window and warps per event (shared
    // with the allocation-free entry point)
    LanePlan lp;
    if (const char* why = lane_plan(p, lp)) return fail(c, TSP_EINVAL, why);
    c->lmax = lp.lmax;
    c->nseg = lp.nseg;
    c->need = lp.need;
    c->maxrows = lp.maxrows;
    c->G = lp.G;
    const int need = lp.need, maxrows = lp.maxrows;
    const double szmax = p.sigma_z * (1.0 + p.kappa_z);
    const double umax = cut * szmax / std::sqrt(2.0);
    const double hy = cut * p.sigma_dl / 2.0 * 1.00001;

    // tiling (see Tiling): angle bins of width 1/16 in tan(theta~) cover the
    // accepted range |t| <= L/2R widened by 6 sigma of its measurement noise
    // (sqrt(2) sigma_z / 2R); events outside go to the outlier path.
    Tiling& tl = c->tl;
    const double dtb = 1.0 / 16.0;
    const double t_max = p.L / (2.0 * p.R) + 6.0 * std::sqrt(2.0) * szmax / (2.0 * p.R);
    tl.nb = (int)std::ceil(2.0 * t_max / dtb);
    tl.dtb = (float)dtb;
    tl.inv_dtb = (float)(1.0 / dtb);
    tl.t0 = (float)(-0.5 * tl.nb * dtb);
    tl.rho_yz = (float)(dy / dz);
    tl.Y0 = p.ny / 2;
    const double smax = (0.5 * tl.nb * dtb) * (dy / dz);
    tl.zs_off = (int)std::ceil(smax * (p.ny / 2 + 1)) + 1;
    tl.HY = (int)std::ceil(hy / dy) + 1;
    // chord half-width, plus the drift of chord centres from the event's
    // sheared centre column: rounding (1.5), sub-pixel centre (|t| rho / 2) and
    // the in-bin angle spread over the rows ((dtb/2) rho HY)
    const double w = umax / dz;
    tl.HZ = (int)std::ceil(w + 1.5 + 0.5 * t_max * (dy / dz) + 0.5 * dtb * (dy / dz) * tl.HY) + 1;
    int RS = 33;
    while (RS - 2 * tl.HZ < std::min(16, p.nz)) RS += 32;
    tl.RS = RS;
    tl.RW = RS;
    tl.TZ = RS - 2 * tl.HZ;
    const size_t budget = 216 * 1024;
    auto fits = [&](int ty) {
        return tiles_region_fits(ty + 2 * tl.HY, RS) &&
               tiles_smem_floats(ty + 2 * tl.HY, RS) * sizeof(float) <= budget;
    };
    int TY = std::max(4, std::min(128, c->sched.ty_cap) / 4 * 4);
    const int ty0 = TY;
    while (TY > 4 && !fits(TY)) TY -= 4;
    c->gld = 0;
    if (!fits(TY)) {
        // windows too large to stage rho' and the accumulator (very fine
        // grids): stage only the accumulator and read rho' from global memory,
        // with two lanes per row; if even that does not fit, no angle bins, so
        // every event takes the global-memory path
        // rho' is then read through L1, which gets what the shared-memory
        // carve-out leaves of the SM's 256 KB: the accumulator region is kept
        // to ~150 KB (at 0.5 mm a pass with a 147 KB region took 28% less
        // time than with 197 KB)
        const size_t gld_budget = 150 * 1024;
        TY = ty0;
        while (TY > 4 && tiles_acc_smem_floats(TY + 2 * tl.HY, RS) * sizeof(float) > gld_budget)
            TY -= 4;
        if (tiles_acc_smem_floats(TY + 2 * tl.HY, RS) * sizeof(float) <= budget) {
            c->gld = 1;
            const int l2 = lane_lmax_split(need);
            if (!l2) return fail(c, TSP_EINVAL, "window chords too long for the lane capacities");
            c->lmax = l2;
            c->nseg = 2;
            c->G = 2 * ((maxrows + 31) / 32);
            if (c->G > kMinWarps)
                return fail(c, TSP_EINVAL, "window has more rows than one block can hold");
        } else {
            tl.nb = 0;
            TY = 4;
        }
    }
    tl.TY = std::min(TY, std::max(p.ny, 4));
    tl.RH = tl.TY + 2 * tl.HY;
    tl.tiles_y = (p.ny + tl.TY - 1) / tl.TY;
    tl.tiles_z = (p.nz + 2 * tl.zs_off + tl.TZ - 1) / tl.TZ;
    c->smem = tl.nb == 0 ? 0
              : (c->gld ? tiles_acc_smem_floats(tl.RH, tl.RS) : tiles_smem_floats(tl.RH, tl.RS)) *
                    sizeof(float);
    c->nbins = tl.nb * tl.tiles_y * tl.tiles_z + 1;
    // The dynamic shared-memory limit is a property of the kernel function,
    // shared by every context: raise it to the device's opt-in maximum (never
    // to this context's size, which could lower it below another context's).
    const size_t limit = dyn_smem_limit(c->dev);
    if (c->smem > limit) return fail(c, TSP_EINVAL, "tile region exceeds the shared memory");
    for (int mode = 0; mode < 3; ++mode) {
        cudaError_t e = prepare_pass(c->lmax, mode, limit);
        if (e != cudaSuccess)
            return fail(c, TSP_ECUDA, std::string("prepare_pass: ") + cudaGetErrorString(e));
    }
    return TSP_OK;
}

int validate(const tsp_params* p, tsp_ctx* c)
{
    if (!p) return fail(c, TSP_EINVAL, "params is NULL");
    auto pos = [](double v) { return std::isfinite(v) && v > 0.0; };
    if (!pos(p->R) || !pos(p->L)) return fail(c, TSP_EINVAL, "R and L must be finite and > 0");
    if (p->ny <= 0 || p->nz <= 0 || (long long)p->ny * p->nz > (1ll << 30))
        return fail(c, TSP_EINVAL, "ny, nz must be > 0 and ny*nz <= 2^30");
    if (!(p->dy == 0.0 || pos(p->dy)) || !(p->dz == 0.0 || pos(p->dz)))
        return fail(c, TSP_EINVAL, "dy, dz must be 0 or finite and > 0");
    if (!pos(p->sigma_z) || !pos(p->sigma_dl))
        return fail(c, TSP_EINVAL, "sigma_z and sigma_dl must be finite and > 0");
    if (!(p->cut == 0.0 || pos(p->cut))) return fail(c, TSP_EINVAL, "cut must be 0 or > 0");
    if (p->flags != 0) return fail(c, TSP_EINVAL, "flags must be 0");
    if (!cinv_valid(*p))
        return fail(c, TSP_EINVAL,
                    "kappa_z must be in [0, 1] and gamma finite with "
                    "2 gamma^2 < 1/((sigma_z (1 + kappa_z))^2 sigma_dl^2)");
    return TSP_OK;
}

int ensure_sensitivity(tsp_ctx* c, cudaStream_t st)
{
    if (c->sens_ready) return TSP_OK;
    const tsp_params& p = c->p;
    TSP_CUDA(c, launch_sensitivity(p.R, p.L, p.ny, p.nz, (double)c->g.dy, (double)c->g.dz, c->s, st));
    c->launches += 1;
    c->sens_ready = true;
    return TSP_OK;
}

// rho' = s rho and sum s rho (into accum->sum_rhop, after clearing the accumulators)
int refresh_rhop(tsp_ctx* c, cudaStream_t st)
{
    TSP_CUDA(c, launch_begin(c->accum, st));
    TSP_CUDA(c, launch_set_rhop(c->npix, c->rho, c->s, c->rhop, c->accum, st));
    c->launches += 2;
    return TSP_OK;
}

PassArgs pass_args(tsp_ctx* c)
{
    PassArgs a;
    a.g = c->g;
    a.tl = c->tl;
    a.evs.geo = c->geo;
    a.evs.geo64 = c->geo64;
    a.evs.rows = c->rows;
    a.items = c->items;
    a.n_items = c->n_items;
    a.outlier_first = (int)c->outlier_first;
    a.outlier_count = (int)c->n_outliers;
    a.rhop = c->rhop;
    a.A = c->A;
    a.accum = c->accum;
    a.G = c->G;
    a.nseg = c->nseg;
    a.gld = c->gld;
    a.grid = c->num_sms;
    a.smem = c->smem;
    return a;
}

// Prepare the uploaded raw events: Eq. 2, windows, binning, work items.
// Event preparation in three steps, so that an upload can be streamed in
// chunks: clear the bin histogram and counters; per chunk, Eq. 2, windows and
// bin keys (k_setup) for events [first, first + n); then the bin offsets, the
// work items and the counting-sort scatter into binned order.
int prep_begin(tsp_ctx* c, cudaStream_t st)
{
    const int nbins = c->nbins;
    dfree(c->bin_count);
    dfree(c->offsets);
    dfree(c->cursor);
    TSP_CUDA(c, dmalloc(&c->bin_count, sizeof(int) * nbins));
    TSP_CUDA(c, dmalloc(&c->offsets, sizeof(long long) * nbins));
    TSP_CUDA(c, dmalloc(&c->cursor, sizeof(int) * nbins));
    TSP_CUDA(c, cudaMemsetAsync(c->bin_count, 0, sizeof(int) * nbins, st));
    TSP_CUDA(c, cudaMemsetAsync(c->cursor, 0, sizeof(int) * nbins, st));
    TSP_CUDA(c, cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long) * 4, st));
    return TSP_OK;
}

int prep_chunk(tsp_ctx* c, long long first, long long n, cudaStream_t st)
{
    if (n <= 0) return TSP_OK;
    TSP_CUDA(c, launch_setup(c->g, c->tl, n, c->zu + first, c->zd + first, c->dl + first,
                             c->geo_u + first, c->geo64_u + first, c->rows_u + first,
                             c->key + first, c->counters, c->bin_count, c->nbins, st));
    c->launches += 1;
    return TSP_OK;
}

int prep_finish(tsp_ctx* c, cudaStream_t st)
{
    const long long n = c->n;
    const int nbins = c->nbins;
    std::vector<int> cnt(nbins);
    TSP_CUDA(c, cudaMemcpyAsync(c->counters_h, c->counters, sizeof(c->counters_h),
                                cudaMemcpyDeviceToHost, st));
    TSP_CUDA(c, cudaMemcpyAsync(cnt.data(), c->bin_count, sizeof(int) * nbins,
                                cudaMemcpyDeviceToHost, st));
    TSP_CUDA(c, cudaStreamSynchronize(st));
    if (c->counters_h[0] != 0) {
        c->uploaded = false;
        c->n = 0;
        return fail(c, TSP_EINVAL, std::to_string(c->counters_h[0]) + " events are not finite");
    }
    std::vector<long long> off(nbins);
    long long acc = 0;
    for (int b = 0; b < nbins; ++b) {
        off[b] = acc;
        acc += cnt[b];
    }
    c->outlier_first = off[nbins - 1];
    c->n_outliers = cnt[nbins - 1];
    if (acc > (1ll << 31) - 1) return fail(c, TSP_EINVAL, "more than 2^31-1 events");
    c->bin_cnt = std::move(cnt);
    c->bin_off = std::move(off);
    const long long placed = acc - c->n_outliers;
    const std::vector<int4> items =
        tile_items(c, item_events(placed, c->sched.items_per_sm, c->num_sms), 0);
    c->n_items = (int)items.size();
    if (c->n_items > c->items_cap) {
        dfree(c->items);
        TSP_CUDA(c, dmalloc(&c->items, sizeof(int4) * std::max(1, c->n_items)));
        c->items_cap = c->n_items;
    }
    if (c->n_items)
        TSP_CUDA(c, cudaMemcpyAsync(c->items, items.data(), sizeof(int4) * c->n_items,
                                    cudaMemcpyHostToDevice, st));
    TSP_CUDA(c, cudaMemcpyAsync(c->offsets, c->bin_off.data(), sizeof(long long) * nbins,
                                cudaMemcpyHostToDevice, st));
    TSP_CUDA(c, launch_scatter(n, nbins, c->key, c->geo_u, c->geo64_u, c->rows_u, c->offsets,
                               c->cursor, c->geo, c->geo64, c->rows, st));
    c->launches += n > 0 ? 1 : 0;
    clear_graphs(c);
    c->uploaded = true;
    return TSP_OK;
}

int prepare_events(tsp_ctx* c, cudaStream_t st)
{
    int rc = prep_begin(c, st);
    if (!rc) rc = prep_chunk(c, 0, c->n, st);
    if (!rc) rc = prep_finish(c, st);
    return rc;
}

long long item_events(long long placed, int items_per_sm, int sms)
{
    const long long E = placed / ((long long)std::max(1, items_per_sm) * std::max(1, sms));
    return std::max(32ll, std::min((long long)kItemMaxEvents, E));
}

std::vector<int4> tile_items(const tsp_ctx* c, long long E, int w)
{
    // the fixed-point accumulator's sums are exact for items of at most
    // kItemMaxEvents events (tsp_device.cuh)
    E = std::max(1ll, std::min(E, (long long)kItemMaxEvents));
    std::vector<int4> items;
    const int nb = (int)c->bin_cnt.size() - 1;     // the last bin holds the outliers
    for (long long k = 0;; ++k) {
        bool any = false;
        const long long first = k * E;
        for (int b = 0; b < nb; ++b) {
            if (first < c->bin_cnt[b]) {
                any = true;
                items.push_back(make_int4(b, (int)(c->bin_off[b] + first),
                                          (int)std::min<long long>(E, c->bin_cnt[b] - first), w));
            }
        }
        if (!any) break;
    }
    return items;
}

int ensure_event_capacity(tsp_ctx* c, long long n)
{
    if (n <= c->cap) return TSP_OK;
    dfree(c->zu);
    dfree(c->zd);
    dfree(c->dl);
    dfree(c->geo_u);
    dfree(c->geo);
    dfree(c->geo64_u);
    dfree(c->geo64);
    dfree(c->rows_u);
    dfree(c->rows);
    dfree(c->key);
    c->cap = 0;
    TSP_CUDA(c, dmalloc(&c->zu, sizeof(float) * n));
    TSP_CUDA(c, dmalloc(&c->zd, sizeof(float) * n));
    TSP_CUDA(c, dmalloc(&c->dl, sizeof(float) * n));
    TSP_CUDA(c, dmalloc(&c->geo_u, sizeof(float4) * n));
    TSP_CUDA(c, dmalloc(&c->geo, sizeof(float4) * n));
    TSP_CUDA(c, dmalloc(&c->geo64_u, sizeof(Ev64) * n));
    TSP_CUDA(c, dmalloc(&c->geo64, sizeof(Ev64) * n));
    TSP_CUDA(c, dmalloc(&c->rows_u, sizeof(int2) * n));
    TSP_CUDA(c, dmalloc(&c->rows, sizeof(int2) * n));
    TSP_CUDA(c, dmalloc(&c->key, sizeof(int) * n));
    c->cap = n;
    return TSP_OK;
}

int capture_iterations(tsp_ctx* c, int n_iter, tsp_ctx::Graph* out)
{
    cudaStream_t cs = c->cap_stream;
    cudaGraph_t graph = nullptr;
    std::vector<cudaEvent_t> ev;
    if (c->profiling) {
        ev.resize(2 * (size_t)n_iter, nullptr);
        for (auto& x : ev) TSP_CUDA(c, cudaEventCreate(&x));
    }
    TSP_CUDA(c, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const PassArgs a = pass_args(c);
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < n_iter && e == cudaSuccess; ++it) {
        e = launch_begin(c->accum, cs);
        if (e == cudaSuccess && c->profiling)
            e = cudaEventRecordWithFlags(ev[2 * it], cs, cudaEventRecordExternal);
        if (e == cudaSuccess) e = launch_mlem_pass(c, a, cs);
        if (e == cudaSuccess && c->profiling)
            e = cudaEventRecordWithFlags(ev[2 * it + 1], cs, cudaEventRecordExternal);
        if (e == cudaSuccess) e = launch_finalize(c->npix, c->rho, c->rhop, c->A, c->s, c->accum, cs);
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(c, TSP_ECUDA, std::string("graph capture: ") +
                                      cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        for (cudaEvent_t x : ev) cudaEventDestroy(x);
        return fail(c, TSP_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    out->exec = exec;
    out->launches = (long long)n_iter * (2 + mlem_pass_launches(c));
    out->ev = std::move(ev);
    return TSP_OK;
}

int copy_floats(tsp_ctx* c, float* dst, const float* src, size_t n, int dst_dev, int src_dev,
                cudaStream_t st)
{
    if (n == 0) return TSP_OK;
    cudaMemcpyKind k = dst_dev ? (src_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice)
                               : (src_dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
    TSP_CUDA(c, cudaMemcpyAsync(dst, src, n * sizeof(float), k, st));
    return TSP_OK;
}

}  // namespace tsp_host

using namespace tsp_host;

extern "C" {

const char* tsp_version(void) { return "tsp 0.1 sm_103a"; }

const char* tsp_last_error(const tsp_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int tsp_create(const tsp_params* params, tsp_ctx** out)
{
    if (!out) return fail(nullptr, TSP_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(params, nullptr);
    if (rc) return rc;
    tsp_ctx* c = new tsp_ctx();
    c->p = *params;
    auto bail = [&](int code) {
        g_create_error = c->err;
        tsp_destroy(c);
        return code;
    };
    if (cudaGetDevice(&c->dev) != cudaSuccess) {
        c->err = "no CUDA device";
        return bail(TSP_ECUDA);
    }
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev) !=
            cudaSuccess ||
        c->num_sms <= 0) {
        cudaGetLastError();
        c->err = "cudaDeviceGetAttribute(MultiProcessorCount) failed";
        return bail(TSP_ECUDA);
    }
    if ((rc = plan(c))) return bail(rc);
    c->npix = params->ny * params->nz;
    const size_t img = sizeof(float) * (size_t)c->npix;
    const size_t padded = img + sizeof(float) * kPadFloats;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dmalloc(&c->rho, img);
    if (e == cudaSuccess) e = dmalloc(&c->rhop, padded);
    if (e == cudaSuccess) e = dmalloc(&c->A, padded);
    if (e == cudaSuccess) e = dmalloc(&c->s, img);
    if (e == cudaSuccess) e = dmalloc(&c->gbuf, img);
    if (e == cudaSuccess) e = dmalloc(&c->accum, sizeof(Accum));
    if (e == cudaSuccess) e = dmalloc(&c->counters, sizeof(unsigned long long) * 4);
    if (e == cudaSuccess) e = dmalloc(&c->flag, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->copy_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->wait_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemset(c->rhop, 0, padded);
    if (e == cudaSuccess) e = cudaMemset(c->A, 0, padded);
    if (e == cudaSuccess) e = cudaMemset(c->accum, 0, sizeof(Accum));
    if (e == cudaSuccess) e = launch_fill(c->rho, c->npix, 1.0f, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        c->err = std::string("tsp_create: ") + cudaGetErrorString(e);
        return bail(e == cudaErrorMemoryAllocation ? TSP_ENOMEM : TSP_ECUDA);
    }
    *out = c;
    return TSP_OK;
}

void tsp_destroy(tsp_ctx* c)
{
    if (!c) return;
    DeviceGuard dg(c->dev);
    cudaDeviceSynchronize();
    clear_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->copy_ev) cudaEventDestroy(c->copy_ev);
    if (c->wait_ev) cudaEventDestroy(c->wait_ev);
    dfree(c->rho); dfree(c->rhop); dfree(c->A); dfree(c->s); dfree(c->gbuf);
    dfree(c->accum); dfree(c->counters); dfree(c->flag);
    dfree(c->zu); dfree(c->zd); dfree(c->dl);
    dfree(c->geo_u); dfree(c->geo); dfree(c->geo64_u); dfree(c->geo64);
    dfree(c->rows_u); dfree(c->rows); dfree(c->key);
    dfree(c->items); dfree(c->bin_count); dfree(c->offsets); dfree(c->cursor);
    delete c;
}

int tsp_begin_events(tsp_ctx* c, int64_t n_total, void* stream)
{
    NvtxRange nvtx_("tsp_begin_events");
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (n_total < 0) return fail(c, TSP_EINVAL, "n_total < 0");
    if (n_total > (1ll << 31) - 1) return fail(c, TSP_EINVAL, "more than 2^31-1 events");
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    c->uploaded = false;
    c->appending = false;
    clear_graphs(c);
    // work already queued on the stream (a previous preparation reading the
    // raw event buffers) finishes before the copy stream overwrites them
    TSP_CUDA(c, cudaEventRecord(c->copy_ev, st));
    TSP_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->copy_ev, 0));
    if ((rc = ensure_event_capacity(c, std::max<long long>(n_total, 1)))) return rc;
    if ((rc = prep_begin(c, st))) return rc;
    c->n = 0;
    c->n_total = n_total;
    c->appending = true;
    return TSP_OK;
}

int tsp_append_events(tsp_ctx* c, const float* zu, const float* zd, const float* dl, int64_t n,
                      int on_device, void* stream)
{
    NvtxRange nvtx_("tsp_append_events");
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (!c->appending) return fail(c, TSP_ESTATE, "append_events without begin_events");
    if (n < 0) return fail(c, TSP_EINVAL, "n < 0");
    if (n > 0 && (!zu || !zd || !dl)) return fail(c, TSP_EINVAL, "event pointer is NULL");
    if (n > c->n_total - c->n) return fail(c, TSP_EINVAL, "more events than begin_events declared");
    if (n == 0) return TSP_OK;
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    const long long first = c->n;
    // host chunks are copied on the context's copy stream, so that the copy of
    // the next chunk overlaps the preparation of this one
    cudaStream_t cs = on_device ? st : c->copy_stream;
    int rc;
    if ((rc = copy_floats(c, c->zu + first, zu, n, 1, on_device, cs))) return rc;
    if ((rc = copy_floats(c, c->zd + first, zd, n, 1, on_device, cs))) return rc;
    if ((rc = copy_floats(c, c->dl + first, dl, n, 1, on_device, cs))) return rc;
    if (!on_device) {
        TSP_CUDA(c, cudaEventRecord(c->copy_ev, cs));
        TSP_CUDA(c, cudaStreamWaitEvent(st, c->copy_ev, 0));
    }
    if (sim_fault() == kSimNan)   // simulated corrupt input: a NaN in the first z_u
        TSP_CUDA(c, cudaMemsetAsync(c->zu + first, 0xff, sizeof(float), st));
    if ((rc = prep_chunk(c, first, n, st))) return rc;
    c->n = first + n;
    return TSP_OK;
}

int tsp_end_events(tsp_ctx* c, void* stream)
{
    NvtxRange nvtx_("tsp_end_events (binning)");
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (!c->appending) return fail(c, TSP_ESTATE, "end_events without begin_events");
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    c->appending = false;
    int rc;
    if ((rc = ensure_sensitivity(c, st))) return rc;
    if ((rc = prep_finish(c, st))) return rc;
    TSP_CUDA(c, launch_fill(c->rho, c->npix, 1.0f, st));
    c->launches += 1;
    if ((rc = refresh_rhop(c, st))) return rc;
    c->iterations = 0;
    return TSP_OK;
}

int tsp_upload_events(tsp_ctx* c, const float* zu, const float* zd, const float* dl, int64_t n,
                      int on_device, void* stream)
{
    NvtxRange nvtx_("tsp_upload_events");
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (n < 0) return fail(c, TSP_EINVAL, "n < 0");
    if (n > 0 && (!zu || !zd || !dl)) return fail(c, TSP_EINVAL, "event pointer is NULL");
    int rc = tsp_begin_events(c, n, stream);
    if (!rc) rc = tsp_append_events(c, zu, zd, dl, n, on_device, stream);
    if (!rc) rc = tsp_end_events(c, stream);
    return rc;
}

int tsp_compute_sensitivity(tsp_ctx* c, float* out, int on_device, void* stream)
{
    NvtxRange nvtx_("tsp_compute_sensitivity");
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_sensitivity(c, st);
    if (rc) return rc;
    if (out) {
        if ((rc = copy_floats(c, out, c->s, c->npix, on_device, 1, st))) return rc;
        if (!on_device) TSP_CUDA(c, cudaStreamSynchronize(st));
    }
    return TSP_OK;
}

int tsp_set_image(tsp_ctx* c, const float* rho, int on_device, void* stream)
{
    NvtxRange nvtx_("tsp_set_image");
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_sensitivity(c, st);
    if (rc) return rc;
    if (rho) {
        if ((rc = copy_floats(c, c->rho, rho, c->npix, 1, on_device, st))) return rc;
        if (!on_device) {
            TSP_CUDA(c, cudaMemsetAsync(c->flag, 0, sizeof(int), st));
            TSP_CUDA(c, launch_check_image(c->npix, c->rho, c->flag, st));
            c->launches += 1;
            int bad = 0;
            TSP_CUDA(c, cudaMemcpyAsync(&bad, c->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
            TSP_CUDA(c, cudaStreamSynchronize(st));
            if (bad) {
                launch_fill(c->rho, c->npix, 1.0f, st);
                refresh_rhop(c, st);
                return fail(c, TSP_EINVAL, "image values must be finite and >= 0");
            }
        }
    } else {
        TSP_CUDA(c, launch_fill(c->rho, c->npix, 1.0f, st));
        c->launches += 1;
    }
    if ((rc = refresh_rhop(c, st))) return rc;
    c->iterations = 0;
    return TSP_OK;
}

int tsp_iterate(tsp_ctx* c, int n_iter, void* stream)
{
    NvtxRange nvtx_("tsp_iterate");
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (n_iter < 0) return fail(c, TSP_EINVAL, "n_iter < 0");
    if (!c->uploaded) return fail(c, TSP_ESTATE, "iterate before upload_events");
    if (n_iter == 0) return TSP_OK;
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    auto it = c->graphs.find(n_iter);
    if (it == c->graphs.end()) {
        tsp_ctx::Graph gr;
        int rc = capture_iterations(c, n_iter, &gr);
        if (rc) return rc;
        it = c->graphs.emplace(n_iter, std::move(gr)).first;
    }
    TSP_CUDA(c, cudaGraphLaunch(it->second.exec, st));
    c->launches += it->second.launches;
    c->last_graph = n_iter;
    c->iterations += n_iter;
    return TSP_OK;
}

int tsp_read_image(tsp_ctx* c, float* out, int which, int on_device, void* stream)
{
    NvtxRange nvtx_("tsp_read_image");
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (!out) return fail(c, TSP_EINVAL, "out is NULL");
    if (which != 0 && which != 1) return fail(c, TSP_EINVAL, "which must be 0 (rho) or 1 (rho')");
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = copy_floats(c, out, which ? c->rhop : c->rho, c->npix, on_device, 1, st);
    if (rc) return rc;
    if (!on_device) TSP_CUDA(c, cudaStreamSynchronize(st));
    return TSP_OK;
}

int tsp_loglik(tsp_ctx* c, double* out, void* stream)
{
    return tsp_loglik_grad(c, out, nullptr, 0, nullptr, stream);
}

int tsp_loglik_grad(tsp_ctx* c, double* L_out, float* g_rho, int g_on_device, double* g_sigma,
                    void* stream)
{
    NvtxRange nvtx_("tsp_loglik_grad");
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (!c->uploaded) return fail(c, TSP_ESTATE, "loglik before upload_events");
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = refresh_rhop(c, st);   // clears the accumulators, sums s rho
    if (rc) return rc;
    const bool grad = g_rho || g_sigma;
    const PassArgs a = pass_args(c);
    TSP_CUDA(c, launch_pass(c->lmax, grad ? kGrad : kLoglik, a, st));
    c->launches += pass_launches(c);
    if (grad) {
        float* gdst = (g_rho && g_on_device) ? g_rho : c->gbuf;
        TSP_CUDA(c, launch_grad_finalize(c->npix, gdst, c->A, c->s, st));
        c->launches += 1;
        if (g_rho && !g_on_device)
            if ((rc = copy_floats(c, g_rho, c->gbuf, c->npix, 0, 1, st))) return rc;
    }
    Accum h;
    TSP_CUDA(c, cudaMemcpyAsync(&h, c->accum, sizeof(Accum), cudaMemcpyDeviceToHost, st));
    TSP_CUDA(c, cudaStreamSynchronize(st));
    if (L_out) *L_out = h.sum_logD - h.sum_rhop;
    if (g_sigma) {
        const double sz = c->p.sigma_z, sl = c->p.sigma_dl;
        g_sigma[0] = h.g_iz * (-2.0 / (sz * sz * sz));   // d iz / d sigma_z = -2 / sigma_z^3
        g_sigma[1] = h.g_il * (-2.0 / (sl * sl * sl));
    }
    return TSP_OK;
}

int tsp_set_sigma(tsp_ctx* c, double sigma_z, double sigma_dl, void* stream)
{
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (!(std::isfinite(sigma_z) && sigma_z > 0 && std::isfinite(sigma_dl) && sigma_dl > 0))
        return fail(c, TSP_EINVAL, "sigmas must be finite and > 0");
    if (c->appending) return fail(c, TSP_ESTATE, "set_sigma between begin_events and end_events");
    {
        tsp_params q = c->p;
        q.sigma_z = sigma_z;
        q.sigma_dl = sigma_dl;
        if (!cinv_valid(q))
            return fail(c, TSP_EINVAL, "sigmas give a C^-1 that is not positive definite with gamma");
    }
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    tsp_params old = c->p;
    c->p.sigma_z = sigma_z;
    c->p.sigma_dl = sigma_dl;
    int rc = plan(c);
    if (rc) {
        c->p = old;
        plan(c);
        return rc;
    }
    clear_graphs(c);
    if (c->uploaded) {
        if ((rc = prepare_events(c, st))) return rc;
        if ((rc = refresh_rhop(c, st))) return rc;
    }
    return TSP_OK;
}

int tsp_stats(tsp_ctx* c, tsp_stats_t* out, void* stream)
{
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (!out) return fail(c, TSP_EINVAL, "out is NULL");
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    Accum h;
    TSP_CUDA(c, cudaMemcpyAsync(&h, c->accum, sizeof(Accum), cudaMemcpyDeviceToHost, st));
    TSP_CUDA(c, cudaStreamSynchronize(st));
    std::memset(out, 0, sizeof(*out));
    out->n_events = c->n;
    out->n_used = (int64_t)h.n_used;
    out->n_empty = (int64_t)c->counters_h[1];
    out->n_outliers = (int64_t)c->n_outliers;
    out->n_window = (int64_t)c->counters_h[3];
    out->iterations = c->iterations;
    out->launches = c->launches;
    out->n_qbad = (int64_t)h.n_qclip;
    out->n_clipped = (int64_t)h.n_lclip;
    out->sum_s_rho = h.sum_rhop;
    out->dbg_violation = (int64_t)h.dbg;
    return TSP_OK;
}

int tsp_set_profiling(tsp_ctx* c, int on)
{
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    DeviceGuard dg(c->dev);
    if ((bool)on != c->profiling) {
        TSP_CUDA(c, cudaDeviceSynchronize());
        clear_graphs(c);
        c->profiling = on != 0;
    }
    return TSP_OK;
}

int tsp_direct_image(tsp_ctx* c, float* out, int on_device, void* stream)
{
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (!out) return fail(c, TSP_EINVAL, "out is NULL");
    if (!c->uploaded) return fail(c, TSP_ESTATE, "direct_image before upload_events");
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    // integer counts in the gradient buffer (reinterpreted); the float image
    // goes to out, or for a host destination to A (all zero between passes),
    // which is copied out and cleared again
    float* dst = on_device ? out : c->A;
    TSP_CUDA(c, launch_direct_image(c->g, c->n, c->zu, c->zd, c->dl,
                                    reinterpret_cast<unsigned*>(c->gbuf), dst, st));
    c->launches += 2;
    if (!on_device) {
        int rc = copy_floats(c, out, c->A, c->npix, 0, 1, st);
        if (rc) return rc;
        TSP_CUDA(c, cudaMemsetAsync(c->A, 0, sizeof(float) * c->npix, st));
        TSP_CUDA(c, cudaStreamSynchronize(st));
    }
    return TSP_OK;
}

int tsp_set_variant(tsp_ctx* c, int variant)
{
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (variant != 0 && variant != 1) return fail(c, TSP_EINVAL, "variant must be 0 or 1");
    if (variant != c->variant) {
        DeviceGuard dg(c->dev);
        TSP_CUDA(c, cudaDeviceSynchronize());
        clear_graphs(c);
        c->variant = variant;
    }
    return TSP_OK;
}

int tsp_get_schedule(tsp_ctx* c, tsp_schedule* out)
{
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (!out) return fail(c, TSP_EINVAL, "out is NULL");
    out->ty_cap = c->sched.ty_cap;
    out->items_per_sm = c->sched.items_per_sm;
    out->order = c->sched.order;
    out->reserved = 0;
    return TSP_OK;
}

int tsp_set_schedule(tsp_ctx* c, const tsp_schedule* s, void* stream)
{
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (!s) return fail(c, TSP_EINVAL, "schedule is NULL");
    if (!schedule_valid(*s)) return fail(c, TSP_EINVAL, TSP_SCHEDULE_RANGES);
    if (c->appending)
        return fail(c, TSP_ESTATE, "set_schedule between begin_events and end_events");
    DeviceGuard dg(c->dev);
    const Schedule old = c->sched;
    c->sched.ty_cap = s->ty_cap;
    c->sched.items_per_sm = s->items_per_sm;
    c->sched.order = s->order;
    int rc = plan(c);
    if (rc) {
        c->sched = old;
        plan(c);
        return rc;
    }
    clear_graphs(c);
    if (c->uploaded && (rc = prepare_events(c, (cudaStream_t)stream))) return rc;
    return TSP_OK;
}

int tsp_autotune(tsp_ctx* c, tsp_schedule* chosen, float* best_ms, void* stream)
{
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (!c->uploaded) return fail(c, TSP_ESTATE, "autotune before upload_events");
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TSP_CUDA(c, cudaEventCreate(&e0));
    TSP_CUDA(c, cudaEventCreate(&e1));
    // best of two MLEM passes; A is cleared afterwards, rho is not touched
    auto time_pass = [&](float* ms) -> int {
        const PassArgs a = pass_args(c);
        float best = 1e30f;
        for (int r = 0; r < 2; ++r) {
            TSP_CUDA(c, launch_begin(c->accum, st));
            TSP_CUDA(c, cudaEventRecord(e0, st));
            TSP_CUDA(c, launch_pass(c->lmax, kMlem, a, st));
            TSP_CUDA(c, cudaEventRecord(e1, st));
            TSP_CUDA(c, launch_fill(c->A, c->npix, 0.0f, st));
            TSP_CUDA(c, cudaEventSynchronize(e1));
            float t = 0.0f;
            TSP_CUDA(c, cudaEventElapsedTime(&t, e0, e1));
            best = std::min(best, t);
            c->launches += 3 + pass_launches(c);
        }
        *ms = best;
        return TSP_OK;
    };
    tsp_schedule best{c->sched.ty_cap, c->sched.items_per_sm, c->sched.order, 0};
    float best_t = 0.0f;
    int rc = time_pass(&best_t);
    auto trial = [&](tsp_schedule s) -> int {
        int r = tsp_set_schedule(c, &s, stream);
        float t = 0.0f;
        if (!r) r = time_pass(&t);
        if (r) return r;
        if (t < best_t) {
            best_t = t;
            best = s;
        }
        return TSP_OK;
    };
    for (int ips : {2, 4, 8, 16, 32}) {
        tsp_schedule s = best;
        s.items_per_sm = ips;
        if (!rc && ips != best.items_per_sm) rc = trial(s);
    }
    for (int ty : {16, 32, 64, 128}) {
        tsp_schedule s = best;
        s.ty_cap = ty;
        if (!rc && ty != best.ty_cap) rc = trial(s);
    }
    if (!rc) rc = tsp_set_schedule(c, &best, stream);
    if (!rc) rc = refresh_rhop(c, st);
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = fail(c, TSP_ECUDA, cudaGetErrorString(e));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = best_t;
    return TSP_OK;
}

int tsp_backproject(tsp_ctx* c, float* A_out, int on_device, void* stream)
{
    NvtxRange nvtx_("tsp_backproject");
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (!A_out) return fail(c, TSP_EINVAL, "A_out is NULL");
    if (!c->uploaded) return fail(c, TSP_ESTATE, "backproject before upload_events");
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = refresh_rhop(c, st);   // clears the pass counters, rho' = s rho, sum s rho
    if (rc) return rc;
    const PassArgs a = pass_args(c);
    TSP_CUDA(c, launch_mlem_pass(c, a, st));
    c->launches += mlem_pass_launches(c);
    if ((rc = copy_floats(c, A_out, c->A, c->npix, on_device, 1, st))) return rc;
    // A is zero between passes (the next pass accumulates into it)
    TSP_CUDA(c, cudaMemsetAsync(c->A, 0, sizeof(float) * c->npix, st));
    if (!on_device) TSP_CUDA(c, cudaStreamSynchronize(st));
    return TSP_OK;
}

int tsp_apply_update(tsp_ctx* c, const float* A, int on_device, void* stream)
{
    NvtxRange nvtx_("tsp_apply_update");
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (!A) return fail(c, TSP_EINVAL, "A is NULL");
    if (c->appending) return fail(c, TSP_ESTATE, "apply_update between begin_events and end_events");
    if (!on_device)
        for (int i = 0; i < c->npix; ++i)
            if (!(std::isfinite(A[i]) && A[i] >= 0.0f))
                return fail(c, TSP_EINVAL, "A must be finite and >= 0");
    DeviceGuard dg(c->dev);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_sensitivity(c, st);
    if (rc) return rc;
    if ((rc = copy_floats(c, c->A, A, c->npix, 1, on_device, st))) return rc;
    // sum s rho is accumulated afresh by the update; the counters of the last
    // back-projection (events used) are kept
    TSP_CUDA(c, cudaMemsetAsync(reinterpret_cast<char*>(c->accum) + offsetof(Accum, sum_rhop), 0,
                                sizeof(double), st));
    TSP_CUDA(c, launch_finalize(c->npix, c->rho, c->rhop, c->A, c->s, c->accum, st));
    c->launches += 1;
    c->iterations += 1;
    if (!on_device) TSP_CUDA(c, cudaStreamSynchronize(st));
    return TSP_OK;
}

int tsp_wait(tsp_ctx* c, void* stream, int timeout_ms)
{
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (timeout_ms < 0) return fail(c, TSP_EINVAL, "timeout_ms < 0");
    DeviceGuard dg(c->dev);
    TSP_CUDA(c, cudaEventRecord(c->wait_ev, (cudaStream_t)stream));
    if (sim_fault() == kSimTimeout)
        return fail(c, TSP_ETIMEOUT, "the work enqueued on the stream did not finish within " +
                                         std::to_string(timeout_ms) + " ms (simulated)");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(c->wait_ev);
        if (e == cudaSuccess) return TSP_OK;
        if (e != cudaErrorNotReady)
            return fail(c, TSP_ECUDA, std::string("cudaEventQuery: ") + cudaGetErrorString(e));
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                            std::chrono::steady_clock::now() - t0)
                            .count();
        if (ms >= timeout_ms)
            return fail(c, TSP_ETIMEOUT, "the work enqueued on the stream did not finish within " +
                                             std::to_string(timeout_ms) + " ms");
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
}

int tsp_pass_times(tsp_ctx* c, float* ms, int max, int* count, void* stream)
{
    if (!c) return fail(nullptr, TSP_EINVAL, "ctx is NULL");
    if (!count || (max > 0 && !ms)) return fail(c, TSP_EINVAL, "NULL output");
    *count = 0;
    DeviceGuard dg(c->dev);
    auto it = c->graphs.find(c->last_graph);
    if (it == c->graphs.end() || it->second.ev.empty()) return TSP_OK;
    TSP_CUDA(c, cudaStreamSynchronize((cudaStream_t)stream));
    const auto& ev = it->second.ev;
    int n = std::min<int>(max, (int)(ev.size() / 2));
    for (int k = 0; k < n; ++k) TSP_CUDA(c, cudaEventElapsedTime(&ms[k], ev[2 * k], ev[2 * k + 1]));
    *count = n;
    return TSP_OK;
}

}  // extern "C"
