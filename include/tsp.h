/*
 * tsp.h -- C ABI of libtsp, a GB300 (sm_103a) implementation of list-mode MLEM
 * reconstruction for the two-strip time-of-flight PET detector of
 * Bialas et al., "GPU accelerated image reconstruction in a two-strip J-PET
 * tomograph" (arXiv:1502.07478).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Units are millimetres.  The strips lie at y = +R (upper) and y = -R
 *    (lower) along z in [-L/2, L/2] (Sec. 2, Fig. 1).
 *  - Image layout: ny x nz float32, row-major, z contiguous; pixel (iy, iz) is
 *    centred at y = -R + (iy + 1/2) dy, z = -L/2 + (iz + 1/2) dz.
 *  - Events are three float32 arrays of length n (structure of arrays): the
 *    measured hit positions z_u, z_d along the upper and lower strip and the
 *    path-length difference delta_l (Sec. 2, Eq. 1).
 *  - on_device = 1 means the pointer is device memory of the current CUDA
 *    device (for example a torch tensor's data_ptr()); 0 means host memory.
 *    Host pointers are only borrowed for the duration of the call; the library
 *    copies what it keeps.  Device pointers given by the caller are never freed
 *    by the library.
 *  - stream is a cudaStream_t (NULL = legacy default stream).  Calls enqueue
 *    work on it; calls that return host-side values synchronise it.
 *  - Return value 0 = success; a negative TSP_E* code on failure, with a
 *    message available from tsp_last_error().  No entry point aborts the
 *    process.  After TSP_ECUDA the context should be destroyed.
 *  - A context is not thread-safe: calls on one context must be serialised by
 *    the caller.  Distinct contexts are independent.
 *  - The library owns all device memory it allocates and frees it in
 *    tsp_destroy().
 *  - Error paths can be exercised without a device fault: the environment
 *    variable TSP_SIM_FAULT = oom (device allocations fail: TSP_ENOMEM),
 *    launch (kernel launches fail before anything is enqueued: TSP_ECUDA),
 *    nan_event (each uploaded chunk gets a NaN z_u: TSP_EINVAL) or timeout
 *    (tsp_wait gives up at once: TSP_ETIMEOUT) simulates that
 *    failure at every site it reaches while it is set.  A context whose call
 *    failed this way can still be destroyed, and new contexts work once the
 *    variable is unset.
 *  - Each entry point that enqueues work opens an NVTX range of its name.
 */
#ifndef TSP_H
#define TSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSP_OK 0
#define TSP_EINVAL (-1)   /* bad argument: sizes, NULL pointers, non-finite events */
#define TSP_ENOMEM (-2)   /* a device or pinned-host allocation failed */
#define TSP_ECUDA (-3)    /* a CUDA call failed (message holds the CUDA error) */
#define TSP_ETIMEOUT (-4) /* a bounded device-side wait gave up */
#define TSP_ESTATE (-5)   /* call out of order, e.g. iterate before any upload */

typedef struct tsp_ctx tsp_ctx;

/* Geometry, grid and resolution of one reconstruction. */
typedef struct {
    double R;          /* half of the strip separation (mm); > 0 */
    double L;          /* strip length (mm); > 0 */
    int32_t ny, nz;    /* image rows (y) and columns (z); > 0 */
    double dy, dz;     /* pixel pitch (mm); 0 selects 2R/ny and L/nz */
    double sigma_z;    /* resolution of z_u, z_d (mm); > 0.  Sec. 3, C^-1 */
    double sigma_dl;   /* resolution of delta_l (mm); > 0.  Sec. 3, C^-1 */
    double cut;        /* window radius in units of sigma; 0 selects 3 (Sec. 3) */
    int32_t flags;     /* reserved, must be 0 */
    int32_t reserved;
    double gamma;      /* cross term of C^-1 between z_u (z_d) and delta_l (Sec. 3):
                          C^-1 = [[1/sz^2, 0, g], [0, 1/sz^2, -g], [g, -g, 1/sdl^2]];
                          0 = diagonal; finite with 2 g^2 < 1/(sz^2 sdl^2 (1+kappa_z)^2) */
    double kappa_z;    /* z dependence of the z resolution (Sec. 3 notes about 10%
                          from the strip centre to its ends, without a form): an
                          event reconstructed at z~ uses
                          sz (1 + kappa_z min(1, (2 z~/L)^2)) in its kernel, window
                          and box; in [0, 1]; 0 = constant sz.  Gradients are with
                          respect to the base sigma_z. */
} tsp_params;

/* Counters of the last upload / pass (filled by tsp_stats). */
typedef struct {
    int64_t n_events;    /* events uploaded */
    int64_t n_used;      /* events with a positive denominator in the last pass */
    int64_t n_empty;     /* events whose window holds no pixel of the grid */
    int64_t n_outliers;  /* events whose window exceeds their tile's halo */
    int64_t n_window;    /* in-window pixels summed over events (pixel evaluations
                            per iteration), counted at upload */
    int64_t iterations;  /* MLEM iterations applied since the last set_image */
    int64_t launches;    /* kernel launches enqueued by this context so far
                            (each replayed graph node counts once) */
    int64_t n_qbad;      /* in-window pixels of the last pass with Q <= 0 (P = 0) */
    int64_t n_clipped;   /* window pixels outside the staged tile region in the
                            last pass (always 0 unless the library is faulty) */
    double sum_s_rho;    /* sum_l s_l rho_l of the current image */
    int64_t dbg_violation; /* a library built with TSP_DEBUG_CHECKS: the first
                            shared-memory access of a tile pass outside its block's
                            window since the context was created, as
                            (site << 32) | (byte offset + 1), the access skipped;
                            0 if none, and always 0 in a release build */
} tsp_stats_t;

/* Create a context for one reconstruction.  Validates params (TSP_EINVAL) and
 * allocates the image-sized device buffers.  The sensitivity map is computed
 * on first use.  *out receives the context; NULL on failure. */
int tsp_create(const tsp_params* params, tsp_ctx** out);

/* Free every resource of the context (NULL is accepted). */
void tsp_destroy(tsp_ctx* ctx);

/* Message of the last failure on ctx (or of the last failed tsp_create when
 * ctx is NULL).  The string lives until the next call on the same context. */
const char* tsp_last_error(const tsp_ctx* ctx);

/* Library version string, e.g. "tsp 0.1 sm_103a". */
const char* tsp_version(void);

/* Upload n events (replacing any previous set) and prepare them for
 * iteration: for each event the direct reconstruction of Eq. 2 (Sec. 2), the
 * 3-sigma window's bounding box of App. B, and the binning of events by the
 * image tile holding their window centre.  zu, zd, dl: n floats each, host or
 * device (on_device).  n = 0 is valid (an empty list).  Non-finite values give
 * TSP_EINVAL and upload nothing.  The image is reset to rho = 1. */
int tsp_upload_events(tsp_ctx* ctx, const float* zu, const float* zd, const float* dl,
                      int64_t n, int on_device, void* stream);

/* Streamed upload: the same result as tsp_upload_events of the concatenated
 * chunks, for event sets that are produced or staged in pieces.
 * tsp_begin_events reserves room for n_total events and clears the binning;
 * each tsp_append_events copies one chunk (host or device) and prepares it
 * (Eq. 2, window, bin key) while later chunks are still arriving: host chunks
 * are copied on a copy stream of the context, so with pinned host memory the
 * copy of chunk k+1 overlaps the preparation of chunk k.  A host chunk must
 * stay valid and unmodified until `stream` has been synchronised (the call
 * returns before the copy ends).  tsp_end_events bins the appended events,
 * resets the image to rho = 1 and synchronises.  Appending more than n_total
 * events gives TSP_EINVAL; append / end without begin, and iterate,
 * set_sigma or set_schedule between begin and end, give TSP_ESTATE. */
int tsp_begin_events(tsp_ctx* ctx, int64_t n_total, void* stream);
int tsp_append_events(tsp_ctx* ctx, const float* zu, const float* zd, const float* dl,
                      int64_t n, int on_device, void* stream);
int tsp_end_events(tsp_ctx* ctx, void* stream);

/* Sensitivity map s(y, z) of Eq. s-yz at the pixel centres (clamped at 0).
 * out (nullable) receives ny*nz floats, host or device (on_device). */
int tsp_compute_sensitivity(tsp_ctx* ctx, float* out, int on_device, void* stream);

/* Set the current image rho (ny*nz floats, host or device); rho = NULL sets
 * the uniform image rho = 1.  Values must be finite and >= 0 (TSP_EINVAL is
 * not checked on device data).  Resets the iteration counter. */
int tsp_set_image(tsp_ctx* ctx, const float* rho, int on_device, void* stream);

/* Apply n_iter >= 0 list-mode MLEM updates of Eq. iter (Sec. 2):
 *   rho_l <- rho_l * sum_j P(e_j|l) / D_j,  D_j = sum_i P(e_j|i) s_i rho_i,
 * with the kernel P of Eq. kernel (Sec. 3) over each event's 3-sigma window.
 * Events with D_j = 0 are skipped.  The iterations are replayed from a CUDA
 * graph captured on the first call with this n_iter.  Requires an upload
 * (TSP_ESTATE otherwise).  Asynchronous on stream. */
int tsp_iterate(tsp_ctx* ctx, int n_iter, void* stream);

/* Event-sharded iteration.  Eq. iter is a sum over events, and given the
 * image rho^t the events are independent: an update over a list split into
 * shards (one context per shard, e.g. one per GPU, every context holding the
 * same image) is the update over the whole list when the shards'
 * back-projections are summed before the image is multiplied.
 *
 * tsp_backproject writes the back-projection of this context's events at the
 * current image,
 *   A_out[l] = sum_j P(e_j|l) / D_j,   D_j = sum_i P(e_j|i) s_i rho_i,
 * over the events with D_j > 0 (ny*nz floats, host or device per on_device),
 * with the kernel P of Eq. kernel (Sec. 3) over each event's window.  At a
 * pixel with s_l rho_l = 0 (which the update keeps at 0 whatever A is) A_out[l]
 * holds only the terms of events on the global-memory path: the tile pass
 * sums the terms P s_l rho_l / D_j and divides by s_l rho_l, so it adds
 * nothing there.  The image is not changed; tsp_stats then reports the events used.  Requires an
 * upload (TSP_ESTATE; an empty list gives A = 0).  A host A_out is filled when
 * the call returns; a device A_out is written asynchronously on stream.
 *
 * tsp_apply_update applies rho_l <- rho_l * A[l] (the last step of Eq. iter)
 * with A given by the caller (ny*nz floats, host or device), typically the sum
 * of every shard's back-projection (an all-reduce); it refreshes rho' = s rho
 * and the sum of s rho and advances the iteration counter by one.  Host
 * values must be finite and >= 0 (TSP_EINVAL, nothing applied); device data
 * is not checked.
 *
 * One context's tsp_backproject followed by tsp_apply_update of its own A is
 * one tsp_iterate(ctx, 1) step up to float rounding order. */
int tsp_backproject(tsp_ctx* ctx, float* A_out, int on_device, void* stream);
int tsp_apply_update(tsp_ctx* ctx, const float* A, int on_device, void* stream);

/* Bounded wait (no counterpart in the paper): wait on the host until the work
 * enqueued on stream so far has finished, for at most timeout_ms >= 0
 * milliseconds.  Returns 0 when it has finished, TSP_ETIMEOUT when the limit
 * ran out first (the work continues; the context stays usable and the call
 * may be repeated), TSP_ECUDA when the stream reports an error. */
int tsp_wait(tsp_ctx* ctx, void* stream, int timeout_ms);

/* Direct-reconstruction image (Eq. 2, Sec. 2): out[iy*nz + iz] = the number of
 * uploaded events whose point (y~, z~) lies in pixel (iy, iz), i.e. y~ in
 * [-R + iy dy, -R + (iy+1) dy) and z~ in [-L/2 + iz dz, -L/2 + (iz+1) dz)
 * (ny*nz floats, host or device; events outside the grid are not counted).
 * Eq. 2 is evaluated in double precision.  Requires an upload (TSP_ESTATE). */
int tsp_direct_image(tsp_ctx* ctx, float* out, int on_device, void* stream);

/* Copy the current image to out (ny*nz floats, host or device).  which = 0:
 * rho of Eq. iter; which = 1: rho' = s * rho of Eq. iter-p. */
int tsp_read_image(tsp_ctx* ctx, float* out, int which, int on_device, void* stream);

/* List-mode Poisson log-likelihood of the current image,
 *   L = sum_j log D_j - sum_i s_i rho_i  (events with D_j = 0 skipped),
 * whose EM step is Eq. iter.  *out receives L (host double).  Synchronises. */
int tsp_loglik(tsp_ctx* ctx, double* out, void* stream);

/* L and its gradient at the current image and resolution, with windows fixed
 * at the current sigmas:
 *   g_rho[l]   = s_l (sum_j P_jl / D_j - 1)                    (ny*nz floats)
 *   g_sigma[k] = sum_j (1/D_j) sum_i s_i rho_i dP_ji/dsigma_k, k = (z, dl)
 * The denominators D_j are recomputed, not stored.  L_out, g_rho (host or
 * device per g_on_device) and g_sigma (host, 2 doubles) are each nullable.
 * Synchronises. */
int tsp_loglik_grad(tsp_ctx* ctx, double* L_out, float* g_rho, int g_on_device,
                    double* g_sigma, void* stream);

/* Change the resolution (sigma_z, sigma_dl > 0) used by the kernel and the
 * windows.  The uploaded events are re-prepared (windows and binning depend on
 * sigma); the image is kept. */
int tsp_set_sigma(tsp_ctx* ctx, double sigma_z, double sigma_dl, void* stream);

/* Fill *out with the counters of the context (synchronises stream). */
int tsp_stats(tsp_ctx* ctx, tsp_stats_t* out, void* stream);

/* Profiling aid (no counterpart in the paper).  With on = 1, graphs captured
 * from now on record a CUDA event pair around each launch of the main MLEM
 * kernel; tsp_pass_times then returns the device durations (ms) of those
 * launches in the last tsp_iterate call, in order.  *count receives the number
 * written (at most max).  Synchronises stream. */
int tsp_set_profiling(tsp_ctx* ctx, int on);
int tsp_pass_times(tsp_ctx* ctx, float* ms, int max, int* count, void* stream);

/* ------------------------------------------------------------------------
 * Tile schedule (no counterpart in the paper, whose kernel takes one event
 * per warp and reads rho through the texture cache, Sec. 4).  Events are
 * binned by the image tile of their window centre; a work item is a run of
 * the events of one tile, staged with its halo in shared memory.  The knobs:
 *   ty_cap        largest tile height in image rows, 4..128 (the shared-
 *                 memory budget may force a smaller one)
 *   items_per_sm  target work items per SM, 1..64: a tile's events are cut
 *                 into items of placed / (items_per_sm * SMs) events,
 *                 clamped to [32, 4096]
 *   order         batches only: 0 = longest estimated item first,
 *                 1 = round robin over the reconstructions
 *   reserved      0
 * Results do not depend on the schedule beyond float rounding order. */
typedef struct {
    int32_t ty_cap;
    int32_t items_per_sm;
    int32_t order;
    int32_t reserved;
} tsp_schedule;

/* MLEM pass variant of tsp_iterate: 0 = the tile kernel (default); 1 = one
 * thread per event (the thread-granularity kernel shape of Sec. 4.2, an
 * ablation: the window is walked row by row by one thread, rho' read from
 * global memory, P evaluated twice, the scatter done by global atomics).
 * Both give the same images up to float rounding order.  Other values give
 * TSP_EINVAL.  The log-likelihood and gradient passes always use the tiles. */
int tsp_set_variant(tsp_ctx* ctx, int variant);

/* Current schedule of ctx (default 128, 8, 0). */
int tsp_get_schedule(tsp_ctx* ctx, tsp_schedule* out);
/* Set the schedule; the uploaded events are re-binned (images are kept).
 * Invalid knobs give TSP_EINVAL and change nothing. */
int tsp_set_schedule(tsp_ctx* ctx, const tsp_schedule* sched, void* stream);
/* Autotuner: time one MLEM pass (best of 2, CUDA events on stream) for
 * candidate schedules by coordinate descent over items_per_sm in
 * {2,4,8,16,32} then ty_cap in {16,32,64,128}, keep the fastest and return it
 * in *chosen and its pass time (ms) in *best_ms (both nullable).  The image
 * is left unchanged.  Requires an upload (TSP_ESTATE).  Synchronises. */
int tsp_autotune(tsp_ctx* ctx, tsp_schedule* chosen, float* best_ms, void* stream);

/* ------------------------------------------------------------------------
 * Batches: k independent reconstructions (each with its own geometry, grid,
 * resolution, events and image) advanced together.  An MLEM iteration of a
 * batch is, whatever k: a reset of the pass accumulators, one persistent tile
 * launch per kernel class present (the reconstructions whose windows need the
 * same lane capacity and row split share one launch over all their work
 * items; plus one launch for outlier events when some reconstruction of the
 * class has them), and the image update of all reconstructions; n iterations
 * are replayed from one CUDA graph.  Results equal those of k
 * separate contexts up to float rounding order.  A batch is not thread-safe.
 * Indices i are 0..k-1; an index out of range gives TSP_EINVAL. */
typedef struct tsp_batch tsp_batch;

/* Create a batch from k >= 1 parameter sets (params[0..k-1]), each validated
 * as by tsp_create.  *out is NULL on failure. */
int tsp_batch_create(const tsp_params* params, int k, tsp_batch** out);
/* Free the batch and every reconstruction in it (NULL is accepted). */
void tsp_batch_destroy(tsp_batch* batch);
/* Message of the last failure on batch (or of the last failed
 * tsp_batch_create when batch is NULL). */
const char* tsp_batch_last_error(const tsp_batch* batch);
/* Number of reconstructions k (0 for NULL). */
int tsp_batch_size(const tsp_batch* batch);
/* As tsp_upload_events / tsp_set_image / tsp_set_sigma, for reconstruction i. */
int tsp_batch_upload_events(tsp_batch* batch, int i, const float* zu, const float* zd,
                            const float* dl, int64_t n, int on_device, void* stream);
int tsp_batch_set_image(tsp_batch* batch, int i, const float* rho, int on_device, void* stream);
int tsp_batch_set_sigma(tsp_batch* batch, int i, double sigma_z, double sigma_dl, void* stream);
/* Apply n_iter >= 0 MLEM updates (Eq. iter) to every reconstruction.  Every
 * reconstruction needs an upload (TSP_ESTATE otherwise).  Asynchronous. */
int tsp_batch_iterate(tsp_batch* batch, int n_iter, void* stream);
/* Copy an image of reconstruction i to out (its ny*nz floats, host or
 * device): which = 0 rho, 1 rho' = s rho, 2 the g_rho of the last
 * tsp_batch_loglik_grad. */
int tsp_batch_read_image(tsp_batch* batch, int i, float* out, int which, int on_device,
                         void* stream);
/* Log-likelihood and gradients (as tsp_loglik_grad) of every reconstruction
 * in one batched pass: L_out[i] (k doubles) and g_sigma[2i], g_sigma[2i+1]
 * (2k doubles), each nullable; g_rho is kept on the device for
 * tsp_batch_read_image(which = 2).  Synchronises. */
int tsp_batch_loglik_grad(tsp_batch* batch, double* L_out, double* g_sigma, void* stream);
/* Counters of reconstruction i (launches counts the batch's launches). */
int tsp_batch_stats(tsp_batch* batch, int i, tsp_stats_t* out, void* stream);
/* Schedule of the batch (shared by its reconstructions) and its autotuner:
 * as tsp_autotune, with item order in {0, 1} tried first, timing one batched
 * MLEM pass per candidate. */
int tsp_batch_get_schedule(tsp_batch* batch, tsp_schedule* out);
int tsp_batch_set_schedule(tsp_batch* batch, const tsp_schedule* sched, void* stream);
int tsp_batch_autotune(tsp_batch* batch, tsp_schedule* chosen, float* best_ms, void* stream);
/* As tsp_set_profiling / tsp_pass_times, for the batched pass. */
int tsp_batch_set_profiling(tsp_batch* batch, int on);
int tsp_batch_pass_times(tsp_batch* batch, float* ms, int max, int* count, void* stream);

/* ------------------------------------------------------------------------
 * Allocation-free MLEM update (no counterpart in the paper: an interface for
 * callers that cannot allocate device memory -- code running under a fixed
 * memory budget handed out by a host framework, real-time acquisition loops
 * where an allocation and the synchronisation it may imply are not allowed,
 * plug-ins that must not touch their host process's allocator).
 *
 * One list-mode MLEM update of Eq. iter, rho_out = rho_in * sum_j P_j / D_j,
 * computed by the same kernels as tsp_iterate.  All pointers except params and
 * errbuf are device pointers owned by the caller: zu, zd, dl (n floats each),
 * s (ny*nz, the sensitivity map, e.g. from tsp_compute_sensitivity), rho_in
 * and rho_out (ny*nz each; rho_out must not alias rho_in).  Non-finite events
 * are skipped.  Enqueued on stream; returns without synchronising.
 *
 * The call allocates nothing: no cudaMalloc, no cudaFree, no host heap.  Its
 * scratch (staged rho', back-projection accumulator, one chunk of prepared
 * events, counters) is a file-scope static device array of
 * TSP_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds
 * until the process exits.  Limits: ny*nz <= TSP_NOALLOC_MAX_PIXELS (larger
 * images return TSP_EINVAL with a message); events are processed in chunks of
 * TSP_NOALLOC_CHUNK, any n >= 0 is accepted.
 *
 * The first call on a device looks up the device address of the scratch array
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call on a device shares the one array and
 * it keeps the last call's contents (the call clears what must start at
 * zero): calls that overlap on the GPU (different streams or host threads)
 * race and give wrong results, so serialise them.
 *
 * errbuf (nullable, errlen bytes) receives a message on failure.  Returns 0 or
 * a TSP_E* code. */
#define TSP_NOALLOC_MAX_PIXELS (1 << 20)
#define TSP_NOALLOC_CHUNK (1 << 16)
#define TSP_NOALLOC_SCRATCH_BYTES (12u << 20)
int tsp_mlem_update_noalloc(const tsp_params* params, const float* zu, const float* zd,
                            const float* dl, int64_t n, const float* s, const float* rho_in,
                            float* rho_out, void* stream, char* errbuf, size_t errlen);

#ifdef __cplusplus
}
#endif

#endif /* TSP_H */
