/*
 * libhp — offloaded silicon-pixel local reconstruction on one GB300 (sm_103a).
 *
 * C ABI of the library.  The calls map onto the External Worker pattern of
 * "Bringing heterogeneity to the CMS software framework" (arXiv:2004.04334):
 *
 *   hp_enqueue_event / hp_enqueue_batch   the non-blocking acquire() (Sec. 2):
 *        read the inputs, queue all device work on a stream and return
 *        without waiting for the device;
 *   hp_on_complete                        the holder that resumes the caller
 *        (Sec. 2; Sec. 4.1: a callback queued into the stream, errors
 *        delivered with it);
 *   hp_fetch_clusters                     produce() (Sec. 2): collect the
 *        result once the stream has signalled completion;
 *   hp_event_* accessors                  the Product<T> wrapper of Sec. 4.2:
 *        device id, stream and CUDA event of the work that made the result;
 *   hp_enqueue_hits                       a second module consuming that
 *        product under the ScopedContext stream rules of Sec. 4.2 (the
 *        clusters -> hits step of Fig. 1);
 *   HP_KEEP_ON_DEVICE, hp_enqueue_transfer   transfer on demand (Sec. 4.3):
 *        results stay on the device unless a transfer module asks for them.
 *
 * Besides: a device-resident entry (hp_reconstruct_device, its CUDA-graph
 * form hp_graph_*, an allocation-free variant), an autotuner for the
 * clustering kernel's launch parameters (hp_autotune), a continuous-batching
 * serving loop (hp_serve_*), stage timers and counters.
 *
 * The device work is the raw -> clusters step of the paper's Fig. 1: decode
 * digi words, bucket them by module, calibrate q = adc * gain[m] - pedestal[m]
 * and keep pixels with q >= pixel_thr, label 8-connected clusters of the kept
 * pixels of each module, and reduce each cluster to its integer charge Q,
 * pixel count and charge-weighted centroid; keep clusters with
 * Q >= cluster_thr, ordered by (event, module, id) where id is the smallest
 * linear pixel index row * cols + col of the cluster.
 *
 * Conventions
 *   - Every call returns an hp_status.  HP_ECUDA means a CUDA runtime call
 *     failed; the context is then unusable and every later call on it
 *     returns HP_ECUDA.
 *   - Threading: all calls may be made from any thread.  Callbacks run on a
 *     CUDA host-function thread (or on the registering thread if the event is
 *     already complete) and must not call CUDA; hp_fetch_clusters,
 *     hp_event_query and hp_release_event make no CUDA call and are safe in a
 *     callback.
 *   - Digi word layout: bits 0-7 row, bits 8-16 column, bits 17-24 ADC,
 *     bits 25-31 zero.  Module ids are uint16.
 */
#ifndef HP_H
#define HP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hp_status {
    HP_OK = 0,
    HP_EAGAIN = 1,    /* over the device budget or the in-flight limit: retry after a completion */
    HP_ENOTREADY = 2, /* the event has not completed yet */
    HP_EINVAL = 3,    /* invalid argument or configuration */
    HP_EBADDIGI = 4,  /* an event holds an invalid digi word or module id */
    HP_EDUP = 5,      /* an event holds the same (module, row, col) twice */
    HP_ECAPACITY = 6, /* an output did not fit the capacity the caller gave */
    HP_ENOMEM = 7,    /* a device or pinned host allocation failed */
    HP_ETIMEOUT = 8,  /* a bounded wait inside a kernel gave up (results invalid) */
    HP_ECUDA = 9      /* a CUDA runtime call failed; the context is unusable */
} hp_status;

/* flags of hp_config.flags and of the enqueue calls */
#define HP_WANT_LABELS 0x1u  /* compute and return one label per input digi */
#define HP_INPUT_NOCOPY 0x2u /* enqueue: the input arrays are pinned host (or device)
                                memory that stays valid until the event completes;
                                they are read directly instead of being staged */
#define HP_KEEP_ON_DEVICE 0x4u /* enqueue: keep the clusters (and labels) in device
                                  memory until release; nothing but per-event status
                                  and offsets goes to the host (see hp_enqueue_transfer) */
#define HP_ALLOW_CPU 0x10u /* hp_config.flags: where no CUDA device is usable, hp_create makes a CPU
                              context (the CPU case of Sec. 3) instead of failing with HP_ECUDA */
#define HP_LABELS_U16 0x8u /* labels in the compact form (implies HP_WANT_LABELS):
                              hp_clusters.label16 and .item_first instead of .label,
                              2 bytes a digi instead of 4 over the host link; not with
                              HP_KEEP_ON_DEVICE (HP_EINVAL) */

/* what of hp_enqueue_transfer */
#define HP_TRANSFER_CLUSTERS 0x1u
#define HP_TRANSFER_LABELS 0x2u

/*
 * Context configuration.  gain and pedestal are host arrays of n_modules
 * entries, copied at hp_create.  Requirements (else HP_EINVAL):
 * 1 <= n_modules <= 65536, 1 <= rows <= 256, 1 <= cols <= 512,
 * rows * cols <= 131072, pixel_thr >= 1, and for every module gain >= 0 and
 * 255 * gain - pedestal <= INT32_MAX / (rows * cols), so that every cluster
 * charge fits in int32.
 */
typedef struct hp_config {
    int device;                 /* CUDA device ordinal */
    uint32_t n_modules;         /* modules per event (1856 for the full detector) */
    uint32_t rows, cols;        /* module geometry (160 x 416) */
    int32_t pixel_thr;          /* keep pixels with q >= pixel_thr (1000 e) */
    int32_t cluster_thr;        /* keep clusters with Q >= cluster_thr (4000 e) */
    const int32_t *gain;        /* [n_modules] e per ADC count */
    const int32_t *pedestal;    /* [n_modules] e */
    size_t device_budget_bytes; /* pooled device bytes that in-flight events may hold; 0 = no limit */
    uint32_t max_inflight;      /* events (or batches) in flight; 0 = 256 */
    uint32_t n_streams;         /* stream pool size; 0 = 4 */
    uint32_t flags;             /* default flags for enqueue (HP_WANT_LABELS) */
} hp_config;

typedef struct hp_ctx hp_ctx;
typedef struct hp_event hp_event;

/* Completion callback: called exactly once per event with its final status. */
typedef void (*hp_callback)(void *user, hp_event *ev, hp_status st);

/*
 * Host view of a completed event (library-owned pinned memory, valid until
 * hp_release_event).  Clusters of event e are [cluster_offsets[e],
 * cluster_offsets[e+1]).  An event whose event_status is not HP_OK has an
 * unspecified cluster slice and labels; the others are exact.
 */
typedef struct hp_clusters {
    uint32_t n_events;
    uint64_t n_digis;
    uint64_t n_clusters;
    uint64_t tag;
    const uint64_t *cluster_offsets; /* [n_events + 1] */
    const int32_t *event_status;     /* [n_events] hp_status of each event */
    const uint32_t *module;          /* [n_clusters] module index */
    const int32_t *id;               /* smallest linear index row * cols + col */
    const int32_t *charge;           /* Q = sum of q over the cluster (e) */
    const int32_t *npix;             /* pixels in the cluster */
    const float *x;                  /* charge-weighted mean row */
    const float *y;                  /* charge-weighted mean column */
    const int32_t *label;            /* [n_digis] cluster id, -1 (pixel below threshold),
                                        -2 (cluster below threshold); NULL without HP_WANT_LABELS
                                        and with HP_LABELS_U16 */
    /* HP_LABELS_U16 (else NULL).  Digi i of event e on module m belongs to
     * cluster cluster_offsets[e] + item_first[e * n_modules + m] + label16[i]
     * when label16[i] < 0xFFFE; 0xFFFF marks a pixel below threshold, 0xFFFE
     * a cluster below threshold (the -1 and -2 of .label).  A module holds at
     * most ceil(rows/2) * ceil(cols/2) <= 32768 clusters, so the rank fits. */
    const uint16_t *label16;         /* [n_digis] rank of the digi's cluster among its module's */
    const uint32_t *item_first;      /* [n_events * n_modules] first cluster of (e, m), from e's first */
} hp_clusters;

/*
 * Output arrays of hp_reconstruct_device, all device pointers owned by the
 * caller.  capacity is the room in the six cluster arrays; a batch never
 * has more clusters than digis, so capacity >= n_digis always suffices.
 */
typedef struct hp_device_clusters {
    uint64_t capacity;
    uint32_t *module;
    int32_t *id, *charge, *npix;
    float *x, *y;
    uint64_t *cluster_offsets; /* [n_events + 1] */
    int32_t *event_status;     /* [n_events] hp_status of each event */
    int32_t *label;            /* [n_digis] or NULL (labels not computed) */
} hp_device_clusters;

/* Launch settings of the clustering kernel (see hp_autotune). */
typedef struct hp_tuning {
    uint32_t tile_slots;
    uint32_t blocks_per_sm;
    uint32_t ticket_items;
    uint32_t warp_max;
    uint32_t label_store;  /* HP_STORE_BITMAP or HP_STORE_HASH */
    uint32_t item_threads; /* threads per item: 512 with the bitmap store; 128, 256 or 512 with the hash store */
} hp_tuning;

#define HP_STORE_BITMAP 0u
#define HP_STORE_HASH 1u

/* Counters of the context (monotonic unless stated). */
typedef struct hp_stats {
    uint64_t device_mallocs;    /* cudaMalloc calls made by the caching pool */
    uint64_t host_mallocs;      /* cudaHostAlloc calls made by the caching pool */
    uint64_t pool_hits;         /* allocations served from the cache */
    uint64_t device_bytes_in_use; /* current: bytes held by in-flight work */
    uint64_t device_bytes_cached; /* current: bytes held by the pool in total */
    uint64_t events_enqueued;
    uint64_t events_completed;
    uint64_t inflight;          /* current */
    uint64_t h2d_bytes, d2h_bytes; /* bytes moved by cudaMemcpyAsync */
    uint64_t kernel_launches;   /* kernels launched by the library */
    uint64_t serve_batches;     /* batches launched by the serving loop */
    uint64_t serve_requests;    /* requests accepted by hp_submit */
    uint64_t consumer_stream_reuses; /* consumer calls (hits, transfer) that took the product's own stream */
    uint64_t consumer_stream_waits;  /* consumer calls that queued cudaStreamWaitEvent */
    uint64_t serve_submit_ns;   /* serving: total time spent inside hp_submit (all threads) */
    uint64_t serve_launch_ns;   /* serving: total admitter time launching batches */
    uint64_t serve_complete_ns; /* serving: total time in batch completion host functions (callbacks included) */
    uint64_t serve_max_batch;   /* serving: most requests in one batch */
} hp_stats;

/* Serving loop configuration (hp_serve_start). */
typedef struct hp_serve_config {
    size_t device_budget_bytes;    /* device bytes in-flight batches may hold; 0 = no limit */
    uint32_t max_batch_events;     /* requests per batch; 0 = 256 */
    uint64_t max_batch_digis;      /* digis per batch; 0 = 32 Mi */
    uint32_t max_inflight_batches; /* batches on the device at once; 0 = 3 */
    uint32_t max_pending;          /* queued requests before hp_submit says HP_EAGAIN; 0 = 65536 */
    uint32_t flags;                /* HP_WANT_LABELS or HP_LABELS_U16; HP_INPUT_NOCOPY: hp_submit does not
                                      copy the inputs, the batch's gather kernel reads them in place
                                      (pinned memory, or any host memory on hosts whose device reads
                                      pageable memory), else one DMA each; they must stay valid until
                                      the request completes */
} hp_serve_config;

const char *hp_status_string(hp_status st);

/*
 * Create a context on cfg->device: the stream pool and the caching device
 * and pinned-host allocators from which every event draws its memory
 * (Sec. 4.1: no allocation or synchronisation on the event path once the
 * pools are warm), and device copies of the calibration tables.  *out
 * receives the context.
 *
 * The choice of technology (Sec. 3, the SwitchProducer) is made here, at
 * run time, when the caller asks for it: with HP_ALLOW_CPU in cfg->flags
 * and no usable CUDA device cfg->device, or with the environment variable
 * HP_FORCE_CPU set to anything but "0", the context is a CPU context.
 * Without either, a missing device is an error (HP_ECUDA): the library
 * never falls back to the host on its own.  It produces the same hp_clusters (same fields, order, labels in
 * either form, per-event statuses) with the host's cores (HP_CPU_THREADS
 * threads; default one per hardware thread), and each product's provenance
 * says HP_PATH_CPU and names the host.  A CPU context takes hp_enqueue_event,
 * hp_enqueue_batch (not HP_KEEP_ON_DEVICE), hp_on_complete, hp_event_query,
 * hp_fetch_clusters, hp_release_event, hp_event_provenance, hp_get_stats and
 * hp_destroy; the device entries, graphs, the autotuner, serving, hits and
 * transfers return HP_EINVAL.  Its events run in submission order, each
 * spread over the threads; callbacks run on the context's dispatcher thread.
 * Errors: HP_EINVAL (see hp_config), HP_ENOMEM, HP_ECUDA.
 */
hp_status hp_create(const hp_config *cfg, hp_ctx **out);

/*
 * Drain every in-flight event (this blocks: teardown is outside event
 * processing), then free all memory, the pools of Sec. 4.1 included.
 * Events not yet released are released.
 */
hp_status hp_destroy(hp_ctx *ctx);

/*
 * acquire() for one event (Sec. 2): n_digis digis, words[i] with module id
 * module_ids[i], in any order.  Unless HP_INPUT_NOCOPY is set the inputs are
 * copied into pooled pinned staging before the call returns, so the caller
 * may reuse them at once.  The call queues the host-to-device copy, the
 * kernels, the device-to-host transfer and a completion callback on one
 * stream of the pool and returns without waiting for the device.
 * flags: HP_WANT_LABELS, HP_INPUT_NOCOPY, HP_KEEP_ON_DEVICE (ORed with
 * hp_config.flags).
 * Errors: HP_EINVAL (NULL pointers with n_digis > 0, n_digis >= 2^32 - 1),
 * HP_EAGAIN (budget or in-flight limit), HP_ENOMEM, HP_ECUDA.
 */
hp_status hp_enqueue_event(hp_ctx *ctx, const uint32_t *words, const uint16_t *module_ids, uint64_t n_digis,
                           uint64_t tag, uint32_t flags, hp_event **out);

/*
 * acquire() for a batch of n_events independent events concatenated in
 * words/module_ids: event e owns digis [offsets[e], offsets[e+1]), offsets
 * has n_events + 1 entries, offsets[0] == 0 and is non-decreasing.  The whole
 * batch runs as one device pass; completion, callback and view are per
 * batch, with per-event status and cluster offsets.
 * Errors: as hp_enqueue_event, plus HP_EINVAL for bad offsets.
 */
hp_status hp_enqueue_batch(hp_ctx *ctx, uint32_t n_events, const uint64_t *offsets, const uint32_t *words,
                           const uint16_t *module_ids, uint64_t tag, uint32_t flags, hp_event **out);

/*
 * Register the completion callback (the holder of Sec. 2 / Sec. 4.1).  It is
 * called exactly once: on the CUDA host-function thread when the event
 * completes, or right here on the calling thread if it already has.  At most
 * one callback per event (else HP_EINVAL).
 */
hp_status hp_on_complete(hp_event *ev, hp_callback cb, void *user);

/* Non-blocking: HP_ENOTREADY while running, else the event's final status. */
hp_status hp_event_query(hp_event *ev);

/*
 * produce() (Sec. 2): fill *view with the event's results.  HP_ENOTREADY if
 * the event has not completed; otherwise returns the event's status (the
 * view is filled in every case once complete).  Works on clusters events of
 * the host path, serving requests and transfer events (arrays a transfer
 * did not carry are NULL); HP_EINVAL for hits events and for events kept on
 * the device (HP_KEEP_ON_DEVICE).  Makes no CUDA call.
 */
hp_status hp_fetch_clusters(hp_event *ev, hp_clusters *view);

/*
 * Return the event's buffers to the pool (Sec. 4.1).  This ends the product
 * holder's lifetime of Sec. 2: before completion the release is deferred
 * until the event completes (after its callback), and while consumers (hits,
 * transfers) still read its outputs, until they have run.  The event
 * pointer and its views are invalid afterwards.  Makes no CUDA call.
 */
hp_status hp_release_event(hp_event *ev);

/*
 * Provenance (Sec. 3: the framework records, per event, on which technology
 * a product was made): the device (name, ordinal, compute capability), the
 * library build, the path that made the product and, for clustering
 * products, the clustering kernel's settings (hp_tuning) it ran with.
 * Valid until hp_release_event; makes no CUDA call.
 */
#define HP_PATH_EVENT 1u    /* hp_enqueue_event */
#define HP_PATH_BATCH 2u    /* hp_enqueue_batch */
#define HP_PATH_SERVING 3u  /* a serving request (hp_submit) */
#define HP_PATH_HITS 4u     /* hp_enqueue_hits */
#define HP_PATH_TRANSFER 5u /* hp_enqueue_transfer */
#define HP_PATH_CPU 6u      /* the CPU case (Sec. 3): hp_enqueue_event / _batch on a context without a GPU */
typedef struct hp_provenance {
    char device_name[64];
    int device;
    int cc_major, cc_minor;
    const char *library; /* static string */
    uint32_t path;       /* HP_PATH_* */
    hp_tuning tuning;    /* zero for hits and transfer products */
} hp_provenance;
hp_status hp_event_provenance(const hp_event *ev, hp_provenance *out);

/* Product<T> metadata (Sec. 4.2): device ordinal, producing stream
 * (cudaStream_t) and the CUDA event recorded after the work. */
int hp_event_device(const hp_event *ev);
void *hp_event_stream(const hp_event *ev);
void *hp_event_cuda_event(const hp_event *ev);
/* Host wall-clock nanoseconds from enqueue to completion (0 before). */
uint64_t hp_event_latency_ns(const hp_event *ev);

/*
 * Device-resident entry: inputs are already in device memory and outputs go
 * to caller-owned device memory; the work is queued on `stream` (a
 * cudaStream_t, NULL for the legacy default stream) and the call returns
 * without waiting.  d_words is 4-byte aligned, d_module_ids 2-byte aligned,
 * d_offsets has n_events + 1 entries with offsets[n_events] == n_digis.
 * Scratch comes from a per-stream workspace of the context; the first call on
 * a stream, or a call that needs more scratch than earlier ones, allocates
 * it (and synchronises that stream); later calls allocate nothing, so the
 * call can be captured in a CUDA graph once warmed up.  Errors found on the
 * device are reported per event in out->event_status.
 * Errors: HP_EINVAL, HP_ENOMEM, HP_ECUDA.
 */
hp_status hp_reconstruct_device(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                                const uint32_t *d_words, const uint16_t *d_module_ids,
                                const hp_device_clusters *out, void *stream);

/*
 * Allocation-free variant of hp_reconstruct_device, for callers that cannot
 * allocate device memory: code that runs where cudaMalloc/cudaFree are not
 * allowed or would stall the device (they synchronise), or under a
 * framework whose own allocator owns the device memory.  (The paper has no
 * counterpart; it is an addition of this library.)
 *
 * Same arguments, work and outputs as hp_reconstruct_device, but the scratch
 * is one fixed 24 MiB device array inside the library, so the call makes no
 * cudaMalloc, cudaFree or other allocating call.  That array exists on every
 * GPU where the library is used, for the life of the process.
 * Limits: n_digis <= 131072 and n_events * n_modules <= 16384 per call, else
 * HP_ECAPACITY (nothing is launched).  The first call on a device looks the
 * array up on that device (cudaGetSymbolAddress) and keeps its address for
 * the life of the process; make that first call before any stream capture,
 * and do not call the entry point after a cudaDeviceReset.  All calls share the one array and each call
 * overwrites what the previous one left in it: calls whose work overlaps on
 * the GPU (different streams, or another thread) race and corrupt each
 * other; serialise them, e.g. on one stream.
 * Argument checks are those of hp_reconstruct_device; a CUDA error marks the
 * context failed (HP_ECUDA for every later call), as there.
 * Errors: HP_EINVAL, HP_ECAPACITY, HP_ECUDA.
 */
hp_status hp_reconstruct_device_noalloc(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                                        const uint32_t *d_words, const uint16_t *d_module_ids,
                                        const hp_device_clusters *out, void *stream);

/*
 * Autotuner.  The clustering kernel has launch parameters whose best values
 * depend on the launch shape (how many (event, module) items, how many
 * digis per item):
 *   tile_slots     capacity of the shared-memory tile of the block tier:
 *                  items with more digis are clustered in global scratch;
 *   blocks_per_sm  resident clustering blocks per SM, 1, 2 or 3 (1 allows
 *                  the largest tile; 3 caps the kernel at 40 registers a
 *                  thread and needs a smaller tile);
 *   ticket_items   (event, module) items per work-queue ticket, 16, 8, 4
 *                  or 2 (halved for launches too small to fill the GPU: down
 *                  to 4 for items of under 64 digis on average, to 1 for
 *                  larger ones);
 *   warp_max       largest item (digis) clustered by a single warp, 32 or 64;
 *   label_store    how the items above the warp tier look up a pixel's
 *                  neighbours: HP_STORE_BITMAP,
 *                  module-sized occupancy and survivor bitmaps with
 *                  row-major slots, one block (512 threads) an item; or
 *                  HP_STORE_HASH, an open-addressing table keyed by linear
 *                  pixel index with two slots a digi, so that its memory
 *                  follows the item's size, for items up to the hash
 *                  store's capacity (larger ones take the bitmap tiers);
 *   item_threads   threads clustering one item of the hash store, 128, 256
 *                  or 512 (a block runs 512 / item_threads items side by
 *                  side, each in its share of the block's shared memory;
 *                  the capacity is what that share holds at 28 bytes a digi,
 *                  at most 8 digis a thread, 5 at three blocks per SM).
 * Labels and clusters are the same for every setting; only speed differs.
 * Settings are kept per shape bucket (log2 of n_events * n_modules, log2 of
 * the mean digis per item) and used by every later launch in the bucket
 * (host, device, graph and serving paths).  A bucket without an entry takes
 * the entry of the nearest tuned bucket (distance |d items_log2| +
 * 4 |d digis_per_item_log2|, at most 8), else the defaults: 4096 slots, 2
 * blocks, 16 items, 64 digis, bitmap store, or, for a mean of 1024 digis
 * per item or more, the single-block tile with 4 items a ticket and 32
 * digis, bitmap store.
 *
 * hp_autotune times every candidate (hp_tuning_candidates) on the given
 * device-resident inputs, `reps` passes each after one warm-up, on a private
 * stream (blocking: a set-up call), stores the fastest for the shape's
 * bucket and returns it; cand_ms[i] (if given, up to cap entries) receives
 * candidate i's mean pass time in milliseconds.  `out` receives a valid
 * result of the inputs.
 * Environment: HP_TUNE=off ignores stored settings (defaults only);
 * HP_TUNE=search makes hp_reconstruct_device tune a bucket the first time
 * it sees it (that call blocks); HP_TUNE_CACHE=<path> loads settings from
 * that file at hp_create (one JSON object per line, entries of other
 * devices or module sizes ignored) and hp_autotune appends its results.
 * Errors: as hp_reconstruct_device; hp_set_tuning returns HP_EINVAL for a
 * setting outside the candidates' ranges (t == NULL clears the bucket).
 */
hp_status hp_tuning_candidates(hp_ctx *ctx, uint32_t cap, hp_tuning *list, uint32_t *n);
hp_status hp_get_tuning(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, hp_tuning *out);
hp_status hp_set_tuning(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const hp_tuning *t);
hp_status hp_autotune(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                      const uint32_t *d_words, const uint16_t *d_module_ids, const hp_device_clusters *out,
                      uint32_t reps, uint32_t cap, double *cand_ms, hp_tuning *best, double *best_ms);

/*
 * CUDA-graph form of the device-resident entry: hp_graph_capture records
 * one hp_reconstruct_device pass (a memset and six kernels) for fixed
 * arguments into an executable CUDA graph with its own scratch;
 * hp_graph_launch replays it on `stream` (one cudaGraphLaunch, no
 * allocation, no host work per launch).  The graph keeps the pointers and
 * sizes it was captured with: refill the same input buffers between
 * launches.  Launches of one graph are serialised by CUDA.  (The paper
 * found graphs too restrictive for its framework, Sec. 4; for a fixed-shape
 * batch they only remove launch overhead.)  hp_graph_destroy waits for the
 * device (it frees the scratch); hp_destroy destroys graphs left over.
 * Errors: as hp_reconstruct_device; HP_ECUDA if capture fails.
 */
typedef struct hp_graph hp_graph;
hp_status hp_graph_capture(hp_ctx *ctx, uint32_t n_events, uint64_t n_digis, const uint64_t *d_offsets,
                           const uint32_t *d_words, const uint16_t *d_module_ids, const hp_device_clusters *out,
                           hp_graph **graph);
hp_status hp_graph_launch(hp_graph *graph, void *stream);
hp_status hp_graph_destroy(hp_graph *graph);

/*
 * Hits: the clusters -> hits step of the paper's Fig. 1, the stage after the
 * clusters, run as a second module of a GPU chain (Sec. 4.2).
 *
 * Placement of module m: origin[3m .. 3m+2] (cm) and the row-major rotation
 * rot[9m .. 9m+8].  A cluster with centroid (x, y) in pixel units (pixel
 * (r, c) has its centre at (r, c)) lies at local
 *   u = (x - (rows - 1) / 2) * pitch_row,  v = (y - (cols - 1) / 2) * pitch_col
 * about the module centre, and its hit at origin + rot * (u, v, 0).  The
 * kernel computes in FP32.
 *
 * hp_set_geometry copies the placement (host arrays of n_modules entries) to
 * the device; it blocks (set-up call).  Calling it again installs a new
 * placement for later hp_enqueue_hits calls; work already queued keeps the
 * one it was queued with.  Errors: HP_EINVAL (NULL arrays, pitches not
 * finite and > 0), HP_ENOMEM, HP_ECUDA.
 */
hp_status hp_set_geometry(hp_ctx *ctx, const float *origin, const float *rot, float pitch_row, float pitch_col);

/*
 * Host view of a completed hits event (library-owned pinned memory, valid
 * until hp_release_event).  Hit i is cluster i of the consumed event: same
 * order, same per-event offsets and status.
 */
typedef struct hp_hits {
    uint32_t n_events;
    uint64_t n_hits;
    uint64_t tag;
    const uint64_t *hit_offsets;   /* [n_events + 1] */
    const int32_t *event_status;   /* [n_events] */
    const uint32_t *module;        /* [n_hits] */
    const float *x, *y, *z;        /* [n_hits] global position (cm) */
} hp_hits;

/*
 * A consumer of a clusters event (the Product<T> of an hp_enqueue_event or
 * hp_enqueue_batch call), following the ScopedContext rules of Sec. 4.2:
 * the work runs on the product's device; the first consumer of a product
 * queues its kernel on the product's own stream (stream order is the
 * synchronisation); every later consumer takes another stream of the
 * context and, if the product's CUDA event has not completed yet, queues
 * cudaStreamWaitEvent on it.  The call never waits for the device.  The
 * result is a new event (*out) with its own completion, callback
 * (hp_on_complete), query, stream and CUDA event, read with hp_fetch_hits
 * and released with hp_release_event.  The consumer holds the product: a
 * product released while consumers are queued is freed only once they have
 * run.  The product must not have been released before this call, and must
 * be a clusters event of hp_enqueue_event/hp_enqueue_batch (not a serving
 * request, not a hits or transfer event).  flags is reserved (0).  It
 * makes CUDA calls, so it must not be called from a completion callback.
 * Errors: HP_EINVAL (no geometry set, wrong kind of event), HP_ENOMEM,
 * HP_ECUDA.
 */
hp_status hp_enqueue_hits(hp_event *clusters, uint32_t flags, hp_event **out);

/* produce() of a hits event: as hp_fetch_clusters (HP_ENOTREADY before
 * completion, else the status of the consumed product). */
hp_status hp_fetch_hits(hp_event *ev, hp_hits *view);

/*
 * Transfer on demand (Sec. 4.3).  An event enqueued with HP_KEEP_ON_DEVICE
 * keeps its results in device memory (held, and charged to the device
 * budget, until hp_release_event); hp_fetch_clusters refuses it (HP_EINVAL).
 * Device consumers read it in place: hp_enqueue_hits, or
 * hp_event_device_clusters, which fills *view with the device addresses
 * (valid until release; safe to read after completion or in the product's
 * stream order).  hp_enqueue_transfer is the transfer module: a consumer
 * under the same stream rules as hp_enqueue_hits that copies to pinned host
 * memory the per-event offsets and statuses and, as `what` asks, the
 * clusters (only those that exist: a kernel reads their count on the device
 * and writes them over the C2C link) and/or the labels (the product must
 * have been enqueued with HP_WANT_LABELS).  The result is a new event read
 * with hp_fetch_clusters; arrays not transferred are NULL in its view.
 * Errors: HP_EINVAL (product not kept on the device, bad `what`, labels not
 * computed), HP_ENOMEM, HP_ECUDA.
 */
hp_status hp_event_device_clusters(hp_event *ev, hp_device_clusters *view);
hp_status hp_enqueue_transfer(hp_event *product, uint32_t what, hp_event **out);

/*
 * Device-resident hits: reads the clusters that hp_reconstruct_device wrote
 * (d_cluster_offsets[n_events] clusters, at most capacity, in d_module,
 * d_x, d_y) and writes the hit positions to d_hx, d_hy, d_hz (capacity
 * entries each); all device pointers owned by the caller.  Queued on
 * `stream` behind the clusters (the same stream gives the ordering); the
 * call returns without waiting and allocates nothing.
 * Errors: HP_EINVAL (no geometry set, NULL pointers), HP_ECUDA.
 */
hp_status hp_hits_device(hp_ctx *ctx, uint32_t n_events, uint64_t capacity, const uint64_t *d_cluster_offsets,
                         const uint32_t *d_module, const float *d_x, const float *d_y, float *d_hx, float *d_hy,
                         float *d_hz, void *stream);

/*
 * Serving (continuous batching).  hp_serve_start starts an admitter thread.
 * hp_submit is a non-blocking acquire() of one event (Sec. 2): it copies the
 * inputs into pooled pinned staging (or, with HP_INPUT_NOCOPY in the serving
 * flags, keeps the caller's pointers for the batch to copy by DMA) and
 * queues the request; it returns
 * HP_EAGAIN only when max_pending requests already wait.  The admitter
 * launches everything queued as one batch whenever fewer than
 * max_inflight_batches batches run and the batch fits the device budget
 * (Sec. 4.1: only asynchronous calls, pooled memory; batches overlap on the
 * context's streams, so copies of one batch overlap compute of another).
 * Each request is an hp_event with its own completion (cb, if given, is its
 * hp_on_complete callback), status, latency and one-event view
 * (hp_fetch_clusters); release each with hp_release_event.  hp_serve_stop
 * launches what is still queued and waits for every batch (blocking;
 * hp_destroy does it too).  hp_serve_start reserves, in the context's
 * caching pools, one block of the largest batch the loop can form per
 * in-flight batch (within the device budget), so that the loop itself never
 * calls cudaMalloc or cudaHostAlloc (this is setup: it blocks, and holds
 * that memory until hp_destroy).
 * Errors: HP_EINVAL (not serving / already serving / bad arguments),
 * HP_EAGAIN, HP_ENOMEM, HP_ECUDA.
 */
hp_status hp_serve_start(hp_ctx *ctx, const hp_serve_config *cfg);
hp_status hp_submit(hp_ctx *ctx, const uint32_t *words, const uint16_t *module_ids, uint64_t n_digis, uint64_t tag,
                    hp_callback cb, void *user, hp_event **out);
hp_status hp_serve_stop(hp_ctx *ctx);

/*
 * Load driver for the serving loop (Sec. 2: several threads acquire
 * concurrently, none blocks on the device): n_threads native submitter
 * threads replay a schedule of n_requests arrivals.  Request i arrives
 * arrival_ns[i] after the start (non-decreasing per thread is not required)
 * and submits pool event event_index[i] (pool_words/pool_modules/pool_n, n_pool
 * events, host memory; with HP_INPUT_NOCOPY serving a pool that is not all
 * in pinned memory is first copied into one pinned block, as a data source
 * writing to pinned buffers would provide it).  Each completion callback records the request's
 * submit-to-completion latency in latency_ns[i] and its status in status[i],
 * then releases it.  The call returns when every request has completed;
 * *span_ns is the time from the start to the last completion.  Requires a
 * running serving loop (hp_serve_start).  Returns the first hp_submit error
 * other than HP_EAGAIN (which is retried), else HP_OK.
 */
hp_status hp_serve_replay(hp_ctx *ctx, uint32_t n_threads, uint64_t n_requests, const uint64_t *arrival_ns,
                          const uint32_t *event_index, uint32_t n_pool, const uint32_t *const *pool_words,
                          const uint16_t *const *pool_modules, const uint64_t *pool_n, uint64_t *latency_ns,
                          int32_t *status, uint64_t *span_ns);

hp_status hp_get_stats(hp_ctx *ctx, hp_stats *out);

/*
 * Stage timers (tracing).  After hp_profile_enable(ctx, n), the next n
 * launches of the context record a CUDA event before and after each of their
 * kernels on the launching stream (asynchronous, no host wait); n = 0 stops
 * and clears.  hp_profile_read waits for the recorded events (a blocking
 * call: use it outside event processing) and returns, per kernel name, the
 * number of timed launches and their summed device time in milliseconds.
 * names[i] are static strings.  *n_kernels receives the number of kernels
 * (at most cap are written).
 */
/*
 * Serving trace (tracing of the loop of hp_serve_start).  After
 * hp_serve_trace_enable(ctx, cap) the next cap batches record, when their
 * completion host function ends: the submit time of their oldest request,
 * when the admitter took them, when their launch had been queued, and when
 * their completion host function started and ended (ns, one monotonic
 * clock, the one of hp_event_latency_ns), with their event and digi counts.
 * hp_serve_trace_read copies up to cap records (oldest first) and reports
 * how many there are; cap 0 in hp_serve_trace_enable stops and clears.  No
 * CUDA call.  Errors: HP_EINVAL.
 */
typedef struct hp_serve_trace_record {
    uint64_t t_first_submit, t_admit, t_launched, t_done_start, t_done_end;
    uint64_t n_digis;
    uint32_t n_events, stream;
    uint64_t t_pooled;  /* the batch's blocks taken from the pools */
    uint64_t t_inputs;  /* its input copies queued */
    uint64_t t_kernels; /* its kernels queued */
    /* device times (CUDA events on the batch's stream, ns from the earliest
     * traced batch's start; -1 if not taken): the batch's start, its inputs
     * copied, its kernels done, its outputs copied */
    int64_t gpu_start, gpu_inputs, gpu_kernels, gpu_outputs;
} hp_serve_trace_record;
hp_status hp_serve_trace_enable(hp_ctx *ctx, uint64_t cap);
hp_status hp_serve_trace_read(hp_ctx *ctx, hp_serve_trace_record *out, uint64_t cap, uint64_t *n);

hp_status hp_profile_enable(hp_ctx *ctx, uint32_t max_launches);
hp_status hp_profile_read(hp_ctx *ctx, uint32_t cap, const char **names, double *total_ms, uint64_t *launches,
                          uint32_t *n_kernels);

/*
 * Test hook (host-side fault injection): the next `count` pool allocations
 * of the context fail with HP_ENOMEM.
 */
hp_status hp_debug_fail_allocations(hp_ctx *ctx, uint32_t count);

/*
 * Test hook for failure detection: in the next `count` launches (host or
 * device entry; not serving batches or graphs captured later) the
 * clustering kernel keeps one work ticket's cluster count back, so its one
 * kind of device-side wait (the ordered output's wait for earlier tickets)
 * expires after its limit of one second instead of completing.  The launch
 * then ends normally with every event's status HP_ETIMEOUT (results
 * invalid), and the context stays usable.  Nothing faults or hangs.
 */
hp_status hp_debug_expire_waits(hp_ctx *ctx, uint32_t count);

#ifdef __cplusplus
}
#endif

#endif /* HP_H */
