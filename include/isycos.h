/*
 * isycos.h -- C ABI of libisycos.so, the GB300 (sm_103a) window-MI engine for iSYCOS
 * (Ho et al., "A Unified Approach for Multi-Scale Synchronous Correlation Search in Big
 * Time Series", arXiv 2204.09131).
 *
 * The library evaluates the window-level KSG mutual information of two time series over
 * many candidate windows (series pair, start, size) on the GPU, and runs the paper's
 * top-down (SYCOS_TD, Algorithm 1) and bottom-up (SYCOS_BU, Algorithm 2) searches with
 * the MI-based noise pruning of Sec. 6 on top of it, one query at a time or as a served
 * stream of queries.
 *
 * Conventions for every call:
 *  - Return value: ISYCOS_OK (0), a negative error code, or ISYCOS_PENDING (> 0, polling).
 *    After an error, isycos_last_error() describes it.
 *  - The caller owns every buffer it passes.  The library owns the resident series and
 *    its device work memory, allocated at isycos_create / isycos_put_series / first use
 *    and released by isycos_destroy.
 *  - "host" pointers are ordinary (pageable or pinned) CPU memory; "device" pointers are
 *    CUDA device memory of the context's device (e.g. torch tensors' data_ptr()).
 *  - cuda_stream is a cudaStream_t of the context's device, or NULL for the library's
 *    own stream.
 *  - A context is not thread-safe, except isycos_serve_submit / isycos_serve_poll /
 *    isycos_serve_cancel, which may be called from any thread.
 *  - Windows are inclusive ranges [start, start + m - 1] of 0-based time indices
 *    (Def. 3.2: a window of size m holds m values); search ranges are half-open
 *    [t_begin, t_end).
 */
#ifndef ISYCOS_H
#define ISYCOS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t isycos_status;

#define ISYCOS_OK 0
#define ISYCOS_E_INVAL (-1)    /* bad argument: size, range, pointer, parameter      */
#define ISYCOS_E_NOMEM (-2)    /* device memory or the context's budget exhausted    */
#define ISYCOS_E_CUDA (-3)     /* a CUDA call failed (message in isycos_last_error)  */
#define ISYCOS_E_TIMEOUT (-4)  /* a bounded device wait ran out                      */
#define ISYCOS_E_TRUNC (-5)    /* output capacity too small; *n_out holds the need   */
#define ISYCOS_E_AGAIN (-6)    /* serving: admission queue full, retry later         */
#define ISYCOS_E_NOTFOUND (-7) /* unknown series id or ticket                        */
#define ISYCOS_E_CANCELED (-8) /* serving: the query was cancelled                   */
#define ISYCOS_PENDING 1       /* serving: the query has not finished yet            */

/* Largest window size the kernels accept (one window's two series fit in shared memory). */
#define ISYCOS_MAX_M 16384
/* Largest number of neighbours k. */
#define ISYCOS_MAX_K 8
/* Largest LAHC idle limit T_maxIdle of SYCOS_BU (its rings reach N_{T_maxIdle + 1}). */
#define ISYCOS_MAX_IDLE 64
/* Most series resident in one context at a time. */
#define ISYCOS_MAX_SERIES (1 << 20)

typedef struct isycos_ctx isycos_ctx;

/* One candidate window of a pair of resident series (Def. 3.4: a synchronous pair of
 * windows [start, start + m - 1] of series xs and ys).  24 bytes. */
typedef struct {
    int32_t xs;        /* series id of X                                   */
    int32_t ys;        /* series id of Y                                   */
    int64_t start;     /* first time index                                  */
    int32_t m;         /* window size, k + 1 <= m <= ISYCOS_MAX_M           */
    int32_t reserved;  /* must be 0                                         */
} isycos_window;

/* Result for one window.  40 bytes.
 *  mi    : Eq. KSGmi (Sec. 4.2), Kraskov's second estimator under the max-norm, in nats:
 *          psi(k) - 1/k + psi(m) - (1/m) sum_i [psi(n_x,i) + psi(n_y,i)]
 *  h_w   : plug-in joint entropy of the window's (x, y) values (Sec. 5.4),
 *          ln m - (1/m) sum_i ln c_i, c_i the multiplicity of (x_i, y_i)
 *  nmi   : mi / h_w (Eq. normalizedMI), 0 when h_w == 0
 *  s_psi : sum_i psi_fx[n_x,i] + psi_fx[n_y,i], psi_fx[n] = round(psi(n) 2^32)
 *  s_log : sum_i log_fx[c_i], log_fx[c] = round(ln(c) 2^32)
 * The scalars are evaluated in binary64 from the exact integer sums in the fixed order
 * ((psi(k) - 1/k) + psi(m)) - (s_psi 2^-32) / m, with psi(k), psi(m), ln m taken from the
 * same 2^-32 tables, so that every value is reproducible bit for bit. */
typedef struct {
    double mi;
    double h_w;
    double nmi;
    int64_t s_psi;
    int64_t s_log;
} isycos_mi_out;

/* Search parameters (Algorithms 1-3 and Sec. 6).  Zero / negative fields take the
 * defaults noted; isycos_params_default() fills every field. */
typedef struct {
    int32_t k;           /* KSG neighbours, 1..ISYCOS_MAX_K (default 4)                  */
    int32_t score_kind;  /* 0: normalised I/H (Sec. 5.4, default); 1: raw I in nats      */
    double sigma;        /* correlation threshold (Def. 3.5), default 0.2                */
    double tau;          /* noise threshold (Def. 6.2); < 0: sigma / 4 (Sec. 8.3)        */
    int32_t s_min;       /* smallest window size, >= k + 1                               */
    int32_t s_max;       /* largest window size, <= ISYCOS_MAX_M                         */
    int32_t delta_td;    /* TD sliding step; <= 0: max(k + 1, s_w / 4) per layer         */
    int32_t delta_bu;    /* BU moving step; <= 0: max(1, s_min / 4)                      */
    int32_t h;           /* LAHC history length; <= 0: 8                                 */
    int32_t t_max_idle;  /* LAHC idle limit; < 0: 3; > ISYCOS_MAX_IDLE: ISYCOS_E_INVAL    */
    int32_t p;           /* consecutive noise detections before pruning; <= 0: 3         */
    int32_t mode;        /* 0: SYCOS_TD, 1: SYCOS_BU, 2: iSYCOS selection (Alg. 3)       */
    int32_t pruning;     /* 0 off, 1 noise pruning (Sec. 6) on                           */
    int32_t max_steps;   /* LAHC steps per climb; <= 0: 10000                            */
    uint64_t seed;       /* seed of the LAHC history-index stream and of Alg. 3 sampling  */
    int32_t sel_partitions; /* Alg. 3: M equal partitions of the range; <= 0: 20           */
    int32_t sel_samples;    /* Alg. 3: m partitions sampled; <= 0: 6                       */
    double sel_alpha;       /* Alg. 3: weight of the runtime factor; < 0: 0.5               */
    double sel_rho;         /* Alg. 3: a window is small iff size <= rho * s_max; <= 0: 0.5 */
    int32_t chunks;         /* Alg. 4: n_p overlapping chunks searched independently
                               (chunk i = [i L - s_max, (i + 1) L) of the range, L = floor(
                               length / n_p), clipped); their windows concatenated and
                               sorted by t_s, so windows of different chunks may overlap;
                               <= 1: one search over the whole range                    */
    int32_t estimator;      /* 0: Kraskov estimator 2 (default); 1: Kraskov estimator 1    */
} isycos_params;   /* 104 bytes */

/* One correlated window found by a search.  32 bytes. */
typedef struct {
    int64_t t_s;
    int64_t t_e;      /* inclusive end                                   */
    double score;     /* the value compared with sigma (nmi or mi)        */
    double mi;        /* raw MI in nats                                   */
} isycos_result_window;

/* Counters since isycos_create (or the last isycos_reset_stats). */
typedef struct {
    int64_t windows;        /* window MIs evaluated on the GPU                        */
    int64_t pairs;          /* brute-force-equivalent ordered pairs, sum m (m - 1)    */
    int64_t launches;       /* kernels launched by the library                        */
    int64_t batches;        /* batched evaluations (one or more launches each)        */
    int64_t incr_windows;   /* windows evaluated by the incremental update            */
    int64_t incr_full_points; /* points whose neighbours the incremental update searched
                               again in full (the rest took +-1 count updates)       */
    int64_t queries_done;   /* served queries completed                               */
    int64_t decided_windows;/* window scores read by the searches' decisions: the count
                               of MI evaluations the sequential Algorithms 1 and 2
                               make (speculatively evaluated windows that no decision
                               read are in `windows` only)                          */
    double mi_kernel_ms;    /* device busy time of the batched MI kernels: the union of
                               their [start, stop] intervals (CUDA events on each
                               launching stream; concurrent launches counted once)    */
    int64_t mi_kernel_launches; /* launches timed in mi_kernel_ms                      */
    /* Per size bucket b = 0 .. 14 (windows with 2^(b-1) < m <= 2^b; b = 0: m = 1):      */
    int64_t windows_by_size[15];   /* batched windows evaluated                          */
    int64_t launches_by_size[15];  /* batched launches whose largest window is in b       */
    double launch_ms_by_size[15];  /* their event-timed durations, summed (not a union)   */
    int64_t decided_by_size[15];   /* decided_windows by the same size buckets            */
    /* Device-resident searches (ISYCOS_OPT_BU_DEVICE): */
    int64_t dev_queries;           /* queries searched                                   */
    int64_t dev_rounds;            /* decide / evaluate rounds, summed over queries      */
    int64_t dev_cycles[3];         /* SM cycles of their CTAs in decide + ask, evaluate,
                                      finish (clock64 of the CTA's first thread)          */
    /* Work the MI kernels did, in the units of the method's own algorithm (the roofline of
     * the work actually run, not of a brute-force equivalent): */
    int64_t work_bf;               /* brute-force passes: point x candidate distance
                                      evaluations (pass 1 and pass 2 count once together) */
    int64_t work_scan;             /* sorted path, phase A: point x candidate visits of the
                                      outward scans                                       */
    int64_t work_search;           /* sorted path, phase B: binary-search steps and
                                      duplicate-scan steps, per point                     */
    int64_t work_sort;             /* sorted path: compare-exchange steps of the bitonic
                                      sorts, per element pair                             */
} isycos_stats;   /* 632 bytes */

/* Create a context on CUDA device `device`.  mem_budget_bytes caps the device memory the
 * context may hold for series and work buffers (0: 90% of the free memory at creation).
 * Errors: E_INVAL (bad device / NULL out), E_CUDA, E_NOMEM. */
isycos_status isycos_create(isycos_ctx **out, int32_t device, uint64_t mem_budget_bytes);

/* Stop the serving thread, free every device and host resource, and free ctx. */
isycos_status isycos_destroy(isycos_ctx *ctx);

/* NUL-terminated description of the last error on this context (never NULL). */
const char *isycos_last_error(const isycos_ctx *ctx);

/* Fill p with the defaults listed in isycos_params. */
void isycos_params_default(isycos_params *p);

/* Make a series resident (Def. 3.1): copies n float32 values from `data` (device memory if
 * on_device != 0, else host memory) into library-owned device memory and returns its id.
 * Non-finite values are rejected (E_INVAL): the estimator's distances need finite input.
 * May be called while served queries run (they only read the series they named).
 * Errors: E_INVAL (n < 1, NULL, non-finite), E_NOMEM (budget, or ISYCOS_MAX_SERIES series
 * resident), E_CUDA. */
isycos_status isycos_put_series(isycos_ctx *ctx, const float *data, int64_t n,
                                int32_t on_device, int32_t *series_id);

/* Make count series resident in one call: series s is data[s][0 .. n[s] - 1] (device memory
 * if on_device != 0, else host memory); series_ids[s] receives its id.  The copies are
 * queued together and the call synchronises once (isycos_put_series synchronises per
 * series).  Same checks and errors as isycos_put_series; on any error no series of the call
 * is made resident. */
isycos_status isycos_put_series_many(isycos_ctx *ctx, int32_t count, const float *const *data,
                                     const int64_t *n, int32_t on_device, int32_t *series_ids);

/* Release a resident series.  Its device memory is kept by the context for a later series of
 * about its size (so that a put / drop cycle allocates nothing), and freed by isycos_destroy
 * or when the context's budget needs it.  A call still reading the series must have
 * completed (every synchronous call has).  Errors: E_NOTFOUND. */
isycos_status isycos_drop_series(isycos_ctx *ctx, int32_t series_id);

/* Device address and length of a resident series (read-only for the caller). */
isycos_status isycos_series_info(isycos_ctx *ctx, int32_t series_id, const float **device_ptr,
                                 int64_t *n);

/* Window-level KSG MI (Sec. 4.2 Eq. KSGmi, Def. 4.2; counting rule of the Sec. 7.1
 * example; score of Sec. 5.4) for n_w windows, batched on the GPU in size buckets by one
 * persistent launch.
 *   windows : host array of n_w windows
 *   k       : neighbours, 1..ISYCOS_MAX_K
 *   out     : host array of n_w results, written in input order
 * Synchronous: returns when `out` is written.
 * Errors: E_INVAL (any window out of range, m < k + 1, m > ISYCOS_MAX_M, unknown series,
 *         reserved != 0; nothing is written), E_NOMEM, E_CUDA. */
isycos_status isycos_mi_windows(isycos_ctx *ctx, const isycos_window *windows, int64_t n_w,
                                int32_t k, isycos_mi_out *out, void *cuda_stream);

/* As isycos_mi_windows, with both arrays in device memory.  Asynchronous on cuda_stream:
 * the call enqueues validation, bucketing and the persistent MI kernel and returns.  Its
 * work buffers belong to the context: two such calls must not overlap on different streams
 * (calls on one stream are ordered), and dropping a series that a pending call reads is an
 * error of the caller.
 *   max_m : an upper bound of the windows' sizes (sizes the kernel's shared memory)
 * Invalid windows are detected on the device: their results are NaN and the next call
 * of isycos_device_status() reports E_INVAL. */
isycos_status isycos_mi_windows_device(isycos_ctx *ctx, const isycos_window *d_windows,
                                       int64_t n_w, int32_t k, int32_t max_m,
                                       isycos_mi_out *d_out, void *cuda_stream);

/* Synchronise cuda_stream and report (then clear) errors flagged by device-side checks
 * of earlier asynchronous calls.  Returns ISYCOS_OK, E_INVAL or E_CUDA. */
isycos_status isycos_device_status(isycos_ctx *ctx, void *cuda_stream);

/* As isycos_mi_windows, also returning the per-point integers that the MI is built from,
 * for parity checks.  nx, ny, c: host arrays of sum_w m_w entries, window after window in
 * input order, point i of a window at offset i:
 *   nx[i] = #{j != i : |x_i - x_j| <= d_x,i},  ny likewise,  c[i] = #{j : (x_j,y_j) = (x_i,y_i)}
 * where d_x,i, d_y,i are the largest per-dimension distances from point i to its k nearest
 * neighbours (max-norm, ties broken toward the smaller time index). */
isycos_status isycos_mi_windows_points(isycos_ctx *ctx, const isycos_window *windows,
                                       int64_t n_w, int32_t k, isycos_mi_out *out,
                                       int32_t *nx, int32_t *ny, int32_t *c,
                                       void *cuda_stream);

/* The plain form: one window per kernel launch (the window's points spread over CTAs,
 * sums combined by the last CTA).  Same results as isycos_mi_windows; it exists as the
 * baseline that the batched form is measured against.  Host arrays, synchronous. */
isycos_status isycos_mi_windows_plain(isycos_ctx *ctx, const isycos_window *windows,
                                      int64_t n_w, int32_t k, isycos_mi_out *out,
                                      void *cuda_stream);

/* Incremental window MI (Sec. 7.1, influenced regions, Lemmas 3-6): evaluates the windows
 * [starts[i], starts[i] + sizes[i] - 1], i = 0 .. n_steps - 1, of one pair in order,
 * deriving each window's neighbour state from the previous window's by the removed and
 * added points: a point keeps its neighbours unless a removed or added point lies in its
 * influenced region (the closed square of half-side eps_i around it), in which case its
 * neighbours are searched again; marginal counts change by one for each removed or added
 * point inside its influenced marginal regions.  Results equal isycos_mi_windows bit for
 * bit.  A long sequence is cut into segments (at least 16 windows each) that run in
 * parallel, each starting from scratch.  Host arrays, synchronous.
 * Errors: as isycos_mi_windows. */
isycos_status isycos_mi_chain(isycos_ctx *ctx, int32_t xs, int32_t ys, const int64_t *starts,
                              const int32_t *sizes, int64_t n_steps, int32_t k,
                              isycos_mi_out *out, void *cuda_stream);

/* Correlation search on one pair (Sec. 3, the SYCOS problem): all non-overlapping windows
 * [t_s, t_e] inside [t_begin, t_end) with s_min <= size <= s_max whose score >= sigma, found
 * by SYCOS_TD (Algorithm 1) or SYCOS_BU (Algorithm 2) per params->mode, with the noise
 * pruning of Sec. 6 when params->pruning.  Window MIs run on the GPU in batches (TD: all
 * sliding positions of a layer at once, then the sequential decisions are replayed; BU:
 * one neighbourhood ring per step).  Output sorted by t_s.
 *   out, cap : host array of capacity cap; *n_out receives the number of windows found
 * Errors: E_INVAL, E_NOTFOUND (series), E_TRUNC (cap too small; *n_out = needed), E_CUDA. */
isycos_status isycos_search(isycos_ctx *ctx, int32_t xs, int32_t ys, int64_t t_begin,
                            int64_t t_end, const isycos_params *params,
                            isycos_result_window *out, int64_t cap, int64_t *n_out);

/* Searches on many pairs at once: n_q independent queries (xs[i], ys[i], t_begin[i],
 * t_end[i]) with shared params; their frontiers are merged into common batches.
 * Results of query i go to out + offsets[i] .. out + offsets[i] + n_out[i] - 1, where
 * offsets[i] = i * cap_per_query.  Errors as isycos_search (E_TRUNC if any query overflows). */
isycos_status isycos_search_many(isycos_ctx *ctx, int64_t n_q, const int32_t *xs,
                                 const int32_t *ys, const int64_t *t_begin,
                                 const int64_t *t_end, const isycos_params *params,
                                 isycos_result_window *out, int64_t cap_per_query,
                                 int64_t *n_out);

/* One search query: a pair, a range [t_begin, t_end) and its own parameters. */
typedef struct {
    int32_t xs;
    int32_t ys;
    int64_t t_begin;
    int64_t t_end;
    isycos_params params;
} isycos_query;

/* As isycos_search_many, with parameters per query (e.g. SYCOS_TD and SYCOS_BU queries of the
 * same pairs in one call: their frontiers run concurrently and share the GPU).  Results of
 * query i go to out + i * cap_per_query; n_out[i] receives their number. */
isycos_status isycos_search_queries(isycos_ctx *ctx, int64_t n_q, const isycos_query *queries,
                                    isycos_result_window *out, int64_t cap_per_query,
                                    int64_t *n_out);

/* Serving (continuous batching).  submit enqueues a search query and returns a ticket at
 * once; a library thread admits queued queries while device memory allows, merges the
 * window frontiers of all admitted queries into shared GPU batches, and completes them
 * independently.  Errors: E_INVAL, E_NOTFOUND (series), E_AGAIN (queue full). */
isycos_status isycos_serve_submit(isycos_ctx *ctx, int32_t xs, int32_t ys, int64_t t_begin,
                                  int64_t t_end, const isycos_params *params,
                                  uint64_t *ticket);

/* Poll a ticket.  Returns ISYCOS_PENDING while the query runs; on completion writes the
 * windows (as isycos_search), the latency from submit to completion in milliseconds, and
 * releases the ticket.  E_TRUNC leaves the ticket in place with *n_out = needed. */
isycos_status isycos_serve_poll(isycos_ctx *ctx, uint64_t ticket, isycos_result_window *out,
                                int64_t cap, int64_t *n_out, double *latency_ms);

/* As isycos_serve_poll, also returning the query's admission wait: the milliseconds from
 * submission until a slot and device memory were free and the query joined the running
 * ones (wait_ms may be NULL). */
isycos_status isycos_serve_poll_ex(isycos_ctx *ctx, uint64_t ticket, isycos_result_window *out,
                                   int64_t cap, int64_t *n_out, double *latency_ms,
                                   double *wait_ms);

/* Cancel a queued or running query; a later poll returns E_CANCELED. */
isycos_status isycos_serve_cancel(isycos_ctx *ctx, uint64_t ticket);

/* Counters (see isycos_stats). */
isycos_status isycos_get_stats(isycos_ctx *ctx, isycos_stats *out);
isycos_status isycos_reset_stats(isycos_ctx *ctx);

/* Copy the library's fixed-point tables (psi_fx, log_fx as in isycos_mi_out) for
 * n = 0 .. n_max (n_max <= ISYCOS_MAX_M + 1) to host arrays of n_max + 1 entries. */
isycos_status isycos_tables(isycos_ctx *ctx, int32_t n_max, int64_t *psi_fx, int64_t *log_fx);

/* Autotuner.  The paper has no counterpart: its kNN search is a CPU index (Sec. 7.1).  For
 * k neighbours, times launches on a seeded probe pair (x ~ N(0,1), y = 0.6 x + 0.8 N(0,1),
 * 65,536 points, uploaded and dropped by the call) and keeps, for this context and k (used
 * while ISYCOS_OPT_KERNEL is 0, the default):
 *  - the faster of the brute-force and sorted-strip MI paths per size bucket the sorted path
 *    can take (257..16384 points), each timed on n_windows windows of the bucket's middle
 *    size (fewer for the two largest buckets);
 *  - the crossover inside the smallest sorted bucket: windows below sort_min keep the
 *    brute-force path (probed at 1/8, 2/8 and 3/8 into the bucket);
 *  - nt_switch: launches whose largest sorted window exceeds it run 1024-thread CTAs, others
 *    256-thread CTAs (512 or 1024, timed on windows of 768 points when their bucket is
 *    sorted).
 * Results are identical on every choice; only speed changes.  Statistics are left as they
 * were.  When the environment names a file in ISYCOS_TUNING_FILE, the choice is stored there
 * under the GPU's name and k (one line of JSON per entry), and isycos_create loads the
 * entries of its GPU from it.  out may be NULL.
 * Errors: E_INVAL (k), E_NOMEM (budget), E_CUDA. */
typedef struct {
    int32_t k;
    uint32_t sorted_buckets;   /* bit b set: windows with 2^(b-1) < m <= 2^b take the sorted
                                  path                                                      */
    int32_t window_size[15];   /* probe window size per bucket (0: bucket not probed)       */
    int32_t n_windows;         /* windows per probe launch (8 per SM; 2 and 1 per SM for the
                                  buckets of 4097..8192 and 8193..16384 points)             */
    double brute_ms[15];       /* best of three launch times, brute-force path               */
    double sorted_ms[15];      /* best of three launch times, sorted-strip path              */
    int32_t sort_min;          /* smallest window size that takes the sorted path           */
    int32_t nt_switch;         /* largest sorted window of a 256-thread launch               */
    int32_t cross_size[3];     /* crossover probe sizes (0: not probed)                      */
    int32_t pad;
    double cross_brute_ms[3];  /* their launch times, brute force and sorted                 */
    double cross_sorted_ms[3];
    double nt_ms[2];           /* 768-point sorted windows in 256- and 1024-thread CTAs      */
} isycos_tuning;   /* 400 bytes */
isycos_status isycos_autotune(isycos_ctx *ctx, int32_t k, isycos_tuning *out);

/* The tuning a context uses for k (from isycos_autotune or the tuning file): sorted buckets
 * (bits as in isycos_tuning), sort_min and nt_switch.  E_NOTFOUND when k is not tuned (the
 * defaults apply: buckets of 1025..16384 points sorted, sort_min 0, nt_switch 1024). */
isycos_status isycos_get_tuning(isycos_ctx *ctx, int32_t k, uint32_t *sorted_buckets,
                                int32_t *sort_min, int32_t *nt_switch);

/* Options (isycos_set_option).  Values are documented per option. */
#define ISYCOS_OPT_KERNEL 1        /* 0 auto (default: the buckets isycos_autotune chose, else
                                      sorted for 1025..16384 points), 1 brute force, 2 sorted
                                      for every window of 257..16384 points                 */
#define ISYCOS_OPT_INCREMENTAL 2   /* searches: 0 off, 1 auto (default), 2 always           */
#define ISYCOS_OPT_SERVE_SLOTS 3   /* serving: most queries admitted at once (default 64)   */
#define ISYCOS_OPT_SERVE_QUEUE 4   /* serving: most queries waiting (default 100000)        */
#define ISYCOS_OPT_LANES 5         /* searches: most engine lanes (host thread + stream +
                                      work buffers), 1 .. 16 (default: the host cores, at
                                      most 16); a call that mixes SYCOS_TD with other
                                      queries gives a quarter of them to the TD queries     */
#define ISYCOS_OPT_ESTIMATOR 6     /* estimator of isycos_mi_windows, _points, _device and
                                      _plain: 0 Kraskov's second (Eq. KSGmi, default), 1
                                      Kraskov's first, psi(k) + psi(m) - <psi(n_x + 1) +
                                      psi(n_y + 1)> with strict counts in strips of half-width
                                      eps_i (searches take isycos_params.estimator)          */
#define ISYCOS_OPT_SPECULATION 7   /* SYCOS_BU: climbs whose first windows are asked ahead,
                                      assuming each ends where it starts; 0 .. 64 (default
                                      24).  Changes the GPU work only, never the results     */
#define ISYCOS_OPT_BU_DEVICE 8     /* SYCOS_BU queries of isycos_search / _many / _queries:
                                      1 the whole search runs on the GPU, one launch for all
                                      BU queries of a call, every LAHC decision made on the
                                      device next to the window MIs it reads (one CTA per
                                      query); 0 (default) the host search machines, one launch
                                      per round of all queries' windows over the whole GPU.
                                      Same results either way; queries with h > 64,
                                      t_max_idle > 31, chunks or selection, and every query
                                      while ISYCOS_OPT_INCREMENTAL is 2, take the host
                                      machines                                              */
#define ISYCOS_OPT_TIME_LIMIT_MS 9 /* device-resident searches: a launch stops once it has run
                                      this long (milliseconds, checked between rounds against
                                      the GPU's global timer) and the call returns
                                      ISYCOS_E_TIMEOUT with no windows; 0 = no limit (default
                                      60000)                                                */
isycos_status isycos_set_option(isycos_ctx *ctx, int32_t option, int64_t value);

/* Window MI that allocates nothing.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc -- code running under a runtime that owns
 * all device memory (a framework's caching allocator, a process held to a fixed device
 * budget it hands out itself) and latency-critical loops where cudaMalloc / cudaFree would
 * synchronise the device.  It needs no context and evaluates the same MI as
 * isycos_mi_windows_device with the same persistent kernel, for windows of ONE pair:
 *   d_x, d_y : device arrays of n float32 values (finite; not checked here)
 *   d_starts : device array of n_w window starts (int64); d_sizes: n_w sizes (int32)
 *   k, max_m : as for isycos_mi_windows_device (max_m bounds every size)
 *   d_out    : device array of n_w results, input order
 * Its work memory (window items, bucket table, counters; about 2.6 MiB) is one static
 * device array, and its tables are static device arrays: every GPU that loads the library
 * holds them until the process exits.  The first call on a device (with that device
 * current) resolves the array's address with cudaGetSymbolAddress and uploads the tables,
 * so it should come before any stream capture.  Calls share the array, which keeps the last
 * call's contents: calls that overlap on the GPU race.  Every window takes the brute-force
 * MI path (the sorted path's work memory would not fit a static array of modest size), so
 * windows above about 1,000 points run slower than through a context that chose the sorted
 * path; results are the same.  Asynchronous on cuda_stream: windows outside [0, n) or with
 * m < k + 1 or m > max_m get NaN mi, h_w and nmi and zero sums, which is the only report of
 * them (the call reads nothing back from the device).
 * Errors: E_INVAL (k, max_m, NULL pointers, or n_w > ISYCOS_NOALLOC_MAX_WINDOWS, the size
 * of the static scratch), E_CUDA. */
#define ISYCOS_NOALLOC_MAX_WINDOWS 65536
isycos_status isycos_mi_windows_noalloc(const float *d_x, const float *d_y, int64_t n,
                                        const int64_t *d_starts, const int32_t *d_sizes,
                                        int64_t n_w, int32_t k, int32_t max_m,
                                        isycos_mi_out *d_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* ISYCOS_H */
