// Host runtime of libisycos: the context, resident series, device work buffers and the
// batch engine that turns window lists into persistent MI launches.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <unordered_map>
#include <vector>

#include "isycos.h"
#include "isycos_internal.h"

namespace isy {

// Lane indices: searches use 0 .. kMaxLanes - 1 (default priority) and kPrioLaneBase + i
// (highest stream priority, for latency-bound searches); serving workers kServeLaneBase + w.
constexpr int kMaxLanes = 16;
constexpr int kMaxSeries = ISYCOS_MAX_SERIES;   // resident series per context
constexpr int kServeLaneBase = 32;
constexpr int kPrioLaneBase = 48;
constexpr int kLaneSlots = 64;


class Server;

// A growable device buffer whose bytes count against the context's budget.
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

// A growable pinned host buffer.
struct HostBuf {
    void *p = nullptr;     // pinned and mapped
    void *dev = nullptr;   // its device address
    size_t cap = 0;
};

// An independent engine lane: a stream with its own work buffers, so that several host
// threads can drive batches at once (one lane per thread).
struct Lane {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevBuf d_items, d_queue, d_out, d_nx, d_ny, d_c;
    DevBuf d_chain_desc, d_chain_steps, d_chain_state, d_chain_recomp, d_chain_out;
    DevBuf d_gscratch;                 // sorted-path scratch of windows above kSortMax points
    HostBuf h_items, h_table;          // pinned staging: table + items; results
    bool queue_clean = false;          // d_queue holds zeroed work counters
    int slot_share = 4;                // quarters of the GPU's resident-CTA slots a launch
                                       // of this lane may take (4: all)
    // the open launch of engine_launch
    struct Open {
        bool open = false;
        cudaStream_t st = nullptr;
        int64_t n = 0, pairs = 0, total_pts = 0;
        int32_t *nx = nullptr, *ny = nullptr, *c = nullptr;
        int32_t count[15] = {0};
        int max_m = 0;
        int64_t work_bf = 0, work_sort = 0;   // known from the sizes
        size_t work_off = 0;                   // byte offset of the device-counted work in h_table
    } open;
    std::vector<int32_t> h_slot;       // per-call bucket slots (reused)
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
};

// One window of a resident pair as the engine sees it (already validated).
struct HostWindow {
    int32_t xs, ys;
    int64_t start;
    int32_t m;
};

}  // namespace isy

struct isycos_ctx {
    int device = 0;
    int n_sm = 0;
    uint64_t budget = 0;
    std::atomic<uint64_t> used{0};
    cudaStream_t stream = nullptr;
    std::string err;
    mutable std::mutex err_mu;

    // 2^-32 fixed-point digamma and log tables (host copy and device copy).
    std::vector<long long> h_psi_fx, h_log_fx;
    long long *d_psi_fx = nullptr, *d_log_fx = nullptr;

    // Resident series.
    std::vector<float *> series_ptr;
    std::vector<int64_t> series_len;
    std::vector<size_t> series_cap;                  // bytes allocated for each series
    std::multimap<size_t, float *> series_pool;      // buffers of dropped series, by bytes
    std::atomic<uint64_t> series_bytes{0};           // device bytes of all series buffers
                                                     // (resident and kept), read by serving
    isy::DevBuf d_series_ptr, d_series_len;
    bool series_dirty = true;

    // Engine state (guarded by engine_mu; lanes other than 0 are driven by helper threads
    // while the calling thread holds engine_mu).
    std::mutex engine_mu;
    // engine lanes by index (created on first use by get_lane under lane_mu, never moved;
    // lane 0 uses `stream`)
    std::atomic<isy::Lane *> lanes[isy::kLaneSlots] = {};
    std::mutex lane_mu;
    int max_lanes = 8;
    isy::DevBuf d_table, d_slot, d_pos, d_bcount, d_status, d_plain_acc;
    isy::DevBuf d_dev_items, d_dev_queue, d_dev_table;   // asynchronous device-array path
    std::mutex launch_mu;                 // occupancy cache and function attributes
    std::unordered_map<uint64_t, int> occupancy;   // CTAs per SM by (k, threads, smem)
    size_t smem_set[2] = {0, 0};   // dynamic smem attribute set per (nt = 256, 1024), all k

    isycos_stats stats{};
    std::mutex stats_mu;
    cudaEvent_t ev_ref = nullptr;                        // origin of the kernel intervals
    std::vector<std::pair<float, float>> kernel_iv;      // MI kernel [start, stop] in ms

    // Options.
    int opt_kernel = 0;
    int opt_incremental = 1;
    int opt_estimator = 0;   // estimator of the direct window-MI entry points
    int opt_spec_climbs = 24; // SYCOS_BU climbs speculated ahead
    int opt_bu_device = 0;    // SYCOS_BU on the device (bu_device.cu)
    int64_t opt_time_limit_ms = 60000;   // device-resident searches: time limit per launch
    isy::DevBuf d_bu_q, d_bu_res, d_bu_found, d_bu_queue;   // device SYCOS_BU
    cudaEvent_t ev_bu[2] = {nullptr, nullptr};
    // sorted-path buckets chosen by isycos_autotune, per k (0: not tuned, use the default)
    uint32_t tuned_sort_mask[ISYCOS_MAX_K + 1] = {0};
    int tuned_sort_min[ISYCOS_MAX_K + 1] = {0};     // windows below it keep brute force
    int tuned_nt_switch[ISYCOS_MAX_K + 1] = {0};    // 0: 1024 (see batched_threads)
    bool tuned[ISYCOS_MAX_K + 1] = {false};
    int serve_slots = 64;
    int serve_queue = 100000;

    isy::Server *server = nullptr;
};

namespace isy {

// Error helpers: record a message on the context and return the status.
isycos_status fail(isycos_ctx *ctx, isycos_status st, const char *fmt, ...);
isycos_status cuda_fail(isycos_ctx *ctx, cudaError_t e, const char *what);

// Device buffer management with budget accounting.
isycos_status dev_reserve(isycos_ctx *ctx, DevBuf &b, size_t bytes);
void dev_release(isycos_ctx *ctx, DevBuf &b);
isycos_status host_reserve(isycos_ctx *ctx, HostBuf &b, size_t bytes);

// Validation of a window against the resident series (host side).
isycos_status check_window(isycos_ctx *ctx, const isycos_window &w, int k);

// Evaluate n windows (validated) with lane L's buffers on stream st, synchronously; results
// in input order into the host array `out`.  Per-point arrays (host) are optional.
isycos_status engine_eval(isycos_ctx *ctx, Lane &L, const HostWindow *w, int64_t n, int k,
                          isycos_mi_out *out, int32_t *nx, int32_t *ny, int32_t *c,
                          cudaStream_t st, int est = 0);
// The same in two halves: engine_launch stages and launches (asynchronous on st), and
// engine_collect waits for that launch and writes the results.  One launch per lane may be
// open at a time.
// The window [start, start + m - 1] of series xs and ys lies inside both series (and m is a
// valid window size for k).  The engines check every window they are given with it.
bool window_in_series(const isycos_ctx *ctx, int32_t xs, int32_t ys, int64_t start, int32_t m, int k);
isycos_status engine_launch(isycos_ctx *ctx, Lane &L, const HostWindow *w, int64_t n, int k,
                            int est, int32_t *nx, int32_t *ny, int32_t *c, cudaStream_t st);
isycos_status engine_collect(isycos_ctx *ctx, Lane &L, isycos_mi_out *out);

// Lane i of the context (created on first use; lane 0 runs on ctx->stream).
isycos_status get_lane(isycos_ctx *ctx, int i, Lane **out);

// Free a lane's device work buffers (they are allocated again on next use).
void lane_release(isycos_ctx *ctx, Lane &L);

void add_stats(isycos_ctx *ctx, int64_t windows, int64_t pairs, int64_t launches,
               int64_t batches, int64_t incr_windows);

cudaStream_t pick_stream(isycos_ctx *ctx, void *s);

// Size buckets whose windows take the sorted (sub-quadratic) MI path for k neighbours, the
// smallest window that takes it, and the largest sorted window of a 256-thread launch.
uint32_t sort_mask(const isycos_ctx *ctx, int k);
int sort_min_size(const isycos_ctx *ctx, int k);
int nt_switch(const isycos_ctx *ctx, int k);
// Tunings kept in the file named by ISYCOS_TUNING_FILE (autotune.cu): load this device's
// entries into the context; store one.
void load_tunings(isycos_ctx *ctx);
void store_tuning(const isycos_ctx *ctx, int k);

// A window sequence of one pair for the incremental kernel: result i goes to out[out_idx[i]]
// (out_idx < 0: evaluated for its state only, result dropped).
struct ChainSpec {
    int32_t xs = 0, ys = 0;
    std::vector<int64_t> starts;
    std::vector<int32_t> sizes;
    std::vector<int64_t> out_idx;
};

// Incremental evaluation of chains (chain.cu), one CTA per chain segment, synchronous;
// results into the host array out of n_out entries.  Caller holds engine_mu.
isycos_status engine_eval_chains(isycos_ctx *ctx, Lane &L, const ChainSpec *specs, size_t n_specs,
                                 int k, isycos_mi_out *out, int64_t n_out, cudaStream_t st);

// Stop and free the serving thread of a context (serve.cu).
void serve_shutdown(isycos_ctx *ctx);

}  // namespace isy
