// Host runtime of libisycos: context, resident series, window-MI entry points.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <thread>
#include <vector>

#include "runtime.h"

using namespace isy;

namespace isy {

isycos_status fail(isycos_ctx *ctx, isycos_status st, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        std::lock_guard<std::mutex> g(ctx->err_mu);
        ctx->err = buf;
    }
    return st;
}

isycos_status cuda_fail(isycos_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, ISYCOS_E_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

isycos_status dev_reserve(isycos_ctx *ctx, DevBuf &b, size_t bytes) {
    if (bytes <= b.cap) return ISYCOS_OK;
    size_t want = std::max(bytes, b.cap + b.cap / 2);
    want = (want + 255) & ~(size_t)255;
    if (ctx->used.load() - b.cap + want > ctx->budget) {
        want = (bytes + 255) & ~(size_t)255;
        if (ctx->used.load() - b.cap + want > ctx->budget)
            return fail(ctx, ISYCOS_E_NOMEM, "device budget exceeded: need %zu more bytes",
                        want - b.cap);
    }
    if (b.p) {
        cudaFree(b.p);
        ctx->used -= b.cap;
        b.p = nullptr;
        b.cap = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, ISYCOS_E_NOMEM, "cudaMalloc(%zu): %s", want, cudaGetErrorString(e));
    }
    b.p = p;
    b.cap = want;
    ctx->used += want;
    return ISYCOS_OK;
}

void dev_release(isycos_ctx *ctx, DevBuf &b) {
    if (b.p) {
        cudaFree(b.p);
        ctx->used -= b.cap;
    }
    b.p = nullptr;
    b.cap = 0;
}

isycos_status host_reserve(isycos_ctx *ctx, HostBuf &b, size_t bytes) {
    if (bytes <= b.cap) return ISYCOS_OK;
    size_t want = std::max(bytes, b.cap + b.cap / 2);
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.dev = nullptr;
    b.cap = 0;
    cudaError_t e = cudaHostAlloc(&b.p, want, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaHostAlloc");
    e = cudaHostGetDevicePointer(&b.dev, b.p, 0);
    if (e != cudaSuccess) {
        cudaFreeHost(b.p);
        b.p = nullptr;
        return cuda_fail(ctx, e, "cudaHostGetDevicePointer");
    }
    b.cap = want;
    return ISYCOS_OK;
}

void add_stats(isycos_ctx *ctx, int64_t windows, int64_t pairs, int64_t launches,
               int64_t batches, int64_t incr_windows) {
    std::lock_guard<std::mutex> g(ctx->stats_mu);
    ctx->stats.windows += windows;
    ctx->stats.pairs += pairs;
    ctx->stats.launches += launches;
    ctx->stats.batches += batches;
    ctx->stats.incr_windows += incr_windows;
}

cudaStream_t pick_stream(isycos_ctx *ctx, void *s) {
    return s ? reinterpret_cast<cudaStream_t>(s) : ctx->stream;
}

isycos_status check_window(isycos_ctx *ctx, const isycos_window &w, int k) {
    const int64_t ns = (int64_t)ctx->series_ptr.size();
    if (w.reserved != 0) return fail(ctx, ISYCOS_E_INVAL, "window.reserved must be 0");
    if (w.xs < 0 || w.xs >= ns || !ctx->series_ptr[w.xs] || w.ys < 0 || w.ys >= ns ||
        !ctx->series_ptr[w.ys])
        return fail(ctx, ISYCOS_E_INVAL, "unknown series id (%d, %d)", w.xs, w.ys);
    if (w.m < k + 1 || w.m > kMaxM)
        return fail(ctx, ISYCOS_E_INVAL, "window size %d outside [k + 1 = %d, %d]", w.m, k + 1, kMaxM);
    const int64_t n = std::min(ctx->series_len[w.xs], ctx->series_len[w.ys]);
    if (w.start < 0 || w.start + w.m > n)
        return fail(ctx, ISYCOS_E_INVAL, "window [%lld, %lld] outside the series (length %lld)",
                    (long long)w.start, (long long)(w.start + w.m - 1), (long long)n);
    return ISYCOS_OK;
}

// Buckets that take the sorted (sub-quadratic) path: ISYCOS_OPT_KERNEL 1 keeps everything on
// the brute-force path, 2 sends every eligible window (257..kSortMax points, one per CTA) to
// the sorted path, 0 (auto) uses the buckets isycos_autotune chose for k, else 1025..4096.
uint32_t sort_mask(const isycos_ctx *ctx, int k) {
    if (ctx->opt_kernel == 1) return 0;
    if (ctx->opt_kernel == 2) return kSortBuckets;
    if (k >= 1 && k <= kMaxK && ctx->tuned[k]) return ctx->tuned_sort_mask[k];
    return kDefaultSortBuckets;
}

int sort_min_size(const isycos_ctx *ctx, int k) {
    if (ctx->opt_kernel != 0 || k < 1 || k > kMaxK || !ctx->tuned[k]) return 0;
    return ctx->tuned_sort_min[k];
}

int nt_switch(const isycos_ctx *ctx, int k) {
    if (ctx->opt_kernel != 0 || k < 1 || k > kMaxK || !ctx->tuned[k] || ctx->tuned_nt_switch[k] <= 0) return 1024;
    return ctx->tuned_nt_switch[k];
}

// Build the persistent launch's bucket table for items already sorted by slot.
static void build_table(BucketTable &T, const int32_t *count, int nt) { fill_bucket_table(&T, count, nt); }

// The batched kernels' dynamic shared-memory limit is a property of the function, shared by
// every thread and context of the process: it is set once to the device's maximum (less room
// for the kernels' static shared memory), the same value every caller sets, and never
// lowered, so that a launch on one lane cannot find the limit lowered by another.
static isycos_status ensure_smem(isycos_ctx *ctx, int k, int nt, size_t smem) {
    std::lock_guard<std::mutex> g(ctx->launch_mu);
    int idx = nt == 1024 ? 1 : 0;
    if (smem <= ctx->smem_set[idx]) return ISYCOS_OK;
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaDeviceGetAttribute");
    const size_t limit = (size_t)optin - 1024;
    if (smem > limit) return fail(ctx, ISYCOS_E_INVAL, "a launch needs %zu bytes of shared memory", smem);
    for (int kk = 1; kk <= kMaxK; ++kk) {
        e = set_batched_smem(kk, nt, limit);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute");
    }
    (void)k;
    ctx->smem_set[idx] = limit;
    return ISYCOS_OK;
}

static isycos_status launch_grid(isycos_ctx *ctx, int k, int nt, size_t smem, int jobs_hint,
                                 int share, int *grid) {
    int per_sm = 0;
    const uint64_t key = ((uint64_t)k << 48) | ((uint64_t)nt << 32) | (uint64_t)smem;
    std::lock_guard<std::mutex> g(ctx->launch_mu);
    auto it = ctx->occupancy.find(key);
    if (it != ctx->occupancy.end()) {
        per_sm = it->second;
    } else {
        cudaError_t e = batched_occupancy(k, nt, smem, &per_sm);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "occupancy");
        ctx->occupancy[key] = per_sm;
    }
    if (per_sm < 1) return fail(ctx, ISYCOS_E_INVAL, "kernel does not fit on an SM (smem %zu)", smem);
    int gsz = ctx->n_sm * per_sm;
    if (share > 0 && share < 4) gsz = std::max(1, gsz * share / 4);
    if (jobs_hint > 0 && jobs_hint < gsz) gsz = jobs_hint;
    *grid = std::max(gsz, 1);
    return ISYCOS_OK;
}

bool window_in_series(const isycos_ctx *ctx, int32_t xs, int32_t ys, int64_t start, int32_t m, int k) {
    const int32_t ns = (int32_t)ctx->series_len.size();
    if (xs < 0 || xs >= ns || ys < 0 || ys >= ns || m < k + 1 || m > kMaxM || start < 0) return false;
    return start + m <= std::min(ctx->series_len[(size_t)xs], ctx->series_len[(size_t)ys]);
}

isycos_status engine_launch(isycos_ctx *ctx, Lane &L, const HostWindow *w, int64_t n, int k,
                            int est, int32_t *nx, int32_t *ny, int32_t *c, cudaStream_t st) {
    L.open.open = false;
    if (n <= 0) return ISYCOS_OK;
    if (n > INT32_MAX / 2) return fail(ctx, ISYCOS_E_INVAL, "too many windows in one call");
    int max_m = 0, max_sorted = 0, max_sorted_glob = 0;
    const uint32_t smask = sort_mask(ctx, k);
    const int smin = sort_min_size(ctx, k);
    int64_t pairs = 0, total_pts = 0;
    int32_t count[kBuckets] = {0};
    // for the work counters: sum of m^2 per size bucket, and the windows below sort_min in its
    // bucket (the only bucket the sorted path splits)
    int64_t m2_by_size[kBuckets] = {0}, m2_below = 0, n_below = 0;
    const int b_smin = smin > 1 ? size_bucket(smin) : -1;
    std::vector<int32_t> &slot = L.h_slot;
    slot.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        // every window must lie inside its resident series: the kernel reads it unchecked
        if (!window_in_series(ctx, w[i].xs, w[i].ys, w[i].start, w[i].m, k))
            return fail(ctx, ISYCOS_E_INVAL, "window %lld ([%lld, +%d] of series %d, %d) is outside its series",
                        (long long)i, (long long)w[i].start, w[i].m, w[i].xs, w[i].ys);
        max_m = std::max(max_m, w[i].m);
        if (((smask >> size_bucket(w[i].m)) & 1u) && w[i].m >= smin) {
            if (w[i].m <= kSortMax) max_sorted = std::max(max_sorted, w[i].m);
            else max_sorted_glob = std::max(max_sorted_glob, w[i].m);
        }
        pairs += (int64_t)w[i].m * (w[i].m - 1);
        slot[i] = bucket_slot(w[i].m);
        count[slot[i]]++;
        total_pts += w[i].m;
        const int64_t m2 = (int64_t)w[i].m * w[i].m;
        const int b = kBuckets - 1 - slot[i];
        m2_by_size[b] += m2;
        if (b == b_smin && w[i].m < smin) {
            m2_below += m2;
            ++n_below;
        }
    }
    const int nt = batched_threads(max_m, std::max(max_sorted, max_sorted_glob), nt_switch(ctx, k));
    const size_t smem = batched_smem(max_m, nt, max_sorted);
    isycos_status rc;
    if ((rc = ensure_smem(ctx, k, nt, smem))) return rc;

    // One pinned staging block: the bucket table, then the items sorted by bucket slot
    // (largest windows first); one host-to-device copy.
    const size_t tab_bytes = (sizeof(BucketTable) + 255) & ~(size_t)255;
    const size_t stage_bytes = tab_bytes + sizeof(WorkItem) * n;
    if ((rc = host_reserve(ctx, L.h_items, stage_bytes))) return rc;
    // results, then the sorted path's device-counted work (two counters)
    const size_t work_off = (sizeof(isycos_mi_out) * (size_t)n + 15) & ~(size_t)15;
    if ((rc = host_reserve(ctx, L.h_table, work_off + 16))) return rc;
    unsigned char *stage = reinterpret_cast<unsigned char *>(L.h_items.p);
    BucketTable &T = *reinterpret_cast<BucketTable *>(stage);
    build_table(T, count, nt);
    int32_t fill[kBuckets];
    for (int q = 0; q < kBuckets; ++q) fill[q] = T.item_off[q];
    WorkItem *items = reinterpret_cast<WorkItem *>(stage + tab_bytes);
    int64_t pts = 0;
    for (int64_t i = 0; i < n; ++i) {
        WorkItem &it = items[fill[slot[i]]++];
        it.x = ctx->series_ptr[w[i].xs] + w[i].start;
        it.y = ctx->series_ptr[w[i].ys] + w[i].start;
        it.m = w[i].m;
        it.out = (int32_t)i;
        it.pts = nx ? pts : -1;
        pts += w[i].m;
    }

    if ((rc = dev_reserve(ctx, L.d_items, stage_bytes))) return rc;
    if (!L.d_queue.p) L.queue_clean = false;
    if ((rc = dev_reserve(ctx, L.d_queue, 256))) return rc;
    if (nx) {
        if ((rc = dev_reserve(ctx, L.d_nx, 4 * total_pts))) return rc;
        if ((rc = dev_reserve(ctx, L.d_ny, 4 * total_pts))) return rc;
        if ((rc = dev_reserve(ctx, L.d_c, 4 * total_pts))) return rc;
    }
    // The work counters are zeroed once; every launch leaves them at zero.
    cudaError_t e = cudaSuccess;
    if (!L.queue_clean) e = cudaMemsetAsync(L.d_queue.p, 0, 128, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_items.p, stage, stage_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "staging the window list");
    L.queue_clean = true;

    int grid;
    if ((rc = launch_grid(ctx, k, nt, smem, batched_grid_need(T, nt), L.slot_share, &grid))) return rc;
    // sorted-path scratch of the windows above kSortMax points: one slice per CTA
    size_t g_stride = 0;
    if (max_sorted_glob > 0) {
        g_stride = (sorted_scratch(max_sorted_glob) + 255) & ~(size_t)255;
        if ((rc = dev_reserve(ctx, L.d_gscratch, g_stride * (size_t)grid))) return rc;
    }
    BatchArgs a;
    a.items = reinterpret_cast<const WorkItem *>(reinterpret_cast<unsigned char *>(L.d_items.p) + tab_bytes);
    a.table = reinterpret_cast<const BucketTable *>(L.d_items.p);
    a.queue = reinterpret_cast<int32_t *>(L.d_queue.p);
    a.psi_fx = ctx->d_psi_fx;
    a.log_fx = ctx->d_log_fx;
    // results go straight to the pinned, mapped host buffer (no copy back)
    a.out = reinterpret_cast<isycos_mi_out *>(L.h_table.dev);
    a.nx = nx ? reinterpret_cast<int32_t *>(L.d_nx.p) : nullptr;
    a.ny = nx ? reinterpret_cast<int32_t *>(L.d_ny.p) : nullptr;
    a.c = nx ? reinterpret_cast<int32_t *>(L.d_c.p) : nullptr;
    a.k = k;
    a.nt = nt;
    a.sort_mask = smask;
    a.est = est;
    a.sort_min = smin;
    a.inv_k = est ? 0.0 : 1.0 / (double)k;
    a.gscratch = max_sorted_glob > 0 ? reinterpret_cast<unsigned char *>(L.d_gscratch.p) : nullptr;
    a.gscratch_stride = (int64_t)g_stride;
    // work counters: device accumulators after the work counters of d_queue
    a.work = reinterpret_cast<unsigned long long *>(reinterpret_cast<unsigned char *>(L.d_queue.p) + 64);
    a.work_out = reinterpret_cast<unsigned long long *>(reinterpret_cast<unsigned char *>(L.h_table.dev) + work_off);
    // per bucket: the path is the same for all its windows (but those below sort_min); a
    // sorted window's sort work depends on its bucket's slot count only
    int64_t work_bf = 0, work_sort = 0;
    for (int b = 0; b < kBuckets; ++b) {
        const int64_t nb = count[kBuckets - 1 - b];
        if (nb == 0) continue;
        if (b >= 7 && takes_sorted_path(1 << b, nt, smask, a.gscratch != nullptr)) {
            const int64_t below = b == b_smin ? n_below : 0;
            work_sort += (nb - below) * sort_cx_steps(1 << b);
            work_bf += b == b_smin ? m2_below : 0;
        } else {
            work_bf += m2_by_size[b];
        }
    }
    e = cudaEventRecord(L.ev_start, st);
    if (e == cudaSuccess) e = launch_batched(a, grid, smem, st);
    if (e == cudaSuccess) e = cudaEventRecord(L.ev_stop, st);
    if (e != cudaSuccess) {
        L.queue_clean = false;
        return cuda_fail(ctx, e, "MI kernel launch");
    }
    if (nx) {
        e = cudaMemcpyAsync(nx, L.d_nx.p, 4 * total_pts, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ny, L.d_ny.p, 4 * total_pts, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c, L.d_c.p, 4 * total_pts, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) {
            L.queue_clean = false;
            return cuda_fail(ctx, e, "per-point results");
        }
    }
    Lane::Open &o = L.open;
    o.open = true;
    o.st = st;
    o.n = n;
    o.pairs = pairs;
    o.total_pts = total_pts;
    o.nx = nx;
    o.ny = ny;
    o.c = c;
    o.max_m = max_m;
    o.work_bf = work_bf;
    o.work_sort = work_sort;
    o.work_off = work_off;
    for (int q = 0; q < kBuckets; ++q) o.count[q] = count[q];
    return ISYCOS_OK;
}

constexpr int kSpinUs = 200;

isycos_status engine_collect(isycos_ctx *ctx, Lane &L, isycos_mi_out *out) {
    Lane::Open &o = L.open;
    if (!o.open) return ISYCOS_OK;
    o.open = false;
    // A search round's launch usually finishes within tens of microseconds, and a blocking
    // synchronise adds the host thread's wake-up to every round: poll the launch's stop event
    // for up to kSpinUs first (the results are in mapped host memory once it has passed),
    // then block.  Per-point outputs are copied after the launch: those wait for the stream.
    cudaError_t e = cudaSuccess;
    bool done = false;
    if (!o.nx) {
        const auto t_spin = std::chrono::steady_clock::now();
        for (;;) {
            e = cudaEventQuery(L.ev_stop);
            if (e != cudaErrorNotReady) {
                done = e == cudaSuccess;
                break;
            }
            if (std::chrono::steady_clock::now() - t_spin > std::chrono::microseconds(kSpinUs)) {
                e = cudaSuccess;
                break;
            }
        }
    }
    if (!done && e == cudaSuccess) e = cudaStreamSynchronize(o.st);
    float t0 = 0.0f, t1 = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t0, ctx->ev_ref, L.ev_start);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, ctx->ev_ref, L.ev_stop);
    if (e != cudaSuccess) {
        L.queue_clean = false;
        return cuda_fail(ctx, e, "MI kernel");
    }
    memcpy(out, L.h_table.p, sizeof(isycos_mi_out) * o.n);
    add_stats(ctx, o.n, o.pairs, 1, 1, 0);
    {
        // kernel intervals on the device timeline (lanes may overlap); their union is the
        // kernel's busy time reported by isycos_get_stats
        std::lock_guard<std::mutex> g(ctx->stats_mu);
        ctx->kernel_iv.push_back({t0, t1});
        ctx->stats.mi_kernel_launches += 1;
        for (int q = 0; q < kBuckets; ++q) ctx->stats.windows_by_size[kBuckets - 1 - q] += o.count[q];
        const int bmax = kBuckets - 1 - bucket_slot(o.max_m);
        ctx->stats.launches_by_size[bmax] += 1;
        ctx->stats.launch_ms_by_size[bmax] += (double)(t1 - t0);
        const unsigned long long *wk =
            reinterpret_cast<const unsigned long long *>(reinterpret_cast<const unsigned char *>(L.h_table.p) + o.work_off);
        ctx->stats.work_bf += o.work_bf;
        ctx->stats.work_sort += o.work_sort;
        ctx->stats.work_scan += (int64_t)wk[0];
        ctx->stats.work_search += (int64_t)wk[1];
    }
    return ISYCOS_OK;
}

isycos_status engine_eval(isycos_ctx *ctx, Lane &L, const HostWindow *w, int64_t n, int k,
                          isycos_mi_out *out, int32_t *nx, int32_t *ny, int32_t *c,
                          cudaStream_t st, int est) {
    isycos_status rc = engine_launch(ctx, L, w, n, k, est, nx, ny, c, st);
    if (rc) return rc;
    return engine_collect(ctx, L, out);
}

isycos_status get_lane(isycos_ctx *ctx, int i, Lane **out) {
    if (i < 0 || i >= kLaneSlots) return fail(ctx, ISYCOS_E_INVAL, "lane %d out of range", i);
    Lane *have = ctx->lanes[i].load(std::memory_order_acquire);
    if (have) {
        *out = have;
        return ISYCOS_OK;
    }
    std::lock_guard<std::mutex> g(ctx->lane_mu);
    if ((have = ctx->lanes[i].load(std::memory_order_acquire))) {
        *out = have;
        return ISYCOS_OK;
    }
    Lane *L = new Lane();
    cudaError_t e = cudaSuccess;
    if (i == 0) {
        L->stream = ctx->stream;
    } else {
        // latency-bound searches get the highest stream priority, so that their small
        // launches take CTA slots ahead of the waiting CTAs of large launches
        int least = 0, greatest = 0;
        if (i >= kPrioLaneBase) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithPriority(&L->stream, cudaStreamNonBlocking,
                                             i >= kPrioLaneBase ? greatest : least);
        L->own_stream = true;
    }
    if (e == cudaSuccess) e = cudaEventCreate(&L->ev_start);
    if (e == cudaSuccess) e = cudaEventCreate(&L->ev_stop);
    if (e != cudaSuccess) {
        if (L->own_stream && L->stream) cudaStreamDestroy(L->stream);
        delete L;
        return cuda_fail(ctx, e, "lane creation");
    }
    ctx->lanes[i].store(L, std::memory_order_release);
    *out = L;
    return ISYCOS_OK;
}

void lane_release(isycos_ctx *ctx, Lane &L) {
    cudaStreamSynchronize(L.stream);
    DevBuf *bufs[] = {&L.d_items, &L.d_queue, &L.d_out, &L.d_nx, &L.d_ny, &L.d_c,
                      &L.d_chain_desc, &L.d_chain_steps, &L.d_chain_state,
                      &L.d_chain_recomp, &L.d_chain_out, &L.d_gscratch};
    for (DevBuf *b : bufs) dev_release(ctx, *b);
}

static void free_lane(isycos_ctx *ctx, Lane *L) {
    DevBuf *bufs[] = {&L->d_items, &L->d_queue, &L->d_out, &L->d_nx, &L->d_ny, &L->d_c,
                      &L->d_chain_desc, &L->d_chain_steps, &L->d_chain_state,
                      &L->d_chain_recomp, &L->d_chain_out, &L->d_gscratch};
    for (DevBuf *b : bufs) dev_release(ctx, *b);
    if (L->h_items.p) cudaFreeHost(L->h_items.p);
    if (L->h_table.p) cudaFreeHost(L->h_table.p);
    if (L->ev_start) cudaEventDestroy(L->ev_start);
    if (L->ev_stop) cudaEventDestroy(L->ev_stop);
    if (L->own_stream) cudaStreamDestroy(L->stream);
    delete L;
}

static isycos_status sync_series_table(isycos_ctx *ctx, cudaStream_t st) {
    if (!ctx->series_dirty) return ISYCOS_OK;
    const size_t ns = std::max<size_t>(ctx->series_ptr.size(), 1);
    isycos_status rc;
    if ((rc = dev_reserve(ctx, ctx->d_series_ptr, sizeof(float *) * ns))) return rc;
    if ((rc = dev_reserve(ctx, ctx->d_series_len, sizeof(int64_t) * ns))) return rc;
    if (!ctx->series_ptr.empty()) {
        cudaError_t e = cudaMemcpyAsync(ctx->d_series_ptr.p, ctx->series_ptr.data(),
                                        sizeof(float *) * ctx->series_ptr.size(),
                                        cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->d_series_len.p, ctx->series_len.data(),
                                sizeof(int64_t) * ctx->series_len.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "series table upload");
    }
    ctx->series_dirty = false;
    return ISYCOS_OK;
}

void fill_fixed_tables(long long *psi_fx, long long *log_fx) {
    // psi(1) = -gamma, psi(n + 1) = psi(n) + 1/n (binary64 forward recurrence); values
    // rounded to the nearest multiple of 2^-32.
    const double gamma = 0.57721566490153286060651209008240243;
    psi_fx[0] = 0;
    log_fx[0] = 0;
    double psi = -gamma;
    for (int n = 1; n < kTableN; ++n) {
        psi_fx[n] = llround(ldexp(psi, 32));
        log_fx[n] = llround(ldexp(log((double)n), 32));
        psi = psi + 1.0 / (double)n;
    }
}

static void build_tables(std::vector<long long> &psi_fx, std::vector<long long> &log_fx) {
    psi_fx.assign(kTableN, 0);
    log_fx.assign(kTableN, 0);
    fill_fixed_tables(psi_fx.data(), log_fx.data());
}

}  // namespace isy

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------

extern "C" {

void isycos_params_default(isycos_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->k = 4;
    p->score_kind = 0;
    p->sigma = 0.2;
    p->tau = -1.0;   /* sigma / 4 */
    p->s_min = 32;
    p->s_max = 256;
    p->delta_td = 0;
    p->delta_bu = 0;
    p->h = 8;
    p->t_max_idle = 3;
    p->p = 3;
    p->mode = 0;
    p->pruning = 0;
    p->max_steps = 10000;
    p->seed = 0;
    p->sel_partitions = 20;
    p->sel_samples = 6;
    p->sel_alpha = 0.5;
    p->sel_rho = 0.5;
    p->chunks = 1;
    p->estimator = 0;
}

isycos_status isycos_create(isycos_ctx **out, int32_t device, uint64_t mem_budget_bytes) {
    if (!out) return ISYCOS_E_INVAL;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ISYCOS_E_CUDA;
    }
    if (device < 0 || device >= ndev) return ISYCOS_E_INVAL;
    isycos_ctx *ctx = new isycos_ctx();
    ctx->device = device;
    // the series tables never reallocate: serving threads read them while the caller adds
    // series
    ctx->series_ptr.reserve(kMaxSeries);
    ctx->series_len.reserve(kMaxSeries);
    e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    size_t free_b = 0, total_b = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
        delete ctx;
        return ISYCOS_E_CUDA;
    }
    ctx->budget = mem_budget_bytes ? mem_budget_bytes : (uint64_t)(0.9 * (double)free_b);
    build_tables(ctx->h_psi_fx, ctx->h_log_fx);
    void *p = nullptr, *q = nullptr;
    e = cudaMalloc(&p, sizeof(long long) * kTableN);
    if (e == cudaSuccess) e = cudaMalloc(&q, sizeof(long long) * kTableN);
    if (e == cudaSuccess)
        e = cudaMemcpy(p, ctx->h_psi_fx.data(), sizeof(long long) * kTableN, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(q, ctx->h_log_fx.data(), sizeof(long long) * kTableN, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (p) cudaFree(p);
        if (q) cudaFree(q);
        cudaStreamDestroy(ctx->stream);
        delete ctx;
        return ISYCOS_E_CUDA;
    }
    ctx->d_psi_fx = reinterpret_cast<long long *>(p);
    ctx->d_log_fx = reinterpret_cast<long long *>(q);
    ctx->used += 2 * sizeof(long long) * kTableN;
    if (cudaEventCreate(&ctx->ev_ref) != cudaSuccess || cudaEventRecord(ctx->ev_ref, ctx->stream) != cudaSuccess ||
        cudaEventSynchronize(ctx->ev_ref) != cudaSuccess) {
        isycos_destroy(ctx);
        return ISYCOS_E_CUDA;
    }
    {
        unsigned hw = std::thread::hardware_concurrency();
        ctx->max_lanes = (int)std::max(1u, std::min((unsigned)kMaxLanes, hw));
        load_tunings(ctx);   // choices isycos_autotune stored for this GPU, if any
        Lane *L0 = nullptr;
        if (get_lane(ctx, 0, &L0) != ISYCOS_OK) {
            isycos_destroy(ctx);
            return ISYCOS_E_CUDA;
        }
    }
    *out = ctx;
    return ISYCOS_OK;
}

isycos_status isycos_destroy(isycos_ctx *ctx) {
    if (!ctx) return ISYCOS_E_INVAL;
    cudaSetDevice(ctx->device);
    serve_shutdown(ctx);
    cudaStreamSynchronize(ctx->stream);
    for (float *p : ctx->series_ptr)
        if (p) cudaFree(p);
    for (auto &kv : ctx->series_pool) cudaFree(kv.second);
    ctx->series_pool.clear();
    for (int i = 0; i < kLaneSlots; ++i) {
        Lane *L = ctx->lanes[i].exchange(nullptr);
        if (!L) continue;
        cudaStreamSynchronize(L->stream);
        free_lane(ctx, L);
    }
    DevBuf *bufs[] = {&ctx->d_series_ptr, &ctx->d_series_len, &ctx->d_table, &ctx->d_slot,
                      &ctx->d_pos, &ctx->d_bcount, &ctx->d_status, &ctx->d_plain_acc,
                      &ctx->d_dev_items, &ctx->d_dev_queue, &ctx->d_dev_table,
                      &ctx->d_bu_q, &ctx->d_bu_res, &ctx->d_bu_found, &ctx->d_bu_queue};
    for (DevBuf *b : bufs) dev_release(ctx, *b);
    if (ctx->ev_ref) cudaEventDestroy(ctx->ev_ref);
    if (ctx->ev_bu[0]) cudaEventDestroy(ctx->ev_bu[0]);
    if (ctx->ev_bu[1]) cudaEventDestroy(ctx->ev_bu[1]);
    if (ctx->d_psi_fx) cudaFree(ctx->d_psi_fx);
    if (ctx->d_log_fx) cudaFree(ctx->d_log_fx);
    cudaStreamDestroy(ctx->stream);
    delete ctx;
    return ISYCOS_OK;
}

const char *isycos_last_error(const isycos_ctx *ctx) {
    if (!ctx) return "null context";
    std::lock_guard<std::mutex> g(ctx->err_mu);
    return ctx->err.c_str();
}

// Device memory for a series of `bytes`: a buffer kept from a dropped series when one of
// between `bytes` and twice that is free, else a new allocation (buffers kept from dropped
// series are freed first when the budget or the device runs short).  Caller holds engine_mu.
static isycos_status series_alloc(isycos_ctx *ctx, size_t bytes, float **out, size_t *cap) {
    auto it = ctx->series_pool.lower_bound(bytes);
    if (it != ctx->series_pool.end() && it->first <= 2 * bytes) {
        *out = it->second;
        *cap = it->first;
        ctx->series_pool.erase(it);
        return ISYCOS_OK;
    }
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (ctx->used.load() + bytes <= ctx->budget) {
            float *d = nullptr;
            if (cudaMalloc(&d, bytes) == cudaSuccess) {
                ctx->used += bytes;
                ctx->series_bytes += bytes;
                *out = d;
                *cap = bytes;
                return ISYCOS_OK;
            }
            cudaGetLastError();
        }
        if (ctx->series_pool.empty()) break;
        for (auto &kv : ctx->series_pool) {   // give the kept buffers back and try again
            cudaFree(kv.second);
            ctx->used -= kv.first;
            ctx->series_bytes -= kv.first;
        }
        ctx->series_pool.clear();
    }
    return fail(ctx, ISYCOS_E_NOMEM, "put_series: no device memory for %zu bytes within the budget", bytes);
}

static void series_release(isycos_ctx *ctx, float *d, size_t cap) {
    ctx->series_pool.emplace(cap, d);
}

// Make `count` series resident: one copy each on the context's stream, one device-side
// finiteness check over the series given in device memory, one synchronisation.  On any
// error nothing is made resident.
static isycos_status put_series_list(isycos_ctx *ctx, int32_t count, const float *const *data,
                                     const int64_t *n, int32_t on_device, int32_t *ids) {
    if (count < 0 || (count > 0 && (!data || !n || !ids))) return fail(ctx, ISYCOS_E_INVAL, "put_series: bad arguments");
    for (int32_t s = 0; s < count; ++s)
        if (!data[s] || n[s] < 1) return fail(ctx, ISYCOS_E_INVAL, "put_series: bad arguments (series %d)", s);
    std::lock_guard<std::mutex> g(ctx->engine_mu);
    cudaSetDevice(ctx->device);
    size_t free_slots = 0;
    for (float *p : ctx->series_ptr) free_slots += p ? 0 : 1;
    if (ctx->series_ptr.size() - free_slots + (size_t)count > (size_t)kMaxSeries)
        return fail(ctx, ISYCOS_E_NOMEM, "put_series: at most %d series resident", kMaxSeries);
    std::vector<float *> dev((size_t)count, nullptr);
    std::vector<size_t> caps((size_t)count, 0);
    auto undo = [&](int32_t upto) {
        for (int32_t s = 0; s < upto; ++s) series_release(ctx, dev[s], caps[s]);
    };
    isycos_status rc;
    for (int32_t s = 0; s < count; ++s)
        if ((rc = series_alloc(ctx, sizeof(float) * (size_t)n[s], &dev[s], &caps[s]))) {
            undo(s);
            return rc;
        }
    cudaError_t e = cudaSuccess;
    for (int32_t s = 0; s < count && e == cudaSuccess; ++s)
        e = cudaMemcpyAsync(dev[s], data[s], sizeof(float) * (size_t)n[s],
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream);
    // every value is checked on the device once it is there (host input included: a scan on
    // the device is faster than one on the host, and there is one synchronisation either way)
    int32_t bad = 0;
    if (e == cudaSuccess) {
        if ((rc = dev_reserve(ctx, ctx->d_status, 256))) {
            cudaStreamSynchronize(ctx->stream);
            undo(count);
            return rc;
        }
        int32_t *flag = reinterpret_cast<int32_t *>(ctx->d_status.p) + 8;
        e = cudaMemsetAsync(flag, 0, 4, ctx->stream);
        for (int32_t s = 0; s < count && e == cudaSuccess; ++s) e = launch_check_finite(dev[s], n[s], flag, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, flag, 4, cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess || bad) {
        cudaStreamSynchronize(ctx->stream);
        undo(count);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "put_series");
        return fail(ctx, ISYCOS_E_INVAL, "put_series: a series holds non-finite values");
    }
    size_t scan = 0;
    for (int32_t s = 0; s < count; ++s) {
        int32_t id = -1;
        for (; scan < ctx->series_ptr.size(); ++scan)
            if (!ctx->series_ptr[scan]) {
                id = (int32_t)scan++;
                break;
            }
        if (id < 0) {
            id = (int32_t)ctx->series_ptr.size();
            ctx->series_ptr.push_back(nullptr);
            ctx->series_len.push_back(0);
            ctx->series_cap.push_back(0);
            scan = ctx->series_ptr.size();
        }
        ctx->series_ptr[id] = dev[s];
        ctx->series_len[id] = n[s];
        ctx->series_cap[id] = caps[s];
        ids[s] = id;
    }
    ctx->series_dirty = true;
    return ISYCOS_OK;
}

isycos_status isycos_put_series(isycos_ctx *ctx, const float *data, int64_t n, int32_t on_device,
                                int32_t *series_id) {
    if (!ctx) return ISYCOS_E_INVAL;
    if (!data || n < 1 || !series_id) return fail(ctx, ISYCOS_E_INVAL, "put_series: bad arguments");
    return put_series_list(ctx, 1, &data, &n, on_device, series_id);
}

isycos_status isycos_put_series_many(isycos_ctx *ctx, int32_t count, const float *const *data,
                                     const int64_t *n, int32_t on_device, int32_t *series_ids) {
    if (!ctx) return ISYCOS_E_INVAL;
    return put_series_list(ctx, count, data, n, on_device, series_ids);
}

isycos_status isycos_drop_series(isycos_ctx *ctx, int32_t series_id) {
    if (!ctx) return ISYCOS_E_INVAL;
    std::lock_guard<std::mutex> g(ctx->engine_mu);
    if (series_id < 0 || series_id >= (int32_t)ctx->series_ptr.size() || !ctx->series_ptr[series_id])
        return fail(ctx, ISYCOS_E_NOTFOUND, "unknown series %d", series_id);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    // the memory is kept for the next series of about its size
    series_release(ctx, ctx->series_ptr[series_id], ctx->series_cap[series_id]);
    ctx->series_ptr[series_id] = nullptr;
    ctx->series_len[series_id] = 0;
    ctx->series_cap[series_id] = 0;
    ctx->series_dirty = true;
    return ISYCOS_OK;
}

isycos_status isycos_series_info(isycos_ctx *ctx, int32_t series_id, const float **device_ptr,
                                 int64_t *n) {
    if (!ctx) return ISYCOS_E_INVAL;
    if (series_id < 0 || series_id >= (int32_t)ctx->series_ptr.size() || !ctx->series_ptr[series_id])
        return fail(ctx, ISYCOS_E_NOTFOUND, "unknown series %d", series_id);
    if (device_ptr) *device_ptr = ctx->series_ptr[series_id];
    if (n) *n = ctx->series_len[series_id];
    return ISYCOS_OK;
}

static isycos_status host_windows(isycos_ctx *ctx, const isycos_window *windows, int64_t n_w,
                                  int32_t k, std::vector<HostWindow> &hw) {
    if (k < 1 || k > kMaxK) return fail(ctx, ISYCOS_E_INVAL, "k = %d outside [1, %d]", k, kMaxK);
    if (n_w < 0 || (n_w > 0 && !windows)) return fail(ctx, ISYCOS_E_INVAL, "bad window list");
    hw.resize((size_t)n_w);
    for (int64_t i = 0; i < n_w; ++i) {
        isycos_status rc = check_window(ctx, windows[i], k);
        if (rc) return fail(ctx, rc, "window %lld: %s", (long long)i, ctx->err.c_str());
        hw[i] = HostWindow{windows[i].xs, windows[i].ys, windows[i].start, windows[i].m};
    }
    return ISYCOS_OK;
}

isycos_status isycos_mi_windows(isycos_ctx *ctx, const isycos_window *windows, int64_t n_w,
                                int32_t k, isycos_mi_out *out, void *cuda_stream) {
    if (!ctx) return ISYCOS_E_INVAL;
    if (n_w > 0 && !out) return fail(ctx, ISYCOS_E_INVAL, "out is NULL");
    std::lock_guard<std::mutex> g(ctx->engine_mu);
    cudaSetDevice(ctx->device);
    std::vector<HostWindow> hw;
    isycos_status rc = host_windows(ctx, windows, n_w, k, hw);
    if (rc) return rc;
    return engine_eval(ctx, *ctx->lanes[0].load(), hw.data(), n_w, k, out, nullptr, nullptr, nullptr,
                       pick_stream(ctx, cuda_stream), ctx->opt_estimator);
}

isycos_status isycos_mi_windows_points(isycos_ctx *ctx, const isycos_window *windows,
                                       int64_t n_w, int32_t k, isycos_mi_out *out, int32_t *nx,
                                       int32_t *ny, int32_t *c, void *cuda_stream) {
    if (!ctx) return ISYCOS_E_INVAL;
    if (n_w > 0 && (!out || !nx || !ny || !c))
        return fail(ctx, ISYCOS_E_INVAL, "output arrays must not be NULL");
    std::lock_guard<std::mutex> g(ctx->engine_mu);
    cudaSetDevice(ctx->device);
    std::vector<HostWindow> hw;
    isycos_status rc = host_windows(ctx, windows, n_w, k, hw);
    if (rc) return rc;
    return engine_eval(ctx, *ctx->lanes[0].load(), hw.data(), n_w, k, out, nx, ny, c,
                       pick_stream(ctx, cuda_stream), ctx->opt_estimator);
}

isycos_status isycos_mi_windows_device(isycos_ctx *ctx, const isycos_window *d_windows,
                                       int64_t n_w, int32_t k, int32_t max_m,
                                       isycos_mi_out *d_out, void *cuda_stream) {
    if (!ctx) return ISYCOS_E_INVAL;
    if (k < 1 || k > kMaxK) return fail(ctx, ISYCOS_E_INVAL, "k = %d outside [1, %d]", k, kMaxK);
    if (max_m < k + 1 || max_m > kMaxM)
        return fail(ctx, ISYCOS_E_INVAL, "max_m = %d outside [k + 1, %d]", max_m, kMaxM);
    if (n_w < 0 || n_w > INT32_MAX / 2 || (n_w > 0 && (!d_windows || !d_out)))
        return fail(ctx, ISYCOS_E_INVAL, "bad window list");
    if (n_w == 0) return ISYCOS_OK;
    std::lock_guard<std::mutex> g(ctx->engine_mu);
    cudaSetDevice(ctx->device);
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    isycos_status rc;
    if ((rc = sync_series_table(ctx, st))) return rc;
    const uint32_t smask = sort_mask(ctx, k);
    // windows are sized on the device: room for the largest window a set bucket allows
    int max_sorted = 0;
    for (int b = 1; b < 31; ++b)
        if (((smask >> b) & 1u) && (1 << (b - 1)) < max_m) max_sorted = std::min(std::min(max_m, 1 << b), kSortMax);
    const int nt = batched_threads(max_m, max_sorted, nt_switch(ctx, k));
    const size_t smem = batched_smem(max_m, nt, max_sorted);
    if ((rc = ensure_smem(ctx, k, nt, smem))) return rc;
    if ((rc = dev_reserve(ctx, ctx->d_dev_items, sizeof(WorkItem) * n_w))) return rc;
    if ((rc = dev_reserve(ctx, ctx->d_slot, 4 * n_w))) return rc;
    if ((rc = dev_reserve(ctx, ctx->d_pos, 4 * n_w))) return rc;
    if ((rc = dev_reserve(ctx, ctx->d_bcount, 4 * kBuckets + 64))) return rc;
    if ((rc = dev_reserve(ctx, ctx->d_dev_table, sizeof(BucketTable)))) return rc;
    if ((rc = dev_reserve(ctx, ctx->d_dev_queue, 256))) return rc;
    if ((rc = dev_reserve(ctx, ctx->d_status, 256))) return rc;
    PrepArgs pa;
    pa.windows = d_windows;
    pa.n_w = n_w;
    pa.k = k;
    pa.max_m = max_m;
    pa.series_ptr = reinterpret_cast<const float *const *>(ctx->d_series_ptr.p);
    pa.series_len = reinterpret_cast<const int64_t *>(ctx->d_series_len.p);
    pa.n_series = (int32_t)ctx->series_ptr.size();
    pa.nt = nt;
    pa.items = reinterpret_cast<WorkItem *>(ctx->d_dev_items.p);
    pa.bucket_count = reinterpret_cast<int32_t *>(ctx->d_bcount.p);
    pa.slot_of = reinterpret_cast<int32_t *>(ctx->d_slot.p);
    pa.pos_of = reinterpret_cast<int32_t *>(ctx->d_pos.p);
    pa.table = reinterpret_cast<BucketTable *>(ctx->d_dev_table.p);
    pa.status = reinterpret_cast<int32_t *>(ctx->d_status.p);
    pa.out = d_out;
    cudaError_t e = cudaMemsetAsync(ctx->d_bcount.p, 0, 4 * kBuckets, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_dev_queue.p, 0, 16, st);
    int launches = 0;
    if (e == cudaSuccess) e = launch_prep(pa, st, &launches);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "window preparation");
    int grid;
    if ((rc = launch_grid(ctx, k, nt, smem, 0, 4, &grid))) return rc;
    BatchArgs a;
    a.items = pa.items;
    a.table = pa.table;
    a.queue = reinterpret_cast<int32_t *>(ctx->d_dev_queue.p);
    a.psi_fx = ctx->d_psi_fx;
    a.log_fx = ctx->d_log_fx;
    a.out = d_out;
    a.nx = a.ny = a.c = nullptr;
    a.k = k;
    a.nt = nt;
    a.sort_mask = smask;
    a.est = ctx->opt_estimator;
    a.sort_min = sort_min_size(ctx, k);
    a.inv_k = a.est ? 0.0 : 1.0 / (double)k;
    a.gscratch = nullptr;   // windows above kSortMax points take the brute-force path here
    a.gscratch_stride = 0;
    e = launch_batched(a, grid, smem, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "MI kernel launch");
    add_stats(ctx, n_w, 0, launches + 1, 1, 0);
    return ISYCOS_OK;
}

isycos_status isycos_device_status(isycos_ctx *ctx, void *cuda_stream) {
    if (!ctx) return ISYCOS_E_INVAL;
    std::lock_guard<std::mutex> g(ctx->engine_mu);
    cudaSetDevice(ctx->device);
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device status");
    if (!ctx->d_status.p) return ISYCOS_OK;
    int32_t flag = 0;
    e = cudaMemcpyAsync(&flag, ctx->d_status.p, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status.p, 0, 4, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device status");
    if (flag & 1) return fail(ctx, ISYCOS_E_INVAL, "an asynchronous call received invalid windows");
    return ISYCOS_OK;
}

isycos_status isycos_mi_windows_plain(isycos_ctx *ctx, const isycos_window *windows,
                                      int64_t n_w, int32_t k, isycos_mi_out *out,
                                      void *cuda_stream) {
    if (!ctx) return ISYCOS_E_INVAL;
    if (n_w > 0 && !out) return fail(ctx, ISYCOS_E_INVAL, "out is NULL");
    std::lock_guard<std::mutex> g(ctx->engine_mu);
    cudaSetDevice(ctx->device);
    std::vector<HostWindow> hw;
    isycos_status rc = host_windows(ctx, windows, n_w, k, hw);
    if (rc) return rc;
    if (n_w == 0) return ISYCOS_OK;
    cudaStream_t st = pick_stream(ctx, cuda_stream);
    if ((rc = dev_reserve(ctx, ctx->lanes[0].load()->d_out, sizeof(isycos_mi_out) * n_w))) return rc;
    if (!ctx->d_plain_acc.p) {
        if ((rc = dev_reserve(ctx, ctx->d_plain_acc, 256))) return rc;
        cudaError_t e = cudaMemset(ctx->d_plain_acc.p, 0, 256);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
    }
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(ctx->d_plain_acc.p);
    int32_t *done = reinterpret_cast<int32_t *>(acc + 2);
    isycos_mi_out *d_out = reinterpret_cast<isycos_mi_out *>(ctx->lanes[0].load()->d_out.p);
    int launches = 0;
    int64_t pairs = 0;
    for (int64_t i = 0; i < n_w; ++i) {
        WorkItem it;
        it.x = ctx->series_ptr[hw[i].xs] + hw[i].start;
        it.y = ctx->series_ptr[hw[i].ys] + hw[i].start;
        it.m = hw[i].m;
        it.out = (int32_t)i;
        it.pts = -1;
        pairs += (int64_t)it.m * (it.m - 1);
        cudaError_t e = launch_plain(it, k, ctx->d_psi_fx, ctx->d_log_fx, acc, done, d_out + i,
                                     nullptr, nullptr, nullptr, ctx->opt_estimator, st, &launches);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "plain MI kernel launch");
    }
    cudaError_t e = cudaMemcpyAsync(out, d_out, sizeof(isycos_mi_out) * n_w, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plain MI kernel");
    add_stats(ctx, n_w, pairs, launches, n_w, 0);
    return ISYCOS_OK;
}

isycos_status isycos_get_stats(isycos_ctx *ctx, isycos_stats *out) {
    if (!ctx || !out) return ISYCOS_E_INVAL;
    std::lock_guard<std::mutex> g(ctx->stats_mu);
    *out = ctx->stats;
    // union of the MI kernel intervals
    std::vector<std::pair<float, float>> iv = ctx->kernel_iv;
    std::sort(iv.begin(), iv.end());
    double busy = 0.0, lo = 0.0, hi = -1.0;
    for (const auto &p : iv) {
        if (p.first > hi) {
            if (hi > lo) busy += hi - lo;
            lo = p.first;
            hi = p.second;
        } else if (p.second > hi) {
            hi = p.second;
        }
    }
    if (hi > lo) busy += hi - lo;
    out->mi_kernel_ms = busy;
    return ISYCOS_OK;
}

isycos_status isycos_reset_stats(isycos_ctx *ctx) {
    if (!ctx) return ISYCOS_E_INVAL;
    std::lock_guard<std::mutex> g(ctx->stats_mu);
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->kernel_iv.clear();
    return ISYCOS_OK;
}

isycos_status isycos_tables(isycos_ctx *ctx, int32_t n_max, int64_t *psi_fx, int64_t *log_fx) {
    if (!ctx) return ISYCOS_E_INVAL;
    if (n_max < 0 || n_max >= kTableN || !psi_fx || !log_fx)
        return fail(ctx, ISYCOS_E_INVAL, "tables: n_max must be in [0, %d]", kTableN - 1);
    for (int32_t n = 0; n <= n_max; ++n) {
        psi_fx[n] = ctx->h_psi_fx[n];
        log_fx[n] = ctx->h_log_fx[n];
    }
    return ISYCOS_OK;
}

isycos_status isycos_set_option(isycos_ctx *ctx, int32_t option, int64_t value) {
    if (!ctx) return ISYCOS_E_INVAL;
    switch (option) {
        case ISYCOS_OPT_KERNEL:
            if (value < 0 || value > 2) break;
            ctx->opt_kernel = (int)value;
            return ISYCOS_OK;
        case ISYCOS_OPT_INCREMENTAL:
            if (value < 0 || value > 2) break;
            ctx->opt_incremental = (int)value;
            return ISYCOS_OK;
        case ISYCOS_OPT_SERVE_SLOTS:
            if (value < 1 || value > 1 << 20) break;
            ctx->serve_slots = (int)value;
            return ISYCOS_OK;
        case ISYCOS_OPT_SERVE_QUEUE:
            if (value < 1 || value > 1 << 24) break;
            ctx->serve_queue = (int)value;
            return ISYCOS_OK;
        case ISYCOS_OPT_LANES:
            if (value < 1 || value > kMaxLanes) break;
            ctx->max_lanes = (int)value;
            return ISYCOS_OK;
        case ISYCOS_OPT_ESTIMATOR:
            if (value < 0 || value > 1) break;
            ctx->opt_estimator = (int)value;
            return ISYCOS_OK;
        case ISYCOS_OPT_SPECULATION:
            if (value < 0 || value > 64) break;
            ctx->opt_spec_climbs = (int)value;
            return ISYCOS_OK;
        case ISYCOS_OPT_BU_DEVICE:
            if (value < 0 || value > 1) break;
            ctx->opt_bu_device = (int)value;
            return ISYCOS_OK;
        case ISYCOS_OPT_TIME_LIMIT_MS:
            if (value < 0 || value > 86400000) break;
            ctx->opt_time_limit_ms = value;
            return ISYCOS_OK;
        default:
            return fail(ctx, ISYCOS_E_INVAL, "unknown option %d", option);
    }
    return fail(ctx, ISYCOS_E_INVAL, "option %d: value %lld out of range", option, (long long)value);
}

}  // extern "C"
