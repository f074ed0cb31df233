// Internal declarations shared by the host runtime and the CUDA kernels of libisycos.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "isycos.h"

namespace isy {

constexpr int kMaxM = ISYCOS_MAX_M;
constexpr int kMaxK = ISYCOS_MAX_K;
constexpr int kTableN = kMaxM + 2;      // psi_fx / log_fx entries 0 .. kMaxM + 1
constexpr int kBuckets = 15;            // size buckets: m <= 2^b, b = 0 .. 14, stored largest first
// Points per lane in the CTA jobs of the brute-force kernels.  One point per lane spreads a
// window over twice as many warps as two would, which shortens the dependent chains of a
// launch of small windows (the latency of a SYCOS_BU round) at the same total work.
constexpr int kPoints = 1;
constexpr int kBlockPts = 32 * kPoints; // points per warp block
constexpr int kWarpSlicePts = 64;       // staging slice of one warp in the small-window phase

// One resolved window: device pointers to its first X and Y values.  32 bytes.
struct WorkItem {
    const float *x;
    const float *y;
    int32_t m;
    int32_t out;      // index of the result in the output array (input order)
    int64_t pts;      // offset of the window's points in the per-point arrays, or -1
};

// Work layout of one persistent launch: items sorted by size bucket, largest bucket first.
// Windows of more than 64 points are CTA jobs: one item (large windows, all warps of the CTA)
// or several items of one bucket (`wpw` warps each).  Windows of at most 64 points (bucket
// slots >= kSmallSlot) are taken one per warp, with no CTA barrier, once a CTA runs out of
// CTA jobs.
constexpr int kSmallSlot = kBuckets - 7;   // m <= 2^6
static_assert((1 << (kBuckets - 1 - kSmallSlot)) <= kWarpSlicePts,
              "a warp's staging slice holds the largest single-warp window");
struct BucketTable {
    int32_t total_jobs;          // CTA jobs
    int32_t n_items;
    int32_t small_first;         // first item taken by single warps
    int32_t pad;
    int32_t item_off[kBuckets];  // first item of bucket slot q
    int32_t count[kBuckets];     // items in bucket slot q
    int32_t job_off[kBuckets];   // first CTA job of bucket slot q
    int32_t wpw[kBuckets];       // warps per item in bucket slot q
};

struct BatchArgs {
    const WorkItem *items;
    const BucketTable *table;
    int32_t *queue;              // CTA jobs, warp items, CTAs finished: zero at launch; the
                                 // last CTA to finish zeroes them again
    const long long *psi_fx;
    const long long *log_fx;
    isycos_mi_out *out;
    int32_t *nx;                 // optional per-point outputs (nullptr: skip)
    int32_t *ny;
    int32_t *c;
    int32_t k;
    int32_t nt;                  // threads per CTA of the launch
    uint32_t sort_mask;          // bit b set: windows of bucket b (2^(b-1) < m <= 2^b) that
                                 // run one per CTA take the sorted path
    int32_t est;                 // 0: Kraskov's second estimator (Eq. KSGmi), 1: the first
    int32_t sort_min;            // windows below this size keep the brute-force path
    double inv_k;                // 1 / k correctly rounded (estimator 0), or 0 (estimator 1)
    unsigned char *gscratch;     // sorted-path scratch of windows above kSortMax points: one
    int64_t gscratch_stride;     // slice of gscratch_stride bytes per CTA (nullptr: none)
    // Work counters of the sorted path (nullptr: not counted): device accumulators, zero at
    // launch, which the last CTA copies to work_out and zeroes again.
    unsigned long long *work = nullptr;      // [0] phase A point x candidate visits, [1] phase B steps
    unsigned long long *work_out = nullptr;
};

// Device-side preparation of a window list held in device memory.
struct PrepArgs {
    const isycos_window *windows;
    int64_t n_w;
    int32_t k;
    int32_t max_m;
    const float *const *series_ptr;  // device table of resident series
    const int64_t *series_len;
    int32_t n_series;
    int32_t nt;                      // threads per CTA of the MI launch that follows
    WorkItem *items;                 // n_w entries (sorted output)
    int32_t *bucket_count;           // kBuckets counters (zeroed before launch)
    int32_t *slot_of;                // n_w scratch: bucket slot of each window or -1
    int32_t *pos_of;                 // n_w scratch: position inside the bucket
    BucketTable *table;
    int32_t *status;                 // error flags (bit 0: invalid window)
    isycos_mi_out *out;              // invalid windows get NaN results
};

// The 2^-32 fixed-point digamma and log tables, entries 0 .. kTableN - 1 (runtime.cu):
// psi_fx[n] = round(psi(n) 2^32) by the binary64 forward recurrence from psi(1) = -gamma,
// log_fx[n] = round(ln(n) 2^32); entry 0 of both is 0.
void fill_fixed_tables(long long *psi_fx, long long *log_fx);

// Launchers (kernels.cu).  Return cudaSuccess or the launch error.
cudaError_t launch_batched(const BatchArgs &a, int grid, size_t smem, cudaStream_t st);
cudaError_t batched_occupancy(int k, int nt, size_t smem, int *blocks_per_sm);
cudaError_t set_batched_smem(int k, int nt, size_t smem);
cudaError_t launch_plain(const WorkItem &it, int k, const long long *psi_fx,
                         const long long *log_fx, unsigned long long *acc, int32_t *done,
                         isycos_mi_out *out, int32_t *nx, int32_t *ny, int32_t *c, int est,
                         cudaStream_t st, int *launches);
cudaError_t launch_prep(const PrepArgs &a, cudaStream_t st, int *launches);
cudaError_t launch_check_finite(const float *d, int64_t n, int32_t *flag, cudaStream_t st);

__host__ __device__ inline int size_bucket(int m);
// Bucket of a window size: smallest b with m <= 2^b; slot q = kBuckets - 1 - b (largest first).
inline int bucket_slot(int m) { return kBuckets - 1 - size_bucket(m); }

// Warps per item for bucket slot q in a CTA of nt threads.
__host__ __device__ inline int warps_per_item(int q, int nt) {
    const int w = nt / 32;
    const int b = kBuckets - 1 - q;
    const int need = ((1 << b) + kBlockPts - 1) / kBlockPts;
    int wpw = 1;
    while (wpw < need && wpw < w) wpw *= 2;
    return wpw;
}

// Fill the bucket table from the per-slot item counts (same layout on host and device).
__host__ __device__ inline void fill_bucket_table(BucketTable *T, const int32_t *count, int nt) {
    const int W = nt / 32;
    int items = 0, jobs = 0;
    for (int q = 0; q < kBuckets; ++q) {
        const int wpw = q < kSmallSlot ? warps_per_item(q, nt) : 1;
        T->item_off[q] = items;
        T->count[q] = count[q];
        T->job_off[q] = jobs;
        T->wpw[q] = wpw;
        items += count[q];
        if (q < kSmallSlot) jobs += (count[q] + (W / wpw) - 1) / (W / wpw);
    }
    T->total_jobs = jobs;
    T->n_items = items;
    T->small_first = T->item_off[kSmallSlot];
    T->pad = 0;
}

// CTAs a launch needs at most: its CTA jobs plus enough warps for the small windows.
inline int batched_grid_need(const BucketTable &T, int nt) {
    const int W = nt / 32;
    return T.total_jobs + (T.n_items - T.small_first + W - 1) / W;
}

// Largest window whose sorted-path scratch (sort keys, records) shares the CTA's shared
// memory; larger windows, up to kMaxM, keep it in a slice of global memory per CTA (it stays
// in L2).
constexpr int kSortMax = 4096;
// Buckets the sorted path can take: windows of 257..4096 points, which run one per CTA (a
// 256-thread CTA up to 1024 points, a 1024-thread CTA above); the path is used for 1025..4096
// points unless isycos_autotune chose otherwise.
constexpr uint32_t kSortBuckets = (1u << 9) | (1u << 10) | (1u << 11) | (1u << 12) | (1u << 13) | (1u << 14);
constexpr uint32_t kDefaultSortBuckets = (1u << 11) | (1u << 12) | (1u << 13) | (1u << 14);
__host__ __device__ inline int size_bucket(int m) {   // smallest b with m <= 2^b
    if (m <= 1) return 0;
#ifdef __CUDA_ARCH__
    return 32 - __clz(m - 1);
#else
    return 32 - __builtin_clz((unsigned)(m - 1));
#endif
}

// Sorted path layout in shared memory after the window's m float2 values: the sort keys
// (8 bytes per slot, the slot count rounded up to a power of two; the y order once the x
// order is in the records), the x-ordered records (16 bytes per point), per-point d_x, d_y
// and multiplicity (12 bytes), four counters, one bit per point of the y order (a word per
// 32 points).
__host__ __device__ inline size_t sorted_off(int m) { return ((size_t)m * 8 + 15) & ~(size_t)15; }
__host__ __device__ inline size_t sorted_scratch(int m) {   // the part after the window
    int n = 1;
    while (n < m) n <<= 1;
    return (size_t)8 * n + (size_t)16 * m + (size_t)12 * m + 16 + (size_t)4 * ((m + 31) / 32);
}
__host__ __device__ inline size_t sorted_smem(int m) { return sorted_off(m) + sorted_scratch(m); }

// Work the brute-force and sort parts of a launch do, known from the window sizes alone
// (the data-dependent parts are counted on the device):
//  - a window on the brute-force path: m x m point x candidate distance evaluations per pass
//    (the point itself included);
//  - a window on the sorted path: the compare-exchange steps of its two bitonic sorts over
//    N = 2^ceil(log2 m) slots, each (N / 2) x log2(N) x (log2(N) + 1) / 2 (both together are
//    returned).
__host__ __device__ inline long long sort_cx_steps(int m) {
    int lg = 0;
    while ((1 << lg) < m) ++lg;
    const long long N = 1ll << lg;
    return N * (long long)lg * (long long)(lg + 1) / 2;
}
// Whether a window of m points in a launch of nt-thread CTAs takes the sorted path (the
// batched kernel's rule: windows of more than 64 points that run one per CTA, in a bucket of
// sort_mask, with their scratch in shared memory or in the launch's global scratch).
__host__ __device__ inline bool takes_sorted_path(int m, int nt, uint32_t sort_mask, bool gscratch,
                                                  int sort_min = 0) {
    if (m <= 64 || m < sort_min) return false;
    const int q = kBuckets - 1 - size_bucket(m);
    const bool one_per_cta = nt / 32 / warps_per_item(q, nt) == 1;
    return one_per_cta && ((sort_mask >> size_bucket(m)) & 1u) && (m <= kSortMax || gscratch);
}

// Shared memory of a batched launch whose largest window has max_m points; max_sorted is the
// largest window that takes the sorted path (0: none).
inline size_t batched_smem(int max_m, int nt, int max_sorted = 0) {
    size_t a = (size_t)max_m * 8;
    size_t b = (size_t)(nt / 32) * kWarpSlicePts * 8;   // the warps' small-window slices
    size_t c = max_sorted > 0 ? sorted_smem(max_sorted) : 0;
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

// Threads per CTA chosen for a batch whose largest window has max_m points and whose
// largest sorted-path window has max_sorted points (the sorted path runs one window per CTA:
// above nt_switch points, 1024 by default or as isycos_autotune chose, it takes 1024 threads,
// which hide its dependent loads).  max_sorted counts only windows whose scratch is in
// shared memory (at most kSortMax points).
inline int batched_threads(int max_m, int max_sorted = 0, int nt_switch = 1024) {
    return (max_m > 8192 || max_sorted > nt_switch) ? 1024 : 256;
}

}  // namespace isy
