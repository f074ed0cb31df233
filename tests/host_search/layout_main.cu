// Host-only checks of the launch layout shared by the host runtime and the batched MI
// kernel (csrc/isycos_internal.h) -- TEST INFRASTRUCTURE ONLY.  Prints "ok" or the first
// violated invariant and exits non-zero.
#include <stdio.h>
#include <stdlib.h>

#include "isycos_internal.h"

using namespace isy;

static int ref_bucket(int m) {   // smallest b with m <= 2^b, by definition
    int b = 0;
    while ((1 << b) < m) ++b;
    return b;
}

#define CHECK(cond, ...)                                                      \
    do {                                                                      \
        if (!(cond)) {                                                        \
            printf("FAIL %s:%d: ", __FILE__, __LINE__);                       \
            printf(__VA_ARGS__);                                              \
            printf("\n");                                                    \
            return 1;                                                         \
        }                                                                     \
    } while (0)

int main() {
    // size buckets (count of leading zeros) against the definition
    for (int m = 1; m <= 4 * kMaxM; ++m) {
        CHECK(size_bucket(m) == ref_bucket(m), "size_bucket(%d) = %d, want %d", m, size_bucket(m), ref_bucket(m));
        if (m <= kMaxM) CHECK(bucket_slot(m) == kBuckets - 1 - ref_bucket(m), "bucket_slot(%d)", m);
    }
    // every window size fits its bucket's warps, and a warp's staging slice holds the
    // largest single-warp window
    CHECK((1 << (kBuckets - 1 - kSmallSlot)) <= kWarpSlicePts, "warp slice");
    for (int nt : {256, 1024}) {
        const int W = nt / 32;
        for (int q = 0; q < kSmallSlot; ++q) {
            const int b = kBuckets - 1 - q, wpw = warps_per_item(q, nt);
            CHECK(wpw >= 1 && wpw <= W && (wpw & (wpw - 1)) == 0, "wpw %d (q %d nt %d)", wpw, q, nt);
            CHECK(wpw * kBlockPts >= (1 << b) || wpw == W, "wpw %d too small for 2^%d (nt %d)", wpw, b, nt);
            // several items of a job share the tile: their slices must fit the small-window
            // staging area
            if (W / wpw > 1)
                CHECK((size_t)(W / wpw) * wpw * kBlockPts * 8 <= batched_smem(1 << b, nt),
                      "job slices of bucket %d exceed the tile (nt %d)", b, nt);
        }
    }
    // bucket tables for random counts: offsets are prefix sums, jobs cover every CTA-job item
    // once, the warp phase starts at the first small item, the grid covers the work
    srand(7);
    for (int trial = 0; trial < 20000; ++trial) {
        const int nt = (trial & 1) ? 1024 : 256, W = nt / 32;
        int32_t count[kBuckets];
        for (int q = 0; q < kBuckets; ++q) count[q] = (rand() % 4 == 0) ? 0 : rand() % 300;
        BucketTable T;
        fill_bucket_table(&T, count, nt);
        int items = 0, jobs = 0;
        for (int q = 0; q < kBuckets; ++q) {
            CHECK(T.item_off[q] == items, "item_off[%d]", q);
            CHECK(T.job_off[q] == jobs, "job_off[%d]", q);
            CHECK(T.count[q] == count[q], "count[%d]", q);
            items += count[q];
            if (q < kSmallSlot) {
                const int per_job = W / T.wpw[q];
                CHECK(per_job >= 1 && per_job * T.wpw[q] <= W, "per_job (q %d)", q);
                jobs += (count[q] + per_job - 1) / per_job;
            } else {
                CHECK(T.wpw[q] == 1, "wpw of a small bucket");
            }
        }
        CHECK(T.n_items == items && T.total_jobs == jobs, "totals");
        CHECK(T.small_first == T.item_off[kSmallSlot], "small_first");
        const int n_small = items - T.small_first;
        CHECK(batched_grid_need(T, nt) * W >= jobs * W + n_small, "grid need");
    }
    // shared memory of a launch covers the largest window, the small-window slices and the
    // sorted path's layout; the sorted layout is its offset plus its scratch
    for (int m = 2; m <= kSortMax; m += (m < 600 ? 1 : 37)) {
        CHECK(sorted_smem(m) == sorted_off(m) + sorted_scratch(m), "sorted_smem(%d)", m);
        CHECK(sorted_off(m) >= (size_t)m * 8 && sorted_off(m) % 16 == 0, "sorted_off(%d)", m);
        for (int nt : {256, 1024}) {
            const size_t s = batched_smem(m, nt, m > 256 ? m : 0);
            CHECK(s >= (size_t)m * 8 && s >= (size_t)(nt / 32) * kWarpSlicePts * 8, "batched_smem(%d, %d)", m, nt);
            if (m > 256) CHECK(s >= sorted_smem(m), "sorted smem(%d, %d)", m, nt);
        }
    }
    CHECK(batched_threads(8193) == 1024 && batched_threads(4096, 1025) == 1024 &&
              batched_threads(4096, 1024) == 256 && batched_threads(100) == 256,
          "batched_threads");
    printf("ok\n");
    return 0;
}
