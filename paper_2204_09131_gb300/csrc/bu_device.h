// Device-resident SYCOS_BU (arXiv 2204.09131, Sec. 5.2, Algorithm 2, with the noise pruning
// of Sec. 6.3): every climb decision runs on the GPU, next to the window-MI evaluations it
// reads, so a whole search is one kernel launch instead of one launch per climb step.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "isycos.h"

namespace isy {

// Largest LAHC history length and idle limit the device search keeps on chip (larger ones
// take the host search).
constexpr int kBuMaxH = 64;
constexpr int kBuMaxIdle = 31;

// One SYCOS_BU query as the kernel reads it (parameters already resolved).
struct DevBuQuery {
    const float *x;
    const float *y;
    int64_t t_begin, t_end;   // [t_begin, t_end)
    double sigma, tau;
    uint64_t seed;
    int32_t k, score_kind, s_min, s_max, delta, h, t_max_idle, p, pruning, max_steps, est;
    int32_t pad;
};

// What the kernel reports per query.
struct DevBuResult {
    int64_t n_found;          // correlated windows found (only the first `cap` are stored)
    int64_t evals;            // window scores read by the decisions (Algorithm 2's evaluations)
    int64_t windows;          // windows evaluated on the GPU (with the speculative ones)
    int64_t pairs;            // their brute-force ordered pairs, sum m (m - 1)
    int64_t rounds;           // evaluate / decide rounds of the query's CTA
    int64_t units;            // brute-force work units (32 or 64 points of one window)
    int64_t work_bf;          // brute-force point x candidate evaluations (both passes)
    int64_t cycles[3];        // clock64 cycles in decide + ask, evaluate, finish
    int64_t evals_by_size[15];
    int64_t windows_by_size[15];
    int32_t status;           // 0 done, 1 time limit reached before the search finished
    int32_t pad;
};

struct BuLaunch {
    const DevBuQuery *q;
    int32_t n_q;
    int32_t spec_climbs;      // climbs asked ahead, assuming each ends where it starts
    DevBuResult *res;         // n_q entries
    isycos_result_window *found;   // query i's windows at found + i * cap
    int64_t cap;
    int32_t *queue;           // next query to take (zero at launch)
    const long long *psi_fx;
    const long long *log_fx;
    uint64_t limit_ns;        // a CTA stops taking rounds this long after it started (0: none)
};

// Score slots of a CTA's shared-memory cache (16 bytes each: window key, score).
constexpr int kBuCacheSlots = 8192;
// Points of the series tile a CTA keeps in shared memory around its search cursor.
constexpr int kBuTile = 4096;
// Threads per CTA of the device search.
constexpr int kBuThreads = 512;

// Dynamic shared memory of one CTA and CTAs per SM for k neighbours.
size_t bu_device_smem();
cudaError_t bu_device_prepare(int k, int *blocks_per_sm);
cudaError_t bu_device_launch(const BuLaunch &a, int k, int grid, cudaStream_t st);

}  // namespace isy
