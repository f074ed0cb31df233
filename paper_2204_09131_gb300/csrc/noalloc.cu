// Window MI with no allocation: isycos_mi_windows_noalloc.
//
// Some callers cannot call cudaMalloc: code that runs under a runtime which owns all device
// memory (a framework's caching allocator, or a process held to a fixed device-memory
// budget that it hands out itself), and latency-critical loops where cudaMalloc / cudaFree
// would synchronise the device.  For them this entry point runs the same persistent,
// size-bucketed MI kernel as isycos_mi_windows_device, but takes every byte of its work
// memory (window items, bucket table, counters) from one file-scope static device array,
// and its digamma / log tables from static device arrays filled once per device.  The
// caller passes the inputs (one pair of series, window starts and sizes) and the output
// array, all in device memory.
//
// The static array lives on every GPU that loads the library until the process exits.  Its
// device address is obtained with cudaGetSymbolAddress on the first call on each device
// (with that device current); that first call also uploads the tables, so it should come
// before any stream capture.  All calls share the array and it keeps the last call's
// contents, so calls that overlap on the GPU (different streams, or host threads) race;
// every call clears the counters it needs before use.
#include <stdint.h>

#include <mutex>

#include "isycos_internal.h"

namespace isy {
namespace {

constexpr int kNoallocMaxDevices = 64;
constexpr size_t kCtlBytes = 1024;                       // counters and bucket table
constexpr size_t kItemBytes = sizeof(WorkItem);          // 32
constexpr size_t kScratchBytes =
    kCtlBytes + (size_t)ISYCOS_NOALLOC_MAX_WINDOWS * (kItemBytes + 2 * sizeof(int32_t));

static_assert(128 + sizeof(BucketTable) <= kCtlBytes, "control block too small");

// The scratch array (about 2.6 MiB for 65,536 windows) and the fixed-point tables.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) long long g_psi_fx[kTableN];
static __device__ __align__(256) long long g_log_fx[kTableN];

// Host-side images of the tables, built once (static storage, no allocation).
static long long h_psi_fx[kTableN];
static long long h_log_fx[kTableN];
static bool h_tables_built = false;

struct DevState {
    bool ready = false;
    unsigned char *scratch = nullptr;
    long long *psi_fx = nullptr;
    long long *log_fx = nullptr;
};
static DevState g_dev[kNoallocMaxDevices];
static std::mutex g_mu;

struct NoallocPrep {
    const float *x;
    const float *y;
    int64_t n;
    const int64_t *starts;
    const int32_t *sizes;
    int64_t n_w;
    int32_t k;
    int32_t max_m;
    int32_t nt;
    unsigned char *scratch;
    isycos_mi_out *out;
};

__device__ __forceinline__ int32_t *ctl_counts(unsigned char *s) { return reinterpret_cast<int32_t *>(s); }
__device__ __forceinline__ BucketTable *ctl_table(unsigned char *s) {
    return reinterpret_cast<BucketTable *>(s + 128);
}
__device__ __forceinline__ WorkItem *ctl_items(unsigned char *s) {
    return reinterpret_cast<WorkItem *>(s + kCtlBytes);
}
__device__ __forceinline__ int32_t *ctl_slot(unsigned char *s) {
    return reinterpret_cast<int32_t *>(s + kCtlBytes + (size_t)ISYCOS_NOALLOC_MAX_WINDOWS * kItemBytes);
}
__device__ __forceinline__ int32_t *ctl_pos(unsigned char *s) {
    return ctl_slot(s) + ISYCOS_NOALLOC_MAX_WINDOWS;
}

// Validate each window against the pair and take its place in its size bucket.
__global__ void noalloc_classify(NoallocPrep a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_w) return;
    const int64_t s = a.starts[i];
    const int32_t m = a.sizes[i];
    const bool ok = m >= a.k + 1 && m <= a.max_m && s >= 0 && s + m <= a.n;
    if (!ok) {
        ctl_slot(a.scratch)[i] = -1;   // invalid: its NaN result is the only report
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        a.out[i].mi = nan;
        a.out[i].h_w = nan;
        a.out[i].nmi = nan;
        a.out[i].s_psi = 0;
        a.out[i].s_log = 0;
        return;
    }
    const int b = 32 - __clz(m - 1);
    const int q = kBuckets - 1 - b;
    ctl_slot(a.scratch)[i] = q;
    ctl_pos(a.scratch)[i] = atomicAdd(ctl_counts(a.scratch) + q, 1);
}

__global__ void noalloc_table(NoallocPrep a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    fill_bucket_table(ctl_table(a.scratch), ctl_counts(a.scratch), a.nt);
}

__global__ void noalloc_scatter(NoallocPrep a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_w) return;
    const int q = ctl_slot(a.scratch)[i];
    if (q < 0) return;
    WorkItem it;
    it.x = a.x + a.starts[i];
    it.y = a.y + a.starts[i];
    it.m = a.sizes[i];
    it.out = (int32_t)i;
    it.pts = -1;
    ctl_items(a.scratch)[ctl_table(a.scratch)->item_off[q] + ctl_pos(a.scratch)[i]] = it;
}

// The tables the batched kernel reads, built by the same routine as a context's.
void build_host_tables() {
    if (h_tables_built) return;
    fill_fixed_tables(h_psi_fx, h_log_fx);
    h_tables_built = true;
}

// Once per device, with the device current: resolve the static arrays' device addresses
// and upload the tables.
isycos_status setup_device(int dev) {
    std::lock_guard<std::mutex> g(g_mu);
    DevState &d = g_dev[dev];
    if (d.ready) return ISYCOS_OK;
    build_host_tables();
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return ISYCOS_E_CUDA;
    d.scratch = reinterpret_cast<unsigned char *>(p);
    if (cudaGetSymbolAddress(&p, g_psi_fx) != cudaSuccess) return ISYCOS_E_CUDA;
    d.psi_fx = reinterpret_cast<long long *>(p);
    if (cudaGetSymbolAddress(&p, g_log_fx) != cudaSuccess) return ISYCOS_E_CUDA;
    d.log_fx = reinterpret_cast<long long *>(p);
    if (cudaMemcpyToSymbol(g_psi_fx, h_psi_fx, sizeof(h_psi_fx)) != cudaSuccess) return ISYCOS_E_CUDA;
    if (cudaMemcpyToSymbol(g_log_fx, h_log_fx, sizeof(h_log_fx)) != cudaSuccess) return ISYCOS_E_CUDA;
    d.ready = true;
    return ISYCOS_OK;
}

}  // namespace
}  // namespace isy

using namespace isy;

extern "C" isycos_status isycos_mi_windows_noalloc(const float *d_x, const float *d_y, int64_t n,
                                                   const int64_t *d_starts, const int32_t *d_sizes,
                                                   int64_t n_w, int32_t k, int32_t max_m,
                                                   isycos_mi_out *d_out, void *cuda_stream) {
    if (k < 1 || k > kMaxK) return ISYCOS_E_INVAL;
    if (n_w < 0 || n_w > ISYCOS_NOALLOC_MAX_WINDOWS) return ISYCOS_E_INVAL;   // beyond the scratch
    if (max_m < k + 1 || max_m > kMaxM) return ISYCOS_E_INVAL;
    if (n_w == 0) return ISYCOS_OK;
    if (!d_x || !d_y || n < 1 || !d_starts || !d_sizes || !d_out) return ISYCOS_E_INVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return ISYCOS_E_CUDA;
    isycos_status rc = setup_device(dev);
    if (rc) return rc;
    const DevState &d = g_dev[dev];
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);

    const int nt = batched_threads(max_m);
    const size_t smem = batched_smem(max_m, nt);
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return ISYCOS_E_CUDA;
    // Raise the kernel's dynamic shared-memory limit to the device maximum: never lower it,
    // so that other callers of the same kernel keep the limit they set.
    if (set_batched_smem(k, nt, (size_t)optin - 1024) != cudaSuccess) return ISYCOS_E_CUDA;
    int per_sm = 0, n_sm = 0;
    if (batched_occupancy(k, nt, smem, &per_sm) != cudaSuccess || per_sm < 1) return ISYCOS_E_CUDA;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ISYCOS_E_CUDA;

    NoallocPrep pa;
    pa.x = d_x;
    pa.y = d_y;
    pa.n = n;
    pa.starts = d_starts;
    pa.sizes = d_sizes;
    pa.n_w = n_w;
    pa.k = k;
    pa.max_m = max_m;
    pa.nt = nt;
    pa.scratch = d.scratch;
    pa.out = d_out;
    // bucket counters and the three work counters start at zero on every call
    if (cudaMemsetAsync(d.scratch, 0, 128, st) != cudaSuccess) return ISYCOS_E_CUDA;
    const int blocks = (int)((n_w + 255) / 256);
    noalloc_classify<<<blocks, 256, 0, st>>>(pa);
    noalloc_table<<<1, 32, 0, st>>>(pa);
    noalloc_scatter<<<blocks, 256, 0, st>>>(pa);
    if (cudaGetLastError() != cudaSuccess) return ISYCOS_E_CUDA;

    BatchArgs a;
    a.items = reinterpret_cast<const WorkItem *>(d.scratch + kCtlBytes);
    a.table = reinterpret_cast<const BucketTable *>(d.scratch + 128);
    a.queue = reinterpret_cast<int32_t *>(d.scratch) + kBuckets;
    a.psi_fx = d.psi_fx;
    a.log_fx = d.log_fx;
    a.out = d_out;
    a.nx = a.ny = a.c = nullptr;
    a.k = k;
    a.nt = nt;
    a.sort_mask = 0;          // brute-force path only
    a.est = 0;                // Kraskov's second estimator (Eq. KSGmi)
    a.sort_min = 0;
    a.inv_k = 1.0 / (double)k;
    a.gscratch = nullptr;
    a.gscratch_stride = 0;
    if (launch_batched(a, n_sm * per_sm, smem, st) != cudaSuccess) return ISYCOS_E_CUDA;
    return ISYCOS_OK;
}
