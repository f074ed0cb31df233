// isycos_autotune: choose, per window-size bucket, between the brute-force and the
// sorted-strip MI paths by timing both on this GPU.  Both paths give identical results (every
// comparison is the same binary32 operation), so the choice changes speed only.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "isycos_internal.h"
#include "runtime.h"

namespace isy {
namespace {

// The probe pair: x ~ N(0, 1), y = 0.6 x + 0.8 N(0, 1) (a moderately dependent pair, so that
// the outward scans of the sorted path see typical neighbour distances), from SplitMix64 and
// the Box-Muller transform.
void probe_pair(int64_t n, std::vector<float> &x, std::vector<float> &y) {
    uint64_t state = 0x243F6A8885A308D3ULL;
    auto next = [&state]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    };
    auto unif = [&next]() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
    auto normal = [&unif]() {
        const double u = unif(), v = unif();
        return sqrt(-2.0 * log(u)) * cos(6.283185307179586 * v);
    };
    x.resize((size_t)n);
    y.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const double a = normal(), b = normal();
        x[(size_t)i] = (float)a;
        y[(size_t)i] = (float)(0.6 * a + 0.8 * b);
    }
}

}  // namespace
}  // namespace isy

using namespace isy;

extern "C" isycos_status isycos_autotune(isycos_ctx *ctx, int32_t k, isycos_tuning *out) {
    if (!ctx) return ISYCOS_E_INVAL;
    if (k < 1 || k > kMaxK) return fail(ctx, ISYCOS_E_INVAL, "autotune: k = %d outside [1, %d]", k, kMaxK);
    constexpr int64_t kLen = 1 << 16;
    std::vector<float> hx, hy;
    probe_pair(kLen, hx, hy);
    int32_t xs = -1, ys = -1;
    isycos_status rc = isycos_put_series(ctx, hx.data(), kLen, 0, &xs);
    if (!rc) rc = isycos_put_series(ctx, hy.data(), kLen, 0, &ys);
    isycos_tuning res;
    memset(&res, 0, sizeof(res));
    res.k = k;
    if (!rc) {
        std::lock_guard<std::mutex> g(ctx->engine_mu);
        cudaSetDevice(ctx->device);
        // the probes are not the caller's work: keep the counters as they were
        isycos_stats saved_stats;
        std::vector<std::pair<float, float>> saved_iv;
        {
            std::lock_guard<std::mutex> g2(ctx->stats_mu);
            saved_stats = ctx->stats;
            saved_iv = ctx->kernel_iv;
        }
        const int saved_opt = ctx->opt_kernel;
        const bool saved_tuned = ctx->tuned[k];
        const uint32_t saved_mask = ctx->tuned_sort_mask[k];
        ctx->opt_kernel = 0;
        ctx->tuned[k] = true;
        Lane &L = *ctx->lanes[0].load();
        // several waves, as in a TD layer (fewer for the largest windows, whose brute-force
        // launches take tens of milliseconds)
        const int n_sm = std::max(1, ctx->n_sm);
        res.n_windows = 8 * n_sm;
        uint32_t chosen = 0;
        std::vector<HostWindow> w((size_t)res.n_windows);
        std::vector<isycos_mi_out> r((size_t)res.n_windows);
        for (int b = 0; b < 15 && !rc; ++b) {
            if (!((kSortBuckets >> b) & 1u)) continue;
            const int n_w = b <= 12 ? 8 * n_sm : (b == 13 ? 2 * n_sm : n_sm);
            const int m = 3 << (b - 2);   // the middle of bucket b: 2^(b-1) < m <= 2^b
            res.window_size[b] = m;
            for (int i = 0; i < n_w; ++i)
                w[(size_t)i] = HostWindow{xs, ys, (int64_t)i * ((kLen - m) / n_w), m};
            double best[2] = {0.0, 0.0};
            for (int path = 0; path < 2 && !rc; ++path) {
                ctx->tuned_sort_mask[k] = path ? (1u << b) : 0u;
                double t = 1e30;
                for (int rep = 0; rep < 4 && !rc; ++rep) {   // one warm-up, best of three
                    rc = engine_eval(ctx, L, w.data(), n_w, k, r.data(), nullptr, nullptr, nullptr,
                                     L.stream, 0);
                    float ms = 0.0f;
                    if (!rc && cudaEventElapsedTime(&ms, L.ev_start, L.ev_stop) != cudaSuccess)
                        rc = fail(ctx, ISYCOS_E_CUDA, "autotune: event timing");
                    if (rep > 0) t = std::min(t, (double)ms);
                }
                best[path] = t;
            }
            res.brute_ms[b] = best[0];
            res.sorted_ms[b] = best[1];
            if (best[1] < best[0]) chosen |= 1u << b;
        }
        ctx->opt_kernel = saved_opt;
        if (!rc) {
            ctx->tuned[k] = true;
            ctx->tuned_sort_mask[k] = chosen;
            res.sorted_buckets = chosen;
        } else {
            ctx->tuned[k] = saved_tuned;
            ctx->tuned_sort_mask[k] = saved_mask;
        }
        std::lock_guard<std::mutex> g2(ctx->stats_mu);
        ctx->stats = saved_stats;
        ctx->kernel_iv = saved_iv;
    }
    if (xs >= 0) isycos_drop_series(ctx, xs);
    if (ys >= 0) isycos_drop_series(ctx, ys);
    if (!rc && out) *out = res;
    return rc;
}
