// isycos_autotune: choose, per window-size bucket, between the brute-force and the
// sorted-strip MI paths by timing both on this GPU.  Both paths give identical results (every
// comparison is the same binary32 operation), so the choice changes speed only.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
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

// One launch of n windows of m points spread over the probe pair, best of three timed runs
// after one warm-up, with the tuning fields of k set as given.
isycos_status time_launch(isycos_ctx *ctx, Lane &L, int k, int32_t xs, int32_t ys, int64_t len,
                          int m, int n, std::vector<HostWindow> &w, std::vector<isycos_mi_out> &r,
                          double *ms_out) {
    w.resize((size_t)n);
    r.resize((size_t)n);
    for (int i = 0; i < n; ++i) w[(size_t)i] = HostWindow{xs, ys, (int64_t)i * ((len - m) / n), m};
    double t = 1e30;
    isycos_status rc = ISYCOS_OK;
    for (int rep = 0; rep < 4 && !rc; ++rep) {
        rc = engine_eval(ctx, L, w.data(), n, k, r.data(), nullptr, nullptr, nullptr, L.stream, 0);
        float ms = 0.0f;
        if (!rc && cudaEventElapsedTime(&ms, L.ev_start, L.ev_stop) != cudaSuccess)
            rc = fail(ctx, ISYCOS_E_CUDA, "autotune: event timing");
        if (rep > 0) t = std::min(t, (double)ms);
    }
    *ms_out = t;
    return rc;
}

std::string gpu_name(const isycos_ctx *ctx) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, ctx->device) != cudaSuccess) return "unknown";
    std::string n(prop.name);
    for (char &c : n)
        if (c == '"' || c == '\\' || c == '\n') c = '_';
    return n;
}

// One line of the tuning file:
// {"gpu": "<name>", "k": 4, "sorted_buckets": 32256, "sort_min": 288, "nt_switch": 1024}
struct TuneLine {
    std::string gpu;
    int k = 0, sort_min = 0, nt_switch = 0;
    unsigned long sorted_buckets = 0;
    bool ok = false;
};

TuneLine parse_line(const std::string &line) {
    TuneLine t;
    const size_t g = line.find("\"gpu\": \"");
    if (g == std::string::npos) return t;
    const size_t a = g + 8, b = line.find('"', a);
    if (b == std::string::npos) return t;
    t.gpu = line.substr(a, b - a);
    auto num = [&line](const char *key, long *v) {
        const size_t p = line.find(key);
        if (p == std::string::npos) return false;
        return sscanf(line.c_str() + p + strlen(key), "%ld", v) == 1;
    };
    long k = 0, sb = 0, smin = 0, nts = 0;
    t.ok = num("\"k\": ", &k) && num("\"sorted_buckets\": ", &sb) && num("\"sort_min\": ", &smin) &&
           num("\"nt_switch\": ", &nts) && k >= 1 && k <= kMaxK && sb >= 0 && smin >= 0 &&
           (nts == 512 || nts == 1024);
    t.k = (int)k;
    t.sorted_buckets = (unsigned long)sb & kSortBuckets;
    t.sort_min = (int)smin;
    t.nt_switch = (int)nts;
    return t;
}

}  // namespace

void load_tunings(isycos_ctx *ctx) {
    const char *path = getenv("ISYCOS_TUNING_FILE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    const std::string me = gpu_name(ctx);
    char buf[512];
    while (fgets(buf, sizeof(buf), f)) {
        const TuneLine t = parse_line(buf);
        if (!t.ok || t.gpu != me) continue;
        ctx->tuned[t.k] = true;
        ctx->tuned_sort_mask[t.k] = (uint32_t)t.sorted_buckets;
        ctx->tuned_sort_min[t.k] = t.sort_min;
        ctx->tuned_nt_switch[t.k] = t.nt_switch;
    }
    fclose(f);
}

void store_tuning(const isycos_ctx *ctx, int k) {
    const char *path = getenv("ISYCOS_TUNING_FILE");
    if (!path || !*path) return;
    const std::string me = gpu_name(ctx);
    std::vector<std::string> keep;
    if (FILE *f = fopen(path, "r")) {
        char buf[512];
        while (fgets(buf, sizeof(buf), f)) {
            const TuneLine t = parse_line(buf);
            if (t.ok && !(t.gpu == me && t.k == k)) keep.push_back(std::string(buf));
        }
        fclose(f);
    }
    char line[512];
    snprintf(line, sizeof(line),
             "{\"gpu\": \"%s\", \"k\": %d, \"sorted_buckets\": %u, \"sort_min\": %d, \"nt_switch\": %d}\n",
             me.c_str(), k, ctx->tuned_sort_mask[k], ctx->tuned_sort_min[k],
             ctx->tuned_nt_switch[k] > 0 ? ctx->tuned_nt_switch[k] : 1024);
    keep.push_back(line);
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    bool ok = true;
    for (const std::string &l : keep) ok = ok && fputs(l.c_str(), f) >= 0;
    ok = (fclose(f) == 0) && ok;
    if (ok) rename(tmp.c_str(), path);
    else remove(tmp.c_str());
}

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
        const int saved_min = ctx->tuned_sort_min[k], saved_nts = ctx->tuned_nt_switch[k];
        ctx->opt_kernel = 0;
        ctx->tuned[k] = true;
        ctx->tuned_sort_min[k] = 0;
        ctx->tuned_nt_switch[k] = 0;
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
        // The crossover inside the smallest sorted bucket b (sorted won at its middle, 3/4 of
        // 2^b): probe 1/8, 2/8 and 3/8 into it; the first size where sorted wins is sort_min.
        int sort_min = 0;
        int b0 = -1;
        for (int b = 0; b < 15; ++b)
            if ((chosen >> b) & 1u) {
                b0 = b;
                break;
            }
        if (!rc && b0 >= 9 && b0 <= 12) {
            const int lo = 1 << (b0 - 1);
            sort_min = res.window_size[b0];
            for (int j = 0; j < 3 && !rc; ++j) {
                const int m = lo + (j + 1) * lo / 8;
                res.cross_size[j] = m;
                double t[2];
                for (int path = 0; path < 2 && !rc; ++path) {
                    ctx->tuned_sort_mask[k] = path ? (1u << b0) : 0u;
                    rc = time_launch(ctx, L, k, xs, ys, kLen, m, 8 * n_sm, w, r, &t[path]);
                }
                res.cross_brute_ms[j] = t[0];
                res.cross_sorted_ms[j] = t[1];
                if (!rc && t[1] < t[0] && sort_min == res.window_size[b0]) sort_min = m;
            }
        }
        // Threads of a launch whose largest sorted window has 513..1024 points: 256 (the
        // sort in registers, several windows' CTAs per SM) or 1024.
        int nt_sw = 1024;
        if (!rc && ((chosen >> 10) & 1u)) {
            ctx->tuned_sort_mask[k] = 1u << 10;
            double t[2];
            for (int v = 0; v < 2 && !rc; ++v) {
                ctx->tuned_nt_switch[k] = v == 0 ? 1024 : 512;
                rc = time_launch(ctx, L, k, xs, ys, kLen, 768, 8 * n_sm, w, r, &t[v]);
            }
            res.nt_ms[0] = t[0];
            res.nt_ms[1] = t[1];
            if (!rc && t[1] < t[0]) nt_sw = 512;
        }
        ctx->opt_kernel = saved_opt;
        if (!rc) {
            ctx->tuned[k] = true;
            ctx->tuned_sort_mask[k] = chosen;
            ctx->tuned_sort_min[k] = sort_min;
            ctx->tuned_nt_switch[k] = nt_sw;
            res.sorted_buckets = chosen;
            res.sort_min = sort_min;
            res.nt_switch = nt_sw;
            store_tuning(ctx, k);
        } else {
            ctx->tuned[k] = saved_tuned;
            ctx->tuned_sort_mask[k] = saved_mask;
            ctx->tuned_sort_min[k] = saved_min;
            ctx->tuned_nt_switch[k] = saved_nts;
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

extern "C" isycos_status isycos_get_tuning(isycos_ctx *ctx, int32_t k, uint32_t *sorted_buckets,
                                           int32_t *sort_min, int32_t *nt_switch) {
    if (!ctx) return ISYCOS_E_INVAL;
    if (k < 1 || k > kMaxK) return fail(ctx, ISYCOS_E_INVAL, "k = %d outside [1, %d]", k, kMaxK);
    if (!ctx->tuned[k]) return fail(ctx, ISYCOS_E_NOTFOUND, "k = %d is not tuned", k);
    if (sorted_buckets) *sorted_buckets = ctx->tuned_sort_mask[k];
    if (sort_min) *sort_min = ctx->tuned_sort_min[k];
    if (nt_switch) *nt_switch = ctx->tuned_nt_switch[k] > 0 ? ctx->tuned_nt_switch[k] : 1024;
    return ISYCOS_OK;
}
