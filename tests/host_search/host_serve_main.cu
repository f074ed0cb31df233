// Host-only test driver for the serving loop of libisycos (csrc/serve.cu) -- TEST
// INFRASTRUCTURE ONLY.
//
// The library's server threads admit, batch and retire the submitted queries as they do on
// the GPU, but every window of a round is scored by a stand-in engine with the CPU oracle's
// estimator (as in host_search_main.cu), so the results of served queries can be compared
// with the oracle's searches without a GPU, and the host threads can run under a race
// detector.
//
// usage: host_serve <series file> <queries file> [batch]
//   batch: run all queries in one isycos_search_queries call (engine lanes on host threads,
//   SYCOS_TD queries on lanes of their own) instead of serving them
//   series file: as for host_search
//   queries file: one query per line: pair mode t_begin t_end k s_min s_max pruning seed
//                 estimator cancel(0/1)
// output: per query "Q <index> <status> <found>" then "W <t_s> <t_e> <score> <mi>" lines.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <memory>
#include <thread>
#include <vector>

#include "search.h"
#include "bu_device.h"

extern "C" {
typedef struct {
    double mi, h_w, nmi;
    int64_t s_psi, s_log;
    double mi_exact, h_exact;
} orc_mi;
int orc_ksg_window_est(const float *x, const float *y, int64_t m, int32_t k, int32_t est,
                       int32_t *nx, int32_t *ny, int32_t *c, float *eps, float *dxm, float *dym,
                       orc_mi *out);
}

namespace {
std::vector<std::vector<float>> g_x, g_y;    // pair p: series ids 2p (x) and 2p + 1 (y)
thread_local std::vector<isycos_mi_out> t_open;   // each worker thread drives one lane

isycos_status score(int32_t xs, int32_t ys, int64_t start, int32_t m, int k, int est,
                    isycos_mi_out *o) {
    const std::vector<float> &x = g_x[(size_t)xs / 2], &y = g_y[(size_t)ys / 2];
    if (start < 0 || m < k + 1 || start + m > (int64_t)x.size()) return ISYCOS_E_INVAL;
    orc_mi r;
    if (orc_ksg_window_est(x.data() + start, y.data() + start, m, k, est, nullptr, nullptr, nullptr,
                           nullptr, nullptr, nullptr, &r) != 0)
        return ISYCOS_E_INVAL;
    *o = isycos_mi_out{r.mi, r.h_w, r.nmi, r.s_psi, r.s_log};
    return ISYCOS_OK;
}
}  // namespace

namespace isy {
isycos_status fail(isycos_ctx *, isycos_status st, const char *, ...) { return st; }
isycos_status cuda_fail(isycos_ctx *, cudaError_t, const char *) { return ISYCOS_E_CUDA; }
// The device-resident search and the buffer / statistics helpers it calls are not used by
// this harness (it drives the machines directly); they only have to link.
isycos_status dev_reserve(isycos_ctx *, DevBuf &, size_t) { return ISYCOS_E_NOMEM; }
cudaError_t bu_device_prepare(int, int *) { return cudaErrorNotSupported; }
cudaError_t bu_device_launch(const BuLaunch &, int, int, cudaStream_t) { return cudaErrorNotSupported; }
void add_stats(isycos_ctx *, int64_t, int64_t, int64_t, int64_t, int64_t) {}
static Lane g_lanes[kLaneSlots];
isycos_status get_lane(isycos_ctx *, int i, Lane **out) {
    if (i < 0 || i >= kLaneSlots) return ISYCOS_E_INVAL;
    *out = &g_lanes[i];
    return ISYCOS_OK;
}
void lane_release(isycos_ctx *, Lane &) {}
isycos_status engine_launch(isycos_ctx *, Lane &L, const HostWindow *w, int64_t n, int k, int est,
                            int32_t *, int32_t *, int32_t *, cudaStream_t) {
    t_open.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        isycos_status rc = score(w[i].xs, w[i].ys, w[i].start, w[i].m, k, est, &t_open[(size_t)i]);
        if (rc) return rc;
    }
    L.open.open = true;
    L.open.n = n;
    return ISYCOS_OK;
}
isycos_status engine_collect(isycos_ctx *, Lane &L, isycos_mi_out *out) {
    if (!L.open.open) return ISYCOS_OK;
    L.open.open = false;
    memcpy(out, t_open.data(), sizeof(isycos_mi_out) * (size_t)L.open.n);
    return ISYCOS_OK;
}
isycos_status engine_eval(isycos_ctx *ctx, Lane &L, const HostWindow *w, int64_t n, int k,
                          isycos_mi_out *out, int32_t *nx, int32_t *ny, int32_t *c, cudaStream_t st,
                          int est) {
    isycos_status rc = engine_launch(ctx, L, w, n, k, est, nx, ny, c, st);
    if (rc) return rc;
    return engine_collect(ctx, L, out);
}
isycos_status engine_eval_chains(isycos_ctx *, Lane &, const ChainSpec *specs, size_t n, int k,
                                 isycos_mi_out *out, int64_t n_out, cudaStream_t) {
    for (size_t c = 0; c < n; ++c)
        for (size_t i = 0; i < specs[c].starts.size(); ++i) {
            const int64_t o = specs[c].out_idx[i];
            if (o < 0) continue;
            if (o >= n_out) return ISYCOS_E_INVAL;
            isycos_status rc = score(specs[c].xs, specs[c].ys, specs[c].starts[i], specs[c].sizes[i],
                                     k, 0, &out[o]);
            if (rc) return rc;
        }
    return ISYCOS_OK;
}
}  // namespace isy

using namespace isy;

extern "C" isycos_status isycos_serve_submit(isycos_ctx *, int32_t, int32_t, int64_t, int64_t,
                                             const isycos_params *, uint64_t *);
extern "C" isycos_status isycos_serve_poll(isycos_ctx *, uint64_t, isycos_result_window *, int64_t,
                                           int64_t *, double *);
extern "C" isycos_status isycos_serve_cancel(isycos_ctx *, uint64_t);
extern "C" isycos_status isycos_search_queries(isycos_ctx *, int64_t, const isycos_query *,
                                               isycos_result_window *, int64_t, int64_t *);

int main(int argc, char **argv) {
    if (argc < 3) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    int32_t n_pairs = 0;
    int64_t n = 0;
    if (fread(&n_pairs, 4, 1, f) != 1 || fread(&n, 8, 1, f) != 1 || n_pairs <= 0 || n <= 0) return 2;
    g_x.assign((size_t)n_pairs, std::vector<float>((size_t)n));
    g_y.assign((size_t)n_pairs, std::vector<float>((size_t)n));
    for (int32_t p = 0; p < n_pairs; ++p)
        if (fread(g_x[(size_t)p].data(), 4, (size_t)n, f) != (size_t)n ||
            fread(g_y[(size_t)p].data(), 4, (size_t)n, f) != (size_t)n)
            return 2;
    fclose(f);

    {   // the oracle fills its tables on first use, single-threaded: do it before the server
        isycos_mi_out o;
        if (score(0, 1, 0, 16, 4, 0, &o) != ISYCOS_OK) return 2;
    }
    auto ctx = std::make_unique<isycos_ctx>();
    ctx->budget = (uint64_t)1 << 40;
    ctx->max_lanes = 4;
    ctx->opt_bu_device = 0;   // the host search machines (the device search needs a GPU)
    ctx->serve_slots = 6;   // fewer slots than queries: admission waits for retirements
    for (int32_t p = 0; p < n_pairs; ++p) {   // resident series: the host copies stand in
        ctx->series_ptr.push_back(g_x[(size_t)p].data());
        ctx->series_len.push_back(n);
        ctx->series_ptr.push_back(g_y[(size_t)p].data());
        ctx->series_len.push_back(n);
    }

    struct Q {
        isycos_params prm;
        int pair;
        int64_t tb, te;
        int cancel;
        uint64_t ticket = 0;
    };
    std::vector<Q> qs;
    FILE *qf = fopen(argv[2], "r");
    if (!qf) return 2;
    int pair, mode, k, s_min, s_max, pruning, est, cancel;
    long long tb, te;
    unsigned long long seed;
    while (fscanf(qf, "%d %d %lld %lld %d %d %d %d %llu %d %d", &pair, &mode, &tb, &te, &k, &s_min,
                  &s_max, &pruning, &seed, &est, &cancel) == 11) {
        Q q;
        memset(&q.prm, 0, sizeof(q.prm));
        q.prm.k = k;
        q.prm.sigma = 0.2;
        q.prm.tau = -1.0;
        q.prm.s_min = s_min;
        q.prm.s_max = s_max;
        q.prm.t_max_idle = -1;
        q.prm.sel_alpha = -1.0;
        q.prm.mode = mode;
        q.prm.pruning = pruning;
        q.prm.seed = seed;
        q.prm.estimator = est;
        q.pair = pair;
        q.tb = tb;
        q.te = te;
        q.cancel = cancel;
        qs.push_back(q);
    }
    fclose(qf);

    if (argc > 3 && strcmp(argv[3], "batch") == 0) {
        ctx->max_lanes = 8;
        std::vector<isycos_query> qa(qs.size());
        for (size_t i = 0; i < qs.size(); ++i)
            qa[i] = isycos_query{2 * qs[i].pair, 2 * qs[i].pair + 1, qs[i].tb, qs[i].te, qs[i].prm};
        const int64_t cap = 4096;
        std::vector<isycos_result_window> out(qs.size() * (size_t)cap);
        std::vector<int64_t> n_out(qs.size());
        const isycos_status st = isycos_search_queries(ctx.get(), (int64_t)qs.size(), qa.data(),
                                                       out.data(), cap, n_out.data());
        for (size_t i = 0; i < qs.size(); ++i) {
            printf("Q %zu %d %lld\n", i, (int)st, (long long)(st == ISYCOS_OK ? n_out[i] : 0));
            if (st == ISYCOS_OK)
                for (int64_t w = 0; w < n_out[i]; ++w) {
                    const isycos_result_window &r = out[i * (size_t)cap + (size_t)w];
                    printf("W %lld %lld %.17g %.17g\n", (long long)r.t_s, (long long)r.t_e, r.score, r.mi);
                }
        }
        return 0;
    }
    // submit from two threads at once, then poll every query to completion
    std::thread t2([&] {
        for (size_t i = 1; i < qs.size(); i += 2)
            if (isycos_serve_submit(ctx.get(), 2 * qs[i].pair, 2 * qs[i].pair + 1, qs[i].tb, qs[i].te,
                                    &qs[i].prm, &qs[i].ticket) != ISYCOS_OK)
                qs[i].ticket = 0;
    });
    for (size_t i = 0; i < qs.size(); i += 2)
        if (isycos_serve_submit(ctx.get(), 2 * qs[i].pair, 2 * qs[i].pair + 1, qs[i].tb, qs[i].te,
                                &qs[i].prm, &qs[i].ticket) != ISYCOS_OK)
            qs[i].ticket = 0;
    t2.join();
    for (Q &q : qs)
        if (q.cancel && q.ticket) isycos_serve_cancel(ctx.get(), q.ticket);
    std::vector<isycos_result_window> buf(1 << 16);
    for (size_t i = 0; i < qs.size(); ++i) {
        if (!qs[i].ticket) {
            printf("Q %zu submit-failed 0\n", i);
            continue;
        }
        for (int spin = 0;; ++spin) {
            int64_t n_out = 0;
            const isycos_status st = isycos_serve_poll(ctx.get(), qs[i].ticket, buf.data(),
                                                       (int64_t)buf.size(), &n_out, nullptr);
            if (st == ISYCOS_PENDING) {
                if (spin > 600000) return 5;   // ten minutes
                std::this_thread::sleep_for(std::chrono::milliseconds(1));
                continue;
            }
            printf("Q %zu %d %lld\n", i, (int)st, (long long)(st == ISYCOS_OK ? n_out : 0));
            if (st == ISYCOS_OK)
                for (int64_t w = 0; w < n_out; ++w)
                    printf("W %lld %lld %.17g %.17g\n", (long long)buf[(size_t)w].t_s,
                           (long long)buf[(size_t)w].t_e, buf[(size_t)w].score, buf[(size_t)w].mi);
            break;
        }
    }
    serve_shutdown(ctx.get());
    return 0;
}
