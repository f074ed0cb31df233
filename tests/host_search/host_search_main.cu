// Host-only test driver for the search machines of libisycos (SYCOS_TD, SYCOS_BU, the
// selection of Algorithm 3, the chunks of Algorithm 4) -- TEST INFRASTRUCTURE ONLY.
//
// It links the library's search logic (csrc/search.cu) with a stand-in for the GPU engine
// whose window scores come from the CPU oracle (oracle/isycos_oracle.c).  Every round of
// windows the machines ask for is scored window by window on the host, so the decisions,
// the found windows and the decided-window counts can be compared with the oracle's own
// searches without a GPU.  The MI kernels themselves are covered by the GPU tests.
//
// usage: host_search <series file> key=value ...
//   series file: int32 n_pairs, int64 n, then per pair n float32 x values and n y values
//   keys: the isycos_params fields (k, score_kind, sigma, tau, s_min, s_max, delta_td,
//         delta_bu, h, t_max_idle, p, mode, pruning, max_steps, seed, sel_partitions,
//         sel_samples, sel_alpha, sel_rho, chunks, estimator), t_begin, t_end,
//         spec (climbs asked ahead), incremental (0, 1, 2),
//         table (a text file of "t_s t_e score" lines: every window then scores from it, MI and
//         normalised score alike, instead of the oracle's estimator), table_default (the score
//         of a window the table does not list, 0 by default)
// output: per pair "M <pair> <found> <decided>" then "W <t_s> <t_e> <score> <mi>" lines.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "search.h"
#include "bu_device.h"

extern "C" {
// The oracle's window estimator (see oracle/isycos_oracle.c for its contract).
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
std::vector<std::vector<float>> g_x, g_y;   // series by id: pair p has ids 2p (x), 2p + 1 (y)
std::vector<isycos_mi_out> g_open;          // results of the open launch
int64_t g_windows = 0, g_rounds = 0;
bool g_use_table = false;                                   // scores from a table, not the estimator
std::map<std::pair<int64_t, int64_t>, double> g_table;     // (t_s, t_e) -> score
double g_table_default = 0.0;

isycos_status score(int32_t xs, int32_t ys, int64_t start, int32_t m, int k, int est,
                    isycos_mi_out *o) {
    const std::vector<float> &x = g_x[(size_t)xs / 2], &y = g_y[(size_t)ys / 2];
    if (start < 0 || m < k + 1 || start + m > (int64_t)x.size()) return ISYCOS_E_INVAL;
    if (g_use_table) {
        auto it = g_table.find({start, start + m - 1});
        const double v = it == g_table.end() ? g_table_default : it->second;
        *o = isycos_mi_out{v, 1.0, v, 0, 0};
        ++g_windows;
        return ISYCOS_OK;
    }
    orc_mi r;
    if (orc_ksg_window_est(x.data() + start, y.data() + start, m, k, est, nullptr, nullptr, nullptr,
                           nullptr, nullptr, nullptr, &r) != 0)
        return ISYCOS_E_INVAL;
    *o = isycos_mi_out{r.mi, r.h_w, r.nmi, r.s_psi, r.s_log};
    ++g_windows;
    return ISYCOS_OK;
}
}  // namespace

namespace isy {
isycos_status fail(isycos_ctx *, isycos_status st, const char *fmt, ...) {
    fprintf(stderr, "fail: %s\n", fmt);
    return st;
}
isycos_status cuda_fail(isycos_ctx *, cudaError_t, const char *) { return ISYCOS_E_CUDA; }
// The device-resident search and the buffer / statistics helpers it calls are not used by
// this harness (it drives the machines directly); they only have to link.
isycos_status dev_reserve(isycos_ctx *, DevBuf &, size_t) { return ISYCOS_E_NOMEM; }
cudaError_t bu_device_prepare(int, int *) { return cudaErrorNotSupported; }
cudaError_t bu_device_launch(const BuLaunch &, int, int, cudaStream_t) { return cudaErrorNotSupported; }
void add_stats(isycos_ctx *, int64_t, int64_t, int64_t, int64_t, int64_t) {}
isycos_status get_lane(isycos_ctx *, int, Lane **) { return ISYCOS_E_INVAL; }
isycos_status engine_launch(isycos_ctx *, Lane &L, const HostWindow *w, int64_t n, int k, int est,
                            int32_t *, int32_t *, int32_t *, cudaStream_t) {
    g_open.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        isycos_status rc = score(w[i].xs, w[i].ys, w[i].start, w[i].m, k, est, &g_open[(size_t)i]);
        if (rc) return rc;
    }
    ++g_rounds;
    L.open.open = true;
    L.open.n = n;
    return ISYCOS_OK;
}
isycos_status engine_collect(isycos_ctx *, Lane &L, isycos_mi_out *out) {
    if (!L.open.open) return ISYCOS_OK;
    L.open.open = false;
    memcpy(out, g_open.data(), sizeof(isycos_mi_out) * (size_t)L.open.n);
    return ISYCOS_OK;
}
isycos_status engine_eval(isycos_ctx *ctx, Lane &L, const HostWindow *w, int64_t n, int k,
                          isycos_mi_out *out, int32_t *nx, int32_t *ny, int32_t *c, cudaStream_t st,
                          int est) {
    isycos_status rc = engine_launch(ctx, L, w, n, k, est, nx, ny, c, st);
    if (rc) return rc;
    return engine_collect(ctx, L, out);
}
// Chains are scored window by window (the incremental kernel gives the same results).
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

int main(int argc, char **argv) {
    if (argc < 2) {
        fprintf(stderr, "usage: host_search <series file> key=value ...\n");
        return 2;
    }
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

    isycos_params in;
    memset(&in, 0, sizeof(in));
    in.k = 4;
    in.sigma = 0.2;
    in.tau = -1.0;
    in.s_min = 32;
    in.s_max = 256;
    in.t_max_idle = -1;
    in.sel_alpha = -1.0;
    int64_t t_begin = 0, t_end = n;
    auto ctx = std::make_unique<isycos_ctx>();
    for (int a = 2; a < argc; ++a) {
        const char *eq = strchr(argv[a], '=');
        if (!eq) return 2;
        const std::string key(argv[a], (size_t)(eq - argv[a]));
        const char *v = eq + 1;
        if (key == "k") in.k = atoi(v);
        else if (key == "score_kind") in.score_kind = atoi(v);
        else if (key == "sigma") in.sigma = atof(v);
        else if (key == "tau") in.tau = atof(v);
        else if (key == "s_min") in.s_min = atoi(v);
        else if (key == "s_max") in.s_max = atoi(v);
        else if (key == "delta_td") in.delta_td = atoi(v);
        else if (key == "delta_bu") in.delta_bu = atoi(v);
        else if (key == "h") in.h = atoi(v);
        else if (key == "t_max_idle") in.t_max_idle = atoi(v);
        else if (key == "p") in.p = atoi(v);
        else if (key == "mode") in.mode = atoi(v);
        else if (key == "pruning") in.pruning = atoi(v);
        else if (key == "max_steps") in.max_steps = atoi(v);
        else if (key == "seed") in.seed = strtoull(v, nullptr, 10);
        else if (key == "sel_partitions") in.sel_partitions = atoi(v);
        else if (key == "sel_samples") in.sel_samples = atoi(v);
        else if (key == "sel_alpha") in.sel_alpha = atof(v);
        else if (key == "sel_rho") in.sel_rho = atof(v);
        else if (key == "chunks") in.chunks = atoi(v);
        else if (key == "estimator") in.estimator = atoi(v);
        else if (key == "t_begin") t_begin = atoll(v);
        else if (key == "t_end") t_end = atoll(v);
        else if (key == "spec") ctx->opt_spec_climbs = atoi(v);
        else if (key == "incremental") ctx->opt_incremental = atoi(v);
        else if (key == "table_default") g_table_default = atof(v);
        else if (key == "table") {
            FILE *tf = fopen(v, "r");
            if (!tf) return 2;
            long long a, b;
            double sc;
            while (fscanf(tf, "%lld %lld %lf", &a, &b, &sc) == 3) g_table[{a, b}] = sc;
            fclose(tf);
            g_use_table = true;
        }
        else {
            fprintf(stderr, "unknown key %s\n", key.c_str());
            return 2;
        }
    }
    SearchParams prm;
    if (resolve_params(ctx.get(), &in, &prm) != ISYCOS_OK) return 3;
    std::vector<std::unique_ptr<SearchMachine>> own;
    std::vector<SearchMachine *> ms;
    for (int32_t p = 0; p < n_pairs; ++p) {
        own.push_back(make_machine(2 * p, 2 * p + 1, t_begin, t_end, prm));
        ms.push_back(own.back().get());
    }
    Lane lane;
    if (run_machines(ctx.get(), lane, ms, nullptr) != ISYCOS_OK) return 4;
    for (int32_t p = 0; p < n_pairs; ++p) {
        const SearchMachine &m = *ms[(size_t)p];
        printf("M %d %zu %lld\n", p, m.found.size(), (long long)m.evals);
        for (const isycos_result_window &w : m.found)
            printf("W %lld %lld %.17g %.17g\n", (long long)w.t_s, (long long)w.t_e, w.score, w.mi);
    }
    printf("R %lld %lld\n", (long long)g_rounds, (long long)g_windows);
    return 0;
}
