// Search state machines: SYCOS_TD (Algorithm 1) and SYCOS_BU (Algorithm 2) with the noise
// pruning of Sec. 6, written as resumable machines that ask for window scores in batches.
#pragma once

#include <stdint.h>

#include <memory>
#include <unordered_map>
#include <vector>

#include "runtime.h"

namespace isy {

// Parameters after defaults are resolved.
struct SearchParams {
    int k;
    int score_kind;
    double sigma, tau;
    int s_min, s_max;
    int delta_td;      // <= 0: per-layer rule max(k + 1, s_w / 4)
    int delta_bu;
    int h, t_max_idle, p, mode, pruning, max_steps;
    uint64_t seed;
};

isycos_status resolve_params(isycos_ctx *ctx, const isycos_params *in, SearchParams *out);

// One window the machine wants scored: [start, start + m - 1] of its pair.
struct WinReq {
    int64_t start;
    int32_t m;
};

class SearchMachine {
public:
    virtual ~SearchMachine() = default;
    // Append the windows to evaluate next.  Returns false once the search has finished.
    virtual bool want(std::vector<WinReq> &req) = 0;
    // Results for the windows of the last want(), in the same order.
    virtual void give(const isycos_mi_out *res, size_t n) = 0;

    int32_t xs = 0, ys = 0;
    int64_t t_begin = 0, t_end = 0;
    SearchParams prm{};
    std::vector<isycos_result_window> found;
    int64_t evals = 0;       // window scores consumed by the decisions

protected:
    double score_of(const isycos_mi_out &r) const { return prm.score_kind == 1 ? r.mi : r.nmi; }
    static uint64_t key(int64_t start, int32_t m) { return ((uint64_t)start << 15) ^ (uint64_t)m; }
    struct Val {
        double score, mi;
    };
    std::unordered_map<uint64_t, Val> cache_;
    std::vector<WinReq> asked_;
    bool lookup(int64_t start, int32_t m, Val *v) const {
        auto it = cache_.find(key(start, m));
        if (it == cache_.end()) return false;
        *v = it->second;
        return true;
    }
    void absorb(const isycos_mi_out *res, size_t n) {
        for (size_t i = 0; i < n && i < asked_.size(); ++i)
            cache_[key(asked_[i].start, asked_[i].m)] = Val{score_of(res[i]), res[i].mi};
    }
};

std::unique_ptr<SearchMachine> make_machine(int32_t xs, int32_t ys, int64_t t_begin,
                                            int64_t t_end, const SearchParams &p);

// Drive machines to completion, merging their requests into common GPU batches.
// Caller holds ctx->engine_mu.
isycos_status run_machines(isycos_ctx *ctx, std::vector<SearchMachine *> &ms, cudaStream_t st);

// One round for the serving loop: collect requests, evaluate them in one batch, deliver.
// Returns the number of windows evaluated.  Caller holds ctx->engine_mu.
isycos_status step_machines(isycos_ctx *ctx, std::vector<SearchMachine *> &ms,
                            std::vector<bool> &finished, cudaStream_t st, int64_t *n_eval);

}  // namespace isy
