// Search state machines: SYCOS_TD (Algorithm 1) and SYCOS_BU (Algorithm 2) with the noise
// pruning of Sec. 6, written as resumable machines that ask for window scores in batches.
#pragma once

#include <stdint.h>

#include <memory>
#include <vector>

#include "runtime.h"

namespace isy {

constexpr int kMaxIdle = ISYCOS_MAX_IDLE;   // largest LAHC idle limit (rings up to N_{T+1})

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
    int sel_partitions, sel_samples;   // Algorithm 3
    double sel_alpha, sel_rho;
    int chunks;                        // Algorithm 4 (<= 1: unchunked)
    int estimator;                     // 0: KSG estimator 2, 1: KSG estimator 1
    int spec_climbs;                   // SYCOS_BU climbs speculated ahead (context option)
};

isycos_status resolve_params(isycos_ctx *ctx, const isycos_params *in, SearchParams *out);

// One window the machine wants scored: [start, start + m - 1] of its pair.
struct WinReq {
    int64_t start;
    int32_t m;
    int32_t chain = -1;   // >= 0: consecutive requests with this id form one chain (in order)
    bool base = false;    // the chain's first window, asked only as the chain's start state
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
    int64_t evals_by_size[kBuckets] = {};   // the same by size bucket (m <= 2^b)
    double cost = 0.0;       // their pair comparisons, sum m (m - 1): the search's "runtime"

    // Take over another machine's evaluation counts (sub-searches of selection and chunks).
    void add_evals(const SearchMachine &o) {
        evals += o.evals;
        for (int b = 0; b < kBuckets; ++b) evals_by_size[b] += o.evals_by_size[b];
    }
    void clear_evals() {
        evals = 0;
        for (int b = 0; b < kBuckets; ++b) evals_by_size[b] = 0;
    }

protected:
    void count(int64_t m) {
        ++evals;
        ++evals_by_size[size_bucket((int)m)];
        cost += (double)m * (double)(m - 1);
    }
    double score_of(const isycos_mi_out &r) const { return prm.score_kind == 1 ? r.mi : r.nmi; }
    static uint64_t key(int64_t start, int32_t m) { return ((uint64_t)start << 15) | (uint64_t)m; }
    struct Val {
        double score, mi;
    };
    // Scores of windows already evaluated: open addressing with linear probing, cleared in
    // O(1) by a generation counter (no allocation per insert).
    class FlatCache {
    public:
        bool find(uint64_t k, Val *v) const {
            if (slots_.empty()) return false;
            for (size_t i = hash(k) & mask_;; i = (i + 1) & mask_) {
                const Slot &s = slots_[i];
                if (s.gen != gen_) return false;
                if (s.key == k) {
                    *v = s.val;
                    return true;
                }
            }
        }
        void put(uint64_t k, const Val &v) {
            if ((used_ + 1) * 2 > slots_.size()) grow();
            for (size_t i = hash(k) & mask_;; i = (i + 1) & mask_) {
                Slot &s = slots_[i];
                if (s.gen != gen_) {
                    s.gen = gen_;
                    s.key = k;
                    s.val = v;
                    ++used_;
                    return;
                }
                if (s.key == k) {
                    s.val = v;
                    return;
                }
            }
        }
        void clear() {
            ++gen_;
            used_ = 0;
        }
        size_t size() const { return used_; }

    private:
        struct Slot {
            uint64_t key;
            uint32_t gen;
            Val val;
        };
        static size_t hash(uint64_t k) {
            k ^= k >> 33;
            k *= 0xff51afd7ed558ccdULL;
            k ^= k >> 33;
            return (size_t)k;
        }
        void grow() {
            std::vector<Slot> old;
            old.swap(slots_);
            const size_t cap = old.empty() ? 1024 : old.size() * 2;
            slots_.assign(cap, Slot{0, 0, Val{0.0, 0.0}});
            mask_ = cap - 1;
            const uint32_t g = gen_;
            gen_ = 1;
            used_ = 0;
            for (const Slot &s : old)
                if (s.gen == g) put(s.key, s.val);
        }
        std::vector<Slot> slots_;
        size_t mask_ = 0, used_ = 0;
        uint32_t gen_ = 1;
    };
    FlatCache cache_;
    std::vector<WinReq> asked_;
    bool lookup(int64_t start, int32_t m, Val *v) const { return cache_.find(key(start, m), v); }
    void absorb(const isycos_mi_out *res, size_t n) {
        for (size_t i = 0; i < n && i < asked_.size(); ++i)
            if (!asked_[i].base) cache_.put(key(asked_[i].start, asked_[i].m), Val{score_of(res[i]), res[i].mi});
    }
};

std::unique_ptr<SearchMachine> make_machine(int32_t xs, int32_t ys, int64_t t_begin,
                                            int64_t t_end, const SearchParams &p);

// Drive machines to completion, merging their requests into common GPU batches.
// Caller holds ctx->engine_mu.
isycos_status run_machines(isycos_ctx *ctx, Lane &L, std::vector<SearchMachine *> &ms,
                           cudaStream_t st);

// One round for the serving loop: collect requests, evaluate them in one batch, deliver.
// Returns the number of windows evaluated.  Caller holds ctx->engine_mu.
isycos_status step_machines(isycos_ctx *ctx, Lane &L, std::vector<SearchMachine *> &ms,
                            std::vector<bool> &finished, cudaStream_t st, int64_t *n_eval);

// A round split in two: round_begin collects the requests and launches their batch on lane
// L (asynchronously), round_end waits for it and delivers the results.
struct Round {
    std::vector<SearchMachine *> *ms = nullptr;
    std::vector<bool> *finished = nullptr;
    Lane *L = nullptr;
    std::vector<std::vector<WinReq>> reqs;
    std::vector<size_t> first;
    std::vector<char> active;
    size_t total = 0;
    std::vector<isycos_mi_out> res, tmp;
    std::vector<HostWindow> batch;
    std::vector<size_t> where;
    int open_k = 0;
};
isycos_status round_begin(isycos_ctx *ctx, Lane &L, std::vector<SearchMachine *> &ms,
                          std::vector<bool> &finished, cudaStream_t st, Round &rd);
isycos_status round_end(isycos_ctx *ctx, Round &rd);


}  // namespace isy
