// SYCOS_TD (arXiv 2204.09131 Sec. 5.1, Algorithm 1) and SYCOS_BU (Sec. 5.2, Algorithm 2)
// with the MI-based noise pruning of Sec. 6 (Def. 6.2; Secs. 6.2 and 6.3), as resumable
// machines whose window scores are evaluated in batches on the GPU.
//
// TD: the decisions of one layer scan are sequential (a correlated window moves the next
// start to t_e + 1), but every window a scan can visit lies on the sliding grid
// t_0 + i * delta when delta divides s_w.  The machine therefore asks for the whole grid
// of every partition of a layer at once and replays the sequential scan on the cached
// scores; an off-grid window (delta not dividing s_w) is asked for in a later round, with
// the grid that continues from it.
// BU: each LAHC step asks for its whole neighbourhood ring (and the noise-test extension
// windows) at once; many pairs' climbs share a batch.
// The decisions are those of the sequential algorithms: the scores are a pure function of
// the window, so batching changes which windows are computed, not which are chosen.
#include <string.h>

#include <algorithm>

#include "search.h"

namespace isy {

isycos_status resolve_params(isycos_ctx *ctx, const isycos_params *in, SearchParams *o) {
    if (!in) return fail(ctx, ISYCOS_E_INVAL, "params is NULL");
    o->k = in->k > 0 ? in->k : 4;
    if (o->k > kMaxK) return fail(ctx, ISYCOS_E_INVAL, "k = %d > %d", o->k, kMaxK);
    o->score_kind = in->score_kind;
    if (o->score_kind != 0 && o->score_kind != 1)
        return fail(ctx, ISYCOS_E_INVAL, "score_kind must be 0 or 1");
    o->sigma = in->sigma;
    o->tau = in->tau < 0.0 ? in->sigma / 4.0 : in->tau;
    o->s_min = in->s_min;
    o->s_max = in->s_max;
    if (o->s_min < o->k + 1) return fail(ctx, ISYCOS_E_INVAL, "s_min = %d < k + 1", o->s_min);
    if (o->s_max < o->s_min || o->s_max > kMaxM)
        return fail(ctx, ISYCOS_E_INVAL, "s_max = %d outside [s_min, %d]", o->s_max, kMaxM);
    o->delta_td = in->delta_td;
    o->delta_bu = in->delta_bu > 0 ? in->delta_bu : std::max(1, o->s_min / 4);
    o->h = in->h > 0 ? in->h : 8;
    o->t_max_idle = in->t_max_idle >= 0 ? in->t_max_idle : 3;
    o->p = in->p > 0 ? in->p : 3;
    o->mode = in->mode;
    if (o->mode != 0 && o->mode != 1) return fail(ctx, ISYCOS_E_INVAL, "mode must be 0 (TD) or 1 (BU)");
    o->pruning = in->pruning ? 1 : 0;
    o->max_steps = in->max_steps > 0 ? in->max_steps : 10000;
    o->seed = in->seed;
    return ISYCOS_OK;
}

namespace {

// ---------------------------------------------------------------------------------------
// SYCOS_TD
// ---------------------------------------------------------------------------------------
class TdMachine : public SearchMachine {
public:
    TdMachine() = default;

    bool want(std::vector<WinReq> &req) override {
        asked_.clear();
        for (;;) {
            if (finished_) return false;
            if (!layer_started_) start_layer();
            bool all_done = true;
            for (Scan &sc : scans_) {
                if (sc.done) continue;
                replay(sc);
                if (!sc.done) all_done = false;
            }
            if (!asked_.empty()) {
                req.insert(req.end(), asked_.begin(), asked_.end());
                return true;
            }
            if (!all_done) continue;   // cannot happen: an unfinished scan always asks
            // Layer finished: reduce(s_w).
            if (s_w_ <= prm.s_min) {
                finish();
                return false;
            }
            s_w_ = std::max<int64_t>(prm.s_min, s_w_ / 2);
            layer_started_ = false;
            cache_.clear();
        }
    }

    void give(const isycos_mi_out *res, size_t n) override { absorb(res, n); }

    void init() { s_w_ = prm.s_max; }

private:
    struct Scan {
        int64_t a, b;        // partition [a, b]
        int64_t t;           // next window start
        bool shifted;        // the window at t is the previous one moved by delta
        int run;             // consecutive noise detections
        bool done;
    };

    int64_t delta() const {
        if (prm.delta_td > 0) return prm.delta_td;
        return std::max<int64_t>(prm.k + 1, s_w_ / 4);
    }

    void start_layer() {
        std::sort(found.begin(), found.end(),
                  [](const isycos_result_window &u, const isycos_result_window &v) { return u.t_s < v.t_s; });
        scans_.clear();
        int64_t cur = t_begin;
        auto add = [&](int64_t a, int64_t b) {
            if (b - a + 1 >= s_w_) scans_.push_back(Scan{a, b, a, false, 0, false});
        };
        for (const auto &w : found) {
            if (w.t_s > cur) add(cur, w.t_s - 1);
            cur = w.t_e + 1;
        }
        if (cur <= t_end - 1) add(cur, t_end - 1);
        layer_started_ = true;
    }

    // Ask for the grid windows of a scan from position t to the partition's end.
    void ask_grid(const Scan &sc) {
        const int64_t d = delta();
        bool shifted = sc.shifted;
        for (int64_t t = sc.t; t + s_w_ - 1 <= sc.b; t += d) {
            Val v;
            if (!lookup(t, (int32_t)s_w_, &v)) asked_.push_back(WinReq{t, (int32_t)s_w_});
            if (prm.pruning && shifted) ask_subs(t);
            shifted = true;
        }
    }

    void ask_subs(int64_t t) {
        const int64_t d = delta();
        const int64_t mo = s_w_ - d;
        if (mo < prm.k + 1 || d < prm.k + 1) return;
        Val v;
        if (!lookup(t, (int32_t)mo, &v)) asked_.push_back(WinReq{t, (int32_t)mo});
        if (!lookup(t + mo, (int32_t)d, &v)) asked_.push_back(WinReq{t + mo, (int32_t)d});
    }

    // Run the sequential scan on cached scores until a score is missing or the scan ends.
    void replay(Scan &sc) {
        const int64_t d = delta();
        while (!sc.done) {
            if (sc.t + s_w_ - 1 > sc.b) {
                sc.done = true;
                return;
            }
            Val w;
            if (!lookup(sc.t, (int32_t)s_w_, &w)) {
                ask_grid(sc);
                return;
            }
            if (w.score >= prm.sigma) {
                found.push_back(isycos_result_window{sc.t, sc.t + s_w_ - 1, w.score, w.mi});
                ++evals;
                sc.t += s_w_;
                sc.shifted = false;
                sc.run = 0;
                continue;
            }
            bool noise = false;
            if (prm.pruning && sc.shifted) {
                const int64_t mo = s_w_ - d;
                if (mo >= prm.k + 1 && d >= prm.k + 1) {
                    Val o, e;
                    if (!lookup(sc.t, (int32_t)mo, &o) || !lookup(sc.t + mo, (int32_t)d, &e)) {
                        ask_grid(sc);
                        return;
                    }
                    // Def. 6.2 with w = w_o, w' = w_delta, w'' = the shifted window.
                    noise = (o.score > 0.0) && (e.score < prm.tau) && (w.score < o.score);
                    evals += 2;
                }
            }
            ++evals;
            sc.run = noise ? sc.run + 1 : 0;
            if (sc.run >= prm.p) {
                sc.t += s_w_;          // Sec. 6.2: skip to just after the current window
                sc.run = 0;
                sc.shifted = false;
            } else {
                sc.t += d;
                sc.shifted = true;
            }
        }
    }

    void finish() {
        std::sort(found.begin(), found.end(),
                  [](const isycos_result_window &u, const isycos_result_window &v) { return u.t_s < v.t_s; });
        finished_ = true;
    }

    int64_t s_w_ = 0;
    bool layer_started_ = false;
    bool finished_ = false;
    std::vector<Scan> scans_;
};

// ---------------------------------------------------------------------------------------
// SYCOS_BU
// ---------------------------------------------------------------------------------------
inline uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
    uint64_t z = seed + n * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

class BuMachine : public SearchMachine {
public:
    bool want(std::vector<WinReq> &req) override {
        asked_.clear();
        for (;;) {
            if (finished_) return false;
            if (phase_ == kStart) {
                if (c_ + prm.s_min > t_end) {
                    finish();
                    return false;
                }
                ws_ = c_;
                we_ = c_ + prm.s_min - 1;
                Val v;
                if (!lookup(ws_, (int32_t)(we_ - ws_ + 1), &v)) {
                    asked_.push_back(WinReq{ws_, (int32_t)(we_ - ws_ + 1)});
                    phase_ = kWaitStart;
                    break;
                }
                begin_climb(v);
                continue;
            }
            if (phase_ == kWaitStart) {
                Val v;
                lookup(ws_, (int32_t)(we_ - ws_ + 1), &v);
                begin_climb(v);
                continue;
            }
            if (phase_ == kRing) {
                build_ring();
                for (const Cand &cd : ring_) {
                    Val v;
                    if (!lookup(cd.ts, (int32_t)(cd.te - cd.ts + 1), &v))
                        asked_.push_back(WinReq{cd.ts, (int32_t)(cd.te - cd.ts + 1)});
                }
                for (int s = 0; s < 2; ++s) {
                    if (!ext_[s].use) continue;
                    Val v;
                    if (!lookup(ext_[s].ts, (int32_t)(ext_[s].te - ext_[s].ts + 1), &v))
                        asked_.push_back(WinReq{ext_[s].ts, (int32_t)(ext_[s].te - ext_[s].ts + 1)});
                }
                phase_ = kDecide;
                if (!asked_.empty()) break;
                continue;
            }
            if (phase_ == kDecide) {
                decide();
                continue;
            }
        }
        // de-duplicate requests of this round
        req.insert(req.end(), asked_.begin(), asked_.end());
        return true;
    }

    void give(const isycos_mi_out *res, size_t n) override { absorb(res, n); }

    void init() {
        c_ = t_begin;
        last_end_ = t_begin - 1;
        L_.assign(prm.h, 0.0);
    }

private:
    enum Phase { kStart, kWaitStart, kRing, kDecide };
    struct Cand {
        int64_t ts, te;
        int a, b;
    };
    struct Ext {
        bool use;
        int64_t ts, te;
        bool pure_found;   // the pure extension neighbour is part of the ring
    };

    void begin_climb(const Val &v) {
        Iw_ = v.score;
        mw_ = v.mi;
        ++evals;
        for (double &x : L_) x = Iw_;
        t_idle_ = 0;
        step_ = 0;
        run_[0] = run_[1] = 0;
        dropped_[0] = dropped_[1] = false;
        if (t_idle_ <= prm.t_max_idle && step_ < (uint64_t)prm.max_steps)
            phase_ = kRing;
        else
            end_climb();
    }

    void build_ring() {
        ring_.clear();
        const int64_t r = t_idle_ + 1, d = prm.delta_bu;
        ext_[0] = Ext{false, 0, 0, false};
        ext_[1] = Ext{false, 0, 0, false};
        for (int64_t a = -r; a <= r; ++a)
            for (int64_t b = -r; b <= r; ++b) {
                if (std::max(a < 0 ? -a : a, b < 0 ? -b : b) != r) continue;
                if (dropped_[0] && a < 0) continue;
                if (dropped_[1] && b > 0) continue;
                const int64_t ts = ws_ + a * d, te = we_ + b * d, mm = te - ts + 1;
                if (mm < prm.s_min || mm > prm.s_max) continue;
                if (ts < t_begin || te > t_end - 1 || ts <= last_end_) continue;
                ring_.push_back(Cand{ts, te, (int)a, (int)b});
                if (prm.pruning && a == -r && b == 0) ext_[0].pure_found = true;
                if (prm.pruning && a == 0 && b == r) ext_[1].pure_found = true;
            }
        if (prm.pruning) {
            if (ext_[0].pure_found && r * d >= prm.k + 1) {
                ext_[0].use = true;
                ext_[0].ts = ws_ - r * d;
                ext_[0].te = ws_ - 1;
            }
            if (ext_[1].pure_found && r * d >= prm.k + 1) {
                ext_[1].use = true;
                ext_[1].ts = we_ + 1;
                ext_[1].te = we_ + r * d;
            }
        }
    }

    void decide() {
        const int64_t r = t_idle_ + 1;
        bool have = false;
        Cand best{};
        Val bv{0.0, 0.0};
        double pure_sc[2] = {0.0, 0.0};
        for (const Cand &cd : ring_) {
            Val v;
            lookup(cd.ts, (int32_t)(cd.te - cd.ts + 1), &v);
            ++evals;
            if (!have || v.score > bv.score) {
                have = true;
                best = cd;
                bv = v;
            }
            if (cd.a == -r && cd.b == 0) pure_sc[0] = v.score;
            if (cd.a == 0 && cd.b == r) pure_sc[1] = v.score;
        }
        if (prm.pruning) {
            for (int s = 0; s < 2; ++s) {
                if (!ext_[s].pure_found) continue;
                bool noise = false;
                if (ext_[s].use) {
                    Val e;
                    lookup(ext_[s].ts, (int32_t)(ext_[s].te - ext_[s].ts + 1), &e);
                    ++evals;
                    // Def. 6.2 with w = current window, w' = extension, w'' = the neighbour.
                    noise = (Iw_ > 0.0) && (e.score < prm.tau) && (pure_sc[s] < Iw_);
                }
                run_[s] = noise ? run_[s] + 1 : 0;
                if (run_[s] >= prm.p) dropped_[s] = true;
            }
        }
        const int v = (int)(splitmix64_at(prm.seed, (climb_ << 32) + step_ + 1) % (uint64_t)prm.h);
        if (have && (bv.score > L_[v] || bv.score > Iw_)) {
            ws_ = best.ts;
            we_ = best.te;
            Iw_ = bv.score;
            mw_ = bv.mi;
            t_idle_ = 0;
        } else {
            t_idle_ += 1;
        }
        if (Iw_ > L_[v]) L_[v] = Iw_;
        ++step_;
        if (t_idle_ <= prm.t_max_idle && step_ < (uint64_t)prm.max_steps)
            phase_ = kRing;
        else
            end_climb();
    }

    void end_climb() {
        if (Iw_ >= prm.sigma) {
            found.push_back(isycos_result_window{ws_, we_, Iw_, mw_});
            last_end_ = we_;
        }
        c_ = std::max(we_ + 1, c_ + prm.s_min);
        ++climb_;
        phase_ = kStart;
        if (cache_.size() > (1u << 16)) cache_.clear();
    }

    void finish() {
        std::sort(found.begin(), found.end(),
                  [](const isycos_result_window &u, const isycos_result_window &v) { return u.t_s < v.t_s; });
        finished_ = true;
    }

    Phase phase_ = kStart;
    bool finished_ = false;
    int64_t c_ = 0, last_end_ = -1, ws_ = 0, we_ = 0;
    double Iw_ = 0.0, mw_ = 0.0;
    std::vector<double> L_;
    int t_idle_ = 0;
    uint64_t step_ = 0, climb_ = 0;
    int run_[2] = {0, 0};
    bool dropped_[2] = {false, false};
    std::vector<Cand> ring_;
    Ext ext_[2];
};

}  // namespace

std::unique_ptr<SearchMachine> make_machine(int32_t xs, int32_t ys, int64_t t_begin, int64_t t_end,
                                            const SearchParams &p) {
    if (p.mode == 0) {
        auto m = std::make_unique<TdMachine>();
        m->xs = xs;
        m->ys = ys;
        m->t_begin = t_begin;
        m->t_end = t_end;
        m->prm = p;
        m->init();
        return m;
    }
    auto m = std::make_unique<BuMachine>();
    m->xs = xs;
    m->ys = ys;
    m->t_begin = t_begin;
    m->t_end = t_end;
    m->prm = p;
    m->init();
    return m;
}

isycos_status step_machines(isycos_ctx *ctx, std::vector<SearchMachine *> &ms,
                            std::vector<bool> &finished, cudaStream_t st, int64_t *n_eval) {
    std::vector<HostWindow> batch;
    std::vector<size_t> first(ms.size(), 0), count(ms.size(), 0);
    std::vector<WinReq> req;
    int k = 0;
    for (size_t q = 0; q < ms.size(); ++q) {
        if (finished[q]) continue;
        req.clear();
        if (!ms[q]->want(req)) {
            finished[q] = true;
            continue;
        }
        k = ms[q]->prm.k;
        first[q] = batch.size();
        count[q] = req.size();
        for (const WinReq &r : req) batch.push_back(HostWindow{ms[q]->xs, ms[q]->ys, r.start, r.m});
    }
    if (n_eval) *n_eval = (int64_t)batch.size();
    if (batch.empty()) return ISYCOS_OK;
    // Machines of one call share k (the batch kernel is specialised on k); group otherwise.
    std::vector<isycos_mi_out> res(batch.size());
    bool mixed = false;
    for (size_t q = 0; q < ms.size(); ++q)
        if (count[q] && ms[q]->prm.k != k) mixed = true;
    if (!mixed) {
        isycos_status rc = engine_eval(ctx, batch.data(), (int64_t)batch.size(), k, res.data(),
                                       nullptr, nullptr, nullptr, st);
        if (rc) return rc;
    } else {
        for (int kk = 1; kk <= kMaxK; ++kk) {
            std::vector<HostWindow> sub;
            std::vector<size_t> where;
            for (size_t q = 0; q < ms.size(); ++q)
                if (count[q] && ms[q]->prm.k == kk)
                    for (size_t i = 0; i < count[q]; ++i) {
                        sub.push_back(batch[first[q] + i]);
                        where.push_back(first[q] + i);
                    }
            if (sub.empty()) continue;
            std::vector<isycos_mi_out> r2(sub.size());
            isycos_status rc = engine_eval(ctx, sub.data(), (int64_t)sub.size(), kk, r2.data(),
                                           nullptr, nullptr, nullptr, st);
            if (rc) return rc;
            for (size_t i = 0; i < sub.size(); ++i) res[where[i]] = r2[i];
        }
    }
    for (size_t q = 0; q < ms.size(); ++q)
        if (count[q]) ms[q]->give(res.data() + first[q], count[q]);
    return ISYCOS_OK;
}

isycos_status run_machines(isycos_ctx *ctx, std::vector<SearchMachine *> &ms, cudaStream_t st) {
    std::vector<bool> finished(ms.size(), false);
    for (;;) {
        int64_t n = 0;
        isycos_status rc = step_machines(ctx, ms, finished, st, &n);
        if (rc) return rc;
        bool all = true;
        for (bool f : finished) all = all && f;
        if (all) return ISYCOS_OK;
    }
}

}  // namespace isy

using namespace isy;

static isycos_status check_query(isycos_ctx *ctx, int32_t xs, int32_t ys, int64_t t_begin,
                                 int64_t t_end) {
    const int32_t ns = (int32_t)ctx->series_ptr.size();
    if (xs < 0 || xs >= ns || !ctx->series_ptr[xs] || ys < 0 || ys >= ns || !ctx->series_ptr[ys])
        return fail(ctx, ISYCOS_E_NOTFOUND, "unknown series id (%d, %d)", xs, ys);
    const int64_t n = std::min(ctx->series_len[xs], ctx->series_len[ys]);
    if (t_begin < 0 || t_end < t_begin || t_end > n)
        return fail(ctx, ISYCOS_E_INVAL, "range [%lld, %lld) outside the series (length %lld)",
                    (long long)t_begin, (long long)t_end, (long long)n);
    return ISYCOS_OK;
}

extern "C" {

isycos_status isycos_search(isycos_ctx *ctx, int32_t xs, int32_t ys, int64_t t_begin,
                            int64_t t_end, const isycos_params *params,
                            isycos_result_window *out, int64_t cap, int64_t *n_out) {
    return isycos_search_many(ctx, 1, &xs, &ys, &t_begin, &t_end, params, out, cap, n_out);
}

isycos_status isycos_search_many(isycos_ctx *ctx, int64_t n_q, const int32_t *xs,
                                 const int32_t *ys, const int64_t *t_begin,
                                 const int64_t *t_end, const isycos_params *params,
                                 isycos_result_window *out, int64_t cap_per_query,
                                 int64_t *n_out) {
    if (!ctx) return ISYCOS_E_INVAL;
    if (n_q < 0 || (n_q > 0 && (!xs || !ys || !t_begin || !t_end || !n_out)) || cap_per_query < 0 ||
        (cap_per_query > 0 && n_q > 0 && !out))
        return fail(ctx, ISYCOS_E_INVAL, "search: bad arguments");
    SearchParams p;
    isycos_status rc = resolve_params(ctx, params, &p);
    if (rc) return rc;
    std::lock_guard<std::mutex> g(ctx->engine_mu);
    cudaSetDevice(ctx->device);
    std::vector<std::unique_ptr<SearchMachine>> own;
    std::vector<SearchMachine *> ms;
    for (int64_t q = 0; q < n_q; ++q) {
        if ((rc = check_query(ctx, xs[q], ys[q], t_begin[q], t_end[q]))) return rc;
        own.push_back(make_machine(xs[q], ys[q], t_begin[q], t_end[q], p));
        ms.push_back(own.back().get());
    }
    if ((rc = run_machines(ctx, ms, ctx->stream))) return rc;
    isycos_status result = ISYCOS_OK;
    for (int64_t q = 0; q < n_q; ++q) {
        const auto &f = ms[q]->found;
        n_out[q] = (int64_t)f.size();
        if ((int64_t)f.size() > cap_per_query) {
            result = fail(ctx, ISYCOS_E_TRUNC, "query %lld found %lld windows, capacity %lld",
                          (long long)q, (long long)f.size(), (long long)cap_per_query);
            continue;
        }
        if (!f.empty())
            memcpy(out + q * cap_per_query, f.data(), sizeof(isycos_result_window) * f.size());
    }
    return result;
}

}  // extern "C"
