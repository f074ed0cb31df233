// Serving loop: continuous batching of correlation-search queries.
//
// Queries (pair, time range, parameters) are submitted from any thread and receive a ticket.
// Library worker threads (one engine lane each: a CUDA stream with its own buffers) admit
// queued queries while the number of running queries stays below the slot limit and their
// estimated device work memory fits in what the context's budget leaves after the resident
// series; an admitted query joins the least loaded worker.  Every round a worker collects the
// pending window requests of its running queries (TD layer grids, BU rings), evaluates them in
// one persistent GPU batch, hands each query its results and retires the queries that
// finished; queries that arrive meanwhile join at the next round.  Workers run concurrently,
// so their batches overlap on the GPU.  The decisions of a query do not depend on which other
// queries share its batches, so a query's result is the same alone and in the mix.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <string.h>
#include <thread>
#include <unordered_map>

#include "search.h"

namespace isy {

using Clock = std::chrono::steady_clock;

class Server {
public:
    // Worker threads, each with its own engine lane (stream and buffers), each stepping its
    // own share of the running queries; the lanes are separate from those of the searches.
    explicit Server(isycos_ctx *ctx) : ctx_(ctx) {
        int n = std::max(1, std::min(ctx->max_lanes, 8));
        {
            std::lock_guard<std::mutex> g(ctx->engine_mu);
            cudaSetDevice(ctx->device);
            for (int w = 0; w < n; ++w) {
                Lane *L = nullptr;
                if (get_lane(ctx, kServeLaneBase + w, &L) != ISYCOS_OK) break;
                lanes_.push_back(L);
            }
        }
        running_.resize(lanes_.size());
        for (size_t w = 0; w < lanes_.size(); ++w) th_.emplace_back([this, w] { loop((int)w); });
    }

    ~Server() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : th_) t.join();
    }


    isycos_status submit(int32_t xs, int32_t ys, int64_t tb, int64_t te, const SearchParams &p,
                         uint64_t *ticket) {
        auto q = std::make_unique<Query>();
        q->xs = xs;
        q->ys = ys;
        q->tb = tb;
        q->te = te;
        q->prm = p;
        q->t_submit = Clock::now();
        q->bytes = estimate_bytes(te - tb, p);
        std::lock_guard<std::mutex> g(mu_);
        if ((int64_t)queue_.size() >= ctx_->serve_queue)
            return fail(ctx_, ISYCOS_E_AGAIN, "serve: admission queue full");
        const uint64_t t = next_++;
        q->ticket = t;
        queue_.push_back(t);
        all_[t] = std::move(q);
        *ticket = t;
        cv_.notify_all();
        return ISYCOS_OK;
    }

    isycos_status poll(uint64_t ticket, isycos_result_window *out, int64_t cap, int64_t *n_out,
                       double *latency_ms, double *wait_ms = nullptr) {
        std::lock_guard<std::mutex> g(mu_);
        auto it = all_.find(ticket);
        if (it == all_.end()) return fail(ctx_, ISYCOS_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
        Query &q = *it->second;
        if (q.state == kQueued || q.state == kRunning) return ISYCOS_PENDING;
        if (q.state == kCanceled) {
            all_.erase(it);
            return fail(ctx_, ISYCOS_E_CANCELED, "query %llu was cancelled", (unsigned long long)ticket);
        }
        if (q.state == kFailed) {
            const isycos_status st = q.status;
            all_.erase(it);
            return fail(ctx_, st, "query %llu failed", (unsigned long long)ticket);
        }
        if (n_out) *n_out = (int64_t)q.result.size();
        if (latency_ms) *latency_ms = q.latency_ms;
        if (wait_ms) *wait_ms = q.wait_ms;
        if ((int64_t)q.result.size() > cap || (!out && !q.result.empty()))
            return fail(ctx_, ISYCOS_E_TRUNC, "query %llu found %lld windows, capacity %lld",
                        (unsigned long long)ticket, (long long)q.result.size(), (long long)cap);
        if (!q.result.empty()) memcpy(out, q.result.data(), sizeof(isycos_result_window) * q.result.size());
        all_.erase(it);
        return ISYCOS_OK;
    }

    isycos_status cancel(uint64_t ticket) {
        std::lock_guard<std::mutex> g(mu_);
        auto it = all_.find(ticket);
        if (it == all_.end()) return fail(ctx_, ISYCOS_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
        Query &q = *it->second;
        if (q.state == kQueued) {
            for (auto qi = queue_.begin(); qi != queue_.end(); ++qi)
                if (*qi == ticket) {
                    queue_.erase(qi);
                    break;
                }
            q.state = kCanceled;
        } else if (q.state == kRunning) {
            q.cancel = true;
        }
        return ISYCOS_OK;
    }

private:
    enum State { kQueued, kRunning, kDone, kCanceled, kFailed };
    struct Query {
        uint64_t ticket = 0;
        int32_t xs = 0, ys = 0;
        int64_t tb = 0, te = 0;
        SearchParams prm{};
        std::unique_ptr<SearchMachine> sm;
        Clock::time_point t_submit;
        double wait_ms = 0.0;   // from submission to admission
        State state = kQueued;
        bool cancel = false;
        std::vector<isycos_result_window> result;
        double latency_ms = 0.0;
        isycos_status status = ISYCOS_OK;
        size_t bytes = 0;
        int worker = 0;
    };

    // Device bytes the engine may need for this query's largest batch: a full TD layer grid
    // (with the two pruning sub-windows per position) or a BU ring, per window one work item
    // and one result.
    static size_t estimate_bytes(int64_t len, const SearchParams &p) {
        int64_t windows;
        if (p.mode == 0) {
            int64_t d = p.delta_td > 0 ? p.delta_td : std::max<int64_t>(p.k + 1, p.s_min / 4);
            windows = len / std::max<int64_t>(d, 1) + 1;
            if (p.pruning) windows *= 3;
        } else {
            windows = 8 * (int64_t)(p.t_max_idle + 1) + 2;
        }
        // twice: the engine's buffers grow by half their size at a time
        return 2 * (size_t)windows * (sizeof(WorkItem) + sizeof(isycos_mi_out));
    }

    size_t capacity() const {
        // (an atomic total: the series tables may grow under another thread meanwhile)
        const size_t fixed = (size_t)ctx_->series_bytes.load() + 2 * sizeof(long long) * kTableN;
        return ctx_->budget > fixed ? ctx_->budget - fixed : 0;
    }

    size_t n_running() const {
        size_t n = 0;
        for (const auto &r : running_) n += r.size();
        return n;
    }

    void admit() {  // holds mu_
        const size_t cap = capacity();
        bool any = false;
        while (!queue_.empty() && (int)n_running() < ctx_->serve_slots) {
            Query &q = *all_[queue_.front()];
            if (reserved_ + q.bytes > cap && n_running() > 0) break;   // wait for memory
            if (q.bytes > cap) {
                q.state = kFailed;
                q.status = ISYCOS_E_NOMEM;
                queue_.pop_front();
                continue;
            }
            queue_.pop_front();
            q.sm = make_machine(q.xs, q.ys, q.tb, q.te, q.prm);
            q.state = kRunning;
            q.wait_ms = std::chrono::duration<double, std::milli>(Clock::now() - q.t_submit).count();
            reserved_ += q.bytes;
            size_t w = 0;
            for (size_t i = 1; i < running_.size(); ++i)
                if (running_[i].size() < running_[w].size()) w = i;
            q.worker = (int)w;
            running_[w].push_back(&q);
            any = true;
        }
        if (any) cv_.notify_all();
    }

    void retire(Query *q, State st, isycos_status status) {  // holds mu_
        q->state = st;
        q->status = status;
        q->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - q->t_submit).count();
        if (st == kDone) {
            q->result = q->sm->found;
            std::lock_guard<std::mutex> g(ctx_->stats_mu);
            ctx_->stats.decided_windows += q->sm->evals;
            for (int b = 0; b < kBuckets; ++b) ctx_->stats.decided_by_size[b] += q->sm->evals_by_size[b];
        }
        q->sm.reset();
        reserved_ -= q->bytes;
    }

    void loop(int w) {
        Lane &L = *lanes_[w];
        cudaSetDevice(ctx_->device);
        std::vector<Query *> batch;
        std::vector<SearchMachine *> ms;
        std::vector<bool> finished;
        auto &mine = running_[w];
        for (;;) {
            {
                std::unique_lock<std::mutex> g(mu_);
                for (size_t i = 0; i < mine.size();) {
                    if (mine[i]->cancel) {
                        retire(mine[i], kCanceled, ISYCOS_E_CANCELED);
                        mine.erase(mine.begin() + i);
                    } else {
                        ++i;
                    }
                }
                admit();
                if (mine.empty()) {
                    if (stop_) return;
                    if (L.d_items.p) lane_release(ctx_, L);   // idle: give the memory back
                    cv_.wait_for(g, std::chrono::milliseconds(20));
                    continue;
                }
                if (stop_) {
                    for (Query *q : mine) retire(q, kCanceled, ISYCOS_E_CANCELED);
                    mine.clear();
                    return;
                }
                batch = mine;
            }
            ms.clear();
            for (Query *q : batch) ms.push_back(q->sm.get());
            finished.assign(ms.size(), false);
            int64_t n = 0;
            const isycos_status rc = step_machines(ctx_, L, ms, finished, L.stream, &n);
            std::lock_guard<std::mutex> g(mu_);
            for (size_t i = 0; i < batch.size(); ++i) {
                if (rc != ISYCOS_OK) {
                    retire(batch[i], kFailed, rc);
                } else if (finished[i]) {
                    retire(batch[i], kDone, ISYCOS_OK);
                    std::lock_guard<std::mutex> sg(ctx_->stats_mu);
                    ctx_->stats.queries_done++;
                } else {
                    continue;
                }
                for (size_t r = 0; r < mine.size(); ++r)
                    if (mine[r] == batch[i]) {
                        mine.erase(mine.begin() + r);
                        break;
                    }
            }
        }
    }

    isycos_ctx *ctx_;
    std::mutex mu_;
    std::condition_variable cv_;
    bool stop_ = false;
    uint64_t next_ = 1;
    std::deque<uint64_t> queue_;
    std::unordered_map<uint64_t, std::unique_ptr<Query>> all_;
    std::vector<std::vector<Query *>> running_;   // per worker
    std::vector<Lane *> lanes_;
    size_t reserved_ = 0;
    std::vector<std::thread> th_;
};

static std::mutex g_server_create_mu;

static Server *get_server(isycos_ctx *ctx) {
    std::lock_guard<std::mutex> g(g_server_create_mu);
    if (!ctx->server) ctx->server = new Server(ctx);
    return ctx->server;
}

void serve_shutdown(isycos_ctx *ctx) {
    std::lock_guard<std::mutex> g(g_server_create_mu);
    delete ctx->server;
    ctx->server = nullptr;
}

}  // namespace isy

using namespace isy;

extern "C" {

isycos_status isycos_serve_submit(isycos_ctx *ctx, int32_t xs, int32_t ys, int64_t t_begin,
                                  int64_t t_end, const isycos_params *params, uint64_t *ticket) {
    if (!ctx) return ISYCOS_E_INVAL;
    if (!ticket) return fail(ctx, ISYCOS_E_INVAL, "ticket is NULL");
    SearchParams p;
    isycos_status rc = resolve_params(ctx, params, &p);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> g(ctx->engine_mu);
        const int32_t ns = (int32_t)ctx->series_ptr.size();
        if (xs < 0 || xs >= ns || !ctx->series_ptr[xs] || ys < 0 || ys >= ns || !ctx->series_ptr[ys])
            return fail(ctx, ISYCOS_E_NOTFOUND, "unknown series id (%d, %d)", xs, ys);
        const int64_t n = std::min(ctx->series_len[xs], ctx->series_len[ys]);
        if (t_begin < 0 || t_end < t_begin || t_end > n)
            return fail(ctx, ISYCOS_E_INVAL, "range outside the series");
    }
    return get_server(ctx)->submit(xs, ys, t_begin, t_end, p, ticket);
}

isycos_status isycos_serve_poll(isycos_ctx *ctx, uint64_t ticket, isycos_result_window *out,
                                int64_t cap, int64_t *n_out, double *latency_ms) {
    if (!ctx) return ISYCOS_E_INVAL;
    return get_server(ctx)->poll(ticket, out, cap, n_out, latency_ms);
}

isycos_status isycos_serve_poll_ex(isycos_ctx *ctx, uint64_t ticket, isycos_result_window *out,
                                   int64_t cap, int64_t *n_out, double *latency_ms,
                                   double *wait_ms) {
    if (!ctx) return ISYCOS_E_INVAL;
    return get_server(ctx)->poll(ticket, out, cap, n_out, latency_ms, wait_ms);
}

isycos_status isycos_serve_cancel(isycos_ctx *ctx, uint64_t ticket) {
    if (!ctx) return ISYCOS_E_INVAL;
    return get_server(ctx)->cancel(ticket);
}

}  // extern "C"
