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
#include <thread>
#include <unordered_map>

#include "search.h"
#include "bu_device.h"

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
    if (o->t_max_idle > kMaxIdle)
        return fail(ctx, ISYCOS_E_INVAL, "t_max_idle = %d > %d", o->t_max_idle, kMaxIdle);
    o->p = in->p > 0 ? in->p : 3;
    o->mode = in->mode;
    if (o->mode < 0 || o->mode > 2)
        return fail(ctx, ISYCOS_E_INVAL, "mode must be 0 (TD), 1 (BU) or 2 (selection)");
    o->pruning = in->pruning ? 1 : 0;
    o->max_steps = in->max_steps > 0 ? in->max_steps : 10000;
    o->seed = in->seed;
    o->sel_partitions = in->sel_partitions > 0 ? in->sel_partitions : 20;
    o->sel_samples = in->sel_samples > 0 ? in->sel_samples : 6;
    o->sel_alpha = in->sel_alpha >= 0.0 ? in->sel_alpha : 0.5;
    o->sel_rho = in->sel_rho > 0.0 ? in->sel_rho : 0.5;
    if (o->sel_partitions > (1 << 20)) return fail(ctx, ISYCOS_E_INVAL, "sel_partitions too large");
    o->chunks = in->chunks > 1 ? in->chunks : 1;
    if (o->chunks > (1 << 20)) return fail(ctx, ISYCOS_E_INVAL, "chunks too large");
    o->estimator = in->estimator;
    if (o->estimator != 0 && o->estimator != 1)
        return fail(ctx, ISYCOS_E_INVAL, "estimator must be 0 or 1");
    o->spec_climbs = ctx->opt_spec_climbs;
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
        dest_.clear();
        next_chain_ = 0;
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

    void give(const isycos_mi_out *res, size_t n) override {
        for (size_t i = 0; i < n && i < asked_.size(); ++i) {
            const Val v{score_of(res[i]), res[i].mi};
            const Dest &d = dest_[i];
            if (d.slot >= 0) {
                Slot &q = slots_[(size_t)d.slot];
                q.v[d.kind] = v;
                q.have |= (uint8_t)(1u << d.kind);
            } else {
                cache_.put(key(asked_[i].start, asked_[i].m), v);
            }
        }
    }

    void init() { s_w_ = prm.s_max; }

private:
    struct Scan {
        int64_t a, b;        // partition [a, b]
        int64_t t;           // next window start
        bool shifted;        // the window at t is the previous one moved by delta
        int run;             // consecutive noise detections
        bool done;
        int64_t off;         // first score slot of the partition in this layer
    };
    // Scores of one layer, one slot per grid position a + i delta of a partition: the grid
    // window (kind 0) and the noise test's sub-windows w_o = [t, t + s_w - delta - 1] (kind 1)
    // and w_delta = [t + s_w - delta, t + s_w - 1] (kind 2).  The scans ask and read them in
    // position order, so the slots are filled and read sequentially.  A window off the grid
    // (delta not dividing a jump) goes to the hashed cache.
    struct Slot {
        Val v[3];
        uint8_t have = 0;
    };
    struct Dest {
        int64_t slot;        // -1: the hashed cache
        int kind;
    };

    int64_t delta() const {
        if (prm.delta_td > 0) return prm.delta_td;
        return std::max<int64_t>(prm.k + 1, s_w_ / 4);
    }

    void start_layer() {
        std::sort(found.begin(), found.end(),
                  [](const isycos_result_window &u, const isycos_result_window &v) { return u.t_s < v.t_s; });
        scans_.clear();
        const int64_t d = delta();
        int64_t cur = t_begin, slots = 0;
        auto add = [&](int64_t a, int64_t b) {
            if (b - a + 1 >= s_w_) {
                scans_.push_back(Scan{a, b, a, false, 0, false, slots});
                slots += (b - a) / d + 1;
            }
        };
        for (const auto &w : found) {
            if (w.t_s > cur) add(cur, w.t_s - 1);
            cur = w.t_e + 1;
        }
        if (cur <= t_end - 1) add(cur, t_end - 1);
        slots_.assign((size_t)slots, Slot{});
        layer_started_ = true;
    }

    // Slot of position t of scan sc, or -1 when t is off the partition's grid.
    int64_t slot_of(const Scan &sc, int64_t t) const {
        const int64_t d = delta(), r = t - sc.a;
        return r % d == 0 ? sc.off + r / d : -1;
    }
    // Score of the window of `kind` at position t of scan sc (m points), if known.
    bool score(const Scan &sc, int64_t t, int kind, int32_t m, Val *v) const {
        const int64_t q = slot_of(sc, t);
        if (q < 0) return lookup(kind == 2 ? t + s_w_ - delta() : t, m, v);
        const Slot &z = slots_[(size_t)q];
        if (!(z.have & (1u << kind))) return false;
        *v = z.v[kind];
        return true;
    }
    void ask(const Scan &sc, int64_t t, int kind, int32_t m, int32_t chain) {
        const int64_t start = kind == 2 ? t + s_w_ - delta() : t;
        asked_.push_back(WinReq{start, m, chain, false});
        dest_.push_back(Dest{slot_of(sc, t), kind});
    }

    // Ask for the grid windows of a scan from position t to the partition's end; the grid
    // windows of one scan form a chain (each is the previous one moved by delta).
    void ask_grid(const Scan &sc) {
        const int64_t d = delta();
        bool shifted = sc.shifted;
        const int32_t chain = next_chain_++;
        for (int64_t t = sc.t; t + s_w_ - 1 <= sc.b; t += d) {
            Val v;
            if (!score(sc, t, 0, (int32_t)s_w_, &v)) ask(sc, t, 0, (int32_t)s_w_, chain);
            if (prm.pruning && shifted) ask_subs(sc, t);
            shifted = true;
        }
    }

    void ask_subs(const Scan &sc, int64_t t) {
        const int64_t d = delta();
        const int64_t mo = s_w_ - d;
        if (mo < prm.k + 1 || d < prm.k + 1) return;
        Val v;
        if (!score(sc, t, 1, (int32_t)mo, &v)) ask(sc, t, 1, (int32_t)mo, -1);
        if (!score(sc, t, 2, (int32_t)d, &v)) ask(sc, t, 2, (int32_t)d, -1);
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
            if (!score(sc, sc.t, 0, (int32_t)s_w_, &w)) {
                ask_grid(sc);
                return;
            }
            if (w.score >= prm.sigma) {
                found.push_back(isycos_result_window{sc.t, sc.t + s_w_ - 1, w.score, w.mi});
                count(s_w_);
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
                    if (!score(sc, sc.t, 1, (int32_t)mo, &o) || !score(sc, sc.t, 2, (int32_t)d, &e)) {
                        ask_grid(sc);
                        return;
                    }
                    // Def. 6.2 with w = w_o, w' = w_delta, w'' = the shifted window.
                    noise = (o.score > 0.0) && (e.score < prm.tau) && (w.score < o.score);
                    count(mo);
                    count(d);
                }
            }
            count(s_w_);
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
    int32_t next_chain_ = 0;
    bool layer_started_ = false;
    bool finished_ = false;
    std::vector<Scan> scans_;
    std::vector<Slot> slots_;
    std::vector<Dest> dest_;
};

// ---------------------------------------------------------------------------------------
// SYCOS_BU
// ---------------------------------------------------------------------------------------
// Division by a lattice step that is usually a power of two (delta = s_min / 4): a shift
// when it is one (the quotients taken here are exact multiples, or non-negative).
struct StepDiv {
    int64_t d = 1;
    int sh = 0;   // log2(d) when d is a power of two, else -1
    void set(int64_t delta) {
        d = std::max<int64_t>(1, delta);
        sh = (d & (d - 1)) == 0 ? __builtin_ctzll((unsigned long long)d) : -1;
    }
    int64_t div(int64_t x) const { return sh >= 0 ? (x >> sh) : x / d; }
    bool divides(int64_t x) const { return sh >= 0 ? (x & (d - 1)) == 0 : x % d == 0; }
};

// A set of positions near a moving cursor: direct mapped over position / step (exact
// positions kept), so that nothing needs clearing as the cursor advances; positions
// kSlots steps apart share a slot (the later one wins: a lost position is merely
// speculated again).
struct PosSet {
    static constexpr int kSlots = 1024;
    StepDiv dv;
    std::vector<int64_t> key = std::vector<int64_t>(kSlots, INT64_MIN);
    void init(int64_t step) { dv.set(step); }
    void clear() { std::fill(key.begin(), key.end(), INT64_MIN); }
    size_t slot(int64_t p) const { return (size_t)(dv.div(std::max<int64_t>(0, p)) & (kSlots - 1)); }
    bool has(int64_t p) const { return key[slot(p)] == p; }
    void add(int64_t p) { key[slot(p)] = p; }
};

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
        dest_.clear();
        next_chain_ = 0;
        ++round_;
        for (;;) {
            if (finished_) return false;
            if (phase_ == kStart) {
                if (c_ + prm.s_min > t_end) {
                    finish();
                    return false;
                }
                ws_ = c_;
                we_ = c_ + prm.s_min - 1;
                // scores are pure functions of the window: keep the cells of earlier climbs
                // when this start lies on their lattice
                if (!grid_.on_lattice(ws_, we_, prm.delta_bu)) {
                    grid_.reset(ws_, we_, prm.delta_bu);
                    spec_starts_.clear();
                }
                // a climb always evaluates ring N_1 of its first window next: ask it now
                int64_t ac, bc;
                grid_.centre(ws_, we_, &ac, &bc);
                if (!grid_.get(ac, bc, &start_val_)) ask_cell(ac, bc, ws_, we_, kDestStart, -1, -1);
                if (prm.t_max_idle >= 0 && prm.max_steps > 0)
                    for (int rr = 1; rr <= std::min(prm.t_max_idle + 1, spec_depth()); ++rr)
                        ask_ring(rr, false, false, false);
                phase_ = kWaitStart;
                if (asked_.empty()) continue;
                speculate_next_climbs();
                speculate_ext_moves();
                break;
            }
            if (phase_ == kWaitStart) {
                begin_climb(start_val_);
                continue;
            }
            if (phase_ == kRing) {
                // Some score of ring N_r is missing.  After a rejection the window stays put
                // and the rings N_r .. N_{T+1} are evaluated until one improves: ask for all
                // of them at once.
                const int r = t_idle_ + 1;
                int r_last = t_idle_ >= 1 ? prm.t_max_idle + 1 : r;
                // Small windows are cheap on the GPU and every round trip costs the same: also
                // ask the outer rings now, which cover the next step's ring N_1 when the
                // climb moves by one delta and the remaining rings when it does not.
                r_last = std::max(r_last, std::min(prm.t_max_idle + 1, spec_depth()));
                const size_t before = asked_.size();
                ask_ring(r, dropped_[0], dropped_[1], stuck_);
                // speculate only when this step needs a round trip anyway
                if (asked_.size() > before) {
                    for (int rr = r + 1; rr <= r_last; ++rr) ask_ring(rr, dropped_[0], dropped_[1], false);
                    speculate_next_climbs();
                    speculate_ext_moves();
                }
                // (a ring whose scores are all cached has nothing to ask; if its decision
                // still finds one missing, the next ask ignores the caches)
                stuck_ = asked_.size() == before;
                phase_ = kDecide;
                if (asked_.empty()) continue;
                break;
            }
            if (phase_ == kDecide) {
                if (!decide(t_idle_ + 1)) phase_ = kRing;
                else stuck_ = false;
                continue;
            }
        }
        req.insert(req.end(), asked_.begin(), asked_.end());
        return true;
    }

    void give(const isycos_mi_out *res, size_t n) override {
        for (size_t i = 0; i < n && i < dest_.size(); ++i) {
            const Dest &d = dest_[i];
            const Val v{score_of(res[i]), res[i].mi};
            if (d.kind == kDestStart || d.kind == kDestCell) {
                if (d.kind == kDestStart) start_val_ = v;
                grid_.put(d.a, d.b, v);
            } else if (d.kind == kDestExt) {
                ext_.put(d.a, d.b, v);
                // the extension windows of the rings asked for the next decisions are also
                // kept by ring and side: the slotted cache may still lose one of them to
                // another window of the same round (P deltas away, or a ring beyond the
                // eighth sharing its slot)
                if (d.r >= 0) ring_ext_[(size_t)(2 * d.r + d.side)] = RingExt{d.a, d.b, v};
            }
        }
    }

    void init() {
        c_ = t_begin;
        last_end_ = t_begin - 1;
        L_.assign(prm.h, 0.0);
        ring_ext_.assign((size_t)2 * (prm.t_max_idle + 2), RingExt{});
        ext_.init(prm.delta_bu, prm.t_max_idle + 1);
        spec_starts_.init(prm.delta_bu);
        ext_left_.init(prm.delta_bu);
        ext_right_.init(prm.delta_bu);
        // the cells one round asks span T_maxIdle + 1 cells around the window and the windows
        // of the climbs asked ahead, s_min / delta cells apart: the direct-mapped array must
        // be wider than that span so that they do not evict one another
        const int64_t step = std::max<int64_t>(1, prm.s_min / std::max(1, prm.delta_bu));
        grid_.init((int)((prm.spec_climbs + 1) * step + 2 * (prm.t_max_idle + 2) + 4));
    }

private:
    enum Phase { kStart, kWaitStart, kRing, kDecide };
    enum DestKind { kDestStart, kDestCell, kDestExt, kDestNone };
    struct Dest {
        int kind, r, side;
        int64_t a, b;   // grid cell, or (start, size) of an extension window
    };
    // Scores of windows on the delta lattice of the climbs: window [bs + a d, be + b d] at
    // cell (a, b).  The array is direct mapped (cell (a, b) in slot (a mod G, b mod G), with
    // its coordinates kept to tell it from the cells that share the slot), so it follows the
    // search along the series without copying.
    struct GridCache {
        // One record per slot, so that a lookup touches one cache line.
        struct Slot {
            int64_t ka = 0, kb = 0;   // the cell that owns the slot
            Val val{0.0, 0.0};
            uint32_t tag = 0;         // == gen: val holds the score of cell (ka, kb)
            uint32_t asked = 0;       // round in which (ka, kb) was last asked
        };
        int G = 64, lg = 6;
        int64_t bs = 0, be = 0, d = 1;
        StepDiv dv;
        uint32_t gen = 1;
        bool valid = false;
        std::vector<Slot> cell;
        void init(int min_side) {
            G = 64;
            lg = 6;
            // (at most 256 x 256 cells, 2.6 MB: beyond that, cells of one round may share a
            // slot, which costs a re-ask but never a wrong score)
            while (G < min_side && G < 256) {
                G <<= 1;
                ++lg;
            }
            cell.assign((size_t)G * G, Slot{});
        }
        bool on_lattice(int64_t ws, int64_t we, int64_t delta) const {
            return valid && delta == d && dv.divides(ws - bs) && dv.divides(we - be);
        }
        void reset(int64_t s, int64_t e, int64_t delta) {
            bs = s;
            be = e;
            d = delta;
            dv.set(delta);
            ++gen;
            valid = true;
        }
        // (ws, we) on the lattice: the quotients are exact
        void centre(int64_t ws, int64_t we, int64_t *a, int64_t *b) const {
            *a = dv.div(ws - bs);
            *b = dv.div(we - be);
        }
        size_t slot(int64_t a, int64_t b) const {
            return ((size_t)(a & (G - 1)) << lg) | (size_t)(b & (G - 1));
        }
        bool get(int64_t a, int64_t b, Val *v) const {
            const Slot &c = cell[slot(a, b)];
            if (c.tag != gen || c.ka != a || c.kb != b) return false;
            *v = c.val;
            return true;
        }
        // (a, b) has a score, or was asked in round `round`
        bool known_or_asked(int64_t a, int64_t b, uint32_t round) const {
            const Slot &c = cell[slot(a, b)];
            return c.ka == a && c.kb == b && (c.tag == gen || c.asked == round);
        }
        // the slot of (a, b) holds another cell asked in round `round`
        bool taken(int64_t a, int64_t b, uint32_t round) const {
            const Slot &c = cell[slot(a, b)];
            return c.asked == round && (c.ka != a || c.kb != b);
        }
        // mark (a, b) as asked in round `round`; false if it already was
        bool mark(int64_t a, int64_t b, uint32_t round) {
            Slot &c = cell[slot(a, b)];
            if (c.asked == round && c.ka == a && c.kb == b) return false;
            if (c.ka != a || c.kb != b) c.tag = 0;   // the slot now belongs to (a, b)
            c.asked = round;
            c.ka = a;
            c.kb = b;
            return true;
        }
        void put(int64_t a, int64_t b, const Val &v) {
            Slot &c = cell[slot(a, b)];
            c.val = v;
            c.tag = gen;
            c.ka = a;
            c.kb = b;
        }
    };
    // Scores of the noise test's extension windows.  The left one of a window starting at p
    // is [p - r delta, p - 1], the right one of a window ending at q is [q + 1, q + r delta]
    // (r = 1 .. T_maxIdle + 1); one window can be both.  Slot: start / delta mod P and r, so
    // that the windows near the search cursor never evict one another (the window itself is
    // kept to tell it from the windows P deltas away that share the slot).
    struct ExtCache {
        static constexpr int P = 2048;
        int R = 1, rmask = 0;   // rmask = R - 1 when R is a power of two, else -1
        StepDiv dv;
        struct E {
            int64_t s = -1, m = 0;
            uint32_t asked = 0;
            bool have = false;
            Val v{0.0, 0.0};
        };
        std::vector<E> e;
        void init(int64_t delta, int rmax) {
            dv.set(delta);
            R = std::max(1, std::min(rmax, 8));   // larger r share slots (r mod 8)
            rmask = (R & (R - 1)) == 0 ? R - 1 : -1;
            e.assign((size_t)P * R, E{});
        }
        size_t slot(int64_t s, int64_t m) const {
            const int64_t r1 = std::max<int64_t>(1, dv.div(m)) - 1;
            const int64_t rq = rmask >= 0 ? (r1 & rmask) : r1 % R;
            return (size_t)(dv.div(std::max<int64_t>(0, s)) & (P - 1)) * (size_t)R + (size_t)rq;
        }
        bool get(int64_t s, int64_t m, Val *v) const {
            const E &x = e[slot(s, m)];
            if (!x.have || x.s != s || x.m != m) return false;
            *v = x.v;
            return true;
        }
        bool mark(int64_t s, int64_t m, uint32_t round) {
            E &x = e[slot(s, m)];
            if (x.s == s && x.m == m && (x.have || x.asked == round)) return false;
            if (x.s != s || x.m != m) x.have = false;
            x.s = s;
            x.m = m;
            x.asked = round;
            return true;
        }
        void put(int64_t s, int64_t m, const Val &v) {
            E &x = e[slot(s, m)];
            x.s = s;
            x.m = m;
            x.have = true;
            x.v = v;
        }
    };
    // Score of the extension window (s, m) last delivered for a ring and side.
    struct RingExt {
        int64_t s = -1, m = 0;
        Val v{0.0, 0.0};
    };
    bool ext_score(int r, int side, int64_t s, int64_t m, Val *v) const {
        if (ext_.get(s, m, v)) return true;
        const RingExt &e = ring_ext_[(size_t)(2 * r + side)];
        if (e.s != s || e.m != m) return false;
        *v = e.v;
        return true;
    }

    void ask_cell(int64_t a, int64_t b, int64_t ts, int64_t te, int kind, int r, int32_t chain) {
        asked_.push_back(WinReq{ts, (int32_t)(te - ts + 1), chain, false});
        dest_.push_back(Dest{kind, r, 0, a, b});
        grid_.mark(a, b, round_);
    }
    void ask_ext(int64_t ts, int64_t te, int r, int side) {
        asked_.push_back(WinReq{ts, (int32_t)(te - ts + 1), -1, false});
        dest_.push_back(Dest{kDestExt, r, side, ts, te - ts + 1});
    }

    // A candidate of ring N_r around (ws_, we_) passes the filters of the search.
    bool keep(int64_t a, int64_t b, int64_t r, bool drop_left, bool drop_right, int64_t *ts,
              int64_t *te) const {
        if (std::max(a < 0 ? -a : a, b < 0 ? -b : b) != r) return false;
        if (drop_left && a < 0) return false;
        if (drop_right && b > 0) return false;
        const int64_t d = prm.delta_bu;
        *ts = ws_ + a * d;
        *te = we_ + b * d;
        const int64_t mm = *te - *ts + 1;
        if (mm < prm.s_min || mm > prm.s_max) return false;
        if (*ts < t_begin || *te > t_end - 1 || *ts <= last_end_) return false;
        return true;
    }

    // Ask for ring N_r around the current window: the candidates walked along the perimeter
    // from (-r, -r) so that consecutive windows differ by one delta at one end (the current
    // window starts the chain), then the noise-test extension windows.
    void ask_ring(int r, bool drop_left, bool drop_right, bool all) {
        const int32_t chain = next_chain_++;
        const size_t first = asked_.size();
        int64_t ac, bc;
        grid_.centre(ws_, we_, &ac, &bc);
        auto visit = [&](int a, int b) {
            int64_t ts, te;
            if (!keep(a, b, r, drop_left, drop_right, &ts, &te)) return;
            // evaluated earlier, or asked in this round
            if (!all && grid_.known_or_asked(ac + a, bc + b, round_)) return;
            ask_cell(ac + a, bc + b, ts, te, kDestCell, r, chain);
        };
        for (int b = -r; b <= r; ++b) visit(-r, b);
        for (int a = -r + 1; a <= r; ++a) visit(a, r);
        for (int b = r - 1; b >= -r; --b) visit(r, b);
        for (int a = r - 1; a > -r; --a) visit(a, -r);
        if (asked_.size() > first + 1) {
            asked_.insert(asked_.begin() + first, WinReq{ws_, (int32_t)(we_ - ws_ + 1), chain, true});
            dest_.insert(dest_.begin() + first, Dest{kDestNone, r, 0, 0, 0});
        } else if (asked_.size() == first + 1) {
            asked_.back().chain = -1;
        }
        if (prm.pruning && (int64_t)r * prm.delta_bu >= prm.k + 1) {
            int64_t ts, te;
            const int64_t span = (int64_t)r * prm.delta_bu;
            const int64_t es[2] = {ws_ - span, we_ + 1}, ee[2] = {ws_ - 1, we_ + span};
            for (int sd = 0; sd < 2; ++sd) {
                if (!keep(sd == 0 ? -r : 0, sd == 0 ? 0 : r, r, drop_left, drop_right, &ts, &te)) continue;
                Val v;
                if (all || !ext_.get(es[sd], ee[sd] - es[sd] + 1, &v)) {
                    ext_.mark(es[sd], ee[sd] - es[sd] + 1, round_);
                    ask_ext(es[sd], ee[sd], r, sd);
                }
            }
        }
    }

    // Speculation across climbs.  Most climbs end where they stand; the next climb then starts
    // at max(t_e + 1, c + s_min) with a window of s_min points and first asks its start
    // window and rings.  When a round goes to the GPU anyway, also ask those windows for the
    // next prm.spec_climbs climbs, assuming each ends at its start.  Their scores are cached
    // and read only if a climb does start there; the decisions are unchanged.
    void speculate_next_climbs() {
        if (prm.t_max_idle < 0 || prm.max_steps <= 0) return;
        const int64_t d = prm.delta_bu, sm = prm.s_min;
        const int depth = std::min(prm.t_max_idle + 1, spec_depth_for(sm));
        int64_t c = std::max(we_ + 1, c_ + sm);
        for (int j = 0; j < prm.spec_climbs; ++j, c += sm) {
            if (c + sm > t_end) return;
            const int64_t cs = c, ce = c + sm - 1;
            if (!grid_.on_lattice(cs, ce, d)) return;   // cached only on the grid's lattice
            if (spec_starts_.has(c)) continue;   // asked in an earlier round
            spec_starts_.add(c);
            // When the start one delta earlier was asked ahead too, its square of cells
            // (offsets up to `depth` around it) holds every cell of this one but those at
            // offset +depth in a or b: ask only those (a cell the cache has lost since is asked
            // again when a decision needs it).
            const bool near = spec_starts_.has(c - d);
            int64_t ac, bc;
            grid_.centre(cs, ce, &ac, &bc);
            if (!near) spec_cell(ac, bc, cs, ce);
            for (int r = 1; r <= depth; ++r) {
                for (int a = -r; a <= r; ++a)
                    for (int b = -r; b <= r; b += (a == -r || a == r) ? 1 : 2 * r) {
                        if (near && a != depth && b != depth) continue;
                        const int64_t ts = cs + a * d, te = ce + b * d, mm = te - ts + 1;
                        if (mm < prm.s_min || mm > prm.s_max) continue;
                        if (ts < t_begin || te > t_end - 1 || ts <= last_end_) continue;
                        spec_cell(ac + a, bc + b, ts, te);
                    }
                if (prm.pruning && (int64_t)r * d >= prm.k + 1) {
                    const int64_t span = (int64_t)r * d;
                    if (cs - span >= t_begin && cs - span > last_end_) spec_ext(cs - span, cs - 1, 0);
                    if (ce + span <= t_end - 1) spec_ext(ce + 1, ce + span, 1);
                }
            }
        }
    }
    // Speculation within a climb, for the noise test (Sec. 6.2).  The test at a window needs
    // the extension windows [t_s - r delta, t_s - 1] and [t_e + 1, t_e + r delta], r = 1 ..
    // T_maxIdle + 1, which depend on the window's own ends: after each move the next decision
    // would wait for them.  When a round goes to the GPU anyway, also ask those of the ends
    // up to kExtMoves deltas away (positions asked before are remembered; the scores are
    // cached and read only if the climb gets there).
    static constexpr int kExtMoves = 8;
    void speculate_ext_moves() {
        if (!prm.pruning || prm.t_max_idle < 0) return;
        const int64_t d = prm.delta_bu;
        for (int a = -kExtMoves; a <= kExtMoves; ++a) {
            const int64_t p = ws_ + a * d, q = we_ + a * d;
            if (!ext_left_.has(p)) {
                ext_left_.add(p);
                for (int r = 1; r <= prm.t_max_idle + 1; ++r) {
                    const int64_t span = (int64_t)r * d;
                    if (p - span >= t_begin && p - span > last_end_ && p <= t_end) spec_ext(p - span, p - 1, 0);
                }
            }
            if (!ext_right_.has(q)) {
                ext_right_.add(q);
                for (int r = 1; r <= prm.t_max_idle + 1; ++r) {
                    const int64_t span = (int64_t)r * d;
                    if (q + 1 >= t_begin && q + 1 > last_end_ && q + span <= t_end - 1) spec_ext(q + 1, q + span, 1);
                }
            }
        }
    }
    void spec_cell(int64_t a, int64_t b, int64_t ts, int64_t te) {
        if (ts < t_begin || te > t_end - 1) return;   // inside the range only
        if (grid_.known_or_asked(a, b, round_)) return;
        // never take a slot that holds a cell asked in this round
        if (grid_.taken(a, b, round_)) return;
        ask_cell(a, b, ts, te, kDestCell, -1, -1);
    }
    void spec_ext(int64_t ts, int64_t te, int side) {
        const int64_t m = te - ts + 1;
        if (m < prm.k + 1 || ts < t_begin || te > t_end - 1) return;   // inside the range only
        Val v;
        if (ext_.get(ts, m, &v)) return;
        if (!ext_.mark(ts, m, round_)) return;
        ask_ext(ts, te, -1, side);
    }

    // Rings asked per round for the current window size (speculation depth).
    int spec_depth() const { return spec_depth_for(we_ - ws_ + 1); }
    static int spec_depth_for(int64_t m) {
        if (m <= 256) return 4;
        if (m <= 2048) return 2;
        return 1;
    }

    void begin_climb(const Val &v) {
        Iw_ = v.score;
        mw_ = v.mi;
        count(we_ - ws_ + 1);
        for (double &x : L_) x = Iw_;
        t_idle_ = 0;
        step_ = 0;
        run_[0] = run_[1] = 0;
        dropped_[0] = dropped_[1] = false;
        if (t_idle_ <= prm.t_max_idle && step_ < (uint64_t)prm.max_steps)
            phase_ = kDecide;   // ring N_1 was asked together with the start window
        else
            end_climb();
    }

    // One LAHC step on ring N_r (Algorithm 2), with the current dropped directions, read from
    // the score caches.  Returns false, with nothing changed, when a score it needs is not
    // cached (not asked yet, or its slot was taken by another window since).
    bool decide(int r) {
        int64_t ac, bc;
        grid_.centre(ws_, we_, &ac, &bc);
        // One pass over the ring: the best candidate, the pure extensions' scores and the
        // counts to add, committed only once every score is at hand (the counts are whole
        // numbers far below 2^53, so their sums do not depend on the order).
        bool have = false;
        int64_t bs = 0, be = 0, n_read = 0;
        int64_t by_size[kBuckets] = {};
        double pairs_read = 0.0;
        Val bv{0.0, 0.0};
        bool pure[2] = {false, false};   // candidates (-r, 0) and (0, r): the pure extensions
        double pure_sc[2] = {0.0, 0.0};
        for (int64_t a = -r; a <= r; ++a)
            // the perimeter of the square, b ascending within each a
            for (int64_t b = -r; b <= r; b += (a == -r || a == r) ? 1 : 2 * r) {
                int64_t ts, te;
                if (!keep(a, b, r, dropped_[0], dropped_[1], &ts, &te)) continue;
                Val v;
                if (!grid_.get(ac + a, bc + b, &v)) return false;
                const int64_t m = te - ts + 1;
                ++n_read;
                ++by_size[size_bucket((int)m)];
                pairs_read += (double)m * (double)(m - 1);
                if (!have || v.score > bv.score) {        // first maximum wins
                    have = true;
                    bs = ts;
                    be = te;
                    bv = v;
                }
                if (a == -r && b == 0) {
                    pure[0] = true;
                    pure_sc[0] = v.score;
                }
                if (a == 0 && b == r) {
                    pure[1] = true;
                    pure_sc[1] = v.score;
                }
            }
        // the noise test's extension windows (Def. 6.2): the r delta points added on that side
        const bool test = prm.pruning && (int64_t)r * prm.delta_bu >= prm.k + 1;
        Val ext[2];
        if (test) {
            const int64_t span = (int64_t)r * prm.delta_bu;
            const int64_t es[2] = {ws_ - span, we_ + 1};
            for (int sd = 0; sd < 2; ++sd)
                if (pure[sd] && !ext_score(r, sd, es[sd], span, &ext[sd])) return false;
        }
        // every score is at hand: the step
        evals += n_read;
        for (int b = 0; b < kBuckets; ++b) evals_by_size[b] += by_size[b];
        cost += pairs_read;
        if (prm.pruning) {
            for (int sd = 0; sd < 2; ++sd) {
                if (!pure[sd]) continue;
                bool noise = false;
                if (test) {
                    count((int64_t)r * prm.delta_bu);
                    // Def. 6.2 with w = current window, w' = extension, w'' = the neighbour.
                    noise = (Iw_ > 0.0) && (ext[sd].score < prm.tau) && (pure_sc[sd] < Iw_);
                }
                run_[sd] = noise ? run_[sd] + 1 : 0;
                if (run_[sd] >= prm.p) dropped_[sd] = true;
            }
        }
        const int v = (int)(splitmix64_at(prm.seed, (climb_ << 32) + step_ + 1) % (uint64_t)prm.h);
        if (have && (bv.score > L_[v] || bv.score > Iw_)) {
            ws_ = bs;
            we_ = be;
            Iw_ = bv.score;
            mw_ = bv.mi;
            t_idle_ = 0;
        } else {
            t_idle_ += 1;
        }
        if (Iw_ > L_[v]) L_[v] = Iw_;
        ++step_;
        if (t_idle_ <= prm.t_max_idle && step_ < (uint64_t)prm.max_steps)
            phase_ = kDecide;
        else
            end_climb();
        return true;
    }

    void end_climb() {
        if (Iw_ >= prm.sigma) {
            found.push_back(isycos_result_window{ws_, we_, Iw_, mw_});
            last_end_ = we_;
        }
        c_ = std::max(we_ + 1, c_ + prm.s_min);
        ++climb_;
        phase_ = kStart;
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
    Val start_val_{0.0, 0.0};
    std::vector<double> L_;
    int t_idle_ = 0;
    uint64_t step_ = 0, climb_ = 0;
    int run_[2] = {0, 0};
    bool dropped_[2] = {false, false};
    std::vector<RingExt> ring_ext_;
    bool stuck_ = false;
    std::vector<Dest> dest_;
    GridCache grid_;
    ExtCache ext_;
    uint32_t round_ = 0;
    PosSet spec_starts_;   // climb starts whose windows were asked speculatively
    PosSet ext_left_;      // window starts whose left extension windows were asked ahead
    PosSet ext_right_;     // window ends whose right extension windows were asked ahead
    int32_t next_chain_ = 0;
};

// ---------------------------------------------------------------------------------------
// iSYCOS selection (Sec. 5.3, Algorithm 3)
// ---------------------------------------------------------------------------------------
// Sample m of M equal partitions of the range, run SYCOS_TD and SYCOS_BU on each sample
// (their frontiers batched together), score both with the normalised efficiency scores
// (Eqs. normalizeruntime, normalizedwindows, normalizedeffscore), where the runtime of a
// search is the number of pair comparisons m (m - 1) of the windows it scores (a
// deterministic stand-in for wall-clock time), then run the selected search on the range.
class SelectMachine : public SearchMachine {
public:
    bool want(std::vector<WinReq> &req) override {
        if (phase_ == 0) {
            bool any = false;
            int32_t chain_base = 0;
            from_.clear();
            for (size_t i = 0; i < subs_.size(); ++i) {
                if (sub_done_[i]) continue;
                std::vector<WinReq> r;
                if (!subs_[i]->want(r)) {
                    sub_done_[i] = true;
                    continue;
                }
                int32_t top = 0;
                for (WinReq &w : r) {
                    if (w.chain >= 0) {
                        top = std::max(top, w.chain + 1);
                        w.chain += chain_base;
                    }
                }
                chain_base += top;
                from_.push_back({i, r.size()});
                req.insert(req.end(), r.begin(), r.end());
                any = true;
            }
            if (any) return true;
            select();
        }
        std::vector<WinReq> r;
        if (!final_->want(r)) {
            found = final_->found;
            clear_evals();
            add_evals(*final_);
            add_evals(sub_evals_);
            cost = final_->cost;
            return false;
        }
        req.insert(req.end(), r.begin(), r.end());
        return true;
    }

    void give(const isycos_mi_out *res, size_t n) override {
        if (phase_ == 0) {
            size_t off = 0;
            for (const auto &f : from_) {
                subs_[f.first]->give(res + off, f.second);
                off += f.second;
            }
            (void)n;
            return;
        }
        final_->give(res, n);
    }

    void init() {
        const int64_t N = t_end - t_begin;
        const int M = prm.sel_partitions;
        const int ms = std::min(prm.sel_samples, M);
        const int64_t L = N / M;
        std::vector<int> idx((size_t)M);
        for (int i = 0; i < M; ++i) idx[i] = i;
        for (int i = 0; i < ms; ++i) {   // partial Fisher-Yates shuffle, SplitMix64 draws
            const uint64_t r = splitmix64_at(prm.seed ^ 0x5E1EC7ULL, (uint64_t)i + 1);
            const int j = i + (int)(r % (uint64_t)(M - i));
            std::swap(idx[i], idx[j]);
        }
        n_samples_ = ms;
        if (L > 0) {
            for (int i = 0; i < ms; ++i) {
                const int64_t a = t_begin + (int64_t)idx[i] * L;
                SearchParams p = prm;
                p.chunks = 1;   // the samples are searched whole
                for (int mode = 0; mode < 2; ++mode) {
                    p.mode = mode;
                    subs_.push_back(make_machine(xs, ys, a, a + L, p));
                }
            }
        }
        sub_done_.assign(subs_.size(), false);
    }

    int selected = -1;
    double nscore[2] = {0.0, 0.0};

private:
    void select() {
        double t_td = 0.0, t_bu = 0.0, nl_td = 0.0, ns_bu = 0.0;
        sub_evals_.clear_evals();
        for (size_t i = 0; i < subs_.size(); ++i) {
            const SearchMachine &m = *subs_[i];
            const bool td = (i % 2) == 0;
            sub_evals_.add_evals(m);
            (td ? t_td : t_bu) += m.cost;
            for (const auto &w : m.found) {
                const bool small = (double)(w.t_e - w.t_s + 1) <= prm.sel_rho * (double)prm.s_max;
                if (td && !small) nl_td += 1.0;
                if (!td && small) ns_bu += 1.0;
            }
        }
        if (n_samples_ > 0) {
            t_td /= (double)n_samples_;
            t_bu /= (double)n_samples_;
        }
        const double tt = t_td + t_bu;
        const double rt_td = tt > 0.0 ? t_td / tt : 0.5, rt_bu = tt > 0.0 ? t_bu / tt : 0.5;
        const double nn = ns_bu + nl_td;
        const double wl_td = nn > 0.0 ? nl_td / nn : 0.0, ws_bu = nn > 0.0 ? ns_bu / nn : 0.0;
        nscore[0] = prm.sel_alpha * (1.0 / rt_td) + (1.0 - prm.sel_alpha) * wl_td;
        nscore[1] = prm.sel_alpha * (1.0 / rt_bu) + (1.0 - prm.sel_alpha) * ws_bu;
        selected = nscore[0] > nscore[1] ? 0 : 1;
        SearchParams p = prm;
        p.mode = selected;
        final_ = make_machine(xs, ys, t_begin, t_end, p);
        subs_.clear();
        phase_ = 1;
    }

    int phase_ = 0;
    int n_samples_ = 0;
    // evaluation counts of the sampled searches (a machine that never runs, used as a tally)
    struct Tally : SearchMachine {
        bool want(std::vector<WinReq> &) override { return false; }
        void give(const isycos_mi_out *, size_t) override {}
    } sub_evals_;
    std::vector<std::unique_ptr<SearchMachine>> subs_;
    std::vector<bool> sub_done_;
    std::vector<std::pair<size_t, size_t>> from_;
    std::unique_ptr<SearchMachine> final_;
};

// ---------------------------------------------------------------------------------------
// Chunked search (Sec. 7.3, Algorithm 4)
// ---------------------------------------------------------------------------------------
// The range is cut into overlapping chunks [i - s_max, i + L) for i = 0, L, 2L, ... (L =
// floor(length / n_p), clipped to the range); the selected search runs on every chunk
// independently (their frontiers batched together), and the windows of all chunks are
// concatenated in chunk order and sorted by t_s (stable).  Windows found by neighbouring
// chunks may overlap, as in the paper's collected result.
class ChunkMachine : public SearchMachine {
public:
    bool want(std::vector<WinReq> &req) override {
        bool any = false;
        int32_t chain_base = 0;
        from_.clear();
        for (size_t i = 0; i < subs_.size(); ++i) {
            if (done_[i]) continue;
            std::vector<WinReq> r;
            if (!subs_[i]->want(r)) {
                done_[i] = true;
                continue;
            }
            int32_t top = 0;
            for (WinReq &w : r)
                if (w.chain >= 0) {
                    top = std::max(top, w.chain + 1);
                    w.chain += chain_base;
                }
            chain_base += top;
            from_.push_back({i, r.size()});
            req.insert(req.end(), r.begin(), r.end());
            any = true;
        }
        if (any) return true;
        found.clear();
        clear_evals();
        cost = 0.0;
        for (const auto &m : subs_) {
            found.insert(found.end(), m->found.begin(), m->found.end());
            add_evals(*m);
            cost += m->cost;
        }
        std::stable_sort(found.begin(), found.end(),
                         [](const isycos_result_window &u, const isycos_result_window &v) { return u.t_s < v.t_s; });
        return false;
    }

    void give(const isycos_mi_out *res, size_t n) override {
        size_t off = 0;
        for (const auto &f : from_) {
            subs_[f.first]->give(res + off, f.second);
            off += f.second;
        }
        (void)n;
    }

    void init() {
        const int64_t N = t_end - t_begin;
        const int64_t L = std::max<int64_t>(1, N / prm.chunks);
        SearchParams p = prm;
        p.chunks = 1;
        for (int64_t i = 0; i < N; i += L) {
            const int64_t a = t_begin + std::max<int64_t>(0, i - prm.s_max);
            const int64_t b = t_begin + std::min<int64_t>(N, i + L);
            subs_.push_back(make_machine(xs, ys, a, b, p));
        }
        done_.assign(subs_.size(), false);
    }

private:
    std::vector<std::unique_ptr<SearchMachine>> subs_;
    std::vector<bool> done_;
    std::vector<std::pair<size_t, size_t>> from_;
};

}  // namespace

std::unique_ptr<SearchMachine> make_machine(int32_t xs, int32_t ys, int64_t t_begin, int64_t t_end,
                                            const SearchParams &p) {
    if (p.chunks > 1 && p.mode != 2) {
        auto m = std::make_unique<ChunkMachine>();
        m->xs = xs;
        m->ys = ys;
        m->t_begin = t_begin;
        m->t_end = t_end;
        m->prm = p;
        m->init();
        return m;
    }
    if (p.mode == 2) {
        auto m = std::make_unique<SelectMachine>();
        m->xs = xs;
        m->ys = ys;
        m->t_begin = t_begin;
        m->t_end = t_end;
        m->prm = p;
        m->init();
        return m;
    }
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

namespace {

// Work of a chain in units of pair comparisons: the first window from scratch, then per step
// the points moved times the window (influence checks, re-searched and added points).
double chain_cost(const std::vector<const WinReq *> &g, int k) {
    double c = (double)g[0]->m * g[0]->m;
    for (size_t i = 1; i < g.size(); ++i) {
        const int64_t s0 = g[i - 1]->start, e0 = s0 + g[i - 1]->m - 1;
        const int64_t s1 = g[i]->start, e1 = s1 + g[i]->m - 1;
        const int64_t inter = std::max<int64_t>(0, std::min(e0, e1) - std::max(s0, s1) + 1);
        const int64_t moved = (e0 - s0 + 1) + (e1 - s1 + 1) - 2 * inter;
        c += (double)moved * g[i]->m * (k + 3);
    }
    return c;
}

double scratch_cost(const std::vector<const WinReq *> &g) {
    double c = 0.0;
    for (const WinReq *r : g)
        if (!r->base) c += (double)r->m * r->m;
    return c;
}

}  // namespace

// Machines are batched together when they share k and the estimator.
constexpr int kBatchKeys = 2 * (kMaxK + 1);
inline int batch_key(const SearchMachine &m) { return m.prm.k + (kMaxK + 1) * m.prm.estimator; }

// Collect the machines' requests and start their evaluation on lane L: chains (rare) run
// synchronously, batched windows of every k but the last too, and the last batch is left
// open on the lane; round_end() waits for it and hands the results to the machines.
isycos_status round_begin(isycos_ctx *ctx, Lane &L, std::vector<SearchMachine *> &ms,
                          std::vector<bool> &finished, cudaStream_t st, Round &rd) {
    rd.ms = &ms;
    rd.finished = &finished;
    rd.L = &L;
    rd.open_k = 0;
    if (rd.reqs.size() < ms.size()) rd.reqs.resize(ms.size());
    for (size_t q = 0; q < ms.size(); ++q) rd.reqs[q].clear();
    rd.first.assign(ms.size(), 0);
    rd.active.assign(ms.size(), 0);
    size_t total = 0;
    int k = 0;
    for (size_t q = 0; q < ms.size(); ++q)
        if (!finished[q]) rd.active[q] = ms[q]->want(rd.reqs[q]) ? 1 : 0;
    for (size_t q = 0; q < ms.size(); ++q) {
        if (finished[q]) continue;
        if (!rd.active[q]) {
            finished[q] = true;
            continue;
        }
        if (k && batch_key(*ms[q]) != k) k = -1;
        if (k == 0) k = batch_key(*ms[q]);
        rd.first[q] = total;
        total += rd.reqs[q].size();
    }
    rd.total = total;
    if (total == 0) return ISYCOS_OK;
    rd.res.resize(total);
    bool present[kBatchKeys] = {false};
    int last_k = 0;
    for (size_t q = 0; q < ms.size(); ++q)
        if (!finished[q] && !rd.reqs[q].empty()) {
            present[batch_key(*ms[q])] = true;
            last_k = std::max(last_k, batch_key(*ms[q]));
        }
    // Per (k, estimator) (machines of one call normally share them), split the requests into
    // the batched list and the chains that the incremental kernel takes.  Only keys with
    // requests are visited: the last one's batch stays open in rd.batch / rd.where.
    for (int kk = 1; kk < kBatchKeys; ++kk) {
        if (!present[kk] || (k > 0 && kk != k)) continue;
        const int k_nb = kk % (kMaxK + 1), est = kk / (kMaxK + 1);
        std::vector<HostWindow> &batch = rd.batch;
        std::vector<size_t> &where = rd.where;
        batch.clear();
        where.clear();
        std::vector<ChainSpec> chains;
        for (size_t q = 0; q < ms.size(); ++q) {
            if (finished[q] || rd.reqs[q].empty() || batch_key(*ms[q]) != kk) continue;
            const auto &rq = rd.reqs[q];
            // the incremental kernel implements the second estimator only
            const bool chains_on = ctx->opt_incremental != 0 && est == 0;
            // A chain's requests are consecutive (its base window first): walk the runs.
            size_t i = 0;
            while (i < rq.size()) {
                size_t e = i + 1;
                if (chains_on && rq[i].chain >= 0)
                    while (e < rq.size() && rq[e].chain == rq[i].chain) ++e;
                bool use = false;
                if (e - i >= 2) {
                    thread_local std::vector<const WinReq *> g;
                    g.clear();
                    for (size_t u = i; u < e; ++u) g.push_back(&rq[u]);
                    if (ctx->opt_incremental == 2) use = true;
                    if (ctx->opt_incremental == 1) use = chain_cost(g, k_nb) < 0.5 * scratch_cost(g);
                }
                if (use) {
                    ChainSpec sp;
                    sp.xs = ms[q]->xs;
                    sp.ys = ms[q]->ys;
                    for (size_t u = i; u < e; ++u) {
                        sp.starts.push_back(rq[u].start);
                        sp.sizes.push_back(rq[u].m);
                        sp.out_idx.push_back(rq[u].base ? -1 : (int64_t)(rd.first[q] + u));
                    }
                    chains.push_back(std::move(sp));
                } else {
                    for (size_t u = i; u < e; ++u) {
                        if (rq[u].base) continue;
                        batch.push_back(HostWindow{ms[q]->xs, ms[q]->ys, rq[u].start, rq[u].m});
                        where.push_back(rd.first[q] + u);
                    }
                }
                i = e;
            }
        }
        if (!chains.empty()) {
            isycos_status rc = engine_eval_chains(ctx, L, chains.data(), chains.size(), k_nb, rd.res.data(),
                                                  (int64_t)total, st);
            if (rc) return rc;
        }
        if (!batch.empty()) {
            isycos_status rc = engine_launch(ctx, L, batch.data(), (int64_t)batch.size(), k_nb, est,
                                             nullptr, nullptr, nullptr, st);
            if (rc) return rc;
            if (kk == last_k) {
                rd.open_k = kk;   // left open for round_end
            } else {
                rd.tmp.resize(batch.size());
                if ((rc = engine_collect(ctx, L, rd.tmp.data()))) return rc;
                for (size_t i = 0; i < batch.size(); ++i) rd.res[where[i]] = rd.tmp[i];
            }
        }
    }
    return ISYCOS_OK;
}

isycos_status round_end(isycos_ctx *ctx, Round &rd) {
    if (rd.total == 0) return ISYCOS_OK;
    if (rd.open_k) {
        rd.tmp.resize(rd.batch.size());
        isycos_status rc = engine_collect(ctx, *rd.L, rd.tmp.data());
        rd.open_k = 0;
        if (rc) return rc;
        for (size_t i = 0; i < rd.batch.size(); ++i) rd.res[rd.where[i]] = rd.tmp[i];
    }
    std::vector<SearchMachine *> &ms = *rd.ms;
    for (size_t q = 0; q < ms.size(); ++q)
        if (!(*rd.finished)[q] && !rd.reqs[q].empty()) ms[q]->give(rd.res.data() + rd.first[q], rd.reqs[q].size());
    return ISYCOS_OK;
}

isycos_status step_machines(isycos_ctx *ctx, Lane &L, std::vector<SearchMachine *> &ms,
                            std::vector<bool> &finished, cudaStream_t st, int64_t *n_eval) {
    thread_local Round rd;
    isycos_status rc = round_begin(ctx, L, ms, finished, st, rd);
    if (n_eval) *n_eval = (int64_t)rd.total;
    if (rc) return rc;
    return round_end(ctx, rd);
}

isycos_status run_machines(isycos_ctx *ctx, Lane &L, std::vector<SearchMachine *> &ms,
                           cudaStream_t st) {
    std::vector<bool> finished(ms.size(), false);
    for (;;) {
        int64_t n = 0;
        isycos_status rc = step_machines(ctx, L, ms, finished, st, &n);
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

}  // extern "C"

// ---------------------------------------------------------------------------------------
// SYCOS_BU on the device (bu_device.cu): all eligible BU queries of a call in one launch per
// k, started before the host lanes run the other queries and collected after them.
// ---------------------------------------------------------------------------------------
struct BuDeviceRun {
    std::vector<int64_t> idx;            // query indices of the call, grouped by k
    std::vector<int> group_k;
    std::vector<int64_t> group_off;
    int64_t cap = 0;
    bool open = false;
    cudaStream_t st = nullptr;
    std::vector<DevBuResult> res;
};

static bool bu_device_eligible(const isycos_ctx *ctx, const SearchParams &p) {
    // (ISYCOS_OPT_INCREMENTAL = 2 asks for the incremental chains, which only the host
    // machines form)
    return ctx->opt_bu_device && ctx->opt_incremental != 2 && p.mode == 1 && p.chunks <= 1 &&
           p.h <= kBuMaxH && p.t_max_idle <= kBuMaxIdle;
}

static isycos_status bu_device_begin(isycos_ctx *ctx, BuDeviceRun &R, const int32_t *xs,
                                     const int32_t *ys, const int64_t *t_begin,
                                     const int64_t *t_end, const SearchParams *prm,
                                     size_t prm_stride, int64_t cap) {
    std::stable_sort(R.idx.begin(), R.idx.end(), [&](int64_t a, int64_t b) {
        return prm[a * prm_stride].k < prm[b * prm_stride].k;
    });
    const size_t n = R.idx.size();
    std::vector<DevBuQuery> qs(n);
    for (size_t i = 0; i < n; ++i) {
        const int64_t q = R.idx[i];
        const SearchParams &p = prm[q * prm_stride];
        DevBuQuery &d = qs[i];
        d.x = ctx->series_ptr[xs[q]];
        d.y = ctx->series_ptr[ys[q]];
        d.t_begin = t_begin[q];
        d.t_end = t_end[q];
        d.sigma = p.sigma;
        d.tau = p.tau;
        d.seed = p.seed;
        d.k = p.k;
        d.score_kind = p.score_kind;
        d.s_min = p.s_min;
        d.s_max = p.s_max;
        d.delta = p.delta_bu;
        d.h = p.h;
        d.t_max_idle = p.t_max_idle;
        d.p = p.p;
        d.pruning = p.pruning;
        d.max_steps = p.max_steps;
        d.est = p.estimator;
        d.pad = 0;
        if (i == 0 || qs[i - 1].k != d.k) {
            R.group_k.push_back(d.k);
            R.group_off.push_back((int64_t)i);
        }
    }
    R.group_off.push_back((int64_t)n);
    R.cap = std::max<int64_t>(1, cap);
    isycos_status rc;
    Lane *L = nullptr;
    if ((rc = get_lane(ctx, kLaneSlots - 1, &L))) return rc;   // highest stream priority
    R.st = L->stream;
    std::vector<int> grids;
    for (size_t g = 0; g < R.group_k.size(); ++g) {
        int per_sm = 0;
        cudaError_t e = bu_device_prepare(R.group_k[g], &per_sm);
        if (e != cudaSuccess || per_sm < 1) return cuda_fail(ctx, e != cudaSuccess ? e : cudaErrorInvalidConfiguration, "device SYCOS_BU setup");
        const int64_t nq = R.group_off[g + 1] - R.group_off[g];
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nq, (int64_t)ctx->n_sm * per_sm));
        grids.push_back(grid);
    }
    const size_t n_groups = R.group_k.size();
    if ((rc = dev_reserve(ctx, ctx->d_bu_q, sizeof(DevBuQuery) * n))) return rc;
    if ((rc = dev_reserve(ctx, ctx->d_bu_res, sizeof(DevBuResult) * n))) return rc;
    if ((rc = dev_reserve(ctx, ctx->d_bu_found, sizeof(isycos_result_window) * n * (size_t)R.cap))) return rc;
    if ((rc = dev_reserve(ctx, ctx->d_bu_queue, 4 * n_groups + 16))) return rc;
    cudaError_t e = cudaSuccess;
    if (!ctx->ev_bu[0]) e = cudaEventCreate(&ctx->ev_bu[0]);
    if (e == cudaSuccess && !ctx->ev_bu[1]) e = cudaEventCreate(&ctx->ev_bu[1]);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->d_bu_q.p, qs.data(), sizeof(DevBuQuery) * n, cudaMemcpyHostToDevice, R.st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_bu_queue.p, 0, 4 * n_groups, R.st);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_bu[0], R.st);
    for (size_t g = 0; g < n_groups && e == cudaSuccess; ++g) {
        BuLaunch a;
        const int64_t off = R.group_off[g];
        a.q = reinterpret_cast<const DevBuQuery *>(ctx->d_bu_q.p) + off;
        a.n_q = (int32_t)(R.group_off[g + 1] - off);
        a.spec_climbs = ctx->opt_spec_climbs;
        a.res = reinterpret_cast<DevBuResult *>(ctx->d_bu_res.p) + off;
        a.found = reinterpret_cast<isycos_result_window *>(ctx->d_bu_found.p) + off * R.cap;
        a.cap = R.cap;
        a.queue = reinterpret_cast<int32_t *>(ctx->d_bu_queue.p) + g;
        a.psi_fx = ctx->d_psi_fx;
        a.log_fx = ctx->d_log_fx;
        a.limit_ns = (uint64_t)ctx->opt_time_limit_ms * 1000000ull;
        e = bu_device_launch(a, R.group_k[g], grids[g], R.st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_bu[1], R.st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device SYCOS_BU launch");
    R.open = true;
    return ISYCOS_OK;
}

// Wait for the device searches and fetch their windows into found[i] (query R.idx[i]).
static isycos_status bu_device_end(isycos_ctx *ctx, BuDeviceRun &R,
                                   std::vector<std::vector<isycos_result_window>> &found,
                                   int64_t *decided) {
    if (!R.open) return ISYCOS_OK;
    R.open = false;
    const size_t n = R.idx.size();
    R.res.resize(n);
    cudaError_t e = cudaMemcpyAsync(R.res.data(), ctx->d_bu_res.p, sizeof(DevBuResult) * n,
                                    cudaMemcpyDeviceToHost, R.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(R.st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device SYCOS_BU");
    found.assign(n, {});
    bool timeout = false;
    int64_t windows = 0, pairs = 0;
    for (size_t i = 0; i < n; ++i) {
        const DevBuResult &r = R.res[i];
        timeout |= r.status != 0;
        const int64_t keep = std::min<int64_t>(r.n_found, R.cap);
        found[i].resize((size_t)r.n_found);
        if (keep > 0)
            e = cudaMemcpyAsync(found[i].data(),
                                reinterpret_cast<isycos_result_window *>(ctx->d_bu_found.p) + (int64_t)i * R.cap,
                                sizeof(isycos_result_window) * (size_t)keep, cudaMemcpyDeviceToHost, R.st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "device SYCOS_BU results");
        windows += r.windows;
        pairs += r.pairs;
        *decided += r.evals;
    }
    e = cudaStreamSynchronize(R.st);
    float t0 = 0.0f, t1 = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t0, ctx->ev_ref, ctx->ev_bu[0]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, ctx->ev_ref, ctx->ev_bu[1]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device SYCOS_BU results");
    add_stats(ctx, windows, pairs, (int64_t)R.group_k.size(), 1, 0);
    {
        std::lock_guard<std::mutex> g(ctx->stats_mu);
        ctx->kernel_iv.push_back({t0, t1});
        ctx->stats.mi_kernel_launches += (int64_t)R.group_k.size();
        ctx->stats.dev_queries += (int64_t)n;
        for (size_t i = 0; i < n; ++i) {
            const DevBuResult &r = R.res[i];
            for (int b = 0; b < kBuckets; ++b) {
                ctx->stats.windows_by_size[b] += r.windows_by_size[b];
                ctx->stats.decided_by_size[b] += r.evals_by_size[b];
            }
            ctx->stats.dev_rounds += r.rounds;
            for (int j = 0; j < 3; ++j) ctx->stats.dev_cycles[j] += r.cycles[j];
            ctx->stats.work_bf += r.work_bf;
        }
    }
    if (timeout)
        return fail(ctx, ISYCOS_E_TIMEOUT, "device SYCOS_BU: the time limit of %lld ms ran out",
                    (long long)ctx->opt_time_limit_ms);
    return ISYCOS_OK;
}

// Run independent queries (each with its own parameters) to completion.
static isycos_status run_queries(isycos_ctx *ctx, int64_t n_q, const int32_t *xs, const int32_t *ys,
                                 const int64_t *t_begin, const int64_t *t_end,
                                 const SearchParams *prm, size_t prm_stride,
                                 isycos_result_window *out, int64_t cap_per_query, int64_t *n_out) {
    isycos_status rc;
    std::vector<std::unique_ptr<SearchMachine>> own;
    std::vector<SearchMachine *> ms;
    std::vector<int64_t> host_of((size_t)n_q, -1);   // index into ms, or -1: on the device
    BuDeviceRun bu;
    for (int64_t q = 0; q < n_q; ++q) {
        if ((rc = check_query(ctx, xs[q], ys[q], t_begin[q], t_end[q]))) return rc;
        if (bu_device_eligible(ctx, prm[q * prm_stride])) {
            bu.idx.push_back(q);
            continue;
        }
        own.push_back(make_machine(xs[q], ys[q], t_begin[q], t_end[q], prm[q * prm_stride]));
        host_of[q] = (int64_t)ms.size();
        ms.push_back(own.back().get());
    }
    // the device searches start first, on the highest-priority stream, so that their CTAs
    // take their SMs before the host lanes' launches fill the GPU
    if (!bu.idx.empty()) {
        if ((rc = bu_device_begin(ctx, bu, xs, ys, t_begin, t_end, prm, prm_stride, cap_per_query)))
            return rc;
    }
    // Independent queries split over engine lanes, one host thread per lane: each thread runs
    // its machines' rounds on its own stream, so that the sequential decision logic of many
    // queries proceeds in parallel and their batches overlap on the GPU.
    const int n_lanes = (int)std::max<int64_t>(1, std::min<int64_t>(ctx->max_lanes, ((int64_t)ms.size() + 3) / 4));
    // SYCOS_TD queries make few, large launches (throughput-bound); the others many small
    // ones (latency-bound).  When both are present they get separate lanes: the TD lanes'
    // launches leave a quarter of the GPU's CTA slots free and the others run on
    // high-priority streams, so that their rounds overlap the large launches instead of
    // waiting behind them.  The TD lanes take a quarter of the lanes, the latency-bound
    // queries the rest, so that the call keeps one host thread per lane.
    std::vector<SearchMachine *> thr, lat;
    for (SearchMachine *m : ms) (m->prm.mode == 0 ? thr : lat).push_back(m);
    const bool split = !thr.empty() && !lat.empty();
    int n_thr = 0, n_all = n_lanes;
    if (split) {
        n_thr = (int)std::max<int64_t>(1, std::min<int64_t>(std::max(1, ctx->max_lanes / 4), ((int64_t)thr.size() + 3) / 4));
        const int n_lat = (int)std::max<int64_t>(
            1, std::min<int64_t>(std::max(1, ctx->max_lanes - n_thr), ((int64_t)lat.size() + 3) / 4));
        n_all = n_thr + n_lat;
    }
    std::vector<Lane *> lanes((size_t)n_all);
    std::vector<std::vector<SearchMachine *>> parts((size_t)n_all);
    for (int i = 0; i < n_all; ++i) {
        const bool prio = split && i >= n_thr;
        if ((rc = get_lane(ctx, prio ? kPrioLaneBase + (i - n_thr) : i, &lanes[i]))) return rc;
        lanes[i]->slot_share = split && !prio ? 3 : 4;
    }
    if (split) {
        for (size_t q = 0; q < thr.size(); ++q) parts[q % n_thr].push_back(thr[q]);
        for (size_t q = 0; q < lat.size(); ++q) parts[n_thr + q % (n_all - n_thr)].push_back(lat[q]);
    } else {
        for (size_t q = 0; q < ms.size(); ++q) parts[q % n_lanes].push_back(ms[q]);
    }
    std::vector<isycos_status> st((size_t)n_all, ISYCOS_OK);
    std::vector<std::thread> th;
    const int dev = ctx->device;
    for (int i = 1; i < n_all; ++i)
        th.emplace_back([&, i] {
            cudaSetDevice(dev);
            st[i] = run_machines(ctx, *lanes[i], parts[i], lanes[i]->stream);
        });
    if (!ms.empty()) st[0] = run_machines(ctx, *lanes[0], parts[0], lanes[0]->stream);
    for (auto &t : th) t.join();
    std::vector<std::vector<isycos_result_window>> dev_found;
    int64_t decided = 0;
    const isycos_status st_bu = bu_device_end(ctx, bu, dev_found, &decided);
    for (isycos_status s1 : st)
        if (s1) return s1;
    if (st_bu) return st_bu;
    std::vector<int64_t> dev_of((size_t)n_q, -1);
    for (size_t i = 0; i < bu.idx.size(); ++i) dev_of[bu.idx[i]] = (int64_t)i;
    isycos_status result = ISYCOS_OK;
    {
        std::lock_guard<std::mutex> g2(ctx->stats_mu);
        for (SearchMachine *m : ms) {
            decided += m->evals;
            for (int b = 0; b < kBuckets; ++b) ctx->stats.decided_by_size[b] += m->evals_by_size[b];
        }
        ctx->stats.decided_windows += decided;
    }
    for (int64_t q = 0; q < n_q; ++q) {
        const auto &f = host_of[q] >= 0 ? ms[host_of[q]]->found : dev_found[dev_of[q]];
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

extern "C" {

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
    return run_queries(ctx, n_q, xs, ys, t_begin, t_end, &p, 0, out, cap_per_query, n_out);
}

isycos_status isycos_search_queries(isycos_ctx *ctx, int64_t n_q, const isycos_query *queries,
                                    isycos_result_window *out, int64_t cap_per_query,
                                    int64_t *n_out) {
    if (!ctx) return ISYCOS_E_INVAL;
    if (n_q < 0 || (n_q > 0 && (!queries || !n_out)) || cap_per_query < 0 ||
        (cap_per_query > 0 && n_q > 0 && !out))
        return fail(ctx, ISYCOS_E_INVAL, "search: bad arguments");
    std::vector<SearchParams> prm((size_t)n_q);
    std::vector<int32_t> xs((size_t)n_q), ys((size_t)n_q);
    std::vector<int64_t> tb((size_t)n_q), te((size_t)n_q);
    for (int64_t q = 0; q < n_q; ++q) {
        isycos_status rc = resolve_params(ctx, &queries[q].params, &prm[q]);
        if (rc) return rc;
        xs[q] = queries[q].xs;
        ys[q] = queries[q].ys;
        tb[q] = queries[q].t_begin;
        te[q] = queries[q].t_end;
    }
    std::lock_guard<std::mutex> g(ctx->engine_mu);
    cudaSetDevice(ctx->device);
    return run_queries(ctx, n_q, xs.data(), ys.data(), tb.data(), te.data(), prm.data(), 1, out,
                       cap_per_query, n_out);
}

}  // extern "C"
