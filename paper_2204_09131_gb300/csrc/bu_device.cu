// Device-resident SYCOS_BU: Algorithm 2 of arXiv 2204.09131 (Sec. 5.2, LAHC climbs over
// the ring neighbourhoods N_r) with the noise pruning of Sec. 6.3, run entirely on the GPU.
//
// One CTA runs one query at a time (queries come from a counter).  The CTA alternates
//   decide + ask (warp 0): replay Algorithm 2 on the scores at hand until one is missing,
//       then list the windows the next decision needs (ring N_r of the current window and
//       the noise test's extension windows) and, speculatively, windows later decisions are
//       likely to need (the outer rings, the first windows of the next climbs assuming each
//       climb ends where it starts, the extension windows of nearby window ends);
//   evaluate (all warps): the listed windows' MI by the brute-force block of the batched
//       kernel (the same binary32 and int64 arithmetic, so every score is bit-identical);
//   finish (all threads): the binary64 scalars of each window, into the CTA's score cache.
// The score cache (window key and score) and a tile of the pair's series around the search
// cursor live in shared memory, so a decision step and a window's staging cost shared-memory
// latency only.  The MI of a found window (reported beside its score) is evaluated once more
// when the query ends.
// The decisions are those of the sequential algorithm: scores are a pure function of the
// window, so speculation changes which windows are evaluated, never which are chosen.
// Termination: every round completes at least one decision (the windows the next decision
// needs are kept in a step buffer that nothing else overwrites), and a query ends after
// finitely many climbs; a %globaltimer deadline bounds a launch's time all the same.
//
// Readings shared with the oracle (Sec. 5.2): ring N_r = offsets (a, b) with max(|a|, |b|)
// = r of the window [t_s + a delta, t_e + b delta]; the first maximum in a-major, b-minor
// order wins; acceptance is strict (> the history entry or > the current score); history
// index SplitMix64((climb << 32) + step + 1) mod h; after a climb the cursor moves to
// max(t_e + 1, c + s_min); the noise test (Def. 6.2) runs on the pure extensions (-r, 0) and
// (0, r) with the extension alone as w'; p consecutive detections drop that side.
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "bu_device.h"
#include "isycos_internal.h"
#include "ksg_device.cuh"

namespace isy {

using namespace dev;

namespace {

constexpr int kNT = kBuThreads;
constexpr int kW = kNT / 32;
constexpr int kRoundCap = 512;                         // windows per round
constexpr int kStepCap = 8 * (kBuMaxIdle + 1) + 2;     // ring N_r cells + 2 extensions
constexpr int kSetSlots = 256;
constexpr int kExtMoves = 8;
static_assert(kStepCap <= kRoundCap, "the needed windows of one decision fit a round");
constexpr unsigned long long kPend = 1ull << 62;       // slot claimed in this round
constexpr unsigned long long kEmpty = 1ull << 63;
enum { kPhStart = 0, kPhClimb = 1, kPhDone = 2 };

struct Shared {
    // score cache: direct mapped by a hash of the window key
    unsigned long long c_key[kBuCacheSlots];
    double c_score[kBuCacheSlots];
    // the pair's values at [tile_lo, tile_lo + kBuTile)
    float2 tile[kBuTile];
    // the round's window list
    long long l_start[kRoundCap];
    long long acc_psi[kRoundCap];
    long long acc_log[kRoundCap];
    // step buffer: the windows of the decision the list was made for
    double st_score[kStepCap];
    // positions asked ahead (direct mapped over position / delta)
    long long set_spec[kSetSlots];
    long long set_left[kSetSlots];
    long long set_right[kSetSlots];
    double L[kBuMaxH];
    unsigned long long evals_by[15];
    unsigned long long win_by[15];
    unsigned long long pairs;
    unsigned long long units;
    unsigned long long work_bf;
    long long tile_lo, tile_hi;   // tile_hi: one past the last point held
    int l_m[kRoundCap];
    int l_slot[kRoundCap];
    int l_step[kRoundCap];
    int l_ubase[kRoundCap + 1];
    signed char st_have[kStepCap];
};
static_assert(sizeof(Shared) <= 200 * 1024, "one CTA's shared memory fits an SM with room to spare");

// The climb state, kept in registers of warp 0 (every lane holds the same values) during
// the decide + ask phase and in shared memory between phases.
struct Climb {
    long long c, last_end, ws, we;
    double Iw;
    unsigned long long step, climb;
    int phase, t_idle, run0, run1, drop0, drop1;
};

struct StepKey {
    int valid, phase, r, d0, d1;
    long long ws, we;
};

__host__ __device__ inline unsigned long long splitmix64_at(unsigned long long seed, unsigned long long n) {
    unsigned long long z = seed + n * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long wkey(long long ts, int m) {
    return ((unsigned long long)ts << 16) | (unsigned long long)m;
}
__device__ __forceinline__ int slot_of(unsigned long long key) {
    key ^= key >> 29;
    key *= 0xBF58476D1CE4E5B9ull;
    key ^= key >> 32;
    return (int)(key & (unsigned long long)(kBuCacheSlots - 1));
}
__device__ __forceinline__ int size_bucket_d(int m) { return m <= 1 ? 0 : 32 - __clz(m - 1); }
// Position of the n-th (0-based) set bit of mask (n < popc(mask)).
__device__ __forceinline__ int nth_set_bit(unsigned mask, int n) {
    for (int i = 0; i < n; ++i) mask &= mask - 1;
    return __ffs(mask) - 1;
}

// Score of window (ts, m) from the CTA's cache.
__device__ __forceinline__ bool cache_get(const Shared &S, long long ts, int m, double *sc) {
    const unsigned long long key = wkey(ts, m);
    const int s = slot_of(key);
    if (S.c_key[s] != key) return false;
    *sc = S.c_score[s];
    return true;
}

// Ring N_r cell idx (0 .. 8r - 1) in Algorithm 2's enumeration order: a from -r to r (outer),
// b from -r to r (inner) over the perimeter max(|a|, |b|) = r.
__device__ __forceinline__ void perim(int r, int idx, int *a, int *b) {
    const int row = 2 * r + 1;
    if (idx < row) {
        *a = -r;
        *b = -r + idx;
    } else if (idx < row + 2 * (2 * r - 1)) {
        const int t = idx - row;
        *a = -r + 1 + (t >> 1);
        *b = (t & 1) ? r : -r;
    } else {
        *a = r;
        *b = -r + (idx - row - 2 * (2 * r - 1));
    }
}

// Rings asked per round for a window of m points (the host search's speculation depth).
__device__ __forceinline__ int spec_depth(long long m) { return m <= 256 ? 4 : (m <= 2048 ? 2 : 1); }

struct Ctx {
    Shared &S;
    const DevBuQuery &q;
    int lane;
};

// A candidate of ring N_r around (ws, we) that passes the search's filters (Algorithm 2's
// neighbourhood with the sizes, range, dropped sides and non-overlap with found windows).
__device__ __forceinline__ bool keep(const DevBuQuery &q, const Climb &C, int a, int b, int r,
                                     int d0, int d1, long long *ts, long long *te) {
    if (max(abs(a), abs(b)) != r) return false;
    if (d0 && a < 0) return false;
    if (d1 && b > 0) return false;
    *ts = C.ws + (long long)a * q.delta;
    *te = C.we + (long long)b * q.delta;
    const long long mm = *te - *ts + 1;
    if (mm < q.s_min || mm > q.s_max) return false;
    if (*ts < q.t_begin || *te > q.t_end - 1 || *ts <= C.last_end) return false;
    return true;
}

// ---------------------------------------------------------------------------------------
// Asking for windows (warp 0): each lane brings one candidate; hits fill the step buffer,
// misses claim their cache slot and join the round's list.
// ---------------------------------------------------------------------------------------
struct Asker {
    int n;          // list length (warp-uniform)
    bool full;
    long long lo, hi;   // range of the listed windows (this lane's part)
};

__device__ void ask_batch(Ctx &X, Asker &A, bool valid, long long ts, int m, int step) {
    Shared &S = X.S;
    unsigned long long key = 0, k0 = 0;
    int s = -1;
    // 0 nothing, 1 claim a slot, 2 list without a slot (needed, slot busy this round)
    int want = 0;
    if (valid) {
        key = wkey(ts, m);
        s = slot_of(key);
        k0 = S.c_key[s];
        if (k0 == key) {   // cached
            if (step >= 0) {
                S.st_score[step] = S.c_score[s];
                S.st_have[step] = 1;
            }
        } else if (k0 & kPend) {   // this window, or another one, was listed in this round
            if (step >= 0) want = 2;
        } else {
            want = 1;
        }
    }
    const unsigned mask = __ballot_sync(kFull, want != 0);
    if (mask == 0) return;
    const int pos = A.n + __popc(mask & ((1u << X.lane) - 1));
    if (want) {
        int slot = -1;
        if (pos >= kRoundCap) {
            want = 0;   // only speculative windows can overflow (the needed ones come first)
        } else if (want == 1) {
            const unsigned long long old = atomicCAS(&S.c_key[s], k0, key | kPend);
            if (old == k0) slot = s;
            else if (step < 0) m = 0;   // lost the slot to another window of this batch: drop
        }
        if (want) {
            S.l_start[pos] = ts;
            S.l_m[pos] = m;
            S.l_slot[pos] = slot;
            S.l_step[pos] = step;
            S.acc_psi[pos] = 0;
            S.acc_log[pos] = 0;
            if (m > 0) {
                A.lo = min(A.lo, ts);
                A.hi = max(A.hi, ts + m);
            }
        }
    }
    A.n = min(kRoundCap, A.n + __popc(mask));
    A.full = A.n >= kRoundCap;
}

// Ring N_r around the current window with the given dropped sides, and (pruning) the noise
// test's extension windows of its pure extensions; needed: into the step buffer.
__device__ void ask_ring(Ctx &X, Asker &A, const Climb &C, int r, int d0, int d1, bool needed) {
    const DevBuQuery &q = X.q;
    const int n = 8 * r;
    for (int base = 0; base < n; base += 32) {
        if (!needed && A.full) return;
        const int idx = base + X.lane;
        long long ts = 0, te = 0;
        bool ok = false;
        if (idx < n) {
            int a, b;
            perim(r, idx, &a, &b);
            ok = keep(q, C, a, b, r, d0, d1, &ts, &te);
        }
        ask_batch(X, A, ok, ts, (int)(te - ts + 1), needed ? idx : -1);
    }
    if (q.pruning && (long long)r * q.delta >= q.k + 1) {
        const long long span = (long long)r * q.delta;
        bool ok = false;
        long long ts = 0, te = 0;
        if (X.lane < 2) {
            const int sd = X.lane;
            long long t1, t2;
            if (keep(q, C, sd == 0 ? -r : 0, sd == 0 ? 0 : r, r, d0, d1, &t1, &t2)) {
                ok = true;
                ts = sd == 0 ? C.ws - span : C.we + 1;
                te = ts + span - 1;
            }
        }
        ask_batch(X, A, ok, ts, (int)(te - ts + 1), needed ? n + X.lane : -1);
    }
}

__device__ __forceinline__ int set_slot(long long p, int delta) {
    return (int)(((p < 0 ? 0 : p) / delta) & (kSetSlots - 1));
}

// The first windows of the next climbs, assuming each climb ends at its start: the start
// window, rings N_1 .. N_depth around it and the extension windows of those rings.  Climb
// starts asked in an earlier round are skipped; the candidates of the new ones are spread
// over the lanes.
__device__ void spec_next_climbs(Ctx &X, Asker &A, const Climb &C, int n_climbs) {
    const DevBuQuery &q = X.q;
    Shared &S = X.S;
    const long long sm = q.s_min, d = q.delta;
    const int depth = min(q.t_max_idle + 1, spec_depth(sm));
    const int n_ring = 4 * depth * (depth + 1);
    const int per = 1 + n_ring + (q.pruning ? 2 * depth : 0);   // candidates per climb
    const long long c0 = max(C.we + 1, C.c + sm);
    for (int jb = 0; jb < n_climbs && !A.full; jb += 32) {
        // climb j starts at c0 + j s_min (lane j - jb checks whether it was asked before)
        const int j = jb + X.lane;
        const long long cj = c0 + (long long)j * sm;
        bool fresh = false;
        if (j < n_climbs && cj + sm <= q.t_end) {
            const int sl = set_slot(cj, (int)d);
            fresh = S.set_spec[sl] != cj;
        }
        // (lanes whose starts share a slot both ask; the slot keeps one of them)
        const unsigned fm0 = __ballot_sync(kFull, fresh);
        if (fresh) S.set_spec[set_slot(cj, (int)d)] = cj;
        __syncwarp();
        const unsigned fm = fm0;
        const int total = __popc(fm) * per;
        for (int base = 0; base < total && !A.full; base += 32) {
            const int idx = base + X.lane;
            bool ok = false;
            long long ts = 0, te = 0;
            if (idx < total) {
                const int kc = idx / per, t0 = idx % per;
                const int src = nth_set_bit(fm, kc);
                const long long cs = c0 + (long long)(jb + src) * sm, ce = cs + sm - 1;
                if (t0 == 0) {
                    ts = cs;
                    te = ce;
                    ok = cs >= q.t_begin && ce <= q.t_end - 1;
                } else if (t0 < 1 + n_ring) {
                    int t = t0 - 1, r = 1;
                    while (t >= 8 * r) {
                        t -= 8 * r;
                        ++r;
                    }
                    int a, b;
                    perim(r, t, &a, &b);
                    ts = cs + a * d;
                    te = ce + b * d;
                    const long long mm = te - ts + 1;
                    ok = mm >= q.s_min && mm <= q.s_max && ts >= q.t_begin && te <= q.t_end - 1 &&
                         ts > C.last_end;
                } else {
                    const int t = t0 - 1 - n_ring;
                    const int r = 1 + t / 2, sd = t & 1;
                    const long long span = (long long)r * d;
                    if (span >= q.k + 1) {
                        if (sd == 0) {
                            ts = cs - span;
                            te = cs - 1;
                            ok = ts >= q.t_begin && ts > C.last_end;
                        } else {
                            ts = ce + 1;
                            te = ce + span;
                            ok = te <= q.t_end - 1;
                        }
                    }
                }
            }
            ask_batch(X, A, ok, ts, (int)(te - ts + 1), -1);
        }
    }
}

// Extension windows of the window ends up to kExtMoves deltas away from the current ones
// (the noise test after a move needs them): lanes 0 .. 2 kExtMoves hold one left end
// ws + a delta and one right end we + a delta each; the (end, r) candidates of the ends not
// asked before are spread over the lanes.
__device__ void spec_ext_moves(Ctx &X, Asker &A, const Climb &C) {
    const DevBuQuery &q = X.q;
    Shared &S = X.S;
    if (!q.pruning || A.full) return;
    const long long d = q.delta;
    const int R = q.t_max_idle + 1;
    const bool lane_ok = X.lane <= 2 * kExtMoves;
    const long long a = X.lane - kExtMoves;
    const long long pl = C.ws + a * d, pr = C.we + a * d;
    bool fl = false, fr = false;
    if (lane_ok) {   // distinct lanes hold distinct positions, in distinct slots
        const int sl = set_slot(pl, (int)d), sr = set_slot(pr, (int)d);
        fl = S.set_left[sl] != pl;
        fr = S.set_right[sr] != pr;
        if (fl) S.set_left[sl] = pl;
        if (fr) S.set_right[sr] = pr;
    }
    __syncwarp();
    const unsigned ml = __ballot_sync(kFull, fl), mr = __ballot_sync(kFull, fr);
    const int nl = __popc(ml), total = (nl + __popc(mr)) * R;
    for (int base = 0; base < total && !A.full; base += 32) {
        const int idx = base + X.lane;
        bool ok = false;
        long long ts = 0, te = 0;
        if (idx < total) {
            const int kpos = idx / R, r = idx % R + 1;
            const bool left = kpos < nl;
            const int src = left ? nth_set_bit(ml, kpos) : nth_set_bit(mr, kpos - nl);
            const long long span = (long long)r * d;
            if (span >= q.k + 1) {
                if (left) {
                    const long long p = C.ws + (long long)(src - kExtMoves) * d;
                    ts = p - span;
                    te = p - 1;
                    ok = ts >= q.t_begin && ts > C.last_end && p <= q.t_end;
                } else {
                    const long long p = C.we + (long long)(src - kExtMoves) * d;
                    ts = p + 1;
                    te = p + span;
                    ok = ts >= q.t_begin && ts > C.last_end && te <= q.t_end - 1;
                }
            }
        }
        ask_batch(X, A, ok, ts, (int)(te - ts + 1), -1);
    }
}

// ---------------------------------------------------------------------------------------
// Deciding (warp 0, all lanes in step).
// ---------------------------------------------------------------------------------------
struct Found {
    isycos_result_window *out;
    long long cap;
};

__device__ __forceinline__ void count_eval(Ctx &X, long long m, long long *evals) {
    *evals += 1;
    if (X.lane == 0) atomicAdd(&X.S.evals_by[size_bucket_d((int)m)], 1ull);
}

__device__ void end_climb(Ctx &X, Climb &C, long long *n_found, const Found &F) {
    const DevBuQuery &q = X.q;
    if (C.Iw >= q.sigma) {
        if (X.lane == 0 && *n_found < F.cap)   // (its MI is evaluated when the query ends)
            F.out[*n_found] = isycos_result_window{C.ws, C.we, C.Iw, 0.0};
        *n_found += 1;
        C.last_end = C.we;
    }
    C.c = max(C.we + 1, C.c + (long long)q.s_min);
    C.climb += 1;
    C.phase = kPhStart;
}

__device__ void begin_climb(Ctx &X, Climb &C, double sc, long long *evals, long long *n_found,
                            const Found &F) {
    const DevBuQuery &q = X.q;
    C.Iw = sc;
    count_eval(X, C.we - C.ws + 1, evals);
    for (int i = X.lane; i < q.h; i += 32) X.S.L[i] = sc;
    __syncwarp();
    C.t_idle = 0;
    C.step = 0;
    C.run0 = C.run1 = 0;
    C.drop0 = C.drop1 = 0;
    if (C.t_idle <= q.t_max_idle && C.step < (unsigned long long)q.max_steps) C.phase = kPhClimb;
    else end_climb(X, C, n_found, F);
}

// One LAHC step on ring N_r (Algorithm 2 with the Sec. 6.3 test).  Returns false, with
// nothing changed, when a score it needs is not at hand.
__device__ bool decide(Ctx &X, Climb &C, const StepKey &K, long long *evals, long long *n_found,
                       const Found &F) {
    const DevBuQuery &q = X.q;
    Shared &S = X.S;
    const int r = C.t_idle + 1;
    const bool sb = K.valid && K.phase == kPhClimb && K.r == r && K.ws == C.ws && K.we == C.we &&
                    K.d0 == C.drop0 && K.d1 == C.drop1;
    const int n = 8 * r;
    bool miss = false, have = false;
    double bsc = 0.0;
    int bidx = 0x7fffffff, n_read = 0;
    double pure_sc0 = 0.0, pure_sc1 = 0.0;
    bool pure0 = false, pure1 = false;
    for (int base = 0; base < n; base += 32) {
        const int idx = base + X.lane;
        if (idx < n) {
            int a, b;
            perim(r, idx, &a, &b);
            long long ts, te;
            if (keep(q, C, a, b, r, C.drop0, C.drop1, &ts, &te)) {
                double sc;
                bool got;
                if (sb) {
                    got = S.st_have[idx] != 0;
                    sc = S.st_score[idx];
                } else {
                    got = cache_get(S, ts, (int)(te - ts + 1), &sc);
                }
                if (!got) {
                    miss = true;
                } else {
                    ++n_read;
                    if (!have || sc > bsc) {   // this lane's cells come in enumeration order
                        have = true;
                        bsc = sc;
                        bidx = idx;
                    }
                    if (a == -r && b == 0) {
                        pure0 = true;
                        pure_sc0 = sc;
                    }
                    if (a == 0 && b == r) {
                        pure1 = true;
                        pure_sc1 = sc;
                    }
                }
            }
        }
    }
    if (__any_sync(kFull, miss)) return false;
    // the first maximum over the ring: larger score, then smaller enumeration index
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double osc = __shfl_xor_sync(kFull, bsc, o);
        const int oidx = __shfl_xor_sync(kFull, bidx, o);
        const bool ohave = __shfl_xor_sync(kFull, have, o);
        if (ohave && (!have || osc > bsc || (osc == bsc && oidx < bidx))) {
            have = true;
            bsc = osc;
            bidx = oidx;
        }
    }
    const int own0 = r & 31, own1 = (4 * r) & 31;   // lanes of cells (-r, 0) and (0, r)
    pure0 = __shfl_sync(kFull, pure0, own0);
    pure_sc0 = __shfl_sync(kFull, pure_sc0, own0);
    pure1 = __shfl_sync(kFull, pure1, own1);
    pure_sc1 = __shfl_sync(kFull, pure_sc1, own1);
    // the noise test's extension windows (Def. 6.2): the r delta points added on that side
    const bool test = q.pruning && (long long)r * q.delta >= q.k + 1;
    const long long span = (long long)r * q.delta;
    double ext0 = 0.0, ext1 = 0.0;
    if (test) {
        if (pure0) {
            const bool got = sb ? S.st_have[n] != 0 : cache_get(S, C.ws - span, (int)span, &ext0);
            if (sb) ext0 = S.st_score[n];
            if (!got) return false;
        }
        if (pure1) {
            const bool got = sb ? S.st_have[n + 1] != 0 : cache_get(S, C.we + 1, (int)span, &ext1);
            if (sb) ext1 = S.st_score[n + 1];
            if (!got) return false;
        }
    }
    // every score is at hand: the step
    for (int base = 0; base < n; base += 32) {   // evaluation counts by window size
        const int idx = base + X.lane;
        if (idx < n) {
            int a, b;
            perim(r, idx, &a, &b);
            long long ts, te;
            if (keep(q, C, a, b, r, C.drop0, C.drop1, &ts, &te))
                atomicAdd(&S.evals_by[size_bucket_d((int)(te - ts + 1))], 1ull);
        }
    }
    int tot = n_read;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(kFull, tot, o);
    *evals += tot;
    if (q.pruning) {
        for (int sd = 0; sd < 2; ++sd) {
            const bool pure = sd == 0 ? pure0 : pure1;
            if (!pure) continue;
            bool noise = false;
            if (test) {
                count_eval(X, span, evals);
                const double e = sd == 0 ? ext0 : ext1, ps = sd == 0 ? pure_sc0 : pure_sc1;
                noise = (C.Iw > 0.0) && (e < q.tau) && (ps < C.Iw);
            }
            int &run = sd == 0 ? C.run0 : C.run1;
            run = noise ? run + 1 : 0;
            if (run >= q.p) (sd == 0 ? C.drop0 : C.drop1) = 1;
        }
    }
    const int v = (int)(splitmix64_at(q.seed, (C.climb << 32) + C.step + 1) % (unsigned long long)q.h);
    const double Lv = S.L[v];
    if (have && (bsc > Lv || bsc > C.Iw)) {
        int a, b;
        perim(r, bidx, &a, &b);
        C.ws += (long long)a * q.delta;
        C.we += (long long)b * q.delta;
        C.Iw = bsc;
        C.t_idle = 0;
    } else {
        C.t_idle += 1;
    }
    __syncwarp();
    if (C.Iw > Lv && X.lane == 0) S.L[v] = C.Iw;
    __syncwarp();
    C.step += 1;
    if (!(C.t_idle <= q.t_max_idle && C.step < (unsigned long long)q.max_steps)) end_climb(X, C, n_found, F);
    return true;
}

// Replay decisions until a score is missing or the query is done.
__device__ void decide_loop(Ctx &X, Climb &C, const StepKey &K, long long *evals,
                            long long *n_found, const Found &F) {
    const DevBuQuery &q = X.q;
    Shared &S = X.S;
    for (;;) {
        if (C.phase == kPhDone) return;
        if (C.phase == kPhStart) {
            if (C.c + q.s_min > q.t_end) {
                C.phase = kPhDone;
                return;
            }
            C.ws = C.c;
            C.we = C.c + q.s_min - 1;
            double sc;
            bool got;
            if (K.valid && K.phase == kPhStart && K.ws == C.ws) {
                got = S.st_have[0] != 0;
                sc = S.st_score[0];
            } else {
                got = cache_get(S, C.ws, q.s_min, &sc);
            }
            if (!__all_sync(kFull, got)) return;
            begin_climb(X, C, sc, evals, n_found, F);
            continue;
        }
        if (!decide(X, C, K, evals, n_found, F)) return;
    }
}

// The list for the next round: the needed windows first, then speculation.  Returns the
// list's length; l_ubase[0 .. n] holds the work units' prefix.
__device__ int ask(Ctx &X, Climb &C, StepKey &K, int spec_climbs, long long *lo, long long *hi) {
    const DevBuQuery &q = X.q;
    Shared &S = X.S;
    Asker A{0, false, LLONG_MAX, LLONG_MIN};
    K.valid = 1;
    K.phase = C.phase;
    K.ws = C.ws;
    K.we = C.we;
    K.d0 = C.drop0;
    K.d1 = C.drop1;
    if (C.phase == kPhStart) {
        K.r = 0;
        if (X.lane == 0) S.st_have[0] = 0;
        __syncwarp();
        ask_batch(X, A, X.lane == 0, C.ws, q.s_min, 0);
        const int depth = min(q.t_max_idle + 1, spec_depth(q.s_min));
        for (int rr = 1; rr <= depth && !A.full; ++rr) ask_ring(X, A, C, rr, 0, 0, false);
    } else {
        const int r = C.t_idle + 1;
        K.r = r;
        for (int i = X.lane; i < 8 * r + 2; i += 32) S.st_have[i] = 0;
        __syncwarp();
        ask_ring(X, A, C, r, C.drop0, C.drop1, true);
        int r_last = C.t_idle >= 1 ? q.t_max_idle + 1 : r;
        r_last = max(r_last, min(q.t_max_idle + 1, spec_depth(C.we - C.ws + 1)));
        for (int rr = r + 1; rr <= r_last && !A.full; ++rr) ask_ring(X, A, C, rr, C.drop0, C.drop1, false);
    }
    spec_next_climbs(X, A, C, spec_climbs);
    spec_ext_moves(X, A, C);
    // work units: one per window of up to 32 points, else one per 64 points
    int carry = 0;
    for (int base = 0; base < A.n; base += 32) {
        const int e = base + X.lane;
        const int m = e < A.n ? S.l_m[e] : 0;
        const int u = m == 0 ? 0 : (m <= 32 ? 1 : (m + 63) / 64);
        int inc = u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, inc, o);
            if (X.lane >= o) inc += t;
        }
        if (e < A.n) S.l_ubase[e] = carry + inc - u;
        carry += __shfl_sync(kFull, inc, 31);
    }
    if (X.lane == 0) S.l_ubase[A.n] = carry;
    __syncwarp();
    long long l = A.lo, h = A.hi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l = min(l, __shfl_xor_sync(kFull, l, o));
        h = max(h, __shfl_xor_sync(kFull, h, o));
    }
    *lo = l;
    *hi = h;
    return A.n;
}

// ---------------------------------------------------------------------------------------
// The kernel.
// ---------------------------------------------------------------------------------------

// Evaluate the listed windows (entries 0 .. n - 1, nu work units) with all warps: a unit is a
// window of up to 32 points or 64 points of a larger one; its sums go to the window's
// accumulators.  Windows inside the shared series tile read it; others read global memory.
template <int K1>
__device__ void eval_units(Shared &S, const DevBuQuery &q, const BuLaunch &a, int n, int nu,
                           int *ctr, int warp, int lane) {
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(ctr, 1);
        u = __shfl_sync(kFull, u, 0);
        if (u >= nu) break;
        int lo = 0, hi = n - 1;   // the last entry whose first unit is <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (S.l_ubase[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        const int e = lo;
        const int m = S.l_m[e];
        const int blk = u - S.l_ubase[e];
        const long long ts = S.l_start[e];
        long long lp = 0, ll = 0;
        if (ts >= S.tile_lo && ts + m <= S.tile_hi) {
            const float2 *s = S.tile + (ts - S.tile_lo);
            if (m <= 32)
                ksg_block<K1, 1>(s, m, 0, lane, a.psi_fx, a.log_fx, lp, ll, nullptr, nullptr, nullptr, q.est);
            else
                ksg_block<K1, 2>(s, m, blk * 64, lane, a.psi_fx, a.log_fx, lp, ll, nullptr, nullptr,
                                 nullptr, q.est);
        } else {
            const PairSrc src{q.x + ts, q.y + ts};
            if (m <= 32)
                ksg_block<K1, 1, PairSrc>(src, m, 0, lane, a.psi_fx, a.log_fx, lp, ll, nullptr, nullptr,
                                          nullptr, q.est);
            else
                ksg_block<K1, 2, PairSrc>(src, m, blk * 64, lane, a.psi_fx, a.log_fx, lp, ll, nullptr,
                                          nullptr, nullptr, q.est);
        }
        lp = warp_sum64(lp);
        ll = warp_sum64(ll);
        if (lane == 0) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&S.acc_psi[e]), (unsigned long long)lp);
            atomicAdd(reinterpret_cast<unsigned long long *>(&S.acc_log[e]), (unsigned long long)ll);
        }
    }
}

// Load the series tile so that it holds [lo, hi) if that range fits (all threads).
__device__ void load_tile(Shared &S, const DevBuQuery &q, long long lo, long long hi) {
    if (lo >= S.tile_lo && hi <= S.tile_hi) return;   // (uniform: shared values)
    __syncthreads();
    if (hi - lo > kBuTile) return;   // does not fit: those windows read global memory
    // room behind the range (the cursor moves forward)
    long long base = max((long long)q.t_begin, lo - 256);
    if (base + kBuTile > q.t_end) base = max((long long)q.t_begin, (long long)q.t_end - kBuTile);
    const long long top = min((long long)q.t_end, base + kBuTile);
    stage_pair(S.tile, q.x + base, q.y + base, (int)(top - base), threadIdx.x, kNT);
    __syncthreads();
    if (threadIdx.x == 0) {
        S.tile_lo = base;
        S.tile_hi = top;
    }
    __syncthreads();
}

template <int K1>
__global__ void __launch_bounds__(kNT, 1) bu_climb_kernel(BuLaunch a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shared &S = *reinterpret_cast<Shared *>(smem_raw);
    __shared__ DevBuQuery q;
    __shared__ Climb Cs;
    __shared__ StepKey Ks;
    __shared__ int s_query, s_n, s_units, s_ctr, s_stop;
    __shared__ long long s_evals, s_found, s_rounds, s_lo, s_hi;
    __shared__ unsigned long long s_deadline;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        unsigned long long now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
        s_deadline = a.limit_ns ? now + a.limit_ns : 0ull;
    }
    for (;;) {
        if (threadIdx.x == 0) s_query = atomicAdd(a.queue, 1);
        __syncthreads();
        const int qi = s_query;
        if (qi >= a.n_q) break;
        if (threadIdx.x == 0) {
            q = a.q[qi];
            Cs.c = q.t_begin;
            Cs.last_end = q.t_begin - 1;
            Cs.ws = Cs.we = 0;
            Cs.Iw = 0.0;
            Cs.step = Cs.climb = 0;
            Cs.phase = kPhStart;
            Cs.t_idle = Cs.run0 = Cs.run1 = Cs.drop0 = Cs.drop1 = 0;
            Ks.valid = 0;
            s_evals = s_found = s_rounds = 0;
            s_stop = 0;
            S.pairs = 0;
            S.units = 0;
            S.work_bf = 0;
            S.tile_lo = 0;
            S.tile_hi = 0;
        }
        for (int i = threadIdx.x; i < kBuCacheSlots; i += kNT) S.c_key[i] = kEmpty;
        for (int i = threadIdx.x; i < kSetSlots; i += kNT) {
            S.set_spec[i] = -1;
            S.set_left[i] = -1;
            S.set_right[i] = -1;
        }
        if (threadIdx.x < 15) {
            S.evals_by[threadIdx.x] = 0;
            S.win_by[threadIdx.x] = 0;
        }
        __syncthreads();
        const Found F{a.found + (size_t)qi * (size_t)a.cap, a.cap};
        const double inv_k = q.est ? 0.0 : __ddiv_rn(1.0, (double)q.k);
        long long cyc[3] = {0, 0, 0};   // (thread 0) decide + ask, evaluate, finish
        for (;;) {
            long long t_a = clock64();
            // decide + ask (warp 0)
            if (warp == 0) {
                Ctx X{S, q, lane};
                Climb C = Cs;
                StepKey K = Ks;
                long long evals = s_evals, n_found = s_found;
                bool stop = false;
                if (s_deadline) {
                    unsigned long long now;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
                    stop = __shfl_sync(kFull, now, 0) > s_deadline;
                }
                int n = 0;
                long long lo = 0, hi = 0;
                if (!stop) {
                    decide_loop(X, C, K, &evals, &n_found, F);
                    if (C.phase != kPhDone) n = ask(X, C, K, a.spec_climbs, &lo, &hi);
                }
                if (lane == 0) {
                    Cs = C;
                    Ks = K;
                    s_evals = evals;
                    s_found = n_found;
                    s_n = n;
                    s_units = n > 0 ? S.l_ubase[n] : 0;
                    s_lo = lo;
                    s_hi = hi;
                    s_ctr = 0;
                    s_stop = stop ? 1 : (C.phase == kPhDone ? 2 : 0);
                    s_rounds += 1;
                }
            }
            __syncthreads();
            long long t_b = clock64();
            cyc[0] += t_b - t_a;
            if (s_stop) break;
            const int n = s_n, nu = s_units;
            if (nu > 0) {
                load_tile(S, q, s_lo, s_hi);
                eval_units<K1>(S, q, a, n, nu, &s_ctr, warp, lane);
                __syncthreads();
                const long long t_c = clock64();
                cyc[1] += t_c - t_b;
                t_b = t_c;
                // finish: the binary64 scalars, into the cache slot and the step buffer
                for (int e = threadIdx.x; e < n; e += kNT) {
                    const int m = S.l_m[e];
                    if (m == 0) continue;
                    isycos_mi_out o;
                    write_result(&o, q.k, m, S.acc_psi[e], S.acc_log[e], a.psi_fx, a.log_fx, inv_k);
                    const double sc = q.score_kind == 1 ? o.mi : o.nmi;
                    const int slot = S.l_slot[e];
                    if (slot >= 0) {
                        S.c_score[slot] = sc;
                        S.c_key[slot] = wkey(S.l_start[e], m);
                    }
                    const int st = S.l_step[e];
                    if (st >= 0) {
                        S.st_score[st] = sc;
                        S.st_have[st] = 1;
                    }
                    atomicAdd(&S.win_by[size_bucket_d(m)], 1ull);
                    atomicAdd(&S.pairs, (unsigned long long)m * (unsigned long long)(m - 1));
                    atomicAdd(&S.work_bf, (unsigned long long)m * (unsigned long long)m);
                }
                if (threadIdx.x == 0) S.units += (unsigned long long)nu;
                __syncthreads();
                cyc[2] += clock64() - t_b;
            }
        }
        // The found windows' MI (the search compared their scores; the result reports both).
        if (s_stop == 2) {
            const long long nf = min(s_found, (long long)a.cap);
            for (long long f0 = 0; f0 < nf; f0 += kRoundCap) {
                const int n = (int)min((long long)kRoundCap, nf - f0);
                if (warp == 0) {
                    int carry = 0;
                    for (int base = 0; base < n; base += 32) {
                        const int e = base + lane;
                        int u = 0;
                        if (e < n) {
                            const isycos_result_window w = F.out[f0 + e];
                            const int m = (int)(w.t_e - w.t_s + 1);
                            S.l_start[e] = w.t_s;
                            S.l_m[e] = m;
                            S.acc_psi[e] = 0;
                            S.acc_log[e] = 0;
                            u = m <= 32 ? 1 : (m + 63) / 64;
                        }
                        int inc = u;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int t = __shfl_up_sync(kFull, inc, o);
                            if (lane >= o) inc += t;
                        }
                        if (e < n) S.l_ubase[e] = carry + inc - u;
                        carry += __shfl_sync(kFull, inc, 31);
                    }
                    if (lane == 0) {
                        S.l_ubase[n] = carry;
                        s_units = carry;
                        s_ctr = 0;
                    }
                }
                __syncthreads();
                eval_units<K1>(S, q, a, n, s_units, &s_ctr, warp, lane);
                __syncthreads();
                for (int e = threadIdx.x; e < n; e += kNT) {
                    isycos_mi_out o;
                    write_result(&o, q.k, S.l_m[e], S.acc_psi[e], S.acc_log[e], a.psi_fx, a.log_fx, inv_k);
                    F.out[f0 + e].mi = o.mi;
                }
                __syncthreads();
            }
        }
        // the query's results
        if (threadIdx.x == 0) {
            DevBuResult &R = a.res[qi];
            R.n_found = s_found;
            R.evals = s_evals;
            long long w = 0;
            for (int b = 0; b < 15; ++b) {
                R.evals_by_size[b] = (long long)S.evals_by[b];
                R.windows_by_size[b] = (long long)S.win_by[b];
                w += (long long)S.win_by[b];
            }
            R.windows = w;
            R.pairs = (long long)S.pairs;
            R.rounds = s_rounds;
            R.units = (long long)S.units;
            R.work_bf = (long long)S.work_bf;
            for (int j = 0; j < 3; ++j) R.cycles[j] = cyc[j];
            R.status = s_stop == 1 ? 1 : 0;
            R.pad = 0;
        }
        __syncthreads();
    }
}

template <int K1>
cudaError_t prep_one(size_t smem, int *per_sm) {
    cudaError_t e = cudaFuncSetAttribute(bu_climb_kernel<K1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(bu_climb_kernel<K1>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, bu_climb_kernel<K1>, kNT, smem);
}

}  // namespace

size_t bu_device_smem() { return sizeof(Shared); }

cudaError_t bu_device_prepare(int k, int *blocks_per_sm) {
    const size_t smem = sizeof(Shared);
    switch (k) {
        case 1: return prep_one<2>(smem, blocks_per_sm);
        case 2: return prep_one<3>(smem, blocks_per_sm);
        case 3: return prep_one<4>(smem, blocks_per_sm);
        case 4: return prep_one<5>(smem, blocks_per_sm);
        case 5: return prep_one<6>(smem, blocks_per_sm);
        case 6: return prep_one<7>(smem, blocks_per_sm);
        case 7: return prep_one<8>(smem, blocks_per_sm);
        case 8: return prep_one<9>(smem, blocks_per_sm);
    }
    return cudaErrorInvalidValue;
}

cudaError_t bu_device_launch(const BuLaunch &a, int k, int grid, cudaStream_t st) {
    const size_t smem = sizeof(Shared);
    switch (k) {
        case 1: bu_climb_kernel<2><<<grid, kNT, smem, st>>>(a); break;
        case 2: bu_climb_kernel<3><<<grid, kNT, smem, st>>>(a); break;
        case 3: bu_climb_kernel<4><<<grid, kNT, smem, st>>>(a); break;
        case 4: bu_climb_kernel<5><<<grid, kNT, smem, st>>>(a); break;
        case 5: bu_climb_kernel<6><<<grid, kNT, smem, st>>>(a); break;
        case 6: bu_climb_kernel<7><<<grid, kNT, smem, st>>>(a); break;
        case 7: bu_climb_kernel<8><<<grid, kNT, smem, st>>>(a); break;
        case 8: bu_climb_kernel<9><<<grid, kNT, smem, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace isy
