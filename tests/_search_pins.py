"""Hand-traced pins of the oracle's searches (SYCOS_TD, Algorithm 1; SYCOS_BU, Algorithm 2;
the noise pruning of Sec. 6) on mocked score tables.

The paper prints no numbers for its searches, so each pin fixes one reading of the text by
a trace worked out by hand in its comment: which windows are scored, in which order, and
what comes out.  Each ``pin_*`` raises AssertionError when the oracle disagrees:

- ``pin_td_layers``: layer sizes s_max, s_max / 2, ..., the step delta = max(k + 1, s_w / 4),
  uncorrelated partitions and the literal partition end of Algorithm 1;
- ``pin_td_tail_not_scored``: a layer stops at the last grid window that fits its partition;
  a window ending at the partition end off that grid is never scored;
- ``pin_td_size_floor``: reduce(s_w) stops at s_min (a layer of s_min points, not s_w / 2);
- ``pin_td_noise_skip``: w_o = [t_s1, t_e0], w_delta = [t_e0 + 1, t_e1] and the skip after p
  detections (Def. 6.2 in SYCOS_TD); no test when w_delta has fewer than k + 1 points;
- ``pin_td_noise_run_resets``: only consecutive detections count toward p;
- ``pin_td_noise_needs_positive_overlap``: Def. 6.2 only holds when I_{w_o} > 0;
- ``pin_bu_single_peak``: a climb over a single-peak table;
- ``pin_bu_plateau``: the ring N_1 (not the whole square), strict acceptance of Algorithm 2,
  and the next climb starting at max(t_e + 1, c + s_min);
- ``pin_bu_first_maximum``: the first maximum of a ring, a outer and b inner, wins;
- ``pin_bu_restart_after_left_move``: a climb that ends left of its start does not move the
  next start back;
- ``pin_bu_noise_drops_one_side``: a noisy extension drops only the neighbours that extend
  that side;
- ``pin_bu_noise_run_resets``: each side's detections count toward p only while consecutive;
- ``pin_bu_late_acceptance``: the late-acceptance history of Algorithm 2 (h entries, the
  step's index drawn from SplitMix64, the same entry compared and then updated);
- ``pin_chunks_overlap``: the chunks of Algorithm 4 reach s_max points back, and a window
  found by two chunks is returned twice;
- ``pin_selection_sampling``: which partitions Algorithm 3 samples for a seed, M and m (the
  partial Fisher-Yates shuffle over SplitMix64 outputs 1 .. m), traced by hand from the
  generator's published reference outputs, and that the sample decides the selection;
- ``pin_selection_runtime``: Algorithm 3's runtime of a search is the pair comparisons of
  the windows it scores, averaged over the sampled partitions, and its window counts split
  at rho * s_max.

tests/test_oracle_mutations.py runs them against planted mistakes of the oracle's searches.
"""
from __future__ import annotations

from oracle import oracle as O
from paper_2204_09131_gb300 import synth


def _score(table, log=None, default=0.0):
    """A window score from a dict {(t_s, t_e): score} or a function (t_s, t_e) -> score; every
    call is appended to ``log``."""
    def score(ts, te):
        if log is not None:
            log.append((ts, te))
        v = table(ts, te) if callable(table) else table.get((ts, te), default)
        return v, v
    return score


def _spans(wins):
    return [(a, b) for a, b, _, _ in wins]


# Score tables of the traces below ((t_s, t_e) -> score; unlisted windows score 0).
_NOISE_SKIP = {(0, 15): 0.2, (4, 19): 0.1, (4, 15): 0.3, (16, 19): 0.05,
               (8, 23): 0.1, (8, 19): 0.3, (20, 23): 0.05, (24, 39): 0.6}
_NOISE_RUN = {(0, 15): 0.2, (4, 19): 0.1, (4, 15): 0.3, (16, 19): 0.05,
              (8, 23): 0.1, (8, 19): 0.3, (20, 23): 0.5,
              (12, 27): 0.1, (12, 23): 0.3, (24, 27): 0.05}
_NOISE_OVERLAP_ZERO = {(0, 15): 0.2, (4, 19): -0.1, (4, 15): 0.0, (16, 19): 0.05}
_LATE = {(4, 11): 0.5, (4, 15): 0.3, (4, 19): 0.9, (0, 7): 0.1}


def pin_td_layers():
    # Correlated iff the window lies inside [20, 40).  Range [0, 48), s_max 16, s_min 8,
    # k = 1 so delta = max(k+1, s_w/4) = 4 then 2.
    # Layer 16: starts 0,4,8,12,16 uncorrelated, [20,35] correlated, next start 36 does
    # not fit.  Layer 8: partitions [0,19] (starts 0..12 step 2) and [36,47] (36,38,40).
    log = []
    score = _score(lambda ts, te: 1.0 if ts >= 20 and te < 40 else 0.0, log)
    wins, n = O.search_td(score, t_begin=0, t_end=48, k=1, s_min=8, s_max=16, sigma=0.5)
    assert _spans(wins) == [(20, 35)], wins
    assert n == 16 and len(log) == 16, (n, log)
    assert log[:6] == [(t, t + 15) for t in (0, 4, 8, 12, 16, 20)], log
    assert log[6:] == [(t, t + 7) for t in range(0, 13, 2)] + [(36, 43), (38, 45), (40, 47)], log


def pin_td_tail_not_scored():
    # One layer of 16 points (s_min = s_max = 16), k = 1, delta 4, range [0, 50).  The scan
    # takes starts 0, 4, ..., 32; start 36 would end at 51 > 49, so the layer stops (Alg. 1
    # loops while the window ends inside its partition).  The window [34, 49] that would end
    # exactly at the partition end is not on that grid and is never scored, although the
    # table makes it the only correlated window.
    log = []
    wins, n = O.search_td(_score(lambda ts, te: 0.9 if ts == 34 and te == 49 else 0.0, log),
                          t_begin=0, t_end=50, k=1, s_min=16, s_max=16, sigma=0.5)
    assert wins == [] and n == 9, (wins, n)
    assert log == [(t, t + 15) for t in range(0, 33, 4)], log


def pin_td_size_floor():
    # Nothing is correlated on [0, 48); s_max 24, s_min 16, k = 1.  Layer 24: delta = 6,
    # starts 0..24.  reduce(24) = 12 is below s_min, so the second and last layer has 16
    # points: delta = 4, starts 0..32.
    log = []
    wins, n = O.search_td(_score(lambda ts, te: 0.0, log), t_begin=0, t_end=48, k=1, s_min=16,
                          s_max=24, sigma=0.5)
    assert wins == [] and n == 14, (wins, n)
    assert log == [(t, t + 23) for t in range(0, 25, 6)] + [(t, t + 15) for t in range(0, 33, 4)], log


def pin_td_noise_skip():
    # One layer of size 16, delta 4, p = 2, sigma 0.5, tau 0.1.  Windows [4,19] and
    # [8,23] are each noise w.r.t. their overlap (I_delta < tau and I_w < I_o), so after
    # the second detection the scan jumps to t_e + 1 = 24, where [24,39] is correlated.
    table = _NOISE_SKIP
    log = []
    wins, n = O.search_td(_score(table, log), t_begin=0, t_end=48, k=1, s_min=16, s_max=16,
                          delta_td=4, sigma=0.5, tau=0.1, p=2, pruning=1)
    assert _spans(wins) == [(24, 39)], wins
    assert log == [(0, 15), (4, 19), (4, 15), (16, 19), (8, 23), (8, 19), (20, 23), (24, 39)], log
    # Without pruning the scan shifts through 12, 16, 20 before reaching 24.
    log2 = []
    wins2, _ = O.search_td(_score(table, log2), t_begin=0, t_end=48, k=1, s_min=16, s_max=16,
                           delta_td=4, sigma=0.5, tau=0.1, p=2)
    assert _spans(wins2) == [(24, 39)], wins2
    assert log2 == [(t, t + 15) for t in range(0, 25, 4)], log2
    # With k = 4 the extension w_delta of 4 points is below k + 1 and is never scored: no
    # noise test runs, and the pruned scan is the unpruned one.
    log3 = []
    wins3, _ = O.search_td(_score(table, log3), t_begin=0, t_end=48, k=4, s_min=16, s_max=16,
                           delta_td=4, sigma=0.5, tau=0.1, p=2, pruning=1)
    assert _spans(wins3) == [(24, 39)], wins3
    assert log3 == [(t, t + 15) for t in range(0, 25, 4)], log3


def pin_td_noise_run_resets():
    # One layer of size 16, delta 4, p = 2, sigma 0.5, tau 0.1.  [4,19] is noise (as in
    # pin_td_noise_skip), [8,23] is not (its w_delta [20,23] scores 0.5 >= tau), [12,27] is
    # noise again: the detections are not consecutive, so the count restarts at [8,23] and
    # the scan never skips; every other window scores 0 (w_o at 0: no noise).  Starts 0..32.
    table = _NOISE_RUN
    log = []
    wins, _ = O.search_td(_score(table, log), t_begin=0, t_end=48, k=1, s_min=16, s_max=16,
                          delta_td=4, sigma=0.5, tau=0.1, p=2, pruning=1)
    assert wins == [], wins
    assert [w for w in log if w[1] - w[0] + 1 == 16] == [(t, t + 15) for t in range(0, 33, 4)], log


def pin_td_noise_needs_positive_overlap():
    # As above with p = 1, but the overlap [4,15] of the shifted window [4,19] scores 0: with
    # I_{w_o} = 0, Def. 6.2 does not hold even though I_delta = 0.05 < tau and I_w = -0.1 <
    # I_{w_o}, so the layer keeps shifting by 4 (every other window scores 0 and is never
    # noise) through the last start 32.
    table = _NOISE_OVERLAP_ZERO
    log = []
    wins, _ = O.search_td(_score(table, log), t_begin=0, t_end=48, k=1, s_min=16, s_max=16,
                          delta_td=4, sigma=0.5, tau=0.1, p=1, pruning=1)
    assert wins == [], wins
    assert [w for w in log if w[1] - w[0] + 1 == 16] == [(t, t + 15) for t in range(0, 33, 4)], log


def pin_bu_single_peak():
    # Score 1 - (|t_s - 20| + |t_e - 39|) / 100: a single peak at [20, 39].  From
    # w0 = [0, 7] the climb moves both ends by delta = 4 until t_s = 20, then the end
    # until 39, where every ring-1 neighbour is worse (T_maxIdle = 0 stops the climb).
    score = _score(lambda ts, te: 1.0 - (abs(ts - 20) + abs(te - 39)) / 100.0)
    wins, _ = O.search_bu(score, t_begin=0, t_end=100, k=1, s_min=8, s_max=40, delta_bu=4,
                          h=1, t_max_idle=0, sigma=0.9, seed=3)
    assert _spans(wins) == [(20, 39)], wins
    assert abs(wins[0][2] - 1.0) < 1e-12, wins


def pin_bu_plateau():
    # Every window scores 0.5; range [0, 24), s_min 8, s_max 16, delta 4, h = 1, T_maxIdle 0,
    # sigma 0.4.  Climb 0 from [0,7]: of ring N_1 only [0,11] (a=0, b=1) and [4,11] (a=1,
    # b=1) have 8..16 points inside the range; neither beats 0.5 strictly, so the climb ends
    # where it started and [0,7] is kept.  The next climb starts at max(7 + 1, 0 + 8) = 8:
    # its ring has [8,19] and [12,19] (a = -1 would start at 4 <= 7).  The last climb at
    # [16,23] has no neighbour inside the range.
    log = []
    wins, n = O.search_bu(_score(lambda ts, te: 0.5, log), t_begin=0, t_end=24, k=1, s_min=8,
                          s_max=16, delta_bu=4, h=1, t_max_idle=0, sigma=0.4, seed=5)
    assert _spans(wins) == [(0, 7), (8, 15), (16, 23)], wins
    assert log == [(0, 7), (0, 11), (4, 11), (8, 15), (8, 19), (12, 19), (16, 23)], log
    assert n == 7


def pin_bu_first_maximum():
    # [0,11] and [4,11] both score 0.9, every other window 0.1; range [0, 40), s_min 8,
    # s_max 16, delta 4, h = 1, T_maxIdle 0, sigma 0.5.  Ring N_1 of [0,7] lists [0,11]
    # (a = 0) before [4,11] (a = 1): the climb moves to [0,11], where [4,11] ties and is not
    # accepted.  The later climbs (starts 12, 20, 28) only see 0.1.
    table = {(0, 11): 0.9, (4, 11): 0.9}
    wins, _ = O.search_bu(_score(table, default=0.1), t_begin=0, t_end=40, k=1, s_min=8,
                          s_max=16, delta_bu=4, h=1, t_max_idle=0, sigma=0.5, seed=5)
    assert _spans(wins) == [(0, 11)], wins


def pin_bu_restart_after_left_move():
    # [6,13] scores 0.9, every other window 0.1; range [0, 24), s_min 8, s_max 16, delta 2,
    # h = 1, T_maxIdle 0, sigma 0.5.
    # Climb 0 at [0,7]: ring [0,9], [2,9]; nothing better, nothing kept; next start 8.
    # Climb 1 at [8,15]: ring (a outer, b inner) [6,13], [6,15], [6,17], [8,17], [10,17];
    # it moves left to [6,13], whose ring [4,11], [4,13], [4,15], [6,15], [8,15] is worse.
    # [6,13] is kept and the next start is max(13 + 1, 8 + 8) = 16, not 14: climb 2 at
    # [16,23] has ring [14,21], [14,23].
    log = []
    wins, _ = O.search_bu(_score({(6, 13): 0.9}, log, default=0.1), t_begin=0, t_end=24, k=1,
                          s_min=8, s_max=16, delta_bu=2, h=1, t_max_idle=0, sigma=0.5, seed=5)
    assert _spans(wins) == [(6, 13)], wins
    assert log == [(0, 7), (0, 9), (2, 9),
                   (8, 15), (6, 13), (6, 15), (6, 17), (8, 17), (10, 17),
                   (4, 11), (4, 13), (4, 15), (6, 15), (8, 15),
                   (16, 23), (14, 21), (14, 23)], log


def _noise_table(ts, te):
    # Windows of at least 8 points: 0.3 + 0.01 t_e - 0.1 |t_s - 4|, best at t_s = 4 and the
    # longest window.  Shorter windows (the extension windows of 4 points): 0 for [0,3]
    # (noise), 0.5 elsewhere.
    if te - ts + 1 < 8:
        return 0.0 if te < 4 else 0.5
    return 0.3 + 0.01 * te - 0.1 * abs(ts - 4)


def pin_bu_noise_drops_one_side():
    # Range [0, 64), k = 1, s_min 8, s_max 24, delta 4, h = 1, T_maxIdle 0, p = 1, tau 0.1,
    # sigma 0.5, pruning on.
    # [0,7] (-0.03): best of the ring is [4,11] (0.41); the right extension [8,11] scores 0.5,
    #   no noise.  Move.
    # [4,11]: the left neighbour [0,11] (0.01) with extension [0,3] (0 < tau, 0.01 < 0.41,
    #   I_w > 0) is noise: with p = 1 the left side is dropped.  Move to [4,15] (0.45).
    # [4,15] -> [4,19] (0.49) -> [4,23] (0.53) -> [4,27] (0.57, 24 points): only neighbours
    #   with a >= 0 are left, and those that extend the right end keep improving.
    # At [4,27] no neighbour is better, so [4,27] (0.57 >= sigma) is kept; the next climb
    #   starts at [28,35] and every later one scores below 0.  (Had the noise dropped both
    #   sides, the first climb would have ended at [4,15] (0.45 < sigma) and the second would
    #   have started at [16,23].)
    log = []
    wins, _ = O.search_bu(_score(_noise_table, log), t_begin=0, t_end=64, k=1, s_min=8,
                          s_max=24, delta_bu=4, h=1, t_max_idle=0, p=1, tau=0.1, sigma=0.5,
                          pruning=1, seed=5)
    assert _spans(wins) == [(4, 27)], wins
    assert abs(wins[0][2] - 0.57) < 1e-12, wins
    assert (28, 35) in log and (16, 23) not in log, log


def _history_indices(seed, h, n):
    # The history index of step s of climb 0: SplitMix64 output s + 1 of the seed, mod h
    # (the generator module's own SplitMix64, pinned to reference outputs elsewhere).
    return [int(z) % h for z in synth.splitmix64(seed, n, offset=0)]


def _shift_table(ts, te):
    # W_j = [4j, 4j + 7] scores 0.1 + 0.1 j for j = 0..5, other windows of 8+ points 0; of the
    # 4-point extension windows, [0,3] and [8,11] score 0 (noise) and the rest 0.5.
    if te - ts + 1 < 8:
        return 0.0 if (ts, te) in ((0, 3), (8, 11)) else 0.5
    if te - ts == 7 and ts % 4 == 0 and ts <= 20:
        return 0.1 + 0.1 * (ts // 4)
    return 0.0


def pin_bu_noise_run_resets():
    # Range [0, 64), k = 1, s_min 8, s_max 16, delta 4, h = 1, T_maxIdle 0, p = 2, tau 0.1,
    # sigma 0.5, pruning on.  The climb shifts right one delta per step, W_0 -> W_5: the ring of
    # W_j is W_{j-1}, [4j-4, 4j+7], [4j-4, 4j+11], [4j, 4j+11] (all 0 or lower) and W_{j+1}.
    # Left extension [4j-4, 4j-1] of W_j (its neighbour [4j-4, 4j+7] scores 0 < I_w):
    #   j = 1: [0,3] noise (count 1); j = 2: [4,7] not noise (count 0); j = 3: [8,11] noise
    #   (count 1 < p): the left side stays, and at W_4 = [16,23] the neighbour (a = -1, b = 1)
    #   [12,27] is scored.
    # Right extension [4j+8, 4j+11]: noise at j = 0 only ([8,11]), never twice in a row.
    # At W_5 nothing is better: [20,27] (0.6) is kept.
    log = []
    wins, _ = O.search_bu(_score(_shift_table, log), t_begin=0, t_end=64, k=1, s_min=8,
                          s_max=16, delta_bu=4, h=1, t_max_idle=0, p=2, tau=0.1, sigma=0.5,
                          pruning=1, seed=5)
    assert _spans(wins) == [(20, 27)], wins
    assert (12, 27) in log, log


def _late_seeds():
    # the first seeds whose first two history indices (h = 2) differ (True) and coincide (False)
    seeds = {}
    for seed in range(1, 64):
        v = _history_indices(seed, 2, 2)
        seeds.setdefault(v[0] != v[1], seed)
    assert set(seeds) == {True, False}
    return seeds


def pin_bu_late_acceptance():
    # Late acceptance (Algorithm 2 with h = 2): a neighbour is taken when it beats the
    # current window OR the history entry L[v] of this step, and L[v] is raised to the
    # current score after the step.  Range [0, 40), s_min 8, s_max 16, delta 4, T_maxIdle 0,
    # sigma 0.35.  Scores: [4,11] 0.5, [4,15] 0.3, [4,19] 0.9, [0,7] 0.1, the rest 0.05.
    # Climb 0 from [0,7] (L = [0.1, 0.1]):
    #   step 0, index v0: [4,11] (0.5) beats 0.1: move; L[v0] = 0.5.
    #   step 1, index v1: the best of the ring of [4,11] is [4,15] (0.3), worse than 0.5.
    #     v1 != v0: 0.3 > L[v1] = 0.1, so the worse window is taken; from there [4,19] (0.9)
    #     is the best of the next ring, and [4,19] is kept.
    #     v1 == v0: 0.3 < L[v0] = 0.5: the climb stops and [4,11] is kept.
    # Later climbs start at 20 or 12 and only see 0.05.
    kw = dict(t_begin=0, t_end=40, k=1, s_min=8, s_max=16, delta_bu=4, h=2, t_max_idle=0,
              sigma=0.35)
    seeds = _late_seeds()
    wins, _ = O.search_bu(_score(_LATE, default=0.05), seed=seeds[True], **kw)
    assert _spans(wins) == [(4, 19)], wins
    wins, _ = O.search_bu(_score(_LATE, default=0.05), seed=seeds[False], **kw)
    assert _spans(wins) == [(4, 11)], wins


def pin_chunks_overlap():
    # Algorithm 4 with n_p = 2 on [0, 64): L = 32, chunks [0, 32) and [32 - s_max, 64) =
    # [16, 64).  One TD layer of 16 points (s_min = s_max = 16, k = 1, delta 4); only [16,31]
    # is correlated.  Chunk 0 scores starts 0, 4, 8, 12, 16 and keeps [16,31]; chunk 1 keeps
    # [16,31] at its first start, then scores 32, 36, 40, 44, 48.  Both copies are returned
    # (11 windows scored).
    log = []
    wins, n = O.search_chunked(_score(lambda ts, te: 0.9 if (ts, te) == (16, 31) else 0.0, log),
                               None, 0, 64, mode=0, chunks=2, k=1, s_min=16, s_max=16, sigma=0.5)
    assert _spans(wins) == [(16, 31), (16, 31)], wins
    assert n == 11 and log == [(t, t + 15) for t in (0, 4, 8, 12, 16, 16, 32, 36, 40, 44, 48)], (n, log)


def pin_selection_runtime():
    # Algorithm 3 with M = m = 2 partitions of [0, 64) (both sampled), alpha 0.5, rho 0.5;
    # TD: s_min 8, s_max 16, k = 1 (deltas 4 and 2); BU: delta 4, h = 1, T_maxIdle 0.  The
    # runtime of a search is the pair comparisons m (m - 1) of the windows it scores,
    # averaged over the partitions.
    # Nothing correlated, per partition of 32 points:
    #   TD: 5 windows of 16 (starts 0..16) and 13 of 8 (starts 0..24): 5*240 + 13*56 = 1928.
    #   BU: climbs at 0, 8, 16, 24 score 3, 6, 6 and 3 windows: [0,7] + [0,11], [4,11];
    #     [8,15] + [4,11], [4,15], [4,19], [8,19], [12,19]; [16,23] + five likewise;
    #     [24,31] + [20,27], [20,31]: 244 + 672 + 672 + 244 = 1832.
    #   No window found: nscore_TD = 0.5 * 3760 / 1928, nscore_BU = 0.5 * 3760 / 1832; BU.
    kw = dict(k=1, s_min=8, s_max=16, delta_bu=4, h=1, t_max_idle=0, sigma=0.5, seed=7)
    wins, _, sel, sc = O.search_auto(_score(lambda ts, te: 0.0), None, 0, 64, partitions=2,
                                     samples=2, alpha=0.5, rho=0.5, **kw)
    assert wins == [] and sel == 1, (wins, sel)
    assert abs(sc[0] - 0.5 * 3760 / 1928) < 1e-12 and abs(sc[1] - 0.5 * 3760 / 1832) < 1e-12, sc
    # [0,15] correlated: in partition [0, 32) TD keeps it at its first window, then scores
    # [16,31] and, in layer 8, the partition [16, 31] (starts 16..24): 2*240 + 5*56 = 760,
    # one large window (16 > rho * s_max).  BU never scores [0,15] (it is not in a ring of
    # its climbs) and costs 1832 as before.  t_TD = (760 + 1928) / 2 = 1344, t_BU = 1832:
    # nscore_TD = 0.5 * 3176 / 1344 + 0.5 * 1, nscore_BU = 0.5 * 3176 / 1832 + 0; TD runs on
    # the whole range and keeps [0,15].
    wins, _, sel, sc = O.search_auto(_score(lambda ts, te: 0.9 if (ts, te) == (0, 15) else 0.0),
                                     None, 0, 64, partitions=2, samples=2, alpha=0.5, rho=0.5, **kw)
    assert _spans(wins) == [(0, 15)] and sel == 0, (wins, sel)
    assert abs(sc[0] - (0.5 * 3176 / 1344 + 0.5)) < 1e-12 and abs(sc[1] - 0.5 * 3176 / 1832) < 1e-12, sc


def pin_selection_sampling():
    # Algorithm 3's random sampling (Sec. 5.3) as read here: m of M partitions chosen by a
    # partial Fisher-Yates shuffle of 0 .. M-1 whose i-th swap (i = 0 .. m-1) takes position
    # i + (r_(i+1) mod (M - i)), r_n the n-th SplitMix64 output of the stream seed ^ 0x5E1EC7.
    # seed = 1234567 ^ 0x5E1EC7 = 5032000 makes that stream the one with state 1234567,
    # whose first outputs are Vigna's reference values r_1 = 6457827717110365317 and
    # r_2 = 3203168211198807973.  With M = 10, m = 2, by hand:
    #   r_1 mod 10 = 7 (its last digit): swap positions 0 and 7 -> partition 7 first;
    #   r_2 mod 9 = 7 (its digit sum 79 = 8 * 9 + 7): swap positions 1 and 1 + 7 = 8 ->
    #   partition 8 second.
    # On [0, 320) the partitions have L = 32 points, so the sample is [224, 256) then
    # [256, 288), each searched by SYCOS_TD and then SYCOS_BU, before the selected search
    # runs on the whole range from 0.
    seed = 1234567 ^ 0x5E1EC7
    assert seed == 5032000
    kw = dict(k=1, s_min=8, s_max=16, delta_bu=4, h=1, t_max_idle=0, sigma=0.5, seed=seed)
    log = []
    O.search_auto(_score(lambda ts, te: 0.0, log), None, 0, 320, partitions=10, samples=2,
                  alpha=0.5, rho=0.5, **kw)
    parts = []
    for ts, te in log:
        q = ts // 32
        if not parts or parts[-1] != q:
            parts.append(q)
    assert parts[:3] == [7, 8, 0], parts[:3]
    # the sampled searches stay inside their partitions: TD then BU on [224, 256), then on
    # [256, 288)
    n_sample = next(i for i, (ts, _) in enumerate(log) if ts < 224)
    assert n_sample > 0 and all(224 <= ts and te < 32 * (ts // 32 + 1) for ts, te in log[:n_sample])
    # The sample decides the choice: [224, 239] (16 points, large: > rho s_max = 8) is the
    # only correlated window.  TD finds it in partition 7, BU (windows of 8..12 points
    # around its climbs, all scoring 0) does not, so nl_TD = 1, ns_BU = 0 and nscore_TD =
    # 0.5 / rt_TD + 0.5 > nscore_BU = 0.5 / rt_BU (both rt near 1/2): SYCOS_TD runs on the
    # whole range and returns the window.  A sample without partition 7 finds nothing, and
    # the cheaper BU would run and miss it.
    wins, _, sel, _ = O.search_auto(_score(lambda ts, te: 0.9 if (ts, te) == (224, 239) else 0.0),
                                    None, 0, 320, partitions=10, samples=2, alpha=0.5, rho=0.5, **kw)
    assert sel == 0 and _spans(wins) == [(224, 239)], (sel, wins)


SEARCH_PINS = [pin_td_layers, pin_td_tail_not_scored, pin_selection_sampling, pin_td_size_floor,
               pin_td_noise_skip, pin_td_noise_run_resets,
               pin_td_noise_needs_positive_overlap, pin_bu_single_peak, pin_bu_plateau,
               pin_bu_first_maximum, pin_bu_restart_after_left_move, pin_bu_noise_drops_one_side,
               pin_bu_noise_run_resets, pin_bu_late_acceptance, pin_chunks_overlap,
               pin_selection_runtime]


def _table(t, default=0.0):
    return lambda ts, te: t.get((ts, te), default)


def machine_cases():
    """The traces above as (name, search, score, t_end, parameters, windows) for other
    implementations of the searches: ``search`` is "td", "bu", "chunked" (parameters carry
    mode and chunks) or "auto" (partitions, samples, alpha, rho); ``score`` maps (t_s, t_e)
    to the window's score on [0, t_end); ``windows`` is the hand-traced result."""
    td1 = dict(k=1, s_min=16, s_max=16, delta_td=4, sigma=0.5, tau=0.1, pruning=1)
    bu1 = dict(k=1, s_min=8, s_max=16, delta_bu=4, h=1, t_max_idle=0, seed=5)
    seeds = _late_seeds()
    late = dict(k=1, s_min=8, s_max=16, delta_bu=4, h=2, t_max_idle=0, sigma=0.35)
    sel = dict(k=1, s_min=8, s_max=16, delta_bu=4, h=1, t_max_idle=0, sigma=0.5, seed=7,
               partitions=2, samples=2, alpha=0.5, rho=0.5)
    return [
        ("td_layers", "td", lambda ts, te: 1.0 if ts >= 20 and te < 40 else 0.0, 48,
         dict(k=1, s_min=8, s_max=16, sigma=0.5), [(20, 35)]),
        ("td_size_floor", "td", lambda ts, te: 0.0, 48, dict(k=1, s_min=16, s_max=24, sigma=0.5), []),
        ("td_noise_skip", "td", _table(_NOISE_SKIP), 48, dict(td1, p=2), [(24, 39)]),
        ("td_noise_tiny", "td", _table(_NOISE_SKIP), 48, dict(td1, p=2, k=4), [(24, 39)]),
        ("td_noise_run_resets", "td", _table(_NOISE_RUN), 48, dict(td1, p=2), []),
        ("td_noise_needs_positive_overlap", "td", _table(_NOISE_OVERLAP_ZERO), 48, dict(td1, p=1), []),
        ("bu_single_peak", "bu", lambda ts, te: 1.0 - (abs(ts - 20) + abs(te - 39)) / 100.0, 100,
         dict(bu1, s_max=40, sigma=0.9, seed=3), [(20, 39)]),
        ("bu_plateau", "bu", lambda ts, te: 0.5, 24, dict(bu1, sigma=0.4), [(0, 7), (8, 15), (16, 23)]),
        ("bu_first_maximum", "bu", _table({(0, 11): 0.9, (4, 11): 0.9}, 0.1), 40, dict(bu1, sigma=0.5),
         [(0, 11)]),
        ("bu_restart_after_left_move", "bu", _table({(6, 13): 0.9}, 0.1), 24,
         dict(bu1, delta_bu=2, sigma=0.5), [(6, 13)]),
        ("bu_noise_drops_one_side", "bu", _noise_table, 64,
         dict(bu1, s_max=24, p=1, tau=0.1, sigma=0.5, pruning=1), [(4, 27)]),
        ("bu_noise_run_resets", "bu", _shift_table, 64, dict(bu1, p=2, tau=0.1, sigma=0.5, pruning=1),
         [(20, 27)]),
        ("bu_late_acceptance_taken", "bu", _table(_LATE, 0.05), 40, dict(late, seed=seeds[True]), [(4, 19)]),
        ("bu_late_acceptance_same_index", "bu", _table(_LATE, 0.05), 40, dict(late, seed=seeds[False]),
         [(4, 11)]),
        ("chunks_overlap", "chunked", lambda ts, te: 0.9 if (ts, te) == (16, 31) else 0.0, 64,
         dict(mode=0, chunks=2, k=1, s_min=16, s_max=16, sigma=0.5), [(16, 31), (16, 31)]),
        ("selection_nothing_found", "auto", lambda ts, te: 0.0, 64, sel, []),
        ("selection_td", "auto", lambda ts, te: 0.9 if (ts, te) == (0, 15) else 0.0, 64, sel, [(0, 15)]),
        ("selection_sampled_partitions", "auto",
         lambda ts, te: 0.9 if (ts, te) == (224, 239) else 0.0, 320,
         dict(sel, seed=1234567 ^ 0x5E1EC7, partitions=10), [(224, 239)]),
        ("td_tail_not_scored", "td", lambda ts, te: 0.9 if (ts, te) == (34, 49) else 0.0, 50,
         dict(k=1, s_min=16, s_max=16, sigma=0.5), []),
    ]


def oracle_run(search, score, t_end, kw):
    """The oracle's search on a machine case: (windows, evaluated-window count)."""
    sc = _score(score)
    if search == "td":
        return O.search_td(sc, t_begin=0, t_end=t_end, **kw)
    if search == "bu":
        return O.search_bu(sc, t_begin=0, t_end=t_end, **kw)
    if search == "chunked":
        return O.search_chunked(sc, None, 0, t_end, **kw)
    wins, n, _, _ = O.search_auto(sc, None, 0, t_end, **kw)
    return wins, n
