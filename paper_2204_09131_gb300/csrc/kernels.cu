// Window-level KSG mutual information on the GPU (arXiv 2204.09131, Sec. 4.2 Eq. KSGmi,
// Def. 4.2; counting rule of the box-assisted example of Sec. 7.1; score of Sec. 5.4).
//
// For a window {(x_j, y_j)}, j = 0 .. m-1, and every point i:
//   a2  d_ij = max(|x_i - x_j|, |y_i - y_j|) (binary32, exact IEEE sub/abs/max); the
//       k nearest neighbours are the first k points j != i in the order of (d_ij, j);
//   a3  d_x,i, d_y,i = largest |x_i - x_j|, |y_i - y_j| over those neighbours;
//   a4  n_x,i = #{j != i : |x_i - x_j| <= d_x,i}, n_y,i likewise, c_i = #{j : (x_j, y_j) = (x_i, y_i)};
//   a5  S_psi = sum_i psi_fx[n_x,i] + psi_fx[n_y,i], S_log = sum_i log_fx[c_i] (int64, exact)
//       and the scalars of isycos_mi_out in a fixed binary64 order.
//
// Neighbour search keeps, per point, the first k+1 entries of (d_ij, j) over ALL j of the
// window including i itself (d_ii = 0).  Since the point itself is among those k+1 entries,
// or all of them are at distance 0, the k+1 list minus one zero-distance entry is exactly
// the k-neighbour set of j != i; a zero entry adds nothing to the per-dimension maxima, so
// d_x,i and d_y,i are the maxima over the whole list and no per-pair j != i test is needed.
// j is scanned in increasing order and an entry replaces the list's last entry only when
// strictly closer, which realises the tie-break toward the smaller index.
//
// c_i: when the (k+1)-th distance is positive every duplicate of (x_i, y_i), i included, is
// in the list, so c_i = number of zero-distance entries; otherwise a third pass counts them
// (taken by a warp only if one of its points needs it).
//
// Layout: the window's values are staged in shared memory as float2 (x, y); each lane owns
// P points of a block of 32 P points and reads (x_j, y_j) as a broadcast, so every shared
// load serves 32 P pairs.  Work: m (m - 1) pairs per pass; no tensor cores (the path
// is compare-and-count work on the FP32/INT pipes).
#include <cuda_runtime.h>
#include <stdint.h>

#include "isycos_internal.h"
#include "ksg_device.cuh"

namespace isy {

// (warp_sum64, list_insert, write_result and ksg_block live in ksg_device.cuh)
using namespace dev;

namespace {

// ---------------------------------------------------------------------------------------
// Sub-quadratic path for one large window (all threads of the CTA), the sorted-strip form of
// the box-assisted search of Sec. 7.1: the window's points are sorted by x and by y; each
// point's neighbours are searched outward along one of the two orders, nearest first in that
// coordinate, until its distance on both sides exceeds the current k+1-th distance (no
// farther point can enter, since d >= |dx| and d >= |dy|); a point takes the y order when
// its y strip is much shorter than its x strip.  The marginal counts are ranges of the x-
// and y-sorted values found by binary search, because fl(|x_i - x_j|) is monotone along the
// sorted order.  Candidates
// arrive out of time order, so the neighbour list compares (d, j) lexicographically.  Every
// comparison is the same binary32 operation as in the brute-force path: results are equal.
// ---------------------------------------------------------------------------------------

// Order-preserving key of a float (-0 and +0 share a key).
__device__ __forceinline__ uint32_t fkey(float f) {
    const uint32_t u = __float_as_uint(f == 0.0f ? 0.0f : f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <int NT, typename T>
__device__ void bitonic_sort(T *k, int N) {   // N a power of two, called by all threads
    // Element i is handled by thread i mod NT, so a step with partner distance j < 32 pairs
    // elements of the same warp.  Between two steps that both stay inside warps a warp
    // barrier suffices; when either step reaches across warps (j >= 32), the whole CTA must
    // wait.
    for (int k2 = 2; k2 <= N; k2 <<= 1)
        for (int j = k2 >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += NT) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const T a = k[i], b = k[ixj];
                    const bool up = (i & k2) == 0;
                    if ((a > b) == up) {
                        k[i] = b;
                        k[ixj] = a;
                    }
                }
            }
            const int jn = j > 1 ? (j >> 1) : ((k2 << 1) <= N ? k2 : 0);   // the next step's j
            if (j >= 32 || jn >= 32 || jn == 0) __syncthreads();
            else __syncwarp();
        }
}

// The same network with the elements in registers: thread t of warp w holds the E elements
// (w E + q) 32 + lane, q < E (N = NT E).  Steps with partner distance j < 32 pair lanes of one
// warp (shuffles); 32 <= j < 32 E pair registers of one thread; only j >= 32 E goes through
// shared memory with CTA barriers (15 of the 78 steps at N = 4096, E = 4).
template <int NT, int E, typename T>
__device__ void bitonic_sort_reg(T *k, int N) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = k[(w * E + q) * 32 + lane];
    for (int k2 = 2; k2 <= N; k2 <<= 1) {
        int j = k2 >> 1;
        if (j >= 32 * E) {
            __syncthreads();   // every thread has read the previous shared-memory state
#pragma unroll
            for (int q = 0; q < E; ++q) k[(w * E + q) * 32 + lane] = v[q];
            __syncthreads();
            for (; j >= 32 * E; j >>= 1) {
                for (int i = threadIdx.x; i < N; i += NT) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const T a = k[i], b = k[ixj];
                        if ((a > b) == ((i & k2) == 0)) {
                            k[i] = b;
                            k[ixj] = a;
                        }
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int q = 0; q < E; ++q) v[q] = k[(w * E + q) * 32 + lane];
        }
        // (register indices stay compile-time: jq runs over the constants E / 2, ..., 1)
#pragma unroll
        for (int jq = E / 2; jq >= 1; jq >>= 1) {
            if (jq * 32 > (k2 >> 1)) continue;
#pragma unroll
            for (int q = 0; q < E; ++q) {
                if (q & jq) continue;
                const int p = q | jq;
                const bool up = ((((w * E + q) * 32 + lane) & k2) == 0);
                const T a = v[q], b = v[p];
                const bool sw = (a > b) == up;
                v[q] = sw ? b : a;
                v[p] = sw ? a : b;
            }
        }
        for (j = min(16, k2 >> 1); j >= 1; j >>= 1) {
            const bool lower = (lane & j) == 0;
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const T a = v[q];
                const T b = __shfl_xor_sync(kFull, a, j);
                const bool up = ((((w * E + q) * 32 + lane) & k2) == 0);
                v[q] = (lower == up) ? (b < a ? b : a) : (b > a ? b : a);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < E; ++q) k[(w * E + q) * 32 + lane] = v[q];
    __syncthreads();
}

// Sort N (a power of two) keys in shared or global memory with all NT threads: in registers
// when N is 1, 2 or 4 times NT, else in memory throughout.
template <int NT, typename T>
__device__ void sort_keys(T *k, int N) {
    if (N == NT) bitonic_sort_reg<NT, 1>(k, N);
    else if (N == 2 * NT) bitonic_sort_reg<NT, 2>(k, N);
    else if (N == 4 * NT) bitonic_sort_reg<NT, 4>(k, N);
    else bitonic_sort<NT>(k, N);
}

// The same insertion under the lexicographic order of (d, j), for candidates that arrive
// out of index order.
template <int K1>
__device__ __forceinline__ void insert_lex(float (&bd)[K1], int (&bj)[K1], float d, int j) {
    bool c[K1];
#pragma unroll
    for (int r = 0; r < K1; ++r) c[r] = bd[r] > d || (bd[r] == d && bj[r] > j);
#pragma unroll
    for (int r = K1 - 1; r > 0; --r) {
        bd[r] = c[r - 1] ? bd[r - 1] : (c[r] ? d : bd[r]);
        bj[r] = c[r - 1] ? bj[r - 1] : (c[r] ? j : bj[r]);
    }
    bd[0] = c[0] ? d : bd[0];
    bj[0] = c[0] ? j : bj[0];
}

__host__ __device__ inline int pow2_ceil(int m) {
    int n = 1;
    while (n < m) n <<= 1;
    return n;
}

// Value of a y key (fkey of the value in the upper 32 bits); zero decodes to +0, which
// subtracts and compares like -0.
__device__ __forceinline__ float key_val(unsigned long long k) {
    const uint32_t u = (uint32_t)(k >> 32);
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// A candidate of the outward scans as (x, y, j): position u of the x order (a record) or of
// the y order (a key, whose index selects the window's value).
template <bool Y>
__device__ __forceinline__ float4 cand(const float4 *rec, const unsigned long long *keys,
                                       const float2 *s, int u) {
    if constexpr (Y) {
        const int j = (int)(keys[u] & 0xffffffffu);
        const float2 v = s[j];
        return make_float4(v.x, v.y, __int_as_float(j), 0.0f);
    } else {
        return rec[u];
    }
}

// The coordinate a scan in that order is sorted by, at position u.
template <bool Y>
__device__ __forceinline__ float ord_val(const float4 *rec, const unsigned long long *keys, int u) {
    if constexpr (Y) return key_val(keys[u]);
    else return rec[u].x;
}

// Candidates u, u + dir, u + 2 dir, u + 3 dir into the list of the point (xi, yi): loads and
// distances first, then the insertions (the list is the same in any visiting order).
template <int K1, bool Y>
__device__ __forceinline__ void visit4(const float4 *rec, const unsigned long long *keys,
                                       const float2 *s, float xi, float yi, float (&bd)[K1],
                                       int (&bj)[K1], int u, int dir) {
    float4 c[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] = cand<Y>(rec, keys, s, u + q * dir);
    float d[4];
    bool any = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        d[q] = fmaxf(fabsf(xi - c[q].x), fabsf(yi - c[q].y));
        any |= d[q] <= bd[K1 - 1];
    }
    if (any) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int jj = __float_as_int(c[q].z);
            if (d[q] < bd[K1 - 1] || (d[q] == bd[K1 - 1] && jj < bj[K1 - 1]))
                insert_lex<K1>(bd, bj, d[q], jj);
        }
    }
}

template <int K1, bool Y>
__device__ __forceinline__ void visit1(const float4 *rec, const unsigned long long *keys,
                                       const float2 *s, float xi, float yi, float (&bd)[K1],
                                       int (&bj)[K1], int u) {
    const float4 c = cand<Y>(rec, keys, s, u);
    const float d = fmaxf(fabsf(xi - c.x), fabsf(yi - c.y));
    const int jj = __float_as_int(c.z);
    if (d < bd[K1 - 1] || (d == bd[K1 - 1] && jj < bj[K1 - 1])) insert_lex<K1>(bd, bj, d, jj);
}

// Positions base + q dir, q < n (n <= 32): every lane marks, in a mask, the candidates that
// would enter its list as it stands (no other can enter later: its last entry only
// decreases), then the lanes insert their own marked candidates together, as many rounds as
// the most marked, instead of one warp-wide insertion per candidate that some lane takes.
// (Used for the second half of the seeds, where most candidates enter no list; in the
// outward extensions, eight at a time, the marking costs more than it saves.)
template <int K1, bool Y>
__device__ __forceinline__ void visit_masked(const float4 *rec, const unsigned long long *keys,
                                             const float2 *s, float xi, float yi, float (&bd)[K1],
                                             int (&bj)[K1], int base, int dir, int n) {
    const float t = bd[K1 - 1];
    const int tj = bj[K1 - 1];
    unsigned mk = 0u;
    int q = 0;
    for (; q + 4 <= n; q += 4) {
        float4 c[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) c[r] = cand<Y>(rec, keys, s, base + (q + r) * dir);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float d = fmaxf(fabsf(xi - c[r].x), fabsf(yi - c[r].y));
            const bool in = d < t || (d == t && __float_as_int(c[r].z) < tj);
            mk |= (in ? 1u : 0u) << (q + r);
        }
    }
    for (; q < n; ++q) {
        const float4 c = cand<Y>(rec, keys, s, base + q * dir);
        const float d = fmaxf(fabsf(xi - c.x), fabsf(yi - c.y));
        const bool in = d < t || (d == t && __float_as_int(c.z) < tj);
        mk |= (in ? 1u : 0u) << q;
    }
    while (__any_sync(kFull, mk != 0u)) {
        if (mk != 0u) {
            const int b = __ffs(mk) - 1;
            mk &= mk - 1u;
            visit1<K1, Y>(rec, keys, s, xi, yi, bd, bj, base + b * dir);
        }
    }
}

// Positions [a0, a1) of the order, every lane of the warp: the first 32 in order (the lists
// are still filling), the rest marked and inserted lane by lane.
template <int K1, bool Y>
__device__ __forceinline__ void visit_range(const float4 *rec, const unsigned long long *keys,
                                            const float2 *s, float xi, float yi, float (&bd)[K1],
                                            int (&bj)[K1], int a0, int a1) {
    const int ah = min(a1, a0 + 32);
    int u = a0;
    for (; u + 4 <= ah; u += 4) visit4<K1, Y>(rec, keys, s, xi, yi, bd, bj, u, 1);
    for (; u < ah; ++u) visit1<K1, Y>(rec, keys, s, xi, yi, bd, bj, u);
    for (; u < a1; u += 32) visit_masked<K1, Y>(rec, keys, s, xi, yi, bd, bj, u, 1, min(32, a1 - u));
}

// Extend the scanned positions (L, R) outward, 8 at a time on each side, while the next
// position on that side is within the bound of some active lane along the order's coordinate
// ci.  The bound is the lane's current k+1-th distance, or bnd if smaller (an upper bound of
// the final one): a point farther than it along the coordinate cannot enter the list
// (d >= that coordinate's distance), and along the order that distance only grows (binary32
// subtraction is monotone) while the bounds only shrink.  Control is warp-uniform: every
// lane visits the same candidates (broadcast shared loads).
template <int K1, bool Y>
__device__ __forceinline__ void extend(const float4 *rec, const unsigned long long *keys,
                                       const float2 *s, float xi, float yi, bool act, float bnd,
                                       float (&bd)[K1], int (&bj)[K1], int &L, int &R, int m) {
    const float ci = Y ? yi : xi;
    for (;;) {
        const bool need_l = L >= 0 &&
            __any_sync(kFull, act && fabsf(ci - ord_val<Y>(rec, keys, L)) <= fminf(bd[K1 - 1], bnd));
        const bool need_r = R < m &&
            __any_sync(kFull, act && fabsf(ci - ord_val<Y>(rec, keys, R)) <= fminf(bd[K1 - 1], bnd));
        if (!need_l && !need_r) break;
        if (need_l) {
            if (L >= 7) {
                visit4<K1, Y>(rec, keys, s, xi, yi, bd, bj, L, -1);
                visit4<K1, Y>(rec, keys, s, xi, yi, bd, bj, L - 4, -1);
                L -= 8;
            } else {
                for (; L >= 0; --L) visit1<K1, Y>(rec, keys, s, xi, yi, bd, bj, L);
            }
        }
        if (need_r) {
            if (R + 8 <= m) {
                visit4<K1, Y>(rec, keys, s, xi, yi, bd, bj, R, 1);
                visit4<K1, Y>(rec, keys, s, xi, yi, bd, bj, R + 4, 1);
                R += 8;
            } else {
                for (; R < m; ++R) visit1<K1, Y>(rec, keys, s, xi, yi, bd, bj, R);
            }
        }
    }
}

// The strip [lo, hi] of positions around t (value c at t) whose values v(u) satisfy
// |c - v(u)| <= e, by binary search (the predicate holds on a range around t, since the
// values ascend); an empty strip (e < 0) leaves [t, t].  steps counts the search steps.
template <typename V>
__device__ __forceinline__ void strip_around(V v, float c, float e, int t, int m, int &lo, int &hi,
                                             int &steps) {
    int l0 = 0, l1 = t;
    while (l0 < l1) {
        ++steps;
        const int mid = (l0 + l1) >> 1;
        if (fabsf(c - v(mid)) <= e) l1 = mid;
        else l0 = mid + 1;
    }
    int r0 = t, r1 = m - 1;
    while (r0 < r1) {
        ++steps;
        const int mid = (r0 + r1 + 1) >> 1;
        if (fabsf(c - v(mid)) <= e) r0 = mid;
        else r1 = mid - 1;
    }
    lo = l0;
    hi = r0;
}

// A point searches along the y order instead of the x order when the y values around it are
// this many times sparser than the x values around it (mean gaps over 64 positions of each
// order), so that the same bound holds that many times fewer points in its y strip.
constexpr float kYSparser = 2.0f;
// Windows of at most this many points keep every search on the x order.
constexpr int kYOrderMin = 1024;
// The seed of a chunk's scans: the positions [c0 - kSeedBefore, c0 + kSeedAfter) of the order
// around a chunk of 32 positions from c0.
constexpr int kSeedBefore = 16, kSeedAfter = 48;

// work (optional): [0] += phase A point x candidate visits, [1] += search and
// duplicate-scan steps.
template <int K1, int NT>
__device__ void ksg_window_sorted(const float2 *__restrict__ s, int m, unsigned char *scratch,
                                  const long long *__restrict__ psi_fx,
                                  const long long *__restrict__ log_fx, long long &acc_psi,
                                  long long &acc_log, int32_t *nx_out, int32_t *ny_out,
                                  int32_t *c_out, int est, unsigned long long *work) {
    const float kInf = __int_as_float(0x7f800000);
    const int N = pow2_ceil(m);
    const int n_chunks = (m + 31) >> 5;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(scratch);
    float4 *rec = reinterpret_cast<float4 *>(scratch + (size_t)8 * N);
    float *pdx = reinterpret_cast<float *>(scratch + (size_t)8 * N + (size_t)16 * m);
    float *pdy = pdx + m;
    int *pcc = reinterpret_cast<int *>(pdy + m);
    int *ctr = pcc + m;
    unsigned *ymask = reinterpret_cast<unsigned *>(ctr + 4);

    // The x order as records (x, y, j, y position), then the y order as keys (value, j) in the
    // same slots (pcc holds each point's x position meanwhile); a window that keeps every
    // search on the x order needs only the sorted y values there.
    const bool two = m > kYOrderMin;
    float *ysf = reinterpret_cast<float *>(keys);
    for (int i = threadIdx.x; i < N; i += NT)
        keys[i] = i < m ? (((unsigned long long)fkey(s[i].x) << 32) | (unsigned)i) : ~0ull;
    __syncthreads();
    sort_keys<NT>(keys, N);
    for (int t = threadIdx.x; t < m; t += NT) {
        const int j = (int)(keys[t] & 0xffffffffu);
        rec[t] = make_float4(s[j].x, s[j].y, __int_as_float(j), 0.0f);
        pcc[j] = t;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_chunks; i += NT) ymask[i] = 0u;
    if (threadIdx.x < 4) ctr[threadIdx.x] = 0;
    if (two) {
        for (int i = threadIdx.x; i < N; i += NT)
            keys[i] = i < m ? (((unsigned long long)fkey(s[i].y) << 32) | (unsigned)i) : ~0ull;
        __syncthreads();
        sort_keys<NT>(keys, N);
        for (int p = threadIdx.x; p < m; p += NT)
            rec[pcc[(int)(keys[p] & 0xffffffffu)]].w = __int_as_float(p);
    } else {
        for (int i = threadIdx.x; i < N; i += NT) ysf[i] = i < m ? s[i].y : kInf;
        __syncthreads();
        sort_keys<NT>(ysf, N);
    }
    __syncthreads();

    // Phase A: the neighbour lists, by outward scans along one of the two orders (the list is
    // the first k + 1 entries of (d, j) over the window, whatever the order of the visits).
    // Per point it leaves, indexed by j, d_x, d_y and the multiplicity (or -1 when the
    // (k+1)-th distance is 0 and the duplicates must be counted in phase B).
    const int lane = threadIdx.x & 31;
    int steps = 0;          // this thread's search and scan steps
    unsigned visits = 0;    // this warp's point x candidate visits (< 2^32 per window)
    auto finish = [&](float xi, float yi, int ji, const float (&bd)[K1], const int (&bj)[K1]) {
        float dxm = 0.0f, dym = 0.0f;
        int cc = 0;
#pragma unroll
        for (int r = 0; r < K1; ++r) {
            const float2 v = s[bj[r]];
            dxm = fmaxf(dxm, fabsf(xi - v.x));
            dym = fmaxf(dym, fabsf(yi - v.y));
            cc += bd[r] == 0.0f ? 1 : 0;
        }
        if (est) {   // Kraskov's first estimator: strict strips of half-width eps
            const float e = bd[K1 - 1];
            dxm = dym = e > 0.0f ? __int_as_float(__float_as_int(e) - 1) : -1.0f;
        }
        pdx[ji] = dxm;
        pdy[ji] = dym;
        pcc[ji] = bd[K1 - 1] == 0.0f ? -1 : cc;
    };
    // A1: a warp takes 32 consecutive points of the x order (a chunk, from a shared counter)
    // and scans the seed positions of the x order around it, which gives every point a list
    // of k + 1 and so a bound b on its (k+1)-th distance.  In a window of more than kYOrderMin
    // points, a point whose strip reaches past the seed and whose y neighbourhood is kYSparser
    // times sparser than its x neighbourhood leaves its search to A2 (a bit at its y position)
    // with b; the other points of the chunk go on outward along the x order.
    for (;;) {
        int chunk = 0;
        if (lane == 0) chunk = atomicAdd(ctr, 1);
        chunk = __shfl_sync(kFull, chunk, 0);
        if (chunk >= n_chunks) break;
        const int c0 = chunk << 5;
        const int t = c0 + lane;
        const bool valid = t < m;
        float xi = kInf, yi = kInf;
        int ji = 0, py = 0;
        if (valid) {
            const float4 me = rec[t];
            xi = me.x;
            yi = me.y;
            ji = __float_as_int(me.z);
            py = __float_as_int(me.w);
        }
        // (a list at -inf takes no candidate: lanes without a point skip the insertions)
        float bd[K1];
        int bj[K1];
#pragma unroll
        for (int r = 0; r < K1; ++r) {
            bd[r] = valid ? kInf : -kInf;
            bj[r] = 0x7fffffff;
        }
        const int a0 = max(0, c0 - kSeedBefore), a1 = min(m, c0 + kSeedAfter);
        visit_range<K1, false>(rec, keys, s, xi, yi, bd, bj, a0, a1);
        visits += (unsigned)(a1 - a0) * (unsigned)min(32, m - c0);
        int L = a0 - 1, R = a1;
        bool act = valid;
        const bool more = valid && ((L >= 0 && fabsf(xi - rec[L].x) <= bd[K1 - 1]) ||
                                    (R < m && fabsf(xi - rec[R].x) <= bd[K1 - 1]));
        if (__any_sync(kFull, more)) {
            if (more && two) {
                // mean gaps: x over the seed positions, y over 64 positions around py
                const int pl = max(0, py - 32), pr = min(m - 1, py + 32);
                const float gx = (rec[a1 - 1].x - rec[a0].x) * (float)(pr - pl);
                const float gy = (key_val(keys[pr]) - key_val(keys[pl])) * (float)(a1 - 1 - a0);
                if (gy > kYSparser * gx) {
                    act = false;
                    pdx[ji] = bd[K1 - 1];
                    atomicOr(ymask + (py >> 5), 1u << (py & 31));
#pragma unroll
                    for (int r = 0; r < K1; ++r) bd[r] = -kInf;
                }
            }
            const int w0 = R - L - 1;
            extend<K1, false>(rec, keys, s, xi, yi, act, kInf, bd, bj, L, R, m);
            visits += (unsigned)(R - L - 1 - w0) * (unsigned)__popc(__ballot_sync(kFull, act));
        }
        if (act) finish(xi, yi, ji, bd, bj);
    }
    __syncthreads();
    // A2: a warp takes 32 consecutive positions of the y order whose bits are set and scans
    // the seed positions around them, then outward along the y order, for those points alone
    // (new lists; b bounds the strips from the start).
    while (two) {
        int chunk = 0;
        if (lane == 0) chunk = atomicAdd(ctr + 1, 1);
        chunk = __shfl_sync(kFull, chunk, 0);
        if (chunk >= n_chunks) break;
        const unsigned mk = ymask[chunk];
        if (mk == 0u) continue;
        const int c0 = chunk << 5;
        const bool act = (mk >> lane) & 1u;
        float xi = kInf, yi = kInf, bnd = kInf;
        int ji = 0;
        if (act) {
            ji = (int)(keys[c0 + lane] & 0xffffffffu);
            const float2 v = s[ji];
            xi = v.x;
            yi = v.y;
            bnd = pdx[ji];
        }
        float bd[K1];
        int bj[K1];
#pragma unroll
        for (int r = 0; r < K1; ++r) {
            bd[r] = act ? kInf : -kInf;
            bj[r] = 0x7fffffff;
        }
        const int a0 = max(0, c0 - kSeedBefore), a1 = min(m, c0 + kSeedAfter);
        visit_range<K1, true>(rec, keys, s, xi, yi, bd, bj, a0, a1);
        int L = a0 - 1, R = a1;
        extend<K1, true>(rec, keys, s, xi, yi, act, bnd, bd, bj, L, R, m);
        visits += (unsigned)(R - L - 1) * (unsigned)__popc(mk);
        if (act) finish(xi, yi, ji, bd, bj);
    }
    if (work && lane == 0) atomicAdd(work, (unsigned long long)visits);
    __syncthreads();
    // Phase B: the marginal counts by binary search, and the duplicate counts left open.
    for (int t = threadIdx.x; t < m; t += NT) {
        const float4 me = rec[t];
        const float xi = me.x, yi = me.y;
        const int ji = __float_as_int(me.z);
        const float dxm = pdx[ji], dym = pdy[ji];
        // n_x: the x-sorted range around position t where fabsf(x_i - x) <= d_x
        int l0, r0;
        strip_around([&](int u) { return rec[u].x; }, xi, dxm, t, m, l0, r0, steps);
        const int cx = r0 - l0 + 1;
        // n_y: the same on the y-sorted values, around the point's own y position (or the first
        // value >= y_i)
        int q0, w0;
        if (two) {
            strip_around([&](int u) { return key_val(keys[u]); }, yi, dym, __float_as_int(me.w), m, q0,
                         w0, steps);
        } else {
            int p0 = 0, p1 = m;
            while (p0 < p1) {
                ++steps;
                const int mid = (p0 + p1) >> 1;
                if (ysf[mid] < yi) p0 = mid + 1;
                else p1 = mid;
            }
            strip_around([&](int u) { return ysf[u]; }, yi, dym, p0, m, q0, w0, steps);
        }
        const int cy = w0 - q0 + 1;
        int cc = pcc[ji];
        if (cc < 0) {   // k+1-th distance 0: count the duplicates among the equal x values
            cc = 1;
            for (int u = t - 1; u >= 0 && rec[u].x == xi; --u, ++steps) cc += rec[u].y == yi ? 1 : 0;
            for (int u = t + 1; u < m && rec[u].x == xi; ++u, ++steps) cc += rec[u].y == yi ? 1 : 0;
        }
        // (an empty strip, e < 0, leaves the search ranges at the point itself: count 1)
        const int nxv = cx - 1, nyv = cy - 1;
        acc_psi += __ldg(psi_fx + nxv + est) + __ldg(psi_fx + nyv + est);
        acc_log += __ldg(log_fx + cc);
        if (nx_out) {
            nx_out[ji] = nxv;
            ny_out[ji] = nyv;
            c_out[ji] = cc;
        }
    }
    if (work) {
        unsigned long long w = (unsigned long long)steps;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(kFull, w, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(work + 1, w);
    }
}

// Persistent, size-bucketed batch: CTAs take jobs from a counter; a job is one large window
// (all warps) or several small windows of one bucket (wpw warps each).
template <int K1, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 4 : 1) ksg_batched_kernel(BatchArgs a) {
    extern __shared__ float2 tile[];
    constexpr int W = NT / 32;
    __shared__ long long acc_psi[W], acc_log[W];
    __shared__ int fin_out[W], fin_m[W];   // the job's items, finished by the lanes of warp 0
    __shared__ int job_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const BucketTable *T = a.table;
    for (;;) {
        if (threadIdx.x == 0) job_s = atomicAdd(a.queue, 1);
        __syncthreads();
        const int job = job_s;
        if (job >= T->total_jobs) break;
        int q = 0;
        while (q + 1 < kBuckets && job >= T->job_off[q + 1]) ++q;
        const int wpw = T->wpw[q];
        const int per_job = W / wpw;
        const int slot = warp / wpw, sub = warp % wpw;
        const int first = T->item_off[q] + (job - T->job_off[q]) * per_job;
        const int last = T->item_off[q] + T->count[q];
        const bool has = first + slot < last;
        WorkItem it;
        it.m = 0;
        if (has) it = a.items[first + slot];
        float2 *s = tile + (per_job == 1 ? 0 : slot * (kBlockPts * wpw));
        if (has) stage_pair(s, it.x, it.y, it.m, sub * 32 + lane, wpw * 32);
        if (lane == 0 && sub == 0) {
            acc_psi[slot] = 0;
            acc_log[slot] = 0;
            fin_out[slot] = has ? it.out : -1;
            fin_m[slot] = it.m;
        }
        __syncthreads();
        if (has) {
            long long lp = 0, ll = 0;
            int32_t *nxo = nullptr, *nyo = nullptr, *co = nullptr;
            if (a.nx && it.pts >= 0) {
                nxo = a.nx + it.pts;
                nyo = a.ny + it.pts;
                co = a.c + it.pts;
            }
            const bool sorted = per_job == 1 && ((a.sort_mask >> (32 - __clz(it.m - 1))) & 1u) &&
                                it.m >= a.sort_min && (it.m <= kSortMax || a.gscratch != nullptr);
            if (sorted) {
                unsigned char *scr = it.m <= kSortMax
                                         ? reinterpret_cast<unsigned char *>(tile) + sorted_off(it.m)
                                         : a.gscratch + (size_t)blockIdx.x * (size_t)a.gscratch_stride;
                ksg_window_sorted<K1, NT>(s, it.m, scr, a.psi_fx, a.log_fx, lp, ll, nxo, nyo, co, a.est,
                                          a.work);
            } else {
                const int nblk = (it.m + kBlockPts - 1) / kBlockPts;
                for (int b = sub; b < nblk; b += wpw)
                    ksg_block<K1>(s, it.m, b * kBlockPts, lane, a.psi_fx, a.log_fx, lp, ll, nxo, nyo, co, a.est);
            }
            lp = warp_sum64(lp);
            ll = warp_sum64(ll);
            if (lane == 0) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&acc_psi[slot]), (unsigned long long)lp);
                atomicAdd(reinterpret_cast<unsigned long long *>(&acc_log[slot]), (unsigned long long)ll);
            }
        }
        __syncthreads();
        if (warp == 0 && lane < per_job && fin_out[lane] >= 0)
            write_result(a.out + fin_out[lane], a.k, fin_m[lane], acc_psi[lane], acc_log[lane],
                         a.psi_fx, a.log_fx, a.inv_k);
    }
    // Small windows (m <= 64): one warp each, staged in the warp's own slice, no CTA barrier.
    float2 *ws = tile + warp * kWarpSlicePts;
    const int first = T->small_first, last = T->n_items;
    // lane r keeps the sums of the r-th pending window of this warp; the lanes finish up to
    // 32 windows together
    long long pend_psi = 0, pend_log = 0;
    int pend_m = 0, pend_out = 0, n_pend = 0;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(a.queue + 1, 1);
        idx = __shfl_sync(kFull, idx, 0);
        if (first + idx >= last) break;
        const WorkItem it = a.items[first + idx];
        __syncwarp();
        for (int i = lane; i < it.m; i += 32) ws[i] = make_float2(it.x[i], it.y[i]);
        __syncwarp();
        long long lp = 0, ll = 0;
        int32_t *nxo = nullptr, *nyo = nullptr, *co = nullptr;
        if (a.nx && it.pts >= 0) {
            nxo = a.nx + it.pts;
            nyo = a.ny + it.pts;
            co = a.c + it.pts;
        }
        if (it.m <= 32)
            ksg_block<K1, 1>(ws, it.m, 0, lane, a.psi_fx, a.log_fx, lp, ll, nxo, nyo, co, a.est);
        else
            ksg_block<K1, 2>(ws, it.m, 0, lane, a.psi_fx, a.log_fx, lp, ll, nxo, nyo, co, a.est);
        lp = warp_sum64(lp);
        ll = warp_sum64(ll);
        if (lane == n_pend) {
            pend_psi = lp;
            pend_log = ll;
            pend_m = it.m;
            pend_out = it.out;
        }
        if (++n_pend == 32) {
            write_result(a.out + pend_out, a.k, pend_m, pend_psi, pend_log, a.psi_fx, a.log_fx, a.inv_k);
            n_pend = 0;
        }
    }
    if (lane < n_pend)
        write_result(a.out + pend_out, a.k, pend_m, pend_psi, pend_log, a.psi_fx, a.log_fx, a.inv_k);
    // The last CTA to finish zeroes the work counters for the next launch on this buffer:
    // every other CTA has taken its last job before it counts itself out.
    // (the work counters this CTA added are ordered before its count by the fence)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.queue + 2, 1) == (int)gridDim.x - 1) {
            a.queue[0] = 0;
            a.queue[1] = 0;
            a.queue[2] = 0;
            if (a.work) {
                a.work_out[0] = atomicExch(a.work, 0ull);
                a.work_out[1] = atomicExch(a.work + 1, 0ull);
            }
            __threadfence_system();
        }
    }
}

// Plain form: one window per launch; CTA b handles the blocks b*W .. b*W + W - 1 and the
// last CTA to finish writes the result.
template <int K1, int NT>
__global__ void __launch_bounds__(NT) ksg_plain_kernel(WorkItem it, int k, const long long *psi_fx,
                                                       const long long *log_fx,
                                                       unsigned long long *acc, int32_t *done,
                                                       isycos_mi_out *out, int32_t *nx,
                                                       int32_t *ny, int32_t *c, int est) {
    extern __shared__ float2 tile[];
    constexpr int W = NT / 32;
    __shared__ long long sp[W], sl[W];
    __shared__ bool is_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    stage_pair(tile, it.x, it.y, it.m, threadIdx.x, NT);
    __syncthreads();
    long long lp = 0, ll = 0;
    const int b = blockIdx.x * W + warp;
    const int nblk = (it.m + kBlockPts - 1) / kBlockPts;
    if (b < nblk) ksg_block<K1>(tile, it.m, b * kBlockPts, lane, psi_fx, log_fx, lp, ll, nx, ny, c, est);
    lp = warp_sum64(lp);
    ll = warp_sum64(ll);
    if (lane == 0) {
        sp[warp] = lp;
        sl[warp] = ll;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tp = 0, tl = 0;
        for (int w = 0; w < W; ++w) {
            tp += sp[w];
            tl += sl[w];
        }
        atomicAdd(acc, (unsigned long long)tp);
        atomicAdd(acc + 1, (unsigned long long)tl);
        __threadfence();
        is_last = atomicAdd(done, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
        __threadfence();
        const long long tp = (long long)atomicAdd(acc, 0ull);
        const long long tl = (long long)atomicAdd(acc + 1, 0ull);
        write_result(out, k, it.m, tp, tl, psi_fx, log_fx, est ? 0.0 : __ddiv_rn(1.0, (double)k));
        acc[0] = 0;
        acc[1] = 0;
        *done = 0;
    }
}

// ---------------------------------------------------------------------------------------
// Device-side preparation of window lists that live in device memory.
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ int dev_bucket_slot(int m) {
    int b = 32 - __clz(m - 1);   // smallest b with m <= 2^b (m >= 2)
    if (m <= 1) b = 0;
    return kBuckets - 1 - b;
}

__global__ void prep_classify_kernel(PrepArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_w) return;
    const isycos_window w = a.windows[i];
    bool ok = w.reserved == 0 && w.xs >= 0 && w.xs < a.n_series && w.ys >= 0 &&
              w.ys < a.n_series && w.m >= a.k + 1 && w.m <= a.max_m && w.m <= kMaxM &&
              w.start >= 0;
    if (ok) {
        const int64_t nx = a.series_len[w.xs], ny = a.series_len[w.ys];
        ok = nx > 0 && ny > 0 && w.start + w.m <= nx && w.start + w.m <= ny &&
             a.series_ptr[w.xs] != nullptr && a.series_ptr[w.ys] != nullptr;
    }
    if (!ok) {
        atomicOr(a.status, 1);
        a.slot_of[i] = -1;
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        a.out[i].mi = nan;
        a.out[i].h_w = nan;
        a.out[i].nmi = nan;
        a.out[i].s_psi = 0;
        a.out[i].s_log = 0;
        return;
    }
    const int q = dev_bucket_slot(w.m);
    a.slot_of[i] = q;
    a.pos_of[i] = atomicAdd(a.bucket_count + q, 1);
}

__global__ void prep_table_kernel(PrepArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    fill_bucket_table(a.table, a.bucket_count, a.nt);
}

__global__ void prep_scatter_kernel(PrepArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_w) return;
    const int q = a.slot_of[i];
    if (q < 0) return;
    const isycos_window w = a.windows[i];
    WorkItem it;
    it.x = a.series_ptr[w.xs] + w.start;
    it.y = a.series_ptr[w.ys] + w.start;
    it.m = w.m;
    it.out = (int32_t)i;
    it.pts = -1;
    a.items[a.table->item_off[q] + a.pos_of[i]] = it;
}

__global__ void check_finite_kernel(const float *d, int64_t n, int32_t *flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (; i < n; i += stride) bad |= !isfinite(d[i]);
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// Kernel tables by k (K1 = k + 1).
template <int NT>
struct BatchedTable {
    using Fn = void (*)(BatchArgs);
    static Fn get(int k) {
        switch (k) {
            case 1: return ksg_batched_kernel<2, NT>;
            case 2: return ksg_batched_kernel<3, NT>;
            case 3: return ksg_batched_kernel<4, NT>;
            case 4: return ksg_batched_kernel<5, NT>;
            case 5: return ksg_batched_kernel<6, NT>;
            case 6: return ksg_batched_kernel<7, NT>;
            case 7: return ksg_batched_kernel<8, NT>;
            case 8: return ksg_batched_kernel<9, NT>;
        }
        return nullptr;
    }
};

using PlainFn = void (*)(WorkItem, int, const long long *, const long long *, unsigned long long *,
                         int32_t *, isycos_mi_out *, int32_t *, int32_t *, int32_t *, int);
constexpr int kPlainNT = 256;

PlainFn plain_fn(int k) {
    switch (k) {
        case 1: return ksg_plain_kernel<2, kPlainNT>;
        case 2: return ksg_plain_kernel<3, kPlainNT>;
        case 3: return ksg_plain_kernel<4, kPlainNT>;
        case 4: return ksg_plain_kernel<5, kPlainNT>;
        case 5: return ksg_plain_kernel<6, kPlainNT>;
        case 6: return ksg_plain_kernel<7, kPlainNT>;
        case 7: return ksg_plain_kernel<8, kPlainNT>;
        case 8: return ksg_plain_kernel<9, kPlainNT>;
    }
    return nullptr;
}

void (*batched_fn(int k, int nt))(BatchArgs) {
    if (nt == 256) return BatchedTable<256>::get(k);
    if (nt == 1024) return BatchedTable<1024>::get(k);
    return nullptr;
}

}  // namespace

cudaError_t set_batched_smem(int k, int nt, size_t smem) {
    auto fn = batched_fn(k, nt);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // let the whole unified L1 / shared array serve shared memory (more resident CTAs)
    return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

cudaError_t batched_occupancy(int k, int nt, size_t smem, int *blocks_per_sm) {
    auto fn = batched_fn(k, nt);
    if (!fn) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, nt, smem);
}

cudaError_t launch_batched(const BatchArgs &a, int grid, size_t smem, cudaStream_t st) {
    auto fn = batched_fn(a.k, a.nt);
    if (!fn) return cudaErrorInvalidValue;
    fn<<<grid, a.nt, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_plain(const WorkItem &it, int k, const long long *psi_fx,
                         const long long *log_fx, unsigned long long *acc, int32_t *done,
                         isycos_mi_out *out, int32_t *nx, int32_t *ny, int32_t *c,
                         int est, cudaStream_t st, int *launches) {
    PlainFn fn = plain_fn(k);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = (size_t)it.m * 8;
    if (smem > 48 * 1024) {   // the largest window's limit, the same for every caller
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxM * 8);
        if (e != cudaSuccess) return e;
    }
    const int per_cta = (kPlainNT / 32) * kBlockPts;
    const int grid = (it.m + per_cta - 1) / per_cta;
    fn<<<grid, kPlainNT, smem, st>>>(it, k, psi_fx, log_fx, acc, done, out, nx, ny, c, est);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_prep(const PrepArgs &a, cudaStream_t st, int *launches) {
    const int nt = 256;
    const int grid = (int)((a.n_w + nt - 1) / nt);
    if (grid > 0) prep_classify_kernel<<<grid, nt, 0, st>>>(a);
    prep_table_kernel<<<1, 32, 0, st>>>(a);
    if (grid > 0) prep_scatter_kernel<<<grid, nt, 0, st>>>(a);
    if (launches) *launches += grid > 0 ? 3 : 1;
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const float *d, int64_t n, int32_t *flag, cudaStream_t st) {
    const int nt = 256;
    int64_t blocks = (n + nt - 1) / nt;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    check_finite_kernel<<<(int)blocks, nt, 0, st>>>(d, n, flag);
    return cudaGetLastError();
}

}  // namespace isy
