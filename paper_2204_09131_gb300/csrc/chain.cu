// Incremental window MI along a chain of windows (arXiv 2204.09131 Sec. 7.1, "Incremental
// MI computation with influenced regions", Defs. 7.1-7.2, Lemmas 3-6).
//
// A chain is a sequence of windows of one pair; each window's per-point state is derived
// from the previous window's by the points removed (R) and added (A).  Per point i of the
// window the state is: eps_i (the (k+1)-th smallest (d_ij, j) distance over all j including
// i, which equals the k-th neighbour distance), the per-dimension distances d_x,i, d_y,i,
// the inclusive marginal counts and the multiplicity c_i.
//
// For a point p present in both windows:
//  - influenced region (Def. 7.1): the closed square of half-side eps_p around p.  If some
//    o in R or A has d(p, o) <= eps_p, the neighbour set of p may change (Lemmas 3, 4): p's
//    neighbours are searched again over the new window and its counts recounted;
//  - otherwise no removed point was a neighbour (all neighbours lie inside the square) and
//    no added point can enter (it would have to be inside the square), so d_x,p, d_y,p keep
//    their values, and each removed / added point inside the influenced marginal regions
//    |x_o - x_p| <= d_x,p (resp. y) changes n_x,p (resp. n_y,p) by one (Lemmas 5, 6).
// Every added point is computed in full.  The closed square also flags ties at eps_p, so a
// recomputation happens whenever the tie-break (d, j) could matter; results are identical
// to the from-scratch kernel bit for bit (same binary32 operations, same scan order in j).
//
// Layout: one CTA per chain; the window's (x, y) values live in a shared-memory ring indexed
// by time index mod cap (cap >= the span of two consecutive windows), the per-point state in
// a global scratch area indexed the same way.
#include <cuda_runtime.h>
#include <stdint.h>

#include "chain.h"

namespace isy {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Stable insertion of (d, j) into the ascending list (candidates arrive in increasing j):
// every position is computed from the old list at once, so the dependent depth is one compare
// and two selects; with d >= the last entry nothing changes.
template <int K1>
__device__ __forceinline__ void insert_sorted(float (&bd)[K1], int (&bj)[K1], float d, int j) {
    bool c[K1];
#pragma unroll
    for (int r = 0; r < K1; ++r) c[r] = bd[r] > d;
#pragma unroll
    for (int r = K1 - 1; r > 0; --r) {
        bd[r] = c[r - 1] ? bd[r - 1] : (c[r] ? d : bd[r]);
        bj[r] = c[r - 1] ? bj[r - 1] : (c[r] ? j : bj[r]);
    }
    bd[0] = c[0] ? d : bd[0];
    bj[0] = c[0] ? j : bj[0];
}

// Full neighbour search and counts for one point (time index tp) over the window
// [s, s + m - 1] held in the ring.  Writes the point's state.
template <int K1>
__device__ void full_point(const float2 *__restrict__ ring, int mask, int64_t s, int m,
                           int64_t tp, ChainState st, int slot_base) {
    const float kInf = __int_as_float(0x7f800000);
    const float2 me = ring[(int)(tp & mask)];
    float bd[K1];
    int bj[K1];
#pragma unroll
    for (int r = 0; r < K1; ++r) {
        bd[r] = kInf;
        bj[r] = 0;
    }
    const int s0 = (int)(s & mask);
    for (int j = 0; j < m; ++j) {
        const float2 v = ring[(s0 + j) & mask];
        const float d = fmaxf(fabsf(me.x - v.x), fabsf(me.y - v.y));
        if (d < bd[K1 - 1]) insert_sorted<K1>(bd, bj, d, j);
    }
    float dx = 0.0f, dy = 0.0f;
#pragma unroll
    for (int r = 0; r < K1; ++r) {
        const float2 v = ring[(s0 + bj[r]) & mask];
        dx = fmaxf(dx, fabsf(me.x - v.x));
        dy = fmaxf(dy, fabsf(me.y - v.y));
    }
    int cx = 0, cy = 0;
    for (int j = 0; j < m; ++j) {
        const float2 v = ring[(s0 + j) & mask];
        cx += fabsf(me.x - v.x) <= dx ? 1 : 0;
        cy += fabsf(me.y - v.y) <= dy ? 1 : 0;
    }
    int cc = 0;
#pragma unroll
    for (int r = 0; r < K1; ++r) cc += bd[r] == 0.0f ? 1 : 0;
    if (bd[K1 - 1] == 0.0f) {
        cc = 0;
        for (int j = 0; j < m; ++j) {
            const float2 v = ring[(s0 + j) & mask];
            cc += (me.x == v.x && me.y == v.y) ? 1 : 0;
        }
    }
    const int slot = slot_base + (int)(tp & mask);
    st.eps[slot] = bd[K1 - 1];
    st.dx[slot] = dx;
    st.dy[slot] = dy;
    st.cx[slot] = cx;
    st.cy[slot] = cy;
    st.cc[slot] = cc;
}

__device__ __forceinline__ long long block_sum64(long long v, long long *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    long long t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    __syncthreads();
    return t;   // valid in thread 0
}

__device__ __forceinline__ void write_result(isycos_mi_out *o, int k, int m, long long s_psi,
                                             long long s_log, const long long *psi_fx,
                                             const long long *log_fx) {
    const double two_m32 = 2.3283064365386962890625e-10;  // 2^-32
    const double psi_k = __dmul_rn(__ll2double_rn(psi_fx[k]), two_m32);
    const double psi_m = __dmul_rn(__ll2double_rn(psi_fx[m]), two_m32);
    const double inv_k = __ddiv_rn(1.0, (double)k);
    const double mean_psi = __ddiv_rn(__dmul_rn(__ll2double_rn(s_psi), two_m32), (double)m);
    const double mi = __dsub_rn(__dadd_rn(__dsub_rn(psi_k, inv_k), psi_m), mean_psi);
    const double ln_m = __dmul_rn(__ll2double_rn(log_fx[m]), two_m32);
    const double h = __dsub_rn(ln_m, __ddiv_rn(__dmul_rn(__ll2double_rn(s_log), two_m32), (double)m));
    o->mi = mi;
    o->h_w = h;
    o->nmi = h > 0.0 ? __ddiv_rn(mi, h) : 0.0;
    o->s_psi = s_psi;
    o->s_log = s_log;
}

template <int K1, int NT>
__global__ void __launch_bounds__(NT) ksg_chain_kernel(ChainArgs a) {
    extern __shared__ unsigned char smem[];
    __shared__ long long red[NT / 32];
    __shared__ int n_work;
    __shared__ int n_flag;
    const ChainDesc ch = a.chains[blockIdx.x];
    const int cap = ch.cap, mask = cap - 1;
    float2 *ring = reinterpret_cast<float2 *>(smem);
    int32_t *work = reinterpret_cast<int32_t *>(smem + (size_t)cap * sizeof(float2));  // t - s
    const int slot_base = (int)ch.state_off;
    ChainState st = a.state;
    int64_t ps = 0, pe = -1;   // previous window (empty at the start)
    for (int q = 0; q < ch.n_steps; ++q) {
        const ChainStep sp = a.steps[ch.first_step + q];
        const int64_t s = sp.start, e = sp.start + sp.m - 1;
        const int m = sp.m;
        // kept = [ks, ke]; added = [s, min(e, ps-1)] U [max(s, pe+1), e];
        // removed = [ps, min(pe, s-1)] U [max(ps, e+1), pe]
        const int64_t ks = s > ps ? s : ps, ke = e < pe ? e : pe;
        const int64_t a0s = s, a0e = (e < ps - 1 ? e : ps - 1);
        const int64_t a1s = (s > pe + 1 ? s : pe + 1), a1e = e;
        const int64_t r0s = ps, r0e = (pe < s - 1 ? pe : s - 1);
        const int64_t r1s = (ps > e + 1 ? ps : e + 1), r1e = pe;
        const bool overlap = ks <= ke;
        if (threadIdx.x == 0) {
            n_work = 0;
            n_flag = 0;
        }
        // 1) stage the added points into the ring (all points when nothing overlaps)
        if (!overlap) {
            for (int i = threadIdx.x; i < m; i += NT) {
                const int64_t t = s + i;
                ring[(int)(t & mask)] = make_float2(ch.x[t], ch.y[t]);
            }
        } else {
            for (int64_t t = a0s + threadIdx.x; t <= a0e; t += NT)
                ring[(int)(t & mask)] = make_float2(ch.x[t], ch.y[t]);
            for (int64_t t = a1s + threadIdx.x; t <= a1e; t += NT)
                ring[(int)(t & mask)] = make_float2(ch.x[t], ch.y[t]);
        }
        __syncthreads();
        // 2) points kept from the previous window: influenced-region test and +-1 updates
        if (overlap) {
            for (int64_t p = ks + threadIdx.x; p <= ke; p += NT) {
                const int slot = slot_base + (int)(p & mask);
                const float2 me = ring[(int)(p & mask)];
                const float eps = st.eps[slot], dxm = st.dx[slot], dym = st.dy[slot];
                bool flag = false;
                int dcx = 0, dcy = 0, dcc = 0;
                // removed points
                for (int pass = 0; pass < 2; ++pass) {
                    const int64_t lo = pass == 0 ? r0s : r1s, hi = pass == 0 ? r0e : r1e;
                    for (int64_t t = lo; t <= hi; ++t) {
                        const float2 v = ring[(int)(t & mask)];
                        const float ax = fabsf(me.x - v.x), ay = fabsf(me.y - v.y);
                        flag |= fmaxf(ax, ay) <= eps;
                        dcx -= ax <= dxm ? 1 : 0;
                        dcy -= ay <= dym ? 1 : 0;
                        dcc -= (ax == 0.0f && ay == 0.0f) ? 1 : 0;
                    }
                }
                // added points
                for (int pass = 0; pass < 2; ++pass) {
                    const int64_t lo = pass == 0 ? a0s : a1s, hi = pass == 0 ? a0e : a1e;
                    for (int64_t t = lo; t <= hi; ++t) {
                        const float2 v = ring[(int)(t & mask)];
                        const float ax = fabsf(me.x - v.x), ay = fabsf(me.y - v.y);
                        flag |= fmaxf(ax, ay) <= eps;
                        dcx += ax <= dxm ? 1 : 0;
                        dcy += ay <= dym ? 1 : 0;
                        dcc += (ax == 0.0f && ay == 0.0f) ? 1 : 0;
                    }
                }
                if (flag) {
                    work[atomicAdd(&n_work, 1)] = (int32_t)(p - s);
                    atomicAdd(&n_flag, 1);
                } else {
                    st.cx[slot] += dcx;
                    st.cy[slot] += dcy;
                    st.cc[slot] += dcc;
                }
            }
        }
        __syncthreads();
        // the added points join the work list
        if (!overlap) {
            for (int i = threadIdx.x; i < m; i += NT) work[atomicAdd(&n_work, 1)] = i;
        } else {
            for (int64_t t = a0s + threadIdx.x; t <= a0e; t += NT) work[atomicAdd(&n_work, 1)] = (int32_t)(t - s);
            for (int64_t t = a1s + threadIdx.x; t <= a1e; t += NT) work[atomicAdd(&n_work, 1)] = (int32_t)(t - s);
        }
        __syncthreads();
        // 3) full neighbour search for the work list over the new window
        const int nw = n_work;
        for (int w = threadIdx.x; w < nw; w += NT) full_point<K1>(ring, mask, s, m, s + work[w], st, slot_base);
        __syncthreads();
        // 4) the window's sums
        long long lp = 0, ll = 0;
        for (int i = threadIdx.x; i < m; i += NT) {
            const int slot = slot_base + (int)((s + i) & mask);
            lp += a.psi_fx[st.cx[slot] - 1] + a.psi_fx[st.cy[slot] - 1];
            ll += a.log_fx[st.cc[slot]];
        }
        const long long tp = block_sum64(lp, red);
        const long long tl = block_sum64(ll, red);
        if (threadIdx.x == 0) {
            write_result(a.out + sp.out, a.k, m, tp, tl, a.psi_fx, a.log_fx);
            if (a.recomputed) a.recomputed[sp.out] = nw;
        }
        ps = s;
        pe = e;
        __syncthreads();
    }
}

using ChainFn = void (*)(ChainArgs);

ChainFn chain_fn(int k) {
    switch (k) {
        case 1: return ksg_chain_kernel<2, kChainThreads>;
        case 2: return ksg_chain_kernel<3, kChainThreads>;
        case 3: return ksg_chain_kernel<4, kChainThreads>;
        case 4: return ksg_chain_kernel<5, kChainThreads>;
        case 5: return ksg_chain_kernel<6, kChainThreads>;
        case 6: return ksg_chain_kernel<7, kChainThreads>;
        case 7: return ksg_chain_kernel<8, kChainThreads>;
        case 8: return ksg_chain_kernel<9, kChainThreads>;
    }
    return nullptr;
}

}  // namespace

cudaError_t launch_chain(const ChainArgs &a, int n_chains, int max_cap, cudaStream_t st) {
    ChainFn fn = chain_fn(a.k);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = chain_smem(max_cap);
    // The limit is a property of the function, shared by every lane: always the largest ring's
    // (a smaller value set by one lane would fail another lane's launch of a larger ring).
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)chain_smem(kChainMaxCap));
    if (e != cudaSuccess) return e;
    fn<<<n_chains, kChainThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace isy

// ------------------------------------------------------------------------------------
// Host side: split a window sequence into chains and run them.
// ------------------------------------------------------------------------------------
#include <string.h>

#include <algorithm>
#include <vector>

#include "runtime.h"

namespace isy {

static int pow2_at_least(int64_t v) {
    int c = 1;
    while (c < v) c <<= 1;
    return c;
}

isycos_status engine_eval_chains(isycos_ctx *ctx, Lane &L, const ChainSpec *specs, size_t n_specs,
                                 int k, isycos_mi_out *out, int64_t n_out, cudaStream_t st) {
    // Segments: a new chain starts where two consecutive windows do not fit one ring.
    std::vector<ChainDesc> chains;
    std::vector<ChainStep> steps;
    int64_t state_slots = 0, pairs = 0;
    int max_cap = 1;
    const int32_t dummy = (int32_t)n_out;      // results of discarded steps land here
    // Long chains are cut into segments so that about two segments per SM run at once;
    // each segment starts from scratch, so a segment holds at least 16 windows.
    int64_t total_steps = 0;
    for (size_t c = 0; c < n_specs; ++c) {
        total_steps += (int64_t)specs[c].starts.size();
        for (size_t i = 0; i < specs[c].starts.size(); ++i)
            if (!window_in_series(ctx, specs[c].xs, specs[c].ys, specs[c].starts[i], specs[c].sizes[i], k))
                return fail(ctx, ISYCOS_E_INVAL, "chain window [%lld, +%d] is outside its series",
                            (long long)specs[c].starts[i], specs[c].sizes[i]);
    }
    const int64_t seg_len = std::max<int64_t>(16, (total_steps + 2 * ctx->n_sm - 1) / (2 * ctx->n_sm));
    for (size_t c = 0; c < n_specs; ++c) {
        const ChainSpec &sp = specs[c];
        const int64_t n = (int64_t)sp.starts.size();
        int64_t seg_first = 0;
        int64_t span_need = n ? sp.sizes[0] : 0;
        for (int64_t i = 0; i <= n; ++i) {
            bool cut = (i == n);
            if (!cut && i - seg_first >= seg_len) cut = true;
            if (!cut && i > seg_first) {
                const int64_t lo = std::min(sp.starts[i - 1], sp.starts[i]);
                const int64_t hi = std::max(sp.starts[i - 1] + sp.sizes[i - 1], sp.starts[i] + sp.sizes[i]);
                if (hi - lo > kChainMaxCap) cut = true;
                else span_need = std::max(span_need, hi - lo);
            }
            if (cut && i > seg_first) {
                ChainDesc d;
                d.x = ctx->series_ptr[sp.xs];
                d.y = ctx->series_ptr[sp.ys];
                d.first_step = (int32_t)(steps.size() - (size_t)(i - seg_first));
                d.n_steps = (int32_t)(i - seg_first);
                d.cap = pow2_at_least(span_need);
                d.pad = 0;
                d.state_off = state_slots;
                state_slots += d.cap;
                max_cap = std::max(max_cap, d.cap);
                chains.push_back(d);
                seg_first = i;
                if (i < n) span_need = sp.sizes[i];
            }
            if (i < n) {
                ChainStep s;
                s.start = sp.starts[i];
                s.m = sp.sizes[i];
                s.out = sp.out_idx[i] >= 0 ? (int32_t)sp.out_idx[i] : dummy;
                steps.push_back(s);
                pairs += (int64_t)s.m * (s.m - 1);
            }
        }
    }
    const int64_t n_steps = (int64_t)steps.size();
    if (n_steps == 0) return ISYCOS_OK;
    if (state_slots > INT32_MAX / 2 || n_out > INT32_MAX / 2)
        return fail(ctx, ISYCOS_E_INVAL, "chain state too large");
    isycos_status rc;
    const size_t sb = (size_t)state_slots;
    if ((rc = dev_reserve(ctx, L.d_chain_desc, sizeof(ChainDesc) * chains.size()))) return rc;
    if ((rc = dev_reserve(ctx, L.d_chain_steps, sizeof(ChainStep) * n_steps))) return rc;
    if ((rc = dev_reserve(ctx, L.d_chain_state, 24 * sb))) return rc;
    if ((rc = dev_reserve(ctx, L.d_chain_out, sizeof(isycos_mi_out) * (n_out + 1)))) return rc;
    if ((rc = dev_reserve(ctx, L.d_chain_recomp, 4 * (n_out + 1)))) return rc;
    cudaError_t e = cudaMemcpyAsync(L.d_chain_desc.p, chains.data(), sizeof(ChainDesc) * chains.size(),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.d_chain_steps.p, steps.data(), sizeof(ChainStep) * n_steps,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.d_chain_recomp.p, 0, 4 * (n_out + 1), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "chain staging");
    unsigned char *sbase = reinterpret_cast<unsigned char *>(L.d_chain_state.p);
    ChainArgs a;
    a.chains = reinterpret_cast<const ChainDesc *>(L.d_chain_desc.p);
    a.steps = reinterpret_cast<const ChainStep *>(L.d_chain_steps.p);
    a.state.eps = reinterpret_cast<float *>(sbase);
    a.state.dx = reinterpret_cast<float *>(sbase + 4 * sb);
    a.state.dy = reinterpret_cast<float *>(sbase + 8 * sb);
    a.state.cx = reinterpret_cast<int32_t *>(sbase + 12 * sb);
    a.state.cy = reinterpret_cast<int32_t *>(sbase + 16 * sb);
    a.state.cc = reinterpret_cast<int32_t *>(sbase + 20 * sb);
    a.psi_fx = ctx->d_psi_fx;
    a.log_fx = ctx->d_log_fx;
    a.out = reinterpret_cast<isycos_mi_out *>(L.d_chain_out.p);
    a.recomputed = reinterpret_cast<int32_t *>(L.d_chain_recomp.p);
    a.k = k;
    e = launch_chain(a, (int)chains.size(), max_cap, st);
    if (e != cudaSuccess)
        return fail(ctx, ISYCOS_E_CUDA, "chain kernel launch (%d chains, ring of %d points, %zu bytes of shared memory): %s",
                    (int)chains.size(), max_cap, chain_smem(max_cap), cudaGetErrorString(e));
    std::vector<int32_t> recomp((size_t)n_out + 1);
    std::vector<isycos_mi_out> all((size_t)n_out + 1);
    e = cudaMemcpyAsync(all.data(), L.d_chain_out.p, sizeof(isycos_mi_out) * (n_out + 1),
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(recomp.data(), L.d_chain_recomp.p, 4 * (n_out + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "chain kernel");
    // only the chains' own results: other entries of `out` belong to the caller
    for (const ChainStep &s : steps)
        if (s.out != dummy) out[s.out] = all[s.out];
    int64_t full = 0;
    for (int32_t r : recomp) full += r;
    add_stats(ctx, n_steps, pairs, 1, 1, n_steps);
    {
        std::lock_guard<std::mutex> g(ctx->stats_mu);
        ctx->stats.incr_full_points += full;
    }
    return ISYCOS_OK;
}

}  // namespace isy

extern "C" isycos_status isycos_mi_chain(isycos_ctx *ctx, int32_t xs, int32_t ys,
                                         const int64_t *starts, const int32_t *sizes,
                                         int64_t n_steps, int32_t k, isycos_mi_out *out,
                                         void *cuda_stream) {
    using namespace isy;
    if (!ctx) return ISYCOS_E_INVAL;
    if (k < 1 || k > kMaxK) return fail(ctx, ISYCOS_E_INVAL, "k = %d outside [1, %d]", k, kMaxK);
    if (n_steps < 0 || n_steps > INT32_MAX / 2 || (n_steps > 0 && (!starts || !sizes || !out)))
        return fail(ctx, ISYCOS_E_INVAL, "chain: bad arguments");
    if (n_steps == 0) return ISYCOS_OK;
    std::lock_guard<std::mutex> g(ctx->engine_mu);
    cudaSetDevice(ctx->device);
    ChainSpec sp;
    sp.xs = xs;
    sp.ys = ys;
    for (int64_t i = 0; i < n_steps; ++i) {
        isycos_window w{xs, ys, starts[i], sizes[i], 0};
        isycos_status rc = check_window(ctx, w, k);
        if (rc) return rc;
        sp.starts.push_back(starts[i]);
        sp.sizes.push_back(sizes[i]);
        sp.out_idx.push_back(i);
    }
    return engine_eval_chains(ctx, *ctx->lanes[0].load(), &sp, 1, k, out, n_steps, pick_stream(ctx, cuda_stream));
}
