// Device building blocks of the window-MI kernels (arXiv 2204.09131, Sec. 4.2 Eq. KSGmi,
// Def. 4.2; counting rule of the Sec. 7.1 example; score of Sec. 5.4), shared by the batched
// kernels (kernels.cu) and the device-resident SYCOS_BU search (bu_device.cu).
//
// ksg_block evaluates a2-a5 for a block of 32 P points of one window: every lane owns P
// points and reads the window's values (x_j, y_j) as broadcasts from `s`, which is either a
// float2 array (the window staged in shared memory) or any type with a float2 operator[]
// (the window read from the resident series in global memory).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "isycos_internal.h"

namespace isy {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kUnroll = 4;

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Stable insertion of (d, j) into the ascending list bd/bj of K1 entries.  Every entry is
// computed from the old list at once: position r takes its predecessor when that is larger
// than d (the tail moves back one), d itself at the first position holding a larger value
// (so d lands after equal entries: candidates arrive in increasing j), else stays.  The
// dependent depth is one compare and two selects, against K1 - 1 compare-swap stages of a
// bubbling insertion; with d >= the last entry nothing changes.
template <int K1>
__device__ __forceinline__ void list_insert(float (&bd)[K1], int (&bj)[K1], float d, int j) {
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

// Canonical binary64 evaluation of the window scalars from the exact integer sums.
// inv_k = 1/k (correctly rounded, as computed on the host), or 0 for Kraskov's first
// estimator, which has no -1/k term (psi_k - 0 is psi_k exactly).  The binary64 work here
// runs on a narrow pipe: callers batch windows so that the lanes of one warp finish
// different windows together.
__device__ __forceinline__ void write_result(isycos_mi_out *o, int k, int m, long long s_psi,
                                             long long s_log, const long long *psi_fx,
                                             const long long *log_fx, double inv_k) {
    const double two_m32 = 2.3283064365386962890625e-10;  // 2^-32
    const double psi_k = __dmul_rn(__ll2double_rn(psi_fx[k]), two_m32);
    const double psi_m = __dmul_rn(__ll2double_rn(psi_fx[m]), two_m32);
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

// One block of 32 * P points of a window staged in shared memory `s` (m points): all of
// a2-a5 for points base + p * 32 + lane, p < P.  Adds the block's sums to acc_psi / acc_log.
template <int K1, int P = kPoints, typename Src = const float2 *>
__device__ __forceinline__ void ksg_block(Src s, int m, int base,
                                          int lane, const long long *__restrict__ psi_fx,
                                          const long long *__restrict__ log_fx,
                                          long long &acc_psi, long long &acc_log,
                                          int32_t *nx_out, int32_t *ny_out, int32_t *c_out,
                                          int est) {
    const float kInf = __int_as_float(0x7f800000);
    float xi[P], yi[P];
    bool val[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = base + p * 32 + lane;
        val[p] = i < m;
        const float2 v = val[p] ? s[i] : make_float2(kInf, kInf);  // sentinel never inserts
        xi[p] = v.x;
        yi[p] = v.y;
    }

    // a2: first K1 entries of (d_ij, j) over all j, self included.
    float bd[P][K1];
    int bj[P][K1];
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
        for (int r = 0; r < K1; ++r) {
            bd[p][r] = kInf;
            bj[p][r] = 0;
        }
    // The first 32 candidates, while the lists fill, and those from 512 on, which rarely
    // enter a list: in order, four at a time.
    auto in_order = [&](int j, int jh) {
        for (; j + kUnroll <= jh; j += kUnroll) {
            float2 v[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) v[u] = s[j + u];
            float d[kUnroll][P];
            bool any = false;
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    d[u][p] = fmaxf(fabsf(xi[p] - v[u].x), fabsf(yi[p] - v[u].y));
                    any |= d[u][p] < bd[p][K1 - 1];
                }
            if (any) {
#pragma unroll
                for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                    for (int p = 0; p < P; ++p)
                        if (d[u][p] < bd[p][K1 - 1]) list_insert<K1>(bd[p], bj[p], d[u][p], j + u);
            }
        }
        for (; j < jh; ++j) {
            const float2 v = s[j];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float d = fmaxf(fabsf(xi[p] - v.x), fabsf(yi[p] - v.y));
                if (d < bd[p][K1 - 1]) list_insert<K1>(bd[p], bj[p], d, j);
            }
        }
    };
    in_order(0, min(m, 32));
    // Candidates 32 .. 511 in chunks of 32: a lane marks the candidates closer than its
    // list's last entry at the chunk's start (no other can enter: that entry only shrinks),
    // then the lanes insert their marked candidates together, in increasing j, as many
    // rounds as the most marked (a warp that inserted per candidate would run an insertion
    // for nearly every one, since some lane's list takes it).
    const int jc = min(m, 512);
    for (int j0 = 32; j0 < jc; j0 += 32) {
        const int n = min(32, jc - j0);
        unsigned mk[P];
        float t[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            mk[p] = 0u;
            t[p] = bd[p][K1 - 1];
        }
        int u = 0;
        for (; u + kUnroll <= n; u += kUnroll) {
#pragma unroll
            for (int q = 0; q < kUnroll; ++q) {
                const float2 v = s[j0 + u + q];
#pragma unroll
                for (int p = 0; p < P; ++p)
                    mk[p] |= (fmaxf(fabsf(xi[p] - v.x), fabsf(yi[p] - v.y)) < t[p] ? 1u : 0u) << (u + q);
            }
        }
        for (; u < n; ++u) {
            const float2 v = s[j0 + u];
#pragma unroll
            for (int p = 0; p < P; ++p)
                mk[p] |= (fmaxf(fabsf(xi[p] - v.x), fabsf(yi[p] - v.y)) < t[p] ? 1u : 0u) << u;
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            while (__any_sync(kFull, mk[p] != 0u)) {
                if (mk[p] != 0u) {
                    const int b = __ffs(mk[p]) - 1;
                    mk[p] &= mk[p] - 1u;
                    const float2 v = s[j0 + b];
                    const float d = fmaxf(fabsf(xi[p] - v.x), fabsf(yi[p] - v.y));
                    if (d < bd[p][K1 - 1]) list_insert<K1>(bd[p], bj[p], d, j0 + b);
                }
            }
        }
    }
    in_order(jc, m);

    // a3: per-dimension distances to the neighbours.
    float dxm[P], dym[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        dxm[p] = 0.0f;
        dym[p] = 0.0f;
#pragma unroll
        for (int r = 0; r < K1; ++r) {
            const float2 v = s[bj[p][r]];
            dxm[p] = fmaxf(dxm[p], fabsf(xi[p] - v.x));
            dym[p] = fmaxf(dym[p], fabsf(yi[p] - v.y));
        }
    }

    // Kraskov's first estimator: both strips of half-width eps_i (the k-th neighbour's
    // distance, the last of the k + 1 entries with the point itself), points strictly
    // inside counted: |d| < eps  <=>  |d| <= the float just below eps (eps = 0: none).
    if (est) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float e = bd[p][K1 - 1];
            const float t = e > 0.0f ? __int_as_float(__float_as_int(e) - 1) : -1.0f;
            dxm[p] = t;
            dym[p] = t;
        }
    }

    // a4: marginal counts (inclusive; the point itself is counted and removed below).
    int cx[P], cy[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        cx[p] = 0;
        cy[p] = 0;
    }
    int j = 0;
    for (; j + kUnroll <= m; j += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const float2 v = s[j + u];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                cx[p] += fabsf(xi[p] - v.x) <= dxm[p] ? 1 : 0;
                cy[p] += fabsf(yi[p] - v.y) <= dym[p] ? 1 : 0;
            }
        }
    }
    for (; j < m; ++j) {
        const float2 v = s[j];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            cx[p] += fabsf(xi[p] - v.x) <= dxm[p] ? 1 : 0;
            cy[p] += fabsf(yi[p] - v.y) <= dym[p] ? 1 : 0;
        }
    }

    // Multiplicity of (x_i, y_i).
    int cc[P];
    bool need = false;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        cc[p] = 0;
#pragma unroll
        for (int r = 0; r < K1; ++r) cc[p] += bd[p][r] == 0.0f ? 1 : 0;
        need |= val[p] && bd[p][K1 - 1] == 0.0f;
    }
    if (__any_sync(kFull, need)) {
        int dup[P];
#pragma unroll
        for (int p = 0; p < P; ++p) dup[p] = 0;
        for (int jj = 0; jj < m; ++jj) {
            const float2 v = s[jj];
#pragma unroll
            for (int p = 0; p < P; ++p) dup[p] += (xi[p] == v.x && yi[p] == v.y) ? 1 : 0;
        }
#pragma unroll
        for (int p = 0; p < P; ++p)
            if (bd[p][K1 - 1] == 0.0f) cc[p] = dup[p];
    }

    // a5: fixed-point digamma and log sums.
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (!val[p]) continue;
        // the point itself was counted unless the strips are empty (estimator 1, eps = 0)
        const int nxv = max(cx[p] - 1, 0), nyv = max(cy[p] - 1, 0);
        acc_psi += __ldg(psi_fx + nxv + est) + __ldg(psi_fx + nyv + est);
        acc_log += __ldg(log_fx + cc[p]);
        const int i = base + p * 32 + lane;
        if (nx_out) {
            nx_out[i] = nxv;
            ny_out[i] = nyv;
            c_out[i] = cc[p];
        }
    }
}


// Stage a window's m values of x and y into s as (x, y) pairs, by the threads t = tid,
// tid + nt, ...: 16-byte loads of four consecutive values where x and y are equally aligned
// (series buffers are, and the window's start is common to both), scalar loads for the
// unaligned head and the tail.
__device__ __forceinline__ void stage_pair(float2 *__restrict__ s, const float *__restrict__ x,
                                           const float *__restrict__ y, int m, int tid, int nt) {
    const uintptr_t ax = reinterpret_cast<uintptr_t>(x), ay = reinterpret_cast<uintptr_t>(y);
    int head = m;
    if (((ax ^ ay) & 15) == 0) head = min(m, (int)(((16 - (ax & 15)) & 15) >> 2));
    for (int i = tid; i < head; i += nt) s[i] = make_float2(__ldg(x + i), __ldg(y + i));
    const int nb = (m - head) >> 2;
    const float4 *x4 = reinterpret_cast<const float4 *>(x + head);
    const float4 *y4 = reinterpret_cast<const float4 *>(y + head);
    for (int i = tid; i < nb; i += nt) {
        const float4 a = __ldg(x4 + i), b = __ldg(y4 + i);
        float2 *d = s + head + 4 * i;
        d[0] = make_float2(a.x, b.x);
        d[1] = make_float2(a.y, b.y);
        d[2] = make_float2(a.z, b.z);
        d[3] = make_float2(a.w, b.w);
    }
    for (int i = head + 4 * nb + tid; i < m; i += nt) s[i] = make_float2(__ldg(x + i), __ldg(y + i));
}

// The window read in place from the resident series (broadcast loads through L1).
struct PairSrc {
    const float *x;
    const float *y;
    __device__ __forceinline__ float2 operator[](int j) const { return make_float2(__ldg(x + j), __ldg(y + j)); }
};

}  // namespace dev
}  // namespace isy
