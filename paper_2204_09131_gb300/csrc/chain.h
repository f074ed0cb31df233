// Incremental window MI along chains of windows (chain.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "isycos_internal.h"

namespace isy {

constexpr int kChainThreads = 256;
constexpr int kChainMaxCap = 16384;   // ring capacity limit: two consecutive windows' span

// One chain: windows first_step .. first_step + n_steps - 1 of one pair, in order.
struct ChainDesc {
    const float *x;
    const float *y;
    int32_t first_step;
    int32_t n_steps;
    int32_t cap;          // power of two >= the span of any two consecutive windows
    int32_t pad;
    int64_t state_off;    // first slot of the chain's state (cap slots)
};

struct ChainStep {
    int64_t start;
    int32_t m;
    int32_t out;          // result index
};

// Per-point state, indexed by state_off + (time index mod cap).
struct ChainState {
    float *eps;
    float *dx;
    float *dy;
    int32_t *cx;          // inclusive marginal counts (the point itself counted)
    int32_t *cy;
    int32_t *cc;          // multiplicity of (x, y)
};

struct ChainArgs {
    const ChainDesc *chains;
    const ChainStep *steps;
    ChainState state;
    const long long *psi_fx;
    const long long *log_fx;
    isycos_mi_out *out;
    int32_t *recomputed;  // optional: points searched in full per window
    int32_t k;
};

inline size_t chain_smem(int cap) { return (size_t)cap * (sizeof(float) * 2 + sizeof(int32_t)); }

cudaError_t launch_chain(const ChainArgs &a, int n_chains, int max_cap, cudaStream_t st);

}  // namespace isy
