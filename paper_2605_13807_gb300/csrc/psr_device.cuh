// Device-side helpers shared by the libpsr kernels.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace psr {

// Records the first device-side error in the context's status word.
__device__ __forceinline__ void set_status(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// Gate nonlinearity of the minGRU update (Sec. II.C): sigma(x) = 1/(1+e^-x).
__device__ __forceinline__ float sigmoid_f(float x) { return 1.0f / (1.0f + expf(-x)); }

// Exact (erf) GELU used after the output map (Sec. II.G).
__device__ __forceinline__ float gelu_f(float x) {
    return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}

// d GELU / dx = Phi(x) + x phi(x).
__device__ __forceinline__ float gelu_grad_f(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
           x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// softplus(x) = log(1 + e^x), stable for both signs.
__device__ __forceinline__ float softplus_f(float x) {
    return fmaxf(x, 0.0f) + log1pf(expf(-fabsf(x)));
}

// Two-way conditional: log P(s | .) from the logit difference
// d = logit[1] - logit[0]:  log P(1) = -softplus(-d), log P(0) = -softplus(d).
// forced >= 0 pins the conditional to that value (zero-magnetisation mask).
__device__ __forceinline__ float site_logp(float d, int s, int forced) {
    if (forced >= 0) return (s == forced) ? 0.0f : -INFINITY;
    return s ? -softplus_f(-d) : -softplus_f(d);
}

// Forced value of site t given n_up ups before it (-1 if free).
__device__ __forceinline__ int u1_forced(int u1, int N, int t, int n_up) {
    if (!u1) return -1;
    if (n_up == (N >> 1)) return 0;
    if (t - n_up == (N >> 1)) return 1;
    return -1;
}

// Bits of sites [t0, t0+32) of a bit-packed row (t0 a multiple of 32) and the
// bit of site t0-1, with the flips p and q (-1 = none) applied.
__device__ __forceinline__ void chunk_bits32(const uint64_t *row, int t0, int p, int q,
                                             uint32_t &cur, uint32_t &prev) {
    cur = (uint32_t)(row[t0 >> 6] >> (t0 & 63));
    prev = (t0 > 0) ? (uint32_t)(row[(t0 - 1) >> 6] >> ((t0 - 1) & 63)) & 1u : 0u;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        int x = f ? q : p;
        if (x < 0) continue;
        if (x >= t0 && x < t0 + 32) cur ^= 1u << (x - t0);
        else if (x == t0 - 1) prev ^= 1u;
    }
}

// Number of up spins in sites [0, t) of an (unflipped) bit-packed row.
__device__ __forceinline__ int count_up_before(const uint64_t *row, int t) {
    int n = 0;
    for (int w = 0; w < (t >> 6); ++w) n += __popcll(row[w]);
    if (t & 63) n += __popcll(row[t >> 6] & ((1ull << (t & 63)) - 1ull));
    return n;
}

}  // namespace psr
