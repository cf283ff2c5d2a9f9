// Internal helpers of the C ABI shared by the psr_api*.cu files: the
// context object, workspace carving, host/device staging, argument checks,
// per-stage events, the connected-configuration generator sequence and the
// autotuner's measurement loop.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "psr_internal.cuh"

struct psr_context {
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 1;
    void *ws = nullptr;
    size_t ws_size = 0;
    int *status = nullptr;  // device status word
    bool profiling = false;
    bool capturing = false;  // a CUDA graph is being captured on the stream
    cudaEvent_t ev_begin[PSR_STAGE_COUNT] = {};
    cudaEvent_t ev_end[PSR_STAGE_COUNT] = {};
    bool stage_ran[PSR_STAGE_COUNT] = {};
    uint64_t ws_generation = 0;  // bumped whenever the workspace moves
    bool graphs = false;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<unsigned char> graph_key;  // arguments the cached graph was built for
    uint64_t graph_ws_generation = 0;
    // Autotuner: measured choices per (operation, shape), kept for the
    // context's lifetime.
    bool autotune = false;
    struct Tuned {
        int op;
        int64_t k0, k1, k2;
        int32_t v0, v1;
        float ms;
    };
    std::vector<Tuned> tuned;
    cudaEvent_t tune_ev[2] = {};
    // shape of the fused forward kernels fixed by psr_context_set_fwd_shape
    // ([0] FP32, [1] BF16; 0 = chosen per call: tuned, else the default)
    int fwd_shape_fixed[2] = {0, 0};
    // second workspace: arrays psr_vmc_step keeps across the calls it makes
    void *ws2 = nullptr;
    size_t ws2_size = 0;
};

namespace psr {
namespace apiutil {

// Bump allocator over the workspace.  Each entry point runs its carving
// sequence twice: once with a null base to size it, once for real.
struct Carver {
    char *base = nullptr;
    size_t off = 0;
    template <class T>
    T *get(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

inline int from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return PSR_OK;
    if (e == cudaErrorMemoryAllocation) return PSR_ENOMEM;
    return PSR_ECUDA;
}

#define PSR_TRY(expr)                          \
    do {                                       \
        int _rc = from_cuda(expr);             \
        if (_rc != PSR_OK) return _rc;         \
    } while (0)

inline bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline int ensure_ws(psr_context *ctx, size_t bytes) {
    if (bytes <= ctx->ws_size) return PSR_OK;
    PSR_TRY(cudaStreamSynchronize(ctx->stream));
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_size = 0;
    size_t want = bytes + bytes / 8 + (1u << 20);
    cudaError_t e = cudaMalloc(&ctx->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return PSR_ENOMEM;
    }
    ctx->ws_size = want;
    ctx->ws_generation++;
    return PSR_OK;
}

// Reads and clears the device status word (synchronises the stream).
inline int take_status(psr_context *ctx) {
    PSR_TRY(cudaStreamSynchronize(ctx->stream));
    int st = 0;
    PSR_TRY(cudaMemcpy(&st, ctx->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) PSR_TRY(cudaMemset(ctx->status, 0, sizeof(int)));
    return st;
}

inline int check_params(const psr_params *p, int64_t n, int32_t L) {
    if (!p || !p->ctx || !p->theta) return PSR_EINVAL;
    if (p->n_layers < 1 || p->n_layers > kMaxLayers) return PSR_EINVAL;
    if (p->hidden != 32 && p->hidden != 64 && p->hidden != 128) return PSR_EINVAL;
    if (p->u1_mask != 0 && p->u1_mask != 1) return PSR_EINVAL;
    if (p->precision == PSR_FP16) return PSR_EUNSUPPORTED;  // the 2D model's forward only
    if (p->precision != PSR_FP32 && p->precision != PSR_BF16) return PSR_EINVAL;
    if (n < 1 || L < 1) return PSR_EINVAL;
    if (n > (int64_t)1 << 31) return PSR_EINVAL;
    if (p->u1_mask && (L % 2)) return PSR_EINVAL;
    if (p->precision == PSR_BF16 &&
        (p->hidden != 128 || p->n_layers != 3 || bf16_packed_bytes() == 0))
        return PSR_EUNSUPPORTED;
    return PSR_OK;
}

inline int check_ham(const psr_hamiltonian *h) {
    if (!h) return PSR_EINVAL;
    if (h->kind != PSR_HEISENBERG && h->kind != PSR_TFIM) return PSR_EINVAL;
    if (h->Lx < 1 || h->Ly < 1 || (int64_t)h->Lx * h->Ly > (1 << 24)) return PSR_EINVAL;
    if (h->pbc != 0 && h->pbc != 1) return PSR_EINVAL;
    if (h->marshall != 0 && h->marshall != 1) return PSR_EINVAL;
    if (h->kind == PSR_HEISENBERG && h->marshall) {
        // bipartite unless a wrapped dimension has odd length
        const bool wx = h->pbc && h->Lx >= 3, wy = h->pbc && h->Ly >= 3;
        if ((wx && (h->Lx & 1)) || (wy && (h->Ly & 1))) return PSR_EINVAL;
    }
    return PSR_OK;
}

inline int64_t words_per_row(int N) { return (N + 63) / 64 + 1; }

// Stages an input array: returns the device pointer to use (the caller's own
// if it is device memory, else a workspace copy filled by an async H2D).
template <class T>
inline int stage_in(const T *src, T *dst_ws, size_t count, bool dev, cudaStream_t st, const T **use) {
    if (dev) {
        *use = src;
        return PSR_OK;
    }
    PSR_TRY(cudaMemcpyAsync(dst_ws, src, count * sizeof(T), cudaMemcpyHostToDevice, st));
    *use = dst_ws;
    return PSR_OK;
}

// Records the begin/end event of a stage when profiling is on.
struct StageScope {
    psr_context *ctx;
    int stage;
    StageScope(psr_context *c, int s) : ctx(c), stage(s) {
        if (ctx->profiling && !ctx->capturing) {
            cudaEventRecord(ctx->ev_begin[stage], ctx->stream);
            ctx->stage_ran[stage] = true;
        }
    }
    ~StageScope() {
        if (ctx->profiling && !ctx->capturing) cudaEventRecord(ctx->ev_end[stage], ctx->stream);
    }
};

inline void reset_stages(psr_context *ctx) {
    for (int i = 0; i < PSR_STAGE_COUNT; ++i) ctx->stage_ran[i] = false;
}

// Shared body of psr_connected and the first half of every local-energy call.
struct ConnBufs {
    int32_t *bonds;
    int64_t *counts;
    int64_t *offsets;
    float *diag;
    int32_t *entries;
};

inline int enqueue_connected(psr_context *ctx, const psr_hamiltonian *ham, const uint8_t *sp, int64_t n,
                      const ConnBufs &b, HamDev &hd) {
    cudaStream_t st = ctx->stream;
    const int N = ham->Lx * ham->Ly;
    hd.kind = ham->kind;
    hd.N = N;
    hd.nb = bond_count(ham->Lx, ham->Ly, ham->pbc);
    hd.bonds = b.bonds;
    hd.J = (float)ham->J;
    hd.h = (float)ham->h;
    hd.coeff = ham->kind == PSR_HEISENBERG ? (float)((ham->marshall ? -0.5 : 0.5) * ham->J)
                                           : (float)(-ham->h);
    if (hd.nb > 0) PSR_TRY(launch_bonds(ham->Lx, ham->Ly, ham->pbc, b.bonds, st));
    PSR_TRY(launch_count_connected(hd, sp, n, b.counts, b.diag, st));
    PSR_TRY(launch_exclusive_scan(b.counts, n, b.offsets, st));
    PSR_TRY(launch_fill_connected(hd, sp, n, b.offsets, b.entries, st));
    return PSR_OK;
}

inline int64_t max_entries_per_sample(const psr_hamiltonian *ham) {
    const int N = ham->Lx * ham->Ly;
    return ham->kind == PSR_HEISENBERG ? bond_count(ham->Lx, ham->Ly, ham->pbc) : N;
}

// ---------------------------------------------------------------- autotuner

enum { kTuneScan = 1, kTuneSample = 2, kTuneSample2d = 3, kTuneSampleLru = 4, kTuneFwd = 5 };

// Times run(i) for every candidate i on the context's stream with CUDA
// events (two runs each when a run is short, the second counted) and
// returns the index of the fastest.  Synchronises the stream.
template <class Run>
int measure_candidates(psr_context *ctx, int count, Run run, int *best, float *best_ms) {
    if (!ctx->tune_ev[0]) {
        PSR_TRY(cudaEventCreate(&ctx->tune_ev[0]));
        PSR_TRY(cudaEventCreate(&ctx->tune_ev[1]));
    }
    cudaStream_t st = ctx->stream;
    *best = 0;
    *best_ms = -1.0f;
    for (int i = 0; i < count; ++i) {
        float ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {
            PSR_TRY(cudaEventRecord(ctx->tune_ev[0], st));
            int rc = run(i);
            if (rc != PSR_OK) return rc;
            PSR_TRY(cudaEventRecord(ctx->tune_ev[1], st));
            PSR_TRY(cudaEventSynchronize(ctx->tune_ev[1]));
            PSR_TRY(cudaEventElapsedTime(&ms, ctx->tune_ev[0], ctx->tune_ev[1]));
            if (ms > 50.0f) break;  // long runs: the first is representative
        }
        if (*best_ms < 0.0f || ms < *best_ms) {
            *best_ms = ms;
            *best = i;
        }
    }
    return PSR_OK;
}

inline const psr_context::Tuned *find_tuned(const psr_context *ctx, int op, int64_t k0, int64_t k1,
                                     int64_t k2) {
    for (const auto &t : ctx->tuned)
        if (t.op == op && t.k0 == k0 && t.k1 == k1 && t.k2 == k2) return &t;
    return nullptr;
}

// ------------------------------------------- shapes of the fused forwards
// BF16 (tcgen05) forward: sequences per MMA stream, 1 (four streams, N = 32)
// or 2 (two streams, N = 64).  FP32 forward: scan chunk, 32 or 16 sites.
// Every shape computes the same function; the FP32 chunk changes only the
// summation order of a configuration's log P (the resume points are chunk
// starts), the BF16 shapes give identical results.
constexpr int kFwdShapeDefault[2] = {kChunkF32, 1};
constexpr int kFwdShapes[2][2] = {{kChunkF32, kChunkGrad}, {1, 2}};

inline bool fwd_shape_valid(bool bf16, int shape) {
    return shape == kFwdShapes[bf16][0] || shape == kFwdShapes[bf16][1];
}

// Key of the forward launches of one call: precision, kind of call (0: log
// psi of the samples, 1: samples + connected configurations) and the
// (sites, samples) of every sample set.
struct FwdKey {
    int64_t k0, k1, k2;
};
inline FwdKey fwd_key(bool bf16, int what, int groups, const int *N, const int64_t *n) {
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the sizes
    for (int g = 0; g < groups; ++g) {
        h = (h ^ (uint64_t)N[g]) * 1099511628211ull;
        h = (h ^ (uint64_t)n[g]) * 1099511628211ull;
    }
    return FwdKey{bf16 ? 1 : 0, what, (int64_t)(h >> 1)};
}

// The shape a call uses: the fixed one, else the tuned one, else the default.
inline int fwd_shape(const psr_context *ctx, bool bf16, const FwdKey &k, bool *tuned) {
    *tuned = false;
    if (ctx->fwd_shape_fixed[bf16]) return ctx->fwd_shape_fixed[bf16];
    if (const psr_context::Tuned *t = find_tuned(ctx, kTuneFwd, k.k0, k.k1, k.k2)) {
        *tuned = true;
        return t->v0;
    }
    return kFwdShapeDefault[bf16];
}

// With the autotuner on and the shape neither fixed nor tuned (and no graph
// being captured), times run(shape) for both shapes and records the faster;
// *shape receives the shape to use.  run must enqueue the call's complete
// forward launches (idempotent).  Synchronises the stream when it tunes.
template <class Run>
inline int tune_fwd_shape(psr_context *ctx, bool bf16, const FwdKey &k, Run run, int *shape) {
    bool tuned = false;
    *shape = fwd_shape(ctx, bf16, k, &tuned);
    if (!ctx->autotune || tuned || ctx->capturing || ctx->fwd_shape_fixed[bf16]) return PSR_OK;
    int best = 0;
    float ms = 0.0f;
    int rc = measure_candidates(ctx, 2, [&](int i) { return run(kFwdShapes[bf16][i]); }, &best, &ms);
    if (rc != PSR_OK) return rc;
    psr_context::Tuned t{kTuneFwd, k.k0, k.k1, k.k2, kFwdShapes[bf16][best], 0, ms};
    ctx->tuned.push_back(t);
    *shape = t.v0;
    return PSR_OK;
}

// ------------------------------------------- tensor-core gradient (H = 128)
// Per-sample O_k rows on the tensor cores: used by psr_grad (BF16 precision,
// dout == NULL) and by psr_step_batch for its BF16 gradient items.  Samples
// go through in batches whose stash and layer arrays fit kTcBudget bytes.
constexpr size_t kTcBudget = size_t(16) << 30;

inline bool grad_tc_applies(const psr_params *p, const float *dout) {
    return p->precision == PSR_BF16 && p->hidden == 128 && dout == nullptr;
}

struct GradTcWs {
    int64_t B;          // samples per batch
    float *stash, *gx[2], *gy[2], *gh, *dz, *dc;
    void *images;
};

inline int64_t grad_tc_batch(int nL, int L, int64_t n) {
    const size_t per = (stash_floats_per_sample(nL, 128, L) + 7 * (size_t)128 * stash_npad(L)) * sizeof(float);
    int64_t B = (int64_t)(kTcBudget / per);
    if (B < 1) B = 1;
    if (B > n) B = n;
    return B;
}

// Carves the batch buffers (call with a null-base Carver to size them).
inline void grad_tc_carve(Carver &c, int nL, int L, int64_t B, GradTcWs &w) {
    const size_t arr = (size_t)B * 128 * stash_npad(L);
    w.B = B;
    w.images = c.get<char>(bwd_tc_image_bytes(nL));
    w.stash = c.get<float>((size_t)B * stash_floats_per_sample(nL, 128, L));
    w.gx[0] = c.get<float>(arr);
    w.gx[1] = c.get<float>(arr);
    w.gy[0] = c.get<float>(arr);
    w.gy[1] = c.get<float>(arr);
    w.gh = c.get<float>(arr);
    w.dz = c.get<float>(arr);
    w.dc = c.get<float>(arr);
}

// Enqueues the O_k rows of n samples of L sites (bit-packed `bits`, W words
// per row) into rows [n][P]; pk / theta: packed FP32 weights and the flat
// parameters.  The transposed images are packed here.
inline int enqueue_grad_tc(psr_context *ctx, int nL, int u1, const float *theta, const float *pk,
                           const uint64_t *bits, int64_t n, int L, int W, float *rows, GradTcWs &w) {
    cudaStream_t st = ctx->stream;
    const ThetaLayout tl = theta_layout(nL, 128);
    const F32Layout fl = f32_layout(nL, 128);
    PSR_TRY(launch_pack_bwd_tc(theta, tl, w.images, st));
    for (int64_t s0 = 0; s0 < n; s0 += w.B) {
        const int64_t b = (n - s0 < w.B) ? n - s0 : w.B;
        BwdTcArgs A{};
        A.n = (int)b;
        A.N = L;
        A.Np = stash_npad(L);
        A.W = W;
        A.nL = nL;
        A.P = tl.total;
        A.tl = tl;
        A.stash = w.stash;
        A.stash_stride = (int64_t)stash_floats_per_sample(nL, 128, L);
        A.wd = pk + fl.wd;
        A.images = static_cast<const uint8_t *>(w.images);
        A.bits = bits + s0 * W;
        A.rows = rows + s0 * tl.total;
        A.gh = w.gh;
        A.dz = w.dz;
        A.dc = w.dc;
        A.pk = pk;
        A.fl = fl;
        A.u1 = u1;
        A.status = ctx->status;
        PSR_TRY(launch_fwd_tc(A, ctx->num_sms, st));  // fills the stash of the batch
        for (int l = nL - 1; l >= 0; --l) {
            A.l = l;
            A.gx_in = w.gx[(l + 1) & 1];
            A.gx_out = w.gx[l & 1];
            A.gy = w.gy[l & 1];
            A.gy_up = w.gy[(l + 1) & 1];
            PSR_TRY(launch_bwd_tc_layer(A, ctx->num_sms, st));
        }
    }
    return PSR_OK;
}

}  // namespace apiutil
}  // namespace psr
