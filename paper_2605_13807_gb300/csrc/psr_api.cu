// C ABI of libpsr: argument checks, workspace, host/device staging and the
// launch sequence of each entry point.  All compute happens in the kernels
// of psr_fwd_f32.cu, psr_fwd_bf16.cu, psr_ham.cu and psr_bwd.cu.
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
    // second workspace: arrays psr_vmc_step keeps across the calls it makes
    void *ws2 = nullptr;
    size_t ws2_size = 0;
};

namespace {

using namespace psr;

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

int from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return PSR_OK;
    if (e == cudaErrorMemoryAllocation) return PSR_ENOMEM;
    return PSR_ECUDA;
}

#define PSR_TRY(expr)                          \
    do {                                       \
        int _rc = from_cuda(expr);             \
        if (_rc != PSR_OK) return _rc;         \
    } while (0)

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int ensure_ws(psr_context *ctx, size_t bytes) {
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
int take_status(psr_context *ctx) {
    PSR_TRY(cudaStreamSynchronize(ctx->stream));
    int st = 0;
    PSR_TRY(cudaMemcpy(&st, ctx->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) PSR_TRY(cudaMemset(ctx->status, 0, sizeof(int)));
    return st;
}

int check_params(const psr_params *p, int64_t n, int32_t L) {
    if (!p || !p->ctx || !p->theta) return PSR_EINVAL;
    if (p->n_layers < 1 || p->n_layers > kMaxLayers) return PSR_EINVAL;
    if (p->hidden != 32 && p->hidden != 64 && p->hidden != 128) return PSR_EINVAL;
    if (p->u1_mask != 0 && p->u1_mask != 1) return PSR_EINVAL;
    if (p->precision != PSR_FP32 && p->precision != PSR_BF16) return PSR_EINVAL;
    if (n < 1 || L < 1) return PSR_EINVAL;
    if (n > (int64_t)1 << 31) return PSR_EINVAL;
    if (p->u1_mask && (L % 2)) return PSR_EINVAL;
    if (p->precision == PSR_BF16 &&
        (p->hidden != 128 || p->n_layers != 3 || bf16_packed_bytes() == 0))
        return PSR_EUNSUPPORTED;
    return PSR_OK;
}

int check_ham(const psr_hamiltonian *h) {
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

int64_t words_per_row(int N) { return (N + 63) / 64 + 1; }

// Stages an input array: returns the device pointer to use (the caller's own
// if it is device memory, else a workspace copy filled by an async H2D).
template <class T>
int stage_in(const T *src, T *dst_ws, size_t count, bool dev, cudaStream_t st, const T **use) {
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

void reset_stages(psr_context *ctx) {
    for (int i = 0; i < PSR_STAGE_COUNT; ++i) ctx->stage_ran[i] = false;
}

}  // namespace

extern "C" {

const char *psr_strerror(int code) {
    switch (code) {
        case PSR_OK: return "ok";
        case PSR_EINVAL: return "invalid argument";
        case PSR_ENOMEM: return "device allocation failed";
        case PSR_ECUDA: return "CUDA runtime error";
        case PSR_ETIMEOUT: return "bounded device wait expired";
        case PSR_EDEVICE: return "device-side check failed";
        case PSR_EUNSUPPORTED: return "unsupported configuration";
        default: return "unknown error";
    }
}

int psr_param_count(int32_t n_layers, int32_t hidden, int64_t *P) {
    if (!P || n_layers < 1 || n_layers > kMaxLayers || hidden < 1) return PSR_EINVAL;
    *P = theta_layout(n_layers, hidden).total;
    return PSR_OK;
}

int psr_context_create(psr_context **out, void *stream) {
    if (!out) return PSR_EINVAL;
    *out = nullptr;
    psr_context *ctx = new (std::nothrow) psr_context();
    if (!ctx) return PSR_ENOMEM;
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    int rc = from_cuda(cudaGetDevice(&ctx->device));
    if (rc == PSR_OK)
        rc = from_cuda(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
    if (rc == PSR_OK) rc = from_cuda(cudaMalloc(&ctx->status, sizeof(int)));
    if (rc == PSR_OK) rc = from_cuda(cudaMemset(ctx->status, 0, sizeof(int)));
    if (rc != PSR_OK) {
        if (ctx->status) cudaFree(ctx->status);
        delete ctx;
        return rc;
    }
    *out = ctx;
    return PSR_OK;
}

int psr_context_set_profiling(psr_context *ctx, int enable) {
    if (!ctx || (enable != 0 && enable != 1)) return PSR_EINVAL;
    if (enable && !ctx->ev_begin[0]) {
        for (int i = 0; i < PSR_STAGE_COUNT; ++i) {
            PSR_TRY(cudaEventCreate(&ctx->ev_begin[i]));
            PSR_TRY(cudaEventCreate(&ctx->ev_end[i]));
        }
    }
    ctx->profiling = enable != 0;
    reset_stages(ctx);
    return PSR_OK;
}

int psr_context_stage_ms(psr_context *ctx, int stage, float *ms) {
    if (!ctx || !ms || !ctx->profiling || stage < 0 || stage >= PSR_STAGE_COUNT) return PSR_EINVAL;
    *ms = 0.0f;
    if (!ctx->stage_ran[stage]) return PSR_OK;
    PSR_TRY(cudaEventSynchronize(ctx->ev_end[stage]));
    PSR_TRY(cudaEventElapsedTime(ms, ctx->ev_begin[stage], ctx->ev_end[stage]));
    return PSR_OK;
}

int psr_context_set_graphs(psr_context *ctx, int enable) {
    if (!ctx || (enable != 0 && enable != 1)) return PSR_EINVAL;
    ctx->graphs = enable != 0;
    return PSR_OK;
}

int psr_context_destroy(psr_context *ctx) {
    if (!ctx) return PSR_EINVAL;
    int rc = from_cuda(cudaStreamSynchronize(ctx->stream));
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    for (int i = 0; i < PSR_STAGE_COUNT; ++i) {
        if (ctx->ev_begin[i]) cudaEventDestroy(ctx->ev_begin[i]);
        if (ctx->ev_end[i]) cudaEventDestroy(ctx->ev_end[i]);
    }
    for (int i = 0; i < 2; ++i)
        if (ctx->tune_ev[i]) cudaEventDestroy(ctx->tune_ev[i]);
    if (ctx->ws2) cudaFree(ctx->ws2);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->status) cudaFree(ctx->status);
    delete ctx;
    return rc;
}

int psr_context_sync(psr_context *ctx) {
    if (!ctx) return PSR_EINVAL;
    return take_status(ctx);
}

int psr_logpsi(const psr_params *params, const uint8_t *spins, int64_t n, int32_t L, float *out) {
    int rc = check_params(params, n, L);
    if (rc != PSR_OK) return rc;
    if (!spins || !out) return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden;
    const bool bf16 = params->precision == PSR_BF16;
    const bool d_theta = is_device_ptr(params->theta), d_spins = is_device_ptr(spins),
               d_out = is_device_ptr(out);
    const ThetaLayout tl = theta_layout(nL, H);
    const F32Layout fl = f32_layout(nL, H);
    const int W = (int)words_per_row(L);

    float *theta_ws = nullptr, *pk = nullptr, *out_ws = nullptr;
    uint8_t *spins_ws = nullptr;
    void *pkb = nullptr;
    uint64_t *bits = nullptr;
    unsigned long long *counter = nullptr;
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : tl.total);
        spins_ws = c.get<uint8_t>(d_spins ? 0 : (size_t)n * L);
        out_ws = c.get<float>(d_out ? 0 : n);
        pk = c.get<float>(fl.total);
        pkb = c.get<char>(bf16 ? bf16_packed_bytes() : 0);
        bits = c.get<uint64_t>((size_t)n * W);
        counter = c.get<unsigned long long>(1);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);

    cudaStream_t st = ctx->stream;
    const float *theta = nullptr;
    const uint8_t *sp = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, tl.total, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(spins, spins_ws, (size_t)n * L, d_spins, st, &sp)) != PSR_OK) return rc;
    float *o = d_out ? out : out_ws;

    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_PACK);
        PSR_TRY(launch_pack_theta_f32(theta, tl, fl, pk, st));
        if (bf16) PSR_TRY(launch_pack_theta_bf16(theta, tl, pkb, st));
        PSR_TRY(launch_bitpack(sp, n, L, W, bits, ctx->status, st));
        PSR_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    }
    FwdJobs jb{};
    jb.mode = 0;
    jb.n_groups = 1;
    jb.g[0].u1 = params->u1_mask;
    jb.g[0].N = L;
    jb.g[0].W = W;
    jb.g[0].n_jobs = n;
    jb.g[0].bits = bits;
    jb.g[0].out = o;
    jb.job_counter = counter;
    jb.status = ctx->status;
    {
        StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
        if (bf16) PSR_TRY(launch_fwd_bf16(jb, pkb, pk, fl, ctx->num_sms, st));
        else PSR_TRY(launch_fwd_f32(jb, pk, fl, ctx->num_sms, st));
    }
    if (!d_out) {
        PSR_TRY(cudaMemcpyAsync(out, out_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    }
    if (!d_out || !d_spins || !d_theta) return take_status(ctx);
    return PSR_OK;
}

// Shared body of psr_connected and the first half of psr_local_energy.
namespace {
struct ConnBufs {
    int32_t *bonds;
    int64_t *counts;
    int64_t *offsets;
    float *diag;
    int32_t *entries;
};

int enqueue_connected(psr_context *ctx, const psr_hamiltonian *ham, const uint8_t *sp, int64_t n,
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

int64_t max_entries_per_sample(const psr_hamiltonian *ham) {
    const int N = ham->Lx * ham->Ly;
    return ham->kind == PSR_HEISENBERG ? bond_count(ham->Lx, ham->Ly, ham->pbc) : N;
}
}  // namespace

int psr_connected(psr_context *ctx, const uint8_t *samples, int64_t n, const psr_hamiltonian *ham,
                  int64_t *offsets, int32_t *entries, int64_t capacity, float *diag,
                  int64_t *total) {
    if (!ctx || !samples || !offsets || !entries || !diag || !total || n < 1) return PSR_EINVAL;
    int rc = check_ham(ham);
    if (rc != PSR_OK) return rc;
    const int N = ham->Lx * ham->Ly;
    const int64_t cap = n * max_entries_per_sample(ham);
    if (capacity < cap) return PSR_EINVAL;
    const bool d_s = is_device_ptr(samples), d_o = is_device_ptr(offsets),
               d_e = is_device_ptr(entries), d_d = is_device_ptr(diag);
    const int nb = bond_count(ham->Lx, ham->Ly, ham->pbc);
    uint8_t *s_ws = nullptr;
    ConnBufs b{};
    int64_t *off_ws = nullptr;
    int32_t *ent_ws = nullptr;
    float *diag_ws = nullptr;
    auto carve = [&](Carver &c) {
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        b.bonds = c.get<int32_t>(2 * (size_t)nb + 2);
        b.counts = c.get<int64_t>(n);
        off_ws = c.get<int64_t>(d_o ? 0 : n + 1);
        ent_ws = c.get<int32_t>(d_e ? 0 : 3 * (size_t)cap);
        diag_ws = c.get<float>(d_d ? 0 : n);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    const uint8_t *sp = nullptr;
    if ((rc = stage_in(samples, s_ws, (size_t)n * N, d_s, st, &sp)) != PSR_OK) return rc;
    b.offsets = d_o ? offsets : off_ws;
    b.entries = d_e ? entries : ent_ws;
    b.diag = d_d ? diag : diag_ws;
    HamDev hd{};
    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_GENERATOR);
        if ((rc = enqueue_connected(ctx, ham, sp, n, b, hd)) != PSR_OK) return rc;
    }
    int64_t tot = 0;
    PSR_TRY(cudaMemcpyAsync(&tot, b.offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PSR_TRY(cudaStreamSynchronize(st));
    *total = tot;
    if (!d_o) PSR_TRY(cudaMemcpyAsync(offsets, off_ws, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    if (!d_e && tot > 0)
        PSR_TRY(cudaMemcpyAsync(entries, ent_ws, 3 * (size_t)tot * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (!d_d) PSR_TRY(cudaMemcpyAsync(diag, diag_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    return take_status(ctx);
}

int psr_local_energy(const psr_params *params, const uint8_t *samples, int64_t n,
                     const psr_hamiltonian *ham, float *out, double *stats) {
    int rc = check_ham(ham);
    if (rc != PSR_OK) return rc;
    const int N = ham->Lx * ham->Ly;
    if ((rc = check_params(params, n, N)) != PSR_OK) return rc;
    if (!samples || !out) return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden;
    const bool bf16 = params->precision == PSR_BF16;
    const int CH = bf16 ? kChunkBF16 : kChunkF32;
    const int nch = (N + CH - 1) / CH;
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(samples),
               d_out = is_device_ptr(out), d_stats = stats ? is_device_ptr(stats) : true;
    const ThetaLayout tl = theta_layout(nL, H);
    const F32Layout fl = f32_layout(nL, H);
    const int W = (int)words_per_row(N);
    const int nb = bond_count(ham->Lx, ham->Ly, ham->pbc);
    const int64_t cap = n * max_entries_per_sample(ham);

    float *theta_ws = nullptr, *out_ws = nullptr, *pk = nullptr, *lpsi = nullptr, *logp = nullptr,
          *carries = nullptr, *delta = nullptr;
    double *stats_ws = nullptr;
    uint8_t *s_ws = nullptr;
    void *pkb = nullptr;
    uint64_t *bits = nullptr;
    unsigned long long *counters = nullptr;
    ConnBufs b{};
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : tl.total);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        out_ws = c.get<float>(d_out ? 0 : n);
        stats_ws = c.get<double>(d_stats ? 0 : 3);
        pk = c.get<float>(fl.total);
        pkb = c.get<char>(bf16 ? bf16_packed_bytes() : 0);
        bits = c.get<uint64_t>((size_t)n * W);
        b.bonds = c.get<int32_t>(2 * (size_t)nb + 2);
        b.counts = c.get<int64_t>(n);
        b.offsets = c.get<int64_t>(n + 1);
        b.diag = c.get<float>(n);
        b.entries = c.get<int32_t>(3 * (size_t)cap);
        lpsi = c.get<float>(n);
        logp = c.get<float>((size_t)n * N);
        carries = c.get<float>((size_t)n * nch * nL * H);
        delta = c.get<float>(cap);
        counters = c.get<unsigned long long>(2);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);

    cudaStream_t st = ctx->stream;
    const float *theta = nullptr;
    const uint8_t *sp = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, tl.total, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(samples, s_ws, (size_t)n * N, d_s, st, &sp)) != PSR_OK) return rc;
    float *o = d_out ? out : out_ws;
    double *so = stats ? (d_stats ? stats : stats_ws) : nullptr;

    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_PACK);
        PSR_TRY(launch_pack_theta_f32(theta, tl, fl, pk, st));
        if (bf16) PSR_TRY(launch_pack_theta_bf16(theta, tl, pkb, st));
        PSR_TRY(launch_bitpack(sp, n, N, W, bits, ctx->status, st));
        PSR_TRY(cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st));
    }
    HamDev hd{};
    {
        StageScope sc(ctx, PSR_STAGE_GENERATOR);
        if ((rc = enqueue_connected(ctx, ham, sp, n, b, hd)) != PSR_OK) return rc;
    }

    FwdJobs js{};
    js.mode = 0;
    js.n_groups = 1;
    js.g[0].u1 = params->u1_mask;
    js.g[0].N = N;
    js.g[0].W = W;
    js.g[0].n_jobs = n;
    js.g[0].bits = bits;
    js.g[0].out = lpsi;
    js.g[0].logp_out = logp;
    js.g[0].carries_out = carries;
    js.job_counter = counters;
    js.status = ctx->status;
    FwdJobs jc{};
    jc.mode = 1;
    jc.n_groups = 1;
    jc.g[0].u1 = params->u1_mask;
    jc.g[0].N = N;
    jc.g[0].W = W;
    jc.g[0].n_jobs = cap;
    jc.g[0].n_jobs_dev = b.offsets + n;
    jc.g[0].bits = bits;
    jc.g[0].entries = b.entries;
    jc.g[0].carries_in = carries;
    jc.g[0].logp_ref = logp;
    jc.g[0].out = delta;
    jc.job_counter = counters + 1;
    jc.status = ctx->status;
    {
        StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
        if (bf16) PSR_TRY(launch_fwd_bf16(js, pkb, pk, fl, ctx->num_sms, st));
        else PSR_TRY(launch_fwd_f32(js, pk, fl, ctx->num_sms, st));
    }
    if (cap > 0) {
        StageScope sc(ctx, PSR_STAGE_FWD_CONNECTED);
        if (bf16) PSR_TRY(launch_fwd_bf16(jc, pkb, pk, fl, ctx->num_sms, st));
        else PSR_TRY(launch_fwd_f32(jc, pk, fl, ctx->num_sms, st));
    }
    {
        StageScope sc(ctx, PSR_STAGE_GATHER);
        PSR_TRY(launch_eloc_gather(b.offsets, delta, b.diag, hd.coeff, n, o, st));
        if (so) PSR_TRY(launch_stats(o, n, so, st));
    }
    if (!d_out) PSR_TRY(cudaMemcpyAsync(out, out_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (stats && !d_stats)
        PSR_TRY(cudaMemcpyAsync(stats, stats_ws, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (!d_out || !d_s || !d_theta || !d_stats) return take_status(ctx);
    return PSR_OK;
}

int psr_grad(const psr_params *params, const uint8_t *spins, int64_t n, int32_t L,
             const float *dout, float *dparams) {
    int rc = check_params(params, n, L);
    if (rc != PSR_OK && rc != PSR_EUNSUPPORTED) return rc;
    if (!spins || !dparams) return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden;
    const ThetaLayout tl = theta_layout(nL, H);
    const F32Layout fl = f32_layout(nL, H);
    const int64_t P = tl.total;
    const int W = (int)words_per_row(L);
    const int nch = (L + kChunkGrad - 1) / kChunkGrad;
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(spins),
               d_dout = dout ? is_device_ptr(dout) : true, d_g = is_device_ptr(dparams);
    int per_sm = 1;
    {
        int occ = 0;
        // backward CTA: H threads and bwd_smem_bytes(H) of shared memory
        int dev_smem = 0;
        cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device);
        occ = (int)(dev_smem / (bwd_smem_bytes(H, nL) + 1024));
        per_sm = occ < 1 ? 1 : (occ > 4 ? 4 : occ);
    }
    int64_t grid64 = (int64_t)ctx->num_sms * per_sm;
    if (grid64 > n) grid64 = n;
    const int grid = (int)grid64;
    const size_t grad_rows = dout ? (size_t)grid : (size_t)n;

    float *theta_ws = nullptr, *dout_ws = nullptr, *g_ws = nullptr, *pk = nullptr, *carries = nullptr,
          *lpsi = nullptr, *tape = nullptr, *partial = nullptr;
    uint8_t *s_ws = nullptr;
    uint64_t *bits = nullptr;
    unsigned long long *counter = nullptr;
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : P);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * L);
        dout_ws = c.get<float>(d_dout ? 0 : n);
        g_ws = c.get<float>(d_g ? 0 : (dout ? P : (size_t)n * P));
        pk = c.get<float>(fl.total);
        bits = c.get<uint64_t>((size_t)n * W);
        carries = c.get<float>((size_t)n * nch * nL * H);
        lpsi = c.get<float>(n);
        tape = c.get<float>((size_t)grid * bwd_tape_floats_per_cta(nL, H));
        partial = c.get<float>(dout ? grad_rows * P : 0);
        counter = c.get<unsigned long long>(1);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);

    cudaStream_t st = ctx->stream;
    const float *theta = nullptr;
    const uint8_t *sp = nullptr;
    const float *dv = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, P, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(spins, s_ws, (size_t)n * L, d_s, st, &sp)) != PSR_OK) return rc;
    if (dout && (rc = stage_in(dout, dout_ws, n, d_dout, st, &dv)) != PSR_OK) return rc;
    float *g = d_g ? dparams : g_ws;

    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_PACK);
        PSR_TRY(launch_pack_theta_f32(theta, tl, fl, pk, st));
        PSR_TRY(launch_bitpack(sp, n, L, W, bits, ctx->status, st));
        PSR_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    }
    FwdJobs jb{};
    jb.mode = 0;
    jb.n_groups = 1;
    jb.g[0].u1 = params->u1_mask;
    jb.g[0].N = L;
    jb.g[0].W = W;
    jb.g[0].n_jobs = n;
    jb.g[0].bits = bits;
    jb.g[0].out = lpsi;
    jb.g[0].carries_out = carries;
    jb.job_counter = counter;
    jb.status = ctx->status;
    {
        StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
        PSR_TRY(launch_fwd_f32(jb, pk, fl, ctx->num_sms, st, kChunkGrad));
    }
    {
        StageScope sc(ctx, PSR_STAGE_BWD);
        float *rows = dout ? partial : g;
        PSR_TRY(cudaMemsetAsync(rows, 0, grad_rows * P * sizeof(float), st));
        PSR_TRY(launch_bwd_f32(bits, n, L, W, params->u1_mask, theta, tl, pk, fl, carries, dv, rows,
                               grid, tape, ctx->status, st));
        if (dout) PSR_TRY(launch_reduce_rows(partial, grid, P, g, st));
    }
    if (!d_g)
        PSR_TRY(cudaMemcpyAsync(dparams, g_ws, (dout ? P : (size_t)n * P) * sizeof(float),
                                cudaMemcpyDeviceToHost, st));
    if (!d_g || !d_s || !d_theta || !d_dout) return take_status(ctx);
    return PSR_OK;
}


int psr_local_energy_batch(const psr_params *params, const psr_batch_item *items, int32_t n_items) {
    if (!params || !items || n_items < 1 || n_items > kMaxGroups) return PSR_EINVAL;
    int rc;
    for (int i = 0; i < n_items; ++i) {
        const psr_batch_item &it = items[i];
        if ((rc = check_ham(&it.ham)) != PSR_OK) return rc;
        if (it.u1_mask != 0 && it.u1_mask != 1) return PSR_EINVAL;
        psr_params pi = *params;
        pi.u1_mask = it.u1_mask;
        if ((rc = check_params(&pi, it.n, it.ham.Lx * it.ham.Ly)) != PSR_OK) return rc;
        if (!it.samples || !it.out) return PSR_EINVAL;
    }
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden;
    const bool bf16 = params->precision == PSR_BF16;
    const int CH = bf16 ? kChunkBF16 : kChunkF32;
    const ThetaLayout tl = theta_layout(nL, H);
    const F32Layout fl = f32_layout(nL, H);
    const bool d_theta = is_device_ptr(params->theta);
    bool d_s[kMaxGroups], d_out[kMaxGroups], d_st[kMaxGroups];
    bool all_device = d_theta;
    for (int i = 0; i < n_items; ++i) {
        d_s[i] = is_device_ptr(items[i].samples);
        d_out[i] = is_device_ptr(items[i].out);
        d_st[i] = items[i].stats ? is_device_ptr(items[i].stats) : true;
        all_device = all_device && d_s[i] && d_out[i] && d_st[i];
    }

    struct ItemWs {
        uint8_t *s_ws;
        float *out_ws;
        double *stats_ws;
        uint64_t *bits;
        ConnBufs b;
        float *lpsi, *logp, *carries, *delta;
        int N, W, nch, nb;
        int64_t cap;
    } w[kMaxGroups];
    for (int i = 0; i < n_items; ++i) {
        const psr_hamiltonian &hm = items[i].ham;
        w[i].N = hm.Lx * hm.Ly;
        w[i].W = (int)words_per_row(w[i].N);
        w[i].nch = (w[i].N + CH - 1) / CH;
        w[i].nb = bond_count(hm.Lx, hm.Ly, hm.pbc);
        w[i].cap = items[i].n * max_entries_per_sample(&hm);
    }
    float *theta_ws = nullptr, *pk = nullptr;
    void *pkb = nullptr;
    unsigned long long *counters = nullptr;
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : tl.total);
        pk = c.get<float>(fl.total);
        pkb = c.get<char>(bf16 ? bf16_packed_bytes() : 0);
        counters = c.get<unsigned long long>(2);
        for (int i = 0; i < n_items; ++i) {
            const int64_t n = items[i].n;
            ItemWs &x = w[i];
            x.s_ws = c.get<uint8_t>(d_s[i] ? 0 : (size_t)n * x.N);
            x.out_ws = c.get<float>(d_out[i] ? 0 : n);
            x.stats_ws = c.get<double>(d_st[i] ? 0 : 3);
            x.bits = c.get<uint64_t>((size_t)n * x.W);
            x.b.bonds = c.get<int32_t>(2 * (size_t)x.nb + 2);
            x.b.counts = c.get<int64_t>(n);
            x.b.offsets = c.get<int64_t>(n + 1);
            x.b.diag = c.get<float>(n);
            x.b.entries = c.get<int32_t>(3 * (size_t)x.cap);
            x.lpsi = c.get<float>(n);
            x.logp = c.get<float>((size_t)n * x.N);
            x.carries = c.get<float>((size_t)n * x.nch * nL * H);
            x.delta = c.get<float>(x.cap);
        }
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;

    // graph replay when the arguments are the ones the cached graph was built for
    const bool use_graph = ctx->graphs && all_device && st != nullptr;
    std::vector<unsigned char> key;
    if (use_graph) {
        const unsigned char *pp = reinterpret_cast<const unsigned char *>(params);
        key.assign(pp, pp + sizeof(psr_params));
        const unsigned char *ip = reinterpret_cast<const unsigned char *>(items);
        key.insert(key.end(), ip, ip + sizeof(psr_batch_item) * n_items);
        if (ctx->graph_exec && key == ctx->graph_key && ctx->graph_ws_generation == ctx->ws_generation) {
            reset_stages(ctx);
            PSR_TRY(cudaGraphLaunch(ctx->graph_exec, st));
            return PSR_OK;
        }
        // kernel attributes are set outside the capture
        if (bf16) PSR_TRY(prepare_fwd_bf16());
        PSR_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        ctx->capturing = true;
    }

    auto enqueue = [&]() -> int {
        int r;
        const float *theta = nullptr;
        if ((r = stage_in(params->theta, theta_ws, tl.total, d_theta, st, &theta)) != PSR_OK) return r;
        const uint8_t *sp[kMaxGroups];
        for (int i = 0; i < n_items; ++i)
            if ((r = stage_in(items[i].samples, w[i].s_ws, (size_t)items[i].n * w[i].N, d_s[i], st,
                              &sp[i])) != PSR_OK)
                return r;
        reset_stages(ctx);
        HamDev hd[kMaxGroups];
        {
            StageScope sc(ctx, PSR_STAGE_PACK);
            PSR_TRY(launch_pack_theta_f32(theta, tl, fl, pk, st));
            if (bf16) PSR_TRY(launch_pack_theta_bf16(theta, tl, pkb, st));
            for (int i = 0; i < n_items; ++i)
                PSR_TRY(launch_bitpack(sp[i], items[i].n, w[i].N, w[i].W, w[i].bits, ctx->status, st));
            PSR_TRY(cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st));
        }
        {
            StageScope sc(ctx, PSR_STAGE_GENERATOR);
            for (int i = 0; i < n_items; ++i) {
                hd[i] = HamDev{};
                if ((r = enqueue_connected(ctx, &items[i].ham, sp[i], items[i].n, w[i].b, hd[i])) != PSR_OK)
                    return r;
            }
        }
        FwdJobs js{}, jc{};
        js.mode = 0;
        jc.mode = 1;
        js.n_groups = jc.n_groups = n_items;
        js.job_counter = counters;
        jc.job_counter = counters + 1;
        js.status = jc.status = ctx->status;
        for (int i = 0; i < n_items; ++i) {
            FwdGroup &a = js.g[i];
            a.u1 = items[i].u1_mask;
            a.N = w[i].N;
            a.W = w[i].W;
            a.n_jobs = items[i].n;
            a.bits = w[i].bits;
            a.out = w[i].lpsi;
            a.logp_out = w[i].logp;
            a.carries_out = w[i].carries;
            FwdGroup &b = jc.g[i];
            b.u1 = items[i].u1_mask;
            b.N = w[i].N;
            b.W = w[i].W;
            b.n_jobs = w[i].cap;
            b.n_jobs_dev = w[i].b.offsets + items[i].n;
            b.bits = w[i].bits;
            b.entries = w[i].b.entries;
            b.carries_in = w[i].carries;
            b.logp_ref = w[i].logp;
            b.out = w[i].delta;
        }
        {
            StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
            if (bf16) PSR_TRY(launch_fwd_bf16(js, pkb, pk, fl, ctx->num_sms, st));
            else PSR_TRY(launch_fwd_f32(js, pk, fl, ctx->num_sms, st));
        }
        {
            StageScope sc(ctx, PSR_STAGE_FWD_CONNECTED);
            if (bf16) PSR_TRY(launch_fwd_bf16(jc, pkb, pk, fl, ctx->num_sms, st));
            else PSR_TRY(launch_fwd_f32(jc, pk, fl, ctx->num_sms, st));
        }
        {
            StageScope sc(ctx, PSR_STAGE_GATHER);
            for (int i = 0; i < n_items; ++i) {
                float *o = d_out[i] ? items[i].out : w[i].out_ws;
                double *so = items[i].stats ? (d_st[i] ? items[i].stats : w[i].stats_ws) : nullptr;
                PSR_TRY(launch_eloc_gather(w[i].b.offsets, w[i].delta, w[i].b.diag, hd[i].coeff,
                                           items[i].n, o, st));
                if (so) PSR_TRY(launch_stats(o, items[i].n, so, st));
            }
        }
        for (int i = 0; i < n_items; ++i) {
            if (!d_out[i])
                PSR_TRY(cudaMemcpyAsync(items[i].out, w[i].out_ws, items[i].n * sizeof(float),
                                        cudaMemcpyDeviceToHost, st));
            if (items[i].stats && !d_st[i])
                PSR_TRY(cudaMemcpyAsync(items[i].stats, w[i].stats_ws, 3 * sizeof(double),
                                        cudaMemcpyDeviceToHost, st));
        }
        return PSR_OK;
    };
    rc = enqueue();
    if (use_graph) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        ctx->capturing = false;
        if (rc != PSR_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return from_cuda(e);
        if (ctx->graph_exec) {
            cudaGraphExecDestroy(ctx->graph_exec);
            ctx->graph_exec = nullptr;
        }
        e = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            ctx->graph_exec = nullptr;
            return from_cuda(e);
        }
        ctx->graph_key = key;
        ctx->graph_ws_generation = ctx->ws_generation;
        PSR_TRY(cudaGraphLaunch(ctx->graph_exec, st));
        return PSR_OK;
    }
    if (rc != PSR_OK) return rc;
    if (!all_device) return take_status(ctx);
    return PSR_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ scan

namespace {

enum { kTuneScan = 1, kTuneSample = 2 };

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

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

const psr_context::Tuned *find_tuned(const psr_context *ctx, int op, int64_t k0, int64_t k1,
                                     int64_t k2) {
    for (const auto &t : ctx->tuned)
        if (t.op == op && t.k0 == k0 && t.k1 == k1 && t.k2 == k2) return &t;
    return nullptr;
}

// Tile shape used without measurement: the widest unit block that still
// gives every resident warp a column, and enough chunks per column to give
// each resident warp about two tiles when columns are scarce.
psr_scan_tile scan_default_tile(const psr_context *ctx, int64_t n, int N, int H) {
    const int64_t resident = (int64_t)ctx->num_sms * 32;  // warps at 4 CTAs of 8 warps per SM
    int units = 4;
    const int widths[4] = {128, 32, 16, 4};
    for (int w : widths)
        if (H % w == 0 && n * (H / w) >= resident) {
            units = w;
            break;
        }
    const int64_t cols = n * (H / units);
    int chunk = N;
    if (cols < 2 * resident) {
        const int64_t per_col = (2 * resident + cols - 1) / cols;
        int64_t c = (N + per_col - 1) / per_col;
        c = (c + 31) / 32 * 32;
        if (c < 256) c = 256;
        if (c < N) chunk = (int)c;
    }
    return psr_scan_tile{units, chunk};
}

// Candidate tile shapes measured by the autotuner.
std::vector<psr_scan_tile> scan_candidates(const psr_context *ctx, int64_t n, int N, int H) {
    std::vector<psr_scan_tile> out;
    const int widths[4] = {4, 16, 32, 128};
    const int chunks[4] = {256, 1024, 4096, 0};  // 0: whole sequence
    for (int w : widths) {
        if (H % w) continue;
        for (int c : chunks) {
            const int ch = c == 0 ? N : c;
            if (c != 0 && ch >= N) continue;
            out.push_back(psr_scan_tile{w, ch});
        }
    }
    const psr_scan_tile d = scan_default_tile(ctx, n, N, H);
    bool have = false;
    for (const auto &t : out) have = have || (t.units == d.units && t.chunk == d.chunk);
    if (!have) out.push_back(d);
    return out;
}

// first_ticket > 0 leaves the tiles before it unprocessed (used only by the
// bounded-wait self-test: their look-back flags are never set).
int enqueue_scan(psr_context *ctx, const float *a, const float *b, const float *h0, int64_t n,
                 int N, int H, float *h, psr_scan_tile tile, unsigned long long *counter,
                 int *flags, float *desc, int first_ticket = 0) {
    cudaStream_t st = ctx->stream;
    ScanArgs g{};
    g.a = a;
    g.b = b;
    g.h0 = h0;
    g.h = h;
    g.N = N;
    g.H = H;
    scan_geometry(n, N, H, tile.units, tile.chunk, &g.nch, &g.n_tiles);
    g.C = tile.chunk >= N ? N : tile.chunk;
    g.nub = H / tile.units;
    g.counter = counter;
    g.flags = flags;
    g.desc = desc;
    g.status = ctx->status;
    PSR_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    if (first_ticket > 0 && first_ticket < 256)
        PSR_TRY(cudaMemsetAsync(counter, first_ticket, 1, st));  // low byte (little endian)
    if (g.nch > 1) PSR_TRY(cudaMemsetAsync(flags, 0, (size_t)g.n_tiles * sizeof(int), st));
    PSR_TRY(launch_scan(g, tile.units, ctx->num_sms, st));
    return PSR_OK;
}

int scan_impl(psr_context *ctx, const float *a, const float *b, const float *h0, int64_t n,
              int32_t N, int32_t H, float *h, const psr_scan_tile *forced) {
    if (!ctx || !a || !b || !h) return PSR_EINVAL;
    if (n < 1 || N < 1 || N > (1 << 30) || H < 4 || (H % 4) != 0) return PSR_EINVAL;
    if (forced && !scan_tile_valid(H, forced->units, forced->chunk)) return PSR_EINVAL;
    const bool d_a = is_device_ptr(a), d_b = is_device_ptr(b), d_h = is_device_ptr(h),
               d_h0 = h0 ? is_device_ptr(h0) : true;
    if ((d_a && !aligned16(a)) || (d_b && !aligned16(b)) || (d_h && !aligned16(h)) ||
        (h0 && d_h0 && !aligned16(h0)))
        return PSR_EINVAL;
    const size_t count = (size_t)n * N * H;

    // The tile: forced, tuned (cached or measured now), or the default.
    std::vector<psr_scan_tile> cands;
    psr_scan_tile tile = scan_default_tile(ctx, n, N, H);
    bool tune_now = false;
    if (forced) {
        tile = *forced;
    } else if (const psr_context::Tuned *t = find_tuned(ctx, kTuneScan, n, N, H)) {
        tile = psr_scan_tile{t->v0, t->v1};
    } else if (ctx->autotune && !ctx->capturing) {
        cands = scan_candidates(ctx, n, N, H);
        tune_now = true;
    }
    // Look-back arrays sized for the smallest chunk that may run.
    int64_t max_tiles = 0;
    size_t max_desc = 0;
    {
        std::vector<psr_scan_tile> all = cands;
        all.push_back(tile);
        for (const auto &t : all) {
            int nch;
            int64_t nt;
            scan_geometry(n, N, H, t.units, t.chunk, &nch, &nt);
            if (nch > 1) {
                if (nt > max_tiles) max_tiles = nt;
                const size_t d = (size_t)nt * 3 * t.units;
                if (d > max_desc) max_desc = d;
            }
        }
    }

    float *a_ws = nullptr, *b_ws = nullptr, *h_ws = nullptr, *h0_ws = nullptr, *desc = nullptr;
    unsigned long long *counter = nullptr;
    int *flags = nullptr;
    auto carve = [&](Carver &c) {
        a_ws = c.get<float>(d_a ? 0 : count);
        b_ws = c.get<float>(d_b ? 0 : count);
        h_ws = c.get<float>(d_h ? 0 : count);
        h0_ws = c.get<float>(d_h0 ? 0 : (size_t)n * H);
        counter = c.get<unsigned long long>(1);
        flags = c.get<int>((size_t)max_tiles);
        desc = c.get<float>(max_desc);
    };
    Carver sz;
    carve(sz);
    int rc = ensure_ws(ctx, sz.off);
    if (rc != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    const float *ua = nullptr, *ub = nullptr, *uh0 = nullptr;
    if ((rc = stage_in(a, a_ws, count, d_a, st, &ua)) != PSR_OK) return rc;
    if ((rc = stage_in(b, b_ws, count, d_b, st, &ub)) != PSR_OK) return rc;
    if (h0 && (rc = stage_in(h0, h0_ws, (size_t)n * H, d_h0, st, &uh0)) != PSR_OK) return rc;
    float *uh = d_h ? h : h_ws;

    if (tune_now) {
        // Time every candidate on these inputs and keep the fastest; the
        // run below then produces the result.
        int bi = 0;
        float best = 0.0f;
        rc = measure_candidates(ctx, (int)cands.size(), [&](int i) {
            return enqueue_scan(ctx, ua, ub, uh0, n, N, H, uh, cands[i], counter, flags, desc);
        }, &bi, &best);
        if (rc != PSR_OK) return rc;
        tile = cands[bi];
        ctx->tuned.push_back(psr_context::Tuned{kTuneScan, n, N, H, tile.units, tile.chunk, best});
    }

    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_SCAN);
        if ((rc = enqueue_scan(ctx, ua, ub, uh0, n, N, H, uh, tile, counter, flags, desc)) != PSR_OK)
            return rc;
    }
    if (!d_h) PSR_TRY(cudaMemcpyAsync(h, h_ws, count * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (!d_a || !d_b || !d_h || !d_h0) return take_status(ctx);
    return PSR_OK;
}

}  // namespace

extern "C" {

int psr_selftest_wait_timeout(psr_context *ctx, float *elapsed_ms) {
    if (!ctx || ctx->capturing) return PSR_EINVAL;
    // one sequence, 64 sites, 4 units, two chunks of 32: tile 0 is skipped,
    // so tile 1 waits for a flag that nothing sets
    const int N = 64, H = 4;
    float *a = nullptr, *b = nullptr, *h = nullptr, *desc = nullptr;
    unsigned long long *counter = nullptr;
    int *flags = nullptr;
    auto carve = [&](Carver &c) {
        a = c.get<float>((size_t)N * H);
        b = c.get<float>((size_t)N * H);
        h = c.get<float>((size_t)N * H);
        counter = c.get<unsigned long long>(1);
        flags = c.get<int>(2);
        desc = c.get<float>(2 * 3 * 4);
    };
    Carver sz;
    carve(sz);
    int rc = ensure_ws(ctx, sz.off);
    if (rc != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    if ((rc = take_status(ctx)) != PSR_OK) return rc;  // start from a clean status word
    PSR_TRY(cudaMemsetAsync(a, 0, (size_t)N * H * sizeof(float), st));
    PSR_TRY(cudaMemsetAsync(b, 0, (size_t)N * H * sizeof(float), st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PSR_TRY(cudaEventCreate(&e0));
    PSR_TRY(cudaEventCreate(&e1));
    cudaEventRecord(e0, st);
    rc = enqueue_scan(ctx, a, b, nullptr, 1, N, H, h, psr_scan_tile{4, 32}, counter, flags, desc, 1);
    cudaEventRecord(e1, st);
    const int status = take_status(ctx);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (elapsed_ms) *elapsed_ms = ms;
    if (rc != PSR_OK) return rc;
    return status;
}

int psr_context_set_autotune(psr_context *ctx, int enable) {
    if (!ctx || (enable != 0 && enable != 1)) return PSR_EINVAL;
    ctx->autotune = enable != 0;
    return PSR_OK;
}

int psr_scan(psr_context *ctx, const float *a, const float *b, const float *h0, int64_t n,
             int32_t N, int32_t H, float *h) {
    return scan_impl(ctx, a, b, h0, n, N, H, h, nullptr);
}

int psr_scan_tiled(psr_context *ctx, const float *a, const float *b, const float *h0, int64_t n,
                   int32_t N, int32_t H, float *h, const psr_scan_tile *tile) {
    if (!tile) return PSR_EINVAL;
    return scan_impl(ctx, a, b, h0, n, N, H, h, tile);
}

int psr_scan_tile_for(psr_context *ctx, int64_t n, int32_t N, int32_t H, psr_scan_tile *tile,
                      int32_t *tuned) {
    if (!ctx || !tile || n < 1 || N < 1 || H < 4 || (H % 4) != 0) return PSR_EINVAL;
    const psr_context::Tuned *t = find_tuned(ctx, kTuneScan, n, N, H);
    *tile = t ? psr_scan_tile{t->v0, t->v1} : scan_default_tile(ctx, n, N, H);
    if (tuned) *tuned = t ? 1 : 0;
    return PSR_OK;
}

// --------------------------------------------------------------- sampler

int psr_sample(const psr_params *params, const float *uniforms, int64_t n, int32_t L,
               uint8_t *spins, float *logpsi) {
    int rc = check_params(params, n, L);
    if (rc == PSR_EUNSUPPORTED && params->precision == PSR_BF16) rc = PSR_OK;  // FP32 either way
    if (rc != PSR_OK) return rc;
    if (!uniforms || !spins) return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden;
    const bool d_theta = is_device_ptr(params->theta), d_u = is_device_ptr(uniforms),
               d_s = is_device_ptr(spins), d_lp = logpsi ? is_device_ptr(logpsi) : true;
    const ThetaLayout tl = theta_layout(nL, H);
    const F32Layout fl = f32_layout(nL, H);
    const size_t cells = (size_t)n * L;

    float *theta_ws = nullptr, *u_ws = nullptr, *lp_ws = nullptr, *pk = nullptr;
    uint8_t *s_ws = nullptr;
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : tl.total);
        u_ws = c.get<float>(d_u ? 0 : cells);
        s_ws = c.get<uint8_t>(d_s ? 0 : cells);
        lp_ws = c.get<float>(d_lp ? 0 : n);
        pk = c.get<float>(fl.total);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    const float *theta = nullptr, *uu = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, tl.total, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(uniforms, u_ws, cells, d_u, st, &uu)) != PSR_OK) return rc;
    uint8_t *so = d_s ? spins : s_ws;
    float *lo = logpsi ? (d_lp ? logpsi : lp_ws) : nullptr;

    // samples per CTA: forced by nothing, tuned, or the default
    const int64_t key2 = (int64_t)nL * 1024 + H;
    int per_cta = 8;
    bool tune_now = false;
    if (const psr_context::Tuned *t = find_tuned(ctx, kTuneSample, n, L, key2)) per_cta = t->v0;
    else if (ctx->autotune && !ctx->capturing) tune_now = true;

    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_PACK);
        PSR_TRY(launch_pack_theta_f32(theta, tl, fl, pk, st));
    }
    if (tune_now) {
        const int cands[4] = {4, 8, 16, 32};
        int bi = 0;
        float best = 0.0f;
        rc = measure_candidates(ctx, 4, [&](int i) {
            return from_cuda(launch_sample(cands[i], pk, fl, uu, n, L, params->u1_mask, so, lo, st));
        }, &bi, &best);
        if (rc != PSR_OK) return rc;
        per_cta = cands[bi];
        ctx->tuned.push_back(psr_context::Tuned{kTuneSample, n, L, key2, per_cta, 0, best});
    }
    {
        StageScope sc(ctx, PSR_STAGE_SAMPLE);
        PSR_TRY(launch_sample(per_cta, pk, fl, uu, n, L, params->u1_mask, so, lo, st));
    }
    if (!d_s) PSR_TRY(cudaMemcpyAsync(spins, s_ws, cells, cudaMemcpyDeviceToHost, st));
    if (logpsi && !d_lp) PSR_TRY(cudaMemcpyAsync(logpsi, lp_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (!d_theta || !d_u || !d_s || !d_lp) return take_status(ctx);
    return PSR_OK;
}

int psr_sample_tile_for(psr_context *ctx, int64_t n, int32_t L, int32_t n_layers, int32_t hidden,
                        int32_t *per_cta, int32_t *tuned) {
    if (!ctx || !per_cta || n < 1 || L < 1) return PSR_EINVAL;
    const psr_context::Tuned *t = find_tuned(ctx, kTuneSample, n, L, (int64_t)n_layers * 1024 + hidden);
    *per_cta = t ? t->v0 : 8;
    if (tuned) *tuned = t ? 1 : 0;
    return PSR_OK;
}

// ------------------------------------------- two-dimensional patched minGRU

}  // extern "C"

namespace {

int check_params2d(const psr_params *p, int64_t n, int Lx, int Ly) {
    if (!p || !p->ctx || !p->theta) return PSR_EINVAL;
    if (p->n_layers < 1 || p->n_layers > kMaxLayers) return PSR_EINVAL;
    if (p->hidden != 32 && p->hidden != 64 && p->hidden != 128 && p->hidden != 256) return PSR_EINVAL;
    if (p->hidden == 256 && p->n_layers > 4) return PSR_EUNSUPPORTED;  // shared memory
    if (p->u1_mask != 0 && p->u1_mask != 1) return PSR_EINVAL;
    if (p->precision != PSR_FP32 && p->precision != PSR_BF16) return PSR_EINVAL;
    if (n < 1 || n > (int64_t)1 << 31) return PSR_EINVAL;
    if (Lx < 2 || Ly < 2 || (Lx % 2) || (Ly % 2) || (int64_t)Lx * Ly > (1 << 24)) return PSR_EINVAL;
    if (Lx > 64) return PSR_EUNSUPPORTED;  // at most 32 patches per row
    if (p->precision != PSR_FP32) return PSR_EUNSUPPORTED;
    return PSR_OK;
}

}  // namespace

extern "C" {

int psr2d_param_count(int32_t n_layers, int32_t hidden, int64_t *P) {
    if (!P || n_layers < 1 || n_layers > kMaxLayers || hidden < 1) return PSR_EINVAL;
    *P = param_count2d(n_layers, hidden);
    return PSR_OK;
}

int psr2d_logpsi(const psr_params *params, const uint8_t *spins, int64_t n, int32_t Lx, int32_t Ly,
                 float *out) {
    int rc = check_params2d(params, n, Lx, Ly);
    if (rc != PSR_OK) return rc;
    if (!spins || !out) return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden, N = Lx * Ly;
    const int64_t P = param_count2d(nL, H);
    const F2Layout f = f2_layout(nL, H);
    const int W = (int)words_per_row(N);
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(spins),
               d_out = is_device_ptr(out);
    float *theta_ws = nullptr, *out_ws = nullptr, *pk = nullptr;
    uint8_t *s_ws = nullptr;
    uint64_t *bits = nullptr;
    unsigned long long *counter = nullptr;
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : P);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        out_ws = c.get<float>(d_out ? 0 : n);
        pk = c.get<float>(f.total);
        bits = c.get<uint64_t>((size_t)n * W);
        counter = c.get<unsigned long long>(1);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    const float *theta = nullptr;
    const uint8_t *sp = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, P, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(spins, s_ws, (size_t)n * N, d_s, st, &sp)) != PSR_OK) return rc;
    float *o = d_out ? out : out_ws;
    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_PACK);
        PSR_TRY(launch_pack_theta_f2(theta, f, pk, st));
        PSR_TRY(launch_bitpack(sp, n, N, W, bits, ctx->status, st));  // spin-byte check
        PSR_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    }
    Fwd2Jobs jb{};
    jb.mode = 0;
    jb.g.Lx = Lx;
    jb.g.Ly = Ly;
    jb.g.u1 = params->u1_mask;
    jb.g.n_jobs = n;
    jb.g.spins = sp;
    jb.g.out = o;
    jb.job_counter = counter;
    jb.status = ctx->status;
    {
        StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
        PSR_TRY(launch_fwd2d_f32(jb, pk, f, ctx->num_sms, st));
    }
    if (!d_out) PSR_TRY(cudaMemcpyAsync(out, out_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (!d_out || !d_s || !d_theta) return take_status(ctx);
    return PSR_OK;
}

int psr2d_local_energy(const psr_params *params, const uint8_t *samples, int64_t n,
                       const psr_hamiltonian *ham, float *out, double *stats) {
    int rc = check_ham(ham);
    if (rc != PSR_OK) return rc;
    if ((rc = check_params2d(params, n, ham->Lx, ham->Ly)) != PSR_OK) return rc;
    if (!samples || !out) return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden, Lx = ham->Lx, Ly = ham->Ly;
    const int N = Lx * Ly, Py = Ly / 2, Np = (Lx / 2) * Py;
    const int64_t P = param_count2d(nL, H);
    const F2Layout f = f2_layout(nL, H);
    const int W = (int)words_per_row(N);
    const int nb = bond_count(Lx, Ly, ham->pbc);
    const int64_t cap = n * max_entries_per_sample(ham);
    const size_t ckpt = fwd2d_checkpoint_floats(nL, H);
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(samples),
               d_out = is_device_ptr(out), d_stats = stats ? is_device_ptr(stats) : true;

    float *theta_ws = nullptr, *out_ws = nullptr, *pk = nullptr, *lpsi = nullptr, *logp = nullptr,
          *carries = nullptr, *delta = nullptr;
    double *stats_ws = nullptr;
    uint8_t *s_ws = nullptr;
    uint64_t *bits = nullptr;
    unsigned long long *counters = nullptr;
    ConnBufs b{};
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : P);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        out_ws = c.get<float>(d_out ? 0 : n);
        stats_ws = c.get<double>(d_stats ? 0 : 3);
        pk = c.get<float>(f.total);
        bits = c.get<uint64_t>((size_t)n * W);
        b.bonds = c.get<int32_t>(2 * (size_t)nb + 2);
        b.counts = c.get<int64_t>(n);
        b.offsets = c.get<int64_t>(n + 1);
        b.diag = c.get<float>(n);
        b.entries = c.get<int32_t>(3 * (size_t)cap);
        lpsi = c.get<float>(n);
        logp = c.get<float>((size_t)n * Np);
        carries = c.get<float>((size_t)n * Py * ckpt);
        delta = c.get<float>(cap);
        counters = c.get<unsigned long long>(2);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    const float *theta = nullptr;
    const uint8_t *sp = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, P, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(samples, s_ws, (size_t)n * N, d_s, st, &sp)) != PSR_OK) return rc;
    float *o = d_out ? out : out_ws;
    double *so = stats ? (d_stats ? stats : stats_ws) : nullptr;

    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_PACK);
        PSR_TRY(launch_pack_theta_f2(theta, f, pk, st));
        PSR_TRY(launch_bitpack(sp, n, N, W, bits, ctx->status, st));  // spin-byte check
        PSR_TRY(cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st));
    }
    HamDev hd{};
    {
        StageScope sc(ctx, PSR_STAGE_GENERATOR);
        if ((rc = enqueue_connected(ctx, ham, sp, n, b, hd)) != PSR_OK) return rc;
    }
    Fwd2Jobs js{};
    js.mode = 0;
    js.g.Lx = Lx;
    js.g.Ly = Ly;
    js.g.u1 = params->u1_mask;
    js.g.n_jobs = n;
    js.g.spins = sp;
    js.g.out = lpsi;
    js.g.logp_out = logp;
    js.g.carries_out = carries;
    js.job_counter = counters;
    js.status = ctx->status;
    Fwd2Jobs jc = js;
    jc.mode = 1;
    jc.g.n_jobs = cap;
    jc.g.n_jobs_dev = b.offsets + n;
    jc.g.entries = b.entries;
    jc.g.carries_in = carries;
    jc.g.logp_ref = logp;
    jc.g.out = delta;
    jc.g.logp_out = nullptr;
    jc.g.carries_out = nullptr;
    jc.job_counter = counters + 1;
    {
        StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
        PSR_TRY(launch_fwd2d_f32(js, pk, f, ctx->num_sms, st));
    }
    if (cap > 0) {
        StageScope sc(ctx, PSR_STAGE_FWD_CONNECTED);
        PSR_TRY(launch_fwd2d_f32(jc, pk, f, ctx->num_sms, st));
    }
    {
        StageScope sc(ctx, PSR_STAGE_GATHER);
        PSR_TRY(launch_eloc_gather(b.offsets, delta, b.diag, hd.coeff, n, o, st));
        if (so) PSR_TRY(launch_stats(o, n, so, st));
    }
    if (!d_out) PSR_TRY(cudaMemcpyAsync(out, out_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (stats && !d_stats)
        PSR_TRY(cudaMemcpyAsync(stats, stats_ws, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (!d_out || !d_s || !d_theta || !d_stats) return take_status(ctx);
    return PSR_OK;
}

// ------------------------------------------------------ deep 1D LRU model

}  // extern "C"

namespace {

int check_params_lru(const psr_params *p, int64_t n, int32_t L) {
    if (!p || !p->ctx || !p->theta) return PSR_EINVAL;
    if (p->n_layers < 1 || p->n_layers > kMaxLayers) return PSR_EINVAL;
    if (p->hidden != 32 && p->hidden != 64 && p->hidden != 128) return PSR_EINVAL;
    if (p->u1_mask != 0 && p->u1_mask != 1) return PSR_EINVAL;
    if (p->precision != PSR_FP32 && p->precision != PSR_BF16) return PSR_EINVAL;
    if (n < 1 || L < 1 || n > (int64_t)1 << 31) return PSR_EINVAL;
    if (p->u1_mask && (L % 2)) return PSR_EINVAL;
    if (p->precision != PSR_FP32) return PSR_EUNSUPPORTED;
    return PSR_OK;
}

// Shared body of psr_lru_logpsi (ham == nullptr) and psr_lru_local_energy.
int lru_run(const psr_params *params, const uint8_t *samples, int64_t n, int32_t L,
            const psr_hamiltonian *ham, float *out, double *stats) {
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden, N = L;
    const int64_t P = param_count_lru(nL, H);
    const LruLayout f = lru_layout(nL, H);
    const int W = (int)words_per_row(N);
    const int nch = (N + kChunkLru - 1) / kChunkLru;
    const bool eloc = ham != nullptr;
    const int nb = eloc ? bond_count(ham->Lx, ham->Ly, ham->pbc) : 0;
    const int64_t cap = eloc ? n * max_entries_per_sample(ham) : 0;
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(samples),
               d_out = is_device_ptr(out), d_stats = stats ? is_device_ptr(stats) : true;
    float *theta_ws = nullptr, *out_ws = nullptr, *pk = nullptr, *lpsi = nullptr, *logp = nullptr,
          *carries = nullptr, *delta = nullptr;
    double *stats_ws = nullptr;
    uint8_t *s_ws = nullptr;
    uint64_t *bits = nullptr;
    unsigned long long *counters = nullptr;
    ConnBufs b{};
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : P);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        out_ws = c.get<float>(d_out ? 0 : n);
        stats_ws = c.get<double>(d_stats ? 0 : 3);
        pk = c.get<float>(f.total);
        bits = c.get<uint64_t>((size_t)n * W);
        counters = c.get<unsigned long long>(2);
        if (eloc) {
            b.bonds = c.get<int32_t>(2 * (size_t)nb + 2);
            b.counts = c.get<int64_t>(n);
            b.offsets = c.get<int64_t>(n + 1);
            b.diag = c.get<float>(n);
            b.entries = c.get<int32_t>(3 * (size_t)cap);
            lpsi = c.get<float>(n);
            logp = c.get<float>((size_t)n * N);
            carries = c.get<float>((size_t)n * nch * nL * 2 * H);
            delta = c.get<float>(cap);
        }
    };
    Carver sz;
    carve(sz);
    int rc = ensure_ws(ctx, sz.off);
    if (rc != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    const float *theta = nullptr;
    const uint8_t *sp = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, P, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(samples, s_ws, (size_t)n * N, d_s, st, &sp)) != PSR_OK) return rc;
    float *o = d_out ? out : out_ws;
    double *so = stats ? (d_stats ? stats : stats_ws) : nullptr;
    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_PACK);
        PSR_TRY(launch_pack_theta_lru(theta, f, pk, st));
        PSR_TRY(launch_bitpack(sp, n, N, W, bits, ctx->status, st));
        PSR_TRY(cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st));
    }
    HamDev hd{};
    if (eloc) {
        StageScope sc(ctx, PSR_STAGE_GENERATOR);
        if ((rc = enqueue_connected(ctx, ham, sp, n, b, hd)) != PSR_OK) return rc;
    }
    FwdJobs js{};
    js.mode = 0;
    js.n_groups = 1;
    js.g[0].u1 = params->u1_mask;
    js.g[0].N = N;
    js.g[0].W = W;
    js.g[0].n_jobs = n;
    js.g[0].bits = bits;
    js.g[0].out = eloc ? lpsi : o;
    js.g[0].logp_out = logp;
    js.g[0].carries_out = carries;
    js.job_counter = counters;
    js.status = ctx->status;
    {
        StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
        PSR_TRY(launch_lru_f32(js, pk, f, ctx->num_sms, st));
    }
    if (eloc) {
        FwdJobs jc = js;
        jc.mode = 1;
        jc.g[0].n_jobs = cap;
        jc.g[0].n_jobs_dev = b.offsets + n;
        jc.g[0].entries = b.entries;
        jc.g[0].carries_in = carries;
        jc.g[0].logp_ref = logp;
        jc.g[0].out = delta;
        jc.g[0].logp_out = nullptr;
        jc.g[0].carries_out = nullptr;
        jc.job_counter = counters + 1;
        if (cap > 0) {
            StageScope sc(ctx, PSR_STAGE_FWD_CONNECTED);
            PSR_TRY(launch_lru_f32(jc, pk, f, ctx->num_sms, st));
        }
        StageScope sc(ctx, PSR_STAGE_GATHER);
        PSR_TRY(launch_eloc_gather(b.offsets, delta, b.diag, hd.coeff, n, o, st));
        if (so) PSR_TRY(launch_stats(o, n, so, st));
    }
    if (!d_out) PSR_TRY(cudaMemcpyAsync(out, out_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (stats && !d_stats)
        PSR_TRY(cudaMemcpyAsync(stats, stats_ws, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (!d_out || !d_s || !d_theta || !d_stats) return take_status(ctx);
    return PSR_OK;
}

}  // namespace

extern "C" {

int psr_lru_param_count(int32_t n_layers, int32_t hidden, int64_t *P) {
    if (!P || n_layers < 1 || n_layers > kMaxLayers || hidden < 1) return PSR_EINVAL;
    *P = param_count_lru(n_layers, hidden);
    return PSR_OK;
}

int psr_lru_logpsi(const psr_params *params, const uint8_t *spins, int64_t n, int32_t L, float *out) {
    int rc = check_params_lru(params, n, L);
    if (rc != PSR_OK) return rc;
    if (!spins || !out) return PSR_EINVAL;
    return lru_run(params, spins, n, L, nullptr, out, nullptr);
}

int psr_lru_local_energy(const psr_params *params, const uint8_t *samples, int64_t n,
                         const psr_hamiltonian *ham, float *out, double *stats) {
    int rc = check_ham(ham);
    if (rc != PSR_OK) return rc;
    if ((rc = check_params_lru(params, n, ham->Lx * ham->Ly)) != PSR_OK) return rc;
    if (!samples || !out) return PSR_EINVAL;
    return lru_run(params, samples, n, ham->Lx * ham->Ly, ham, out, stats);
}

// ------------------------------------- c4v symmetrisation and the VMC step

}  // extern "C"

namespace {

// Fills the 8 groups of a forward job list with the images g = 0..7 of n
// configurations (group g: rows g*n .. g*n+n-1 of the image arrays).
void image_groups(FwdJobs &jb, int N, int W, int u1, int64_t n, uint64_t *bits, float *out,
                  float *logp, float *carries, int64_t carry_row) {
    jb.n_groups = 8;
    for (int g = 0; g < 8; ++g) {
        FwdGroup &G = jb.g[g];
        G.N = N;
        G.W = W;
        G.u1 = u1;
        G.n_jobs = n;
        G.bits = bits + (size_t)g * n * W;
        G.out = out + (size_t)g * n;
        G.logp_out = logp ? logp + (size_t)g * n * N : nullptr;
        G.carries_out = carries ? carries + (size_t)g * n * carry_row : nullptr;
    }
}

int launch_fwd_any(const psr_params *p, const FwdJobs &jb, const void *pkb, const float *pk,
                   const F32Layout &fl, psr_context *ctx) {
    if (p->precision == PSR_BF16) PSR_TRY(launch_fwd_bf16(jb, pkb, pk, fl, ctx->num_sms, ctx->stream));
    else PSR_TRY(launch_fwd_f32(jb, pk, fl, ctx->num_sms, ctx->stream));
    return PSR_OK;
}

int ensure_ws2(psr_context *ctx, size_t bytes) {
    if (bytes <= ctx->ws2_size) return PSR_OK;
    PSR_TRY(cudaStreamSynchronize(ctx->stream));
    if (ctx->ws2) cudaFree(ctx->ws2);
    ctx->ws2 = nullptr;
    ctx->ws2_size = 0;
    const size_t want = bytes + bytes / 8 + (1u << 20);
    if (cudaMalloc(&ctx->ws2, want) != cudaSuccess) {
        cudaGetLastError();
        ctx->ws2 = nullptr;
        return PSR_ENOMEM;
    }
    ctx->ws2_size = want;
    return PSR_OK;
}

}  // namespace

extern "C" {

int psr_sym_logpsi(const psr_params *params, const uint8_t *spins, int64_t n, int32_t Lx, int32_t Ly,
                   float *out) {
    if (Lx != Ly || Lx < 2) return PSR_EINVAL;
    const int L = Lx, N = L * L;
    int rc = check_params(params, n, N);
    if (rc != PSR_OK) return rc;
    if (!spins || !out || n > ((int64_t)1 << 28)) return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden;
    const bool bf16 = params->precision == PSR_BF16;
    const ThetaLayout tl = theta_layout(nL, H);
    const F32Layout fl = f32_layout(nL, H);
    const int W = (int)words_per_row(N);
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(spins),
               d_out = is_device_ptr(out);
    float *theta_ws = nullptr, *out_ws = nullptr, *pk = nullptr, *lp8 = nullptr;
    uint8_t *s_ws = nullptr, *imgs = nullptr;
    void *pkb = nullptr;
    uint64_t *bits = nullptr;
    unsigned long long *counter = nullptr;
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : tl.total);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        out_ws = c.get<float>(d_out ? 0 : n);
        pk = c.get<float>(fl.total);
        pkb = c.get<char>(bf16 ? bf16_packed_bytes() : 0);
        imgs = c.get<uint8_t>((size_t)8 * n * N);
        bits = c.get<uint64_t>((size_t)8 * n * W);
        lp8 = c.get<float>((size_t)8 * n);
        counter = c.get<unsigned long long>(1);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    const float *theta = nullptr;
    const uint8_t *sp = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, tl.total, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(spins, s_ws, (size_t)n * N, d_s, st, &sp)) != PSR_OK) return rc;
    float *o = d_out ? out : out_ws;
    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_PACK);
        PSR_TRY(launch_pack_theta_f32(theta, tl, fl, pk, st));
        if (bf16) PSR_TRY(launch_pack_theta_bf16(theta, tl, pkb, st));
        PSR_TRY(launch_c4v_images(sp, n, L, imgs, st));
        PSR_TRY(launch_bitpack(imgs, 8 * n, N, W, bits, ctx->status, st));
        PSR_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    }
    FwdJobs jb{};
    jb.mode = 0;
    image_groups(jb, N, W, params->u1_mask, n, bits, lp8, nullptr, nullptr, 0);
    jb.job_counter = counter;
    jb.status = ctx->status;
    {
        StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
        if ((rc = launch_fwd_any(params, jb, pkb, pk, fl, ctx)) != PSR_OK) return rc;
    }
    PSR_TRY(launch_sym_logpsi(lp8, n, o, st));
    if (!d_out) PSR_TRY(cudaMemcpyAsync(out, out_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (!d_out || !d_s || !d_theta) return take_status(ctx);
    return PSR_OK;
}

int psr_sym_local_energy(const psr_params *params, const uint8_t *samples, int64_t n,
                         const psr_hamiltonian *ham, float *out, double *stats) {
    int rc = check_ham(ham);
    if (rc != PSR_OK) return rc;
    if (ham->Lx != ham->Ly || ham->Lx < 2) return PSR_EINVAL;
    const int L = ham->Lx, N = L * L;
    if ((rc = check_params(params, n, N)) != PSR_OK) return rc;
    if (!samples || !out || n > ((int64_t)1 << 28)) return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden;
    const bool bf16 = params->precision == PSR_BF16;
    const int CH = bf16 ? kChunkBF16 : kChunkF32;
    const int nch = (N + CH - 1) / CH;
    const ThetaLayout tl = theta_layout(nL, H);
    const F32Layout fl = f32_layout(nL, H);
    const int W = (int)words_per_row(N);
    const int nb = bond_count(L, L, ham->pbc);
    const int64_t cap = n * max_entries_per_sample(ham);
    const int64_t carry_row = (int64_t)nch * nL * H;
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(samples),
               d_out = is_device_ptr(out), d_stats = stats ? is_device_ptr(stats) : true;
    float *theta_ws = nullptr, *out_ws = nullptr, *pk = nullptr, *lp8 = nullptr, *logp8 = nullptr,
          *carries8 = nullptr, *delta8 = nullptr, *dsym = nullptr;
    double *stats_ws = nullptr;
    uint8_t *s_ws = nullptr, *imgs = nullptr;
    void *pkb = nullptr;
    uint64_t *bits = nullptr;
    int32_t *ent8 = nullptr;
    unsigned long long *counters = nullptr;
    ConnBufs b{};
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : tl.total);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        out_ws = c.get<float>(d_out ? 0 : n);
        stats_ws = c.get<double>(d_stats ? 0 : 3);
        pk = c.get<float>(fl.total);
        pkb = c.get<char>(bf16 ? bf16_packed_bytes() : 0);
        imgs = c.get<uint8_t>((size_t)8 * n * N);
        bits = c.get<uint64_t>((size_t)8 * n * W);
        b.bonds = c.get<int32_t>(2 * (size_t)nb + 2);
        b.counts = c.get<int64_t>(n);
        b.offsets = c.get<int64_t>(n + 1);
        b.diag = c.get<float>(n);
        b.entries = c.get<int32_t>(3 * (size_t)cap);
        ent8 = c.get<int32_t>((size_t)8 * 3 * cap);
        lp8 = c.get<float>((size_t)8 * n);
        logp8 = c.get<float>((size_t)8 * n * N);
        carries8 = c.get<float>((size_t)8 * n * carry_row);
        delta8 = c.get<float>((size_t)8 * cap);
        dsym = c.get<float>(cap);
        counters = c.get<unsigned long long>(2);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    const float *theta = nullptr;
    const uint8_t *sp = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, tl.total, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(samples, s_ws, (size_t)n * N, d_s, st, &sp)) != PSR_OK) return rc;
    float *o = d_out ? out : out_ws;
    double *so = stats ? (d_stats ? stats : stats_ws) : nullptr;
    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_PACK);
        PSR_TRY(launch_pack_theta_f32(theta, tl, fl, pk, st));
        if (bf16) PSR_TRY(launch_pack_theta_bf16(theta, tl, pkb, st));
        PSR_TRY(launch_c4v_images(sp, n, L, imgs, st));
        PSR_TRY(launch_bitpack(imgs, 8 * n, N, W, bits, ctx->status, st));
        PSR_TRY(cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st));
    }
    HamDev hd{};
    {
        StageScope sc(ctx, PSR_STAGE_GENERATOR);
        if ((rc = enqueue_connected(ctx, ham, sp, n, b, hd)) != PSR_OK) return rc;
        if (cap > 0) PSR_TRY(launch_c4v_entries(b.entries, b.offsets + n, cap, L, ent8, st));
    }
    FwdJobs js{};
    js.mode = 0;
    image_groups(js, N, W, params->u1_mask, n, bits, lp8, logp8, carries8, carry_row);
    js.job_counter = counters;
    js.status = ctx->status;
    {
        StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
        if ((rc = launch_fwd_any(params, js, pkb, pk, fl, ctx)) != PSR_OK) return rc;
    }
    if (cap > 0) {
        FwdJobs jc{};
        jc.mode = 1;
        jc.n_groups = 8;
        for (int g = 0; g < 8; ++g) {
            FwdGroup &G = jc.g[g];
            G.N = N;
            G.W = W;
            G.u1 = params->u1_mask;
            G.n_jobs = cap;
            G.n_jobs_dev = b.offsets + n;
            G.bits = bits + (size_t)g * n * W;
            G.entries = ent8 + (size_t)g * 3 * cap;
            G.carries_in = carries8 + (size_t)g * n * carry_row;
            G.logp_ref = logp8 + (size_t)g * n * N;
            G.out = delta8 + (size_t)g * cap;
        }
        jc.job_counter = counters + 1;
        jc.status = ctx->status;
        StageScope sc(ctx, PSR_STAGE_FWD_CONNECTED);
        if ((rc = launch_fwd_any(params, jc, pkb, pk, fl, ctx)) != PSR_OK) return rc;
        PSR_TRY(launch_sym_delta(b.entries, b.offsets + n, cap, lp8, n, delta8, dsym, st));
    }
    {
        StageScope sc(ctx, PSR_STAGE_GATHER);
        PSR_TRY(launch_eloc_gather(b.offsets, dsym, b.diag, hd.coeff, n, o, st));
        if (so) PSR_TRY(launch_stats(o, n, so, st));
    }
    if (!d_out) PSR_TRY(cudaMemcpyAsync(out, out_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (stats && !d_stats)
        PSR_TRY(cudaMemcpyAsync(stats, stats_ws, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (!d_out || !d_s || !d_theta || !d_stats) return take_status(ctx);
    return PSR_OK;
}

int psr_vmc_step(const psr_params *params, const psr_hamiltonian *ham, int32_t symmetrize,
                 const float *uniforms, const float *sym_uniforms, int64_t n, const psr_adam *adam,
                 float *theta_out, uint8_t *spins_out, float *eloc_out, double *stats_out,
                 float *grad_out) {
    int rc = check_ham(ham);
    if (rc != PSR_OK) return rc;
    const int N = ham->Lx * ham->Ly;
    if ((rc = check_params(params, n, N)) != PSR_OK) return rc;
    if (symmetrize != 0 && symmetrize != 1) return PSR_EINVAL;
    if (symmetrize && (ham->Lx != ham->Ly || !sym_uniforms)) return PSR_EINVAL;
    if (!uniforms || !adam || !adam->m || !adam->v || !theta_out || adam->step < 1) return PSR_EINVAL;
    if (!(adam->lr >= 0.0f) || !(adam->beta1 >= 0.0f && adam->beta1 < 1.0f) ||
        !(adam->beta2 >= 0.0f && adam->beta2 < 1.0f) || !(adam->eps > 0.0f))
        return PSR_EINVAL;
    const void *dev_args[] = {params->theta, uniforms, adam->m, adam->v, theta_out};
    for (const void *p : dev_args)
        if (!is_device_ptr(p)) return PSR_EINVAL;
    if ((symmetrize && !is_device_ptr(sym_uniforms)) || (spins_out && !is_device_ptr(spins_out)) ||
        (eloc_out && !is_device_ptr(eloc_out)) || (stats_out && !is_device_ptr(stats_out)) ||
        (grad_out && !is_device_ptr(grad_out)))
        return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden;
    const int64_t P = theta_layout(nL, H).total;
    const int n_img = symmetrize ? 8 : 1;

    uint8_t *spins = nullptr, *spins_sym = nullptr, *imgs = nullptr;
    float *eloc = nullptr, *lp8 = nullptr, *dout = nullptr, *grad = nullptr;
    double *stats = nullptr;
    auto carve = [&](Carver &c) {
        spins = c.get<uint8_t>(spins_out && !symmetrize ? 0 : (size_t)n * N);
        spins_sym = c.get<uint8_t>(symmetrize && !spins_out ? (size_t)n * N : 0);
        imgs = c.get<uint8_t>(symmetrize ? (size_t)8 * n * N : 0);
        eloc = c.get<float>(eloc_out ? 0 : n);
        stats = c.get<double>(stats_out ? 0 : 3);
        lp8 = c.get<float>(symmetrize ? (size_t)8 * n : 0);
        dout = c.get<float>((size_t)n_img * n);
        grad = c.get<float>(grad_out ? 0 : P);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws2(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws2);
    carve(cv);
    if (spins_out && !symmetrize) spins = spins_out;
    if (symmetrize && spins_out) spins_sym = spins_out;
    if (eloc_out) eloc = eloc_out;
    if (stats_out) stats = stats_out;
    if (grad_out) grad = grad_out;
    cudaStream_t st = ctx->stream;
    psr_params p32 = *params;
    p32.precision = PSR_FP32;

    // 1. exact samples of |psi|^2 (then a uniformly drawn c4v image of each)
    if ((rc = psr_sample(params, uniforms, n, N, spins, nullptr)) != PSR_OK) return rc;
    const uint8_t *used = spins;
    if (symmetrize) {
        PSR_TRY(launch_c4v_pick(spins, sym_uniforms, n, ham->Lx, spins_sym, st));
        used = spins_sym;
    }
    // 2. local energies and their FP64 statistics
    rc = symmetrize ? psr_sym_local_energy(params, used, n, ham, eloc, stats)
                    : psr_local_energy(params, used, n, ham, eloc, stats);
    if (rc != PSR_OK) return rc;
    // 3. centred energy-gradient weights (per image when symmetrised)
    if (symmetrize) {
        PSR_TRY(launch_c4v_images(used, n, ham->Lx, imgs, st));
        if ((rc = psr_logpsi(&p32, imgs, 8 * n, N, lp8)) != PSR_OK) return rc;
    }
    PSR_TRY(launch_vmc_dout(eloc, stats, lp8, n, n_img, dout, st));
    // 4. gradient sum_i dout_i d log psi(s_i) / d theta (FP32 reverse scan)
    if ((rc = psr_grad(params, symmetrize ? imgs : used, n_img * n, N, dout, grad)) != PSR_OK)
        return rc;
    // 5. Adam update
    PSR_TRY(launch_adam(params->theta, grad, P, adam->lr, adam->beta1, adam->beta2, adam->eps,
                        adam->step, adam->m, adam->v, theta_out, st));
    return PSR_OK;
}

}  // extern "C"
