// C ABI: the standalone chunked scan with its autotuner, the bounded-wait
// self-test, and the exact autoregressive sampler.
#include "psr_api_common.cuh"

using namespace psr;
using namespace psr::apiutil;

// ------------------------------------------------------------------ scan

namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

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
    // BF16 shapes the tensor-core sampler does not hold draw in FP32
    if (rc == PSR_EUNSUPPORTED && params->precision == PSR_BF16) rc = PSR_OK;
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
    uint8_t *s_ws = nullptr, *wimg = nullptr;
    // BF16 at the BF16 forward's shape: the tensor-core sampler (the
    // conditionals of the BF16 model); FP32 otherwise
    const bool tc = params->precision == PSR_BF16 && sample_tc_supported(nL, H);
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : tl.total);
        u_ws = c.get<float>(d_u ? 0 : cells);
        s_ws = c.get<uint8_t>(d_s ? 0 : cells);
        lp_ws = c.get<float>(d_lp ? 0 : n);
        pk = c.get<float>(fl.total);
        if (tc) wimg = c.get<uint8_t>(sample_tc_weight_bytes());
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

    if (tc) {
        reset_stages(ctx);
        {
            StageScope sc(ctx, PSR_STAGE_PACK);
            PSR_TRY(launch_pack_theta_f32(theta, tl, fl, pk, st));
        }
        {
            StageScope sc(ctx, PSR_STAGE_SAMPLE);
            PSR_TRY(launch_sample_tc(pk, fl, wimg, uu, n, L, params->u1_mask, so, lo, ctx->status, ctx->num_sms, st));
        }
        if (!d_s) PSR_TRY(cudaMemcpyAsync(spins, s_ws, cells, cudaMemcpyDeviceToHost, st));
        if (logpsi && !d_lp)
            PSR_TRY(cudaMemcpyAsync(logpsi, lp_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
        if (!d_theta || !d_u || !d_s || !d_lp) return take_status(ctx);
        return PSR_OK;
    }
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

}  // extern "C"
