// C ABI of libpsr, chain minGRU model: errors, contexts, log psi, the
// connected-configuration generator, local energy and the gradient (the
// batched forms are in psr_api_batch.cu).  The argument checks, workspace carving and staging are in
// psr_api_common.cuh; all compute happens in the kernels.
#include "psr_api_common.cuh"

using namespace psr;
using namespace psr::apiutil;

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
    const int32_t Ns[1] = {L};
    const int64_t ns[1] = {n};
    const FwdKey key = fwd_key(bf16, 0, 1, Ns, ns);
    auto run_fwd = [&](int shape) -> int {
        StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
        PSR_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
        if (bf16) PSR_TRY(launch_fwd_bf16(jb, pkb, pk, fl, ctx->num_sms, st, shape));
        else PSR_TRY(launch_fwd_f32(jb, pk, fl, ctx->num_sms, st, shape));
        return PSR_OK;
    };
    int shape = 0;
    if ((rc = tune_fwd_shape(ctx, bf16, key, run_fwd, &shape)) != PSR_OK) return rc;
    if ((rc = run_fwd(shape)) != PSR_OK) return rc;
    if (!d_out) {
        PSR_TRY(cudaMemcpyAsync(out, out_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    }
    if (!d_out || !d_spins || !d_theta) return take_status(ctx);
    return PSR_OK;
}

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
    // carries sized for the shortest chunk any forward shape uses
    const int CHmin = bf16 ? kChunkBF16 : kChunkGrad;
    const int nch = (N + CHmin - 1) / CHmin;
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
    const int32_t Ns[1] = {N};
    const int64_t ns[1] = {n};
    const FwdKey key = fwd_key(bf16, 1, 1, Ns, ns);
    auto run_fwd = [&](int shape) -> int {
        PSR_TRY(cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st));
        {
            StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
            if (bf16) PSR_TRY(launch_fwd_bf16(js, pkb, pk, fl, ctx->num_sms, st, shape));
            else PSR_TRY(launch_fwd_f32(js, pk, fl, ctx->num_sms, st, shape));
        }
        if (cap > 0) {
            StageScope sc(ctx, PSR_STAGE_FWD_CONNECTED);
            if (bf16) PSR_TRY(launch_fwd_bf16(jc, pkb, pk, fl, ctx->num_sms, st, shape));
            else PSR_TRY(launch_fwd_f32(jc, pk, fl, ctx->num_sms, st, shape));
        }
        return PSR_OK;
    };
    int shape = 0;
    if ((rc = tune_fwd_shape(ctx, bf16, key, run_fwd, &shape)) != PSR_OK) return rc;
    if ((rc = run_fwd(shape)) != PSR_OK) return rc;
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

// psr_grad on the tensor cores (BF16 precision, per-sample rows, hidden 128).
static int grad_tc_call(const psr_params *params, const uint8_t *spins, int64_t n, int32_t L, float *dparams) {
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers;
    const ThetaLayout tl = theta_layout(nL, 128);
    const F32Layout fl = f32_layout(nL, 128);
    const int64_t P = tl.total;
    const int W = (int)words_per_row(L);
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(spins), d_g = is_device_ptr(dparams);
    const int64_t B = grad_tc_batch(nL, L, n);
    float *theta_ws = nullptr, *g_ws = nullptr, *pk = nullptr;
    uint8_t *s_ws = nullptr;
    uint64_t *bits = nullptr;
    GradTcWs tw{};
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : P);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * L);
        g_ws = c.get<float>(d_g ? 0 : (size_t)n * P);
        pk = c.get<float>(fl.total);
        bits = c.get<uint64_t>((size_t)n * W);
        grad_tc_carve(c, nL, L, B, tw);
    };
    Carver sz;
    carve(sz);
    int rc;
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    const float *theta = nullptr;
    const uint8_t *sp = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, P, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(spins, s_ws, (size_t)n * L, d_s, st, &sp)) != PSR_OK) return rc;
    float *g = d_g ? dparams : g_ws;
    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_PACK);
        PSR_TRY(launch_pack_theta_f32(theta, tl, fl, pk, st));
        PSR_TRY(launch_bitpack(sp, n, L, W, bits, ctx->status, st));
    }
    {
        StageScope sc(ctx, PSR_STAGE_BWD);  // the stash forward and the reverse pass
        if ((rc = enqueue_grad_tc(ctx, nL, params->u1_mask, theta, pk, bits, n, L, W, g, tw)) != PSR_OK) return rc;
    }
    if (!d_g) PSR_TRY(cudaMemcpyAsync(dparams, g_ws, (size_t)n * P * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (!d_g || !d_s || !d_theta) return take_status(ctx);
    return PSR_OK;
}

int psr_grad(const psr_params *params, const uint8_t *spins, int64_t n, int32_t L,
             const float *dout, float *dparams) {
    int rc = check_params(params, n, L);
    if (rc != PSR_OK && rc != PSR_EUNSUPPORTED) return rc;
    if (!spins || !dparams) return PSR_EINVAL;
    if (rc == PSR_OK && grad_tc_applies(params, dout)) return grad_tc_call(params, spins, n, L, dparams);
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


}  // extern "C"
