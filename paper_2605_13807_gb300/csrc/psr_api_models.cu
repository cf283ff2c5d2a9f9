// C ABI: the paper's two-dimensional patched minGRU and deep 1D LRU models.
#include "psr_api_common.cuh"

using namespace psr;
using namespace psr::apiutil;

// ------------------------------------------- two-dimensional patched minGRU

namespace {

int check_params2d(const psr_params *p, int64_t n, int Lx, int Ly) {
    if (!p || !p->ctx || !p->theta) return PSR_EINVAL;
    if (p->n_layers < 1 || p->n_layers > kMaxLayers) return PSR_EINVAL;
    if (p->hidden != 32 && p->hidden != 64 && p->hidden != 128 && p->hidden != 256) return PSR_EINVAL;
    if (p->hidden == 256 && p->n_layers > 4) return PSR_EUNSUPPORTED;  // shared memory
    if (p->u1_mask != 0 && p->u1_mask != 1) return PSR_EINVAL;
    if (p->precision != PSR_FP32 && p->precision != PSR_BF16 && p->precision != PSR_FP16) return PSR_EINVAL;
    if (n < 1 || n > (int64_t)1 << 31) return PSR_EINVAL;
    if (Lx < 2 || Ly < 2 || (Lx % 2) || (Ly % 2) || (int64_t)Lx * Ly > (1 << 24)) return PSR_EINVAL;
    if (Lx > 64) return PSR_EUNSUPPORTED;  // at most 32 patches per row
    // FP16 / BF16: the forward evaluations (log psi, E_loc) on the tensor cores
    if (p->precision != PSR_FP32 && !fwd2d_tc_supported(p->n_layers, p->hidden, Lx)) return PSR_EUNSUPPORTED;
    return PSR_OK;
}

// Workspace of the tensor-core forward (16-bit precisions): the weight slices,
// per-CTA h_V images and residual rows, and a zero image (the h_V of row 0).
struct Tc2 {
    uint8_t *wimg = nullptr, *scratch = nullptr, *zero = nullptr;
    float *res = nullptr;
};

void tc2_carve(Carver &c, psr_context *ctx, int nL, int H, int Lx, Tc2 &t) {
    t.wimg = c.get<uint8_t>(fwd2d_tc_weight_bytes(nL, H));
    t.scratch = c.get<uint8_t>(fwd2d_tc_scratch_bytes(nL, H, Lx, ctx->num_sms));
    t.zero = c.get<uint8_t>(fwd2d_tc_image_bytes(H, Lx));
    t.res = c.get<float>(fwd2d_tc_res_floats(H, ctx->num_sms));
}

cudaError_t tc2_prepare(const float *theta, const T2Layout &tl, int Lx, bool f16, const Tc2 &t,
                        cudaStream_t st) {
    cudaError_t e = launch_pack2d_tc(theta, tl, f16, t.wimg, st);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(t.zero, 0, fwd2d_tc_image_bytes(tl.H, Lx), st);
}

// The jobs of `jb` on the tensor cores; row checkpoints as 16-bit images
// (img_out written in mode 0 when set, img_in read in mode 1).
cudaError_t tc2_run(psr_context *ctx, const Fwd2Jobs &jb, bool f16, const float *theta, const T2Layout &tl,
                    const Tc2 &t, const uint8_t *img_in, uint8_t *img_out) {
    Fwd2TcArgs a{};
    a.mode = jb.mode;
    a.f16 = f16 ? 1 : 0;
    a.Lx = jb.g.Lx;
    a.Ly = jb.g.Ly;
    a.u1 = jb.g.u1;
    a.n_jobs = jb.g.n_jobs;
    a.n_jobs_dev = jb.g.n_jobs_dev;
    a.spins = jb.g.spins;
    a.entries = jb.g.entries;
    a.img_in = img_in;
    a.img_out = img_out;
    a.scratch = t.scratch;
    a.zero_img = t.zero;
    a.res = t.res;
    a.logp_ref = jb.g.logp_ref;
    a.out = jb.g.out;
    a.logp_out = jb.g.logp_out;
    a.theta = theta;
    a.tl = tl;
    a.wimg = t.wimg;
    a.job_counter = jb.job_counter;
    a.status = jb.status;
    if (jb.g.n_jobs >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;  // job indices are 32-bit
    int W, S;
    fwd2d_tc_geometry(a.Lx, &W, &S);
    int64_t grid = (jb.g.n_jobs + S - 1) / S;
    if (grid > ctx->num_sms) grid = ctx->num_sms;
    if (grid < 1) grid = 1;
    return launch_fwd2d_tc(a, (int)grid, ctx->stream);
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
    const T2Layout tl = t2_layout(nL, H);
    const bool tc = params->precision != PSR_FP32, f16 = params->precision == PSR_FP16;
    const int W = (int)words_per_row(N);
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(spins),
               d_out = is_device_ptr(out);
    float *theta_ws = nullptr, *out_ws = nullptr, *pk = nullptr;
    uint8_t *s_ws = nullptr;
    uint64_t *bits = nullptr;
    unsigned long long *counter = nullptr;
    Tc2 t2{};
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : P);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        out_ws = c.get<float>(d_out ? 0 : n);
        pk = c.get<float>(tc ? 0 : f.total);
        bits = c.get<uint64_t>((size_t)n * W);
        counter = c.get<unsigned long long>(1);
        if (tc) tc2_carve(c, ctx, nL, H, Lx, t2);
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
        if (tc) PSR_TRY(tc2_prepare(theta, tl, Lx, f16, t2, st));
        else PSR_TRY(launch_pack_theta_f2(theta, f, pk, st));
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
        if (tc) PSR_TRY(tc2_run(ctx, jb, f16, theta, tl, t2, nullptr, nullptr));
        else PSR_TRY(launch_fwd2d_f32(jb, pk, f, ctx->num_sms, st));
    }
    if (!d_out) PSR_TRY(cudaMemcpyAsync(out, out_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (!d_out || !d_s || !d_theta) return take_status(ctx);
    return PSR_OK;
}

int psr2d_sample(const psr_params *params, const float *uniforms, int64_t n, int32_t Lx, int32_t Ly,
                 uint8_t *spins, float *logpsi) {
    int rc = check_params2d(params, n, Lx, Ly);
    if (rc != PSR_OK) return rc;
    if (!uniforms || !spins) return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden, N = Lx * Ly;
    const int64_t Np = (int64_t)(Lx / 2) * (Ly / 2);
    const int64_t P = param_count2d(nL, H);
    const F2Layout f = f2_layout(nL, H);
    const bool d_theta = is_device_ptr(params->theta), d_u = is_device_ptr(uniforms),
               d_s = is_device_ptr(spins), d_lp = logpsi ? is_device_ptr(logpsi) : true;
    // samples per CTA: the candidates that fit (a thread per logit, shared memory)
    std::vector<int> cands;
    for (int b : {1, 2, 4, 8})
        if (b * 16 <= H && sample2d_smem_bytes(b, nL, H, Lx) <= 220 * 1024) cands.push_back(b);
    if (cands.empty()) return PSR_EUNSUPPORTED;
    float *theta_ws = nullptr, *u_ws = nullptr, *lp_ws = nullptr, *pk = nullptr;
    uint8_t *s_ws = nullptr;
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : P);
        u_ws = c.get<float>(d_u ? 0 : (size_t)n * Np);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        lp_ws = c.get<float>(d_lp ? 0 : n);
        pk = c.get<float>(f.total);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    const float *theta = nullptr, *uu = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, P, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(uniforms, u_ws, (size_t)n * Np, d_u, st, &uu)) != PSR_OK) return rc;
    uint8_t *so = d_s ? spins : s_ws;
    float *lo = logpsi ? (d_lp ? logpsi : lp_ws) : nullptr;
    const int64_t key2 = (int64_t)nL * 1024 + H;
    int per_cta = cands.size() > 2 ? cands[2] : cands.back();  // 4 where it fits
    bool tune_now = false;
    if (const psr_context::Tuned *t = find_tuned(ctx, kTuneSample2d, n, (int64_t)Lx * 65536 + Ly, key2))
        per_cta = t->v0;
    else if (ctx->autotune && !ctx->capturing) tune_now = true;
    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_PACK);
        PSR_TRY(launch_pack_theta_f2(theta, f, pk, st));
    }
    if (tune_now) {
        int bi = 0;
        float best = 0.0f;
        rc = measure_candidates(ctx, (int)cands.size(), [&](int i) {
            return from_cuda(launch_sample2d(cands[i], pk, f, uu, n, Lx, Ly, params->u1_mask, so, lo, st));
        }, &bi, &best);
        if (rc != PSR_OK) return rc;
        per_cta = cands[bi];
        ctx->tuned.push_back(psr_context::Tuned{kTuneSample2d, n, (int64_t)Lx * 65536 + Ly, key2, per_cta, 0,
                                                best});
    }
    {
        StageScope sc(ctx, PSR_STAGE_SAMPLE);
        PSR_TRY(launch_sample2d(per_cta, pk, f, uu, n, Lx, Ly, params->u1_mask, so, lo, st));
    }
    if (!d_s) PSR_TRY(cudaMemcpyAsync(spins, s_ws, (size_t)n * N, cudaMemcpyDeviceToHost, st));
    if (logpsi && !d_lp) PSR_TRY(cudaMemcpyAsync(logpsi, lp_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (!d_theta || !d_u || !d_s || !d_lp) return take_status(ctx);
    return PSR_OK;
}

int psr2d_grad(const psr_params *params, const uint8_t *spins, int64_t n, int32_t Lx, int32_t Ly,
               const float *dout, float *dparams) {
    int rc = check_params2d(params, n, Lx, Ly);
    if (rc != PSR_OK) return rc;
    if (!spins || !dparams) return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden, N = Lx * Ly, Py = Ly / 2;
    const int64_t P = param_count2d(nL, H);
    const F2Layout f = f2_layout(nL, H);
    const T2Layout tl = t2_layout(nL, H);
    const int W = (int)words_per_row(N);
    const size_t ckpt = fwd2d_checkpoint_floats(nL, H, Lx);
    int dev_smem = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device);
    int per_sm = (int)(dev_smem / (bwd2d_smem_bytes(nL, H, Lx) + 1024));
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
    int64_t grid64 = (int64_t)ctx->num_sms * per_sm;
    if (grid64 > n) grid64 = n;
    const int grid = (int)grid64;
    const size_t rows = dout ? (size_t)grid : (size_t)n;
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(spins),
               d_dout = dout ? is_device_ptr(dout) : true, d_g = is_device_ptr(dparams);
    float *theta_ws = nullptr, *dout_ws = nullptr, *g_ws = nullptr, *pk = nullptr, *lpsi = nullptr,
          *carries = nullptr, *scratch = nullptr, *partial = nullptr;
    uint8_t *s_ws = nullptr;
    uint64_t *bits = nullptr;
    unsigned long long *counter = nullptr;
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : P);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        dout_ws = c.get<float>(d_dout ? 0 : n);
        g_ws = c.get<float>(d_g ? 0 : (dout ? P : (size_t)n * P));
        pk = c.get<float>(f.total);
        bits = c.get<uint64_t>((size_t)n * W);
        lpsi = c.get<float>(n);
        carries = c.get<float>((size_t)n * Py * ckpt);
        scratch = c.get<float>((size_t)grid * bwd2d_scratch_floats_per_cta(nL, H));
        partial = c.get<float>(dout ? rows * P : 0);
        counter = c.get<unsigned long long>(1);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    const float *theta = nullptr, *dv = nullptr;
    const uint8_t *sp = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, P, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(spins, s_ws, (size_t)n * N, d_s, st, &sp)) != PSR_OK) return rc;
    if (dout && (rc = stage_in(dout, dout_ws, n, d_dout, st, &dv)) != PSR_OK) return rc;
    float *g = d_g ? dparams : g_ws;
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
    jb.g.out = lpsi;
    jb.g.carries_out = carries;
    jb.job_counter = counter;
    jb.status = ctx->status;
    {
        StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
        PSR_TRY(launch_fwd2d_f32(jb, pk, f, ctx->num_sms, st));
    }
    {
        StageScope sc(ctx, PSR_STAGE_BWD);
        float *out_rows = dout ? partial : g;
        PSR_TRY(cudaMemsetAsync(out_rows, 0, rows * P * sizeof(float), st));
        PSR_TRY(launch_bwd2d(sp, n, Lx, Ly, params->u1_mask, theta, tl, pk, f, carries, dv, out_rows, grid,
                             scratch, st));
        if (dout) PSR_TRY(launch_reduce_rows(partial, grid, P, g, st));
    }
    if (!d_g)
        PSR_TRY(cudaMemcpyAsync(dparams, g_ws, (dout ? P : (size_t)n * P) * sizeof(float),
                                cudaMemcpyDeviceToHost, st));
    if (!d_g || !d_s || !d_theta || !d_dout) return take_status(ctx);
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
    const T2Layout tl = t2_layout(nL, H);
    const bool tc = params->precision != PSR_FP32, f16 = params->precision == PSR_FP16;
    const int W = (int)words_per_row(N);
    const int nb = bond_count(Lx, Ly, ham->pbc);
    const int64_t cap = n * max_entries_per_sample(ham);
    if (params->precision != PSR_FP32 && cap >= ((int64_t)1 << 31)) return PSR_EUNSUPPORTED;
    const size_t ckpt = fwd2d_checkpoint_floats(nL, H, Lx);
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(samples),
               d_out = is_device_ptr(out), d_stats = stats ? is_device_ptr(stats) : true;

    float *theta_ws = nullptr, *out_ws = nullptr, *pk = nullptr, *lpsi = nullptr, *logp = nullptr,
          *carries = nullptr, *delta = nullptr;
    double *stats_ws = nullptr;
    uint8_t *s_ws = nullptr;
    uint64_t *bits = nullptr;
    unsigned long long *counters = nullptr;
    uint8_t *imgs = nullptr;
    Tc2 t2{};
    ConnBufs b{};
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : P);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        out_ws = c.get<float>(d_out ? 0 : n);
        stats_ws = c.get<double>(d_stats ? 0 : 3);
        pk = c.get<float>(tc ? 0 : f.total);
        bits = c.get<uint64_t>((size_t)n * W);
        b.bonds = c.get<int32_t>(2 * (size_t)nb + 2);
        b.counts = c.get<int64_t>(n);
        b.offsets = c.get<int64_t>(n + 1);
        b.diag = c.get<float>(n);
        b.entries = c.get<int32_t>(3 * (size_t)cap);
        lpsi = c.get<float>(n);
        logp = c.get<float>((size_t)n * Np);
        carries = c.get<float>(tc ? 0 : (size_t)n * Py * ckpt);
        imgs = c.get<uint8_t>(tc ? (size_t)n * fwd2d_tc_ckpt_bytes(nL, H, Lx, Ly) : 0);
        if (tc) tc2_carve(c, ctx, nL, H, Lx, t2);
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
        if (tc) PSR_TRY(tc2_prepare(theta, tl, Lx, f16, t2, st));
        else PSR_TRY(launch_pack_theta_f2(theta, f, pk, st));
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
        if (tc) PSR_TRY(tc2_run(ctx, js, f16, theta, tl, t2, nullptr, imgs));
        else PSR_TRY(launch_fwd2d_f32(js, pk, f, ctx->num_sms, st));
    }
    if (cap > 0) {
        StageScope sc(ctx, PSR_STAGE_FWD_CONNECTED);
        if (tc) PSR_TRY(tc2_run(ctx, jc, f16, theta, tl, t2, imgs, nullptr));
        else PSR_TRY(launch_fwd2d_f32(jc, pk, f, ctx->num_sms, st));
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

// ------------------------------------------ c4v-symmetrised 2D patched model

}  // extern "C"

namespace {

// Shared body of psr2d_sym_logpsi (ham == nullptr) and psr2d_sym_local_energy:
// the 8 c4v images of every configuration in one forward launch (with row
// checkpoints and per-patch log P when E_loc follows), the images of every
// connected entry (sites g(p), g(q) flipped) resumed from their image
// sample's checkpoints, one launch per image, then the log-sum-exp
// combinations of the 8 images.
int sym2d_run(const psr_params *params, const uint8_t *samples, int64_t n, int32_t L,
              const psr_hamiltonian *ham, float *out, double *stats) {
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden, N = L * L, Py = L / 2, Np = (L / 2) * Py;
    const int64_t P = param_count2d(nL, H);
    const F2Layout f = f2_layout(nL, H);
    const T2Layout tl = t2_layout(nL, H);
    const bool tc = params->precision != PSR_FP32, f16 = params->precision == PSR_FP16;
    const size_t ckpt_img = tc ? fwd2d_tc_ckpt_bytes(nL, H, L, L) : 0;
    const bool eloc = ham != nullptr;
    const int W = (int)words_per_row(N);
    const int nb = eloc ? bond_count(L, L, ham->pbc) : 0;
    const int64_t cap = eloc ? n * max_entries_per_sample(ham) : 0;
    if (params->precision != PSR_FP32 && cap >= ((int64_t)1 << 31)) return PSR_EUNSUPPORTED;
    const size_t ckpt = fwd2d_checkpoint_floats(nL, H, L);
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(samples),
               d_out = is_device_ptr(out), d_stats = stats ? is_device_ptr(stats) : true;
    float *theta_ws = nullptr, *out_ws = nullptr, *pk = nullptr, *lp8 = nullptr, *logp8 = nullptr,
          *carries8 = nullptr, *delta8 = nullptr, *dsym = nullptr;
    double *stats_ws = nullptr;
    uint8_t *s_ws = nullptr, *imgs = nullptr;
    uint64_t *bits = nullptr;
    int32_t *ent8 = nullptr;
    unsigned long long *counters = nullptr;
    uint8_t *ckimg8 = nullptr;
    Tc2 t2{};
    ConnBufs b{};
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : P);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        out_ws = c.get<float>(d_out ? 0 : n);
        stats_ws = c.get<double>(d_stats ? 0 : 3);
        pk = c.get<float>(tc ? 0 : f.total);
        if (tc) tc2_carve(c, ctx, nL, H, L, t2);
        bits = c.get<uint64_t>((size_t)n * W);
        imgs = c.get<uint8_t>((size_t)8 * n * N);
        lp8 = c.get<float>((size_t)8 * n);
        counters = c.get<unsigned long long>(9);
        if (eloc) {
            b.bonds = c.get<int32_t>(2 * (size_t)nb + 2);
            b.counts = c.get<int64_t>(n);
            b.offsets = c.get<int64_t>(n + 1);
            b.diag = c.get<float>(n);
            b.entries = c.get<int32_t>(3 * (size_t)cap);
            ent8 = c.get<int32_t>((size_t)8 * 3 * cap);
            logp8 = c.get<float>((size_t)8 * n * Np);
            carries8 = c.get<float>(tc ? 0 : (size_t)8 * n * Py * ckpt);
            ckimg8 = c.get<uint8_t>(tc ? (size_t)8 * n * ckpt_img : 0);
            delta8 = c.get<float>((size_t)8 * cap);
            dsym = c.get<float>(cap);
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
        if (tc) PSR_TRY(tc2_prepare(theta, tl, L, f16, t2, st));
        else PSR_TRY(launch_pack_theta_f2(theta, f, pk, st));
        PSR_TRY(launch_bitpack(sp, n, N, W, bits, ctx->status, st));  // spin-byte check
        PSR_TRY(launch_c4v_images(sp, n, L, imgs, st));
        PSR_TRY(cudaMemsetAsync(counters, 0, 9 * sizeof(unsigned long long), st));
    }
    HamDev hd{};
    if (eloc) {
        StageScope sc(ctx, PSR_STAGE_GENERATOR);
        if ((rc = enqueue_connected(ctx, ham, sp, n, b, hd)) != PSR_OK) return rc;
        if (cap > 0) PSR_TRY(launch_c4v_entries(b.entries, b.offsets + n, cap, L, ent8, st));
    }
    Fwd2Jobs js{};
    js.mode = 0;
    js.g.Lx = L;
    js.g.Ly = L;
    js.g.u1 = params->u1_mask;
    js.g.n_jobs = 8 * n;
    js.g.spins = imgs;
    js.g.out = lp8;
    js.g.logp_out = logp8;
    js.g.carries_out = carries8;
    js.job_counter = counters;
    js.status = ctx->status;
    {
        StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
        if (tc) PSR_TRY(tc2_run(ctx, js, f16, theta, tl, t2, nullptr, eloc ? ckimg8 : nullptr));
        else PSR_TRY(launch_fwd2d_f32(js, pk, f, ctx->num_sms, st));
    }
    if (eloc && cap > 0) {
        StageScope sc(ctx, PSR_STAGE_FWD_CONNECTED);
        for (int g = 0; g < 8; ++g) {
            Fwd2Jobs jc = js;
            jc.mode = 1;
            jc.g.n_jobs = cap;
            jc.g.n_jobs_dev = b.offsets + n;
            jc.g.spins = imgs + (size_t)g * n * N;
            jc.g.entries = ent8 + (size_t)g * 3 * cap;
            jc.g.carries_in = tc ? nullptr : carries8 + (size_t)g * n * Py * ckpt;
            jc.g.logp_ref = logp8 + (size_t)g * n * Np;
            jc.g.out = delta8 + (size_t)g * cap;
            jc.g.logp_out = nullptr;
            jc.g.carries_out = nullptr;
            jc.job_counter = counters + 1 + g;
            if (tc) PSR_TRY(tc2_run(ctx, jc, f16, theta, tl, t2, ckimg8 + (size_t)g * n * ckpt_img, nullptr));
            else PSR_TRY(launch_fwd2d_f32(jc, pk, f, ctx->num_sms, st));
        }
        PSR_TRY(launch_sym_delta(b.entries, b.offsets + n, cap, lp8, n, delta8, dsym, st));
    }
    if (eloc) {
        StageScope sc(ctx, PSR_STAGE_GATHER);
        PSR_TRY(launch_eloc_gather(b.offsets, dsym, b.diag, hd.coeff, n, o, st));
        if (so) PSR_TRY(launch_stats(o, n, so, st));
    } else {
        PSR_TRY(launch_sym_logpsi(lp8, n, o, st));
    }
    if (!d_out) PSR_TRY(cudaMemcpyAsync(out, out_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (stats && !d_stats)
        PSR_TRY(cudaMemcpyAsync(stats, stats_ws, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (!d_out || !d_s || !d_theta || !d_stats) return take_status(ctx);
    return PSR_OK;
}

}  // namespace

extern "C" {

int psr2d_sym_logpsi(const psr_params *params, const uint8_t *spins, int64_t n, int32_t Lx, int32_t Ly,
                     float *out) {
    if (Lx != Ly) return PSR_EINVAL;
    int rc = check_params2d(params, n, Lx, Ly);
    if (rc != PSR_OK) return rc;
    if (!spins || !out || n > ((int64_t)1 << 28)) return PSR_EINVAL;
    return sym2d_run(params, spins, n, Lx, nullptr, out, nullptr);
}

int psr2d_sym_local_energy(const psr_params *params, const uint8_t *samples, int64_t n,
                           const psr_hamiltonian *ham, float *out, double *stats) {
    int rc = check_ham(ham);
    if (rc != PSR_OK) return rc;
    if (ham->Lx != ham->Ly) return PSR_EINVAL;
    if ((rc = check_params2d(params, n, ham->Lx, ham->Ly)) != PSR_OK) return rc;
    if (!samples || !out || n > ((int64_t)1 << 28)) return PSR_EINVAL;
    return sym2d_run(params, samples, n, ham->Lx, ham, out, stats);
}

// ------------------------------------------------------ deep 1D LRU model

}  // extern "C"

namespace {

int check_params_lru(const psr_params *p, int64_t n, int32_t L) {
    if (!p || !p->ctx || !p->theta) return PSR_EINVAL;
    if (p->n_layers < 1 || p->n_layers > kMaxLayers) return PSR_EINVAL;
    if (p->hidden != 32 && p->hidden != 64 && p->hidden != 128) return PSR_EINVAL;
    if (p->u1_mask != 0 && p->u1_mask != 1) return PSR_EINVAL;
    if (p->precision != PSR_FP32 && p->precision != PSR_BF16 && p->precision != PSR_FP16) return PSR_EINVAL;
    if (n < 1 || L < 1 || n > (int64_t)1 << 31) return PSR_EINVAL;
    if (p->u1_mask && (L % 2)) return PSR_EINVAL;
    // FP16 / BF16: the forward evaluations (log psi, E_loc) on the tensor cores
    if (p->precision != PSR_FP32 && !lru_tc_supported(p->n_layers, p->hidden)) return PSR_EUNSUPPORTED;
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
    const bool tc = params->precision != PSR_FP32, f16 = params->precision == PSR_FP16;
    if (tc && cap >= ((int64_t)1 << 31)) return PSR_EUNSUPPORTED;  // 32-bit job indices
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(samples),
               d_out = is_device_ptr(out), d_stats = stats ? is_device_ptr(stats) : true;
    float *theta_ws = nullptr, *out_ws = nullptr, *pk = nullptr, *lpsi = nullptr, *logp = nullptr,
          *carries = nullptr, *delta = nullptr;
    uint8_t *wimg = nullptr;
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
        if (tc) wimg = c.get<uint8_t>(lru_tc_weight_bytes(nL));
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
        if (tc) PSR_TRY(launch_pack_lru_tc(pk, f, f16, wimg, st));
        PSR_TRY(launch_bitpack(sp, n, N, W, bits, ctx->status, st));
        PSR_TRY(cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st));
    }
    // the FP32 kernel, or the tensor-core one (one job per slot, 8 slots per CTA)
    auto run = [&](const FwdJobs &jb) -> cudaError_t {
        if (!tc) return launch_lru_f32(jb, pk, f, ctx->num_sms, st);
        LruTcArgs a{};
        a.mode = jb.mode;
        a.nL = nL;
        a.f16 = f16 ? 1 : 0;
        a.g = jb.g[0];
        a.f = f;
        a.pk = pk;
        a.wimg = wimg;
        a.job_counter = jb.job_counter;
        a.status = jb.status;
        int64_t grid = (jb.g[0].n_jobs + 7) / 8;
        if (grid > ctx->num_sms) grid = ctx->num_sms;
        return launch_lru_tc(a, (int)(grid < 1 ? 1 : grid), st);
    };
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
        PSR_TRY(run(js));
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
            PSR_TRY(run(jc));
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

int psr_lru_sample(const psr_params *params, const float *uniforms, int64_t n, int32_t L, uint8_t *spins,
                   float *logpsi) {
    int rc = check_params_lru(params, n, L);
    if (rc != PSR_OK) return rc;
    if (!uniforms || !spins) return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden, N = L;
    const int64_t P = param_count_lru(nL, H);
    const LruLayout f = lru_layout(nL, H);
    const bool d_theta = is_device_ptr(params->theta), d_u = is_device_ptr(uniforms),
               d_s = is_device_ptr(spins), d_lp = logpsi ? is_device_ptr(logpsi) : true;
    float *theta_ws = nullptr, *u_ws = nullptr, *lp_ws = nullptr, *pk = nullptr;
    uint8_t *s_ws = nullptr, *wimg = nullptr;
    // 16-bit precision: the tensor-core sampler (the conditionals of the
    // tensor-core forward) where it holds the model; FP32 otherwise
    const bool tc = params->precision != PSR_FP32 && lru_tc_sample_supported(nL, H);
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : P);
        u_ws = c.get<float>(d_u ? 0 : (size_t)n * N);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        lp_ws = c.get<float>(d_lp ? 0 : n);
        pk = c.get<float>(f.total);
        if (tc) wimg = c.get<uint8_t>(lru_tc_weight_bytes(nL));
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    const float *theta = nullptr, *uu = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, P, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(uniforms, u_ws, (size_t)n * N, d_u, st, &uu)) != PSR_OK) return rc;
    uint8_t *so = d_s ? spins : s_ws;
    float *lo = logpsi ? (d_lp ? logpsi : lp_ws) : nullptr;
    if (tc) {
        const bool f16 = params->precision == PSR_FP16;
        reset_stages(ctx);
        {
            StageScope sc(ctx, PSR_STAGE_PACK);
            PSR_TRY(launch_pack_theta_lru(theta, f, pk, st));
            PSR_TRY(launch_pack_lru_tc(pk, f, f16, wimg, st));
        }
        {
            StageScope sc(ctx, PSR_STAGE_SAMPLE);
            PSR_TRY(launch_sample_lru_tc(pk, f, f16, wimg, uu, n, N, params->u1_mask, so, lo, ctx->status,
                                         ctx->num_sms, st));
        }
        if (!d_s) PSR_TRY(cudaMemcpyAsync(spins, s_ws, (size_t)n * N, cudaMemcpyDeviceToHost, st));
        if (logpsi && !d_lp)
            PSR_TRY(cudaMemcpyAsync(logpsi, lp_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
        if (!d_theta || !d_u || !d_s || !d_lp) return take_status(ctx);
        return PSR_OK;
    }
    // samples per CTA: measured by the autotuner when it is on; otherwise
    // the most that still gives every SM a CTA (weights are read once per
    // CTA and site, so more samples per CTA read less)
    std::vector<int> cands;
    for (int b : {4, 8, 16})
        if (sample_lru_smem_bytes(b, nL, H) <= 220 * 1024) cands.push_back(b);
    int per_cta = 4;
    for (int b : {16, 8})
        if ((n + b - 1) / b >= ctx->num_sms && sample_lru_smem_bytes(b, nL, H) <= 220 * 1024) {
            per_cta = b;
            break;
        }
    const int64_t key2 = (int64_t)nL * 1024 + H;
    bool tune_now = false;
    if (const psr_context::Tuned *t = find_tuned(ctx, kTuneSampleLru, n, N, key2))
        per_cta = t->v0;
    else if (ctx->autotune && !ctx->capturing) tune_now = true;
    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_PACK);
        PSR_TRY(launch_pack_theta_lru(theta, f, pk, st));
    }
    if (tune_now) {
        int bi = 0;
        float best = 0.0f;
        rc = measure_candidates(ctx, (int)cands.size(), [&](int i) {
            return from_cuda(launch_sample_lru(cands[i], pk, f, uu, n, N, params->u1_mask, so, lo, st));
        }, &bi, &best);
        if (rc != PSR_OK) return rc;
        per_cta = cands[bi];
        ctx->tuned.push_back(psr_context::Tuned{kTuneSampleLru, n, N, key2, per_cta, 0, best});
    }
    {
        StageScope sc(ctx, PSR_STAGE_SAMPLE);
        PSR_TRY(launch_sample_lru(per_cta, pk, f, uu, n, N, params->u1_mask, so, lo, st));
    }
    if (!d_s) PSR_TRY(cudaMemcpyAsync(spins, s_ws, (size_t)n * N, cudaMemcpyDeviceToHost, st));
    if (logpsi && !d_lp) PSR_TRY(cudaMemcpyAsync(logpsi, lp_ws, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (!d_theta || !d_u || !d_s || !d_lp) return take_status(ctx);
    return PSR_OK;
}

int psr_lru_grad(const psr_params *params, const uint8_t *spins, int64_t n, int32_t L, const float *dout,
                 float *dparams) {
    int rc = check_params_lru(params, n, L);
    if (rc != PSR_OK) return rc;
    if (!spins || !dparams) return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden, N = L;
    const int64_t P = param_count_lru(nL, H);
    const LruLayout f = lru_layout(nL, H);
    const TLruLayout tl = tlru_layout(nL, H);
    const int W = (int)words_per_row(N);
    const int nch = (N + kChunkLru - 1) / kChunkLru;
    int dev_smem = 0;
    cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device);
    int per_sm = (int)(dev_smem / (bwd_lru_smem_bytes(H) + 1024));
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
    int64_t grid64 = (int64_t)ctx->num_sms * per_sm;
    if (grid64 > n) grid64 = n;
    const int grid = (int)grid64;
    const size_t rows = dout ? (size_t)grid : (size_t)n;
    const bool d_theta = is_device_ptr(params->theta), d_s = is_device_ptr(spins),
               d_dout = dout ? is_device_ptr(dout) : true, d_g = is_device_ptr(dparams);
    float *theta_ws = nullptr, *dout_ws = nullptr, *g_ws = nullptr, *pk = nullptr, *lpsi = nullptr,
          *carries = nullptr, *scratch = nullptr, *partial = nullptr;
    uint8_t *s_ws = nullptr;
    uint64_t *bits = nullptr;
    unsigned long long *counter = nullptr;
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : P);
        s_ws = c.get<uint8_t>(d_s ? 0 : (size_t)n * N);
        dout_ws = c.get<float>(d_dout ? 0 : n);
        g_ws = c.get<float>(d_g ? 0 : (dout ? P : (size_t)n * P));
        pk = c.get<float>(f.total);
        bits = c.get<uint64_t>((size_t)n * W);
        lpsi = c.get<float>(n);
        carries = c.get<float>((size_t)n * nch * nL * 2 * H);
        scratch = c.get<float>((size_t)grid * bwd_lru_scratch_floats_per_cta(nL, H));
        partial = c.get<float>(dout ? rows * P : 0);
        counter = c.get<unsigned long long>(1);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;
    const float *theta = nullptr, *dv = nullptr;
    const uint8_t *sp = nullptr;
    if ((rc = stage_in(params->theta, theta_ws, P, d_theta, st, &theta)) != PSR_OK) return rc;
    if ((rc = stage_in(spins, s_ws, (size_t)n * N, d_s, st, &sp)) != PSR_OK) return rc;
    if (dout && (rc = stage_in(dout, dout_ws, n, d_dout, st, &dv)) != PSR_OK) return rc;
    float *g = d_g ? dparams : g_ws;
    reset_stages(ctx);
    {
        StageScope sc(ctx, PSR_STAGE_PACK);
        PSR_TRY(launch_pack_theta_lru(theta, f, pk, st));
        PSR_TRY(launch_bitpack(sp, n, N, W, bits, ctx->status, st));  // spin-byte check
        PSR_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
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
    js.g[0].carries_out = carries;
    js.job_counter = counter;
    js.status = ctx->status;
    {
        StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
        PSR_TRY(launch_lru_f32(js, pk, f, ctx->num_sms, st));
    }
    {
        StageScope sc(ctx, PSR_STAGE_BWD);
        float *out_rows = dout ? partial : g;
        PSR_TRY(cudaMemsetAsync(out_rows, 0, rows * P * sizeof(float), st));
        PSR_TRY(launch_bwd_lru(bits, n, N, W, params->u1_mask, theta, tl, pk, f, carries, dv, out_rows, grid,
                               scratch, st));
        if (dout) PSR_TRY(launch_reduce_rows(partial, grid, P, g, st));
    }
    if (!d_g)
        PSR_TRY(cudaMemcpyAsync(dparams, g_ws, (dout ? P : (size_t)n * P) * sizeof(float),
                                cudaMemcpyDeviceToHost, st));
    if (!d_g || !d_s || !d_theta || !d_dout) return take_status(ctx);
    return PSR_OK;
}

}  // extern "C"
