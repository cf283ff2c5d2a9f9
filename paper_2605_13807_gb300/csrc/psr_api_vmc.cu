// C ABI: c4v-symmetrised amplitudes and local energies, and the on-device
// VMC step.
#include "psr_api_common.cuh"

using namespace psr;
using namespace psr::apiutil;

// ------------------------------------- c4v symmetrisation and the VMC step

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

int psr2d_vmc_step(const psr_params *params, const psr_hamiltonian *ham, int32_t symmetrize,
                   const float *uniforms, const float *sym_uniforms, int64_t n, const psr_adam *adam,
                   float *theta_out, uint8_t *spins_out, float *eloc_out, double *stats_out,
                   float *grad_out) {
    int rc = check_ham(ham);
    if (rc != PSR_OK) return rc;
    if (!params || !params->ctx || !params->theta) return PSR_EINVAL;
    if (symmetrize != 0 && symmetrize != 1) return PSR_EINVAL;
    if (symmetrize && (ham->Lx != ham->Ly || !sym_uniforms || n > ((int64_t)1 << 28))) return PSR_EINVAL;
    if (!uniforms || !adam || !adam->m || !adam->v || !theta_out || adam->step < 1 || n < 1)
        return PSR_EINVAL;
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
    const int Lx = ham->Lx, Ly = ham->Ly, N = Lx * Ly;
    const int n_img = symmetrize ? 8 : 1;
    int64_t P = 0;
    if ((rc = psr2d_param_count(params->n_layers, params->hidden, &P)) != PSR_OK) return rc;
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
    // BF16 precision selects the tensor-core forward for the local energies
    // only; sampling, the image weights and the gradient run in FP32.
    psr_params p32 = *params;
    p32.precision = PSR_FP32;
    // 1. exact samples of |psi|^2 (then a uniformly drawn c4v image of each)
    if ((rc = psr2d_sample(&p32, uniforms, n, Lx, Ly, spins, nullptr)) != PSR_OK) return rc;
    const uint8_t *used = spins;
    if (symmetrize) {
        PSR_TRY(launch_c4v_pick(spins, sym_uniforms, n, Lx, spins_sym, st));
        used = spins_sym;
    }
    // 2. local energies and their FP64 statistics
    rc = symmetrize ? psr2d_sym_local_energy(params, used, n, ham, eloc, stats)
                    : psr2d_local_energy(params, used, n, ham, eloc, stats);
    if (rc != PSR_OK) return rc;
    // 3. centred energy-gradient weights (per image when symmetrised)
    if (symmetrize) {
        PSR_TRY(launch_c4v_images(used, n, Lx, imgs, st));
        if ((rc = psr2d_logpsi(&p32, imgs, 8 * n, Lx, Ly, lp8)) != PSR_OK) return rc;
    }
    PSR_TRY(launch_vmc_dout(eloc, stats, lp8, n, n_img, dout, st));
    // 4. gradient sum_i dout_i d log psi(s_i) / d theta
    if ((rc = psr2d_grad(&p32, symmetrize ? imgs : used, n_img * n, Lx, Ly, dout, grad)) != PSR_OK)
        return rc;
    // 5. Adam update
    PSR_TRY(launch_adam(params->theta, grad, P, adam->lr, adam->beta1, adam->beta2, adam->eps,
                        adam->step, adam->m, adam->v, theta_out, st));
    return PSR_OK;
}

int psr_lru_vmc_step(const psr_params *params, const psr_hamiltonian *ham, const float *uniforms, int64_t n,
                     const psr_adam *adam, float *theta_out, uint8_t *spins_out, float *eloc_out,
                     double *stats_out, float *grad_out) {
    int rc = check_ham(ham);
    if (rc != PSR_OK) return rc;
    const int N = ham->Lx * ham->Ly;
    int64_t P = 0;
    if (!params || !params->ctx || !params->theta) return PSR_EINVAL;
    if ((rc = psr_lru_param_count(params->n_layers, params->hidden, &P)) != PSR_OK) return rc;
    if (!uniforms || !adam || !adam->m || !adam->v || !theta_out || adam->step < 1 || n < 1)
        return PSR_EINVAL;
    if (!(adam->lr >= 0.0f) || !(adam->beta1 >= 0.0f && adam->beta1 < 1.0f) ||
        !(adam->beta2 >= 0.0f && adam->beta2 < 1.0f) || !(adam->eps > 0.0f))
        return PSR_EINVAL;
    const void *dev_args[] = {params->theta, uniforms, adam->m, adam->v, theta_out};
    for (const void *p : dev_args)
        if (!is_device_ptr(p)) return PSR_EINVAL;
    if ((spins_out && !is_device_ptr(spins_out)) || (eloc_out && !is_device_ptr(eloc_out)) ||
        (stats_out && !is_device_ptr(stats_out)) || (grad_out && !is_device_ptr(grad_out)))
        return PSR_EINVAL;
    psr_context *ctx = params->ctx;
    uint8_t *spins = nullptr;
    float *eloc = nullptr, *dout = nullptr, *grad = nullptr;
    double *stats = nullptr;
    auto carve = [&](Carver &c) {
        spins = c.get<uint8_t>(spins_out ? 0 : (size_t)n * N);
        eloc = c.get<float>(eloc_out ? 0 : n);
        stats = c.get<double>(stats_out ? 0 : 3);
        dout = c.get<float>(n);
        grad = c.get<float>(grad_out ? 0 : P);
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws2(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws2);
    carve(cv);
    if (spins_out) spins = spins_out;
    if (eloc_out) eloc = eloc_out;
    if (stats_out) stats = stats_out;
    if (grad_out) grad = grad_out;
    cudaStream_t st = ctx->stream;
    if ((rc = psr_lru_sample(params, uniforms, n, N, spins, nullptr)) != PSR_OK) return rc;
    if ((rc = psr_lru_local_energy(params, spins, n, ham, eloc, stats)) != PSR_OK) return rc;
    PSR_TRY(launch_vmc_dout(eloc, stats, nullptr, n, 1, dout, st));
    if ((rc = psr_lru_grad(params, spins, n, N, dout, grad)) != PSR_OK) return rc;
    PSR_TRY(launch_adam(params->theta, grad, P, adam->lr, adam->beta1, adam->beta2, adam->eps,
                        adam->step, adam->m, adam->v, theta_out, st));
    return PSR_OK;
}

}  // extern "C"
