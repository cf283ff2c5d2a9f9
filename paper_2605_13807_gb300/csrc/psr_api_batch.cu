// C ABI of libpsr: mixed batches of sample sets (several lattice sizes and
// Hamiltonians sharing one model) evaluated with one launch per kernel of the
// step.  psr_step_batch gives every item what psr_logpsi, psr_local_energy
// and psr_grad would give it; psr_local_energy_batch is its E_loc-only form.
//
// Launches of one call: parameter packing, bit-packing and the connected-set
// generator per item (small), then ONE sample forward over the samples of all
// items, ONE persistent forward over the connected configurations of all
// items (ragged over samples and lattices), the E_loc gathers, ONE FP32
// forward on gradient chunks and ONE reverse-scan gradient over the samples
// of all gradient items.  With graphs enabled the whole sequence is captured
// once per argument set and replayed.
#include "psr_api_common.cuh"

using namespace psr;
using namespace psr::apiutil;

namespace {

struct StepItem {
    const uint8_t *samples;
    int64_t n;
    psr_hamiltonian ham;
    int32_t u1;
    float *logpsi;
    float *eloc;
    double *stats;
    float *grad;
};

int step_batch_impl(const psr_params *params, const StepItem *items, int n_items,
                    const void *key_bytes, size_t key_len) {
    if (!params || !items || n_items < 1 || n_items > kMaxGroups) return PSR_EINVAL;
    int rc;
    for (int i = 0; i < n_items; ++i) {
        const StepItem &it = items[i];
        if ((rc = check_ham(&it.ham)) != PSR_OK) return rc;
        if (it.u1 != 0 && it.u1 != 1) return PSR_EINVAL;
        psr_params pi = *params;
        pi.u1_mask = it.u1;
        if ((rc = check_params(&pi, it.n, it.ham.Lx * it.ham.Ly)) != PSR_OK) return rc;
        if (!it.samples || (!it.logpsi && !it.eloc && !it.grad)) return PSR_EINVAL;
        if (it.stats && !it.eloc) return PSR_EINVAL;
    }
    psr_context *ctx = params->ctx;
    const int nL = params->n_layers, H = params->hidden;
    const bool bf16 = params->precision == PSR_BF16;
    const int CHmin = bf16 ? kChunkBF16 : kChunkGrad;  // E_loc carries sized for the shortest chunk
    const ThetaLayout tl = theta_layout(nL, H);
    const F32Layout fl = f32_layout(nL, H);
    const int64_t P = tl.total;
    const bool d_theta = is_device_ptr(params->theta);
    bool all_device = d_theta;

    struct ItemWs {
        bool d_s, d_lp, d_el, d_st, d_g;
        uint8_t *s_ws;
        float *lp_ws, *el_ws, *g_ws;
        double *st_ws;
        uint64_t *bits;
        ConnBufs b;
        float *lpsi, *logp, *carries, *delta;  // sample forward / E_loc
        float *carries_g, *lpsi_g;             // gradient forward
        int N, W, nb;
        int64_t cap;
    } w[kMaxGroups];
    int64_t n_grad = 0;
    for (int i = 0; i < n_items; ++i) {
        const StepItem &it = items[i];
        ItemWs &x = w[i];
        x.d_s = is_device_ptr(it.samples);
        x.d_lp = it.logpsi ? is_device_ptr(it.logpsi) : true;
        x.d_el = it.eloc ? is_device_ptr(it.eloc) : true;
        x.d_st = it.stats ? is_device_ptr(it.stats) : true;
        x.d_g = it.grad ? is_device_ptr(it.grad) : true;
        all_device = all_device && x.d_s && x.d_lp && x.d_el && x.d_st && x.d_g;
        x.N = it.ham.Lx * it.ham.Ly;
        x.W = (int)words_per_row(x.N);
        x.nb = bond_count(it.ham.Lx, it.ham.Ly, it.ham.pbc);
        x.cap = it.eloc ? it.n * max_entries_per_sample(&it.ham) : 0;
        if (it.grad) n_grad += it.n;
    }
    // gradient launch geometry: as psr_grad (CTAs per SM by shared memory)
    int grad_grid = 0;
    if (n_grad > 0) {
        int dev_smem = 0;
        cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device);
        int occ = (int)(dev_smem / (bwd_smem_bytes(H, nL) + 1024));
        occ = occ < 1 ? 1 : (occ > 4 ? 4 : occ);
        int64_t g = (int64_t)ctx->num_sms * occ;
        grad_grid = (int)(g > n_grad ? n_grad : g);
    }

    // BF16 gradients run on the tensor cores one item after another (as
    // psr_grad does), through one set of batch buffers sized for the largest
    const bool use_tc = bf16 && H == 128;
    size_t tc_stash = 0, tc_arr = 0;
    if (use_tc) {
        for (int i = 0; i < n_items; ++i) {
            if (!items[i].grad) continue;
            const int64_t B = grad_tc_batch(nL, w[i].N, items[i].n);
            const size_t st_i = (size_t)B * stash_floats_per_sample(nL, 128, w[i].N);
            const size_t ar_i = (size_t)B * 128 * stash_npad(w[i].N);
            tc_stash = st_i > tc_stash ? st_i : tc_stash;
            tc_arr = ar_i > tc_arr ? ar_i : tc_arr;
        }
        grad_grid = 0;
    }
    GradTcWs tw{};
    float *theta_ws = nullptr, *pk = nullptr, *tape = nullptr;
    void *pkb = nullptr;
    unsigned long long *counters = nullptr;
    auto carve = [&](Carver &c) {
        theta_ws = c.get<float>(d_theta ? 0 : P);
        pk = c.get<float>(fl.total);
        pkb = c.get<char>(bf16 ? bf16_packed_bytes() : 0);
        counters = c.get<unsigned long long>(3);
        tape = c.get<float>((size_t)grad_grid * bwd_tape_floats_per_cta(nL, H));
        if (use_tc && n_grad > 0) {
            tw.images = c.get<char>(bwd_tc_image_bytes(nL));
            tw.stash = c.get<float>(tc_stash);
            for (int k = 0; k < 2; ++k) {
                tw.gx[k] = c.get<float>(tc_arr);
                tw.gy[k] = c.get<float>(tc_arr);
            }
            tw.gh = c.get<float>(tc_arr);
            tw.dz = c.get<float>(tc_arr);
            tw.dc = c.get<float>(tc_arr);
        }
        for (int i = 0; i < n_items; ++i) {
            const StepItem &it = items[i];
            const int64_t n = it.n;
            ItemWs &x = w[i];
            const bool fwd = it.logpsi || it.eloc;
            const int nch = (x.N + CHmin - 1) / CHmin;
            const int nchg = (x.N + kChunkGrad - 1) / kChunkGrad;
            x.s_ws = c.get<uint8_t>(x.d_s ? 0 : (size_t)n * x.N);
            x.lp_ws = c.get<float>(x.d_lp ? 0 : n);
            x.el_ws = c.get<float>(x.d_el ? 0 : n);
            x.st_ws = c.get<double>(x.d_st ? 0 : 3);
            x.g_ws = c.get<float>(x.d_g ? 0 : (size_t)n * P);
            x.bits = c.get<uint64_t>((size_t)n * x.W);
            x.lpsi = c.get<float>(fwd && !it.logpsi ? n : 0);
            x.b.bonds = c.get<int32_t>(it.eloc ? 2 * (size_t)x.nb + 2 : 0);
            x.b.counts = c.get<int64_t>(it.eloc ? n : 0);
            x.b.offsets = c.get<int64_t>(it.eloc ? n + 1 : 0);
            x.b.diag = c.get<float>(it.eloc ? n : 0);
            x.b.entries = c.get<int32_t>(3 * (size_t)x.cap);
            x.logp = c.get<float>(it.eloc ? (size_t)n * x.N : 0);
            x.carries = c.get<float>(it.eloc ? (size_t)n * nch * nL * H : 0);
            x.delta = c.get<float>(x.cap);
            x.carries_g = c.get<float>(it.grad && !use_tc ? (size_t)n * nchg * nL * H : 0);
            x.lpsi_g = c.get<float>(it.grad && !use_tc ? n : 0);
        }
    };
    Carver sz;
    carve(sz);
    if ((rc = ensure_ws(ctx, sz.off)) != PSR_OK) return rc;
    Carver cv;
    cv.base = static_cast<char *>(ctx->ws);
    carve(cv);
    cudaStream_t st = ctx->stream;

    // forward shape of this batch (tuned on a call that is not captured)
    int Ns[kMaxGroups];
    int64_t ns[kMaxGroups];
    bool any_eloc = false;
    for (int i = 0; i < n_items; ++i) {
        Ns[i] = items[i].eloc ? w[i].N : -w[i].N;  // the key tells E_loc items apart
        ns[i] = items[i].n;
        any_eloc = any_eloc || items[i].eloc;
    }
    const FwdKey fkey = fwd_key(bf16, 2, n_items, Ns, ns);
    bool shape_tuned = false;
    fwd_shape(ctx, bf16, fkey, &shape_tuned);
    const bool tune_now = ctx->autotune && !shape_tuned && !ctx->fwd_shape_fixed[bf16];

    // graph replay when the arguments are the ones the cached graph was built for
    const bool use_graph = ctx->graphs && all_device && st != nullptr && !tune_now;
    std::vector<unsigned char> key;
    if (use_graph) {
        const unsigned char *pp = reinterpret_cast<const unsigned char *>(params);
        key.assign(pp, pp + sizeof(psr_params));
        const unsigned char *ip = static_cast<const unsigned char *>(key_bytes);
        key.insert(key.end(), ip, ip + key_len);
        if (ctx->graph_exec && key == ctx->graph_key && ctx->graph_ws_generation == ctx->ws_generation) {
            reset_stages(ctx);
            PSR_TRY(cudaGraphLaunch(ctx->graph_exec, st));
            return PSR_OK;
        }
        // kernel attributes are set outside the capture
        if (bf16) PSR_TRY(prepare_fwd_bf16());
        if (n_grad > 0 && !use_tc) PSR_TRY(prepare_bwd_f32(H, nL));
        if (n_grad > 0 && use_tc) PSR_TRY(prepare_bwd_tc());
        PSR_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        ctx->capturing = true;
    }

    auto enqueue = [&]() -> int {
        int r;
        const float *theta = nullptr;
        if ((r = stage_in(params->theta, theta_ws, P, d_theta, st, &theta)) != PSR_OK) return r;
        const uint8_t *sp[kMaxGroups];
        for (int i = 0; i < n_items; ++i)
            if ((r = stage_in(items[i].samples, w[i].s_ws, (size_t)items[i].n * w[i].N, w[i].d_s, st,
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
        }
        if (any_eloc) {
            StageScope sc(ctx, PSR_STAGE_GENERATOR);
            for (int i = 0; i < n_items; ++i) {
                hd[i] = HamDev{};
                if (!items[i].eloc) continue;
                if ((r = enqueue_connected(ctx, &items[i].ham, sp[i], items[i].n, w[i].b, hd[i])) != PSR_OK)
                    return r;
            }
        }
        // ---- forwards over the samples and the connected configurations
        FwdJobs js{}, jc{};
        js.mode = 0;
        jc.mode = 1;
        js.job_counter = counters;
        jc.job_counter = counters + 1;
        js.status = jc.status = ctx->status;
        for (int i = 0; i < n_items; ++i) {
            const StepItem &it = items[i];
            if (!it.logpsi && !it.eloc) continue;
            FwdGroup &a = js.g[js.n_groups++];
            a.u1 = it.u1;
            a.N = w[i].N;
            a.W = w[i].W;
            a.n_jobs = it.n;
            a.bits = w[i].bits;
            a.out = it.logpsi ? (w[i].d_lp ? it.logpsi : w[i].lp_ws) : w[i].lpsi;
            a.logp_out = it.eloc ? w[i].logp : nullptr;
            a.carries_out = it.eloc ? w[i].carries : nullptr;
            if (!it.eloc) continue;
            FwdGroup &b = jc.g[jc.n_groups++];
            b.u1 = it.u1;
            b.N = w[i].N;
            b.W = w[i].W;
            b.n_jobs = w[i].cap;
            b.n_jobs_dev = w[i].b.offsets + it.n;
            b.bits = w[i].bits;
            b.entries = w[i].b.entries;
            b.carries_in = w[i].carries;
            b.logp_ref = w[i].logp;
            b.out = w[i].delta;
        }
        auto run_fwd = [&](int shape) -> int {
            PSR_TRY(cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st));
            if (js.n_groups > 0) {
                StageScope sc(ctx, PSR_STAGE_FWD_SAMPLES);
                if (bf16) PSR_TRY(launch_fwd_bf16(js, pkb, pk, fl, ctx->num_sms, st, shape));
                else PSR_TRY(launch_fwd_f32(js, pk, fl, ctx->num_sms, st, shape));
            }
            if (jc.n_groups > 0) {
                StageScope sc(ctx, PSR_STAGE_FWD_CONNECTED);
                if (bf16) PSR_TRY(launch_fwd_bf16(jc, pkb, pk, fl, ctx->num_sms, st, shape));
                else PSR_TRY(launch_fwd_f32(jc, pk, fl, ctx->num_sms, st, shape));
            }
            return PSR_OK;
        };
        int shape = 0;
        if ((r = tune_fwd_shape(ctx, bf16, fkey, run_fwd, &shape)) != PSR_OK) return r;
        if ((r = run_fwd(shape)) != PSR_OK) return r;
        if (any_eloc) {
            StageScope sc(ctx, PSR_STAGE_GATHER);
            for (int i = 0; i < n_items; ++i) {
                const StepItem &it = items[i];
                if (!it.eloc) continue;
                float *o = w[i].d_el ? it.eloc : w[i].el_ws;
                double *so = it.stats ? (w[i].d_st ? it.stats : w[i].st_ws) : nullptr;
                PSR_TRY(launch_eloc_gather(w[i].b.offsets, w[i].delta, w[i].b.diag, hd[i].coeff, it.n, o, st));
                if (so) PSR_TRY(launch_stats(o, it.n, so, st));
            }
        }
        // ---- gradient on the tensor cores (BF16), one item after another
        if (n_grad > 0 && use_tc) {
            StageScope sc(ctx, PSR_STAGE_BWD);
            for (int i = 0; i < n_items; ++i) {
                const StepItem &it = items[i];
                if (!it.grad) continue;
                tw.B = grad_tc_batch(nL, w[i].N, it.n);
                float *rows = w[i].d_g ? it.grad : w[i].g_ws;
                if ((r = enqueue_grad_tc(ctx, nL, it.u1, theta, pk, w[i].bits, it.n, w[i].N, w[i].W, rows, tw)) !=
                    PSR_OK)
                    return r;
            }
        }
        // ---- gradient: FP32 forward on gradient chunks, then the reverse scan
        if (n_grad > 0 && !use_tc) {
            FwdJobs jg{};
            jg.mode = 0;
            jg.job_counter = counters + 2;
            jg.status = ctx->status;
            BwdJobs bj{};
            bj.first[0] = 0;
            for (int i = 0; i < n_items; ++i) {
                const StepItem &it = items[i];
                if (!it.grad) continue;
                FwdGroup &a = jg.g[jg.n_groups++];
                a.u1 = it.u1;
                a.N = w[i].N;
                a.W = w[i].W;
                a.n_jobs = it.n;
                a.bits = w[i].bits;
                a.out = w[i].lpsi_g;
                a.carries_out = w[i].carries_g;
                float *rows = w[i].d_g ? it.grad : w[i].g_ws;
                bj.g[bj.n_groups] = BwdGroup{w[i].bits, w[i].N, w[i].W, it.u1, w[i].carries_g, nullptr, rows};
                bj.first[bj.n_groups + 1] = bj.first[bj.n_groups] + it.n;
                ++bj.n_groups;
            }
            {
                StageScope sc(ctx, PSR_STAGE_BWD);  // the gradient's forward and reverse pass
                PSR_TRY(cudaMemsetAsync(counters + 2, 0, sizeof(unsigned long long), st));
                PSR_TRY(launch_fwd_f32(jg, pk, fl, ctx->num_sms, st, kChunkGrad));
                for (int g = 0; g < bj.n_groups; ++g)
                    PSR_TRY(cudaMemsetAsync(bj.g[g].rows, 0, (size_t)(bj.first[g + 1] - bj.first[g]) * P * sizeof(float), st));
                PSR_TRY(launch_bwd_f32_groups(bj, theta, tl, pk, fl, grad_grid, tape, ctx->status, st));
            }
        }
        // ---- results to host arrays
        for (int i = 0; i < n_items; ++i) {
            const StepItem &it = items[i];
            const ItemWs &x = w[i];
            if (it.logpsi && !x.d_lp)
                PSR_TRY(cudaMemcpyAsync(it.logpsi, x.lp_ws, it.n * sizeof(float), cudaMemcpyDeviceToHost, st));
            if (it.eloc && !x.d_el)
                PSR_TRY(cudaMemcpyAsync(it.eloc, x.el_ws, it.n * sizeof(float), cudaMemcpyDeviceToHost, st));
            if (it.stats && !x.d_st)
                PSR_TRY(cudaMemcpyAsync(it.stats, x.st_ws, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
            if (it.grad && !x.d_g)
                PSR_TRY(cudaMemcpyAsync(it.grad, x.g_ws, (size_t)it.n * P * sizeof(float), cudaMemcpyDeviceToHost, st));
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

}  // namespace

extern "C" {

int psr_step_batch(const psr_params *params, const psr_step_item *items, int32_t n_items) {
    if (!params || !items || n_items < 1 || n_items > kMaxGroups) return PSR_EINVAL;
    StepItem it[kMaxGroups];
    for (int i = 0; i < n_items; ++i)
        it[i] = StepItem{items[i].samples, items[i].n,      items[i].ham,   items[i].u1_mask,
                         items[i].logpsi,  items[i].eloc,   items[i].stats, items[i].grad};
    // the graph key tells psr_step_batch argument sets from psr_local_energy_batch ones
    std::vector<unsigned char> kb(1, 2);
    const unsigned char *ip = reinterpret_cast<const unsigned char *>(items);
    kb.insert(kb.end(), ip, ip + sizeof(psr_step_item) * n_items);
    return step_batch_impl(params, it, n_items, kb.data(), kb.size());
}

int psr_local_energy_batch(const psr_params *params, const psr_batch_item *items, int32_t n_items) {
    if (!params || !items || n_items < 1 || n_items > kMaxGroups) return PSR_EINVAL;
    StepItem it[kMaxGroups];
    for (int i = 0; i < n_items; ++i) {
        if (!items[i].out) return PSR_EINVAL;
        it[i] = StepItem{items[i].samples, items[i].n, items[i].ham, items[i].u1_mask,
                         nullptr,          items[i].out, items[i].stats, nullptr};
    }
    std::vector<unsigned char> kb(1, 1);
    const unsigned char *ip = reinterpret_cast<const unsigned char *>(items);
    kb.insert(kb.end(), ip, ip + sizeof(psr_batch_item) * n_items);
    return step_batch_impl(params, it, n_items, kb.data(), kb.size());
}

int psr_context_set_fwd_shape(psr_context *ctx, int32_t precision, int32_t shape) {
    if (ctx && precision == PSR_FP16) return PSR_EUNSUPPORTED;
    if (!ctx || (precision != PSR_FP32 && precision != PSR_BF16)) return PSR_EINVAL;
    const bool bf16 = precision == PSR_BF16;
    if (shape != 0 && !fwd_shape_valid(bf16, shape)) return PSR_EINVAL;
    ctx->fwd_shape_fixed[bf16] = shape;
    return PSR_OK;
}

int psr_fwd_shape_for(psr_context *ctx, int32_t precision, int32_t what, int32_t n_sets, const int64_t *n,
                      const int32_t *L, int32_t *shape, int32_t *tuned) {
    if (ctx && precision == PSR_FP16) return PSR_EUNSUPPORTED;
    if (!ctx || !shape || !n || !L || (precision != PSR_FP32 && precision != PSR_BF16) || what < 0 ||
        what > 2 || n_sets < 1 || n_sets > kMaxGroups || (what < 2 && n_sets != 1))
        return PSR_EINVAL;
    const bool bf16 = precision == PSR_BF16;
    int32_t Ns[kMaxGroups];
    for (int i = 0; i < n_sets; ++i) {
        if (n[i] < 1 || L[i] < 1) return PSR_EINVAL;
        Ns[i] = L[i];  // batch sets with E_loc (the key of psr_step_batch)
    }
    bool t = false;
    *shape = fwd_shape(ctx, bf16, fwd_key(bf16, what, n_sets, Ns, n), &t);
    if (tuned) *tuned = t ? 1 : 0;
    return PSR_OK;
}

}  // extern "C"
