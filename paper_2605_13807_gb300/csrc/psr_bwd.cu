// Reverse-mode gradient d log psi / d theta (FP32, SIMT).
//
// For each sample the chunks are visited in reverse order.  A chunk is first
// recomputed from the chunk-boundary carries stored by the forward (so no
// hidden state of the whole sequence is kept), writing a per-CTA tape of the
// chunk's inputs u, gates a, candidates h~, states h and pre-activations y.
// The adjoint then runs layer by layer from the top:
//   readout   g_t = 1/2 (s_t - P(1 | .))   on the logit difference
//   output    gy = gx * GELU'(y);  dC += gy h^T,  dD += gy u^T
//             dL/dh (direct) = C^T gy  (+ gy of layer l+1 when l+1 >= 2: the
//             residual s^(l+1) = h^(l))
//   scan      lambda_t = dL/dh_t (direct) + a_{t+1} lambda_{t+1}  (reverse scan
//             of h_t = a_t h_{t-1} + (1 - a_t) h~_t, Sec. II.C)
//             da = lambda (h_{t-1} - h~),  dh~ = lambda (1 - a),  dz = da a (1 - a)
//   inputs    dW_z += dz u^T, dW_h += dh~ u^T, gx(l-1) = W_z^T dz + W_h^T dh~ + D^T gy
// lambda_t and a_{t+1} cross chunk boundaries in shared memory.  Thread j owns
// hidden unit j for the per-unit work and input unit k = j for the
// weight-gradient rows, which makes every parameter update a coalesced
// reduction issued by exactly one thread.  The updates are fire-and-forget
// global reductions (no value returned, so the warp does not wait on memory);
// a single writer per address adds in program order, so the sums are
// deterministic.
#include <cuda_runtime.h>

#include "psr_device.cuh"
#include "psr_internal.cuh"

namespace psr {

namespace {
constexpr int CH = kChunkGrad;
constexpr int LD = CH + 4;
enum { TQ_U = 0, TQ_A = 1, TQ_C = 2, TQ_H = 3, TQ_Y = 4, TQ_N = 5 };
}  // namespace

__host__ __device__ inline size_t tape_floats(int nL, int H) { return (size_t)nL * TQ_N * CH * H; }
size_t bwd_tape_floats_per_cta(int nL, int H) { return tape_floats(nL, H); }

// Shared memory of one CTA.  The per-layer carries that follow the struct
// (hc0, hcar, lam, anext: [nL][H] each) are sized by the layer count.
template <int H>
struct BwdSmem {
    union {
        float xs[H * LD];    // forward recompute: layer input tile [k][t]
        float gy[H * LD];    // layer loop: gy, one padded row per unit [j][t]
    };
    float hs[H * LD];        // forward recompute: hidden tile [k][t]
    float gzc[2 * H * LD];   // gz, gc [j][t] (padded unit rows) in the layer
                             // loop; before it the last-layer output xl [t][k]
    float g1[CH];
    int code[CH];
};
static_assert(CH * (128 + 1) <= 2 * 128 * LD, "xl fits in the gz / gc storage");

template <int H>
__global__ void __launch_bounds__(H, 4) bwd_f32_kernel(
    const __grid_constant__ BwdJobs bj, const float *__restrict__ theta, ThetaLayout tl,
    const float *__restrict__ pk, F32Layout fl, float *__restrict__ tape_all, int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem<H> &S = *reinterpret_cast<BwdSmem<H> *>(smem_raw);
    const int j = threadIdx.x;
    const int nL = tl.nL;
    struct {
        float *hc0, *hcar, *lam, *anext, *gz, *gc, *xl;
    } V;
    {
        float *tail = reinterpret_cast<float *>(smem_raw + sizeof(BwdSmem<H>));
        V.hc0 = tail;               // carry at chunk start (= h_{t0-1})
        V.hcar = tail + nL * H;     // running carry during recompute
        V.lam = tail + 2 * nL * H;  // adjoint carry lambda_{t0+CH}
        V.anext = tail + 3 * nL * H;  // a_{t0+CH} of the later chunk
        V.gz = S.gzc;
        V.gc = S.gzc + H * LD;
        V.xl = S.gzc;
    }
    const int64_t P = tl.total;
    float *tape = tape_all + (size_t)blockIdx.x * tape_floats(nL, H);
    auto T = [&](int l, int q, int t) -> float * {
        return tape + (((size_t)l * TQ_N + q) * CH + t) * H;
    };

    const float a0_0 = pk[fl.A0 + j], a0_1 = pk[fl.A0 + H + j], a0_2 = pk[fl.A0 + 2 * H + j];
    const float b0_0 = pk[fl.B0 + j], b0_1 = pk[fl.B0 + H + j], b0_2 = pk[fl.B0 + 2 * H + j];
    const float d0_0 = pk[fl.DU0 + j], d0_1 = pk[fl.DU0 + H + j], d0_2 = pk[fl.DU0 + 2 * H + j];
    const float c0_0 = pk[fl.CD0 + j], c0_1 = pk[fl.CD0 + H + j], c0_2 = pk[fl.CD0 + 2 * H + j];
    const float bd = pk[fl.bd];
    const float wdj = pk[fl.wd + j];

    // samples of all groups in order; sample s of group gi is sample s - first[gi] there
    for (int64_t sg = blockIdx.x; sg < bj.first[bj.n_groups]; sg += gridDim.x) {
        int gi = 0;
        while (gi + 1 < bj.n_groups && sg >= bj.first[gi + 1]) ++gi;
        const BwdGroup &BG = bj.g[gi];
        const int64_t s = sg - bj.first[gi];
        const int N = BG.N, u1 = BG.u1;
        const int nch = (N + CH - 1) / CH;
        const float *carries = BG.carries;
        const uint64_t *row = BG.bits + s * BG.W;
        const float scale = BG.dout ? BG.dout[s] : 1.0f;
        float *G = BG.dout ? BG.rows + (size_t)blockIdx.x * P : BG.rows + (size_t)s * P;
        for (int l = 0; l < nL; ++l) {
            V.lam[l * H + j] = 0.0f;
            V.anext[l * H + j] = 0.0f;
        }
        float gbz[kMaxLayers], gbh[kMaxLayers];
#pragma unroll
        for (int l = 0; l < kMaxLayers; ++l) { gbz[l] = 0.0f; gbh[l] = 0.0f; }

        for (int c = nch - 1; c >= 0; --c) {
            const int t0 = c * CH;
            // ------------------------------------------------ recompute chunk
            for (int l = 0; l < nL; ++l) {
                const float v = carries[(((int64_t)s * nch + c) * nL + l) * H + j];
                V.hc0[l * H + j] = v;
                V.hcar[l * H + j] = v;
            }
            uint32_t cur, prev;
            chunk_bits32(row, t0, -1, -1, cur, prev);
            const int nvalid = min(CH, N - t0);
            cur &= (1u << nvalid) - 1u;
            const uint32_t prevbits = (cur << 1) | prev;
            if (j < CH) S.code[j] = (t0 + j == 0) ? 0 : 1 + (int)((prevbits >> j) & 1u);
            float hprevl[CH];
            {
                float hv = V.hcar[j];
                float y[CH];
#pragma unroll
                for (int t = 0; t < CH; ++t) {
                    const bool first = (t0 + t == 0);
                    const uint32_t sb = (prevbits >> t) & 1u;
                    const float a = first ? a0_0 : (sb ? a0_2 : a0_1);
                    const float b = first ? b0_0 : (sb ? b0_2 : b0_1);
                    const float cd = first ? c0_0 : (sb ? c0_2 : c0_1);
                    hv = a * hv + b;
                    hprevl[t] = hv;
                    y[t] = first ? d0_0 : (sb ? d0_2 : d0_1);
                    T(0, TQ_A, t)[j] = a;
                    T(0, TQ_C, t)[j] = cd;
                    T(0, TQ_H, t)[j] = hv;
                    S.hs[j * LD + t] = hv;
                }
                __syncthreads();
                const float *Ct = pk + fl.CT[0];
                #pragma unroll 4
                for (int k = 0; k < H; ++k) {
                    const float w = Ct[k * H + j];
                    const float4 *src = reinterpret_cast<const float4 *>(S.hs + k * LD);
#pragma unroll
                    for (int t4 = 0; t4 < CH / 4; ++t4) {
                        float4 v = src[t4];
                        y[4 * t4] += w * v.x; y[4 * t4 + 1] += w * v.y;
                        y[4 * t4 + 2] += w * v.z; y[4 * t4 + 3] += w * v.w;
                    }
                }
#pragma unroll
                for (int t = 0; t < CH; ++t) {
                    T(0, TQ_Y, t)[j] = y[t];
                    S.xs[j * LD + t] = gelu_f(y[t]);
                }
                __syncthreads();
            }
            for (int l = 1; l < nL; ++l) {
                float z[CH], y[CH];
                const float bz = pk[fl.bz[l] + j], bh = pk[fl.bh[l] + j];
#pragma unroll
                for (int t = 0; t < CH; ++t) {
                    z[t] = bz;
                    y[t] = bh;
                    T(l, TQ_U, t)[j] = S.xs[j * LD + t];
                }
                const float *Wz = pk + fl.WzT[l];
                const float *Wh = pk + fl.WhT[l];
                #pragma unroll 4
                for (int k = 0; k < H; ++k) {
                    const float wz = Wz[k * H + j], wh = Wh[k * H + j];
                    const float4 *src = reinterpret_cast<const float4 *>(S.xs + k * LD);
#pragma unroll
                    for (int t4 = 0; t4 < CH / 4; ++t4) {
                        float4 v = src[t4];
                        z[4 * t4] += wz * v.x; z[4 * t4 + 1] += wz * v.y;
                        z[4 * t4 + 2] += wz * v.z; z[4 * t4 + 3] += wz * v.w;
                        y[4 * t4] += wh * v.x; y[4 * t4 + 1] += wh * v.y;
                        y[4 * t4 + 2] += wh * v.z; y[4 * t4 + 3] += wh * v.w;
                    }
                }
                float hn[CH];
                {
                    float hv = V.hcar[l * H + j];
#pragma unroll
                    for (int t = 0; t < CH; ++t) {
                        const float a = sigmoid_f(z[t]);
                        hv = a * hv + (1.0f - a) * y[t];
                        hn[t] = hv;
                        T(l, TQ_A, t)[j] = a;
                        T(l, TQ_C, t)[j] = y[t];
                        T(l, TQ_H, t)[j] = hv;
                    }
                    V.hcar[l * H + j] = hv;
                }
                __syncthreads();  // everyone done reading hs of the previous layer
#pragma unroll
                for (int t = 0; t < CH; ++t) S.hs[j * LD + t] = hn[t];
                __syncthreads();
#pragma unroll
                for (int t = 0; t < CH; ++t) y[t] = (l >= 2) ? hprevl[t] : 0.0f;
                const float *Ct = pk + fl.CT[l];
                const float *Dt = pk + fl.DT[l];
                #pragma unroll 4
                for (int k = 0; k < H; ++k) {
                    const float wc = Ct[k * H + j], wd = Dt[k * H + j];
                    const float4 *sh = reinterpret_cast<const float4 *>(S.hs + k * LD);
                    const float4 *sx = reinterpret_cast<const float4 *>(S.xs + k * LD);
#pragma unroll
                    for (int t4 = 0; t4 < CH / 4; ++t4) {
                        float4 vh = sh[t4], vx = sx[t4];
                        y[4 * t4] += wc * vh.x + wd * vx.x;
                        y[4 * t4 + 1] += wc * vh.y + wd * vx.y;
                        y[4 * t4 + 2] += wc * vh.z + wd * vx.z;
                        y[4 * t4 + 3] += wc * vh.w + wd * vx.w;
                    }
                }
                __syncthreads();
#pragma unroll
                for (int t = 0; t < CH; ++t) {
                    T(l, TQ_Y, t)[j] = y[t];
                    S.xs[j * LD + t] = gelu_f(y[t]);
                    hprevl[t] = hn[t];
                }
                __syncthreads();
            }
            // ------------------------------------------------ readout adjoint
            for (int t = 0; t < CH; ++t) V.xl[t * (H + 1) + j] = S.xs[j * LD + t];
            __syncthreads();
            if (j < CH) {
                const int t = j;
                float d = bd;
                const float *wd = pk + fl.wd;
                for (int k = 0; k < H; ++k) d += wd[k] * V.xl[t * (H + 1) + k];
                float g = 0.0f;
                const int tt = t0 + t;
                if (tt < N) {
                    const int sv = (cur >> t) & 1u;
                    g = 0.5f * ((float)sv - 1.0f / (1.0f + expf(-d)));
                }
                S.g1[t] = g;
            }
            __syncthreads();
            if (u1 && j == 0) {
                // forced sites carry no parameter dependence
                const int n_up0 = count_up_before(row, t0);
                for (int t = 0; t < CH && t0 + t < N; ++t) {
                    const int nu = n_up0 + __popc(cur & ((1u << t) - 1u));
                    if (u1_forced(u1, N, t0 + t, nu) >= 0) S.g1[t] = 0.0f;
                }
            }
            __syncthreads();
            if (j < CH) S.g1[j] *= scale;
            __syncthreads();
            {
                float gw = 0.0f, gb = 0.0f;
                for (int t = 0; t < CH; ++t) {
                    gw += S.g1[t] * V.xl[t * (H + 1) + j];
                    gb += S.g1[t];
                }
                atomicAdd(&G[tl.Wo + H + j], gw);
                atomicAdd(&G[tl.Wo + j], -(gw));
                if (j == 0) {
                    atomicAdd(&G[tl.bo + 1], gb);
                    atomicAdd(&G[tl.bo], -(gb));
                }
            }
            // ------------------------------------------------ layers, top down
            float gx[CH];
#pragma unroll
            for (int t = 0; t < CH; ++t) gx[t] = S.g1[t] * wdj;
            float gy_up[CH];  // gy of layer l+1 (residual path into h^(l))
#pragma unroll
            for (int t = 0; t < CH; ++t) gy_up[t] = 0.0f;
            for (int l = nL - 1; l >= 0; --l) {
                const int din = (l == 0) ? 2 : H;
                float gy[CH];
#pragma unroll
                for (int t = 0; t < CH; ++t) gy[t] = gx[t] * gelu_grad_f(T(l, TQ_Y, t)[j]);
                {
                    float4 *gyr = reinterpret_cast<float4 *>(S.gy + j * LD);
#pragma unroll
                    for (int t4 = 0; t4 < CH / 4; ++t4)
                        gyr[t4] = make_float4(gy[4 * t4], gy[4 * t4 + 1], gy[4 * t4 + 2], gy[4 * t4 + 3]);
                }
                __syncthreads();
                // k-role: direct dL/dh, D^T gy, dC, dD
                float hk[CH], uk[CH], ghd[CH], gud[CH];
#pragma unroll
                for (int t = 0; t < CH; ++t) {
                    hk[t] = T(l, TQ_H, t)[j];
                    uk[t] = (l >= 1) ? T(l, TQ_U, t)[j] : 0.0f;
                    ghd[t] = (l + 1 < nL && l + 1 >= 2) ? gy_up[t] : 0.0f;
                    gud[t] = 0.0f;
                }
                const float *Cw = theta + tl.C[l];
                const float *Dw = theta + tl.D[l];
                // weights of the next jj are fetched one iteration ahead
                float cjk_n = Cw[j];
                float djk_n = (l >= 1) ? Dw[j] : 0.0f;
                for (int jj = 0; jj < H; ++jj) {
                    const float cjk = cjk_n;
                    const float djk = djk_n;
                    if (jj + 1 < H) {
                        cjk_n = Cw[(int64_t)(jj + 1) * H + j];
                        djk_n = (l >= 1) ? Dw[(int64_t)(jj + 1) * H + j] : 0.0f;
                    }
                    float ac = 0.0f, ad = 0.0f;
                    const float4 *gr = reinterpret_cast<const float4 *>(S.gy + jj * LD);
#pragma unroll
                    for (int t4 = 0; t4 < CH / 4; ++t4) {
                        const float4 g4 = gr[t4];
                        const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int t = 4 * t4 + e;
                            const float g = gv[e];
                            ghd[t] += cjk * g;
                            gud[t] += djk * g;
                            ac += g * hk[t];
                            ad += g * uk[t];
                        }
                    }
                    atomicAdd(&G[tl.C[l] + (int64_t)jj * H + j], ac);
                    if (l >= 1) atomicAdd(&G[tl.D[l] + (int64_t)jj * H + j], ad);
                }
                if (l == 0) {
                    float d0 = 0.0f, d1 = 0.0f;
                    for (int t = 0; t < CH; ++t) {
                        const int cd = S.code[t];
                        if (cd == 1) d0 += gy[t];
                        if (cd == 2) d1 += gy[t];
                    }
                    atomicAdd(&G[tl.D[0] + 2 * j], d0);
                    atomicAdd(&G[tl.D[0] + 2 * j + 1], d1);
                }
                // reverse scan (thread j = hidden unit j)
                {
                    float lam = V.lam[l * H + j];
                    float an = V.anext[l * H + j];
                    float sz = 0.0f, sc = 0.0f;
#pragma unroll
                    for (int t = CH - 1; t >= 0; --t) {
                        lam = ghd[t] + an * lam;
                        const float a = T(l, TQ_A, t)[j];
                        const float cd = T(l, TQ_C, t)[j];
                        const float hp = (t > 0) ? hk[t - 1] : V.hc0[l * H + j];
                        const float ga = lam * (hp - cd);
                        const float gcv = lam * (1.0f - a);
                        const float gzv = ga * a * (1.0f - a);
                        ghd[t] = gzv;  // ghd[t] and hk[t] are not read again
                        hk[t] = gcv;
                        sz += gzv;
                        sc += gcv;
                        an = a;
                    }
                    float4 *gzr = reinterpret_cast<float4 *>(V.gz + j * LD);
                    float4 *gcr = reinterpret_cast<float4 *>(V.gc + j * LD);
#pragma unroll
                    for (int t4 = 0; t4 < CH / 4; ++t4) {
                        gzr[t4] = make_float4(ghd[4 * t4], ghd[4 * t4 + 1], ghd[4 * t4 + 2], ghd[4 * t4 + 3]);
                        gcr[t4] = make_float4(hk[4 * t4], hk[4 * t4 + 1], hk[4 * t4 + 2], hk[4 * t4 + 3]);
                    }
                    V.lam[l * H + j] = lam;
                    V.anext[l * H + j] = an;
                    gbz[l] += sz;
                    gbh[l] += sc;
                }
                __syncthreads();
                if (l >= 1) {
                    const float *Wzw = theta + tl.Wz[l];
                    const float *Whw = theta + tl.Wh[l];
                    float gn[CH];
#pragma unroll
                    for (int t = 0; t < CH; ++t) gn[t] = gud[t];
                    float wz_n = Wzw[j], wh_n = Whw[j];
                    for (int jj = 0; jj < H; ++jj) {
                        const float wz = wz_n;
                        const float wh = wh_n;
                        if (jj + 1 < H) {
                            wz_n = Wzw[(int64_t)(jj + 1) * H + j];
                            wh_n = Whw[(int64_t)(jj + 1) * H + j];
                        }
                        float az = 0.0f, ah = 0.0f;
                        const float4 *zr = reinterpret_cast<const float4 *>(V.gz + jj * LD);
                        const float4 *cr = reinterpret_cast<const float4 *>(V.gc + jj * LD);
#pragma unroll
                        for (int t4 = 0; t4 < CH / 4; ++t4) {
                            const float4 z4 = zr[t4], c4 = cr[t4];
                            const float zv[4] = {z4.x, z4.y, z4.z, z4.w}, cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int t = 4 * t4 + e;
                                gn[t] += wz * zv[e] + wh * cv[e];
                                az += zv[e] * uk[t];
                                ah += cv[e] * uk[t];
                            }
                        }
                        atomicAdd(&G[tl.Wz[l] + (int64_t)jj * H + j], az);
                        atomicAdd(&G[tl.Wh[l] + (int64_t)jj * H + j], ah);
                    }
#pragma unroll
                    for (int t = 0; t < CH; ++t) {
                        gx[t] = gn[t];
                        gy_up[t] = gy[t];
                    }
                } else {
                    float z0 = 0.0f, z1 = 0.0f, c0v = 0.0f, c1v = 0.0f;
                    for (int t = 0; t < CH; ++t) {
                        const int cd = S.code[t];
                        const float gzv = V.gz[j * LD + t], gcv = V.gc[j * LD + t];
                        if (cd == 1) { z0 += gzv; c0v += gcv; }
                        if (cd == 2) { z1 += gzv; c1v += gcv; }
                    }
                    atomicAdd(&G[tl.Wz[0] + 2 * j], z0);
                    atomicAdd(&G[tl.Wz[0] + 2 * j + 1], z1);
                    atomicAdd(&G[tl.Wh[0] + 2 * j], c0v);
                    atomicAdd(&G[tl.Wh[0] + 2 * j + 1], c1v);
                }
                (void)din;
                __syncthreads();
            }
        }
        for (int l = 0; l < nL; ++l) {
            atomicAdd(&G[tl.bz[l] + j], gbz[l]);
            atomicAdd(&G[tl.bh[l] + j], gbh[l]);
        }
        __syncthreads();
    }
    (void)status;
}

template <int H>
static cudaError_t prepare_bwd_h(int nL) {
    const size_t smem = sizeof(BwdSmem<H>) + 4 * (size_t)nL * H * sizeof(float);
    return cudaFuncSetAttribute(bwd_f32_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t prepare_bwd_f32(int H, int nL) {
    switch (H) {
        case 32: return prepare_bwd_h<32>(nL);
        case 64: return prepare_bwd_h<64>(nL);
        case 128: return prepare_bwd_h<128>(nL);
        default: return cudaErrorInvalidValue;
    }
}

template <int H>
static cudaError_t launch_bwd_h(const BwdJobs &bj, const float *theta, const ThetaLayout &tl,
                                const float *packed, const F32Layout &fl, int grid, float *tape,
                                int *status, cudaStream_t stream) {
    const size_t smem = sizeof(BwdSmem<H>) + 4 * (size_t)tl.nL * H * sizeof(float);
    cudaError_t e = prepare_bwd_h<H>(tl.nL);
    if (e != cudaSuccess) return e;
    bwd_f32_kernel<H><<<grid, H, smem, stream>>>(bj, theta, tl, packed, fl, tape, status);
    return cudaGetLastError();
}

cudaError_t launch_bwd_f32_groups(const BwdJobs &bj, const float *theta, const ThetaLayout &tl,
                                  const float *packed, const F32Layout &fl, int grid, float *tape,
                                  int *status, cudaStream_t stream) {
    if (bj.n_groups < 1 || bj.n_groups > kMaxGroups) return cudaErrorInvalidValue;
    switch (tl.H) {
        case 32: return launch_bwd_h<32>(bj, theta, tl, packed, fl, grid, tape, status, stream);
        case 64: return launch_bwd_h<64>(bj, theta, tl, packed, fl, grid, tape, status, stream);
        case 128: return launch_bwd_h<128>(bj, theta, tl, packed, fl, grid, tape, status, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_bwd_f32(const uint64_t *bits, int64_t n, int N, int W, int u1,
                           const float *theta, const ThetaLayout &tl, const float *packed,
                           const F32Layout &fl, const float *carries, const float *dout,
                           float *grad_rows, int grid, float *tape, int *status,
                           cudaStream_t stream) {
    BwdJobs bj{};
    bj.n_groups = 1;
    bj.first[0] = 0;
    bj.first[1] = n;
    bj.g[0] = BwdGroup{bits, N, W, u1, carries, dout, grad_rows};
    return launch_bwd_f32_groups(bj, theta, tl, packed, fl, grid, tape, status, stream);
}

size_t bwd_smem_bytes(int H, int nL) {
    const size_t tail = 4 * (size_t)nL * H * sizeof(float);
    switch (H) {
        case 32: return sizeof(BwdSmem<32>) + tail;
        case 64: return sizeof(BwdSmem<64>) + tail;
        default: return sizeof(BwdSmem<128>) + tail;
    }
}

// out[p] = sum_r partial[r][p] in row order (deterministic).
__global__ void reduce_rows_kernel(const float *__restrict__ partial, int rows, int64_t P,
                                   float *__restrict__ out) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int r = 0; r < rows; ++r) acc += partial[(size_t)r * P + p];
        out[p] = acc;
    }
}

cudaError_t launch_reduce_rows(const float *partial, int rows, int64_t P, float *out,
                               cudaStream_t stream) {
    int blocks = (int)((P + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    reduce_rows_kernel<<<blocks, 256, 0, stream>>>(partial, rows, P, out);
    return cudaGetLastError();
}

}  // namespace psr
