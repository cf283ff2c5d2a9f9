// Exact autoregressive sampling on the device (Sec. II.A and Sec. III.B: the
// model's conditionals P(s_t | s_<t) are drawn site by site, so samples are
// exact and independent, with no Markov chain).
//
// One CTA draws B samples; thread j owns hidden unit j of every layer for all
// B samples.  Site by site the CTA runs one step of each minGRU layer
// (Eq. minGRU; output map and residual of Sec. II.F-G) for its B samples,
// forms the logit difference d, and sets s_t = 1 iff u_t < P(s_t = 1) =
// sigmoid(d) (or the value the zero-magnetisation mask forces), using the
// caller's uniform u_t.  The decision feeds the next site's layer-0 input
// onehot(s_t).  Arithmetic is FP32 and its order does not depend on B or on a
// sample's slot in the CTA, so every B draws the same samples.
#include <cuda_runtime.h>

#include "psr_device.cuh"
#include "psr_internal.cuh"

namespace psr {

namespace {

template <int H, int B>
__global__ void __launch_bounds__(H) sample_kernel(const float *__restrict__ pk, F32Layout fl,
                                                   const float *__restrict__ unif, int64_t n, int N,
                                                   int u1, uint8_t *__restrict__ out,
                                                   float *__restrict__ logpsi) {
    constexpr int NW = H / 32;
    extern __shared__ __align__(16) float smem[];
    float *xs = smem;             // [B][H] layer input / output of the current site
    float *hs = xs + B * H;       // [B][H] hidden states of the current layer
    float *red = hs + B * H;      // [NW][B] readout partial sums
    float *hc = red + NW * B;     // [nL][B][H] recurrent carries
    __shared__ int s_prev[B], s_nup[B];
    __shared__ float s_acc[B];

    const int j = threadIdx.x;
    const int lane = j & 31, warp = j >> 5;
    const int nL = fl.nL;
    const int64_t first = (int64_t)blockIdx.x * B;

    for (int i = j; i < nL * B * H; i += H) hc[i] = 0.0f;
    if (j < B) {
        s_prev[j] = 0;
        s_nup[j] = 0;
        s_acc[j] = 0.0f;
    }
    const float a0_0 = pk[fl.A0 + j], a0_1 = pk[fl.A0 + H + j], a0_2 = pk[fl.A0 + 2 * H + j];
    const float b0_0 = pk[fl.B0 + j], b0_1 = pk[fl.B0 + H + j], b0_2 = pk[fl.B0 + 2 * H + j];
    const float d0_0 = pk[fl.DU0 + j], d0_1 = pk[fl.DU0 + H + j], d0_2 = pk[fl.DU0 + 2 * H + j];
    const float wdj = pk[fl.wd + j];
    const float bd = pk[fl.bd];
    __syncthreads();

    for (int t = 0; t < N; ++t) {
        float y[B];
        // layer 0: input onehot(s_{t-1}) (zero at t = 0) -> lookup tables
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int code = (t == 0) ? 0 : 1 + s_prev[b];
            const float a = code == 0 ? a0_0 : (code == 1 ? a0_1 : a0_2);
            const float bb = code == 0 ? b0_0 : (code == 1 ? b0_1 : b0_2);
            const float h = a * hc[b * H + j] + bb;
            hc[b * H + j] = h;
            hs[b * H + j] = h;
            y[b] = code == 0 ? d0_0 : (code == 1 ? d0_1 : d0_2);
        }
        __syncthreads();
        {
            const float *Ct = pk + fl.CT[0];
#pragma unroll 4
            for (int k = 0; k < H; ++k) {
                const float w = Ct[k * H + j];
#pragma unroll
                for (int b = 0; b < B; ++b) y[b] += w * hs[b * H + k];
            }
#pragma unroll
            for (int b = 0; b < B; ++b) xs[b * H + j] = gelu_f(y[b]);
        }
        __syncthreads();

        for (int l = 1; l < nL; ++l) {
            float z[B];
            const float bz = pk[fl.bz[l] + j], bh = pk[fl.bh[l] + j];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                z[b] = bz;
                y[b] = bh;
            }
            const float *Wz = pk + fl.WzT[l];
            const float *Wh = pk + fl.WhT[l];
#pragma unroll 4
            for (int k = 0; k < H; ++k) {
                const float wz = Wz[k * H + j], wh = Wh[k * H + j];
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const float xv = xs[b * H + k];
                    z[b] += wz * xv;
                    y[b] += wh * xv;
                }
            }
            float *hcl = hc + (size_t)l * B * H;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const float a = sigmoid_f(z[b]);
                // explicit rounding order: identical for every samples-per-CTA instance
                const float h = fmaf(a, hcl[b * H + j], __fmul_rn(1.0f - a, y[b]));
                hcl[b * H + j] = h;
                hs[b * H + j] = h;
            }
            __syncthreads();
            // residual s^l = h^(l-1) for l >= 2 (this unit's own carry)
            const float *hres = hc + (size_t)(l - 1) * B * H;
#pragma unroll
            for (int b = 0; b < B; ++b) y[b] = (l >= 2) ? hres[b * H + j] : 0.0f;
            const float *Ct = pk + fl.CT[l];
            const float *Dt = pk + fl.DT[l];
#pragma unroll 4
            for (int k = 0; k < H; ++k) {
                const float wc = Ct[k * H + j], wd = Dt[k * H + j];
#pragma unroll
                for (int b = 0; b < B; ++b) y[b] = fmaf(wd, xs[b * H + k], fmaf(wc, hs[b * H + k], y[b]));
            }
            __syncthreads();
#pragma unroll
            for (int b = 0; b < B; ++b) xs[b * H + j] = gelu_f(y[b]);
            __syncthreads();
        }

        // readout: d_b = bd + sum_j wd_j x_b[j], reduced in a fixed order
#pragma unroll
        for (int b = 0; b < B; ++b) {
            float v = wdj * xs[b * H + j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp * B + b] = v;
        }
        __syncthreads();
        if (j < B) {
            const int b = j;
            float d = bd;
#pragma unroll
            for (int w = 0; w < NW; ++w) d += red[w * B + b];
            const int64_t row = first + b;
            if (row < n) {
                const int forced = u1_forced(u1, N, t, s_nup[b]);
                const float p1 = forced >= 0 ? (float)forced : 1.0f / (1.0f + expf(-d));
                const int s = unif[row * N + t] < p1 ? 1 : 0;
                s_acc[b] += site_logp(d, s, forced);
                s_prev[b] = s;
                s_nup[b] += s;
                out[row * N + t] = (uint8_t)s;
            }
        }
        __syncthreads();
    }
    if (j < B && first + j < n && logpsi) logpsi[first + j] = 0.5f * s_acc[j];
}

template <int H, int B>
cudaError_t launch_sample_hb(const float *packed, const F32Layout &fl, const float *unif,
                             int64_t n, int N, int u1, uint8_t *out, float *logpsi,
                             cudaStream_t stream) {
    const size_t smem = ((size_t)2 * B * H + (size_t)(H / 32) * B + (size_t)fl.nL * B * H) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(sample_kernel<H, B>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (n + B - 1) / B;
    if (grid > 0x7fffffff) return cudaErrorInvalidValue;
    sample_kernel<H, B><<<(int)grid, H, smem, stream>>>(packed, fl, unif, n, N, u1, out, logpsi);
    return cudaGetLastError();
}

template <int H>
cudaError_t launch_sample_h(int B, const float *packed, const F32Layout &fl, const float *unif,
                            int64_t n, int N, int u1, uint8_t *out, float *logpsi,
                            cudaStream_t stream) {
    switch (B) {
        case 4: return launch_sample_hb<H, 4>(packed, fl, unif, n, N, u1, out, logpsi, stream);
        case 8: return launch_sample_hb<H, 8>(packed, fl, unif, n, N, u1, out, logpsi, stream);
        case 16: return launch_sample_hb<H, 16>(packed, fl, unif, n, N, u1, out, logpsi, stream);
        case 32: return launch_sample_hb<H, 32>(packed, fl, unif, n, N, u1, out, logpsi, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_sample(int per_cta, const float *packed, const F32Layout &fl, const float *unif,
                          int64_t n, int N, int u1, uint8_t *out, float *logpsi,
                          cudaStream_t stream) {
    switch (fl.H) {
        case 32: return launch_sample_h<32>(per_cta, packed, fl, unif, n, N, u1, out, logpsi, stream);
        case 64: return launch_sample_h<64>(per_cta, packed, fl, unif, n, N, u1, out, logpsi, stream);
        case 128: return launch_sample_h<128>(per_cta, packed, fl, unif, n, N, u1, out, logpsi, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace psr
