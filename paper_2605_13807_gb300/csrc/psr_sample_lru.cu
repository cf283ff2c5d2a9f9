// Exact autoregressive sampling of the deep 1D LRU ansatz on the device
// (Sec. II.A and Sec. III.B: conditionals drawn site by site, no Markov
// chain; model of Sec. II.B Eq. lru with the GLU blocks of Sec. III.B).
//
// One CTA draws B samples; thread j owns hidden unit j of every layer for all
// B samples, with the complex states h (one (Re, Im) pair per layer and
// sample) in shared memory.  At each site the CTA runs one step of every
// layer, forms the logit difference d and sets s_t = 1 iff u_t < P(s_t = 1)
// = sigmoid(d) (or the value the zero-magnetisation mask forces).  Every sum
// is an explicit fused multiply-add chain in a fixed order, so the samples
// do not depend on B or on a sample's slot in the CTA.
#include <cuda_runtime.h>

#include "psr_device.cuh"
#include "psr_internal.cuh"

namespace psr {

namespace {

template <int H, int B>
__global__ void __launch_bounds__(H) sample_lru_kernel(const float *__restrict__ pk, LruLayout f,
                                                       const float *__restrict__ unif, int64_t n, int N,
                                                       int u1, uint8_t *__restrict__ out,
                                                       float *__restrict__ logpsi) {
    constexpr int NW = H / 32;
    extern __shared__ __align__(16) float smem[];
    float *xs = smem;            // [B][H] block input / output of the current site
    float *hr = xs + B * H;      // [B][H] Re h of the current layer
    float *hi = hr + B * H;      // [B][H] Im h
    float *ys = hi + B * H;      // [B][H] y = Re(C h) + D u
    float *red = ys + B * H;     // [NW][B] readout partial sums
    float *hc = red + NW * B;    // [nL][2][B][H] recurrent states
    __shared__ int s_prev[B], s_nup[B];
    __shared__ float s_acc[B];

    const int j = threadIdx.x;
    const int lane = j & 31, warp = j >> 5;
    const int nL = f.nL;
    const int64_t first = (int64_t)blockIdx.x * B;

    for (int i = j; i < nL * 2 * B * H; i += H) hc[i] = 0.0f;
    if (j < B) {
        s_prev[j] = 0;
        s_nup[j] = 0;
        s_acc[j] = 0.0f;
    }
    const float wdj = pk[f.wd + j];
    const float bd = pk[f.bd];
    __syncthreads();

    for (int t = 0; t < N; ++t) {
        for (int l = 0; l < nL; ++l) {
            float br[B], bi[B], y[B];
            if (l == 0) {
                const float r0 = pk[f.BreT[0] + j], r1 = pk[f.BreT[0] + H + j];
                const float i0 = pk[f.BimT[0] + j], i1 = pk[f.BimT[0] + H + j];
                const float d0 = pk[f.D[0] + j], d1 = pk[f.D[0] + H + j];
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const int code = (t == 0) ? 0 : 1 + s_prev[b];
                    br[b] = code == 0 ? 0.0f : (code == 1 ? r0 : r1);
                    bi[b] = code == 0 ? 0.0f : (code == 1 ? i0 : i1);
                    y[b] = code == 0 ? 0.0f : (code == 1 ? d0 : d1);
                }
            } else {
                const float dj = pk[f.D[l] + j];
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    br[b] = 0.0f;
                    bi[b] = 0.0f;
                    y[b] = __fmul_rn(dj, xs[b * H + j]);
                }
                const float *Br = pk + f.BreT[l], *Bi = pk + f.BimT[l];
#pragma unroll 4
                for (int k = 0; k < H; ++k) {
                    const float wr = Br[k * H + j], wi = Bi[k * H + j];
#pragma unroll
                    for (int b = 0; b < B; ++b) {
                        const float xv = xs[b * H + k];
                        br[b] = fmaf(wr, xv, br[b]);
                        bi[b] = fmaf(wi, xv, bi[b]);
                    }
                }
            }
            // h = lambda h + e^gamma (B u)
            {
                const float lr = pk[f.lre[l] + j], li = pk[f.lim[l] + j], g = pk[f.gam[l] + j];
                float *cr = hc + (size_t)(2 * l) * B * H, *ci = cr + (size_t)B * H;
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const float zr = cr[b * H + j], zi = ci[b * H + j];
                    const float nr = fmaf(lr, zr, fmaf(-li, zi, __fmul_rn(g, br[b])));
                    const float ni = fmaf(lr, zi, fmaf(li, zr, __fmul_rn(g, bi[b])));
                    cr[b * H + j] = nr;
                    ci[b * H + j] = ni;
                    hr[b * H + j] = nr;
                    hi[b * H + j] = ni;
                }
            }
            __syncthreads();
            // y = Re(C h) + D u
            {
                const float *Cr = pk + f.CreT[l], *Ci = pk + f.CimT[l];
#pragma unroll 4
                for (int m = 0; m < H; ++m) {
                    const float wr = Cr[m * H + j], wi = Ci[m * H + j];
#pragma unroll
                    for (int b = 0; b < B; ++b) y[b] = fmaf(-wi, hi[b * H + m], fmaf(wr, hr[b * H + m], y[b]));
                }
#pragma unroll
                for (int b = 0; b < B; ++b) ys[b * H + j] = y[b];
            }
            __syncthreads();
            // GLU + residual
            {
                float a[B], gg[B];
                const float ba = pk[f.ba[l] + j], bg = pk[f.bg[l] + j];
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    a[b] = ba;
                    gg[b] = bg;
                }
                const float *Wa = pk + f.WaT[l], *Wg = pk + f.WgT[l];
#pragma unroll 4
                for (int k = 0; k < H; ++k) {
                    const float wa = Wa[k * H + j], wg = Wg[k * H + j];
#pragma unroll
                    for (int b = 0; b < B; ++b) {
                        const float yv = ys[b * H + k];
                        a[b] = fmaf(wa, yv, a[b]);
                        gg[b] = fmaf(wg, yv, gg[b]);
                    }
                }
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const float r = l >= 1 ? xs[b * H + j] : 0.0f;
                    xs[b * H + j] = fmaf(a[b], sigmoid_f(gg[b]), r);
                }
            }
            __syncthreads();
        }
        // readout: d_b = bd + sum_j wd_j x_b[j], reduced in a fixed order
#pragma unroll
        for (int b = 0; b < B; ++b) {
            float v = __fmul_rn(wdj, xs[b * H + j]);
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
cudaError_t launch_hb(const float *packed, const LruLayout &f, const float *unif, int64_t n, int N, int u1,
                      uint8_t *out, float *logpsi, cudaStream_t stream) {
    const size_t smem = sample_lru_smem_bytes(B, f.nL, H);
    cudaError_t e = cudaFuncSetAttribute(sample_lru_kernel<H, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (n + B - 1) / B;
    if (grid > 0x7fffffff) return cudaErrorInvalidValue;
    sample_lru_kernel<H, B><<<(int)grid, H, smem, stream>>>(packed, f, unif, n, N, u1, out, logpsi);
    return cudaGetLastError();
}

template <int H>
cudaError_t launch_h(int B, const float *packed, const LruLayout &f, const float *unif, int64_t n, int N,
                     int u1, uint8_t *out, float *logpsi, cudaStream_t stream) {
    switch (B) {
        case 4: return launch_hb<H, 4>(packed, f, unif, n, N, u1, out, logpsi, stream);
        case 8: return launch_hb<H, 8>(packed, f, unif, n, N, u1, out, logpsi, stream);
        case 16: return launch_hb<H, 16>(packed, f, unif, n, N, u1, out, logpsi, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t sample_lru_smem_bytes(int per_cta, int nL, int H) {
    return ((size_t)4 * per_cta * H + (size_t)(H / 32) * per_cta + (size_t)nL * 2 * per_cta * H) *
           sizeof(float);
}

cudaError_t launch_sample_lru(int per_cta, const float *packed, const LruLayout &f, const float *unif,
                              int64_t n, int N, int u1, uint8_t *out, float *logpsi, cudaStream_t stream) {
    switch (f.H) {
        case 32: return launch_h<32>(per_cta, packed, f, unif, n, N, u1, out, logpsi, stream);
        case 64: return launch_h<64>(per_cta, packed, f, unif, n, N, u1, out, logpsi, stream);
        case 128: return launch_h<128>(per_cta, packed, f, unif, n, N, u1, out, logpsi, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace psr
