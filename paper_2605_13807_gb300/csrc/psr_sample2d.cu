// Exact autoregressive sampling of the 2D patched minGRU (Sec. II.F
// two-dimensional recurrences; Sec. III.B exact sampling), FP32.
//
// One CTA draws B samples; thread j owns hidden unit j.  Patches are visited
// along the zigzag path of the patch lattice.  For each sample and layer the
// CTA keeps one row of states by column in shared memory, updated in place:
// when patch (i, j) is evaluated, column i still holds the previous row's
// state (its h_V) and the column visited just before holds the current
// row's previous patch (its h_H, zero at the row start); after the patch
// the column holds the new state.  The 16-way conditional of the patch
// (softmax of the readout, restricted by the zero-magnetisation mask) is
// sampled with the caller's uniform: the smallest value v whose cumulative
// probability exceeds u (the last allowed value if rounding leaves u above
// the total).  Per-sample arithmetic does not depend on B, so every B draws
// the same samples.
#include <cuda_runtime.h>

#include "psr_device.cuh"
#include "psr_internal.cuh"

namespace psr {

namespace {

__device__ __forceinline__ int pos2(int Lx, int i, int j) { return j * Lx + ((j & 1) ? Lx - 1 - i : i); }

template <int H, int B>
__global__ void __launch_bounds__(H) sample2d_kernel(const float *__restrict__ pk, F2Layout f,
                                                     const float *__restrict__ unif, int64_t n,
                                                     int Lx, int Ly, int u1,
                                                     uint8_t *__restrict__ out,
                                                     float *__restrict__ logpsi) {
    static_assert(B * 16 <= H, "one thread per (sample, logit)");
    extern __shared__ __align__(16) float smem[];
    const int nL = f.nL;
    const int Px = Lx >> 1, Py = Ly >> 1, N = Lx * Ly, Np = Px * Py;
    float *buf = smem;                          // [B][nL][H][Px] states by column
    float *xs = buf + (size_t)B * nL * H * Px;  // [B][H] layer input / output of the patch
    float *hs = xs + B * H;                     // [B][H] states of the patch's current layer
    float *lg = hs + B * H;                     // [B][16] logits
    __shared__ int s_vprev[B][32];              // previous row's values by column (updated in place)
    __shared__ int s_vlast[B];                  // value of the previous patch on the path
    __shared__ int s_up[B], s_down[B];
    __shared__ float s_acc[B];

    const int j = threadIdx.x;
    const int64_t first = (int64_t)blockIdx.x * B;
    for (size_t i = j; i < (size_t)B * nL * H * Px; i += H) buf[i] = 0.0f;
    if (j < B) {
        s_vlast[j] = -1;
        s_up[j] = 0;
        s_down[j] = 0;
        s_acc[j] = 0.0f;
    }
    for (int i = j; i < B * 32; i += H) s_vprev[i / 32][i % 32] = 0;
    __syncthreads();

    for (int t = 0; t < Np; ++t) {
        const int pj = t / Px, k = t - pj * Px;
        const int pi = (pj & 1) ? Px - 1 - k : k;
        const int pprev = (pj & 1) ? pi + 1 : pi - 1;  // column of the previous patch in the row
        float hres[B];
#pragma unroll
        for (int b = 0; b < B; ++b) hres[b] = 0.0f;
        for (int l = 0; l < nL; ++l) {
            float z[B], c[B], y[B];
            const float bz = pk[f.bz[l] + j], bh = pk[f.bh[l] + j];
            if (l == 0) {
                const float *WzT = pk + f.WzT[0], *WhxT = pk + f.WhxT[0], *DT = pk + f.DT[0];
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const int vh = k > 0 ? (s_vlast[b] & 15) : -1;
                    const int vv = pj > 0 ? (s_vprev[b][pi] & 15) : -1;
                    z[b] = bz + (vh >= 0 ? WzT[vh * H + j] : 0.0f) + (vv >= 0 ? WzT[(16 + vv) * H + j] : 0.0f);
                    c[b] = bh + (vh >= 0 ? WhxT[vh * H + j] : 0.0f) + (vv >= 0 ? WhxT[(16 + vv) * H + j] : 0.0f);
                    y[b] = (vh >= 0 ? DT[vh * H + j] : 0.0f) + (vv >= 0 ? DT[(16 + vv) * H + j] : 0.0f);
                }
            } else {
                const float *WzT = pk + f.WzT[l], *WhxT = pk + f.WhxT[l];
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    z[b] = bz;
                    c[b] = bh;
                }
#pragma unroll 4
                for (int m = 0; m < H; ++m) {
                    const float wz = WzT[m * H + j], wh = WhxT[m * H + j];
#pragma unroll
                    for (int b = 0; b < B; ++b) {
                        const float xv = xs[b * H + m];
                        z[b] += wz * xv;
                        c[b] += wh * xv;
                    }
                }
            }
            if (pj > 0) {
                const float *Wv = pk + f.WhvT[l];
#pragma unroll 4
                for (int m = 0; m < H; ++m) {
                    const float w = Wv[m * H + j];
#pragma unroll
                    for (int b = 0; b < B; ++b) c[b] += w * buf[(((size_t)b * nL + l) * H + m) * Px + pi];
                }
            }
            float h[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const float a = sigmoid_f(z[b]);
                const float hH = k > 0 ? buf[(((size_t)b * nL + l) * H + j) * Px + pprev] : 0.0f;
                // explicit rounding order: identical for every samples-per-CTA instance
                h[b] = fmaf(a, hH, __fmul_rn(1.0f - a, c[b]));
            }
            __syncthreads();  // every read of column pi (h_V) is done
#pragma unroll
            for (int b = 0; b < B; ++b) {
                buf[(((size_t)b * nL + l) * H + j) * Px + pi] = h[b];
                hs[b * H + j] = h[b];
            }
            __syncthreads();
            if (l >= 1) {
#pragma unroll
                for (int b = 0; b < B; ++b) y[b] = (l >= 2) ? hres[b] : 0.0f;
                const float *DT = pk + f.DT[l];
#pragma unroll 4
                for (int m = 0; m < H; ++m) {
                    const float wd = DT[m * H + j];
#pragma unroll
                    for (int b = 0; b < B; ++b) y[b] += wd * xs[b * H + m];
                }
            }
            {
                const float *Ct = pk + f.CT[l];
#pragma unroll 4
                for (int m = 0; m < H; ++m) {
                    const float w = Ct[m * H + j];
#pragma unroll
                    for (int b = 0; b < B; ++b) y[b] += w * hs[b * H + m];
                }
            }
            __syncthreads();  // every read of xs and hs is done
#pragma unroll
            for (int b = 0; b < B; ++b) {
                xs[b * H + j] = gelu_f(y[b]);
                hres[b] = h[b];
            }
            __syncthreads();
        }
        // readout: thread (b, o) computes logit o of sample b
        if (j < B * 16) {
            const int b = j >> 4, o = j & 15;
            const float *Wo = pk + f.Wo;
            float v = Wo[16 * H + o];
            for (int m = 0; m < H; ++m) v += Wo[o * H + m] * xs[b * H + m];
            lg[b * 16 + o] = v;
        }
        __syncthreads();
        if (j < B) {
            const int b = j;
            const int64_t row = first + b;
            if (row >= n) {
                // padding sample of the last CTA: keep its inputs valid codes
                s_vlast[b] = 0;
                s_vprev[b][pi] = 0;
            } else {
                const int up = s_up[b], down = s_down[b];
                auto allowed = [&](int v) {
                    const int pc = __popc(v);
                    return !u1 || (up + pc <= N / 2 && down + 4 - pc <= N / 2);
                };
                float mx = -INFINITY;
                for (int v = 0; v < 16; ++v)
                    if (allowed(v)) mx = fmaxf(mx, lg[b * 16 + v]);
                float ssum = 0.0f;
                for (int v = 0; v < 16; ++v)
                    if (allowed(v)) ssum += expf(lg[b * 16 + v] - mx);
                const float lse = mx + logf(ssum);
                const float u = unif[row * Np + t];
                float cum = 0.0f;
                int pick = -1, last = -1;
                for (int v = 0; v < 16; ++v) {
                    if (!allowed(v)) continue;
                    last = v;
                    cum += expf(lg[b * 16 + v] - lse);
                    if (pick < 0 && u < cum) pick = v;
                }
                if (pick < 0) pick = last;
                if (pick < 0) pick = 0;  // not reached: the mask always leaves a value
                s_acc[b] += lg[b * 16 + pick] - lse;
                s_up[b] = up + __popc(pick);
                s_down[b] = down + 4 - __popc(pick);
                s_vlast[b] = pick;
                s_vprev[b][pi] = pick;
                uint8_t *o = out + row * N;
#pragma unroll
                for (int bit = 0; bit < 4; ++bit)
                    o[pos2(Lx, 2 * pi + (bit & 1), 2 * pj + (bit >> 1))] = (uint8_t)((pick >> bit) & 1);
            }
        }
        __syncthreads();
    }
    if (j < B && first + j < n && logpsi) logpsi[first + j] = 0.5f * s_acc[j];
}

template <int H, int B>
cudaError_t launch_s2_hb(const float *packed, const F2Layout &f, const float *unif, int64_t n, int Lx,
                         int Ly, int u1, uint8_t *out, float *logpsi, cudaStream_t st) {
    const int Px = Lx / 2;
    const size_t smem = ((size_t)B * f.nL * H * Px + 2 * (size_t)B * H + 16 * (size_t)B) * sizeof(float);
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(sample2d_kernel<H, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (n + B - 1) / B;
    if (grid > 0x7fffffff) return cudaErrorInvalidValue;
    sample2d_kernel<H, B><<<(int)grid, H, smem, st>>>(packed, f, unif, n, Lx, Ly, u1, out, logpsi);
    return cudaGetLastError();
}

template <int H>
cudaError_t launch_s2_h(int B, const float *packed, const F2Layout &f, const float *unif, int64_t n,
                        int Lx, int Ly, int u1, uint8_t *out, float *logpsi, cudaStream_t st) {
    switch (B) {
        case 1: return launch_s2_hb<H, 1>(packed, f, unif, n, Lx, Ly, u1, out, logpsi, st);
        case 2: return launch_s2_hb<H, 2>(packed, f, unif, n, Lx, Ly, u1, out, logpsi, st);
        default: break;
    }
    if constexpr (H >= 64) {
        if (B == 4) return launch_s2_hb<H, 4>(packed, f, unif, n, Lx, Ly, u1, out, logpsi, st);
    }
    if constexpr (H >= 128) {
        if (B == 8) return launch_s2_hb<H, 8>(packed, f, unif, n, Lx, Ly, u1, out, logpsi, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

size_t sample2d_smem_bytes(int per_cta, int nL, int H, int Lx) {
    return ((size_t)per_cta * nL * H * (Lx / 2) + 2 * (size_t)per_cta * H + 16 * (size_t)per_cta) *
           sizeof(float);
}

cudaError_t launch_sample2d(int per_cta, const float *packed, const F2Layout &f, const float *unif,
                            int64_t n, int Lx, int Ly, int u1, uint8_t *out, float *logpsi,
                            cudaStream_t stream) {
    switch (f.H) {
        case 32: return launch_s2_h<32>(per_cta, packed, f, unif, n, Lx, Ly, u1, out, logpsi, stream);
        case 64: return launch_s2_h<64>(per_cta, packed, f, unif, n, Lx, Ly, u1, out, logpsi, stream);
        case 128: return launch_s2_h<128>(per_cta, packed, f, unif, n, Lx, Ly, u1, out, logpsi, stream);
        case 256: return launch_s2_h<256>(per_cta, packed, f, unif, n, Lx, Ly, u1, out, logpsi, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace psr
