// Reverse-mode gradient d log psi / d theta of the 2D patched minGRU
// (Sec. II.F two-dimensional recurrences, Sec. II.G residual; the gradient
// the VMC energy estimator needs, Sec. III.B), FP32.
//
// One CTA per sample (grid-stride); thread j owns hidden unit j.  Patch rows
// are visited from the last to the first.  A row is first recomputed from
// its stored checkpoint (the previous row's states of every layer, written
// by the forward), recording its layer inputs u, gates z, candidates h~,
// states h and pre-activations y on a per-CTA tape.  The adjoint then runs
// from the readout down through the layers:
//   readout   g_o = 1/2 ([o == v] - P(o)) over the allowed values
//   output    gy = gx GELU'(y);  dC += gy h^T,  dD += gy u^T
//             dL/dh = C^T gy + [l+1 >= 2] gy^(l+1) + (from the row below)
//   scan      lambda_k = dL/dh_k + z_{k+1} lambda_{k+1} along the row
//             (the row's last patch has no horizontal successor)
//             dz = lambda (h_H - h~) z (1 - z),  dh~ = lambda (1 - z)
//   inputs    dW_z += dz u^T,  dW_h += dh~ [u, h_V]^T,
//             gx^(l-1) = W_z^T dz + W_hx^T dh~ + D^T gy,
//             row above: g_V = W_hv^T dh~, at the same column
// Parameter updates are fire-and-forget reductions with one writer per
// address, so the sums are deterministic.
#include <cuda_runtime.h>

#include "psr_device.cuh"
#include "psr_internal.cuh"

namespace psr {

T2Layout t2_layout(int nL, int H) {
    T2Layout t{};
    t.nL = nL;
    t.H = H;
    int64_t off = 0;
    for (int l = 0; l < nL; ++l) {
        const int64_t din = l == 0 ? 32 : H;
        t.Wz[l] = off; off += H * din;
        t.bz[l] = off; off += H;
        t.Wh[l] = off; off += H * (din + H);
        t.bh[l] = off; off += H;
        t.C[l] = off; off += (int64_t)H * H;
        t.D[l] = off; off += H * din;
    }
    t.Wo = off; off += 16 * (int64_t)H;
    t.bo = off; off += 16;
    t.total = off;
    return t;
}

size_t bwd2d_smem_bytes(int nL, int H, int Lx);

namespace {

constexpr int kR = 32;       // patches per row (max)
constexpr int kLD = kR + 4;  // padded smem rows (same as the forward's checkpoints)
enum { TQ_U = 0, TQ_Z = 1, TQ_C = 2, TQ_H = 3, TQ_Y = 4, TQ_N = 5 };

__device__ __forceinline__ int sp2(int Lx, int i, int j) { return j * Lx + ((j & 1) ? Lx - 1 - i : i); }

// R: patches per row (row2d_width(Lx) >= Lx / 2), held in registers; shared rows
// and row checkpoints are R + 4 floats wide, the tape keeps kR-wide rows.
template <int H, int R>
__global__ void __launch_bounds__(H) bwd2d_kernel(const uint8_t *__restrict__ spins, int64_t n,
                                                  int Lx, int Ly, int u1,
                                                  const float *__restrict__ theta, T2Layout tl,
                                                  const float *__restrict__ pk, F2Layout f,
                                                  const float *__restrict__ carries,
                                                  const float *__restrict__ dout,
                                                  float *__restrict__ grad_rows,
                                                  float *__restrict__ scratch) {
    // Above hidden 128 the previous row's states are read in place from the
    // forward's row checkpoint in HBM (through L1) instead of a shared copy.
    constexpr bool kHvG = H > 128;
    constexpr int LD = R + 4;
    extern __shared__ __align__(16) float smem[];
    const int nL = f.nL;
    const int Px = Lx >> 1, Py = Ly >> 1, N = Lx * Ly;
    float *xs = smem;                 // [H][LD] layer input / output
    float *hs = xs + H * LD;         // [H][LD] states of the current layer
    float *hv_s = hs + H * LD;       // [nL][H][LD] previous row's states (this row's order)
    float *g1 = kHvG ? hv_s : hv_s + nL * H * LD;  // [H][LD] adjoint tile (gy, then dz)
    float *g2 = g1 + H * LD;         // [H][LD] adjoint tile (dh~)
    float *lg = g2 + H * LD;         // [16][LD] logits, then their adjoints
    __shared__ int s_v[kR], s_vprev[kR];
    __shared__ int s_up;

    const int j = threadIdx.x;
    const int64_t P = tl.total;
    const size_t ckpt = (size_t)nL * H * LD;
    float *tape = scratch + (size_t)blockIdx.x * ((size_t)nL * TQ_N * kR * H + 2 * ckpt);
    float *gvb[2] = {tape + (size_t)nL * TQ_N * kR * H, tape + (size_t)nL * TQ_N * kR * H + ckpt};
    auto T = [&](int l, int q, int k) -> float * { return tape + (((size_t)l * TQ_N + q) * kR + k) * H; };

    for (int64_t smp = blockIdx.x; smp < n; smp += gridDim.x) {
        const uint8_t *s = spins + (size_t)smp * N;
        const float scale = dout ? dout[smp] : 1.0f;
        float *G = dout ? grad_rows + (size_t)blockIdx.x * P : grad_rows + (size_t)smp * P;
        float gbz[kMaxLayers], gbh[kMaxLayers];
#pragma unroll
        for (int l = 0; l < kMaxLayers; ++l) { gbz[l] = 0.0f; gbh[l] = 0.0f; }
        int cur = 0;  // gvb[cur]: adjoint into this row's states from the row below
        for (size_t i = j; i < ckpt; i += H) {
            gvb[0][i] = 0.0f;
            gvb[1][i] = 0.0f;
        }

        for (int pj = Py - 1; pj >= 0; --pj) {
            // ------------------------------------------------ recompute the row
            const float *hv = carries + ((size_t)smp * Py + pj) * ckpt;
            if (!kHvG) {
                for (size_t i = j; i < ckpt; i += H) hv_s[i] = hv[i];
                hv = hv_s;
            }
            if (j < Px) {
                const int pi = (pj & 1) ? Px - 1 - j : j;
                int v = 0;
                for (int b = 0; b < 4; ++b) v |= (int)(s[sp2(Lx, 2 * pi + (b & 1), 2 * pj + (b >> 1))] & 1u) << b;
                s_v[j] = v;
                if (pj > 0) {
                    int w = 0;
                    for (int b = 0; b < 4; ++b) w |= (int)(s[sp2(Lx, 2 * j + (b & 1), 2 * pj - 2 + (b >> 1))] & 1u) << b;
                    s_vprev[j] = w;
                }
            }
            if (j == 0) {
                int up = 0;
                for (int t = 0; t < 2 * pj * Lx; ++t) up += s[t] & 1;
                s_up = up;
            }
            __syncthreads();
            float hl[R];
            {   // layer 0
                const float *WzT = pk + f.WzT[0], *WhxT = pk + f.WhxT[0], *DT = pk + f.DT[0];
                const float bz = pk[f.bz[0] + j], bh = pk[f.bh[0] + j];
                float z[R], c[R], y[R];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const int kk = k < Px ? k : Px - 1;
                    const int pi = (pj & 1) ? Px - 1 - kk : kk;
                    const int vh = kk > 0 ? s_v[kk - 1] : -1;
                    const int vv = pj > 0 ? s_vprev[pi] : -1;
                    z[k] = bz + (vh >= 0 ? WzT[vh * H + j] : 0.0f) + (vv >= 0 ? WzT[(16 + vv) * H + j] : 0.0f);
                    c[k] = bh + (vh >= 0 ? WhxT[vh * H + j] : 0.0f) + (vv >= 0 ? WhxT[(16 + vv) * H + j] : 0.0f);
                    y[k] = (vh >= 0 ? DT[vh * H + j] : 0.0f) + (vv >= 0 ? DT[(16 + vv) * H + j] : 0.0f);
                }
                if (pj > 0) {
                    const float *Wv = pk + f.WhvT[0];
#pragma unroll 2
                    for (int m = 0; m < H; ++m) {
                        const float w = Wv[m * H + j];
                        const float4 *sv = reinterpret_cast<const float4 *>(hv + m * LD);
#pragma unroll
                        for (int k4 = 0; k4 < R / 4; ++k4) {
                            const float4 v = sv[k4];
                            c[4 * k4] += w * v.x; c[4 * k4 + 1] += w * v.y;
                            c[4 * k4 + 2] += w * v.z; c[4 * k4 + 3] += w * v.w;
                        }
                    }
                }
                float h = 0.0f;
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const float a = sigmoid_f(z[k]);
                    h = a * h + (1.0f - a) * c[k];
                    hl[k] = h;
                    T(0, TQ_Z, k)[j] = a;
                    T(0, TQ_C, k)[j] = c[k];
                    T(0, TQ_H, k)[j] = h;
                }
                float4 *dh = reinterpret_cast<float4 *>(hs + j * LD);
#pragma unroll
                for (int k4 = 0; k4 < R / 4; ++k4)
                    dh[k4] = make_float4(hl[4 * k4], hl[4 * k4 + 1], hl[4 * k4 + 2], hl[4 * k4 + 3]);
                __syncthreads();
                const float *Ct = pk + f.CT[0];
#pragma unroll 2
                for (int m = 0; m < H; ++m) {
                    const float w = Ct[m * H + j];
                    const float4 *sh = reinterpret_cast<const float4 *>(hs + m * LD);
#pragma unroll
                    for (int k4 = 0; k4 < R / 4; ++k4) {
                        const float4 v = sh[k4];
                        y[4 * k4] += w * v.x; y[4 * k4 + 1] += w * v.y;
                        y[4 * k4 + 2] += w * v.z; y[4 * k4 + 3] += w * v.w;
                    }
                }
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    T(0, TQ_Y, k)[j] = y[k];
                    xs[j * LD + k] = gelu_f(y[k]);
                }
                __syncthreads();
            }
            for (int l = 1; l < nL; ++l) {
                const float *WzT = pk + f.WzT[l], *WhxT = pk + f.WhxT[l], *Wv = pk + f.WhvT[l];
                const float *hvl = hv + (size_t)l * H * LD;
                float z[R], c[R];
                const float bz = pk[f.bz[l] + j], bh = pk[f.bh[l] + j];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    z[k] = bz;
                    c[k] = bh;
                    T(l, TQ_U, k)[j] = xs[j * LD + k];
                }
#pragma unroll 2
                for (int m = 0; m < H; ++m) {
                    const float wz = WzT[m * H + j], wh = WhxT[m * H + j], wv = Wv[m * H + j];
                    const float4 *sx = reinterpret_cast<const float4 *>(xs + m * LD);
                    const float4 *sv = reinterpret_cast<const float4 *>(hvl + m * LD);
#pragma unroll
                    for (int k4 = 0; k4 < R / 4; ++k4) {
                        const float4 x = sx[k4], v = sv[k4];
                        z[4 * k4] += wz * x.x; z[4 * k4 + 1] += wz * x.y;
                        z[4 * k4 + 2] += wz * x.z; z[4 * k4 + 3] += wz * x.w;
                        c[4 * k4] += wh * x.x + wv * v.x; c[4 * k4 + 1] += wh * x.y + wv * v.y;
                        c[4 * k4 + 2] += wh * x.z + wv * v.z; c[4 * k4 + 3] += wh * x.w + wv * v.w;
                    }
                }
                float hn[R];
                float h = 0.0f;
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const float a = sigmoid_f(z[k]);
                    h = a * h + (1.0f - a) * c[k];
                    hn[k] = h;
                    T(l, TQ_Z, k)[j] = a;
                    T(l, TQ_C, k)[j] = c[k];
                    T(l, TQ_H, k)[j] = h;
                }
                __syncthreads();
                float4 *dh = reinterpret_cast<float4 *>(hs + j * LD);
#pragma unroll
                for (int k4 = 0; k4 < R / 4; ++k4)
                    dh[k4] = make_float4(hn[4 * k4], hn[4 * k4 + 1], hn[4 * k4 + 2], hn[4 * k4 + 3]);
                __syncthreads();
                float y[R];
#pragma unroll
                for (int k = 0; k < R; ++k) y[k] = (l >= 2) ? hl[k] : 0.0f;
                const float *Ct = pk + f.CT[l], *DT = pk + f.DT[l];
#pragma unroll 2
                for (int m = 0; m < H; ++m) {
                    const float wc = Ct[m * H + j], wd = DT[m * H + j];
                    const float4 *sh = reinterpret_cast<const float4 *>(hs + m * LD);
                    const float4 *sx = reinterpret_cast<const float4 *>(xs + m * LD);
#pragma unroll
                    for (int k4 = 0; k4 < R / 4; ++k4) {
                        const float4 a = sh[k4], b = sx[k4];
                        y[4 * k4] += wc * a.x + wd * b.x; y[4 * k4 + 1] += wc * a.y + wd * b.y;
                        y[4 * k4 + 2] += wc * a.z + wd * b.z; y[4 * k4 + 3] += wc * a.w + wd * b.w;
                    }
                }
                __syncthreads();
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    T(l, TQ_Y, k)[j] = y[k];
                    xs[j * LD + k] = gelu_f(y[k]);
                    hl[k] = hn[k];
                }
                __syncthreads();
            }

            // ------------------------------------------------ readout adjoint
            {
                const int o = j & 15;
                for (int k = j >> 4; k < Px; k += H / 16) {
                    float v = theta[tl.bo + o];
                    for (int m = 0; m < H; ++m) v += theta[tl.Wo + o * H + m] * xs[m * LD + k];
                    lg[o * LD + k] = v;
                }
            }
            __syncthreads();
            if (j < Px) {
                const int k = j;
                int up = s_up, down = 2 * pj * Lx - s_up;
                for (int kk = 0; kk < k; ++kk) {
                    const int pc = __popc(s_v[kk]);
                    up += pc;
                    down += 4 - pc;
                }
                auto allowed = [&](int v) {
                    const int pc = __popc(v);
                    return !u1 || (up + pc <= N / 2 && down + 4 - pc <= N / 2);
                };
                float mx = -INFINITY;
                for (int v = 0; v < 16; ++v)
                    if (allowed(v)) mx = fmaxf(mx, lg[v * LD + k]);
                float ssum = 0.0f;
                for (int v = 0; v < 16; ++v)
                    if (allowed(v)) ssum += expf(lg[v * LD + k] - mx);
                const int vk = s_v[k];
                for (int v = 0; v < 16; ++v) {
                    const float p = allowed(v) ? expf(lg[v * LD + k] - mx) / ssum : 0.0f;
                    lg[v * LD + k] = 0.5f * scale * ((v == vk ? 1.0f : 0.0f) - p);
                }
            }
            __syncthreads();
            // zero the padding sites' adjoints
            for (int i = j; i < 16 * LD; i += H)
                if ((i % LD) >= Px) lg[i] = 0.0f;
            __syncthreads();
            float gx[R];
            {
#pragma unroll
                for (int k = 0; k < R; ++k) gx[k] = 0.0f;
                for (int o = 0; o < 16; ++o) {
                    const float w = theta[tl.Wo + o * H + j];
                    float gw = 0.0f;
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        const float g = lg[o * LD + k];
                        gx[k] += w * g;
                        gw += g * xs[j * LD + k];
                    }
                    atomicAdd(&G[tl.Wo + o * H + j], gw);
                }
                if (j < 16) {
                    float gb = 0.0f;
                    for (int k = 0; k < Px; ++k) gb += lg[j * LD + k];
                    atomicAdd(&G[tl.bo + j], gb);
                }
            }

            // ------------------------------------------------ layers, top down
            float gy_up[R];
#pragma unroll
            for (int k = 0; k < R; ++k) gy_up[k] = 0.0f;
            float *gv_in = gvb[cur], *gv_out = gvb[cur ^ 1];
            for (int l = nL - 1; l >= 0; --l) {
                const int din = l == 0 ? 32 : H;
                float gy[R];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    gy[k] = k < Px ? gx[k] * gelu_grad_f(T(l, TQ_Y, k)[j]) : 0.0f;
                    g1[j * LD + k] = gy[k];
                }
                __syncthreads();
                // unit j as the input unit m: C^T gy, D^T gy, dC, dD
                float ghd[R], gud[R], hk[R], uk[R];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    hk[k] = T(l, TQ_H, k)[j];
                    uk[k] = (l >= 1) ? T(l, TQ_U, k)[j] : 0.0f;
                    ghd[k] = (l + 1 < nL && l + 1 >= 2 ? gy_up[k] : 0.0f) +
                             gv_in[((size_t)l * H + j) * LD + k];
                    gud[k] = 0.0f;
                }
                {
                    const float *Cw = theta + tl.C[l];
                    const float *Dw = theta + tl.D[l];
                    for (int i = 0; i < H; ++i) {
                        const float cij = Cw[(int64_t)i * H + j];
                        const float dij = (l >= 1) ? Dw[(int64_t)i * H + j] : 0.0f;
                        float ac = 0.0f, ad = 0.0f;
#pragma unroll
                        for (int k = 0; k < R; ++k) {
                            const float g = g1[i * LD + k];
                            ghd[k] += cij * g;
                            gud[k] += dij * g;
                            ac += g * hk[k];
                            ad += g * uk[k];
                        }
                        atomicAdd(&G[tl.C[l] + (int64_t)i * H + j], ac);
                        if (l >= 1) atomicAdd(&G[tl.D[l] + (int64_t)i * H + j], ad);
                    }
                }
                if (l == 0) {  // D^(0) acts on (onehot(v_H), onehot(v_V))
                    for (int k = 0; k < Px; ++k) {
                        const int pi = (pj & 1) ? Px - 1 - k : k;
                        if (k > 0) atomicAdd(&G[tl.D[0] + (int64_t)j * 32 + s_v[k - 1]], gy[k]);
                        if (pj > 0) atomicAdd(&G[tl.D[0] + (int64_t)j * 32 + 16 + s_vprev[pi]], gy[k]);
                    }
                }
                // reverse scan along the row (unit j)
                {
                    float lam = 0.0f, an = 0.0f, sz = 0.0f, sc = 0.0f;
#pragma unroll
                    for (int k = R - 1; k >= 0; --k) {
                        float dz = 0.0f, dc = 0.0f;
                        if (k < Px) {
                            lam = ghd[k] + an * lam;
                            const float a = T(l, TQ_Z, k)[j];
                            const float cd = T(l, TQ_C, k)[j];
                            const float hp = k > 0 ? hk[k - 1] : 0.0f;
                            dz = lam * (hp - cd) * a * (1.0f - a);
                            dc = lam * (1.0f - a);
                            an = a;
                        }
                        sz += dz;
                        sc += dc;
                        ghd[k] = dz;  // reuse as the dz row
                        hk[k] = dc;   // reuse as the dh~ row
                    }
#pragma unroll
                    for (int ll = 0; ll < kMaxLayers; ++ll)
                        if (ll == l) { gbz[ll] += sz; gbh[ll] += sc; }
                }
                __syncthreads();  // every read of g1 (gy) is done
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    g1[j * LD + k] = ghd[k];  // dz
                    g2[j * LD + k] = hk[k];   // dh~
                }
                __syncthreads();
                // unit j as the input unit m: weight gradients, g_V, gx of the layer below
                {
                    const float *Wzw = theta + tl.Wz[l];
                    const float *Whw = theta + tl.Wh[l];
                    const float *hvl = hv + (size_t)l * H * LD;
                    float gn[R], gvo[R];
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        gn[k] = gud[k];
                        gvo[k] = 0.0f;
                    }
                    for (int i = 0; i < H; ++i) {
                        const float wz = (l >= 1) ? Wzw[(int64_t)i * din + j] : 0.0f;
                        const float wh = (l >= 1) ? Whw[(int64_t)i * (din + H) + j] : 0.0f;
                        const float wv = Whw[(int64_t)i * (din + H) + din + j];
                        float az = 0.0f, ah = 0.0f, avv = 0.0f;
#pragma unroll
                        for (int k = 0; k < R; ++k) {
                            const float dz = g1[i * LD + k], dc = g2[i * LD + k];
                            gn[k] += wz * dz + wh * dc;
                            gvo[k] += wv * dc;
                            az += dz * uk[k];
                            ah += dc * uk[k];
                            avv += dc * hvl[j * LD + k];
                        }
                        if (l >= 1) {
                            atomicAdd(&G[tl.Wz[l] + (int64_t)i * din + j], az);
                            atomicAdd(&G[tl.Wh[l] + (int64_t)i * (din + H) + j], ah);
                        }
                        if (pj > 0) atomicAdd(&G[tl.Wh[l] + (int64_t)i * (din + H) + din + j], avv);
                    }
                    if (l == 0) {  // W_z^(0), W_hx^(0) act on the one-hot inputs
                        for (int k = 0; k < Px; ++k) {
                            const int pi = (pj & 1) ? Px - 1 - k : k;
                            const float dz = g1[j * LD + k], dc = g2[j * LD + k];
                            if (k > 0) {
                                atomicAdd(&G[tl.Wz[0] + (int64_t)j * 32 + s_v[k - 1]], dz);
                                atomicAdd(&G[tl.Wh[0] + (int64_t)j * (32 + H) + s_v[k - 1]], dc);
                            }
                            if (pj > 0) {
                                atomicAdd(&G[tl.Wz[0] + (int64_t)j * 32 + 16 + s_vprev[pi]], dz);
                                atomicAdd(&G[tl.Wh[0] + (int64_t)j * (32 + H) + 16 + s_vprev[pi]], dc);
                            }
                        }
                    }
                    // adjoint into the row above (path order of that row: reversed)
#pragma unroll
                    for (int k = 0; k < R; ++k)
                        if (k < Px) gv_out[((size_t)l * H + j) * LD + (Px - 1 - k)] = gvo[k];
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        gx[k] = gn[k];
                        gy_up[k] = gy[k];
                    }
                }
                __syncthreads();
            }
            // the adjoint just written is the next row's input; clear the old one
            for (size_t i = j; i < ckpt; i += H) gv_in[i] = 0.0f;
            cur ^= 1;
            __syncthreads();
        }
        for (int l = 0; l < nL; ++l) {
            float bzv = 0.0f, bhv = 0.0f;
#pragma unroll
            for (int ll = 0; ll < kMaxLayers; ++ll)
                if (ll == l) { bzv = gbz[ll]; bhv = gbh[ll]; }
            atomicAdd(&G[tl.bz[l] + j], bzv);
            atomicAdd(&G[tl.bh[l] + j], bhv);
        }
        __syncthreads();
    }
}

template <int H, int R>
cudaError_t launch_bwd2d_hr(const uint8_t *spins, int64_t n, int Lx, int Ly, int u1, const float *theta,
                           const T2Layout &tl, const float *packed, const F2Layout &f,
                           const float *carries, const float *dout, float *grad_rows, int grid,
                           float *scratch, cudaStream_t st) {
    const size_t smem = bwd2d_smem_bytes(f.nL, H, Lx);
    cudaError_t e = cudaFuncSetAttribute(bwd2d_kernel<H, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    bwd2d_kernel<H, R><<<grid, H, smem, st>>>(spins, n, Lx, Ly, u1, theta, tl, packed, f, carries, dout,
                                            grad_rows, scratch);
    return cudaGetLastError();
}

template <int H>
cudaError_t launch_bwd2d_h(const uint8_t *spins, int64_t n, int Lx, int Ly, int u1, const float *theta,
                           const T2Layout &tl, const float *packed, const F2Layout &f,
                           const float *carries, const float *dout, float *grad_rows, int grid,
                           float *scratch, cudaStream_t st) {
    switch (row2d_width(Lx)) {
        case 8: return launch_bwd2d_hr<H, 8>(spins, n, Lx, Ly, u1, theta, tl, packed, f, carries, dout, grad_rows, grid, scratch, st);
        case 12: return launch_bwd2d_hr<H, 12>(spins, n, Lx, Ly, u1, theta, tl, packed, f, carries, dout, grad_rows, grid, scratch, st);
        case 16: return launch_bwd2d_hr<H, 16>(spins, n, Lx, Ly, u1, theta, tl, packed, f, carries, dout, grad_rows, grid, scratch, st);
        case 24: return launch_bwd2d_hr<H, 24>(spins, n, Lx, Ly, u1, theta, tl, packed, f, carries, dout, grad_rows, grid, scratch, st);
        case 28: return launch_bwd2d_hr<H, 28>(spins, n, Lx, Ly, u1, theta, tl, packed, f, carries, dout, grad_rows, grid, scratch, st);
        default: return launch_bwd2d_hr<H, 32>(spins, n, Lx, Ly, u1, theta, tl, packed, f, carries, dout, grad_rows, grid, scratch, st);
    }
}

}  // namespace

size_t bwd2d_scratch_floats_per_cta(int nL, int H) {
    return (size_t)nL * TQ_N * kR * H + 2 * (size_t)nL * H * kLD;
}

size_t bwd2d_smem_bytes(int nL, int H, int Lx) {
    const size_t ld = (size_t)row2d_width(Lx) + 4;
    return ((size_t)(4 + (H > 128 ? 0 : nL)) * H * ld + 16 * ld) * sizeof(float);
}

cudaError_t launch_bwd2d(const uint8_t *spins, int64_t n, int Lx, int Ly, int u1, const float *theta,
                         const T2Layout &tl, const float *packed, const F2Layout &f, const float *carries,
                         const float *dout, float *grad_rows, int grid, float *scratch,
                         cudaStream_t stream) {
    switch (f.H) {
        case 32: return launch_bwd2d_h<32>(spins, n, Lx, Ly, u1, theta, tl, packed, f, carries, dout, grad_rows, grid, scratch, stream);
        case 64: return launch_bwd2d_h<64>(spins, n, Lx, Ly, u1, theta, tl, packed, f, carries, dout, grad_rows, grid, scratch, stream);
        case 128: return launch_bwd2d_h<128>(spins, n, Lx, Ly, u1, theta, tl, packed, f, carries, dout, grad_rows, grid, scratch, stream);
        case 256: return launch_bwd2d_h<256>(spins, n, Lx, Ly, u1, theta, tl, packed, f, carries, dout, grad_rows, grid, scratch, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace psr
