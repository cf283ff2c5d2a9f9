// Forward of the paper's deep 1D LRU ansatz (Sec. II.B Eq. lru, Sec. II.G 1D
// residual, Sec. III.B: each layer an LRU followed by a single-layer GLU
// feed-forward network), FP32 on CUDA cores.
//
// Per layer, with input u_t (onehot(s_{t-1}) at layer 0, zero at t = 0):
//   h_t = lambda h_{t-1} + e^gamma (B u_t),  lambda = exp(-e^nu + i e^theta)
//   y_t = Re(C h_t) + D u_t                  (D: d x 2 at layer 0, else diag)
//   x_t = (W_a y_t + b_a) sigmoid(W_g y_t + b_g) + [l >= 1] u_t
// followed by the two-logit softmax readout.  The recurrence is diagonal and
// linear with a constant complex coefficient: the parallel-scan form the
// paper uses it for.  Here, as in the minGRU kernels, the sequences of a
// launch supply the parallelism: thread j owns hidden unit j for a chunk of
// 32 sites and runs the complex scan sequentially with the carry in
// registers; B u, C h and the GLU products are batched over the chunk's
// sites from shared memory.  Jobs follow the minGRU forward's modes: 0 for
// samples (optionally writing per-site log P and the complex chunk carries
// [n][nch][nL][2][H]), 1 for connected configurations resumed at the chunk
// of their first flipped site.
#include <cuda_runtime.h>

#include "psr_device.cuh"
#include "psr_internal.cuh"

namespace psr {

LruLayout lru_layout(int nL, int H) {
    LruLayout f{};
    f.nL = nL;
    f.H = H;
    int64_t off = 0;
    auto take = [&](int64_t n) {
        const int64_t o = off;
        off += (n + 3) & ~int64_t(3);
        return o;
    };
    for (int l = 0; l < nL; ++l) {
        const int din = l == 0 ? 2 : H;
        f.lre[l] = take(H);
        f.lim[l] = take(H);
        f.gam[l] = take(H);
        f.BreT[l] = take((int64_t)din * H);
        f.BimT[l] = take((int64_t)din * H);
        f.CreT[l] = take((int64_t)H * H);
        f.CimT[l] = take((int64_t)H * H);
        f.D[l] = take(l == 0 ? 2 * (int64_t)H : H);
        f.WaT[l] = take((int64_t)H * H);
        f.ba[l] = take(H);
        f.WgT[l] = take((int64_t)H * H);
        f.bg[l] = take(H);
    }
    f.wd = take(H);
    f.bd = take(1);
    f.total = off;
    return f;
}

int64_t param_count_lru(int nL, int H) {
    int64_t P = 0;
    for (int l = 0; l < nL; ++l) {
        const int64_t din = l == 0 ? 2 : H;
        P += 3 * (int64_t)H + 2 * H * din + 2 * (int64_t)H * H + (l == 0 ? 2 * (int64_t)H : H) +
             2 * (int64_t)H * H + 2 * (int64_t)H;
    }
    return P + 2 * (int64_t)H + 2;
}

namespace {

// theta (flat LRU layout) -> packed FP32: lambda as (Re, Im), e^gamma,
// transposed matrices, layer-0 D as [2][H], readout as a logit difference.
__global__ void pack_lru_kernel(const float *__restrict__ theta, LruLayout f, float *__restrict__ pk) {
    const int H = f.H;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t src = 0;
    for (int l = 0; l < f.nL; ++l) {
        const int din = l == 0 ? 2 : H;
        const int64_t nu = src, th = nu + H, ga = th + H, Bre = ga + H, Bim = Bre + (int64_t)H * din,
                      Cre = Bim + (int64_t)H * din, Cim = Cre + (int64_t)H * H, D = Cim + (int64_t)H * H,
                      Wa = D + (l == 0 ? 2 * (int64_t)H : H), ba = Wa + (int64_t)H * H, Wg = ba + H,
                      bg = Wg + (int64_t)H * H;
        src = bg + H;
        for (int64_t j = tid; j < H; j += stride) {
            const float r = expf(-expf(theta[nu + j]));
            const float ph = expf(theta[th + j]);
            pk[f.lre[l] + j] = r * cosf(ph);
            pk[f.lim[l] + j] = r * sinf(ph);
            pk[f.gam[l] + j] = expf(theta[ga + j]);
            pk[f.ba[l] + j] = theta[ba + j];
            pk[f.bg[l] + j] = theta[bg + j];
            if (l > 0) pk[f.D[l] + j] = theta[D + j];
        }
        for (int64_t i = tid; i < (int64_t)H * din; i += stride) {
            const int j = (int)(i / din), k = (int)(i % din);
            pk[f.BreT[l] + (int64_t)k * H + j] = theta[Bre + i];
            pk[f.BimT[l] + (int64_t)k * H + j] = theta[Bim + i];
            if (l == 0) pk[f.D[l] + (int64_t)k * H + j] = theta[D + i];  // D^(0) is [H][2]
        }
        for (int64_t i = tid; i < (int64_t)H * H; i += stride) {
            const int j = (int)(i / H), k = (int)(i % H);
            pk[f.CreT[l] + (int64_t)k * H + j] = theta[Cre + i];
            pk[f.CimT[l] + (int64_t)k * H + j] = theta[Cim + i];
            pk[f.WaT[l] + (int64_t)k * H + j] = theta[Wa + i];
            pk[f.WgT[l] + (int64_t)k * H + j] = theta[Wg + i];
        }
    }
    for (int64_t j = tid; j < H; j += stride) pk[f.wd + j] = theta[src + H + j] - theta[src + j];
    if (tid == 0) pk[f.bd] = theta[src + 2 * (int64_t)H + 1] - theta[src + 2 * (int64_t)H];
}

constexpr int CH = 32;
constexpr int LD = CH + 4;

template <int H>
__global__ void __launch_bounds__(H) lru_f32_kernel(const __grid_constant__ FwdJobs jb,
                                                    const float *__restrict__ pk, LruLayout f) {
    extern __shared__ __align__(16) float smem[];
    float *xs = smem;              // [H][LD] layer input / output
    float *hr = xs + H * LD;       // [H][LD] Re h
    float *hi = hr + H * LD;       // [H][LD] Im h
    float *ys = hi + H * LD;       // [H][LD] y = Re(C h) + D u
    __shared__ long long s_job;
    __shared__ long long s_base[kMaxGroups + 1];

    const int j = threadIdx.x;
    const int nL = f.nL;
    if (j == 0) {
        long long b = 0;
        s_base[0] = 0;
        for (int i = 0; i < jb.n_groups; ++i) {
            b += jb.mode == 1 ? (long long)*jb.g[i].n_jobs_dev : (long long)jb.g[i].n_jobs;
            s_base[i + 1] = b;
        }
    }
    __syncthreads();
    const long long njobs = s_base[jb.n_groups];
    const float bd = pk[f.bd];

    for (;;) {
        if (j == 0) s_job = (long long)atomicAdd(jb.job_counter, 1ull);
        __syncthreads();
        const long long job = s_job;
        __syncthreads();
        if (job >= njobs) break;
        int gi = 0;
        while (gi + 1 < jb.n_groups && job >= s_base[gi + 1]) ++gi;
        const FwdGroup &G = jb.g[gi];
        const long long lj = job - s_base[gi];
        const int N = G.N;
        const int nch = (N + CH - 1) / CH;
        int sample, p = -1, q = -1, c0 = 0;
        if (jb.mode == 0) {
            sample = (int)lj;
        } else {
            const int32_t *e = G.entries + 3 * lj;
            sample = e[0];
            p = e[1];
            q = e[2];
            c0 = p / CH;
        }
        const uint64_t *row = G.bits + (int64_t)sample * G.W;
        // complex carries, one (Re, Im) pair per layer, in registers
        float cre[kMaxLayers], cim[kMaxLayers];
#pragma unroll
        for (int l = 0; l < kMaxLayers; ++l) {
            cre[l] = 0.0f;
            cim[l] = 0.0f;
            if (l < nL && c0 > 0) {
                const float *cin = G.carries_in + (((int64_t)sample * nch + c0) * nL + l) * 2 * H;
                cre[l] = cin[j];
                cim[l] = cin[H + j];
            }
        }
        int n_up = G.u1 ? count_up_before(row, c0 * CH) : 0;
        float acc = 0.0f;

        for (int c = c0; c < nch; ++c) {
            const int t0 = c * CH;
            if (G.carries_out) {
#pragma unroll
                for (int l = 0; l < kMaxLayers; ++l)
                    if (l < nL) {
                        float *co = G.carries_out + (((int64_t)sample * nch + c) * nL + l) * 2 * H;
                        co[j] = cre[l];
                        co[H + j] = cim[l];
                    }
            }
            uint32_t cur, prev;
            chunk_bits32(row, t0, p, q, cur, prev);
            const int nvalid = min(CH, N - t0);
            if (nvalid < 32) cur &= (1u << nvalid) - 1u;
            const uint32_t prevbits = (cur << 1) | prev;  // bit t = s_{t0+t-1}

#pragma unroll 1
            for (int l = 0; l < nL; ++l) {
                float br[CH], bi[CH];
                const float g = pk[f.gam[l] + j];
                if (l == 0) {
                    // one-hot input: column gathers of B (zero at the first site)
                    const float r0 = pk[f.BreT[0] + j], r1 = pk[f.BreT[0] + H + j];
                    const float i0 = pk[f.BimT[0] + j], i1 = pk[f.BimT[0] + H + j];
#pragma unroll
                    for (int t = 0; t < CH; ++t) {
                        const bool first = (t0 + t == 0);
                        const bool sb = (prevbits >> t) & 1u;
                        br[t] = first ? 0.0f : (sb ? r1 : r0);
                        bi[t] = first ? 0.0f : (sb ? i1 : i0);
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < CH; ++t) {
                        br[t] = 0.0f;
                        bi[t] = 0.0f;
                    }
                    const float *Br = pk + f.BreT[l], *Bi = pk + f.BimT[l];
#pragma unroll 4
                    for (int k = 0; k < H; ++k) {
                        const float wr = Br[k * H + j], wi = Bi[k * H + j];
                        const float4 *src = reinterpret_cast<const float4 *>(xs + k * LD);
#pragma unroll
                        for (int t4 = 0; t4 < CH / 4; ++t4) {
                            const float4 v = src[t4];
                            br[4 * t4] += wr * v.x; br[4 * t4 + 1] += wr * v.y;
                            br[4 * t4 + 2] += wr * v.z; br[4 * t4 + 3] += wr * v.w;
                            bi[4 * t4] += wi * v.x; bi[4 * t4 + 1] += wi * v.y;
                            bi[4 * t4 + 2] += wi * v.z; bi[4 * t4 + 3] += wi * v.w;
                        }
                    }
                }
                // complex scan h_t = lambda h_{t-1} + e^gamma (B u_t)
                {
                    const float lr = pk[f.lre[l] + j], li = pk[f.lim[l] + j];
                    float zr = 0.0f, zi = 0.0f;
#pragma unroll
                    for (int k = 0; k < kMaxLayers; ++k)
                        if (k == l) { zr = cre[k]; zi = cim[k]; }
#pragma unroll
                    for (int t = 0; t < CH; ++t) {
                        const float nr = fmaf(lr, zr, fmaf(-li, zi, g * br[t]));
                        const float ni = fmaf(lr, zi, fmaf(li, zr, g * bi[t]));
                        zr = nr;
                        zi = ni;
                        br[t] = zr;
                        bi[t] = zi;
                    }
#pragma unroll
                    for (int k = 0; k < kMaxLayers; ++k)
                        if (k == l) { cre[k] = zr; cim[k] = zi; }
                }
                float4 *dr = reinterpret_cast<float4 *>(hr + j * LD);
                float4 *di = reinterpret_cast<float4 *>(hi + j * LD);
#pragma unroll
                for (int t4 = 0; t4 < CH / 4; ++t4) {
                    dr[t4] = make_float4(br[4 * t4], br[4 * t4 + 1], br[4 * t4 + 2], br[4 * t4 + 3]);
                    di[t4] = make_float4(bi[4 * t4], bi[4 * t4 + 1], bi[4 * t4 + 2], bi[4 * t4 + 3]);
                }
                __syncthreads();
                // y = Re(C h) + D u
                float y[CH];
                if (l == 0) {
                    const float d0 = pk[f.D[0] + j], d1 = pk[f.D[0] + H + j];
#pragma unroll
                    for (int t = 0; t < CH; ++t) {
                        const bool first = (t0 + t == 0);
                        const bool sb = (prevbits >> t) & 1u;
                        y[t] = first ? 0.0f : (sb ? d1 : d0);
                    }
                } else {
                    const float dj = pk[f.D[l] + j];
                    const float4 *src = reinterpret_cast<const float4 *>(xs + j * LD);
#pragma unroll
                    for (int t4 = 0; t4 < CH / 4; ++t4) {
                        const float4 v = src[t4];
                        y[4 * t4] = dj * v.x; y[4 * t4 + 1] = dj * v.y;
                        y[4 * t4 + 2] = dj * v.z; y[4 * t4 + 3] = dj * v.w;
                    }
                }
                {
                    const float *Cr = pk + f.CreT[l], *Ci = pk + f.CimT[l];
#pragma unroll 4
                    for (int m = 0; m < H; ++m) {
                        const float wr = Cr[m * H + j], wi = Ci[m * H + j];
                        const float4 *sr = reinterpret_cast<const float4 *>(hr + m * LD);
                        const float4 *si = reinterpret_cast<const float4 *>(hi + m * LD);
#pragma unroll
                        for (int t4 = 0; t4 < CH / 4; ++t4) {
                            const float4 a = sr[t4], b = si[t4];
                            y[4 * t4] += wr * a.x - wi * b.x; y[4 * t4 + 1] += wr * a.y - wi * b.y;
                            y[4 * t4 + 2] += wr * a.z - wi * b.z; y[4 * t4 + 3] += wr * a.w - wi * b.w;
                        }
                    }
                }
                float4 *dy = reinterpret_cast<float4 *>(ys + j * LD);
#pragma unroll
                for (int t4 = 0; t4 < CH / 4; ++t4)
                    dy[t4] = make_float4(y[4 * t4], y[4 * t4 + 1], y[4 * t4 + 2], y[4 * t4 + 3]);
                __syncthreads();
                // GLU + residual
                float a[CH], gg[CH];
                {
                    const float ba = pk[f.ba[l] + j], bg = pk[f.bg[l] + j];
#pragma unroll
                    for (int t = 0; t < CH; ++t) {
                        a[t] = ba;
                        gg[t] = bg;
                    }
                    const float *Wa = pk + f.WaT[l], *Wg = pk + f.WgT[l];
#pragma unroll 4
                    for (int k = 0; k < H; ++k) {
                        const float wa = Wa[k * H + j], wg = Wg[k * H + j];
                        const float4 *src = reinterpret_cast<const float4 *>(ys + k * LD);
#pragma unroll
                        for (int t4 = 0; t4 < CH / 4; ++t4) {
                            const float4 v = src[t4];
                            a[4 * t4] += wa * v.x; a[4 * t4 + 1] += wa * v.y;
                            a[4 * t4 + 2] += wa * v.z; a[4 * t4 + 3] += wa * v.w;
                            gg[4 * t4] += wg * v.x; gg[4 * t4 + 1] += wg * v.y;
                            gg[4 * t4 + 2] += wg * v.z; gg[4 * t4 + 3] += wg * v.w;
                        }
                    }
                }
                float4 *dx = reinterpret_cast<float4 *>(xs + j * LD);
                float xo[CH];
#pragma unroll
                for (int t4 = 0; t4 < CH / 4; ++t4) {
                    float4 r = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (l >= 1) r = dx[t4];  // this unit's own input: residual
                    xo[4 * t4] = a[4 * t4] * sigmoid_f(gg[4 * t4]) + r.x;
                    xo[4 * t4 + 1] = a[4 * t4 + 1] * sigmoid_f(gg[4 * t4 + 1]) + r.y;
                    xo[4 * t4 + 2] = a[4 * t4 + 2] * sigmoid_f(gg[4 * t4 + 2]) + r.z;
                    xo[4 * t4 + 3] = a[4 * t4 + 3] * sigmoid_f(gg[4 * t4 + 3]) + r.w;
                }
                __syncthreads();  // every read of xs (B u) and ys is done
#pragma unroll
                for (int t4 = 0; t4 < CH / 4; ++t4)
                    dx[t4] = make_float4(xo[4 * t4], xo[4 * t4 + 1], xo[4 * t4 + 2], xo[4 * t4 + 3]);
                __syncthreads();
            }

            // readout: thread t < 32 handles site t0 + t
            if (j < 32) {
                const int t = j;
                float v = 0.0f;
                const int tt = t0 + t;
                if (tt < N) {
                    float d = bd;
                    const float *wd = pk + f.wd;
                    for (int k = 0; k < H; ++k) d += wd[k] * xs[k * LD + t];
                    const int s = (cur >> t) & 1u;
                    const int nu = n_up + __popc(cur & ((1u << t) - 1u));
                    const float lp = site_logp(d, s, u1_forced(G.u1, N, tt, nu));
                    if (G.logp_out) G.logp_out[(int64_t)sample * N + tt] = lp;
                    v = (jb.mode == 1) ? lp - G.logp_ref[(int64_t)sample * N + tt] : lp;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (j == 0) acc += v;
            }
            n_up += __popc(cur);
            __syncthreads();
        }
        if (j == 0) G.out[lj] = 0.5f * acc;
    }
}

template <int H>
cudaError_t launch_lru_h(const FwdJobs &jobs, const float *packed, const LruLayout &f, int num_sms,
                         cudaStream_t stream) {
    const size_t smem = (size_t)4 * H * LD * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(lru_f32_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lru_f32_kernel<H>, H, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)num_sms * per_sm;
    const int64_t nj = max_jobs(jobs);
    if (nj < grid) grid = nj;
    if (grid < 1) grid = 1;
    lru_f32_kernel<H><<<(int)grid, H, smem, stream>>>(jobs, packed, f);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pack_theta_lru(const float *theta, const LruLayout &f, float *packed,
                                  cudaStream_t stream) {
    pack_lru_kernel<<<64, 256, 0, stream>>>(theta, f, packed);
    return cudaGetLastError();
}

cudaError_t launch_lru_f32(const FwdJobs &jobs, const float *packed, const LruLayout &f, int num_sms,
                           cudaStream_t stream) {
    switch (f.H) {
        case 32: return launch_lru_h<32>(jobs, packed, f, num_sms, stream);
        case 64: return launch_lru_h<64>(jobs, packed, f, num_sms, stream);
        case 128: return launch_lru_h<128>(jobs, packed, f, num_sms, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace psr
