// FP32 SIMT forward of the PSR-NQS ansatz (the plain path), parameter
// packing and spin bit-packing.
//
// One CTA of H threads evaluates one sequence at a time (thread j owns hidden
// unit j) and walks it chunk by chunk (32 sites).  Inside a chunk:
//   layer 0  : gates from lookup tables of the one-hot input onehot(s_{t-1})
//              (Sec. II.F: zero input at the first site), the recurrence
//              h_t = a_t h_{t-1} + b_t (Sec. II.C) carried in a register,
//              then x^(1) = GELU(C h + D u) (Sec. II.F-G);
//   layer l>0: z = W_z x + b_z, h~ = W_h x + b_h (FP32 FMA over a shared-memory
//              tile), a = sigmoid(z), b = (1 - a) h~, the same scan, and
//              x^(l+1) = GELU(C h + D x + [l >= 2] h^(l-1));
//   readout  : d_t = (W_o[1] - W_o[0]) x_t + (b_o[1] - b_o[0]) and
//              log P(s_t) = -softplus(-+d_t) (two-way softmax), summed over
//              sites; log psi = 1/2 sum_t log P (Sec. III.B).
// The scan carry of each layer crosses chunk boundaries in shared memory, so
// a sequence needs no inter-CTA communication; jobs are handed out by an
// atomic counter for load balance over ragged sequence lengths.
#include <cuda_runtime.h>

#include "psr_device.cuh"
#include "psr_internal.cuh"

namespace psr {

ThetaLayout theta_layout(int nL, int H) {
    ThetaLayout t{};
    t.nL = nL;
    t.H = H;
    int64_t off = 0;
    for (int l = 0; l < nL; ++l) {
        int64_t din = (l == 0) ? 2 : H;
        t.Wz[l] = off; off += H * din;
        t.bz[l] = off; off += H;
        t.Wh[l] = off; off += H * din;
        t.bh[l] = off; off += H;
        t.C[l] = off;  off += (int64_t)H * H;
        t.D[l] = off;  off += H * din;
    }
    t.Wo = off; off += 2 * H;
    t.bo = off; off += 2;
    t.total = off;
    return t;
}

F32Layout f32_layout(int nL, int H) {
    F32Layout f{};
    f.nL = nL;
    f.H = H;
    int64_t off = 0;
    for (int l = 0; l < nL; ++l) {
        int64_t din = (l == 0) ? 2 : H;
        f.WzT[l] = off; off += din * H;
        f.WhT[l] = off; off += din * H;
        f.CT[l] = off;  off += (int64_t)H * H;
        f.DT[l] = off;  off += din * H;
        f.bz[l] = off;  off += H;
        f.bh[l] = off;  off += H;
    }
    f.A0 = off;  off += 3 * H;
    f.B0 = off;  off += 3 * H;
    f.DU0 = off; off += 3 * H;
    f.CD0 = off; off += 3 * H;
    f.wd = off;  off += H;
    f.bd = off;  off += 4;
    f.total = off;
    return f;
}

__global__ void pack_f32_kernel(const float *__restrict__ theta, ThetaLayout tl, F32Layout fl,
                                float *__restrict__ pk) {
    const int H = tl.H;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int l = 0; l < tl.nL; ++l) {
        const int din = (l == 0) ? 2 : H;
        for (int64_t i = tid; i < (int64_t)din * H; i += stride) {
            int k = (int)(i / H), j = (int)(i % H);
            pk[fl.WzT[l] + i] = theta[tl.Wz[l] + (int64_t)j * din + k];
            pk[fl.WhT[l] + i] = theta[tl.Wh[l] + (int64_t)j * din + k];
            pk[fl.DT[l] + i] = theta[tl.D[l] + (int64_t)j * din + k];
        }
        for (int64_t i = tid; i < (int64_t)H * H; i += stride) {
            int k = (int)(i / H), j = (int)(i % H);
            pk[fl.CT[l] + i] = theta[tl.C[l] + (int64_t)j * H + k];
        }
        for (int64_t i = tid; i < H; i += stride) {
            pk[fl.bz[l] + i] = theta[tl.bz[l] + i];
            pk[fl.bh[l] + i] = theta[tl.bh[l] + i];
        }
    }
    for (int64_t i = tid; i < 3 * H; i += stride) {
        int code = (int)(i / H), j = (int)(i % H);
        float zp = theta[tl.bz[0] + j];
        float cd = theta[tl.bh[0] + j];
        float du = 0.0f;
        if (code > 0) {
            zp += theta[tl.Wz[0] + 2 * j + (code - 1)];
            cd += theta[tl.Wh[0] + 2 * j + (code - 1)];
            du = theta[tl.D[0] + 2 * j + (code - 1)];
        }
        float a = sigmoid_f(zp);
        pk[fl.A0 + i] = a;
        pk[fl.B0 + i] = (1.0f - a) * cd;
        pk[fl.DU0 + i] = du;
        pk[fl.CD0 + i] = cd;
    }
    for (int64_t i = tid; i < H; i += stride)
        pk[fl.wd + i] = theta[tl.Wo + H + i] - theta[tl.Wo + i];
    if (tid == 0) pk[fl.bd] = theta[tl.bo + 1] - theta[tl.bo];
}

cudaError_t launch_pack_theta_f32(const float *theta, const ThetaLayout &tl, const F32Layout &fl,
                                  float *packed, cudaStream_t stream) {
    pack_f32_kernel<<<64, 256, 0, stream>>>(theta, tl, fl, packed);
    return cudaGetLastError();
}

// One thread per 64-bit word; a byte other than 0/1 is reported as
// PSR_EDEVICE and treated as its lowest bit.  Words past N are zero.
__global__ void bitpack_kernel(const uint8_t *__restrict__ spins, int64_t n, int N, int W,
                               uint64_t *__restrict__ bits, int *status) {
    const int64_t total = n * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = i / W;
        int w = (int)(i % W);
        const uint8_t *row = spins + s * N;
        uint64_t word = 0;
        int bad = 0;
        for (int b = 0; b < 64; ++b) {
            int t = w * 64 + b;
            if (t >= N) break;
            uint8_t v = row[t];
            bad |= (v > 1);
            word |= (uint64_t)(v & 1u) << b;
        }
        if (bad) set_status(status, PSR_EDEVICE);
        bits[i] = word;
    }
}

cudaError_t launch_bitpack(const uint8_t *spins, int64_t n, int N, int W, uint64_t *bits,
                           int *status, cudaStream_t stream) {
    int64_t total = n * W;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 65535) blocks = 65535;
    if (blocks < 1) blocks = 1;
    bitpack_kernel<<<blocks, 256, 0, stream>>>(spins, n, N, W, bits, status);
    return cudaGetLastError();
}

template <int H, int CH>
__global__ void __launch_bounds__(H) fwd_f32_kernel(const __grid_constant__ FwdJobs jb,
                                                   const float *__restrict__ pk, F32Layout fl) {
    static_assert(CH == 16 || CH == 32, "chunk of 16 or 32 sites");
    constexpr int LD = CH + 4;  // padded row: conflict-free float4 row writes
    extern __shared__ __align__(16) float smem[];
    float *xs = smem;              // [H][LD] layer input / output
    float *hs = xs + H * LD;       // [H][LD] hidden states of the chunk
    float *hcar = hs + H * LD;     // [kMaxLayers][H] scan carries
    __shared__ long long s_job;
    __shared__ long long s_base[kMaxGroups + 1];

    const int j = threadIdx.x;
    const int nL = fl.nL;
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

    const float a0_0 = pk[fl.A0 + j], a0_1 = pk[fl.A0 + H + j], a0_2 = pk[fl.A0 + 2 * H + j];
    const float b0_0 = pk[fl.B0 + j], b0_1 = pk[fl.B0 + H + j], b0_2 = pk[fl.B0 + 2 * H + j];
    const float d0_0 = pk[fl.DU0 + j], d0_1 = pk[fl.DU0 + H + j], d0_2 = pk[fl.DU0 + 2 * H + j];
    const float bd = pk[fl.bd];

    for (;;) {
        if (j == 0) s_job = (long long)atomicAdd((unsigned long long *)jb.job_counter, 1ull);
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
        for (int l = 0; l < nL; ++l)
            hcar[l * H + j] = (c0 == 0) ? 0.0f
                : G.carries_in[(((int64_t)sample * nch + c0) * nL + l) * H + j];
        int n_up = G.u1 ? count_up_before(row, c0 * CH) : 0;
        float acc = 0.0f;

        for (int c = c0; c < nch; ++c) {
            const int t0 = c * CH;
            if (G.carries_out)
                for (int l = 0; l < nL; ++l)
                    G.carries_out[(((int64_t)sample * nch + c) * nL + l) * H + j] = hcar[l * H + j];
            uint32_t cur, prev;
            chunk_bits32(row, t0, p, q, cur, prev);
            const int nvalid = min(CH, N - t0);
            if (nvalid < 32) cur &= (1u << nvalid) - 1u;
            // input code of site t: 0 = first site, 1 + s_{t-1} otherwise
            const uint32_t prevbits = (cur << 1) | prev;  // bit t = s_{t0+t-1}

            float hl[CH];  // h of the current layer (residual source for the next)
            float y[CH];
            {
                float hv = hcar[j];
#pragma unroll
                for (int t = 0; t < CH; ++t) {
                    const bool first = (t0 + t == 0);
                    const uint32_t sb = (prevbits >> t) & 1u;
                    const float a = first ? a0_0 : (sb ? a0_2 : a0_1);
                    const float b = first ? b0_0 : (sb ? b0_2 : b0_1);
                    hv = a * hv + b;
                    hl[t] = hv;
                    y[t] = first ? d0_0 : (sb ? d0_2 : d0_1);
                }
                hcar[j] = hv;
                float4 *dst = reinterpret_cast<float4 *>(hs + j * LD);
#pragma unroll
                for (int t4 = 0; t4 < CH / 4; ++t4)
                    dst[t4] = make_float4(hl[4 * t4], hl[4 * t4 + 1], hl[4 * t4 + 2], hl[4 * t4 + 3]);
            }
            __syncthreads();
            {
                const float *Ct = pk + fl.CT[0];
                #pragma unroll 4
                for (int k = 0; k < H; ++k) {
                    const float w = Ct[k * H + j];
                    const float4 *src = reinterpret_cast<const float4 *>(hs + k * LD);
#pragma unroll
                    for (int t4 = 0; t4 < CH / 4; ++t4) {
                        float4 v = src[t4];
                        y[4 * t4] += w * v.x; y[4 * t4 + 1] += w * v.y;
                        y[4 * t4 + 2] += w * v.z; y[4 * t4 + 3] += w * v.w;
                    }
                }
                float4 *dst = reinterpret_cast<float4 *>(xs + j * LD);
#pragma unroll
                for (int t4 = 0; t4 < CH / 4; ++t4)
                    dst[t4] = make_float4(gelu_f(y[4 * t4]), gelu_f(y[4 * t4 + 1]),
                                          gelu_f(y[4 * t4 + 2]), gelu_f(y[4 * t4 + 3]));
            }
            __syncthreads();

            for (int l = 1; l < nL; ++l) {
                float z[CH];
                const float bz = pk[fl.bz[l] + j], bh = pk[fl.bh[l] + j];
#pragma unroll
                for (int t = 0; t < CH; ++t) { z[t] = bz; y[t] = bh; }
                const float *Wz = pk + fl.WzT[l];
                const float *Wh = pk + fl.WhT[l];
                #pragma unroll 4
                for (int k = 0; k < H; ++k) {
                    const float wz = Wz[k * H + j], wh = Wh[k * H + j];
                    const float4 *src = reinterpret_cast<const float4 *>(xs + k * LD);
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
                    float hv = hcar[l * H + j];
#pragma unroll
                    for (int t = 0; t < CH; ++t) {
                        const float a = sigmoid_f(z[t]);
                        hv = a * hv + (1.0f - a) * y[t];
                        hn[t] = hv;
                    }
                    hcar[l * H + j] = hv;
                    float4 *dst = reinterpret_cast<float4 *>(hs + j * LD);
#pragma unroll
                    for (int t4 = 0; t4 < CH / 4; ++t4)
                        dst[t4] = make_float4(hn[4 * t4], hn[4 * t4 + 1], hn[4 * t4 + 2], hn[4 * t4 + 3]);
                }
                __syncthreads();
#pragma unroll
                for (int t = 0; t < CH; ++t) y[t] = (l >= 2) ? hl[t] : 0.0f;
                const float *Ct = pk + fl.CT[l];
                const float *Dt = pk + fl.DT[l];
                #pragma unroll 4
                for (int k = 0; k < H; ++k) {
                    const float wc = Ct[k * H + j], wd = Dt[k * H + j];
                    const float4 *sh = reinterpret_cast<const float4 *>(hs + k * LD);
                    const float4 *sx = reinterpret_cast<const float4 *>(xs + k * LD);
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
                float4 *dst = reinterpret_cast<float4 *>(xs + j * LD);
#pragma unroll
                for (int t4 = 0; t4 < CH / 4; ++t4)
                    dst[t4] = make_float4(gelu_f(y[4 * t4]), gelu_f(y[4 * t4 + 1]),
                                          gelu_f(y[4 * t4 + 2]), gelu_f(y[4 * t4 + 3]));
#pragma unroll
                for (int t = 0; t < CH; ++t) hl[t] = hn[t];
                __syncthreads();
            }

            // readout: thread t < CH handles site t0 + t (warp 0 reduces)
            if (j < 32) {
                const int t = j;
                float v = 0.0f;
                const int tt = t0 + t;
                if (t < CH && tt < N) {
                    float d = bd;
                    const float *wd = pk + fl.wd;
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

template <int H, int CH>
static cudaError_t launch_fwd_f32_h(const FwdJobs &jobs, const float *packed, const F32Layout &fl,
                                    int num_sms, cudaStream_t stream) {
    const size_t smem = (size_t)(2 * H * (CH + 4) + kMaxLayers * H) * sizeof(float);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fwd_f32_kernel<H, CH>, H, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)num_sms * per_sm;
    const int64_t nj = max_jobs(jobs);
    if (nj < grid) grid = nj;
    if (grid < 1) grid = 1;
    fwd_f32_kernel<H, CH><<<(int)grid, H, smem, stream>>>(jobs, packed, fl);
    return cudaGetLastError();
}

cudaError_t launch_fwd_f32(const FwdJobs &jobs, const float *packed, const F32Layout &fl,
                           int num_sms, cudaStream_t stream, int chunk) {
    if (chunk == kChunkGrad) {
        switch (fl.H) {
            case 32: return launch_fwd_f32_h<32, kChunkGrad>(jobs, packed, fl, num_sms, stream);
            case 64: return launch_fwd_f32_h<64, kChunkGrad>(jobs, packed, fl, num_sms, stream);
            case 128: return launch_fwd_f32_h<128, kChunkGrad>(jobs, packed, fl, num_sms, stream);
            default: return cudaErrorInvalidValue;
        }
    }
    if (chunk != kChunkF32) return cudaErrorInvalidValue;
    switch (fl.H) {
        case 32: return launch_fwd_f32_h<32, kChunkF32>(jobs, packed, fl, num_sms, stream);
        case 64: return launch_fwd_f32_h<64, kChunkF32>(jobs, packed, fl, num_sms, stream);
        case 128: return launch_fwd_f32_h<128, kChunkF32>(jobs, packed, fl, num_sms, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace psr
