// Forward of the paper's two-dimensional patched minGRU (Sec. II.F,
// two-dimensional recurrences; Sec. II.G residual), FP32 on CUDA cores.
//
// The Lx x Ly spin lattice is cut into 2 x 2 patches (value v = sum of
// s(2i+dx, 2j+dy) 2^(2dy+dx), 16-way conditionals) visited along the zigzag
// path of the patch lattice.  The recurrence is evaluated row by row, as the
// paper describes: within a patch row every site's horizontal predecessor is
// the previous site on the path and the row starts from h_H = 0; the vertical
// predecessor (i, j-1) belongs to the previous row, which is complete.  So for
// one row and one layer the gates z = sigma(W_z u + b_z) and candidates
// h~ = W_h [u, h_V] + b_h of all the row's sites are a batched projection
// (the h_V part multiplies the previous row's states), followed by the scan
// h = z h_H + (1 - z) h~ along the row.
//
// One CTA evaluates one configuration at a time (jobs from an atomic
// counter); thread j owns hidden unit j for all sites of the row (up to 32
// patches).  Shared memory holds the row's layer input and states and, per
// layer, the previous row's states stored in the current row's path order
// (consecutive rows run in opposite directions, so column i of the previous
// row sits at path position Px - 1 - k of the current one).
//   mode 0 (samples): log psi, per-patch log P and, optionally, the previous
//     row's states before every row (row checkpoints);
//   mode 1 (connected configurations): the sample with spins p, q flipped,
//     resumed at the patch row holding p from the sample's checkpoint, giving
//     log psi(s') - log psi(s) as a sum of per-patch differences.
#include <cuda_runtime.h>

#include "psr_device.cuh"
#include "psr_internal.cuh"

namespace psr {

F2Layout f2_layout(int nL, int H) {
    F2Layout f{};
    f.nL = nL;
    f.H = H;
    int64_t off = 0;
    auto take = [&](int64_t n) {
        const int64_t o = off;
        off += (n + 3) & ~int64_t(3);  // 16-byte aligned tensors
        return o;
    };
    for (int l = 0; l < nL; ++l) {
        const int din = l == 0 ? 32 : H;
        f.WzT[l] = take((int64_t)din * H);
        f.WhxT[l] = take((int64_t)din * H);
        f.WhvT[l] = take((int64_t)H * H);
        f.CT[l] = take((int64_t)H * H);
        f.DT[l] = take((int64_t)din * H);
        f.bz[l] = take(H);
        f.bh[l] = take(H);
    }
    f.Wo = take(16 * (int64_t)H);
    f.bo = take(16);
    f.total = off;
    return f;
}

int64_t param_count2d(int nL, int H) {
    int64_t P = 0;
    for (int l = 0; l < nL; ++l) {
        const int64_t din = l == 0 ? 32 : H;
        P += H * din + H + H * (din + H) + H + (int64_t)H * H + H * din;
    }
    return P + 16 * (int64_t)H + 16;
}

namespace {

// theta (flat 2D layout) -> transposed FP32 matrices for unit-coalesced reads.
__global__ void pack_f2_kernel(const float *__restrict__ theta, F2Layout f, float *__restrict__ pk) {
    const int H = f.H;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t src = 0;
    for (int l = 0; l < f.nL; ++l) {
        const int din = l == 0 ? 32 : H;
        const int64_t Wz = src, bz = Wz + (int64_t)H * din, Wh = bz + H,
                      bh = Wh + (int64_t)H * (din + H), C = bh + H, D = C + (int64_t)H * H;
        src = D + (int64_t)H * din;
        for (int64_t i = tid; i < (int64_t)H * din; i += stride) {
            const int j = (int)(i / din), k = (int)(i % din);  // row j (output unit), column k
            pk[f.WzT[l] + (int64_t)k * H + j] = theta[Wz + i];
            pk[f.DT[l] + (int64_t)k * H + j] = theta[D + i];
        }
        for (int64_t i = tid; i < (int64_t)H * (din + H); i += stride) {
            const int j = (int)(i / (din + H)), k = (int)(i % (din + H));
            if (k < din) pk[f.WhxT[l] + (int64_t)k * H + j] = theta[Wh + i];
            else pk[f.WhvT[l] + (int64_t)(k - din) * H + j] = theta[Wh + i];
        }
        for (int64_t i = tid; i < (int64_t)H * H; i += stride) {
            const int j = (int)(i / H), k = (int)(i % H);
            pk[f.CT[l] + (int64_t)k * H + j] = theta[C + i];
        }
        for (int64_t i = tid; i < H; i += stride) {
            pk[f.bz[l] + i] = theta[bz + i];
            pk[f.bh[l] + i] = theta[bh + i];
        }
    }
    for (int64_t i = tid; i < 16 * (int64_t)H + 16; i += stride) pk[f.Wo + i] = theta[src + i];
}

constexpr int kRow = 32;       // patches per row handled by one CTA (max)

__device__ __forceinline__ int seq_pos2d(int Lx, int i, int j) {
    return j * Lx + ((j & 1) ? (Lx - 1 - i) : i);
}

// spin at lattice (i, j) of a configuration with sites p and q flipped
__device__ __forceinline__ int spin_at(const uint8_t *s, int Lx, int i, int j, int p, int q) {
    const int pos = seq_pos2d(Lx, i, j);
    return (int)(s[pos] & 1u) ^ (pos == p) ^ (pos == q);
}

// R: patches per row (row2d_width(Lx) >= Lx / 2), held in registers; shared rows
// and row checkpoints are R + 4 floats wide (float4 rows).
template <int H, int R>
__global__ void __launch_bounds__(H) fwd2d_f32_kernel(const __grid_constant__ Fwd2Jobs jb,
                                                      const float *__restrict__ pk, F2Layout f) {
    constexpr int LD = R + 4;
    extern __shared__ __align__(16) float smem[];
    const int nL = f.nL;
    float *xs = smem;                    // [H][LD] layer input / output of the row
    float *hs = xs + H * LD;            // [H][LD] states of the current layer
    float *hv = hs + H * LD;            // [nL][H][LD] previous row's states (path order)
    float *lg = hv + nL * H * LD;       // [16][LD] logits of the row
    __shared__ int s_v[kRow];            // patch values of the row (path order)
    __shared__ int s_vprev[kRow];        // previous row's values by column
    __shared__ float s_part[1];
    __shared__ long long s_job;

    const int j = threadIdx.x;
    const int lane = j & 31;
    const Fwd2Group &G = jb.g;
    const int Lx = G.Lx, Ly = G.Ly, Px = Lx >> 1, Py = Ly >> 1, N = Lx * Ly, Np = Px * Py;
    const long long njobs = jb.mode == 1 ? (long long)*G.n_jobs_dev : (long long)G.n_jobs;
    const float *Wo = pk + f.Wo;
    const size_t ckpt_row = (size_t)nL * H * LD;  // floats of one row checkpoint

    for (;;) {
        if (j == 0) s_job = (long long)atomicAdd(jb.job_counter, 1ull);
        __syncthreads();
        const long long job = s_job;
        __syncthreads();
        if (job >= njobs) break;
        int sample, p = -1, q = -1, r0 = 0;
        if (jb.mode == 0) {
            sample = (int)job;
        } else {
            const int32_t *e = G.entries + 3 * job;
            sample = e[0];
            p = e[1];
            q = e[2];
            r0 = (p / Lx) >> 1;  // patch row of the first flipped spin
        }
        const uint8_t *sp = G.spins + (size_t)sample * N;

        // state before row r0: the previous row's states and values, the
        // up / down counts of every earlier patch (the flips come later)
        if (r0 == 0) {
            for (int i = j; i < nL * H * LD; i += H) hv[i] = 0.0f;
        } else {
            const float *src = G.carries_in + ((size_t)sample * Py + r0) * ckpt_row;
            for (int i = j; i < nL * H * LD; i += H) hv[i] = src[i];
        }
        if (j < Px && r0 > 0) {
            const int pj = r0 - 1;
            int v = 0;
            for (int b = 0; b < 4; ++b) v |= spin_at(sp, Lx, 2 * j + (b & 1), 2 * pj + (b >> 1), -1, -1) << b;
            s_vprev[j] = v;
        }
        int n_up = 0;
        for (int t = j; t < 2 * r0 * Lx; t += H) n_up += sp[t] & 1;
        for (int o = 16; o > 0; o >>= 1) n_up += __shfl_xor_sync(0xffffffffu, n_up, o);
        __shared__ int s_up[H / 32];
        if (lane == 0) s_up[j >> 5] = n_up;
        __syncthreads();
        n_up = 0;
        for (int w = 0; w < H / 32; ++w) n_up += s_up[w];
        int n_down = 2 * r0 * Lx - n_up;
        float acc = 0.0f;

        for (int pj = r0; pj < Py; ++pj) {
            if (jb.mode == 0 && G.carries_out) {
                float *dst = G.carries_out + ((size_t)sample * Py + pj) * ckpt_row;
                for (int i = j; i < nL * H * LD; i += H) dst[i] = hv[i];
            }
            if (j < Px) {
                const int pi = (pj & 1) ? Px - 1 - j : j;
                int v = 0;
                for (int b = 0; b < 4; ++b) v |= spin_at(sp, Lx, 2 * pi + (b & 1), 2 * pj + (b >> 1), p, q) << b;
                s_v[j] = v;
            }
            __syncthreads();

            float hl[R];  // this unit's states of the layer below (residual source)
            // ---------------- layer 0: inputs onehot(v_H), onehot(v_V)
            {
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
                    const float *hv0 = hv;
#pragma unroll 4
                    for (int m = 0; m < H; ++m) {
                        const float w = Wv[m * H + j];
                        const float4 *src = reinterpret_cast<const float4 *>(hv0 + m * LD);
#pragma unroll
                        for (int k4 = 0; k4 < R / 4; ++k4) {
                            const float4 v = src[k4];
                            c[4 * k4] += w * v.x; c[4 * k4 + 1] += w * v.y;
                            c[4 * k4 + 2] += w * v.z; c[4 * k4 + 3] += w * v.w;
                        }
                    }
                }
                float h = 0.0f;  // the row starts from h_H = 0
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const float a = sigmoid_f(z[k]);
                    h = a * h + (1.0f - a) * c[k];
                    hl[k] = h;
                }
                float4 *dst = reinterpret_cast<float4 *>(hs + j * LD);
#pragma unroll
                for (int k4 = 0; k4 < R / 4; ++k4)
                    dst[k4] = make_float4(hl[4 * k4], hl[4 * k4 + 1], hl[4 * k4 + 2], hl[4 * k4 + 3]);
                __syncthreads();  // all reads of hv[0] and writes of hs done
                const float *Ct = pk + f.CT[0];
#pragma unroll 4
                for (int m = 0; m < H; ++m) {
                    const float w = Ct[m * H + j];
                    const float4 *src = reinterpret_cast<const float4 *>(hs + m * LD);
#pragma unroll
                    for (int k4 = 0; k4 < R / 4; ++k4) {
                        const float4 v = src[k4];
                        y[4 * k4] += w * v.x; y[4 * k4 + 1] += w * v.y;
                        y[4 * k4 + 2] += w * v.z; y[4 * k4 + 3] += w * v.w;
                    }
                }
                float4 *xd = reinterpret_cast<float4 *>(xs + j * LD);
#pragma unroll
                for (int k4 = 0; k4 < R / 4; ++k4)
                    xd[k4] = make_float4(gelu_f(y[4 * k4]), gelu_f(y[4 * k4 + 1]), gelu_f(y[4 * k4 + 2]),
                                         gelu_f(y[4 * k4 + 3]));
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if (k < Px) hv[j * LD + (Px - 1 - k)] = hl[k];
                __syncthreads();
            }
            // ---------------- layers l >= 1
            for (int l = 1; l < nL; ++l) {
                const float *WzT = pk + f.WzT[l], *WhxT = pk + f.WhxT[l], *Wv = pk + f.WhvT[l];
                float *hvl = hv + (size_t)l * H * LD;
                float z[R], c[R];
                const float bz = pk[f.bz[l] + j], bh = pk[f.bh[l] + j];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    z[k] = bz;
                    c[k] = bh;
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
                {
                    float h = 0.0f;
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        const float a = sigmoid_f(z[k]);
                        h = a * h + (1.0f - a) * c[k];
                        hn[k] = h;
                    }
                }
                __syncthreads();  // every read of hs (previous layer) and hv[l] is done
                float4 *dst = reinterpret_cast<float4 *>(hs + j * LD);
#pragma unroll
                for (int k4 = 0; k4 < R / 4; ++k4)
                    dst[k4] = make_float4(hn[4 * k4], hn[4 * k4 + 1], hn[4 * k4 + 2], hn[4 * k4 + 3]);
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if (k < Px) hvl[j * LD + (Px - 1 - k)] = hn[k];
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
                __syncthreads();  // every read of xs done
                float4 *xd = reinterpret_cast<float4 *>(xs + j * LD);
#pragma unroll
                for (int k4 = 0; k4 < R / 4; ++k4)
                    xd[k4] = make_float4(gelu_f(y[4 * k4]), gelu_f(y[4 * k4 + 1]), gelu_f(y[4 * k4 + 2]),
                                         gelu_f(y[4 * k4 + 3]));
#pragma unroll
                for (int k = 0; k < R; ++k) hl[k] = hn[k];
                __syncthreads();
            }
            // ---------------- readout: 16 logits per patch, masked softmax
            {
                constexpr int G16 = H / 16;  // site groups
                const int o = j & 15, g = j >> 4;
                const float bo = Wo[16 * H + o];
                for (int k = g; k < Px; k += G16) {
                    float v = bo;
                    for (int m = 0; m < H; ++m) v += Wo[o * H + m] * xs[m * LD + k];
                    lg[o * LD + k] = v;
                }
            }
            __syncthreads();
            if (j < 32) {
                float d = 0.0f;
                const int k = j;
                if (k < Px) {
                    int up_before = n_up, down_before = n_down;
                    for (int kk = 0; kk < k; ++kk) {
                        const int pc = __popc(s_v[kk]);
                        up_before += pc;
                        down_before += 4 - pc;
                    }
                    // zero magnetisation: value u is allowed while neither count
                    // passes N/2 after it
                    auto allowed = [&](int u) {
                        const int pc = __popc(u);
                        return !G.u1 || (up_before + pc <= N / 2 && down_before + 4 - pc <= N / 2);
                    };
                    float mx = -INFINITY;
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        if (allowed(u)) mx = fmaxf(mx, lg[u * LD + k]);
                    float ssum = 0.0f;
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        if (allowed(u)) ssum += expf(lg[u * LD + k] - mx);
                    const int v = s_v[k];
                    const float lp = allowed(v) ? lg[v * LD + k] - mx - logf(ssum) : -INFINITY;
                    const int t = pj * Px + k;
                    if (G.logp_out) G.logp_out[(size_t)sample * Np + t] = lp;
                    d = (jb.mode == 1) ? lp - G.logp_ref[(size_t)sample * Np + t] : lp;
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
                if (j == 0) s_part[0] = d;
            }
            __syncthreads();
            acc += s_part[0];
            {
                int row_up = 0;
                for (int k = 0; k < Px; ++k) row_up += __popc(s_v[k]);
                n_up += row_up;
                n_down += 4 * Px - row_up;
            }
            if (j < Px) s_vprev[(pj & 1) ? Px - 1 - j : j] = s_v[j];
            __syncthreads();
        }
        if (j == 0) G.out[job] = 0.5f * acc;
    }
}

template <int H, int R>
cudaError_t launch_fwd2d_hr(const Fwd2Jobs &jobs, const float *packed, const F2Layout &f, int num_sms,
                            cudaStream_t stream) {
    constexpr int LD = R + 4;
    const size_t smem = ((size_t)(2 + f.nL) * H * LD + 16 * LD) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(fwd2d_f32_kernel<H, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fwd2d_f32_kernel<H, R>, H, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (jobs.g.n_jobs < grid) grid = jobs.g.n_jobs;
    if (grid < 1) grid = 1;
    fwd2d_f32_kernel<H, R><<<(int)grid, H, smem, stream>>>(jobs, packed, f);
    return cudaGetLastError();
}

template <int H>
cudaError_t launch_fwd2d_h(const Fwd2Jobs &jobs, const float *packed, const F2Layout &f, int num_sms,
                           cudaStream_t stream) {
    switch (row2d_width(jobs.g.Lx)) {
        case 8: return launch_fwd2d_hr<H, 8>(jobs, packed, f, num_sms, stream);
        case 12: return launch_fwd2d_hr<H, 12>(jobs, packed, f, num_sms, stream);
        case 16: return launch_fwd2d_hr<H, 16>(jobs, packed, f, num_sms, stream);
        case 24: return launch_fwd2d_hr<H, 24>(jobs, packed, f, num_sms, stream);
        case 28: return launch_fwd2d_hr<H, 28>(jobs, packed, f, num_sms, stream);
        default: return launch_fwd2d_hr<H, 32>(jobs, packed, f, num_sms, stream);
    }
}

}  // namespace

cudaError_t launch_pack_theta_f2(const float *theta, const F2Layout &f, float *packed,
                                 cudaStream_t stream) {
    pack_f2_kernel<<<64, 256, 0, stream>>>(theta, f, packed);
    return cudaGetLastError();
}

int row2d_width(int Lx) {
    const int Px = Lx / 2;
    for (int r : {8, 12, 16, 24, 28})
        if (Px <= r) return r;
    return 32;
}

size_t fwd2d_checkpoint_floats(int nL, int H, int Lx) { return (size_t)nL * H * (row2d_width(Lx) + 4); }

cudaError_t launch_fwd2d_f32(const Fwd2Jobs &jobs, const float *packed, const F2Layout &f,
                             int num_sms, cudaStream_t stream) {
    switch (f.H) {
        case 32: return launch_fwd2d_h<32>(jobs, packed, f, num_sms, stream);
        case 64: return launch_fwd2d_h<64>(jobs, packed, f, num_sms, stream);
        case 128: return launch_fwd2d_h<128>(jobs, packed, f, num_sms, stream);
        case 256: return launch_fwd2d_h<256>(jobs, packed, f, num_sms, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace psr
