// c4v symmetrisation and the pieces of one VMC step that are not a forward
// or a backward: symmetry images of configurations and of connected-entry
// flips, the log-sum-exp combinations of the 8 images, the centred
// energy-gradient weights and the Adam update.
//
// c4v acts on an L x L lattice by its 8 operations g (identity, rotations by
// 90, 180, 270 degrees, reflections in x, in y, in the diagonal and in the
// anti-diagonal); image g of a configuration has (g s)(g(x)) = s(x).  The
// symmetrised amplitude of a positive wave function is
// psi_sym(s) = sqrt(1/8 sum_g psi(g s)^2) (the symmetry the paper imposes on
// its 2D runs, Sec. III.C, in the form of the RNN wave-function work it
// cites).  A connected configuration s' of s (sites p, q flipped) has the
// images g s' = g s with sites g(p), g(q) flipped, so every image of every
// connected configuration is itself a connected entry of an image sample
// and resumes from that image's stored chunk carries.
#include <cuda_runtime.h>
#include <math.h>

#include "psr_device.cuh"
#include "psr_internal.cuh"

namespace psr {

namespace {

__device__ __forceinline__ void seq_coords(int L, int pos, int &i, int &j) {
    j = pos / L;
    const int k = pos - j * L;
    i = (j & 1) ? L - 1 - k : k;
}

__device__ __forceinline__ int seq_pos_sq(int L, int i, int j) {
    return j * L + ((j & 1) ? L - 1 - i : i);
}

// position of g(x) for the site at sequence position pos
__device__ __forceinline__ int c4v_apply(int g, int L, int pos) {
    int i, j;
    seq_coords(L, pos, i, j);
    int a = i, b = j;
    switch (g) {
        case 1: a = L - 1 - j; b = i; break;          // rotation by 90 degrees
        case 2: a = L - 1 - i; b = L - 1 - j; break;  // rotation by 180 degrees
        case 3: a = j; b = L - 1 - i; break;          // rotation by 270 degrees
        case 4: a = L - 1 - i; b = j; break;          // reflection in x
        case 5: a = i; b = L - 1 - j; break;          // reflection in y
        case 6: a = j; b = i; break;                  // reflection in the diagonal
        case 7: a = L - 1 - j; b = L - 1 - i; break;  // reflection in the anti-diagonal
        default: break;                               // identity
    }
    return seq_pos_sq(L, a, b);
}

// out[g][i][g(x)] = s[i][x] for all 8 g (one thread per (i, x), 8 writes)
__global__ void c4v_images_kernel(const uint8_t *__restrict__ s, int64_t n, int L,
                                  uint8_t *__restrict__ out) {
    const int N = L * L;
    const int64_t total = n * N;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / N;
        const int x = (int)(k - i * N);
        const uint8_t v = s[k];
#pragma unroll
        for (int g = 0; g < 8; ++g) out[((int64_t)g * n + i) * N + c4v_apply(g, L, x)] = v;
    }
}

// out[i][x] = image g_i of sample i, g_i = min(7, floor(8 u_i))
__global__ void c4v_pick_kernel(const uint8_t *__restrict__ s, const float *__restrict__ u, int64_t n,
                                int L, uint8_t *__restrict__ out) {
    const int N = L * L;
    const int64_t total = n * N;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / N;
        const int x = (int)(k - i * N);
        const int g = min(7, max(0, (int)floorf(8.0f * u[i])));
        out[i * N + c4v_apply(g, L, x)] = s[k];
    }
}

// entries of image g: (sample, min(g p, g q), max(...)) with q = -1 kept
__global__ void c4v_entries_kernel(const int32_t *__restrict__ entries, const int64_t *__restrict__ count,
                                   int64_t cap, int L, int32_t *__restrict__ out) {
    const int64_t E = *count;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t smp = entries[3 * e], p = entries[3 * e + 1], q = entries[3 * e + 2];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const int gp = c4v_apply(g, L, p);
            const int gq = q >= 0 ? c4v_apply(g, L, q) : -1;
            int32_t *o = out + ((int64_t)g * cap + e) * 3;
            o[0] = smp;
            o[1] = (gq >= 0 && gq < gp) ? gq : gp;
            o[2] = (gq >= 0 && gq < gp) ? gp : gq;
        }
    }
}

__device__ __forceinline__ float lse8(const float (&x)[8]) {
    float m = x[0];
#pragma unroll
    for (int g = 1; g < 8; ++g) m = fmaxf(m, x[g]);
    if (m == -INFINITY) return -INFINITY;
    float s = 0.0f;
#pragma unroll
    for (int g = 0; g < 8; ++g) s += expf(x[g] - m);
    return m + logf(s);
}

// log psi_sym(s_i) = 1/2 (LSE_g 2 lp[g][i] - log 8)
__global__ void sym_logpsi_kernel(const float *__restrict__ lp8, int64_t n, float *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float x[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) x[g] = 2.0f * lp8[(int64_t)g * n + i];
        out[i] = 0.5f * (lse8(x) - 2.0794415416798357f);
    }
}

// log(psi_sym(s'_e) / psi_sym(s)) from the images' log psi and differences
__global__ void sym_delta_kernel(const int32_t *__restrict__ entries, const int64_t *__restrict__ count,
                                 int64_t cap, const float *__restrict__ lp8, int64_t n,
                                 const float *__restrict__ delta8, float *__restrict__ out) {
    const int64_t E = *count;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = entries[3 * e];
        float a[8], b[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            a[g] = 2.0f * lp8[(int64_t)g * n + i];
            b[g] = a[g] + 2.0f * delta8[(int64_t)g * cap + e];
        }
        out[e] = 0.5f * (lse8(b) - lse8(a));
    }
}

// dout[g][i] = 2/n (E_i - mean) w_g(i), w = softmax_g(2 lp8[g][i]); the
// plain (unsymmetrised) case is the single image g = 0 with w = 1.
__global__ void vmc_dout_kernel(const float *__restrict__ eloc, const double *__restrict__ stats,
                                const float *__restrict__ lp8, int64_t n, int n_img,
                                float *__restrict__ dout) {
    const double mean = stats[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float c = (float)(2.0 * ((double)eloc[i] - mean) / (double)n);
        if (n_img == 1) {
            dout[i] = c;
            continue;
        }
        float x[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) x[g] = 2.0f * lp8[(int64_t)g * n + i];
        const float z = lse8(x);
#pragma unroll
        for (int g = 0; g < 8; ++g) dout[(int64_t)g * n + i] = c * expf(x[g] - z);
    }
}

// Adam (Kingma and Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// theta_out = theta - lr m^ / (sqrt(v^) + eps), m^ = m/(1-b1^t), v^ = v/(1-b2^t)
__global__ void adam_kernel(const float *__restrict__ theta, const float *__restrict__ grad, int64_t P,
                            float lr, float b1, float b2, float eps, float c1, float c2,
                            float *__restrict__ m, float *__restrict__ v, float *__restrict__ out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < P;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float g = grad[k];
        const float mk = b1 * m[k] + (1.0f - b1) * g;
        const float vk = b2 * v[k] + (1.0f - b2) * g * g;
        m[k] = mk;
        v[k] = vk;
        out[k] = theta[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

int blocks_for(int64_t work) {
    int64_t b = (work + 255) / 256;
    if (b > 4096) b = 4096;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_c4v_images(const uint8_t *s, int64_t n, int L, uint8_t *out, cudaStream_t st) {
    c4v_images_kernel<<<blocks_for(n * L * L), 256, 0, st>>>(s, n, L, out);
    return cudaGetLastError();
}

cudaError_t launch_c4v_pick(const uint8_t *s, const float *u, int64_t n, int L, uint8_t *out,
                            cudaStream_t st) {
    c4v_pick_kernel<<<blocks_for(n * L * L), 256, 0, st>>>(s, u, n, L, out);
    return cudaGetLastError();
}

cudaError_t launch_c4v_entries(const int32_t *entries, const int64_t *count, int64_t cap, int L,
                               int32_t *out, cudaStream_t st) {
    c4v_entries_kernel<<<blocks_for(cap), 256, 0, st>>>(entries, count, cap, L, out);
    return cudaGetLastError();
}

cudaError_t launch_sym_logpsi(const float *lp8, int64_t n, float *out, cudaStream_t st) {
    sym_logpsi_kernel<<<blocks_for(n), 256, 0, st>>>(lp8, n, out);
    return cudaGetLastError();
}

cudaError_t launch_sym_delta(const int32_t *entries, const int64_t *count, int64_t cap,
                             const float *lp8, int64_t n, const float *delta8, float *out,
                             cudaStream_t st) {
    sym_delta_kernel<<<blocks_for(cap), 256, 0, st>>>(entries, count, cap, lp8, n, delta8, out);
    return cudaGetLastError();
}

cudaError_t launch_vmc_dout(const float *eloc, const double *stats, const float *lp8, int64_t n,
                            int n_img, float *dout, cudaStream_t st) {
    vmc_dout_kernel<<<blocks_for(n), 256, 0, st>>>(eloc, stats, lp8, n, n_img, dout);
    return cudaGetLastError();
}

cudaError_t launch_adam(const float *theta, const float *grad, int64_t P, float lr, float b1, float b2,
                        float eps, int step, float *m, float *v, float *out, cudaStream_t st) {
    const float c1 = (float)(1.0 - pow((double)b1, (double)step));
    const float c2 = (float)(1.0 - pow((double)b2, (double)step));
    adam_kernel<<<blocks_for(P), 256, 0, st>>>(theta, grad, P, lr, b1, b2, eps, c1, c2, m, v, out);
    return cudaGetLastError();
}

}  // namespace psr
