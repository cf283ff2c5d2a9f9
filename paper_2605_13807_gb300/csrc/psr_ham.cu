// Lattice Hamiltonians on the device: bond list, connected-configuration
// generator (count -> exclusive scan -> emit, bit-exact and deterministic),
// the local-energy gather and the FP64 energy statistics.
//
// Heisenberg (Sec. III.C): H = J sum S_p.S_q with S = sigma/2, so the
// diagonal is (J/4) sum sigma_p sigma_q and every antiparallel bond connects
// to the configuration with both spins exchanged (element J/2, times -1
// under the Marshall sign).  TFIM (Sec. III.B): diagonal -J sum sigma sigma,
// every single-site flip connected with element -h.  The local energy sums
// element * psi(s')/psi(s) over the connected set (Sec. II.A).
#include <cuda_runtime.h>

#include "psr_device.cuh"
#include "psr_internal.cuh"

namespace psr {

static inline void wraps(int Lx, int Ly, int pbc, int &wx, int &wy) {
    wx = (pbc && Lx >= 3) ? 1 : 0;
    wy = (pbc && Ly >= 3) ? 1 : 0;
}

int bond_count(int Lx, int Ly, int pbc) {
    int wx, wy;
    wraps(Lx, Ly, pbc, wx, wy);
    const int rx = Lx - 1 + wx;
    return Ly * rx + Lx * (Ly - 1 + wy);
}

__device__ __forceinline__ int zigzag(int Lx, int i, int j) {
    return j * Lx + ((j & 1) ? (Lx - 1 - i) : i);
}

// One thread per lattice site; the position of a site's bonds in the
// canonical order (row-major sites, right then down) is a closed form:
// every earlier row holds rx right bonds and Lx down bonds, and every earlier
// site of the same row holds one right bond and (hasD) one down bond.
__global__ void bonds_kernel(int Lx, int Ly, int wx, int wy, int32_t *bonds) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Lx * Ly) return;
    const int i = r % Lx, j = r / Lx;
    const int rx = Lx - 1 + wx;
    const int hasR = (i < Lx - 1) || wx;
    const int hasD = (j < Ly - 1) || wy;
    int pos = j * (rx + Lx) + i * (1 + hasD);
    const int here = zigzag(Lx, i, j);
    if (hasR) {
        const int o = zigzag(Lx, (i + 1) % Lx, j);
        bonds[2 * pos] = min(here, o);
        bonds[2 * pos + 1] = max(here, o);
        ++pos;
    }
    if (hasD) {
        const int o = zigzag(Lx, i, (j + 1) % Ly);
        bonds[2 * pos] = min(here, o);
        bonds[2 * pos + 1] = max(here, o);
    }
}

cudaError_t launch_bonds(int Lx, int Ly, int pbc, int32_t *bonds, cudaStream_t stream) {
    int wx, wy;
    wraps(Lx, Ly, pbc, wx, wy);
    const int n = Lx * Ly;
    bonds_kernel<<<(n + 255) / 256, 256, 0, stream>>>(Lx, Ly, wx, wy, bonds);
    return cudaGetLastError();
}

// One warp per sample: number of connected entries and diagonal energy.
__global__ void count_connected_kernel(HamDev hd, const uint8_t *__restrict__ spins, int64_t n,
                                       int64_t *__restrict__ counts, float *__restrict__ diag) {
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= n) return;
    const uint8_t *x = spins + s * hd.N;
    int zz = 0, anti = 0;
    for (int b = lane; b < hd.nb; b += 32) {
        const int sp = x[hd.bonds[2 * b]] & 1, sq = x[hd.bonds[2 * b + 1]] & 1;
        const int d = sp ^ sq;
        anti += d;
        zz += 1 - 2 * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        zz += __shfl_xor_sync(0xffffffffu, zz, o);
        anti += __shfl_xor_sync(0xffffffffu, anti, o);
    }
    if (lane == 0) {
        if (hd.kind == PSR_HEISENBERG) {
            counts[s] = anti;
            diag[s] = 0.25f * hd.J * (float)zz;
        } else {
            counts[s] = hd.N;
            diag[s] = -hd.J * (float)zz;
        }
    }
}

cudaError_t launch_count_connected(const HamDev &hd, const uint8_t *spins, int64_t n,
                                   int64_t *counts, float *diag, cudaStream_t stream) {
    const int64_t threads = n * 32;
    const int blocks = (int)((threads + 255) / 256);
    count_connected_kernel<<<blocks, 256, 0, stream>>>(hd, spins, n, counts, diag);
    return cudaGetLastError();
}

// Exclusive scan of n int64 counts into offsets[0..n] by one CTA: each
// thread sums a contiguous segment, the segment sums are scanned in shared
// memory, then each thread writes its segment.  Deterministic.
__global__ void __launch_bounds__(1024) scan_kernel(const int64_t *__restrict__ counts, int64_t n,
                                                    int64_t *__restrict__ offsets) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t seg = (n + 1023) / 1024;
    const int64_t lo = min(n, t * seg), hi = min(n, lo + seg);
    int64_t sum = 0;
    for (int64_t i = lo; i < hi; ++i) sum += counts[i];
    part[t] = sum;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        int64_t v = (t >= d) ? part[t - d] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - sum;  // exclusive prefix of this segment
    for (int64_t i = lo; i < hi; ++i) {
        offsets[i] = run;
        run += counts[i];
    }
    if (t == 1023) offsets[n] = part[1023];
}

cudaError_t launch_exclusive_scan(const int64_t *counts, int64_t n, int64_t *offsets,
                                  cudaStream_t stream) {
    scan_kernel<<<1, 1024, 0, stream>>>(counts, n, offsets);
    return cudaGetLastError();
}

// One warp per sample: emits (sample, p, q) in canonical bond order using a
// ballot per group of 32 bonds (no atomics; bit-exact).
__global__ void fill_connected_kernel(HamDev hd, const uint8_t *__restrict__ spins, int64_t n,
                                      const int64_t *__restrict__ offsets,
                                      int32_t *__restrict__ entries) {
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= n) return;
    int64_t base = offsets[s];
    if (hd.kind == PSR_TFIM) {
        for (int i = lane; i < hd.N; i += 32) {
            int32_t *e = entries + 3 * (base + i);
            e[0] = (int32_t)s;
            e[1] = i;
            e[2] = -1;
        }
        return;
    }
    const uint8_t *x = spins + s * hd.N;
    for (int b0 = 0; b0 < hd.nb; b0 += 32) {
        const int b = b0 + lane;
        int p = 0, q = 0, anti = 0;
        if (b < hd.nb) {
            p = hd.bonds[2 * b];
            q = hd.bonds[2 * b + 1];
            anti = (x[p] ^ x[q]) & 1;
        }
        const unsigned m = __ballot_sync(0xffffffffu, anti);
        if (anti) {
            const int64_t at = base + __popc(m & ((1u << lane) - 1u));
            int32_t *e = entries + 3 * at;
            e[0] = (int32_t)s;
            e[1] = p;
            e[2] = q;
        }
        base += __popc(m);
    }
}

cudaError_t launch_fill_connected(const HamDev &hd, const uint8_t *spins, int64_t n,
                                  const int64_t *offsets, int32_t *entries, cudaStream_t stream) {
    const int64_t threads = n * 32;
    const int blocks = (int)((threads + 255) / 256);
    fill_connected_kernel<<<blocks, 256, 0, stream>>>(hd, spins, n, offsets, entries);
    return cudaGetLastError();
}

// One warp per sample: E_loc = diag + coeff * sum_e exp(delta_e).
__global__ void eloc_gather_kernel(const int64_t *__restrict__ offsets,
                                   const float *__restrict__ delta, const float *__restrict__ diag,
                                   float coeff, int64_t n, float *__restrict__ eloc) {
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= n) return;
    float acc = 0.0f;
    for (int64_t e = offsets[s] + lane; e < offsets[s + 1]; e += 32) acc += expf(delta[e]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) eloc[s] = diag[s] + coeff * acc;
}

cudaError_t launch_eloc_gather(const int64_t *offsets, const float *delta, const float *diag,
                               float coeff, int64_t n, float *eloc, cudaStream_t stream) {
    const int64_t threads = n * 32;
    const int blocks = (int)((threads + 255) / 256);
    eloc_gather_kernel<<<blocks, 256, 0, stream>>>(offsets, delta, diag, coeff, n, eloc);
    return cudaGetLastError();
}

// FP64 mean, unbiased variance and standard error of n values (one CTA,
// fixed reduction order).
__global__ void __launch_bounds__(1024) stats_kernel(const float *__restrict__ e, int64_t n,
                                                     double *__restrict__ out) {
    __shared__ double red[1024];
    const int t = threadIdx.x;
    double s = 0.0;
    for (int64_t i = t; i < n; i += 1024) s += (double)e[i];
    red[t] = s;
    __syncthreads();
    for (int d = 512; d > 0; d >>= 1) {
        if (t < d) red[t] += red[t + d];
        __syncthreads();
    }
    const double mean = red[0] / (double)n;
    __syncthreads();
    double v = 0.0;
    for (int64_t i = t; i < n; i += 1024) {
        const double d = (double)e[i] - mean;
        v += d * d;
    }
    red[t] = v;
    __syncthreads();
    for (int d = 512; d > 0; d >>= 1) {
        if (t < d) red[t] += red[t + d];
        __syncthreads();
    }
    if (t == 0) {
        const double var = (n > 1) ? red[0] / (double)(n - 1) : 0.0;
        out[0] = mean;
        out[1] = var;
        out[2] = sqrt(var / (double)n);
    }
}

cudaError_t launch_stats(const float *eloc, int64_t n, double *stats, cudaStream_t stream) {
    stats_kernel<<<1, 1024, 0, stream>>>(eloc, n, stats);
    return cudaGetLastError();
}

}  // namespace psr
