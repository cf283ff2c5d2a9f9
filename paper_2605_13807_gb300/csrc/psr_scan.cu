// Standalone chunked scan of the diagonal linear recurrence
//     h_t = a_t * h_{t-1} + b_t   (element-wise over H units)
// over many sequences held in HBM: the parallel-scan form of the minGRU
// recurrence (Sec. II.A, parallel-scan paragraph; Eq. minGRU with
// a_t = 1 - z_t, b_t = z_t h~_t).
//
// Layout: a, b, h are FP32 [n][N][H] (H contiguous), h0 is [n][H] or absent
// (zero).  A tile is (sequence, block of U = 4Q units, chunk of C sites).
// One warp owns a tile; lane (s, q) = (lane / Q, lane % Q) holds the float4
// of units 4q..4q+3 of site s of each S = 32 / Q site step, so every load and
// store is a coalesced 16-byte access (a step covers S rows of 16Q bytes).
//
// Inside a chunk each step is an inclusive warp-shuffle scan over its S sites
// of the affine maps h -> a h + b (composition (A2, B2) o (A1, B1) =
// (A2 A1, A2 B1 + B2)), applied to the running carry that the last site lane
// of the previous step broadcasts.  Between chunks of one column the carry
// travels through a look-back descriptor array in global memory: a chunk
// first publishes the aggregate map of its sites (flag 1), then walks back
// over its predecessors, composing aggregates until it finds one that has
// published its inclusive end value (flag 2), publishes its own inclusive
// value and rescans its chunk (now an L2 hit) with the carry, storing h.
// Chunk 0 of a column needs no look-back and makes a single pass.  Tiles are
// handed out by an atomic ticket with the chunk index fastest, so a warp only
// ever waits on tiles owned by warps that are already running.  Every wait is
// bounded (2 s of %globaltimer); an expiry records PSR_ETIMEOUT and the warp
// carries on with a zero carry so that nothing downstream waits again.
#include <cuda_runtime.h>

#include "psr_device.cuh"
#include "psr_internal.cuh"

namespace psr {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanUnroll = 4;  // site steps loaded ahead of the scan
constexpr unsigned long long kScanWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long scan_clock() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ float4 f4(float x) { return make_float4(x, x, x, x); }

__device__ __forceinline__ float4 fma4(float4 a, float4 x, float4 b) {
    return make_float4(fmaf(a.x, x.x, b.x), fmaf(a.y, x.y, b.y), fmaf(a.z, x.z, b.z),
                       fmaf(a.w, x.w, b.w));
}

__device__ __forceinline__ float4 mul4(float4 a, float4 b) {
    return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}

__device__ __forceinline__ float4 shfl_up4(float4 v, int d) {
    return make_float4(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d),
                       __shfl_up_sync(0xffffffffu, v.z, d), __shfl_up_sync(0xffffffffu, v.w, d));
}

__device__ __forceinline__ float4 shfl4(float4 v, int src) {
    return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                       __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}

// Waits (bounded) until *flag != 0 and returns it; 0 after a timeout, or at
// once when another wait of this launch has already timed out.
__device__ int wait_flag(const int *flag, int *status) {
    int v = ld_acquire_gpu(flag);
    if (v) return v;
    const unsigned long long t0 = scan_clock();
    for (unsigned it = 1;; ++it) {
        __nanosleep(64);
        v = ld_acquire_gpu(flag);
        if (v) return v;
        if ((it & 31u) == 0) {
            if (*(volatile int *)status == PSR_ETIMEOUT) return 0;
            if (scan_clock() - t0 > kScanWaitNs || it > (1u << 28)) {
                set_status(status, PSR_ETIMEOUT);
                return 0;
            }
        }
    }
}

// Scans sites [t_begin, t_end) of one tile, starting from the running map
// (runA, runB): h = runA * h_before + runB.  kStore: write h_t = B of the
// composed map (runA is then 0 and not tracked) and stream it out; otherwise
// only compose, so that (runA, runB) ends as the aggregate map of the range.
template <int Q, bool kStore>
__device__ __forceinline__ void scan_sites(const float4 *__restrict__ a4, const float4 *__restrict__ b4,
                                           float4 *__restrict__ h4, long long base4, int H4,
                                           int t_begin, int t_end, int s, int q, float4 &runA,
                                           float4 &runB) {
    constexpr int S = 32 / Q;
    const int last = (S - 1) * Q + q;
    for (int t0 = t_begin; t0 < t_end; t0 += S * kScanUnroll) {
        float4 av[kScanUnroll], bv[kScanUnroll];
#pragma unroll
        for (int k = 0; k < kScanUnroll; ++k) {
            const int t = t0 + k * S + s;
            if (t < t_end) {
                const long long i = base4 + (long long)t * H4;
                av[k] = __ldg(a4 + i);
                bv[k] = __ldg(b4 + i);
            } else {
                av[k] = f4(1.0f);  // identity map past the end
                bv[k] = f4(0.0f);
            }
        }
#pragma unroll
        for (int k = 0; k < kScanUnroll; ++k) {
            float4 A = av[k], B = bv[k];
#pragma unroll
            for (int off = 1; off < S; off <<= 1) {
                const float4 Au = shfl_up4(A, off * Q);
                const float4 Bu = shfl_up4(B, off * Q);
                if (s >= off) {
                    B = fma4(A, Bu, B);
                    A = mul4(A, Au);
                }
            }
            const float4 hB = fma4(A, runB, B);
            if (kStore) {
                const int t = t0 + k * S + s;
                if (t < t_end) __stcs(h4 + base4 + (long long)t * H4, hB);
                runB = shfl4(hB, last);
            } else {
                const float4 hA = mul4(A, runA);
                runA = shfl4(hA, last);
                runB = shfl4(hB, last);
            }
        }
    }
}

template <int Q>
__global__ void __launch_bounds__(kScanThreads) scan_kernel(const __grid_constant__ ScanArgs g) {
    const int lane = threadIdx.x & 31;
    const int q = lane % Q, s = lane / Q;
    const int H4 = g.H >> 2;
    const float4 *a4 = reinterpret_cast<const float4 *>(g.a);
    const float4 *b4 = reinterpret_cast<const float4 *>(g.b);
    const float4 *h04 = reinterpret_cast<const float4 *>(g.h0);
    float4 *h4 = reinterpret_cast<float4 *>(g.h);
    float4 *d4 = reinterpret_cast<float4 *>(g.desc);  // [tile][3][Q] float4: A, B, inclusive

    for (;;) {
        unsigned long long tile = 0;
        if (lane == 0) tile = atomicAdd(g.counter, 1ull);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= (unsigned long long)g.n_tiles) break;
        const long long col = (long long)(tile / (unsigned long long)g.nch);
        const int c = (int)((long long)tile - col * g.nch);
        const long long seq = col / g.nub;
        const int ub = (int)(col - seq * g.nub);
        const int t_begin = c * g.C;
        const int t_end = min(g.N, t_begin + g.C);
        const long long base4 = seq * (long long)g.N * H4 + (long long)ub * Q + q;

        float4 carry = f4(0.0f);
        if (c == 0) {
            if (h04) carry = __ldg(h04 + seq * H4 + (long long)ub * Q + q);
        } else {
            float4 A = f4(1.0f), B = f4(0.0f);
            scan_sites<Q, false>(a4, b4, h4, base4, H4, t_begin, t_end, s, q, A, B);
            const long long me = (long long)tile;
            if (s == 0) {
                d4[(me * 3 + 0) * Q + q] = A;
                d4[(me * 3 + 1) * Q + q] = B;
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release_gpu(g.flags + me, 1);
            // look back over the chunks of this column
            float4 accA = f4(1.0f), accB = f4(0.0f);
            for (long long k = me - 1;; --k) {
                const int f = wait_flag(g.flags + k, g.status);
                if (f == 0) {
                    accA = f4(0.0f);
                    accB = f4(0.0f);
                    break;
                }
                if (f == 2) {
                    accB = fma4(accA, d4[(k * 3 + 2) * Q + q], accB);
                    break;
                }
                accB = fma4(accA, d4[(k * 3 + 1) * Q + q], accB);
                accA = mul4(accA, d4[(k * 3 + 0) * Q + q]);
            }
            carry = accB;
            __syncwarp();
            if (s == 0) d4[(me * 3 + 2) * Q + q] = fma4(A, carry, B);
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release_gpu(g.flags + me, 2);
        }
        float4 runA = f4(0.0f), runB = carry;
        scan_sites<Q, true>(a4, b4, h4, base4, H4, t_begin, t_end, s, q, runA, runB);
        if (c == 0 && g.nch > 1) {
            const long long me = (long long)tile;
            if (s == 0) d4[(me * 3 + 2) * Q + q] = runB;
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release_gpu(g.flags + me, 2);
        }
    }
}

template <int Q>
cudaError_t launch_scan_q(const ScanArgs &g, int num_sms, cudaStream_t stream) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_kernel<Q>,
                                                                  kScanThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int warps = kScanThreads / 32;
    long long grid = (long long)num_sms * per_sm;
    const long long need = (g.n_tiles + warps - 1) / warps;
    if (need < grid) grid = need;
    if (grid < 1) grid = 1;
    scan_kernel<Q><<<(int)grid, kScanThreads, 0, stream>>>(g);
    return cudaGetLastError();
}

}  // namespace

bool scan_tile_valid(int H, int units, int chunk) {
    if (units != 4 && units != 16 && units != 32 && units != 128) return false;
    if (H % units != 0) return false;
    return chunk >= 1;
}

void scan_geometry(int64_t n, int N, int H, int units, int chunk, int *nch, int64_t *n_tiles) {
    const int c = chunk >= N ? N : chunk;
    *nch = (N + c - 1) / c;
    *n_tiles = n * (int64_t)(H / units) * (*nch);
}

cudaError_t launch_scan(const ScanArgs &g, int units, int num_sms, cudaStream_t stream) {
    switch (units) {
        case 4: return launch_scan_q<1>(g, num_sms, stream);
        case 16: return launch_scan_q<4>(g, num_sms, stream);
        case 32: return launch_scan_q<8>(g, num_sms, stream);
        case 128: return launch_scan_q<32>(g, num_sms, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace psr
