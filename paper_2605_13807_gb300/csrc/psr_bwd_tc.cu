// Reverse-mode gradient on the tensor cores (hidden 128): per-sample
// O_k = d log psi / d theta of the minGRU chain (derivative of Eq. minGRU
// and of the output map, Sec. II.F-G; the energy-gradient estimates of
// Sec. III.B use these rows), computed layer by layer over whole samples.
//
// The FP32 forward stores, for every sample, layer l and site t, the gate a,
// the candidate c = W_h u + b_h, the state h and the output-map
// pre-activation y (unit-major [unit][site], sites padded to a multiple of
// 64 with zeros), and the readout adjoint g_t = 1/2 (s_t - P(1 | s_<t)).
// Then, from the top layer down:
//   gy  = gx (.) GELU'(y)                 gx = g wd at the top layer
//   g_h = C^T gy (+ gy of layer l+1, the residual s^{l+1} = h^l, l+1 >= 2)
//   lambda_t = g_h,t + a_{t+1} lambda_{t+1}          (reverse scan, FP32)
//   dz = lambda (h_{t-1} - c) a (1 - a),  dc = lambda (1 - a)
//   gx  = W_z^T dz + W_h^T dc + D^T gy               (input of layer l-1)
//   dC = sum_t gy h^T,  dD = sum_t gy u^T,  dW_z = sum_t dz u^T,
//   dW_h = sum_t dc u^T  (u = GELU(y of layer l-1)),  biases: sums
// Layer 0's input is one-hot, so its W_z, W_h, D gradients are sums of dz,
// dc, gy over the sites of each input code.
//
// Every product runs as tcgen05 MMAs on BF16 operands with FP32
// accumulation, each operand split into a high and a low BF16 part
// (x = hi + lo; hi.hi + hi.lo + lo.hi), which keeps about 16 mantissa bits:
// single BF16 operands leave a relative gradient error near 2e-3, above the
// 1e-3 bound; split operands about 5e-6.  Scans, derivatives and sums stay
// FP32.
//
// Kernels (one launch each per layer, samples of a batch):
//   gy_gh_kernel  feature-major MMAs D[unit][site] = C^T . gy, four
//                 warpgroup streams per SM, C^T images in TMEM;
//   scan_bwd_kernel  one CTA per sample, thread j = unit j walks the sites
//                 backwards in steps of 8 (32-byte loads), writes dz, dc and
//                 the bias / one-hot / readout rows of O_k;
//   gx_kernel     feature-major MMAs of W_z^T, W_h^T, D^T (images in TMEM),
//                 two streams per SM;
//   wgrad_kernel  per sample D[j][k] = sum_t A[j][t] B[k][t], both operands
//                 K-major over sites, four 128 x 128 accumulators in TMEM.
// Every mbarrier wait is bounded (PSR_ETIMEOUT in the status word).
#include <cstddef>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "psr_device.cuh"
#include "psr_internal.cuh"
#include "psr_tc.cuh"

namespace psr {

namespace {

using namespace tc;

constexpr int H = 128;
constexpr int TS = 64;                      // sites per tile (one 128-byte swizzle row)
constexpr uint32_t kTile = 128 * TS * 2;    // [128 rows][64 sites] bf16 = 16 KB
constexpr uint32_t kImg = 32768;            // 128 x 128 bf16 image
constexpr int kImgPerLayer = 16;            // C, W_z, W_h, D transposed (backward), then as
                                            // stored (forward), each hi and lo
constexpr int kImgPlain = 8;                // first plain image of a layer
enum { IM_C = 0, IM_WZ = 1, IM_WH = 2, IM_D = 3 };

// kind::f16, D = F32, A = B = BF16, M = 128.
// Feature-major: A K-major (TMEM), B MN-major (sites contiguous), N = 64.
constexpr uint32_t kIdescFM = (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (1u << 16) |
                              ((uint32_t)(TS >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
// Weight gradient: A and B K-major (sites contiguous), N = 128.
constexpr uint32_t kIdescWG = (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (0u << 16) |
                              ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

// 128-byte-swizzled tile descriptors.  A tile holds 128 rows of 64 BF16
// (128 bytes per row, 8-row atoms of 1024 bytes).  As an MN-major B operand
// (rows = K) the 64 sites are one atom wide, so only the K stride (1024) is
// used; as a K-major operand (rows = M or N) the row-group stride is 1024.
__device__ __forceinline__ uint64_t tdesc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(1024u >> 4) << 16) |
           ((uint64_t)(1024u >> 4) << 32) | (1ull << 46) | (2ull << 61);
}
// K = 16 slice kk of a feature-major B tile: 16 rows further (2048 bytes)
__device__ __forceinline__ uint64_t fm_boff(int kk) { return (uint64_t)((kk * 2048) >> 4); }
// K = 16 slice kk (0..3) of a K-major tile: 32 bytes further along the row
__device__ __forceinline__ uint64_t km_off(int kk) { return (uint64_t)((kk * 32) >> 4); }

// Row r of a tile from 64 FP32 values: the high BF16 parts into `hi`, the
// low parts (v - hi) into `lo`; 16-byte chunk c at position c ^ (r & 7).
__device__ __forceinline__ void store_row_split(uint8_t *hi, uint8_t *lo, int r, const float (&v)[TS]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint32_t wh[4], wl[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float x0 = v[8 * c + 2 * i], x1 = v[8 * c + 2 * i + 1];
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
            const float2 hf = __bfloat1622float2(h2);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
            wh[i] = *reinterpret_cast<const uint32_t *>(&h2);
            wl[i] = *reinterpret_cast<const uint32_t *>(&l2);
        }
        const uint32_t off = (uint32_t)r * 128u + ((uint32_t)(c ^ (r & 7)) << 4);
        *reinterpret_cast<uint4 *>(hi + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        *reinterpret_cast<uint4 *>(lo + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    }
}

// Half a row (32 values, chunks c0 .. c0 + 3) of the same layout.
__device__ __forceinline__ void store_half_split(uint8_t *hi, uint8_t *lo, int r, int c0, const float (&v)[32]) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t wh[4], wl[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float x0 = v[8 * c + 2 * i], x1 = v[8 * c + 2 * i + 1];
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
            const float2 hf = __bfloat1622float2(h2);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
            wh[i] = *reinterpret_cast<const uint32_t *>(&h2);
            wl[i] = *reinterpret_cast<const uint32_t *>(&l2);
        }
        const uint32_t off = (uint32_t)r * 128u + ((uint32_t)((c0 + c) ^ (r & 7)) << 4);
        *reinterpret_cast<uint4 *>(hi + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        *reinterpret_cast<uint4 *>(lo + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    }
}

template <int K>
__device__ __forceinline__ void loadk(const float *src, float (&v)[K]) {
    const float4 *p = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int i = 0; i < K / 4; ++i) {
        const float4 w = p[i];
        v[4 * i] = w.x;
        v[4 * i + 1] = w.y;
        v[4 * i + 2] = w.z;
        v[4 * i + 3] = w.w;
    }
}

template <int K>
__device__ __forceinline__ void storek(float *dst, const float (&v)[K]) {
    float4 *p = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int i = 0; i < K / 4; ++i) p[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

__device__ __forceinline__ void load64(const float *src, float (&v)[TS]) {
    const float4 *p = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int i = 0; i < TS / 4; ++i) {
        const float4 w = p[i];
        v[4 * i] = w.x;
        v[4 * i + 1] = w.y;
        v[4 * i + 2] = w.z;
        v[4 * i + 3] = w.w;
    }
}

__device__ __forceinline__ void store64(float *dst, const float (&v)[TS]) {
    float4 *p = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int i = 0; i < TS / 4; ++i) p[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// TMEM image of one transposed matrix (rows of 256 bytes) into columns
// col .. col + 63 of this thread's lane; called by all 128 threads of a
// warpgroup (thread j = lane j).
__device__ __forceinline__ void image_to_tmem(const uint8_t *img, uint32_t tmem, uint32_t lane_off, uint32_t col,
                                              int j) {
    const uint32_t *row = reinterpret_cast<const uint32_t *>(img + (size_t)j * 256);
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
        uint32_t r[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) r[q] = row[part * 32 + q];
        tmem_st32(tmem + lane_off + col + part * 32, r);
    }
}

__device__ __forceinline__ void tmem_alloc_all(uint32_t dst_smem, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free_all(uint32_t tmem, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
}

struct TcMisc {
    uint64_t mbar[4];
    uint32_t tmem_base;
    int abort_flag;
};

}  // namespace

size_t bwd_tc_image_bytes(int nL) { return (size_t)nL * kImgPerLayer * kImg; }

// Images of C, W_z, W_h, D of every layer (layer 0: C only; its other
// matrices act on the one-hot input), high and low BF16 parts, in the TMEM
// row layout (image row m, element k at m * 256 + 2 k): transposed (value
// M[k][m], the backward's products) and as stored (value M[m][k], the
// forward's products).
__global__ void pack_bwd_tc_kernel(const float *__restrict__ theta, ThetaLayout tl, uint8_t *__restrict__ out) {
    const int64_t total = (int64_t)tl.nL * 4 * H * H;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(i / (4 * H * H));
        const int mat = (int)((i / (H * H)) % 4);
        const int e = (int)(i % (H * H));
        const int m = e / H, k = e % H;
        if (l == 0 && mat != IM_C) continue;
        const int64_t src = mat == IM_C ? tl.C[l] : mat == IM_WZ ? tl.Wz[l] : mat == IM_WH ? tl.Wh[l] : tl.D[l];
#pragma unroll
        for (int plain = 0; plain < 2; ++plain) {
            const float v = plain ? theta[src + (int64_t)m * H + k] : theta[src + (int64_t)k * H + m];
            const __nv_bfloat16 hv = __float2bfloat16_rn(v);
            const __nv_bfloat16 lv = __float2bfloat16_rn(v - __bfloat162float(hv));
            const size_t base = ((size_t)l * kImgPerLayer + plain * kImgPlain + 2 * mat) * kImg + (size_t)m * 256 +
                                (size_t)k * 2;
            *reinterpret_cast<__nv_bfloat16 *>(out + base) = hv;
            *reinterpret_cast<__nv_bfloat16 *>(out + base + kImg) = lv;
        }
    }
}

cudaError_t launch_pack_bwd_tc(const float *theta, const ThetaLayout &tl, void *images, cudaStream_t stream) {
    if (tl.H != H) return cudaErrorInvalidValue;
    pack_bwd_tc_kernel<<<128, 256, 0, stream>>>(theta, tl, static_cast<uint8_t *>(images));
    return cudaGetLastError();
}

// --------------------------------------------------------------- gy, g_h
// Two streams (warpgroups) per CTA, up to two CTAs per SM (256 TMEM columns
// each: C^T high and low parts at 128 and 192, accumulators at 0 and 64);
// stream s takes items blockIdx.x * 2 + s, stepping by gridDim.x * 2.  An
// item is (sample, 64-site tile).
constexpr int kGhStreams = 2;
constexpr uint32_t kGhSmem = kGhStreams * 2 * kTile + 256 + 1024;

__global__ void __launch_bounds__(128 * kGhStreams, 1) gy_gh_kernel(const __grid_constant__ BwdTcArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    TcMisc &M = *reinterpret_cast<TcMisc *>(smem + kGhStreams * 2 * kTile);
    const int tid = threadIdx.x, s = tid >> 7, j = tid & 127, warp = tid >> 5;
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    uint8_t *thi = smem + (2 * s) * kTile, *tlo = thi + kTile;
    if (warp == 0) tmem_alloc_all(smem_u32(&M.tmem_base), 256);
    if (tid == 0) {
        for (int i = 0; i < kGhStreams; ++i) mbar_init(smem_u32(&M.mbar[i]), 1);
        M.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = M.tmem_base;
    // C^T of this layer, high part at column 128, low part at 192
    const uint8_t *img = A.images + (size_t)A.l * kImgPerLayer * kImg;
    if (s == 0) image_to_tmem(img + (2 * IM_C) * kImg, tmem, lane_off, 128, j);
    else image_to_tmem(img + (2 * IM_C + 1) * kImg, tmem, lane_off, 192, j);
    tmem_wait_st();
    tc_before();
    __syncthreads();
    tc_after();
    // columns are relative to the allocation, which may start at 0 or 256
    const bool ok_tmem = ((tmem & 0xFFFFu) == 0 || (tmem & 0xFFFFu) == 256) && (tmem >> 16) == 0;
    if (!ok_tmem && tid == 0) set_status(A.status, PSR_EDEVICE);
    const uint32_t acc = 64u * (uint32_t)s;
    const uint32_t bar = smem_u32(&M.mbar[s]);
    const int bar_id = 1 + s;
    uint32_t phase = 0;
    const int ntile = A.Np / TS;
    const int64_t items = ok_tmem ? (int64_t)A.n * ntile : 0;
    const bool top = (A.l == A.nL - 1);
    const float wdj = top ? A.wd[j] : 0.0f;
    for (int64_t it = (int64_t)blockIdx.x * kGhStreams + s; it < items; it += (int64_t)gridDim.x * kGhStreams) {
        const int64_t sample = it / ntile;
        const int t0 = (int)(it % ntile) * TS;
        const float *st = A.stash + sample * A.stash_stride;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {  // 32 sites at a time
            const int th = t0 + 32 * hh;
            float v[32], y[32];
            loadk<32>(st + ((int64_t)(A.l * kStashQ + kStashY) * H + j) * A.Np + th, y);
            if (top) {
                loadk<32>(st + (int64_t)A.nL * kStashQ * H * A.Np + th, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] *= wdj;
            } else {
                loadk<32>(A.gx_in + (sample * H + j) * A.Np + th, v);
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] *= gelu_grad(y[i]);
            storek<32>(A.gy + (sample * H + j) * A.Np + th, v);
            store_half_split(thi, tlo, j, 4 * hh, v);
        }
        fence_proxy_async();
        tc_before();
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        tc_after();
        if (j == 0) {
            const uint64_t bh = tdesc(smem_u32(thi)), bl = tdesc(smem_u32(tlo));
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(tmem + acc, tmem + 128 + kk * 8, bh + fm_boff(kk), kk > 0);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(tmem + acc, tmem + 128 + kk * 8, bl + fm_boff(kk), 1);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(tmem + acc, tmem + 192 + kk * 8, bh + fm_boff(kk), 1);
            mma_commit(bar);
        }
        if (!mbar_wait(bar, phase)) {
            M.abort_flag = 1;
            set_status(A.status, PSR_ETIMEOUT);
        }
        phase ^= 1u;
        tc_after();
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            uint32_t r[32];
            tmem_ld32(tmem + lane_off + acc + 32 * hh, r);
            tmem_wait_ld32(r);
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
            storek<32>(A.gh + (sample * H + j) * A.Np + t0 + 32 * hh, v);
        }
        tc_before();
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        tc_after();
        if (M.abort_flag) break;
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        tmem_free_all(tmem, 256);
    }
}

// --------------------------------------------------------------- gx
// Two streams per CTA; images W_z^T, W_h^T, D^T (hi, lo) in TMEM columns
// 128 .. 511, accumulators at 0 and 64.
constexpr int kGxStreams = 2;
constexpr uint32_t kGxSmem = kGxStreams * 6 * kTile + 256 + 1024;

__global__ void __launch_bounds__(128 * kGxStreams, 1) gx_kernel(const __grid_constant__ BwdTcArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    TcMisc &M = *reinterpret_cast<TcMisc *>(smem + kGxStreams * 6 * kTile);
    const int tid = threadIdx.x, s = tid >> 7, j = tid & 127, warp = tid >> 5;
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    uint8_t *tiles = smem + (6 * s) * kTile;  // dz hi, lo, dc hi, lo, gy hi, lo
    if (warp == 0) tmem_alloc_all(smem_u32(&M.tmem_base), 512);
    if (tid == 0) {
        for (int i = 0; i < kGxStreams; ++i) mbar_init(smem_u32(&M.mbar[i]), 1);
        M.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = M.tmem_base;
    const uint8_t *img = A.images + (size_t)A.l * kImgPerLayer * kImg;
    if (s == 0) {
        image_to_tmem(img + (2 * IM_WZ) * kImg, tmem, lane_off, 128, j);
        image_to_tmem(img + (2 * IM_WZ + 1) * kImg, tmem, lane_off, 192, j);
        image_to_tmem(img + (2 * IM_WH) * kImg, tmem, lane_off, 256, j);
        tmem_wait_st();
    } else {
        image_to_tmem(img + (2 * IM_WH + 1) * kImg, tmem, lane_off, 320, j);
        image_to_tmem(img + (2 * IM_D) * kImg, tmem, lane_off, 384, j);
        image_to_tmem(img + (2 * IM_D + 1) * kImg, tmem, lane_off, 448, j);
        tmem_wait_st();
    }
    tc_before();
    __syncthreads();
    tc_after();
    const bool ok_tmem = (tmem == 0);
    if (!ok_tmem && tid == 0) set_status(A.status, PSR_EDEVICE);
    const uint32_t acc = 64u * (uint32_t)s;
    const uint32_t bar = smem_u32(&M.mbar[s]);
    const int bar_id = 1 + s;
    uint32_t phase = 0;
    const int ntile = A.Np / TS;
    const int64_t items = ok_tmem ? (int64_t)A.n * ntile : 0;
    for (int64_t it = (int64_t)blockIdx.x * kGxStreams + s; it < items; it += (int64_t)gridDim.x * kGxStreams) {
        const int64_t sample = it / ntile;
        const int t0 = (int)(it % ntile) * TS;
        const int64_t off = (sample * H + j) * A.Np + t0;
        {
            float v[TS];
            load64(A.dz + off, v);
            store_row_split(tiles, tiles + kTile, j, v);
            load64(A.dc + off, v);
            store_row_split(tiles + 2 * kTile, tiles + 3 * kTile, j, v);
            load64(A.gy + off, v);
            store_row_split(tiles + 4 * kTile, tiles + 5 * kTile, j, v);
        }
        fence_proxy_async();
        tc_before();
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        tc_after();
        if (j == 0) {
            const uint32_t tb = smem_u32(tiles);
            bool first = true;
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {  // (W_z^T, dz), (W_h^T, dc), (D^T, gy)
                const uint32_t ahi = 128u + 128u * (uint32_t)pr, alo = ahi + 64u;
                const uint64_t bh = tdesc(tb + (2 * pr) * kTile), bl = tdesc(tb + (2 * pr + 1) * kTile);
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    mma_ts<kIdescFM>(acc, ahi + kk * 8, bh + fm_boff(kk), first ? 0u : 1u);
                    first = false;
                }
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(acc, ahi + kk * 8, bl + fm_boff(kk), 1);
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(acc, alo + kk * 8, bh + fm_boff(kk), 1);
            }
            mma_commit(bar);
        }
        if (!mbar_wait(bar, phase)) {
            M.abort_flag = 1;
            set_status(A.status, PSR_ETIMEOUT);
        }
        phase ^= 1u;
        tc_after();
        uint32_t r0[32], r1[32];
        tmem_ld32(tmem + lane_off + acc, r0);
        tmem_ld32(tmem + lane_off + acc + 32, r1);
        tmem_wait_ld32(r0);
        tmem_wait_ld32(r1);
        float v[TS];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            v[i] = __uint_as_float(r0[i]);
            v[32 + i] = __uint_as_float(r1[i]);
        }
        store64(A.gx_out + off, v);
        tc_before();
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        tc_after();
        if (M.abort_flag) break;
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        tmem_free_all(tmem, 512);
    }
}

// --------------------------------------------------------------- reverse scan
// One CTA per sample, thread j = unit j; sites from the last padded one down
// in steps of 8 (two 16-byte loads per array and step).
__global__ void __launch_bounds__(H) scan_bwd_kernel(const __grid_constant__ BwdTcArgs A) {
    const int j = threadIdx.x;
    const int64_t sample = blockIdx.x;
    const int l = A.l, Np = A.Np;
    const float *st = A.stash + sample * A.stash_stride;
    const float *ar = st + ((int64_t)(l * kStashQ + kStashA) * H + j) * Np;
    const float *cr = st + ((int64_t)(l * kStashQ + kStashC) * H + j) * Np;
    const float *hr = st + ((int64_t)(l * kStashQ + kStashH) * H + j) * Np;
    const float *gr = A.gh + (sample * H + j) * Np;
    const bool resid = (l + 1 < A.nL) && (l + 1 >= 2);
    const float *rr = resid ? A.gy_up + (sample * H + j) * Np : nullptr;
    float *dzr = A.dz + (sample * H + j) * Np;
    float *dcr = A.dc + (sample * H + j) * Np;
    const bool top = (l == A.nL - 1);
    const float *yr = top ? st + ((int64_t)(l * kStashQ + kStashY) * H + j) * Np : nullptr;
    const float *gd = st + (int64_t)A.nL * kStashQ * H * Np;
    const float *gyr = (l == 0) ? A.gy + (sample * H + j) * Np : nullptr;
    const uint64_t *bits = (l == 0) ? A.bits + sample * A.W : nullptr;
    float *row = A.rows + sample * A.P;

    float lam = 0.0f, an = 0.0f;
    float sz = 0.0f, sc = 0.0f, swo = 0.0f, sbo = 0.0f;
    float z1 = 0.0f, z2 = 0.0f, c1 = 0.0f, c2 = 0.0f, d1 = 0.0f, d2 = 0.0f;  // layer 0: codes 1, 2
    // the next (lower) step's inputs are fetched while this one is computed
    float ng[8], na[8], nc[8], nh[8], nr[8], nhb = 0.0f;
    auto fetch = [&](int t) {
        const float4 *g4 = reinterpret_cast<const float4 *>(gr + t);
        const float4 *a4 = reinterpret_cast<const float4 *>(ar + t);
        const float4 *c4 = reinterpret_cast<const float4 *>(cr + t);
        const float4 *h4 = reinterpret_cast<const float4 *>(hr + t);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float4 gv = g4[q], av = a4[q], cv = c4[q], hv = h4[q];
            ng[4 * q] = gv.x; ng[4 * q + 1] = gv.y; ng[4 * q + 2] = gv.z; ng[4 * q + 3] = gv.w;
            na[4 * q] = av.x; na[4 * q + 1] = av.y; na[4 * q + 2] = av.z; na[4 * q + 3] = av.w;
            nc[4 * q] = cv.x; nc[4 * q + 1] = cv.y; nc[4 * q + 2] = cv.z; nc[4 * q + 3] = cv.w;
            nh[4 * q] = hv.x; nh[4 * q + 1] = hv.y; nh[4 * q + 2] = hv.z; nh[4 * q + 3] = hv.w;
            if (resid) {
                const float4 rv = reinterpret_cast<const float4 *>(rr + t)[q];
                nr[4 * q] = rv.x; nr[4 * q + 1] = rv.y; nr[4 * q + 2] = rv.z; nr[4 * q + 3] = rv.w;
            } else {
                nr[4 * q] = nr[4 * q + 1] = nr[4 * q + 2] = nr[4 * q + 3] = 0.0f;
            }
        }
        nhb = (t > 0) ? hr[t - 1] : 0.0f;
    };
    fetch(Np - 8);
    for (int t = Np - 8; t >= 0; t -= 8) {
        float g[8], a[8], c[8], h[8], r[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            g[i] = ng[i];
            a[i] = na[i];
            c[i] = nc[i];
            h[i] = nh[i];
            r[i] = nr[i];
        }
        const float hbefore = nhb;
        if (t >= 8) fetch(t - 8);
        float dz[8], dc[8];
#pragma unroll
        for (int i = 7; i >= 0; --i) {
            lam = g[i] + r[i] + an * lam;
            const float hp = (i > 0) ? h[i - 1] : hbefore;
            const float ai = a[i];
            const float da = lam * (hp - c[i]);
            dz[i] = da * ai * (1.0f - ai);
            dc[i] = lam * (1.0f - ai);
            an = ai;
            sz += dz[i];
            sc += dc[i];
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            reinterpret_cast<float4 *>(dzr + t)[q] = make_float4(dz[4 * q], dz[4 * q + 1], dz[4 * q + 2], dz[4 * q + 3]);
            reinterpret_cast<float4 *>(dcr + t)[q] = make_float4(dc[4 * q], dc[4 * q + 1], dc[4 * q + 2], dc[4 * q + 3]);
        }
        if (top) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float gi = gd[t + i];
                swo += gi * gelu_f(yr[t + i]);
                sbo += gi;
            }
        }
        if (l == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int tt = t + i;
                if (tt == 0 || tt >= A.N) continue;  // code 0 (first site) or padding
                const int sprev = (int)((bits[(tt - 1) >> 6] >> ((tt - 1) & 63)) & 1ull);
                const float gyv = gyr[tt];
                if (sprev) { z2 += dz[i]; c2 += dc[i]; d2 += gyv; }
                else { z1 += dz[i]; c1 += dc[i]; d1 += gyv; }
            }
        }
    }
    const ThetaLayout &tl = A.tl;
    row[tl.bz[l] + j] = sz;
    row[tl.bh[l] + j] = sc;
    if (l == 0) {
        // W[j][0] acts on s_{t-1} = 0 (code 1), W[j][1] on s_{t-1} = 1 (code 2)
        row[tl.Wz[0] + 2 * j] = z1;
        row[tl.Wz[0] + 2 * j + 1] = z2;
        row[tl.Wh[0] + 2 * j] = c1;
        row[tl.Wh[0] + 2 * j + 1] = c2;
        row[tl.D[0] + 2 * j] = d1;
        row[tl.D[0] + 2 * j + 1] = d2;
    }
    if (top) {
        // readout: logit difference d = (W_o[1] - W_o[0]) x + (b_o[1] - b_o[0])
        row[tl.Wo + H + j] = swo;
        row[tl.Wo + j] = -swo;
        if (j == 0) {
            row[tl.bo + 1] = sbo;
            row[tl.bo] = -sbo;
        }
    }
}

// --------------------------------------------------------------- weight gradients
// One warpgroup per CTA; item = sample.  Per 64-site tile: A operands gy, dz,
// dc and B operands h, u (hi and lo each) in shared memory; four 128 x 128
// FP32 accumulators in TMEM (layer 0: dC only).
constexpr uint32_t kWgSmem = 10 * kTile + 256 + 1024;

__global__ void __launch_bounds__(128, 1) wgrad_kernel(const __grid_constant__ BwdTcArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    TcMisc &M = *reinterpret_cast<TcMisc *>(smem + 10 * kTile);
    const int tid = threadIdx.x, j = tid, warp = tid >> 5;
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    // tiles: 0,1 gy; 2,3 dz; 4,5 dc; 6,7 h; 8,9 u (hi, lo)
    if (warp == 0) tmem_alloc_all(smem_u32(&M.tmem_base), 512);
    if (tid == 0) {
        mbar_init(smem_u32(&M.mbar[0]), 1);
        M.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = M.tmem_base;
    const bool ok_tmem = (tmem == 0);
    if (!ok_tmem && tid == 0) set_status(A.status, PSR_EDEVICE);
    const uint32_t bar = smem_u32(&M.mbar[0]);
    uint32_t phase = 0;
    const int l = A.l, Np = A.Np, ntile = Np / TS;
    const bool full = (l >= 1);
    const uint32_t tb = smem_u32(smem);
    const int64_t items = ok_tmem ? A.n : 0;
    for (int64_t sample = blockIdx.x; sample < items; sample += gridDim.x) {
        const float *st = A.stash + sample * A.stash_stride;
        const int64_t off = (sample * H + j) * Np;
        for (int tile = 0; tile < ntile; ++tile) {
            const int t0 = tile * TS;
            float v[TS];
            load64(A.gy + off + t0, v);
            store_row_split(smem, smem + kTile, j, v);
            load64(st + ((int64_t)(l * kStashQ + kStashH) * H + j) * Np + t0, v);
            store_row_split(smem + 6 * kTile, smem + 7 * kTile, j, v);
            if (full) {
                load64(A.dz + off + t0, v);
                store_row_split(smem + 2 * kTile, smem + 3 * kTile, j, v);
                load64(A.dc + off + t0, v);
                store_row_split(smem + 4 * kTile, smem + 5 * kTile, j, v);
                // u = x^l = GELU(y^{l-1}) (zero at padded sites, where y = 0)
                load64(st + ((int64_t)((l - 1) * kStashQ + kStashY) * H + j) * Np + t0, v);
#pragma unroll
                for (int i = 0; i < TS; ++i) v[i] = gelu_f(v[i]);
                store_row_split(smem + 8 * kTile, smem + 9 * kTile, j, v);
            }
            fence_proxy_async();
            tc_before();
            __syncthreads();
            tc_after();
            if (tid == 0) {
                // (accumulator, A tile, B tile): dC = gy h^T, dD = gy u^T, dW_z = dz u^T, dW_h = dc u^T
                const int na = full ? 4 : 1;
#pragma unroll 1
                for (int q = 0; q < na; ++q) {
                    const int at = (q == 0 || q == 1) ? 0 : (q == 2 ? 2 : 4);
                    const int bt = (q == 0) ? 6 : 8;
                    const uint32_t d = 128u * (uint32_t)q;
                    const uint64_t ah = tdesc(tb + at * kTile), al = tdesc(tb + (at + 1) * kTile);
                    const uint64_t bh = tdesc(tb + bt * kTile), bl = tdesc(tb + (bt + 1) * kTile);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_ss<kIdescWG>(d, ah + km_off(kk), bh + km_off(kk), (tile > 0 || kk > 0) ? 1u : 0u);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) mma_ss<kIdescWG>(d, ah + km_off(kk), bl + km_off(kk), 1);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) mma_ss<kIdescWG>(d, al + km_off(kk), bh + km_off(kk), 1);
                }
                mma_commit(bar);
            }
            if (!mbar_wait(bar, phase)) {
                M.abort_flag = 1;
                set_status(A.status, PSR_ETIMEOUT);
            }
            phase ^= 1u;
            tc_after();
            __syncthreads();
            if (M.abort_flag) break;
        }
        if (M.abort_flag) break;
        // accumulators -> this sample's O_k row: row j of each 128 x 128 block
        float *row = A.rows + sample * A.P;
        const ThetaLayout &tl = A.tl;
        const int na = full ? 4 : 1;
#pragma unroll 1
        for (int q = 0; q < na; ++q) {
            const int64_t dst = (q == 0 ? tl.C[l] : q == 1 ? tl.D[l] : q == 2 ? tl.Wz[l] : tl.Wh[l]) + (int64_t)j * H;
#pragma unroll 1
            for (int part = 0; part < 4; ++part) {
                uint32_t r[32];
                tmem_ld32(tmem + lane_off + 128u * (uint32_t)q + 32u * (uint32_t)part, r);
                tmem_wait_ld32(r);
                // scalar stores: a row of P floats need not start 16-byte aligned
                float *p = row + dst + 32 * part;
#pragma unroll
                for (int i = 0; i < 32; ++i) p[i] = __uint_as_float(r[i]);
            }
        }
        tc_before();
        __syncthreads();
        tc_after();
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        tmem_free_all(tmem, 512);
    }
}

// --------------------------------------------------------------- stash forward
// The forward the backward needs, layer by layer over whole samples on the
// same tensor-core path: layer l >= 1 projections z = W_z u + b_z,
// c = W_h u + b_h (u = GELU(y of layer l-1)), a = sigmoid(z); the scan
// h_t = a_t h_{t-1} + (1 - a_t) c_t in FP32 (layer 0: a, c from the one-hot
// lookup tables); the output map y = C h + D u (+ h of layer l-1 for l >= 2;
// layer 0: C0 h + D0 onehot(s_{t-1})); then the readout adjoint g.  The
// products use the split BF16 operands of the backward.
constexpr int kFwStreams = 2;
constexpr uint32_t kFwSmem = kFwStreams * 4 * kTile + 256 + 1024;

// layer l >= 1: a and c of every site into the stash
__global__ void __launch_bounds__(128 * kFwStreams, 1) proj_fwd_kernel(const __grid_constant__ BwdTcArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    TcMisc &M = *reinterpret_cast<TcMisc *>(smem + kFwStreams * 4 * kTile);
    const int tid = threadIdx.x, s = tid >> 7, j = tid & 127, warp = tid >> 5;
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    uint8_t *tiles = smem + (4 * s) * kTile;  // u hi, lo
    if (warp == 0) tmem_alloc_all(smem_u32(&M.tmem_base), 512);
    if (tid == 0) {
        for (int i = 0; i < kFwStreams; ++i) mbar_init(smem_u32(&M.mbar[i]), 1);
        M.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = M.tmem_base;
    const int l = A.l;
    const uint8_t *img = A.images + ((size_t)l * kImgPerLayer + kImgPlain) * kImg;
    if (s == 0) {
        image_to_tmem(img + (2 * IM_WZ) * kImg, tmem, lane_off, 256, j);
        image_to_tmem(img + (2 * IM_WZ + 1) * kImg, tmem, lane_off, 320, j);
    } else {
        image_to_tmem(img + (2 * IM_WH) * kImg, tmem, lane_off, 384, j);
        image_to_tmem(img + (2 * IM_WH + 1) * kImg, tmem, lane_off, 448, j);
    }
    tmem_wait_st();
    tc_before();
    __syncthreads();
    tc_after();
    const bool ok_tmem = (tmem == 0);
    if (!ok_tmem && tid == 0) set_status(A.status, PSR_EDEVICE);
    const uint32_t accz = 128u * (uint32_t)s, accc = accz + 64u;
    const uint32_t bar = smem_u32(&M.mbar[s]);
    const int bar_id = 1 + s;
    uint32_t phase = 0;
    const int Np = A.Np, ntile = Np / TS;
    const float bz = A.pk[A.fl.bz[l] + j], bh = A.pk[A.fl.bh[l] + j];
    const int64_t items = ok_tmem ? (int64_t)A.n * ntile : 0;
    for (int64_t it = (int64_t)blockIdx.x * kFwStreams + s; it < items; it += (int64_t)gridDim.x * kFwStreams) {
        const int64_t sample = it / ntile;
        const int t0 = (int)(it % ntile) * TS;
        float *st = const_cast<float *>(A.stash) + sample * A.stash_stride;
#pragma unroll 1
        for (int hh = 0; hh < 2; ++hh) {
            float v[32];
            loadk<32>(st + ((int64_t)((l - 1) * kStashQ + kStashY) * H + j) * Np + t0 + 32 * hh, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = gelu_f(v[i]);
            store_half_split(tiles, tiles + kTile, j, 4 * hh, v);
        }
        fence_proxy_async();
        tc_before();
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        tc_after();
        if (j == 0) {
            const uint64_t bh_ = tdesc(smem_u32(tiles)), bl_ = tdesc(smem_u32(tiles + kTile));
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                const uint32_t d = w ? accc : accz, ahi = w ? 384u : 256u, alo = ahi + 64u;
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(d, ahi + kk * 8, bh_ + fm_boff(kk), kk > 0);
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(d, ahi + kk * 8, bl_ + fm_boff(kk), 1);
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(d, alo + kk * 8, bh_ + fm_boff(kk), 1);
            }
            mma_commit(bar);
        }
        if (!mbar_wait(bar, phase)) {
            M.abort_flag = 1;
            set_status(A.status, PSR_ETIMEOUT);
        }
        phase ^= 1u;
        tc_after();
#pragma unroll 1
        for (int hh = 0; hh < 2; ++hh) {
            uint32_t rz[32], rc[32];
            tmem_ld32(tmem + lane_off + accz + 32 * hh, rz);
            tmem_ld32(tmem + lane_off + accc + 32 * hh, rc);
            tmem_wait_ld32(rz);
            tmem_wait_ld32(rc);
            float av[32], cv[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const bool in = (t0 + 32 * hh + i) < A.N;
                av[i] = in ? sigmoid_f(__uint_as_float(rz[i]) + bz) : 0.0f;
                cv[i] = in ? __uint_as_float(rc[i]) + bh : 0.0f;
            }
            storek<32>(st + ((int64_t)(l * kStashQ + kStashA) * H + j) * Np + t0 + 32 * hh, av);
            storek<32>(st + ((int64_t)(l * kStashQ + kStashC) * H + j) * Np + t0 + 32 * hh, cv);
        }
        tc_before();
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        tc_after();
        if (M.abort_flag) break;
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        tmem_free_all(tmem, 512);
    }
}

// forward scan of layer l: one CTA per sample, thread j = unit j
__global__ void __launch_bounds__(H) scan_fwd_kernel(const __grid_constant__ BwdTcArgs A) {
    const int j = threadIdx.x;
    const int64_t sample = blockIdx.x;
    const int l = A.l, Np = A.Np, N = A.N;
    float *st = const_cast<float *>(A.stash) + sample * A.stash_stride;
    float *ar = st + ((int64_t)(l * kStashQ + kStashA) * H + j) * Np;
    float *cr = st + ((int64_t)(l * kStashQ + kStashC) * H + j) * Np;
    float *hr = st + ((int64_t)(l * kStashQ + kStashH) * H + j) * Np;
    const uint64_t *bits = A.bits + sample * A.W;
    float ta[3] = {0, 0, 0}, tb[3] = {0, 0, 0}, tc_[3] = {0, 0, 0};
    if (l == 0) {
#pragma unroll
        for (int code = 0; code < 3; ++code) {
            ta[code] = A.pk[A.fl.A0 + code * H + j];
            tb[code] = A.pk[A.fl.B0 + code * H + j];
            tc_[code] = A.pk[A.fl.CD0 + code * H + j];
        }
    }
    float h = 0.0f;
    float na[8], nc[8];
    auto fetch = [&](int t, float (&a)[8], float (&c)[8]) {
        if (l == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int tt = t + i;
                const int code = (tt == 0) ? 0 : 1 + (int)((bits[(tt - 1) >> 6] >> ((tt - 1) & 63)) & 1ull);
                a[i] = ta[code];
                c[i] = tc_[code];
            }
        } else {
            const float4 *a4 = reinterpret_cast<const float4 *>(ar + t);
            const float4 *c4 = reinterpret_cast<const float4 *>(cr + t);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float4 av = a4[q], cv = c4[q];
                a[4 * q] = av.x; a[4 * q + 1] = av.y; a[4 * q + 2] = av.z; a[4 * q + 3] = av.w;
                c[4 * q] = cv.x; c[4 * q + 1] = cv.y; c[4 * q + 2] = cv.z; c[4 * q + 3] = cv.w;
            }
        }
    };
    fetch(0, na, nc);
    for (int t = 0; t < Np; t += 8) {
        float a[8], c[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            a[i] = na[i];
            c[i] = nc[i];
        }
        if (t + 8 < Np) fetch(t + 8, na, nc);  // the next step's inputs, in flight meanwhile
        float hv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const bool in = (t + i) < N;
            if (l == 0) {
                const int tt = t + i;
                const int code = (tt == 0) ? 0 : 1 + (int)((bits[(tt - 1) >> 6] >> ((tt - 1) & 63)) & 1ull);
                h = a[i] * h + tb[code];
            } else {
                h = a[i] * h + (1.0f - a[i]) * c[i];
            }
            hv[i] = in ? h : 0.0f;
            if (!in) { a[i] = 0.0f; c[i] = 0.0f; }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            reinterpret_cast<float4 *>(hr + t)[q] = make_float4(hv[4 * q], hv[4 * q + 1], hv[4 * q + 2], hv[4 * q + 3]);
            if (l == 0) {
                reinterpret_cast<float4 *>(ar + t)[q] = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
                reinterpret_cast<float4 *>(cr + t)[q] = make_float4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]);
            }
        }
    }
}

// output map of layer l: y into the stash
__global__ void __launch_bounds__(128 * kFwStreams, 1) outmap_fwd_kernel(const __grid_constant__ BwdTcArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    TcMisc &M = *reinterpret_cast<TcMisc *>(smem + kFwStreams * 4 * kTile);
    const int tid = threadIdx.x, s = tid >> 7, j = tid & 127, warp = tid >> 5;
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    uint8_t *tiles = smem + (4 * s) * kTile;  // h hi, lo, u hi, lo
    if (warp == 0) tmem_alloc_all(smem_u32(&M.tmem_base), 512);
    if (tid == 0) {
        for (int i = 0; i < kFwStreams; ++i) mbar_init(smem_u32(&M.mbar[i]), 1);
        M.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = M.tmem_base;
    const int l = A.l;
    const uint8_t *img = A.images + ((size_t)l * kImgPerLayer + kImgPlain) * kImg;
    if (s == 0) {
        image_to_tmem(img + (2 * IM_C) * kImg, tmem, lane_off, 256, j);
        image_to_tmem(img + (2 * IM_C + 1) * kImg, tmem, lane_off, 320, j);
    } else if (l >= 1) {
        image_to_tmem(img + (2 * IM_D) * kImg, tmem, lane_off, 384, j);
        image_to_tmem(img + (2 * IM_D + 1) * kImg, tmem, lane_off, 448, j);
    }
    tmem_wait_st();
    tc_before();
    __syncthreads();
    tc_after();
    const bool ok_tmem = (tmem == 0);
    if (!ok_tmem && tid == 0) set_status(A.status, PSR_EDEVICE);
    const uint32_t acc = 64u * (uint32_t)s;
    const uint32_t bar = smem_u32(&M.mbar[s]);
    const int bar_id = 1 + s;
    uint32_t phase = 0;
    const int Np = A.Np, ntile = Np / TS;
    float du[3] = {0, 0, 0};
    if (l == 0) {
#pragma unroll
        for (int code = 0; code < 3; ++code) du[code] = A.pk[A.fl.DU0 + code * H + j];
    }
    const int64_t items = ok_tmem ? (int64_t)A.n * ntile : 0;
    for (int64_t it = (int64_t)blockIdx.x * kFwStreams + s; it < items; it += (int64_t)gridDim.x * kFwStreams) {
        const int64_t sample = it / ntile;
        const int t0 = (int)(it % ntile) * TS;
        float *st = const_cast<float *>(A.stash) + sample * A.stash_stride;
#pragma unroll 1
        for (int hh = 0; hh < 2; ++hh) {
            float v[32];
            loadk<32>(st + ((int64_t)(l * kStashQ + kStashH) * H + j) * Np + t0 + 32 * hh, v);
            store_half_split(tiles, tiles + kTile, j, 4 * hh, v);
            if (l >= 1) {
                loadk<32>(st + ((int64_t)((l - 1) * kStashQ + kStashY) * H + j) * Np + t0 + 32 * hh, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = gelu_f(v[i]);
                store_half_split(tiles + 2 * kTile, tiles + 3 * kTile, j, 4 * hh, v);
            }
        }
        fence_proxy_async();
        tc_before();
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        tc_after();
        if (j == 0) {
            const uint64_t hh_ = tdesc(smem_u32(tiles)), hl_ = tdesc(smem_u32(tiles + kTile));
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(acc, 256 + kk * 8, hh_ + fm_boff(kk), kk > 0);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(acc, 256 + kk * 8, hl_ + fm_boff(kk), 1);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(acc, 320 + kk * 8, hh_ + fm_boff(kk), 1);
            if (l >= 1) {
                const uint64_t uh = tdesc(smem_u32(tiles + 2 * kTile)), ul = tdesc(smem_u32(tiles + 3 * kTile));
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(acc, 384 + kk * 8, uh + fm_boff(kk), 1);
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(acc, 384 + kk * 8, ul + fm_boff(kk), 1);
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) mma_ts<kIdescFM>(acc, 448 + kk * 8, uh + fm_boff(kk), 1);
            }
            mma_commit(bar);
        }
        if (!mbar_wait(bar, phase)) {
            M.abort_flag = 1;
            set_status(A.status, PSR_ETIMEOUT);
        }
        phase ^= 1u;
        tc_after();
        const uint64_t *bits = A.bits + sample * A.W;
#pragma unroll 1
        for (int hh = 0; hh < 2; ++hh) {
            uint32_t r[32];
            tmem_ld32(tmem + lane_off + acc + 32 * hh, r);
            tmem_wait_ld32(r);
            float y[32];
            if (l >= 2) loadk<32>(st + ((int64_t)((l - 1) * kStashQ + kStashH) * H + j) * Np + t0 + 32 * hh, y);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int tt = t0 + 32 * hh + i;
                float v = __uint_as_float(r[i]);
                if (l >= 2) v += y[i];
                if (l == 0) {
                    const int code = (tt == 0) ? 0 : 1 + (int)((bits[(tt - 1) >> 6] >> ((tt - 1) & 63)) & 1ull);
                    v += du[code];
                }
                y[i] = (tt < A.N) ? v : 0.0f;
            }
            storek<32>(st + ((int64_t)(l * kStashQ + kStashY) * H + j) * Np + t0 + 32 * hh, y);
        }
        tc_before();
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        tc_after();
        if (M.abort_flag) break;
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        tmem_free_all(tmem, 512);
    }
}

// readout adjoint g_t = 1/2 (s_t - sigmoid(d_t)) with d = wd . GELU(y) + bd
// of the top layer (0 at forced sites and at t >= N): one thread per site
__global__ void readout_fwd_kernel(const __grid_constant__ BwdTcArgs A) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int Np = A.Np, N = A.N;
    if (i >= (int64_t)A.n * Np) return;
    const int64_t sample = i / Np;
    const int t = (int)(i % Np);
    float *st = const_cast<float *>(A.stash) + sample * A.stash_stride;
    float g = 0.0f;
    if (t < N) {
        const float *y = st + ((int64_t)((A.nL - 1) * kStashQ + kStashY) * H) * Np + t;
        float d = A.pk[A.fl.bd];
        for (int k = 0; k < H; ++k) d += A.wd[k] * gelu_f(y[(int64_t)k * Np]);
        const uint64_t *row = A.bits + sample * A.W;
        const int sv = (int)((row[t >> 6] >> (t & 63)) & 1ull);
        const int forced = u1_forced(A.u1, N, t, A.u1 ? count_up_before(row, t) : 0);
        g = (forced >= 0) ? 0.0f : 0.5f * ((float)sv - 1.0f / (1.0f + expf(-d)));
    }
    st[(int64_t)A.nL * kStashQ * H * Np + t] = g;
}

cudaError_t launch_fwd_tc(const BwdTcArgs &A0, int num_sms, cudaStream_t stream) {
    cudaError_t e = prepare_bwd_tc();  // declared in psr_internal.cuh
    if (e != cudaSuccess) return e;
    BwdTcArgs A = A0;
    const int64_t items = (int64_t)A.n * (A.Np / TS);
    int g = num_sms;
    if ((int64_t)g * kFwStreams > items) g = (int)((items + kFwStreams - 1) / kFwStreams);
    if (g < 1) g = 1;
    for (int l = 0; l < A.nL; ++l) {
        A.l = l;
        if (l >= 1) {
            proj_fwd_kernel<<<g, 128 * kFwStreams, kFwSmem, stream>>>(A);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        scan_fwd_kernel<<<A.n, H, 0, stream>>>(A);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        outmap_fwd_kernel<<<g, 128 * kFwStreams, kFwSmem, stream>>>(A);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int64_t sites = (int64_t)A.n * A.Np;
    readout_fwd_kernel<<<(unsigned)((sites + 255) / 256), 256, 0, stream>>>(A);
    return cudaGetLastError();
}

cudaError_t prepare_bwd_tc() {
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(gy_gh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGhSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gx_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGxSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(proj_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(outmap_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwSmem);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

// One layer of the backward for the samples of a batch (A.l set by the
// caller): gy and g_h, the reverse scan, the input gradient (l >= 1) and the
// weight gradients.
cudaError_t launch_bwd_tc_layer(const BwdTcArgs &A, int num_sms, cudaStream_t stream) {
    cudaError_t e = prepare_bwd_tc();
    if (e != cudaSuccess) return e;
    const int64_t items = (int64_t)A.n * (A.Np / TS);
    int g = num_sms;
    if ((int64_t)g * kGhStreams > items) g = (int)((items + kGhStreams - 1) / kGhStreams);
    gy_gh_kernel<<<g < 1 ? 1 : g, 128 * kGhStreams, kGhSmem, stream>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    scan_bwd_kernel<<<A.n, H, 0, stream>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (A.l >= 1) {
        g = num_sms;
        if ((int64_t)g * kGxStreams > items) g = (int)((items + kGxStreams - 1) / kGxStreams);
        gx_kernel<<<g < 1 ? 1 : g, 128 * kGxStreams, kGxSmem, stream>>>(A);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    g = num_sms < A.n ? num_sms : A.n;
    wgrad_kernel<<<g < 1 ? 1 : g, 128, kWgSmem, stream>>>(A);
    return cudaGetLastError();
}

}  // namespace psr
