// Exact autoregressive sampling of the chain minGRU on the tensor cores
// (Sec. II.A and Sec. III.B: conditionals drawn site by site; Eq. minGRU with
// the output map and residual of Sec. II.F-G), hidden 128, 3 layers, BF16
// operands with FP32 accumulation, FP32 gates, scan, GELU and readout: the
// conditionals of the model the BF16 forward (psr_fwd_bf16.cu) evaluates,
// with its activation forms (tanh-form GELU where the output is rounded to
// BF16, the A&S erf GELU for the readout's input, sigmoid via tanh).
//
// One CTA draws blocks of 32 samples, one sample per MMA column (N = 32).  At
// each site the products of every layer run as MMAs with the weights as A
// (M = 128 hidden units) and the block's activations as B (K-major, 128-byte
// swizzle): C0 h0;  W_z1 x1, W_h1 x1;  C1 h1 + D1 x1;  W_z2 x2, W_h2 x2;
// C2 h2 + D2 x2.  Seven of the nine weight matrices stay in tensor memory as
// A operands for the whole launch, D1 and D2 in shared memory.  Thread
// (warpgroup s, lane j of its quarter) owns hidden unit j for the block's
// samples 8 s .. 8 s + 7, with the three layers' carries in registers; the
// readout w_d x3 is reduced over the units on the CUDA cores and warp 0
// draws s_t = [u_t < P(s_t = 1)] (or the value the zero-magnetisation mask
// forces) for the 32 samples.  Each sample's arithmetic is independent of the
// others, so the draws do not depend on how samples are grouped into blocks.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "psr_bf16_math.cuh"
#include "psr_device.cuh"
#include "psr_internal.cuh"
#include "psr_tc.cuh"

namespace psr {

namespace {

using namespace tc;
using namespace bf16m;

constexpr int kHc = 128;                 // hidden width
constexpr int kLc = 3;                   // layers
constexpr int kBc = 32;                  // samples per block (MMA N)
constexpr int kEpiC = 512;               // epilogue threads
constexpr uint32_t kMatC = 32768;        // one 128 x 128 BF16 matrix
constexpr int kTmMats = 7;               // C0, Wz1, Wh1, C1, Wz2, Wh2, C2 in tensor memory
constexpr uint32_t kTileC = 2 * 4096;    // B tile: 32 rows x K 128 (two 64-wide K chunks)
constexpr size_t kSmemPadC = 120 * 1024; // at least this much, so one CTA holds an SM (all of TMEM)
// tensor-memory columns: accumulators z (or y) at 0, c at 32; the weights
enum { kTmZ = 0, kTmH = 32, kTmW = 64 };
enum { kWC0, kWWz1, kWWh1, kWC1, kWWz2, kWWh2, kWC2 };
// per-unit constants in shared memory [kind][unit]
enum { kKA0, kKA1, kKA2, kKB0, kKB1, kKB2, kKD0, kKD1, kKD2, kKHbz1, kKBh1, kKHbz2, kKBh2, kKWd, kKCst };

template <int NN>
constexpr uint32_t idesc_c() {  // kind::f16, D F32, A = B = BF16, both K-major, M = 128
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ uint64_t kdesc_c(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(1024u >> 4) << 16) |
           ((uint64_t)(1024u >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

struct MiscC {
    uint64_t e2m, m2e, wload;
    uint32_t tmem_base;
    int abort_flag;
    uint32_t spins;  // the block's draws at the current site, bit b = sample b
};

__device__ __forceinline__ bool wait_abc(uint32_t bar, uint32_t parity, const volatile int *ab) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u && (*ab || globaltimer() - t0 > kWaitNs)) return false;
    }
    return false;
}

__device__ __forceinline__ bool bar_or_c(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(kEpiC)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
    uint16_t h;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(x));
    return h;
}

__global__ void __launch_bounds__(kEpiC + 32, 1)
    sample_tc_kernel(const float *__restrict__ pk, F32Layout fl, const uint8_t *__restrict__ wimg,
                     const float *__restrict__ unif, int64_t n, int N, int u1, uint8_t *__restrict__ out,
                     float *__restrict__ logpsi, int *status) {
    constexpr int NW = kEpiC / 32;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    MiscC &M = *reinterpret_cast<MiscC *>(smem_raw);
    uint8_t *wd = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + sizeof(MiscC) + 1023) & ~uintptr_t(1023));
    uint8_t *tileX = wd + 2 * kMatC;  // D1, D2: 2 x 2 slices of 16 KB
    uint8_t *tileH = tileX + kTileC;
    float *cst = reinterpret_cast<float *>(tileH + kTileC);
    float *part = cst + kKCst * kHc;  // readout partial sums [warpgroup][quarter][sample]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const volatile int *ab = &M.abort_flag;
    const int64_t nblk = (n + kBc - 1) / kBc;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&M.tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&M.e2m), kEpiC / 32);  // one arrival per epilogue warp
        mbar_init(smem_u32(&M.m2e), 1);
        mbar_init(smem_u32(&M.wload), 1);
        M.abort_flag = 0;
        M.spins = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < kKCst * kHc; i += blockDim.x) {
        const int u = i % kHc, k = i / kHc;
        int64_t o;
        switch (k) {
            case kKA0: case kKA1: case kKA2: o = fl.A0 + (int64_t)(k - kKA0) * kHc + u; break;
            case kKB0: case kKB1: case kKB2: o = fl.B0 + (int64_t)(k - kKB0) * kHc + u; break;
            case kKD0: case kKD1: case kKD2: o = fl.DU0 + (int64_t)(k - kKD0) * kHc + u; break;
            case kKHbz1: o = fl.bz[1] + u; break;
            case kKBh1: o = fl.bh[1] + u; break;
            case kKHbz2: o = fl.bz[2] + u; break;
            case kKBh2: o = fl.bh[2] + u; break;
            default: o = fl.wd + u; break;
        }
        cst[i] = (k == kKHbz1 || k == kKHbz2) ? 0.5f * pk[o] : pk[o];
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = M.tmem_base;
    if (tmem != 0) {  // the kernel owns all 512 columns, from column 0
        if (tid == 0) set_status(status, PSR_EDEVICE);
        M.abort_flag = 1;
    }
    // the tensor-memory weights (warpgroup 0: row m = TMEM lane m) and the
    // shared-memory ones (bulk copy)
    if (warp < 4 && !M.abort_flag) {
        const int m = tid;
#pragma unroll 1
        for (int t = 0; t < kTmMats; ++t) {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(wimg + (size_t)t * kMatC + (size_t)m * 256);
#pragma unroll 1
            for (int part_ = 0; part_ < 2; ++part_) {
                uint32_t r[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) r[q] = row[part_ * 32 + q];
                tmem_st32(tmem + ((uint32_t)(warp * 32) << 16) + kTmW + t * 64 + part_ * 32, r);
            }
        }
        tmem_wait_st();
    }
    if (tid == 0 && !M.abort_flag) {
        mbar_arrive_tx(smem_u32(&M.wload), 2 * kMatC);
        for (int i = 0; i < 4; ++i)
            bulk_g2s(smem_u32(wd + (size_t)i * 16384), wimg + (size_t)kTmMats * kMatC + (size_t)i * 16384, 16384,
                     smem_u32(&M.wload));
        if (!mbar_wait(smem_u32(&M.wload), 0)) {
            M.abort_flag = 1;
            set_status(status, PSR_ETIMEOUT);
        }
    }
    tc_before();
    __syncthreads();
    tc_after();

    if (warp == NW) {
        // ------------------------------------------------ MMA issue
        if (lane == 0 && !M.abort_flag) {
            const uint32_t e2m = smem_u32(&M.e2m), m2e = smem_u32(&M.m2e);
            const uint64_t bx = kdesc_c(smem_u32(tileX)), bh = kdesc_c(smem_u32(tileH)),
                           ad0 = kdesc_c(smem_u32(wd));
            uint32_t pe = 0;
            bool ok = true;
            // K step kk (16 inputs) of a B tile: chunk kk / 4 (4 KB apart), 32 bytes per step
            auto bk = [](uint64_t b, int kk) { return b + (uint64_t)(((kk >> 2) * 4096 + (kk & 3) * 32) >> 4); };
            auto wait_e = [&]() -> bool {
                if (!wait_abc(e2m, pe, ab)) return false;
                pe ^= 1u;
                tc_after();
                return true;
            };
            // A from tensor memory (weight t), B tile b, accumulate onto D at column dc
            auto mm_t = [&](uint32_t dc, int t, uint64_t b, bool acc0) {
#pragma unroll
                for (int kk = 0; kk < 8; ++kk)
                    mma_ts<idesc_c<kBc>()>(tmem + dc, tmem + kTmW + t * 64 + kk * 8, bk(b, kk),
                                           (kk > 0 || acc0) ? 1u : 0u);
            };
            // A from shared memory (D1 or D2: two 16 KB slices of K 64), accumulating
            auto mm_s = [&](uint32_t dc, int which, uint64_t b) {
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const uint64_t a = ad0 + (uint64_t)(((which * 2 + (kk >> 2)) * 16384 + (kk & 3) * 32) >> 4);
                    mma_ss<idesc_c<kBc>()>(tmem + dc, a, bk(b, kk), 1u);
                }
            };
            for (int64_t blk = blockIdx.x; blk < nblk && ok; blk += gridDim.x) {
                for (int t = 0; t < N && ok; ++t) {
                    if (!(ok = wait_e())) break;  // h0
                    mm_t(kTmZ, kWC0, bh, false);
                    mma_commit(m2e);
                    if (!(ok = wait_e())) break;  // x1
                    mm_t(kTmZ, kWWz1, bx, false);
                    mm_t(kTmH, kWWh1, bx, false);
                    mma_commit(m2e);
                    if (!(ok = wait_e())) break;  // h1
                    mm_t(kTmZ, kWC1, bh, false);
                    mm_s(kTmZ, 0, bx);
                    mma_commit(m2e);
                    if (!(ok = wait_e())) break;  // x2
                    mm_t(kTmZ, kWWz2, bx, false);
                    mm_t(kTmH, kWWh2, bx, false);
                    mma_commit(m2e);
                    if (!(ok = wait_e())) break;  // h2
                    mm_t(kTmZ, kWC2, bh, false);
                    mm_s(kTmZ, 1, bx);
                    mma_commit(m2e);
                }
            }
            if (!ok) {
                M.abort_flag = 1;
                set_status(status, PSR_ETIMEOUT);
            }
        }
    } else {
        // ------------------------------------------------ epilogue
        const int s = warp >> 2, q4 = warp & 3, j = 32 * q4 + lane;
        const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
        auto K = [&](int k) { return cst[k * kHc + j]; };
        // element j of tile row 8 s + dt (K-major, 128-byte swizzle; K chunk j / 64)
        auto trow = [&](uint8_t *tl) -> uint32_t {
            const int kk = j & 63;
            return smem_u32(tl) + (uint32_t)(j >> 6) * 4096u + (uint32_t)(8 * s) * 128u + ((uint32_t)(kk >> 3) << 4) +
                   (uint32_t)(kk & 7) * 2u;
        };
        const uint32_t rX = trow(tileX), rH = trow(tileH);
        auto tst = [&](uint32_t b, int dt, float v) {
            asm volatile("st.shared.b16 [%0], %1;" ::"r"((b ^ ((uint32_t)(dt & 7) << 4)) + 128u * dt),
                         "h"(bf16_bits(v)));
        };
        auto ld8 = [&](uint32_t col, float (&v)[8]) {
            uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
            tmem_ld8(tmem + lane_off + col + (uint32_t)(8 * s), r0, r1, r2, r3, r4, r5, r6, r7);
            asm volatile("tcgen05.wait::ld.sync.aligned;"
                         : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3), "+r"(r4), "+r"(r5), "+r"(r6), "+r"(r7)::"memory");
            v[0] = __uint_as_float(r0);
            v[1] = __uint_as_float(r1);
            v[2] = __uint_as_float(r2);
            v[3] = __uint_as_float(r3);
            v[4] = __uint_as_float(r4);
            v[5] = __uint_as_float(r5);
            v[6] = __uint_as_float(r6);
            v[7] = __uint_as_float(r7);
        };
        uint32_t pm_ = 0;
        bool ok = !M.abort_flag;
        auto wait_m2e = [&]() {
            bool w = false;
            if (lane == 0) w = ok && wait_abc(smem_u32(&M.m2e), pm_, ab);
            w = __shfl_sync(0xffffffffu, w ? 1 : 0, 0) != 0;
            if (!w && ok && lane == 0) {
                M.abort_flag = 1;
                set_status(status, PSR_ETIMEOUT);
            }
            ok = ok && w;
            pm_ ^= 1u;
            tc_after();
        };
        auto arrive_e2m = [&]() {
            fence_proxy_async();
            tc_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&M.e2m));
        };
        const float bd = pk[fl.bd];
        // gates and scan of layer l (1 or 2) for the 8 samples; h to the h tile
        auto gates_scan = [&](float (&h)[8], int kh, int kb) {
            float z[8], c[8];
            ld8(kTmZ, z);
            ld8(kTmH, c);
            const float2 hbz2 = make_float2(K(kh), K(kh)), bh2 = make_float2(K(kb), K(kb));
#pragma unroll
            for (int b = 0; b < 8; b += 2) {
                float2 a, bb;
                gates2(make_float2(z[b], z[b + 1]), make_float2(c[b], c[b + 1]), hbz2, bh2, a, bb);
                h[b] = fmaf(a.x, h[b], bb.x);
                h[b + 1] = fmaf(a.y, h[b + 1], bb.y);
                tst(rH, b, h[b]);
                tst(rH, b + 1, h[b + 1]);
            }
        };

        for (int64_t blk = blockIdx.x; blk < nblk && ok; blk += gridDim.x) {
            const int64_t first = blk * kBc;
            float h0[8], h1[8], h2[8];
#pragma unroll
            for (int b = 0; b < 8; ++b) h0[b] = h1[b] = h2[b] = 0.0f;
            int nup = 0;         // warp 0: lane b's up spins so far
            float acc = 0.0f;    // warp 0: lane b's sum of log P
            uint32_t prev = 0;   // the block's draws at the previous site
            for (int t = 0; t < N && ok; ++t) {
                // ---- layer 0: one-hot input (zero at t = 0) -> lookups; scan
                {
                    const float a0 = K(kKA0), a1 = K(kKA1), a2 = K(kKA2), b0 = K(kKB0), b1 = K(kKB1), b2 = K(kKB2);
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        const int code = t == 0 ? 0 : 1 + (int)((prev >> (8 * s + b)) & 1u);
                        const float a = code == 0 ? a0 : (code == 1 ? a1 : a2);
                        const float bb = code == 0 ? b0 : (code == 1 ? b1 : b2);
                        h0[b] = fmaf(a, h0[b], bb);
                        tst(rH, b, h0[b]);
                    }
                }
                arrive_e2m();
                // ---- x1 = GELU(C0 h0 + D0 u)
                wait_m2e();
                if (ok) {
                    float y[8];
                    ld8(kTmZ, y);
                    const float d0 = K(kKD0), d1 = K(kKD1), d2 = K(kKD2);
#pragma unroll
                    for (int b = 0; b < 8; b += 2) {
                        float du[2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int code = t == 0 ? 0 : 1 + (int)((prev >> (8 * s + b + e)) & 1u);
                            du[e] = code == 0 ? d0 : (code == 1 ? d1 : d2);
                        }
                        const float2 x = gelu_bf16out2(make_float2(y[b] + du[0], y[b + 1] + du[1]));
                        tst(rX, b, x.x);
                        tst(rX, b + 1, x.y);
                    }
                }
                arrive_e2m();
                // ---- layer 1: gates and scan
                wait_m2e();
                if (ok) gates_scan(h1, kKHbz1, kKBh1);
                arrive_e2m();
                // ---- x2 = GELU(C1 h1 + D1 x1)
                wait_m2e();
                if (ok) {
                    float y[8];
                    ld8(kTmZ, y);
#pragma unroll
                    for (int b = 0; b < 8; b += 2) {
                        const float2 x = gelu_bf16out2(make_float2(y[b], y[b + 1]));
                        tst(rX, b, x.x);
                        tst(rX, b + 1, x.y);
                    }
                }
                arrive_e2m();
                // ---- layer 2: gates and scan
                wait_m2e();
                if (ok) gates_scan(h2, kKHbz2, kKBh2);
                arrive_e2m();
                // ---- x3 = GELU(C2 h2 + D2 x2 + h1); readout partial sums
                wait_m2e();
                if (ok) {
                    float y[8];
                    ld8(kTmZ, y);
                    const float wdj = K(kKWd);
#pragma unroll
                    for (int b = 0; b < 8; b += 2) {
                        const float2 x = gelu_fast2(__fadd2_rn(make_float2(y[b], y[b + 1]), make_float2(h1[b], h1[b + 1])));
                        float v0 = wdj * x.x, v1 = wdj * x.y;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            v0 += __shfl_xor_sync(0xffffffffu, v0, o);
                            v1 += __shfl_xor_sync(0xffffffffu, v1, o);
                        }
                        if (lane == 0) {
                            part[(s * 4 + q4) * 8 + b] = v0;
                            part[(s * 4 + q4) * 8 + b + 1] = v1;
                        }
                    }
                }
                tc_before();
                if (bar_or_c(!ok || *ab)) ok = false;
                // ---- draws: warp 0, sample 8 s' + b by lane 8 s' + b
                if (ok && warp == 0) {
                    const int sb = lane >> 3, b = lane & 7;
                    float d = bd;
#pragma unroll
                    for (int q = 0; q < 4; ++q) d += part[(sb * 4 + q) * 8 + b];
                    const int64_t row = first + lane;
                    int sv = 0;
                    if (row < n) {
                        const int forced = u1_forced(u1, N, t, nup);
                        const float p1 = forced >= 0 ? (float)forced : 1.0f / (1.0f + expf(-d));
                        sv = unif[row * N + t] < p1 ? 1 : 0;
                        acc += site_logp(d, sv, forced);
                        nup += sv;
                        out[row * N + t] = (uint8_t)sv;
                    }
                    const uint32_t mask = __ballot_sync(0xffffffffu, sv != 0);
                    if (lane == 0) M.spins = mask;
                }
                if (bar_or_c(!ok || *ab)) ok = false;
                prev = *(volatile uint32_t *)&M.spins;
            }
            if (ok && warp == 0 && logpsi && first + lane < n) logpsi[first + lane] = 0.5f * acc;
        }
        if (!ok) {
            M.abort_flag = 1;
            set_status(status, PSR_ETIMEOUT);
        }
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// BF16 weight image: the seven tensor-memory matrices row-major (A[m][k], 256
// bytes a row), then D1, D2 as K-major 128-byte-swizzled slices (rows m, 64
// inputs each: D1 k < 64, D1 k >= 64, D2 k < 64, D2 k >= 64).
__global__ void pack_sample_tc_kernel(const float *__restrict__ pk, F32Layout fl, uint8_t *__restrict__ wimg) {
    const int64_t tm_src[kTmMats] = {fl.CT[0], fl.WzT[1], fl.WhT[1], fl.CT[1], fl.WzT[2], fl.WhT[2], fl.CT[2]};
    const int64_t total = (int64_t)(kTmMats + 2) * kHc * kHc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int mat = (int)(i / (kHc * kHc)), m = (int)((i / kHc) % kHc), k = (int)(i % kHc);
        size_t byte;
        float v;
        if (mat < kTmMats) {
            v = pk[tm_src[mat] + (int64_t)k * kHc + m];
            byte = (size_t)mat * kMatC + (size_t)m * 256 + (size_t)k * 2;
        } else {
            const int w = mat - kTmMats;
            v = pk[(w == 0 ? fl.DT[1] : fl.DT[2]) + (int64_t)k * kHc + m];
            const int sl = w * 2 + (k >> 6), kk = k & 63;
            byte = (size_t)kTmMats * kMatC + (size_t)sl * 16384 + (size_t)m * 128 +
                   ((size_t)((kk >> 3) ^ (m & 7)) << 4) + (size_t)(kk & 7) * 2;
        }
        const __nv_bfloat16 bv = __float2bfloat16_rn(v);
        *reinterpret_cast<__nv_bfloat16 *>(wimg + byte) = bv;
    }
}

}  // namespace

bool sample_tc_supported(int nL, int H) { return nL == kLc && H == kHc; }

size_t sample_tc_weight_bytes() { return (size_t)(kTmMats + 2) * kMatC; }

cudaError_t launch_sample_tc(const float *pk, const F32Layout &fl, uint8_t *wimg, const float *unif, int64_t n,
                             int N, int u1, uint8_t *out, float *logpsi, int *status, int num_sms,
                             cudaStream_t stream) {
    if (!sample_tc_supported(fl.nL, fl.H)) return cudaErrorInvalidValue;
    pack_sample_tc_kernel<<<144, 256, 0, stream>>>(pk, fl, wimg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nblk = (n + kBc - 1) / kBc;
    const int grid = (int)(nblk < num_sms ? nblk : num_sms);
    if (grid < 1) return cudaSuccess;
    size_t smem = sizeof(MiscC) + 1024 + 2 * kMatC + 2 * kTileC + (size_t)kKCst * kHc * sizeof(float) +
                  (size_t)16 * 8 * sizeof(float);
    if (smem < kSmemPadC) smem = kSmemPadC;
    e = cudaFuncSetAttribute(sample_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sample_tc_kernel<<<grid, kEpiC + 32, smem, stream>>>(pk, fl, wimg, unif, n, N, u1, out, logpsi, status);
    return cudaGetLastError();
}

}  // namespace psr
