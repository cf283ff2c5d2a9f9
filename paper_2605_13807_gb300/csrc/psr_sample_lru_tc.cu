// Exact autoregressive sampling of the deep 1D LRU ansatz on the tensor
// cores (Sec. II.A and Sec. III.B: conditionals drawn site by site; model of
// Sec. II.B Eq. lru with the GLU blocks of Sec. III.B), hidden 64, FP16 (or
// BF16) operands with FP32 accumulation, FP32 complex recurrence, GLU and
// readout: the conditionals of the model that the tensor-core forward
// (psr_lru_tc.cu) evaluates.
//
// One CTA draws blocks of 32 samples, one sample per MMA column (N = 32).
// At each site every layer's products run as MMAs with the weights as A
// (M = 128 rows, the same 16 KB slices as the forward, resident in shared
// memory for the whole launch) and the block's activations as B:
//   e^gamma [B_re; B_im] u,  [C_re, -C_im] [h_re; h_im],  [W_a; W_g] y,
// then the readout x^T w_d with the x tile as A (M = 128 rows, the block's 32
// samples in rows 0..31) and w_d as B (N = 16), which leaves sample b's logit
// difference in tensor-memory lane b.  Warp 0 draws s_t = [u_t < P(s_t = 1)]
// for the 32 samples (or the value the zero-magnetisation mask forces) and
// publishes them for the next site's one-hot input.
//
// Thread r = 32 q4 + lane of warpgroup s owns row r of every accumulator
// (unit j = r / 2: its real part on even rows, imaginary part on odd rows)
// for the block's samples 8 s .. 8 s + 7; the complex carry of each layer
// and sample is split across the thread pair (each holds its own part and
// reads the partner's by a shuffle), so it stays in registers.  The y and
// GLU epilogues split the samples by parity across the pair.  Each sample's
// arithmetic is independent of the others, so the draws do not depend on
// how samples are grouped into blocks.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "psr_bf16_math.cuh"
#include "psr_device.cuh"
#include "psr_internal.cuh"
#include "psr_tc.cuh"

namespace psr {

namespace {

using namespace tc;
using namespace bf16m;

constexpr int kHs = 64;              // hidden width
constexpr int kBs = 32;              // samples per block (MMA N)
constexpr int kMaxLs = 3;            // layers whose weights stay resident in shared memory
constexpr uint32_t kSliceS = 16384;  // 128 rows x 64 inputs, 16-bit
constexpr int kEpiS = 512;           // epilogue threads
constexpr uint32_t kTileS = 2 * 16384;  // B tile (and the readout's A): 128 rows x K 128
constexpr uint32_t kWdS = 16 * 128;     // readout B operand: w_d, then 15 zero rows
constexpr int kTmemS = 32;              // tensor-memory columns

// per-unit constants in shared memory, [layer][kind][unit] (as the forward)
enum { kSLre, kSLim, kSD0, kSD1, kSBa, kSBg, kSBr0, kSBr1, kSBi0, kSBi1, kSCst };

template <bool F16, int NN>
constexpr uint32_t idesc_s() {
    return (1u << 4) | ((F16 ? 0u : 1u) << 7) | ((F16 ? 0u : 1u) << 10) | ((uint32_t)(NN >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ uint64_t kdesc_s(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(1024u >> 4) << 16) |
           ((uint64_t)(1024u >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

struct MiscS {
    uint64_t e2m, m2e, wload;
    uint32_t tmem_base;
    int abort_flag;
    uint32_t spins;  // the block's draws at the current site, bit b = sample b
};

__device__ __forceinline__ bool wait_abs(uint32_t bar, uint32_t parity, const volatile int *ab) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u && (*ab || globaltimer() - t0 > kWaitNs)) return false;
    }
    return false;
}

__device__ __forceinline__ bool bar_or_s(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(kEpiS)
        : "memory");
    return r != 0;
}

template <bool F16>
__device__ __forceinline__ uint16_t op16s(float x) {
    uint16_t h;  // round to nearest even; FP16 saturates at +-65504
    if (F16) asm("cvt.rn.satfinite.f16.f32 %0, %1;" : "=h"(h) : "f"(x));
    else asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(x));
    return h;
}

__device__ __forceinline__ void sts16s(uint32_t a, uint16_t v) {
    asm volatile("st.shared.b16 [%0], %1;" ::"r"(a), "h"(v));
}

template <bool F16>
__global__ void __launch_bounds__(kEpiS + 32, 1)
    sample_lru_tc_kernel(const float *__restrict__ pk, LruLayout f, const uint8_t *__restrict__ wimg, int n_slices,
                         const float *__restrict__ unif, int64_t n, int N, int u1, uint8_t *__restrict__ out,
                         float *__restrict__ logpsi, int *status) {
    constexpr int NW = kEpiS / 32;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    MiscS &M = *reinterpret_cast<MiscS *>(smem_raw);
    uint8_t *wts = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + sizeof(MiscS) + 1023) & ~uintptr_t(1023));
    uint8_t *wdb = wts + (size_t)(n_slices - 1) * kSliceS;  // the readout's B operand (w_d rows)
    uint8_t *tile = wdb + kWdS + (1024 - kWdS % 1024) % 1024;
    float *cst = reinterpret_cast<float *>(tile + kTileS);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nL = f.nL;
    const volatile int *ab = &M.abort_flag;
    const int64_t nblk = (n + kBs - 1) / kBs;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&M.tmem_base)),
                     "r"(kTmemS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&M.e2m), kEpiS / 32);  // one arrival per epilogue warp
        mbar_init(smem_u32(&M.m2e), 1);
        mbar_init(smem_u32(&M.wload), 1);
        M.abort_flag = 0;
        M.spins = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < nL * kSCst * kHs; i += blockDim.x) {
        const int u = i % kHs, k = (i / kHs) % kSCst, l = i / (kHs * kSCst);
        int64_t o = -1;
        switch (k) {
            case kSLre: o = f.lre[l] + u; break;
            case kSLim: o = f.lim[l] + u; break;
            case kSD0: o = f.D[l] + u; break;
            case kSD1: o = l == 0 ? f.D[0] + kHs + u : -1; break;
            case kSBa: o = f.ba[l] + u; break;
            case kSBg: o = f.bg[l] + u; break;
            case kSBr0: o = l == 0 ? f.BreT[0] + u : -1; break;
            case kSBr1: o = l == 0 ? f.BreT[0] + kHs + u : -1; break;
            case kSBi0: o = l == 0 ? f.BimT[0] + u : -1; break;
            default: o = l == 0 ? f.BimT[0] + kHs + u : -1; break;
        }
        // layer 0's one-hot B u lookups carry the factor e^gamma
        cst[i] = o >= 0 ? (k >= kSBr0 ? pk[f.gam[0] + u] * pk[o] : pk[o]) : 0.0f;
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = M.tmem_base;
    if (tid == 0) {
        // the weight slices (and the first 2 KB of the w_d slice) by bulk copy
        const uint32_t bytes = (uint32_t)(n_slices - 1) * kSliceS + kWdS;
        mbar_arrive_tx(smem_u32(&M.wload), bytes);
        for (int i = 0; i < n_slices - 1; ++i)
            bulk_g2s(smem_u32(wts + (size_t)i * kSliceS), wimg + (size_t)i * kSliceS, kSliceS, smem_u32(&M.wload));
        bulk_g2s(smem_u32(wdb), wimg + (size_t)(n_slices - 1) * kSliceS, kWdS, smem_u32(&M.wload));
        if (!mbar_wait(smem_u32(&M.wload), 0)) {
            M.abort_flag = 1;
            set_status(status, PSR_ETIMEOUT);
        }
    }
    __syncthreads();

    if (warp == NW) {
        // ------------------------------------------------ MMA issue
        if (lane == 0 && !M.abort_flag) {
            const uint32_t e2m = smem_u32(&M.e2m), m2e = smem_u32(&M.m2e);
            const uint64_t wd0 = kdesc_s(smem_u32(wts)), td = kdesc_s(smem_u32(tile)), wdd = kdesc_s(smem_u32(wdb));
            uint32_t pe = 0;
            bool ok = true;
            // one stage: wait for the epilogue, MMAs over the slices
            // [i0, i0 + ns) (K chunk kc of the tile for the i-th), commit
            auto stage = [&](int i0, int ns) -> bool {
                if (!wait_abs(e2m, pe, ab)) return false;
                pe ^= 1u;
                tc_after();
                for (int k = 0; k < ns; ++k) {
                    const uint64_t ad = wd0 + (uint64_t)((i0 + k) * (kSliceS >> 4)),
                                   bd = td + (uint64_t)((k * 16384u) >> 4);
                    mma_ss<idesc_s<F16, kBs>()>(tmem, ad, bd, k > 0 ? 1u : 0u);
                    mma_ss<idesc_s<F16, kBs>()>(tmem, ad + 2, bd + 2, 1u);
                    mma_ss<idesc_s<F16, kBs>()>(tmem, ad + 4, bd + 4, 1u);
                    mma_ss<idesc_s<F16, kBs>()>(tmem, ad + 6, bd + 6, 1u);
                }
                mma_commit(m2e);
                return true;
            };
            for (int64_t blk = blockIdx.x; blk < nblk && ok; blk += gridDim.x) {
                for (int t = 0; t < N && ok; ++t) {
                    int i = 0;  // slice index in the image's order
                    for (int l = 0; l < nL && ok; ++l) {
                        if (l > 0) {
                            ok = stage(i, 1);  // e^gamma B u
                            ++i;
                        }
                        if (ok) ok = stage(i, 2);  // Re(C h): h_re, h_im
                        i += 2;
                        if (ok) ok = stage(i, 1);  // [W_a; W_g] y
                        ++i;
                    }
                    if (!ok) break;
                    // readout: A = the x tile (samples in rows 0..31), B = w_d
                    if (!wait_abs(e2m, pe, ab)) {
                        ok = false;
                        break;
                    }
                    pe ^= 1u;
                    tc_after();
                    mma_ss<idesc_s<F16, 16>()>(tmem, td, wdd, 0u);
                    mma_ss<idesc_s<F16, 16>()>(tmem, td + 2, wdd + 2, 1u);
                    mma_ss<idesc_s<F16, 16>()>(tmem, td + 4, wdd + 4, 1u);
                    mma_ss<idesc_s<F16, 16>()>(tmem, td + 6, wdd + 6, 1u);
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
        const int s = warp >> 2, q4 = warp & 3, r = 32 * q4 + lane;
        const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
        const uint32_t tacc = tmem + lane_off + (uint32_t)(8 * s);  // this thread's 8 samples
        const int j = r >> 1;
        const bool odd_r = r & 1;
        auto C = [&](int l, int k) { return cst[(l * kSCst + k) * kHs + j]; };
        // element k of row nb + dt of the tile (K-major, 128-byte swizzle),
        // nb and dt with disjoint low three bits
        const uint32_t tiles_s = smem_u32(tile);
        auto tb = [&](int kc, int nb, int k) -> uint32_t {
            return tiles_s + (uint32_t)kc * 16384u + (uint32_t)nb * 128u + ((uint32_t)((k >> 3) ^ (nb & 7)) << 4) +
                   (uint32_t)(k & 7) * 2u;
        };
        auto tst = [&](uint32_t b, int dt, uint16_t v) { sts16s((b ^ ((uint32_t)(dt & 7) << 4)) + 128u * dt, v); };
        const float bd = pk[f.bd];
        uint32_t pm_ = 0;
        bool ok = !M.abort_flag;
        auto wait_m2e = [&]() {
            bool w = false;
            if (lane == 0) w = ok && wait_abs(smem_u32(&M.m2e), pm_, ab);
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

        for (int64_t blk = blockIdx.x; blk < nblk && ok; blk += gridDim.x) {
            const int64_t first = blk * kBs;
            // this thread's part of the complex carries (layer l, sample 8 s + b)
            float cm[kMaxLs][8];
#pragma unroll
            for (int l = 0; l < kMaxLs; ++l)
#pragma unroll
                for (int b = 0; b < 8; ++b) cm[l][b] = 0.0f;
            float xr[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // layer input at samples 8 s + 2 i + odd_r
            int nup = 0;                              // warp 0: lane b's up spins so far
            float acc = 0.0f;                         // warp 0: lane b's sum of log P
            uint32_t prev = 0;                        // the block's draws at the previous site
            for (int t = 0; t < N && ok; ++t) {
#pragma unroll 1
                for (int l = 0; l < nL && ok; ++l) {
                    // ---- h = lambda h + e^gamma B u for the thread's 8 samples
                    if (l > 0) wait_m2e();
                    if (ok) {
                        float pm[8];
                        if (l == 0) {
                            const float br0 = C(0, kSBr0), br1 = C(0, kSBr1), bi0 = C(0, kSBi0), bi1 = C(0, kSBi1);
                            const float m0 = odd_r ? bi0 : br0, m1 = odd_r ? bi1 : br1;
#pragma unroll
                            for (int b = 0; b < 8; ++b)
                                pm[b] = t == 0 ? 0.0f : (((prev >> (8 * s + b)) & 1u) ? m1 : m0);
                        } else {
                            uint32_t v0, v1, v2, v3, v4, v5, v6, v7;
                            tmem_ld8(tacc, v0, v1, v2, v3, v4, v5, v6, v7);
                            asm volatile("tcgen05.wait::ld.sync.aligned;"
                                         : "+r"(v0), "+r"(v1), "+r"(v2), "+r"(v3), "+r"(v4), "+r"(v5), "+r"(v6),
                                           "+r"(v7)::"memory");
                            pm[0] = __uint_as_float(v0);
                            pm[1] = __uint_as_float(v1);
                            pm[2] = __uint_as_float(v2);
                            pm[3] = __uint_as_float(v3);
                            pm[4] = __uint_as_float(v4);
                            pm[5] = __uint_as_float(v5);
                            pm[6] = __uint_as_float(v6);
                            pm[7] = __uint_as_float(v7);
                        }
                        const float lr = C(l, kSLre), lis = odd_r ? C(l, kSLim) : -C(l, kSLim);
                        const uint32_t bh = tb(odd_r ? 1 : 0, 8 * s, j);
#pragma unroll
                        for (int k = 0; k < kMaxLs; ++k) {
                            if (k != l) continue;
#pragma unroll
                            for (int b = 0; b < 8; ++b) {
                                // own part m' = Re(lambda) m + sl Im(lambda) o + (own part
                                // of e^gamma B u), o the partner's part of the carry, sl =
                                // -1 on row 2j (real), +1 on row 2j + 1 (imaginary)
                                const float o = __shfl_xor_sync(0xffffffffu, cm[k][b], 1);
                                const float m = fmaf(lr, cm[k][b], fmaf(lis, o, pm[b]));
                                cm[k][b] = m;
                                tst(bh, b, op16s<F16>(m));
                            }
                        }
                    }
                    arrive_e2m();
                    // ---- y = Re(C h) + D u at the samples of this row's parity
                    wait_m2e();
                    if (ok) {
                        uint32_t v0, v1, v2, v3, v4, v5, v6, v7;
                        tmem_ld8(tacc, v0, v1, v2, v3, v4, v5, v6, v7);
                        asm volatile("tcgen05.wait::ld.sync.aligned;"
                                     : "+r"(v0), "+r"(v1), "+r"(v2), "+r"(v3), "+r"(v4), "+r"(v5), "+r"(v6),
                                       "+r"(v7)::"memory");
                        const float cv[8] = {__uint_as_float(v0), __uint_as_float(v1), __uint_as_float(v2),
                                             __uint_as_float(v3), __uint_as_float(v4), __uint_as_float(v5),
                                             __uint_as_float(v6), __uint_as_float(v7)};
                        const float d0 = C(l, kSD0), d1 = C(l, kSD1);
                        const uint32_t by = tb(0, 8 * s + (odd_r ? 1 : 0), j);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int b = 2 * i + (odd_r ? 1 : 0);
                            const float c = odd_r ? cv[2 * i + 1] : cv[2 * i];
                            float y;
                            if (l == 0) y = c + (t == 0 ? 0.0f : (((prev >> (8 * s + b)) & 1u) ? d1 : d0));
                            else y = fmaf(d0, xr[i], c);
                            tst(by, 2 * i, op16s<F16>(y));
                        }
                    }
                    arrive_e2m();
                    // ---- GLU: rows 2j (W_a y), 2j + 1 (W_g y); new layer input
                    wait_m2e();
                    if (ok) {
                        uint32_t v0, v1, v2, v3, v4, v5, v6, v7;
                        tmem_ld8(tacc, v0, v1, v2, v3, v4, v5, v6, v7);
                        asm volatile("tcgen05.wait::ld.sync.aligned;"
                                     : "+r"(v0), "+r"(v1), "+r"(v2), "+r"(v3), "+r"(v4), "+r"(v5), "+r"(v6),
                                       "+r"(v7)::"memory");
                        const float gv[8] = {__uint_as_float(v0), __uint_as_float(v1), __uint_as_float(v2),
                                             __uint_as_float(v3), __uint_as_float(v4), __uint_as_float(v5),
                                             __uint_as_float(v6), __uint_as_float(v7)};
                        const float ba = C(l, kSBa), bg = C(l, kSBg);
                        const uint32_t bx = tb(0, 8 * s + (odd_r ? 1 : 0), j);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float ve = gv[2 * i], vo = gv[2 * i + 1];
                            const float other = __shfl_xor_sync(0xffffffffu, odd_r ? ve : vo, 1);
                            const float a = (odd_r ? other : ve) + ba, gg = (odd_r ? vo : other) + bg;
                            const float x = a * (0.5f + 0.5f * tanh_approx(0.5f * gg)) + (l >= 1 ? xr[i] : 0.0f);
                            xr[i] = x;
                            tst(bx, 2 * i, op16s<F16>(x));
                        }
                    }
                    arrive_e2m();
                }
                // ---- readout and draws: warp 0, sample b by lane b
                wait_m2e();
                if (ok && warp == 0) {
                    uint32_t dvb;
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                                 : "=r"(dvb)
                                 : "r"(tmem + lane_off)
                                 : "memory");
                    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(dvb)::"memory");
                    const float d = __uint_as_float(dvb) + bd;
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
                tc_before();
                if (bar_or_s(!ok || *ab)) ok = false;
                prev = *(volatile uint32_t *)&M.spins;
            }
            if (ok && warp == 0 && logpsi && first + lane < n) logpsi[first + lane] = 0.5f * acc;
            // next block: the scan of its first site writes the tile after
            // every warp has passed the closing barrier above
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemS) : "memory");
    }
}

}  // namespace

bool lru_tc_sample_supported(int nL, int H) { return H == kHs && nL >= 1 && nL <= kMaxLs; }

size_t sample_lru_tc_smem_bytes(int nL) {
    return sizeof(MiscS) + 1024 + (size_t)(4 * nL - 1) * kSliceS + 1024 * ((kWdS + 1023) / 1024) + kTileS +
           (size_t)nL * kSCst * kHs * sizeof(float);
}

cudaError_t launch_sample_lru_tc(const float *pk, const LruLayout &f, bool f16, const uint8_t *wimg,
                                 const float *unif, int64_t n, int N, int u1, uint8_t *out, float *logpsi,
                                 int *status, int num_sms, cudaStream_t stream) {
    if (!lru_tc_sample_supported(f.nL, f.H)) return cudaErrorInvalidValue;
    const int n_slices = 4 * f.nL;  // the forward's image: its last slice holds w_d
    const size_t smem = sample_lru_tc_smem_bytes(f.nL);
    const int64_t nblk = (n + kBs - 1) / kBs;
    const int grid = (int)(nblk < num_sms ? nblk : num_sms);
    if (grid < 1) return cudaSuccess;
    cudaError_t e;
    if (f16) {
        e = cudaFuncSetAttribute(sample_lru_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        sample_lru_tc_kernel<true><<<grid, kEpiS + 32, smem, stream>>>(pk, f, wimg, n_slices, unif, n, N, u1, out,
                                                                        logpsi, status);
    } else {
        e = cudaFuncSetAttribute(sample_lru_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        sample_lru_tc_kernel<false><<<grid, kEpiS + 32, smem, stream>>>(pk, f, wimg, n_slices, unif, n, N, u1, out,
                                                                         logpsi, status);
    }
    return cudaGetLastError();
}

}  // namespace psr
