// Forward of the paper's deep 1D LRU ansatz (Sec. II.B Eq. lru, Sec. II.G 1D
// residual, Sec. III.B: each layer an LRU followed by a single-layer GLU) on
// the tensor cores, hidden d = d_h = 64 (the paper's Table IV width): FP16
// (or BF16) operands, FP32 accumulation in tensor memory, FP32 complex scan,
// GLU, residual and readout.
//
// The model is the one psr_lru.cu evaluates in FP32:
//   h_t = lambda h_{t-1} + e^gamma (B u_t),   y_t = Re(C h_t) + D u_t,
//   x_t = (W_a y_t + b_a) sigmoid(W_g y_t + b_g) + [l >= 1] u_t,
// with the two-logit readout.  Its dense products become three MMAs per
// layer, each with an M = 128 weight operand (A, K-major, 128-byte swizzle)
// and the sites as B (N = 128 columns):
//   e^gamma [B_re; B_im] u   rows 2j, 2j + 1 = unit j's real / imaginary part
//   [C_re, -C_im] [h_re; h_im]   rows 2j, 2j + 1 both unit j's, K = 128
//   [W_a; W_g] y     rows 2j, 2j + 1 = unit j's W_a / W_g row
// and the readout w_d x with w_d in row 32 q of every lane quarter q (each
// warp reads it from its lane 0 and takes 8 of the chunk's sites).  Layer
// 0's input is one-hot (Sec. II.F), so its B u and D u are lookups.  The
// thread pair of rows 2j, 2j + 1 shares unit j: both run its complex scan
// over the chunk, and the y and GLU epilogues split the sites by parity
// (even sites: row 2j), so the FP32 layer input u_t that D u and the residual
// need stays with the thread that made it (in its tensor-memory lane).
//
// Work layout: one persistent CTA per SM with two groups of 4 slots; a slot
// holds one 32-site chunk of one job (a sample, or a connected configuration
// resumed at the chunk of its first flipped site from the sample's FP32
// complex chunk carries), advances one chunk per step and takes the next job
// from a counter when its sequence ends.  Warpgroup s serves slot s of both
// groups; every stage of a chunk step (scan, y, GLU per layer, readout) runs
// for group 0 and then for group 1, so one group's MMAs (N = 128: its 4
// slots) run while the epilogue works on the other group.  The weights (12
// slices of 16 KB per chunk step at 3 layers) stream from L2 through a ring
// of slices (producer thread), each slice serving both groups; one thread
// issues the MMAs.  The complex carries of the slots stay in shared memory.
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

constexpr int kH = 64;              // hidden width of this kernel
constexpr int kCh = 32;             // sites per chunk (slot width)
constexpr int kSl = 4;              // slots per group (one per epilogue warpgroup)
constexpr int kGroups = 2;          // slot groups, a chunk step apart in phase
constexpr uint32_t kSliceL = 16384; // 128 rows x 64 inputs, 16-bit
constexpr int kMaxRingL = 12;
constexpr int kEpiL = 512;          // epilogue threads
constexpr int kMaxLL = 4;           // layers (rows of the slots' carries in shared memory)

// Tensor memory (columns): group g's accumulator at 128 g (B u, y, GLU and
// readout in turn: each MMA starts after the epilogue has read the previous
// one); warpgroup s's FP32 layer input u_t of group g at 256 + 32 s + 16 g.
// Shared memory: group g's B operand tile at 32 KB g, used in turn by x
// (K = 64), h (K = 128: h_re, then h_im) and y (K = 64).
constexpr uint32_t kTileG = 2 * 16384;
constexpr uint32_t kTilesBytes = kGroups * kTileG;
// per-unit constants of each layer in shared memory, [layer][kind][unit]:
// lambda (re, im), D (one-hot rows 0, 1 at layer 0; the diagonal above),
// b_a, b_g, and layer 0's one-hot e^gamma B u (re, im for inputs 0, 1)
enum { kCLre, kCLim, kCD0, kCD1, kCBa, kCBg, kCBr0, kCBr1, kCBi0, kCBi1, kCst };

template <bool F16>
constexpr uint32_t idesc_l() {
    return (1u << 4) | ((F16 ? 0u : 1u) << 7) | ((F16 ? 0u : 1u) << 10) | (0u << 15) | (0u << 16) |
           ((uint32_t)((kCh * kSl) >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ uint64_t kdesc_l(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(1024u >> 4) << 16) |
           ((uint64_t)(1024u >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

struct SlotL {
    int job;              // -1: needs a job, -2: none left
    int sample, p, q;     // configuration (p, q: flipped sites or -1)
    int c, c0, nch;       // current chunk, first chunk, chunks of the sequence
    int n_up;             // up spins before the current chunk
    int first;            // 1 in the job's first chunk (carries to load)
    float acc;            // sum of log P (mode 0) or of its differences (mode 1)
    float part[4];        // the last chunk's sums over sites 8 q .. 8 q + 7 (warp q4 = q)
    uint32_t cur, pb;     // spins of the current chunk and of the sites before (chunk_bits32)
};

struct MiscL {
    uint64_t full[kMaxRingL], empty[kMaxRingL];
    uint64_t e2m[kGroups], m2e[kGroups], go[2];
    uint32_t tmem_base;
    int abort_flag;
    int go_flag[2];
    SlotL slot[kGroups * kSl];
};

__device__ __forceinline__ bool wait_abl(uint32_t bar, uint32_t parity, const volatile int *ab) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u && (*ab || globaltimer() - t0 > kWaitNs)) return false;
    }
    return false;
}

__device__ __forceinline__ bool bar_or_l(uint32_t id, uint32_t n, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

// FP32 -> 16-bit operand, round to nearest even; FP16 saturates at +-65504
template <bool F16>
__device__ __forceinline__ uint16_t op16(float x) {
    uint16_t h;
    if (F16) asm("cvt.rn.satfinite.f16.f32 %0, %1;" : "=h"(h) : "f"(x));
    else asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(x));
    return h;
}

__device__ __forceinline__ void sts16(uint32_t a, uint16_t v) {
    asm volatile("st.shared.b16 [%0], %1;" ::"r"(a), "h"(v));
}

// op word of a slice: bit 0 K chunk of the B tile, bit 1 accumulate from the
// first K step, bit 2 last slice of its stage (commit to the epilogue).
// Every stage starts after an epilogue arrival of the same group.
enum { kLopKc = 1u, kLopAcc = 2u, kLopEnd = 4u };

template <bool F16>
__global__ void __launch_bounds__(kEpiL + 64, 1) lru_tc_kernel(const __grid_constant__ LruTcArgs A) {
    constexpr int NW = kEpiL / 32;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    MiscL &M = *reinterpret_cast<MiscL *>(smem_raw);
    uint8_t *tiles = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + sizeof(MiscL) + 1023) & ~uintptr_t(1023));
    uint8_t *ring = tiles + kTilesBytes;
    float *cst = reinterpret_cast<float *>(ring + (size_t)A.R * kSliceL);
    float *car = cst + A.nL * kCst * kH;  // complex carries [slot][layer][re, im][unit]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = A.R, nL = A.nL;
    const FwdGroup &G = A.g;
    const int N = G.N;
    const volatile int *ab = &M.abort_flag;
    const float *pk = A.pk;
    const LruLayout &f = A.f;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&M.tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < R; ++i) {
            mbar_init(smem_u32(&M.full[i]), 1);
            mbar_init(smem_u32(&M.empty[i]), 1);
        }
        for (int g = 0; g < kGroups; ++g) {
            mbar_init(smem_u32(&M.e2m[g]), kEpiL / 32);  // one arrival per epilogue warp
            mbar_init(smem_u32(&M.m2e[g]), 1);
        }
        mbar_init(smem_u32(&M.go[0]), 1);
        mbar_init(smem_u32(&M.go[1]), 1);
        M.abort_flag = 0;
        M.go_flag[0] = 1;
        M.go_flag[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < kGroups * kSl) {
        M.slot[tid].job = -1;
        M.slot[tid].acc = 0.0f;
        for (int q = 0; q < 4; ++q) M.slot[tid].part[q] = 0.0f;
    }
    for (int i = tid; i < nL * kCst * kH; i += blockDim.x) {
        const int u = i % kH, k = (i / kH) % kCst, l = i / (kH * kCst);
        int64_t o = -1;
        switch (k) {
            case kCLre: o = f.lre[l] + u; break;
            case kCLim: o = f.lim[l] + u; break;
            case kCD0: o = f.D[l] + u; break;
            case kCD1: o = l == 0 ? f.D[0] + kH + u : -1; break;
            case kCBa: o = f.ba[l] + u; break;
            case kCBg: o = f.bg[l] + u; break;
            case kCBr0: o = l == 0 ? f.BreT[0] + u : -1; break;
            case kCBr1: o = l == 0 ? f.BreT[0] + kH + u : -1; break;
            case kCBi0: o = l == 0 ? f.BimT[0] + u : -1; break;
            default: o = l == 0 ? f.BimT[0] + kH + u : -1; break;
        }
        // layer 0's one-hot B u lookups carry the factor e^gamma
        cst[i] = o >= 0 ? (k >= kCBr0 ? pk[f.gam[0] + u] * pk[o] : pk[o]) : 0.0f;
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = M.tmem_base;
    if (tmem != 0) {
        if (tid == 0) set_status(A.status, PSR_EDEVICE);
        M.abort_flag = 1;
    }
    if (tid == 0) mbar_arrive(smem_u32(&M.go[0]));
    __syncthreads();
    const long long njobs = A.mode == 1 ? (long long)*G.n_jobs_dev : (long long)G.n_jobs;

    if (warp == NW) {
        // ------------------------------------------------ producer: weight stream
        if (lane == 0 && !M.abort_flag) {
            uint32_t q = 0, slot = 0, round = 0;
            const uint32_t fb = smem_u32(&M.full[0]), ebar = smem_u32(&M.empty[0]), rb = smem_u32(ring);
            for (uint32_t row = 0;; ++row) {
                if (!wait_abl(smem_u32(&M.go[row & 1]), (row >> 1) & 1, ab)) break;
                if (!*(volatile int *)&M.go_flag[row & 1]) break;
                bool ok = true;
                const uint8_t *src = A.wimg;
                for (int i = 0; i < A.n_slices; ++i, ++q, src += kSliceL) {
                    if (round > 0 && !wait_abl(ebar + 8 * slot, (round - 1) & 1, ab)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_tx(fb + 8 * slot, kSliceL);
                    bulk_g2s(rb + slot * kSliceL, src, kSliceL, fb + 8 * slot);
                    if (++slot == (uint32_t)R) {
                        slot = 0;
                        ++round;
                    }
                }
                if (!ok) break;
            }
            const uint32_t last = q < (uint32_t)R ? q : (uint32_t)R;
            for (uint32_t t = 0; t < last; ++t) {
                const uint32_t qq = q - 1 - t;
                if (!mbar_wait(smem_u32(&M.full[qq % R]), (qq / R) & 1)) set_status(A.status, PSR_ETIMEOUT);
            }
            if (*ab) set_status(A.status, PSR_ETIMEOUT);
        }
    } else if (warp == NW + 1) {
        // ------------------------------------------------ MMA issue
        // Each stage (the slices up to one marked kLopEnd) runs for group 0,
        // then for group 1, each after that group's epilogue arrival; the
        // stage's ring slots are released after group 1's MMAs.
        if (lane == 0 && !M.abort_flag) {
            uint32_t q = 0, pe0 = 0, pe1 = 0;
            const uint32_t fb = smem_u32(&M.full[0]), ebar = smem_u32(&M.empty[0]);
            const uint64_t tdesc0 = kdesc_l(smem_u32(tiles)), rd = kdesc_l(smem_u32(ring));
            bool ok = true;
            for (uint32_t row = 0; ok; ++row) {
                if (!wait_abl(smem_u32(&M.go[row & 1]), (row >> 1) & 1, ab)) {
                    ok = false;
                    break;
                }
                if (!*(volatile int *)&M.go_flag[row & 1]) break;
                for (int i = 0; i < A.n_slices && ok;) {
                    int ns = 1;
                    while (!(A.op[i + ns - 1] & kLopEnd)) ++ns;
#pragma unroll
                    for (int g = 0; g < kGroups; ++g) {
                        if (!ok) break;
                        uint32_t &pe = g ? pe1 : pe0;
                        if (!wait_abl(smem_u32(&M.e2m[g]), pe, ab)) {
                            ok = false;
                            break;
                        }
                        pe ^= 1u;
                        tc_after();
                        for (int k = 0; k < ns; ++k) {
                            const uint32_t qq = q + k, sl = qq % R;
                            if (g == 0 && !wait_abl(fb + 8 * sl, (qq / R) & 1, ab)) {
                                ok = false;
                                break;
                            }
                            const uint32_t op = A.op[i + k];
                            const uint64_t ad = rd + (uint64_t)(sl * (kSliceL >> 4)),
                                           bd = tdesc0 + (uint64_t)((g * kTileG + (op & kLopKc) * 16384u) >> 4);
                            const uint32_t d = tmem + 128u * g;
                            mma_ss<idesc_l<F16>()>(d, ad, bd, (op & kLopAcc) ? 1u : 0u);
                            mma_ss<idesc_l<F16>()>(d, ad + 2, bd + 2, 1u);
                            mma_ss<idesc_l<F16>()>(d, ad + 4, bd + 4, 1u);
                            mma_ss<idesc_l<F16>()>(d, ad + 6, bd + 6, 1u);
                        }
                        if (!ok) break;
                        mma_commit(smem_u32(&M.m2e[g]));
                    }
                    if (!ok) break;
                    for (int k = 0; k < ns; ++k) mma_commit(ebar + 8 * ((q + k) % R));
                    q += ns;
                    i += ns;
                }
            }
            const uint32_t last = q < (uint32_t)R ? q : (uint32_t)R;
            for (uint32_t t = 0; t < last; ++t) {
                const uint32_t qq = q - 1 - t;
                if (!mbar_wait(smem_u32(&M.empty[qq % R]), (qq / R) & 1)) set_status(A.status, PSR_ETIMEOUT);
            }
            if (!ok) {
                M.abort_flag = 1;
                set_status(A.status, PSR_ETIMEOUT);
            }
        }
    } else {
        // ------------------------------------------------ epilogue
        // warpgroup s = slot s of each group (columns 32 s ..); warp w reads
        // TMEM lanes 32 (w & 3) + lane = row r of every accumulator
        const int s = warp >> 2, q4 = warp & 3, r = 32 * q4 + lane;
        const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
        const int j = r >> 1;        // unit of rows 2j, 2j + 1
        const bool odd_r = r & 1;
        auto C = [&](int l, int k) { return cst[(l * kCst + k) * kH + j]; };
        // accumulator columns of this thread's slot in group g; its layer input
        auto tacc = [&](int g) { return tmem + lane_off + 128u * g + (uint32_t)(kCh * s); };
        auto tres = [&](int g) { return tmem + lane_off + 256u + (uint32_t)(32 * s + 16 * g); };
        // Element k of row n of a B tile (K-major, 128-byte swizzle: the
        // 16-byte group k >> 3 of row n sits at group (k >> 3) ^ (n & 7)).
        // tb(g, kc, nb, k) is the address of element k of row nb of group g's
        // tile; element k of row nb + dt is at (tb ^ ((dt & 7) << 4)) + 128 dt
        // whenever the low three bits of nb and dt share no bit.
        const uint32_t tiles_s = smem_u32(tiles);
        auto tb = [&](int g, int kc, int nb, int k) -> uint32_t {
            return tiles_s + (uint32_t)g * kTileG + (uint32_t)kc * 16384u + (uint32_t)nb * 128u +
                   ((uint32_t)((k >> 3) ^ (nb & 7)) << 4) + (uint32_t)(k & 7) * 2u;
        };
        auto tst = [&](uint32_t b, int dt, uint16_t v) { sts16((b ^ ((uint32_t)(dt & 7) << 4)) + 128u * dt, v); };
        const float bd = pk[f.bd];
        auto carp = [&](int g, int l) { return car + ((s + kSl * g) * kMaxLL + l) * 2 * kH + j; };
        float lref[kGroups] = {0.0f, 0.0f};
        uint32_t pm0 = 0, pm1 = 0;
        bool ok = !M.abort_flag;

        // Inside a chunk step the epilogue warps synchronise with the MMA
        // thread only: each warp waits for the group's MMAs (lane 0 polls,
        // the warp takes its answer) and arrives on the group's e2m barrier
        // once its tensor-memory reads and tile stores are done.  A warp whose
        // wait expires sets the abort flag, which ends every other wait, and
        // all warps meet at the step's closing barrier.
        auto wait_m2e = [&](int g) {
            uint32_t &pm = g ? pm1 : pm0;
            bool w = false;
            if (lane == 0) w = ok && wait_abl(smem_u32(&M.m2e[g]), pm, ab);
            w = __shfl_sync(0xffffffffu, w ? 1 : 0, 0) != 0;
            if (!w && ok && lane == 0) {
                M.abort_flag = 1;
                set_status(A.status, PSR_ETIMEOUT);
            }
            ok = ok && w;
            pm ^= 1u;
            tc_after();
        };
        auto arrive_e2m = [&](int g) {
            fence_proxy_async();
            tc_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&M.e2m[g]));
        };
        // carry of layer l entering the slot's chunk (stored as the chunk's
        // checkpoint in mode 0)
        auto carry_in = [&](int g, int l, const SlotL &st, float &zr, float &zi) {
            const float *cp = carp(g, l);
            zr = cp[0];
            zi = cp[kH];
            if (G.carries_out && !odd_r) {
                float *co = G.carries_out + (((int64_t)st.sample * st.nch + st.c) * nL + l) * 2 * kH;
                co[j] = zr;
                co[kH + j] = zi;
            }
        };
        auto carry_out = [&](int g, int l, float zr, float zi) {
            if (!odd_r) {
                float *cp = carp(g, l);
                cp[0] = zr;
                cp[kH] = zi;
            }
        };
        // h_t = lambda h_{t-1} + e^gamma B u_t over 16 sites (c0 .. c0 + 15)
        // of the slot, on this thread's part m of h (real part: row 2j,
        // imaginary part: row 2j + 1) and the partner's part o:
        //   m' = Re(lambda) m + sl Im(lambda) o + pm,  o' = Re(lambda) o - sl Im(lambda) m + po
        // with sl = -1 on row 2j and +1 on row 2j + 1, pm/po the two parts of
        // e^gamma B u_t; m to the h tile (K chunk 0: real, 1: imaginary)
        auto scan16 = [&](int g, int c0, const float (&pm)[16], const float (&po)[16], float lr, float lis, float &m,
                          float &o) {
            const uint32_t b = tb(g, odd_r ? 1 : 0, kCh * s + c0, j);
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const float nm = fmaf(lr, m, fmaf(lis, o, pm[t]));
                const float no = fmaf(lr, o, fmaf(-lis, m, po[t]));
                m = nm;
                o = no;
                tst(b, t, op16<F16>(m));
            }
        };
        // ---- the complex scan of layer l over the slot's chunk: B u from a
        // lookup of the one-hot input (layer 0) or from the MMA (rows 2j: re,
        // 2j + 1: im)
        auto scan_stage = [&](int g, int l) {
            const SlotL &st = M.slot[s + kSl * g];
            if (st.job < 0) return;
            const uint32_t pb = st.pb;
            const int t0 = st.c * kCh;
            const float lr = C(l, kCLre), lis = odd_r ? C(l, kCLim) : -C(l, kCLim);
            float zr, zi;
            carry_in(g, l, st, zr, zi);
            float m = odd_r ? zi : zr, o = odd_r ? zr : zi;
            if (l == 0) {
                const float br0 = C(0, kCBr0), br1 = C(0, kCBr1), bi0 = C(0, kCBi0), bi1 = C(0, kCBi1);
                const float pm0_ = odd_r ? bi0 : br0, pm1_ = odd_r ? bi1 : br1;
                const float po0_ = odd_r ? br0 : bi0, po1_ = odd_r ? br1 : bi1;
#pragma unroll 1
                for (int hh = 0; hh < 2; ++hh) {
                    float pm[16], po[16];
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        const int tc = 16 * hh + t;
                        const bool first = (t0 + tc == 0), sb = (pb >> tc) & 1u;
                        pm[t] = first ? 0.0f : (sb ? pm1_ : pm0_);
                        po[t] = first ? 0.0f : (sb ? po1_ : po0_);
                    }
                    scan16(g, 16 * hh, pm, po, lr, lis, m, o);
                }
            } else {
#pragma unroll 1
                for (int hh = 0; hh < 2; ++hh) {
                    uint32_t v[16];
                    tmem_ld16(tacc(g) + 16 * hh, v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" : PSR_P16(v, 0)::"memory");
                    float pm[16], po[16];
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        pm[t] = __uint_as_float(v[t]);
                        po[t] = __shfl_xor_sync(0xffffffffu, pm[t], 1);
                    }
                    scan16(g, 16 * hh, pm, po, lr, lis, m, o);
                }
            }
            carry_out(g, l, odd_r ? o : m, odd_r ? m : o);
        };
        // ---- y = Re(C h) + D u: unit j at the sites of this row's parity
        auto y_stage = [&](int g, int l) {
            const SlotL &st = M.slot[s + kSl * g];
            if (st.job < 0) return;
            const uint32_t pb = st.pb;
            const int t0 = st.c * kCh;
            const float d0 = C(l, kCD0), d1 = C(l, kCD1);
            const uint32_t by = tb(g, 0, kCh * s + (odd_r ? 1 : 0), j);
            uint32_t v0[16], v1[16], xv[16];
            tmem_ld16(tacc(g), v0);
            tmem_ld16(tacc(g) + 16, v1);
            if (l > 0) {
                tmem_ld16(tres(g), xv);
                asm volatile("tcgen05.wait::ld.sync.aligned;" : PSR_P16(v0, 0), PSR_P16(v1, 0), PSR_P16(xv, 0)::"memory");
            } else {
                tmem_wait_ld16x2(v0, v1);
            }
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int ii = 8 * hh + i, t = 2 * ii + (odd_r ? 1 : 0);
                    const uint32_t cv = hh ? (odd_r ? v1[2 * i + 1] : v1[2 * i]) : (odd_r ? v0[2 * i + 1] : v0[2 * i]);
                    const float c = __uint_as_float(cv);
                    float y;
                    if (l == 0) {
                        const bool first = (t0 + t == 0), sb = (pb >> t) & 1u;
                        y = c + (first ? 0.0f : (sb ? d1 : d0));
                    } else {
                        y = fmaf(d0, __uint_as_float(xv[ii]), c);
                    }
                    tst(by, 2 * ii, op16<F16>(y));
                }
            }
        };
        // ---- GLU: rows 2j (W_a y), 2j + 1 (W_g y); the new layer input x
        // (+ the residual above layer 0) to the x tile and to tensor memory
        auto glu_stage = [&](int g, int l) {
            const SlotL &st = M.slot[s + kSl * g];
            if (st.job < 0) return;
            const float ba = C(l, kCBa), bg = C(l, kCBg);
            const uint32_t bx = tb(g, 0, kCh * s + (odd_r ? 1 : 0), j);
            uint32_t v0[16], v1[16], xv[16];
            tmem_ld16(tacc(g), v0);
            tmem_ld16(tacc(g) + 16, v1);
            if (l > 0) {
                tmem_ld16(tres(g), xv);
                asm volatile("tcgen05.wait::ld.sync.aligned;" : PSR_P16(v0, 0), PSR_P16(v1, 0), PSR_P16(xv, 0)::"memory");
            } else {
                tmem_wait_ld16x2(v0, v1);
            }
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    // each thread sends its partner the value at the partner's site
                    const float ve = __uint_as_float(hh ? v1[2 * i] : v0[2 * i]),
                                vo = __uint_as_float(hh ? v1[2 * i + 1] : v0[2 * i + 1]);
                    const float other = __shfl_xor_sync(0xffffffffu, odd_r ? ve : vo, 1);
                    const float a = (odd_r ? other : ve) + ba, gg = (odd_r ? vo : other) + bg;
                    const int ii = 8 * hh + i;
                    const float x = a * (0.5f + 0.5f * tanh_approx(0.5f * gg)) + (l >= 1 ? __uint_as_float(xv[ii]) : 0.0f);
                    xv[ii] = __float_as_uint(x);
                    tst(bx, 2 * ii, op16<F16>(x));
                }
            }
            tmem_st16(tres(g), xv);
            tmem_wait_st();
        };
        // ---- readout: d_t = w_d x_t + b_d in row 32 q4 of every lane
        // quarter (lane 0 of each warp); warp q4 takes sites 8 q4 .. 8 q4 + 7,
        // site 8 q4 + i by lane i, and leaves its sum in the slot's part[q4]
        auto readout = [&](int g) {
            SlotL &st = M.slot[s + kSl * g];
            if (st.job < 0) return;
            const uint32_t cur = st.cur;
            const int t0 = st.c * kCh;
            uint32_t v0, v1, v2, v3, v4, v5, v6, v7;
            tmem_ld8(tacc(g) + 8 * q4, v0, v1, v2, v3, v4, v5, v6, v7);
            asm volatile("tcgen05.wait::ld.sync.aligned;"
                         : "+r"(v0), "+r"(v1), "+r"(v2), "+r"(v3), "+r"(v4), "+r"(v5), "+r"(v6), "+r"(v7)::"memory");
            const uint32_t vv[8] = {v0, v1, v2, v3, v4, v5, v6, v7};
            float dv = 0.0f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float x = __shfl_sync(0xffffffffu, __uint_as_float(vv[i]), 0);
                if (i == lane) dv = x;
            }
            const int t = 8 * q4 + lane, tt = t0 + t;
            float lp = 0.0f;
            if (lane < 8 && tt < N) {
                const float d = dv + bd;
                const int sv = (cur >> t) & 1u;
                const int nu = st.n_up + __popc(cur & ((1u << t) - 1u));
                lp = site_logp_fast(d, sv, u1_forced(G.u1, N, tt, nu));
                if (A.mode == 0 && G.logp_out) G.logp_out[(int64_t)st.sample * N + tt] = lp;
                if (A.mode == 1) lp -= lref[g];
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) lp += __shfl_xor_sync(0xffffffffu, lp, o);
            if (lane == 0) st.part[q4] = lp;
        };
        // adds the last chunk's four partial sums to the job's sum, in a
        // fixed order
        auto fold = [&](SlotL &st) {
            st.acc += (st.part[0] + st.part[1]) + (st.part[2] + st.part[3]);
            st.part[0] = st.part[1] = st.part[2] = st.part[3] = 0.0f;
        };
        // the 32 sites' 32-bit spins of the slot's current chunk: cur (bit t =
        // s_{t0+t}) and prevbits (bit t = s_{t0+t-1}, 0 at the first site)
        auto chunk_spins = [&](const SlotL &st, uint32_t &cur, uint32_t &prevbits) {
            const uint64_t *row = G.bits + (int64_t)st.sample * G.W;
            uint32_t prev;
            chunk_bits32(row, st.c * kCh, st.p, st.q, cur, prev);
            const int nvalid = min(kCh, N - st.c * kCh);
            if (nvalid < 32) cur &= (1u << nvalid) - 1u;
            prevbits = (cur << 1) | prev;
        };

        for (uint32_t row_it = 0; ok; ++row_it) {
            // ---- slot update (lanes 0, 1 of warp 4 s: slots s, 4 + s)
            if (q4 == 0 && lane < kGroups) {
                SlotL &st = M.slot[s + kSl * lane];
                fold(st);
                if (row_it > 0 && st.job >= 0 && st.c + 1 >= st.nch) {
                    G.out[st.job] = 0.5f * st.acc;  // the job's last chunk is done
                }
                if (st.job != -2) {
                    if (st.job == -1 || st.c + 1 >= st.nch) {
                        const unsigned long long nj = atomicAdd(A.job_counter, 1ull);
                        if ((long long)nj >= njobs) {
                            st.job = -2;
                        } else {
                            int sample = (int)nj, p = -1, q = -1, c0 = 0;
                            if (A.mode == 1) {
                                const int32_t *e = G.entries + 3 * nj;
                                sample = e[0];
                                p = e[1];
                                q = e[2];
                                c0 = p / kCh;
                            }
                            st.job = (int)nj;
                            st.sample = sample;
                            st.p = p;
                            st.q = q;
                            st.c0 = c0;
                            st.c = c0;
                            st.nch = (N + kCh - 1) / kCh;
                            st.first = 1;
                            st.acc = 0.0f;
                            st.n_up = G.u1 ? count_up_before(G.bits + (int64_t)sample * G.W, c0 * kCh) : 0;
                            uint32_t cur, pb;
                            chunk_spins(st, cur, pb);
                            st.cur = cur;
                            st.pb = pb;
                        }
                    } else {
                        st.n_up += __popc(st.cur);
                        st.c += 1;
                        st.first = 0;
                        uint32_t cur, pb;
                        chunk_spins(st, cur, pb);
                        st.cur = cur;
                        st.pb = pb;
                    }
                }
            }
            if (bar_or_l(1, kEpiL, !ok || *ab)) {
                ok = false;
                break;
            }
            if (tid == 0) {
                bool more = false;
                for (int k = 0; k < kGroups * kSl; ++k)
                    if (M.slot[k].job >= 0 && M.slot[k].c + 1 < M.slot[k].nch) more = true;
                if (!more) more = (long long)atomicAdd(A.job_counter, 0ull) < njobs;
                M.go_flag[(row_it + 1) & 1] = more ? 1 : 0;
                mbar_arrive(smem_u32(&M.go[(row_it + 1) & 1]));
            }
#pragma unroll
            for (int g = 0; g < kGroups; ++g) {
                const SlotL &st = M.slot[s + kSl * g];
                const bool act = st.job >= 0;
                const int t0 = act ? st.c * kCh : 0;
                // carries entering the job's first chunk (zero, or the
                // sample's checkpoint in mode 1), all layers' loads at once
                if (act && st.first && !odd_r) {
                    const bool ld = A.mode == 1 && st.c0 > 0;
                    const float *cin = G.carries_in + ((int64_t)st.sample * st.nch + st.c0) * nL * 2 * kH;
#pragma unroll
                    for (int k = 0; k < kMaxLL; ++k) {
                        if (k >= nL) break;
                        float *cp = carp(g, k);
                        cp[0] = ld ? cin[k * 2 * kH + j] : 0.0f;
                        cp[kH] = ld ? cin[k * 2 * kH + kH + j] : 0.0f;
                    }
                }
                // log P of the reference configuration at this lane's site
                // (mode 1 readout), loaded ahead of the step
                lref[g] = 0.0f;
                if (A.mode == 1 && act && lane < 8 && t0 + 8 * q4 + lane < N)
                    lref[g] = G.logp_ref[(int64_t)st.sample * N + t0 + 8 * q4 + lane];
            }
            __syncwarp();  // the carries written by the even lanes, before both lanes read them

            // ---- the layers: every stage for group 0, then for group 1, so
            // that one group's MMAs run while the other's epilogue works
#pragma unroll
            for (int g = 0; g < kGroups; ++g) {
                if (ok) scan_stage(g, 0);
                arrive_e2m(g);
            }
#pragma unroll 1
            for (int l = 0; l < nL; ++l) {
                if (l > 0) {
#pragma unroll
                    for (int g = 0; g < kGroups; ++g) {
                        wait_m2e(g);
                        if (ok) scan_stage(g, l);
                        arrive_e2m(g);
                    }
                }
#pragma unroll
                for (int g = 0; g < kGroups; ++g) {
                    wait_m2e(g);
                    if (ok) y_stage(g, l);
                    arrive_e2m(g);
                }
#pragma unroll
                for (int g = 0; g < kGroups; ++g) {
                    wait_m2e(g);
                    if (ok) glu_stage(g, l);
                    arrive_e2m(g);
                }
            }
#pragma unroll
            for (int g = 0; g < kGroups; ++g) {
                wait_m2e(g);
                if (ok) readout(g);
            }
            tc_before();
            if (bar_or_l(1, kEpiL, !ok)) {
                ok = false;
                break;
            }
            if (!*(volatile int *)&M.go_flag[(row_it + 1) & 1]) {
                if (q4 == 0 && lane < kGroups) {
                    SlotL &sf = M.slot[s + kSl * lane];
                    fold(sf);
                    if (sf.job >= 0) G.out[sf.job] = 0.5f * sf.acc;
                }
                break;
            }
        }
        if (!ok) {
            M.abort_flag = 1;
            set_status(A.status, PSR_ETIMEOUT);
        }
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// Weight slices (128 rows x 64 inputs) in the MMA thread's order, from the
// packed FP32 matrices (transposed: M^T[k][j]).
struct LruKinds {
    int n;
    uint8_t kind[kLruSchedMax];
};

template <bool F16>
__global__ void pack_lru_tc_kernel(const float *__restrict__ pk, LruLayout f, LruKinds kd,
                                   uint8_t *__restrict__ wimg) {
    constexpr int H = kH;
    const int64_t total = (int64_t)kd.n * 1024;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(id >> 10), m = (int)((id >> 3) & 127), c = (int)(id & 7);
        const int code = kd.kind[i], ty = code >> 4, l = code & 15;
        uint32_t w[4];
#pragma unroll
        for (int e2 = 0; e2 < 4; ++e2) {
            float v2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = 8 * c + 2 * e2 + h;
                float v = 0.0f;
                switch (ty) {
                    case 0:  // e^gamma B
                        v = pk[f.gam[l] + (m >> 1)] * pk[((m & 1) ? f.BimT[l] : f.BreT[l]) + (int64_t)k * H + (m >> 1)];
                        break;
                    case 1: v = pk[f.CreT[l] + (int64_t)k * H + (m >> 1)]; break;                          // C_re
                    case 2: v = -pk[f.CimT[l] + (int64_t)k * H + (m >> 1)]; break;                         // -C_im
                    case 3: v = pk[((m & 1) ? f.WgT[l] : f.WaT[l]) + (int64_t)k * H + (m >> 1)]; break;   // W_a, W_g
                    default: if ((m & 31) == 0) v = pk[f.wd + k]; break;                                  // w_d
                }
                v2[h] = v;
            }
            w[e2] = (uint32_t)op16<F16>(v2[0]) | ((uint32_t)op16<F16>(v2[1]) << 16);
        }
        *reinterpret_cast<uint4 *>(wimg + (size_t)i * kSliceL + m * 128 + ((c ^ (m & 7)) << 4)) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
}

}  // namespace

// Slices of one chunk step and the MMA thread's op words (kLopKc, kLopAcc,
// kLopEnd); kind[i] = matrix type << 4 | layer.
int lru_tc_schedule(int nL, uint8_t *kind, uint32_t *op) {
    int n = 0;
    auto add = [&](int ty, int l, uint32_t fl) {
        kind[n] = (uint8_t)(ty << 4 | l);
        op[n] = fl;
        ++n;
    };
    for (int l = 0; l < nL; ++l) {
        if (l > 0) add(0, l, kLopEnd);  // e^gamma B u: after the previous GLU (x ready)
        add(1, l, 0);                   // Re(C h), K chunk 0 (h_re): after the scan
        add(2, l, kLopKc | kLopAcc | kLopEnd);
        add(3, l, kLopEnd);             // [W_a; W_g] y: y ready
    }
    add(4, 0, kLopEnd);  // readout: x of the last layer ready
    return n;
}

bool lru_tc_supported(int nL, int H) { return H == kH && nL >= 1 && nL <= kMaxLL && 4 * nL <= kLruSchedMax; }

size_t lru_tc_weight_bytes(int nL) { return (size_t)(4 * nL) * kSliceL; }

cudaError_t launch_pack_lru_tc(const float *pk, const LruLayout &f, bool f16, uint8_t *wimg, cudaStream_t stream) {
    LruKinds kd{};
    uint32_t op[kLruSchedMax];
    kd.n = lru_tc_schedule(f.nL, kd.kind, op);
    const int blocks = (int)(((int64_t)kd.n * 1024 + 255) / 256);
    if (f16) pack_lru_tc_kernel<true><<<blocks, 256, 0, stream>>>(pk, f, kd, wimg);
    else pack_lru_tc_kernel<false><<<blocks, 256, 0, stream>>>(pk, f, kd, wimg);
    return cudaGetLastError();
}

cudaError_t launch_lru_tc(LruTcArgs a, int grid, cudaStream_t stream) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    uint8_t kind[kLruSchedMax];
    a.n_slices = lru_tc_schedule(a.nL, kind, a.op);
    const size_t base = sizeof(MiscL) + 1024 + kTilesBytes + (size_t)a.nL * kCst * kH * sizeof(float) +
                        (size_t)kGroups * kSl * kMaxLL * 2 * kH * sizeof(float);
    if ((size_t)optin < base + 2 * kSliceL) return cudaErrorInvalidConfiguration;
    int R = (int)(((size_t)optin - base) / kSliceL);
    a.R = R > kMaxRingL ? kMaxRingL : R;
    const size_t smem = base + (size_t)a.R * kSliceL;
    if (grid < 1) grid = 1;
    if (a.f16) {
        e = cudaFuncSetAttribute(lru_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        lru_tc_kernel<true><<<grid, kEpiL + 64, smem, stream>>>(a);
    } else {
        e = cudaFuncSetAttribute(lru_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        lru_tc_kernel<false><<<grid, kEpiL + 64, smem, stream>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace psr
