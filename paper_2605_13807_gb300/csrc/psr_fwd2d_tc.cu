// Forward of the paper's two-dimensional patched minGRU (Sec. II.F,
// two-dimensional recurrences; Sec. II.G residual and GELU) on the tensor
// cores: BF16 operands, FP32 accumulation in tensor memory, FP32 gates,
// scan, GELU and softmax.
//
// The model is the one psr_fwd2d.cu evaluates in FP32 (2 x 2 patches along
// the zigzag path of the patch lattice, row by row: within a patch row the
// gates and candidates of all sites are one batched projection, the h_V part
// acting on the previous row's states, followed by the scan
// h = a h_H + (1 - a) h~ along the row).  Here every contraction of a row is
// a tcgen05 MMA with the weights as the A operand (M = 128 hidden units, one
// or two halves) and the row's sites as B (N = 128 columns):
//   z = W_z x,  c = W_hx x + W_hv h_V,  y = D x + C h,  logits = W_o x.
// Layer 0's input is the one-hot pair (v_H, v_V) of 32 entries, zero-padded
// to one 64-wide K chunk.
//
// Work layout.  One persistent CTA per SM holds 128 site columns cut into S
// slots of W = 8 ceil(P_x / 8) columns; each slot evaluates one job
// (configuration) and advances one patch row per step, so all slots share
// every weight fetch.  A slot whose job has finished takes the next job from
// a counter.  The weights (about 1.7 MB per row step at d_h = 256) do not fit
// in shared memory: they are stored once, in MMA order, as 16 KB slices
// (128 rows x 64 BF16, 128-byte swizzle) and streamed through a ring of
// slices by bulk copies, from L2, where every CTA's stream hits.
//
// Roles: H epilogue threads (thread j = hidden unit j: its tensor-memory lane
// holds unit j's accumulators for all 128 columns), one producer thread (the
// weight stream) and one MMA thread.  Per row step and layer:
//   MMA  z, c (needs x, then h_V)  ->  epilogue: gates and scan, h -> smem
//   MMA  y = D x + C h             ->  epilogue: GELU(y + residual) -> x
// then the readout MMA and the masked 16-way softmax of every patch.
// The next row's h_V is this row's h, path-reversed (consecutive rows run in
// opposite directions); the scan writes it to global memory as a BF16 image
// in the tile layout, and the next row bulk-copies it into the h tile.  In
// mode 0 these images are the row checkpoints that mode 1 (connected
// configurations, resumed at the patch row of the first flipped spin) reads.
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

constexpr int kCols = 128;          // site columns per CTA (MMA N)
constexpr uint32_t kSlice = 16384;  // 128 rows x 64 BF16
constexpr int kMaxSlots = 16;
constexpr int kMaxRing = 10;

// kind::f16, D = F32, A = B = FP16 (F16) or BF16, both K-major, M = 128,
// N = 128.
template <bool F16>
constexpr uint32_t idesc2() {
    return (1u << 4) | ((F16 ? 0u : 1u) << 7) | ((F16 ? 0u : 1u) << 10) | (0u << 15) | (0u << 16) |
           ((uint32_t)(kCols >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// Descriptor of a K-major, 128-byte-swizzled operand: 8-row atoms of 1024
// bytes stacked along M (or N); K = 16 step kk is 32 bytes along the row.
__device__ __forceinline__ uint64_t kdesc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(1024u >> 4) << 16) |
           ((uint64_t)(1024u >> 4) << 32) | (1ull << 46) | (2ull << 61);
}
__device__ __forceinline__ uint64_t kstep(int kk) { return (uint64_t)((kk * 32) >> 4); }

constexpr int kEpi = 512;  // epilogue threads: 512 / H per hidden unit

struct Slot2 {
    int job;              // -1: needs a job, -2: none left (a launch holds < 2^31 jobs)
    int sample, p, q;     // configuration (p, q: flipped sites or -1)
    int row, r0, n_up;    // current patch row, first row, up spins before it
    float acc;            // sum of log P (mode 0) or of its differences (mode 1)
    float part[4];        // the row's readout sums, per 8-column chunk
    uint8_t v[32];        // patch values of the current row, by column
    uint8_t vprev[32];    // previous row's values, by column
};

struct Misc2 {
    uint64_t full[kMaxRing], empty[kMaxRing];
    uint64_t e2m[2], m2e[2], hv, imgw, go[2];  // e2m, m2e: per unit half
    uint32_t tmem_base;
    int abort_flag;
    int go_flag[2];
    uint32_t hv_armed;                           // h_V image loads issued
    Slot2 slot[kMaxSlots];
};

// Bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool wait_ab(uint32_t bar, uint32_t parity, const volatile int *ab) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u && (*ab || globaltimer() - t0 > kWaitNs)) return false;
    }
    return false;
}

__device__ __forceinline__ int seq_pos2d(int Lx, int i, int j) {
    return j * Lx + ((j & 1) ? (Lx - 1 - i) : i);
}

// Value (0..15) of patch (pi, pj): spin (2 pi + dx, 2 pj + dy) is bit
// 2 dy + dx, with sites p and q flipped.
__device__ __forceinline__ int patch_value(const uint8_t *s, int Lx, int pi, int pj, int p, int q) {
    int v = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int pos = seq_pos2d(Lx, 2 * pi + (b & 1), 2 * pj + (b >> 1));
        v |= ((int)(s[pos] & 1u) ^ (pos == p) ^ (pos == q)) << b;
    }
    return v;
}

// Named barrier `id` of `n` threads.
__device__ __forceinline__ void named_bar(uint32_t id, uint32_t n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Named barrier that also ORs a flag over its threads, so that they all
// take the same exit.
__device__ __forceinline__ bool named_bar_or(uint32_t id, uint32_t n, bool v) {
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
// all epilogue threads (barrier 1)
__device__ __forceinline__ bool epi_bar_or(bool v) { return named_bar_or(1, kEpi, v); }

// Bulk copy shared -> global (bulk-group completion).
__device__ __forceinline__ void bulk_s2g(void *dst, uint32_t src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Operand bits of an FP32 value, rounded to nearest: FP16 (values beyond the
// largest finite FP16 saturate to it) or BF16.
template <bool F16>
__device__ __forceinline__ uint16_t op_bits(float x) {
    if (F16) return __half_as_ushort(__float2half_rn(fminf(fmaxf(x, -65504.0f), 65504.0f)));
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<const uint16_t *>(&b);
}
template <bool F16>
__device__ __forceinline__ uint32_t op_pack(float lo, float hi) {
    return (uint32_t)op_bits<F16>(lo) | ((uint32_t)op_bits<F16>(hi) << 16);
}

// 16 columns (two 8-column TMEM loads) of this thread's lane, columns beyond
// `nc8` chunks left untouched.
__device__ __forceinline__ void tmem_ld_cols16(uint32_t taddr, int nc8, uint32_t (&r)[16]) {
    tmem_ld8(taddr, r[0], r[1], r[2], r[3], r[4], r[5], r[6], r[7]);
    if (nc8 > 1) tmem_ld8(taddr + 8, r[8], r[9], r[10], r[11], r[12], r[13], r[14], r[15]);
}

template <int H, bool F16>
__global__ void __launch_bounds__(kEpi + 64, 1) fwd2d_tc_kernel(const __grid_constant__ Fwd2TcArgs A) {
    constexpr int NH = H / 128;     // unit halves (M tiles)
    constexpr int KC = H / 64;      // K chunks of a hidden-size input
    constexpr int CG = kEpi / H;    // epilogue threads per unit (column groups)
    constexpr int NW = kEpi / 32;   // epilogue warps
    constexpr uint32_t kTileBytes = KC * 16384u;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    Misc2 &M = *reinterpret_cast<Misc2 *>(smem_raw);
    uint8_t *tiles = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + sizeof(Misc2) + 1023) & ~uintptr_t(1023));
    uint8_t *xt = tiles;                    // layer input x (K-major rows = site columns)
    uint8_t *ht = tiles + kTileBytes;       // h_V, then the layer's states h
    uint8_t *ring = tiles + 2 * kTileBytes; // weight slices
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = A.R, S = A.S, W = A.W, Lx = A.Lx, Ly = A.Ly, Px = Lx >> 1, Py = Ly >> 1;
    const int nL = A.tl.nL, N = Lx * Ly, Np = Px * Py;
    const int nch = W >> 3;  // 8-column chunks of a slot
    const uint32_t img_bytes = (uint32_t)KC * (uint32_t)W * 128u;  // one layer's h_V image of a slot
    const volatile int *ab = &M.abort_flag;
    uint8_t *scratch = A.scratch + (size_t)blockIdx.x * S * nL * img_bytes;

    // h_V image of layer l for slot s's current row (source) and for its next
    // row (destination; null after the job's last row)
    auto img_src = [&](const Slot2 &st, int s, int l) -> const uint8_t * {
        if (st.row == st.r0) {
            if (st.r0 == 0) return A.zero_img;
            return A.img_in + (((size_t)st.sample * Py + st.r0) * nL + l) * img_bytes;
        }
        if (A.img_out) return A.img_out + (((size_t)st.sample * Py + st.row) * nL + l) * img_bytes;
        return scratch + ((size_t)s * nL + l) * img_bytes;
    };
    auto img_dst = [&](const Slot2 &st, int s, int l) -> uint8_t * {
        if (st.row + 1 >= Py) return nullptr;
        if (A.img_out) return A.img_out + (((size_t)st.sample * Py + st.row + 1) * nL + l) * img_bytes;
        return scratch + ((size_t)s * nL + l) * img_bytes;
    };

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
        for (int g = 0; g < 2; ++g) {
            mbar_init(smem_u32(&M.e2m[g]), 1);
            mbar_init(smem_u32(&M.m2e[g]), 1);
        }
        M.hv_armed = 0;
        mbar_init(smem_u32(&M.hv), 1);
        mbar_init(smem_u32(&M.imgw), 1);
        mbar_init(smem_u32(&M.go[0]), 1);
        mbar_init(smem_u32(&M.go[1]), 1);
        M.abort_flag = 0;
        M.go_flag[0] = 1;
        M.go_flag[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int s = tid; s < kMaxSlots; s += blockDim.x) {
        M.slot[s].job = -1;
        M.slot[s].acc = 0.0f;
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = M.tmem_base;
    if (tmem != 0) {  // all 512 columns are needed from column 0
        if (tid == 0) set_status(A.status, PSR_EDEVICE);
        M.abort_flag = 1;
    }
    if (tid == 0) mbar_arrive(smem_u32(&M.go[0]));  // row step 0 runs
    __syncthreads();
    const long long njobs = A.mode == 1 ? (long long)*A.n_jobs_dev : (long long)A.n_jobs;
    const uint32_t hvb = smem_u32(&M.hv), imgw = smem_u32(&M.imgw);

    if (warp == NW) {
        // ------------------------------------------------ producer: weight stream
        if (lane == 0 && !M.abort_flag) {
            uint32_t q = 0, slot = 0, round = 0;  // slices issued; ring slot and pass over the ring
            const uint32_t fb = smem_u32(&M.full[0]), ebar = smem_u32(&M.empty[0]), rb = smem_u32(ring);
            for (uint32_t row = 0;; ++row) {
                if (!wait_ab(smem_u32(&M.go[row & 1]), (row >> 1) & 1, ab)) break;
                if (!*(volatile int *)&M.go_flag[row & 1]) break;
                bool ok = true;
                const uint8_t *src = A.wimg;
                for (int i = 0; i < A.n_slices; ++i, ++q, src += kSlice) {
                    if (round > 0 && !wait_ab(ebar + 8 * slot, (round - 1) & 1, ab)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_tx(fb + 8 * slot, kSlice);
                    bulk_g2s(rb + slot * kSlice, src, kSlice, fb + 8 * slot);
                    if (++slot == (uint32_t)R) {
                        slot = 0;
                        ++round;
                    }
                }
                if (!ok) break;
            }
            // copies still in flight land before the CTA may exit
            const uint32_t last = q < (uint32_t)R ? q : (uint32_t)R;
            for (uint32_t t = 0; t < last; ++t) {
                const uint32_t qq = q - 1 - t;
                if (!mbar_wait(smem_u32(&M.full[qq % R]), (qq / R) & 1)) set_status(A.status, PSR_ETIMEOUT);
            }
            if (*ab) set_status(A.status, PSR_ETIMEOUT);
        }
    } else if (warp == NW + 1) {
        // ------------------------------------------------ MMA issue, h_V image stores
        if (lane == 0 && !M.abort_flag) {
            // slices consumed; ring slot and the full barriers' phase; e2m and
            // h_V barrier phases
            uint32_t q = 0, slot = 0, fph = 0, pe0 = 0, pe1 = 0, ph = 0;
            const uint32_t e2m0 = smem_u32(&M.e2m[0]), e2m1 = smem_u32(&M.e2m[1]), m2e0 = smem_u32(&M.m2e[0]),
                           m2e1 = smem_u32(&M.m2e[1]);
            const uint32_t ha = smem_u32(ht), fb = smem_u32(&M.full[0]), ebar = smem_u32(&M.empty[0]);
            const uint64_t xd = kdesc(smem_u32(xt)), hd = kdesc(ha), rd = kdesc(smem_u32(ring));
            bool ok = true;
            for (uint32_t row = 0; ok; ++row) {
                if (!wait_ab(smem_u32(&M.go[row & 1]), (row >> 1) & 1, ab)) {
                    ok = false;
                    break;
                }
                if (!*(volatile int *)&M.go_flag[row & 1]) break;
                for (int i = 0; i < A.n_slices; ++i, ++q) {
                    const uint32_t op = A.sched.op[i];
                    if (op & 0x00FF0000u) {
                        const uint32_t fl = (op >> 16) & 0xFFu;
                        if (fl & (kSchedC0 | kSchedC1)) {
                            bulk_wait_read();  // the h tile may be overwritten once this commit lands
                            if (fl & kSchedC0) mma_commit(m2e0);
                            if (fl & kSchedC1) mma_commit(m2e1);
                        }
                        if (fl & kSchedW0) {
                            if (!wait_ab(e2m0, pe0, ab)) { ok = false; break; }
                            pe0 ^= 1u;
                            tc_after();
                        }
                        if (fl & kSchedW1) {
                            if (!wait_ab(e2m1, pe1, ab)) { ok = false; break; }
                            pe1 ^= 1u;
                            tc_after();
                        }
                        if (fl & kSchedStoreH) {
                            // the scan has written h: it is the next row's h_V of layer l
                            const int l = (int)((op >> 24) & 0xFu);
                            for (int s = 0; s < S; ++s) {
                                const Slot2 &st = M.slot[s];
                                if (st.job < 0) continue;
                                uint8_t *dst = img_dst(st, s, l);
                                if (!dst) continue;
                                for (int c = 0; c < KC; ++c)
                                    bulk_s2g(dst + (size_t)c * W * 128, ha + c * 16384 + s * W * 128,
                                             (uint32_t)W * 128u);
                            }
                            bulk_commit();
                        }
                        if (fl & kSchedWaitHv) {
                            if (!wait_ab(hvb, ph, ab)) { ok = false; break; }
                            ph ^= 1u;
                            tc_after();
                        }
                    }
                    // the weight slice has landed (bulk-copy transactions)
                    if (!wait_ab(fb + 8 * slot, fph, ab)) { ok = false; break; }
                    const uint64_t ad = rd + (uint64_t)(slot * (kSlice >> 4));
                    const uint64_t bd = ((op & (1u << 10)) ? hd : xd) + (uint64_t)(((op >> 12) & 3u) * (16384u >> 4));
                    const uint32_t d = tmem + (op & 0x3FFu);
                    mma_ss<idesc2<F16>()>(d, ad, bd, (op >> 11) & 1u);
                    mma_ss<idesc2<F16>()>(d, ad + kstep(1), bd + kstep(1), 1u);
                    mma_ss<idesc2<F16>()>(d, ad + kstep(2), bd + kstep(2), 1u);
                    mma_ss<idesc2<F16>()>(d, ad + kstep(3), bd + kstep(3), 1u);
                    mma_commit(ebar + 8 * slot);
                    if (++slot == (uint32_t)R) {
                        slot = 0;
                        fph ^= 1u;
                    }
                }
                if (!ok) break;
                // the row's image stores are complete before its successor reads them
                bulk_wait_all();
                mbar_arrive(imgw);
                mma_commit(m2e0);  // logits of the row
                if (NH == 2) mma_commit(m2e1);
            }
            bulk_wait_all();
            // the MMAs of the last slices complete before the CTA may exit
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
        // warp w reads tensor-memory lanes 32 (w & 3) ..; warpgroup w >> 2
        // takes unit half g and column group cg (slots s = cg, cg + CG, ...)
        const int q4 = warp & 3, wg = warp >> 2, g = wg % NH, cg = wg / NH;
        const int j = 128 * g + 32 * q4 + lane;  // hidden unit
        const uint32_t lane_off = (uint32_t)(q4 * 32) << 16;
        const uint32_t tz = tmem + lane_off + 128u * g;          // z, then y
        const uint32_t tcc = tmem + lane_off + 128u * (NH + g);  // c
        const uint32_t tlg = tmem + lane_off + 128u * NH;        // logits (lanes 32 q4 + 0..15)
        // unit j's place in a K-major tile row
        const uint32_t kreg = (uint32_t)(j >> 6) * 16384u;
        const int ch = (j & 63) >> 3;
        const uint32_t eb = (uint32_t)(j & 7) * 2u;
        // unit j's element of tile row nb + k, nb a multiple of 8 (so the
        // 16-byte chunk's swizzle phase is k & 7)
        const uint32_t eoff = kreg + eb, sw = (uint32_t)ch << 4;
        auto tile_st = [&](uint8_t *tile, int nb, int k, uint16_t v) {
            *reinterpret_cast<uint16_t *>(tile + eoff + (uint32_t)nb * 128u + (sw ^ ((uint32_t)(k & 7) << 4)) +
                                          (uint32_t)k * 128u) = v;
        };
        float *res = A.res + (size_t)blockIdx.x * 2 * kCols * H;
        uint32_t pm = 0;  // m2e phase of this thread's unit half
        bool ok = !M.abort_flag;
        // this unit half's barriers, named barrier (2 + g) and leader thread
        const uint32_t e2m = smem_u32(&M.e2m[g]), m2e = smem_u32(&M.m2e[g]);
        const uint32_t hbar = 2u + (uint32_t)g, hcount = (uint32_t)(kEpi / NH);
        const bool leader = tid == 128 * g;

        // thread 0: bulk copies of every active slot's h_V image of layer l
        auto issue_hv = [&](int l) {
            uint32_t bytes = 0;
            for (int s = 0; s < S; ++s)
                if (M.slot[s].job >= 0) bytes += img_bytes;
            mbar_arrive_tx(hvb, bytes);
            for (int s = 0; s < S; ++s) {
                const Slot2 &st = M.slot[s];
                if (st.job < 0) continue;
                const uint8_t *src = img_src(st, s, l);
                for (int kc = 0; kc < KC; ++kc)
                    bulk_g2s(smem_u32(ht + kc * 16384 + s * W * 128), src + (size_t)kc * W * 128, (uint32_t)W * 128u,
                             hvb);
            }
            ++M.hv_armed;
        };
        // One thread polls the MMA thread's barrier and a named barrier
        // releases the others (hundreds of pollers would contend for the
        // shared memory the tensor core reads its operands from); the
        // epilogue's signal is one arrival after a named barrier.
        auto wait_m2e = [&]() {
            bool w = true;
            if (leader) w = ok && wait_ab(m2e, pm, ab);
            const bool bad = named_bar_or(hbar, hcount, !w || !ok);
            if (bad && ok && leader) {
                M.abort_flag = 1;
                set_status(A.status, PSR_ETIMEOUT);
            }
            ok = ok && !bad;
            pm ^= 1u;
            tc_after();
        };
        auto arrive_e2m = [&]() {
            fence_proxy_async();  // this thread's tile writes, before the MMAs read them
            tc_before();
            named_bar(hbar, hcount);
            if (leader) mbar_arrive(e2m);
        };
        // the previous row's readout sums into the job's total (fixed order),
        // and the job's log psi after its last row (slot s, its warp)
        auto fold = [&](int s) {
            Slot2 &st = M.slot[s];
            if (lane == 0 && st.job >= 0) {
                float a = st.acc;
                for (int c = 0; c < nch; ++c) a += st.part[c];
                st.acc = a;
                if (st.row + 1 >= Py) A.out[st.job] = 0.5f * a;
            }
            __syncwarp();
        };

        for (uint32_t row_it = 0; ok; ++row_it) {
            // ---- slot update (warp s for slot s): finished or empty slots
            // take the next job, the others advance one patch row
            for (int s = warp; s < S; s += NW) {
                Slot2 &st = M.slot[s];
                if (row_it > 0) fold(s);
                const int job = st.job;
                if (job == -2) continue;
                const uint8_t *sp;
                int r;
                if (job == -1 || st.row + 1 >= Py) {
                    unsigned long long nj = 0;
                    if (lane == 0) nj = atomicAdd(A.job_counter, 1ull);
                    nj = __shfl_sync(0xffffffffu, nj, 0);
                    if ((long long)nj >= njobs) {
                        if (lane == 0) st.job = -2;
                        __syncwarp();
                        continue;
                    }
                    int sample = (int)nj, p = -1, qq = -1, r0 = 0;
                    if (A.mode == 1) {
                        const int32_t *e = A.entries + 3 * nj;
                        sample = e[0];
                        p = e[1];
                        qq = e[2];
                        r0 = (p / Lx) >> 1;
                    }
                    sp = A.spins + (size_t)sample * N;
                    int up = 0;
                    for (int t = lane; t < 2 * r0 * Lx; t += 32) up += sp[t] & 1;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) up += __shfl_xor_sync(0xffffffffu, up, o);
                    if (lane < Px) {
                        if (r0 > 0) st.vprev[lane] = (uint8_t)patch_value(sp, Lx, lane, r0 - 1, -1, -1);
                        st.v[lane] = (uint8_t)patch_value(sp, Lx, lane, r0, p, qq);
                    }
                    if (lane == 0) {
                        st.job = (int)nj;
                        st.sample = sample;
                        st.p = p;
                        st.q = qq;
                        st.row = r0;
                        st.r0 = r0;
                        st.n_up = up;
                        st.acc = 0.0f;
                    }
                    r = r0;
                } else {
                    r = st.row + 1;
                    sp = A.spins + (size_t)st.sample * N;
                    int pc = 0;
                    if (lane < Px) {
                        const int old = st.v[lane];
                        pc = __popc(old);
                        st.vprev[lane] = (uint8_t)old;
                        st.v[lane] = (uint8_t)patch_value(sp, Lx, lane, r, st.p, st.q);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, o);
                    if (lane == 0) {
                        st.n_up += pc;
                        st.row = r;
                    }
                }
                __syncwarp();
            }
            if (epi_bar_or(!ok || *ab)) {
                ok = false;
                break;
            }
            if (tid == 0) {
                // does a row step follow this one?
                bool more = false;
                for (int s = 0; s < S; ++s)
                    if (M.slot[s].job >= 0 && M.slot[s].row + 1 < Py) more = true;
                if (!more) more = (long long)atomicAdd(A.job_counter, 0ull) < njobs;
                M.go_flag[(row_it + 1) & 1] = more ? 1 : 0;
                mbar_arrive(smem_u32(&M.go[(row_it + 1) & 1]));
                // the previous row's image stores are complete
                if (row_it > 0 && !wait_ab(imgw, (row_it - 1) & 1, ab)) {
                    ok = false;
                    M.abort_flag = 1;
                    set_status(A.status, PSR_ETIMEOUT);
                }
                if (ok) issue_hv(0);
            }
            // ---- layer-0 input: one-hot (v_H, v_V) of every column, K chunk 0
            {
                constexpr uint32_t kOne = F16 ? 0x3C00u : 0x3F80u;  // 1.0
                for (int id = tid; id < kCols * 8; id += kEpi) {
                    const int n = id >> 3, c = id & 7, s = n / W, i = n - s * W;
                    int vh = -1, vv = -1;
                    if (s < S && i < Px) {
                        const Slot2 &st = M.slot[s];
                        if (st.job >= 0) {
                            const bool odd = st.row & 1;
                            // the previous patch on the path: column i - 1 (even rows) or i + 1
                            if (odd ? (i + 1 < Px) : (i > 0)) vh = st.v[odd ? i + 1 : i - 1];
                            if (st.row > 0) vv = 16 + st.vprev[i];
                        }
                    }
                    uint32_t w4[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int e0 = 8 * c + 2 * e, e1 = e0 + 1;
                        const uint32_t lo = (e0 == vh || e0 == vv) ? kOne : 0u;
                        const uint32_t hi = (e1 == vh || e1 == vv) ? kOne : 0u;
                        w4[e] = lo | (hi << 16);
                    }
                    *reinterpret_cast<uint4 *>(xt + n * 128 + ((c ^ (n & 7)) << 4)) =
                        make_uint4(w4[0], w4[1], w4[2], w4[3]);
                }
            }
            arrive_e2m();

            for (int l = 0; l < nL; ++l) {
                // ---- gates and scan along each slot's row (path order)
                wait_m2e();
                {
                    const float hbz = 0.5f * A.theta[A.tl.bz[l] + j], bh = A.theta[A.tl.bh[l] + j];
                    const float2 hbz2 = make_float2(hbz, hbz), bh2 = make_float2(bh, bh);
                    const bool keep_res = (l >= 1) && (l + 1 < nL);
                    float *resw = res + (size_t)(l & 1) * kCols * H;
                    for (int s = cg; s < S; s += CG) {
                        const Slot2 &st = M.slot[s];
                        if (st.job < 0) continue;
                        const int n0 = s * W;
                        const bool odd = st.row & 1;
                        float h = 0.0f;  // the row starts from h_H = 0
                        // two 16-column halves, in path order
                        for (int hh = 0; hh < 2; ++hh) {
                            const int half = odd ? 1 - hh : hh;
                            const int c0 = 16 * half;
                            if (c0 >= Px) continue;
                            const int nc8 = nch - 2 * half;
                            uint32_t zr[16], cr[16];
                            tmem_ld_cols16(tz + n0 + c0, nc8, zr);
                            tmem_ld_cols16(tcc + n0 + c0, nc8, cr);
                            tmem_wait_ld16x2(zr, cr);
                            float av[16], bv[16];
#pragma unroll
                            for (int k = 0; k < 16; k += 2) {
                                float2 a2, b2;
                                gates2(make_float2(__uint_as_float(zr[k]), __uint_as_float(zr[k + 1])),
                                       make_float2(__uint_as_float(cr[k]), __uint_as_float(cr[k + 1])), hbz2, bh2, a2,
                                       b2);
                                av[k] = a2.x;
                                av[k + 1] = a2.y;
                                bv[k] = b2.x;
                                bv[k + 1] = b2.y;
                            }
                            if (!odd) {
#pragma unroll
                                for (int k = 0; k < 16; ++k) {
                                    if (c0 + k < Px) {
                                        h = fmaf(av[k], h, bv[k]);
                                        tile_st(ht, n0 + c0, k, op_bits<F16>(h));
                                        if (keep_res) resw[(size_t)(n0 + c0 + k) * H + j] = h;
                                    }
                                }
                            } else {
#pragma unroll
                                for (int k = 15; k >= 0; --k) {
                                    if (c0 + k < Px) {
                                        h = fmaf(av[k], h, bv[k]);
                                        tile_st(ht, n0 + c0, k, op_bits<F16>(h));
                                        if (keep_res) resw[(size_t)(n0 + c0 + k) * H + j] = h;
                                    }
                                }
                            }
                        }
                    }
                }
                arrive_e2m();

                // ---- output map: x = GELU(y + residual)
                wait_m2e();
                // the last half's output map is committed: every MMA reading
                // the h tile is complete, the next layer's h_V may land in it
                if (leader && g == NH - 1 && l + 1 < nL && ok) issue_hv(l + 1);
                {
                    const bool use_res = (l >= 2);
                    const float *resr = res + (size_t)((l - 1) & 1) * kCols * H;
                    for (int s = cg; s < S; s += CG) {
                        const Slot2 &st = M.slot[s];
                        if (st.job < 0) continue;
                        const int n0 = s * W;
                        for (int half = 0; half < 2; ++half) {
                            const int c0 = 16 * half;
                            if (c0 >= Px) continue;
                            uint32_t yr[16];
                            tmem_ld_cols16(tz + n0 + c0, nch - 2 * half, yr);
                            float rv[16];
#pragma unroll
                            for (int k = 0; k < 16; ++k)
                                rv[k] = (use_res && c0 + k < Px) ? resr[(size_t)(n0 + c0 + k) * H + j] : 0.0f;
                            asm volatile("tcgen05.wait::ld.sync.aligned;" : PSR_P16(yr, 0)::"memory");
#pragma unroll
                            for (int k = 0; k < 16; k += 2) {
                                if (c0 + k < Px) {
                                    const float2 x = gelu_bf16out2(make_float2(__uint_as_float(yr[k]) + rv[k],
                                                                               __uint_as_float(yr[k + 1]) + rv[k + 1]));
                                    tile_st(xt, n0 + c0, k, op_bits<F16>(x.x));
                                    if (c0 + k + 1 < Px)
                                        tile_st(xt, n0 + c0, k + 1, op_bits<F16>(x.y));
                                }
                            }
                        }
                    }
                }
                arrive_e2m();
            }

            // ---- readout: masked 16-way softmax of every patch of the row;
            // warp w takes 8 columns (slot w / nch, chunk w % nch)
            wait_m2e();
            if (ok && warp < S * nch) {
                const int s = warp / nch, c8 = warp - s * nch;
                Slot2 &st = M.slot[s];
                if (st.job >= 0) {
                    const int r = st.row, n0 = s * W, i0 = 8 * c8;
                    const bool odd = r & 1;
                    const float bo = A.theta[A.tl.bo + (lane & 15)];
                    const int pc_lane = __popc(lane & 15);
                    // up spins of the row's patches before path position `lane`
                    int upx;
                    {
                        const int c = odd ? Px - 1 - lane : lane;  // column at path position lane
                        const int pc = lane < Px ? __popc(st.v[c]) : 0;
                        int incl = pc;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int t = __shfl_up_sync(0xffffffffu, incl, o);
                            if (lane >= o) incl += t;
                        }
                        upx = incl - pc;
                    }
                    float ref = 0.0f;
                    if (A.mode == 1 && lane < 8 && i0 + lane < Px) {
                        const int i = i0 + lane, k = odd ? Px - 1 - i : i;
                        ref = A.logp_ref[(size_t)st.sample * Np + r * Px + k];
                    }
                    uint32_t lr[8];
                    tmem_ld8(tlg + n0 + i0, lr[0], lr[1], lr[2], lr[3], lr[4], lr[5], lr[6], lr[7]);
                    asm volatile("tcgen05.wait::ld.sync.aligned;"
                                 : "+r"(lr[0]), "+r"(lr[1]), "+r"(lr[2]), "+r"(lr[3]), "+r"(lr[4]), "+r"(lr[5]),
                                   "+r"(lr[6]), "+r"(lr[7])::"memory");
                    float rsum = 0.0f;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int i = i0 + e;
                        if (i >= Px) break;
                        const int k = odd ? Px - 1 - i : i, v = st.v[i];
                        const int up = st.n_up + __shfl_sync(0xffffffffu, upx, k);
                        const int down = 2 * r * Lx + 4 * k - up;
                        const bool allowed = !A.u1 || (up + pc_lane <= N / 2 && down + 4 - pc_lane <= N / 2);
                        const float lg = __uint_as_float(lr[e]) + bo;
                        float m = allowed ? lg : -INFINITY;
#pragma unroll
                        for (int o = 8; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o, 16));
                        float ex = allowed ? __expf(lg - m) : 0.0f;
#pragma unroll
                        for (int o = 8; o > 0; o >>= 1) ex += __shfl_xor_sync(0xffffffffu, ex, o, 16);
                        float lp = allowed ? lg - m - __logf(ex) : -INFINITY;
                        lp = __shfl_sync(0xffffffffu, lp, v);
                        const float rf = __shfl_sync(0xffffffffu, ref, e);
                        float d = lp;
                        if (A.mode == 1) d = lp - rf;
                        else if (A.logp_out && lane == 0) A.logp_out[(size_t)st.sample * Np + r * Px + k] = lp;
                        rsum += d;
                    }
                    if (lane == 0) st.part[c8] = rsum;
                }
            }
            tc_before();
            if (epi_bar_or(!ok)) {
                ok = false;
                break;
            }
            if (!*(volatile int *)&M.go_flag[(row_it + 1) & 1]) {
                for (int s = warp; s < S; s += NW) fold(s);
                break;
            }
        }
        if (!ok) {
            M.abort_flag = 1;
            set_status(A.status, PSR_ETIMEOUT);
        }
        if (tid == 0 && M.hv_armed > 0 && !mbar_wait(hvb, (M.hv_armed - 1) & 1)) set_status(A.status, PSR_ETIMEOUT);
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

template <int H>
size_t fwd2d_tc_smem(int R) {
    return sizeof(Misc2) + 1024 + 2 * (size_t)(H / 64) * 16384 + (size_t)R * kSlice;
}

template <int H, bool F16>
cudaError_t launch_h(const Fwd2TcArgs &a, int grid, cudaStream_t stream) {
    const size_t smem = fwd2d_tc_smem<H>(a.R);
    cudaError_t e =
        cudaFuncSetAttribute(fwd2d_tc_kernel<H, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fwd2d_tc_kernel<H, F16><<<grid, kEpi + 64, smem, stream>>>(a);
    return cudaGetLastError();
}

// Weight slices in MMA order: 128 rows (units 128 g ..) x 64 inputs (64 kc ..)
// of one matrix, 128-byte swizzle (16-byte chunk c of row m at c ^ (m & 7)).
template <bool F16>
__global__ void pack2d_tc_kernel(const float *__restrict__ theta, T2Layout tl, Sched2 sc,
                                 uint8_t *__restrict__ wimg) {
    const int H = tl.H;
    const int64_t total = (int64_t)sc.n * 1024;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(id >> 10), m = (int)((id >> 3) & 127), c = (int)(id & 7);
        const int ty = sc.type[i], l = sc.l[i], unit = 128 * sc.g[i] + m, k0 = 64 * sc.kc[i] + 8 * c;
        const int din = l == 0 ? 32 : H;
        uint32_t w[4];
#pragma unroll
        for (int e2 = 0; e2 < 4; ++e2) {
            float v2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = k0 + 2 * e2 + h;
                float v = 0.0f;
                switch (ty) {
                    case kMtWz: if (k < din) v = theta[tl.Wz[l] + (int64_t)unit * din + k]; break;
                    case kMtWhx: if (k < din) v = theta[tl.Wh[l] + (int64_t)unit * (din + H) + k]; break;
                    case kMtWhv: v = theta[tl.Wh[l] + (int64_t)unit * (din + H) + din + k]; break;
                    case kMtC: v = theta[tl.C[l] + (int64_t)unit * H + k]; break;
                    case kMtD: if (k < din) v = theta[tl.D[l] + (int64_t)unit * din + k]; break;
                    default:  // W_o in rows 32 q + o of every lane quarter q
                        if ((unit & 31) < 16) v = theta[tl.Wo + (int64_t)(unit & 31) * H + k];
                        break;
                }
                v2[h] = v;
            }
            w[e2] = op_pack<F16>(v2[0], v2[1]);
        }
        *reinterpret_cast<uint4 *>(wimg + (size_t)i * kSlice + m * 128 + ((c ^ (m & 7)) << 4)) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
}

}  // namespace

// Slices of one row step, in the order the MMA thread consumes them, with
// the synchronisation each needs first.
Sched2 fwd2d_tc_schedule(int nL, int H) {
    Sched2 sc{};
    const int NH = H / 128, KC = H / 64;
    int n = 0;
    auto add = [&](int ty, int l, int g, int kc, int fl) {
        sc.type[n] = (uint8_t)ty;
        sc.l[n] = (uint8_t)l;
        sc.g[n] = (uint8_t)g;
        sc.kc[n] = (uint8_t)kc;
        sc.flags[n] = (uint8_t)fl;
        // accumulator column (z / y of half g: 128 g; c: 128 (NH + g); logits:
        // 128 NH), B tile, accumulate flag
        uint32_t dcol = 0, from_h = 0, acc = 0;
        switch (ty) {
            case kMtWz: dcol = 128u * g; acc = kc > 0; break;
            case kMtWhx: dcol = 128u * (NH + g); acc = 1; break;
            case kMtWhv: dcol = 128u * (NH + g); from_h = 1; acc = kc > 0; break;
            case kMtD: dcol = 128u * g; acc = kc > 0; break;
            case kMtC: dcol = 128u * g; from_h = 1; acc = 1; break;
            default: dcol = 128u * NH; acc = kc > 0; break;
        }
        sc.op[n] = dcol | (from_h << 10) | (acc << 11) | ((uint32_t)kc << 12) | ((uint32_t)fl << 16) |
                   ((uint32_t)l << 24);
        ++n;
    };
    const int HL = NH - 1;                                       // last unit half
    const int kC[2] = {kSchedC0, kSchedC1}, kW[2] = {kSchedW0, kSchedW1};
    const int wall = NH == 2 ? (kSchedW0 | kSchedW1) : kSchedW0;  // both halves' epilogues
    for (int l = 0; l < nL; ++l) {
        const int kin = l == 0 ? 1 : KC;
        // W_hv h_V needs only the h_V image of the layer: above layer 0 it
        // runs while the epilogue computes the layer input (after the last
        // half's output map of layer l - 1 has been committed)
        for (int g = 0; g < NH; ++g)
            for (int kc = 0; kc < KC; ++kc) {
                int fl = 0;
                if (g == 0 && kc == 0) fl = kSchedWaitHv | (l > 0 ? kC[HL] : 0);
                add(kMtWhv, l, g, kc, fl);
            }
        // W_z x, W_hx x once x is complete; half g's projections are
        // committed (its scan may start) before half g + 1's are issued
        for (int g = 0; g < NH; ++g) {
            for (int kc = 0; kc < kin; ++kc) {
                int fl = 0;
                if (kc == 0) fl = (g == 0) ? wall : kC[g - 1];
                add(kMtWz, l, g, kc, fl);
            }
            for (int kc = 0; kc < kin; ++kc) add(kMtWhx, l, g, kc, 0);
        }
        // D x of half g once half g's scan has consumed z; C h once every
        // half's scan has written h (then h is also stored as the next row's
        // h_V); half g's output map committed before half g + 1's C
        for (int g = 0; g < NH; ++g)
            for (int kc = 0; kc < kin; ++kc) {
                int fl = 0;
                if (kc == 0) fl = (g == 0 ? kC[HL] : 0) | kW[g] | (g == HL ? kSchedStoreH : 0);
                add(kMtD, l, g, kc, fl);
            }
        for (int g = 0; g < NH; ++g)
            for (int kc = 0; kc < KC; ++kc) add(kMtC, l, g, kc, (kc == 0 && g > 0) ? kC[g - 1] : 0);
    }
    // readout once both halves' layer input of the readout (x) is complete
    for (int kc = 0; kc < KC; ++kc) add(kMtWo, 0, 0, kc, kc == 0 ? (kC[HL] | wall) : 0);
    sc.n = n;
    return sc;
}

bool fwd2d_tc_supported(int nL, int H, int Lx) {
    return (H == 128 || H == 256) && nL >= 1 && nL <= kMaxLayers && Lx >= 2 && Lx <= 64 &&
           fwd2d_tc_schedule(nL, H).n <= kSchedMax;
}

void fwd2d_tc_geometry(int Lx, int *W, int *S) {
    const int Px = Lx / 2;
    *W = 8 * ((Px + 7) / 8);
    *S = kCols / *W;
    if (*S > kMaxSlots) *S = kMaxSlots;
}

size_t fwd2d_tc_image_bytes(int H, int Lx) {
    int W, S;
    fwd2d_tc_geometry(Lx, &W, &S);
    return (size_t)(H / 64) * W * 128;
}

size_t fwd2d_tc_weight_bytes(int nL, int H) { return (size_t)fwd2d_tc_schedule(nL, H).n * kSlice; }

size_t fwd2d_tc_ckpt_bytes(int nL, int H, int Lx, int Ly) {
    return (size_t)(Ly / 2) * nL * fwd2d_tc_image_bytes(H, Lx);
}

size_t fwd2d_tc_scratch_bytes(int nL, int H, int Lx, int grid) {
    int W, S;
    fwd2d_tc_geometry(Lx, &W, &S);
    return (size_t)grid * S * nL * fwd2d_tc_image_bytes(H, Lx);
}

size_t fwd2d_tc_res_floats(int H, int grid) { return (size_t)grid * 2 * kCols * H; }

cudaError_t launch_pack2d_tc(const float *theta, const T2Layout &tl, bool f16, uint8_t *wimg,
                             cudaStream_t stream) {
    const Sched2 sc = fwd2d_tc_schedule(tl.nL, tl.H);
    const int64_t total = (int64_t)sc.n * 1024;
    const int blocks = (int)((total + 255) / 256);
    if (f16) pack2d_tc_kernel<true><<<blocks, 256, 0, stream>>>(theta, tl, sc, wimg);
    else pack2d_tc_kernel<false><<<blocks, 256, 0, stream>>>(theta, tl, sc, wimg);
    return cudaGetLastError();
}

cudaError_t launch_fwd2d_tc(Fwd2TcArgs a, int grid, cudaStream_t stream) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int H = a.tl.H;
    fwd2d_tc_geometry(a.Lx, &a.W, &a.S);
    a.sched = fwd2d_tc_schedule(a.tl.nL, H);
    a.n_slices = a.sched.n;
    const size_t base = (H == 256) ? fwd2d_tc_smem<256>(0) : fwd2d_tc_smem<128>(0);
    if ((size_t)optin < base + 2 * kSlice) return cudaErrorInvalidConfiguration;
    int R = (int)(((size_t)optin - base) / kSlice);
    a.R = R > kMaxRing ? kMaxRing : R;
    if (grid < 1) grid = 1;
    switch (H) {
        case 128: return a.f16 ? launch_h<128, true>(a, grid, stream) : launch_h<128, false>(a, grid, stream);
        case 256: return a.f16 ? launch_h<256, true>(a, grid, stream) : launch_h<256, false>(a, grid, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace psr
