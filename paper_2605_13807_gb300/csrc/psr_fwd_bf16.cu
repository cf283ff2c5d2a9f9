// tcgen05 (5th-generation tensor core) forward of the PSR-NQS ansatz,
// hidden = 128, 3 layers, BF16 operands with FP32 accumulation.
//
// Layout: "feature-major" tiles.  Every MMA computes D[out unit][site] =
// sum_k A[out unit][k] B[site][k] with M = 128 output units (one per TMEM
// lane), N = 64 sites (one scan chunk) and K = 128 input units, so after
// tcgen05.ld thread j of a warpgroup holds hidden unit j for all 64 sites of
// the chunk and the recurrence h_t = a_t h_{t-1} + b_t (Sec. II.C) is a plain
// sequential FP32 loop in registers, with the carry kept across chunks.  The
// activations of the chunk (h and x, BF16) are written straight into the
// next MMA's B operand in shared memory (MN-major, 128-byte swizzle); they
// never touch HBM.  All weights stay on chip for the whole kernel:
//   TMEM (A operand):  W_z^(1), W_h^(1), W_z^(2), W_h^(2)
//   SMEM (A operand):  C^(0), C^(1), D^(1), C^(2), D^(2)   (K-major, SW128)
// Layer 0 has a one-hot input (Sec. II.F), so its gates come from lookup
// tables and only its output map C^(0) h is a contraction.  The readout
// (logit difference, two-way softmax) and log-psi sums are FP32 on CUDA cores.
//
// A CTA (one per SM) runs two independent sequence streams, one per
// warpgroup, each with its own TMEM accumulators, B tiles and mbarrier:
// while one stream runs its epilogue (gates, scan, GELU) the tensor core
// works on the other stream's MMAs.  Jobs (full sequences or connected
// configurations resumed from a stored chunk carry) come from an atomic
// counter.  Every mbarrier wait is bounded; on expiry the CTA records
// PSR_ETIMEOUT, stops issuing work, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "psr_device.cuh"
#include "psr_internal.cuh"

namespace psr {

namespace {

constexpr int H = 128;
constexpr int CH = kChunkBF16;  // 64 sites = MMA N
constexpr int NL = 3;
constexpr int kThreads = 256;   // two warpgroups = two streams
constexpr uint32_t kTileBytes = 16384;     // [K=128 rows][64 sites] bf16
constexpr uint32_t kMatBytes = 32768;      // 128 x 128 bf16
constexpr int kSmemMats = 5;               // C0, C1, D1, C2, D2
constexpr int kTmemMats = 4;               // Wz1, Wh1, Wz2, Wh2
enum { SM_C0 = 0, SM_C1 = 1, SM_D1 = 2, SM_C2 = 3, SM_D2 = 4 };
enum { TM_WZ1 = 0, TM_WH1 = 1, TM_WZ2 = 2, TM_WH2 = 3 };
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kTmemWeightCol = 256;   // weights at columns 256..511

// shared memory map (offsets from a 1024-aligned base)
constexpr uint32_t OFF_W = 0;
constexpr uint32_t OFF_TILES = OFF_W + kSmemMats * kMatBytes;   // per stream: X, H
constexpr uint32_t OFF_MISC = OFF_TILES + 4 * kTileBytes;
constexpr uint32_t MISC_BYTES = 256;
constexpr uint32_t kSmemBytes = OFF_MISC + MISC_BYTES + 1024;   // + alignment slack

// packed global image (bytes)
constexpr size_t PK_SMEM = 0;
constexpr size_t PK_TMEM = PK_SMEM + (size_t)kSmemMats * kMatBytes;
constexpr size_t PK_TOTAL = PK_TMEM + (size_t)kTmemMats * kMatBytes;

// kind::f16 instruction descriptor: D = F32, A = B = BF16, A K-major,
// B MN-major, N = 64, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (1u << 16) |
                            ((uint32_t)(CH >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound per wait

// ------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase completed, false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u && globaltimer() - t0 > kWaitNs) return false;
    }
    return false;
}

__device__ __forceinline__ void named_bar(int id) {
    asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Smem matrix descriptor (tcgen05): start >> 4, LBO >> 4 at bit 16,
// SBO >> 4 at bit 32, version 1 at bit 46, 128-byte swizzle (2) at bit 61.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

#define PSR_R32(x) \
    "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]), "=r"(x[7]), \
    "=r"(x[8]), "=r"(x[9]), "=r"(x[10]), "=r"(x[11]), "=r"(x[12]), "=r"(x[13]), "=r"(x[14]),         \
    "=r"(x[15]), "=r"(x[16]), "=r"(x[17]), "=r"(x[18]), "=r"(x[19]), "=r"(x[20]), "=r"(x[21]),       \
    "=r"(x[22]), "=r"(x[23]), "=r"(x[24]), "=r"(x[25]), "=r"(x[26]), "=r"(x[27]), "=r"(x[28]),       \
    "=r"(x[29]), "=r"(x[30]), "=r"(x[31])
#define PSR_W32(x) \
    "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(x[7]),         \
    "r"(x[8]), "r"(x[9]), "r"(x[10]), "r"(x[11]), "r"(x[12]), "r"(x[13]), "r"(x[14]), "r"(x[15]),    \
    "r"(x[16]), "r"(x[17]), "r"(x[18]), "r"(x[19]), "r"(x[20]), "r"(x[21]), "r"(x[22]), "r"(x[23]),  \
    "r"(x[24]), "r"(x[25]), "r"(x[26]), "r"(x[27]), "r"(x[28]), "r"(x[29]), "r"(x[30]), "r"(x[31])

// 32 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : PSR_R32(r)
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        PSR_W32(r)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Writes 32 consecutive sites [32*half, 32*half+32) of row k of an MN-major
// SW128 B tile: row k is 128 bytes, 16-byte chunk c holds sites 8c..8c+7 and
// sits at physical chunk c ^ (k & 7).
__device__ __forceinline__ void tile_store32(uint8_t *tile, int k, int half, const float *v) {
    uint8_t *row = tile + k * 128;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = half * 4 + q;
        uint4 w;
        w.x = pack_bf16(v[8 * q + 0], v[8 * q + 1]);
        w.y = pack_bf16(v[8 * q + 2], v[8 * q + 3]);
        w.z = pack_bf16(v[8 * q + 4], v[8 * q + 5]);
        w.w = pack_bf16(v[8 * q + 6], v[8 * q + 7]);
        *reinterpret_cast<uint4 *>(row + ((c ^ (k & 7)) << 4)) = w;
    }
}

struct Misc {
    uint64_t mbar[2];
    long long job[2];
    uint32_t tmem_base;
    int abort_flag[2];
};
static_assert(sizeof(Misc) <= MISC_BYTES, "misc block too large");

}  // namespace

size_t bf16_packed_bytes() { return PK_TOTAL; }

// theta (FP32, D5 layout) -> BF16 images: five K-major SW128 shared-memory
// images followed by four row-major TMEM images.
__global__ void pack_bf16_kernel(const float *__restrict__ theta, ThetaLayout tl,
                                 uint8_t *__restrict__ out) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t smem_src[kSmemMats] = {tl.C[0], tl.C[1], tl.D[1], tl.C[2], tl.D[2]};
    const int64_t tmem_src[kTmemMats] = {tl.Wz[1], tl.Wh[1], tl.Wz[2], tl.Wh[2]};
    for (int64_t i = tid; i < (int64_t)(kSmemMats + kTmemMats) * H * H; i += stride) {
        const int mat = (int)(i / (H * H));
        const int e = (int)(i % (H * H));
        const int m = e / H, k = e % H;
        __nv_bfloat16 v;
        size_t byte;
        if (mat < kSmemMats) {
            v = __float2bfloat16_rn(theta[smem_src[mat] + e]);
            const int atom = k >> 6, kin = k & 63, chunk = kin >> 3, within = kin & 7;
            const int group = m >> 3, r = m & 7;
            byte = PK_SMEM + (size_t)mat * kMatBytes + (size_t)atom * 16384 + group * 1024 + r * 128 +
                   ((chunk ^ r) << 4) + within * 2;
        } else {
            const int t = mat - kSmemMats;
            v = __float2bfloat16_rn(theta[tmem_src[t] + e]);
            byte = PK_TMEM + (size_t)t * kMatBytes + (size_t)m * 256 + (size_t)k * 2;
        }
        *reinterpret_cast<__nv_bfloat16 *>(out + byte) = v;
    }
}

cudaError_t launch_pack_theta_bf16(const float *theta, const ThetaLayout &tl, void *packed,
                                   cudaStream_t stream) {
    if (tl.H != H || tl.nL != NL) return cudaErrorInvalidValue;
    pack_bf16_kernel<<<128, 256, 0, stream>>>(theta, tl, static_cast<uint8_t *>(packed));
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kThreads, 1)
fwd_bf16_kernel(FwdJobs jb, const uint8_t *__restrict__ pkb, const float *__restrict__ pk,
                F32Layout fl) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    Misc &M = *reinterpret_cast<Misc *>(smem + OFF_MISC);

    const int tid = threadIdx.x;
    const int g = tid >> 7;          // stream (warpgroup)
    const int j = tid & 127;         // hidden unit = TMEM lane
    const int warp = tid >> 5;
    const int lane_base = (warp & 3) * 32;

    uint8_t *tileX = smem + OFF_TILES + (2 * g) * kTileBytes;
    uint8_t *tileH = tileX + kTileBytes;
    const uint32_t wsm = smem_u32(smem + OFF_W);
    const uint32_t tX = smem_u32(tileX), tH = smem_u32(tileH);
    const uint32_t bar = smem_u32(&M.mbar[g]);

    // ------------------------------------------------------------- set-up
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&M.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&M.mbar[0]), 1);
        mbar_init(smem_u32(&M.mbar[1]), 1);
        M.abort_flag[0] = 0;
        M.abort_flag[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // shared-memory weight images (plain 16-byte copies)
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(pkb + PK_SMEM);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + OFF_W);
        for (int i = tid; i < (int)(kSmemMats * kMatBytes / 16); i += kThreads) dst[i] = src[i];
    }
    fence_proxy_async();
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = M.tmem_base;
    // TMEM weight images: warpgroup 0, lane j = row j
    if (g == 0) {
#pragma unroll 1
        for (int m = 0; m < kTmemMats; ++m) {
            const uint32_t *row =
                reinterpret_cast<const uint32_t *>(pkb + PK_TMEM + (size_t)m * kMatBytes + j * 256);
#pragma unroll 1
            for (int half = 0; half < 2; ++half) {
                uint32_t r[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) r[q] = row[half * 32 + q];
                tmem_st32(tmem + ((uint32_t)lane_base << 16) + kTmemWeightCol + m * 64 + half * 32, r);
            }
        }
        tmem_wait_st();
    }
    tc_before();
    __syncthreads();
    tc_after();

    // per-thread constants (FP32)
    const float a0_0 = pk[fl.A0 + j], a0_1 = pk[fl.A0 + H + j], a0_2 = pk[fl.A0 + 2 * H + j];
    const float b0_0 = pk[fl.B0 + j], b0_1 = pk[fl.B0 + H + j], b0_2 = pk[fl.B0 + 2 * H + j];
    const float d0_0 = pk[fl.DU0 + j], d0_1 = pk[fl.DU0 + H + j], d0_2 = pk[fl.DU0 + 2 * H + j];
    const float bz1 = pk[fl.bz[1] + j], bh1 = pk[fl.bh[1] + j];
    const float bz2 = pk[fl.bz[2] + j], bh2 = pk[fl.bh[2] + j];
    const float wdj = pk[fl.wd + j];
    const float bd = pk[fl.bd];

    const uint32_t lane_off = (uint32_t)lane_base << 16;
    const uint32_t accZ = tmem + lane_off + 128 * g;       // this thread's lane, Z columns
    const uint32_t accC = accZ + 64;
    const uint32_t dZ = tmem + 128 * g;                    // MMA destination (lane 0)
    const uint32_t dC = dZ + 64;
    const uint32_t aW = tmem + kTmemWeightCol;             // TMEM weights (lane 0)

    const int N = jb.N;
    const int nch = (N + CH - 1) / CH;
    const long long njobs = jb.mode == 1 ? (long long)*jb.n_jobs_dev : (long long)jb.n_jobs;
    const int bar_id = 1 + g;
    uint32_t phase = 0;
    bool aborted = false;

    // Issues the MMAs of one step (thread j == 0 of the stream) and waits.
    // Returns false if the wait expired (the whole stream then stops).
    auto sync_wait = [&]() -> bool {
        bool ok = mbar_wait(bar, phase);
        phase ^= 1u;
        if (!ok) {
            M.abort_flag[g] = 1;
            set_status(jb.status, PSR_ETIMEOUT);
        }
        named_bar(bar_id);
        tc_after();
        return M.abort_flag[g] == 0;
    };
    // generic smem writes + TMEM loads done -> visible to the MMA issuer
    auto publish = [&]() {
        fence_proxy_async();
        tc_before();
        named_bar(bar_id);
        tc_after();
    };

    for (;;) {
        if (j == 0) M.job[g] = (long long)atomicAdd(jb.job_counter, 1ull);
        named_bar(bar_id);
        const long long job = M.job[g];
        named_bar(bar_id);
        if (job >= njobs) break;

        int sample, p = -1, q = -1, c0 = 0;
        if (jb.mode == 0) {
            sample = (int)job;
        } else {
            const int32_t *e = jb.entries + 3 * job;
            sample = e[0];
            p = e[1];
            q = e[2];
            c0 = p / CH;
        }
        const uint64_t *row = jb.bits + (int64_t)sample * jb.W;
        float hc0 = 0.0f, hc1 = 0.0f, hc2 = 0.0f;
        if (c0 > 0) {
            const float *cin = jb.carries_in + (((int64_t)sample * nch + c0) * NL) * H + j;
            hc0 = cin[0];
            hc1 = cin[H];
            hc2 = cin[2 * H];
        }
        int n_up = jb.u1 ? count_up_before(row, c0 * CH) : 0;
        float acc = 0.0f;

        for (int c = c0; c < nch && !aborted; ++c) {
            const int t0 = c * CH;
            if (jb.carries_out) {
                float *co = jb.carries_out + (((int64_t)sample * nch + c) * NL) * H + j;
                co[0] = hc0;
                co[H] = hc1;
                co[2 * H] = hc2;
            }
            uint64_t cur = row[c];
            uint32_t prev = (c > 0) ? (uint32_t)(row[c - 1] >> 63) : 0u;
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const int x = f ? q : p;
                if (x >= t0 && x < t0 + CH) cur ^= 1ull << (x - t0);
                else if (x >= 0 && x == t0 - 1) prev ^= 1u;
            }
            const int nvalid = min(CH, N - t0);
            if (nvalid < 64) cur &= (1ull << nvalid) - 1ull;
            const uint64_t prevbits = (cur << 1) | prev;  // bit t = s_{t0+t-1}

            // ---------------- layer 0: lookup gates + scan -> h0 (B tile H)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float hv[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int t = half * 32 + i;
                    const bool first = (t0 + t == 0);
                    const bool sb = (prevbits >> t) & 1ull;
                    const float a = first ? a0_0 : (sb ? a0_2 : a0_1);
                    const float b = first ? b0_0 : (sb ? b0_2 : b0_1);
                    hc0 = a * hc0 + b;
                    hv[i] = hc0;
                }
                tile_store32(tileH, j, half, hv);
            }
            publish();
            if (j == 0) {
#pragma unroll
                for (int kk = 0; kk < 8; ++kk)
                    mma_ss(dZ, sdesc(wsm + SM_C0 * kMatBytes + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024),
                           sdesc(tH + kk * 2048, 1024, 1024), kk > 0);
                mma_commit(bar);
            }
            if (!sync_wait()) { aborted = true; break; }
            // epilogue: x1 = GELU(C0 h0 + D0 u) -> B tile X
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                uint32_t r[32];
                tmem_ld32(accZ + half * 32, r);
                tmem_wait_ld();
                float xv[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int t = half * 32 + i;
                    const bool first = (t0 + t == 0);
                    const bool sb = (prevbits >> t) & 1ull;
                    const float du = first ? d0_0 : (sb ? d0_2 : d0_1);
                    xv[i] = gelu_f(__uint_as_float(r[i]) + du);
                }
                tile_store32(tileX, j, half, xv);
            }
            publish();

            // ---------------- layers 1 and 2
            float h1[CH];
            float x3[CH];
#pragma unroll
            for (int l = 1; l <= 2; ++l) {
                const uint32_t wz = aW + (l == 1 ? TM_WZ1 : TM_WZ2) * 64;
                const uint32_t wh = aW + (l == 1 ? TM_WH1 : TM_WH2) * 64;
                if (j == 0) {
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk)
                        mma_ts(dZ, wz + kk * 8, sdesc(tX + kk * 2048, 1024, 1024), kk > 0);
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk)
                        mma_ts(dC, wh + kk * 8, sdesc(tX + kk * 2048, 1024, 1024), kk > 0);
                    mma_commit(bar);
                }
                if (!sync_wait()) { aborted = true; break; }
                const float bz = (l == 1) ? bz1 : bz2, bh = (l == 1) ? bh1 : bh2;
                float hc = (l == 1) ? hc1 : hc2;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    uint32_t rz[32], rc[32];
                    tmem_ld32(accZ + half * 32, rz);
                    tmem_ld32(accC + half * 32, rc);
                    tmem_wait_ld();
                    float hv[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float a = sigmoid_f(__uint_as_float(rz[i]) + bz);
                        hc = a * hc + (1.0f - a) * (__uint_as_float(rc[i]) + bh);
                        hv[i] = hc;
                        if (l == 1) h1[half * 32 + i] = hc;
                    }
                    tile_store32(tileH, j, half, hv);
                }
                if (l == 1) hc1 = hc; else hc2 = hc;
                publish();
                const int sC = (l == 1) ? SM_C1 : SM_C2, sD = (l == 1) ? SM_D1 : SM_D2;
                if (j == 0) {
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk)
                        mma_ss(dZ, sdesc(wsm + sC * kMatBytes + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024),
                               sdesc(tH + kk * 2048, 1024, 1024), kk > 0);
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk)
                        mma_ss(dZ, sdesc(wsm + sD * kMatBytes + (kk >> 2) * 16384 + (kk & 3) * 32, 16, 1024),
                               sdesc(tX + kk * 2048, 1024, 1024), 1);
                    mma_commit(bar);
                }
                if (!sync_wait()) { aborted = true; break; }
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    uint32_t r[32];
                    tmem_ld32(accZ + half * 32, r);
                    tmem_wait_ld();
                    float xv[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        float y = __uint_as_float(r[i]);
                        if (l == 2) y += h1[half * 32 + i];
                        xv[i] = gelu_f(y);
                        if (l == 2) x3[half * 32 + i] = xv[i];
                    }
                    if (l == 1) tile_store32(tileX, j, half, xv);
                }
                if (l == 1) publish();
            }
            if (aborted) break;
            tc_before();  // TMEM reads of this chunk are done before the next MMA

            // ---------------- readout: d_t = wd . x3_t + bd, reduced over units
            {
                float v[CH];
#pragma unroll
                for (int t = 0; t < CH; ++t) v[t] = wdj * x3[t];
                const int lane = tid & 31;
#pragma unroll
                for (int s = 0; s < 5; ++s) {
                    const int m = 16 >> s;
                    const int half = 32 >> s;
                    const bool upper = (lane & m) != 0;
#pragma unroll
                    for (int i = 0; i < half; ++i) {
                        const float send = upper ? v[i] : v[i + half];
                        const float keep = upper ? v[i + half] : v[i];
                        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
                    }
                }
                // lane L now holds sites 2L and 2L+1 summed over its warp's units
                float *red = reinterpret_cast<float *>(tileX);  // [4 warps][64]
                const int w4 = warp & 3;
                red[w4 * CH + 2 * lane] = v[0];
                red[w4 * CH + 2 * lane + 1] = v[1];
                named_bar(bar_id);
                float sv = 0.0f;
                if (j < CH) {
                    const int t = j;
                    const float d = bd + red[t] + red[CH + t] + red[2 * CH + t] + red[3 * CH + t];
                    const int tt = t0 + t;
                    if (tt < N) {
                        const int s = (int)((cur >> t) & 1ull);
                        const int nu = n_up + __popcll(cur & ((1ull << t) - 1ull));
                        const float lp = site_logp(d, s, u1_forced(jb.u1, N, tt, nu));
                        if (jb.logp_out) jb.logp_out[(int64_t)sample * N + tt] = lp;
                        sv = (jb.mode == 1) ? lp - jb.logp_ref[(int64_t)sample * N + tt] : lp;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
                }
                named_bar(bar_id);  // red[] reads done
                if (j < CH && (j & 31) == 0) red[j >> 5] = sv;
                named_bar(bar_id);
                if (j == 0) acc += red[0] + red[1];
                n_up += __popcll(cur);
                named_bar(bar_id);  // scratch reads done before the next chunk writes X
            }
        }
        if (aborted) break;
        if (j == 0) jb.out[job] = 0.5f * acc;
    }

    // ------------------------------------------------------------ teardown
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
}

cudaError_t launch_fwd_bf16(const FwdJobs &jobs, const void *packed_bf16, const float *packed_f32,
                            const F32Layout &fl, int num_sms, cudaStream_t stream) {
    if (fl.H != H || fl.nL != NL) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fwd_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    int64_t grid = num_sms;
    const int64_t max_jobs_streams = (jobs.n_jobs + 1) / 2;
    if (grid > max_jobs_streams) grid = max_jobs_streams;
    if (grid < 1) grid = 1;
    fwd_bf16_kernel<<<(int)grid, kThreads, kSmemBytes, stream>>>(
        jobs, static_cast<const uint8_t *>(packed_bf16), packed_f32, fl);
    return cudaGetLastError();
}

}  // namespace psr
