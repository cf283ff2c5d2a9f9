// tcgen05 (5th-generation tensor core) forward of the PSR-NQS ansatz,
// hidden = 128, 3 layers, BF16 operands with FP32 accumulation.
//
// Layout: "feature-major" tiles.  Every MMA computes D[out unit][site] =
// sum_k A[out unit][k] B[site][k] with M = 128 output units (one per TMEM
// lane), N = 32 sites (one scan chunk) and K = 128 input units, so after
// tcgen05.ld thread j of a warpgroup holds hidden unit j for all 32 sites of
// the chunk and the recurrence h_t = a_t h_{t-1} + b_t (Sec. II.C) is a plain
// sequential FP32 loop in registers, with the carry kept across chunks.  The
// activations of the chunk (h and x, BF16) are written straight into the
// next MMA's B operand in shared memory (MN-major, 64-byte swizzle); they
// never touch HBM.  All weights stay on chip for the whole kernel:
//   TMEM (A operand):  W_z^(1), W_h^(1), W_z^(2), W_h^(2)
//   SMEM (A operand):  C^(0), C^(1), D^(1), C^(2), D^(2)   (K-major, SW128)
// Layer 0 has a one-hot input (Sec. II.F), so its gates come from lookup
// tables and only its output map C^(0) h is a contraction.  The readout
// (logit difference, two-way softmax) and log-psi sums are FP32 on CUDA cores.
//
// A CTA (one per SM) has four warpgroups, one per sequence in flight, grouped
// into MMA streams of HALVES sequences each (template parameter):
//   HALVES = 1: four streams, MMA N = 32 (one sequence's chunk), 64-byte
//               swizzled activation tiles;
//   HALVES = 2: two streams, MMA N = 64 (the chunks of two sequences side by
//               side), 128-byte swizzled tiles.
// A stream owns 2N TMEM accumulator columns, two B tiles, an mbarrier and a
// named barrier; while one stream waits for its MMAs or its TMEM loads, the
// others issue their epilogues (gates, scan, GELU), and the tensor core works
// through the MMAs of all of them.  The shared-memory weight slices an MMA
// reads (4 KB per K = 16 slice) serve N sites, so the two-sequence streams
// read half the weight bytes per site; the sequences of one stream advance
// chunk by chunk in step, each with its own job.  Jobs (full sequences or
// connected configurations resumed from a stored chunk carry) come from an
// atomic counter.  Every mbarrier wait is bounded; on expiry the CTA records
// PSR_ETIMEOUT, stops issuing work, frees its TMEM and returns.
#include <cstddef>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "psr_bf16_math.cuh"
#include "psr_device.cuh"
#include "psr_internal.cuh"
#include "psr_tc.cuh"

namespace psr {

namespace {

constexpr int H = 128;
constexpr int CH = kChunkBF16;  // 32 sites per sequence and chunk
constexpr int NL = 3;
constexpr int kSeqs = 4;                  // sequences in flight per CTA, one warpgroup each
constexpr int kThreads = 128 * kSeqs;
constexpr uint32_t kTileBytesAll = 2 * kSeqs * 8192;  // X and H tiles of all streams
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
constexpr uint32_t OFF_MISC = OFF_TILES + kTileBytesAll;
constexpr uint32_t MISC_BYTES = 512;
constexpr uint32_t kSmemBytes = OFF_MISC + MISC_BYTES + 1024;   // + alignment slack

// Stream shape: HALVES sequences per MMA stream.
template <int HALVES>
struct Shape {
    static constexpr int kStreams = kSeqs / HALVES;
    static constexpr int kN = CH * HALVES;                    // MMA N (sites)
    static constexpr uint32_t kRowBytes = 2 * kN;             // one K row of a B tile
    static constexpr uint32_t kTileBytes = 128 * kRowBytes;   // [K = 128][kN] bf16
    static constexpr uint32_t kAtom = 8 * kRowBytes;          // 8-row swizzle atom
    static constexpr uint64_t kLayout = HALVES == 1 ? 4ull : 2ull;  // 64- / 128-byte swizzle
    // kind::f16 instruction descriptor: D = F32, A = B = BF16, A K-major,
    // B MN-major, N = kN, M = 128.
    static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (1u << 16) |
                                       ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
};
static_assert(2 * Shape<1>::kStreams * Shape<1>::kTileBytes == kTileBytesAll, "tile budget");
static_assert(2 * Shape<2>::kStreams * Shape<2>::kTileBytes == kTileBytesAll, "tile budget");

// packed global image (bytes)
constexpr size_t PK_SMEM = 0;
constexpr size_t PK_TMEM = PK_SMEM + (size_t)kSmemMats * kMatBytes;
constexpr size_t PK_TOTAL = PK_TMEM + (size_t)kTmemMats * kMatBytes;


using namespace tc;
using namespace bf16m;

// B operand: an activation tile, MN-major (kN sites = kRowBytes per K row),
// 64-byte (kN = 32) or 128-byte (kN = 64) swizzle; 8-row groups of kAtom
// bytes along K.  The kN sites are one swizzle atom wide, so only the
// K-direction stride is ever used; both offsets are given that value.
template <class SH>
__device__ __forceinline__ uint64_t bdesc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(SH::kAtom >> 4) << 16) |
           ((uint64_t)(SH::kAtom >> 4) << 32) | (1ull << 46) | (SH::kLayout << 61);
}

// What the readout of a job's chunks needs after the warpgroup may already
// have moved on to its next job (two slots per warpgroup, alternating by job).
struct RdInfo {
    float *logp;                     // per-site log P row of the sample (mode 0) or null
    float *out;                      // the job's output element
    int N, u1;
};

struct Misc {
    uint64_t mbar[kSeqs];            // per stream
    long long job[kSeqs];            // per warpgroup
    long long base[kMaxGroups + 1];  // first job of each group
    RdInfo info[kSeqs][2];           // per warpgroup
    uint32_t tmem_base;
    int abort_flag[kSeqs];           // per stream
    int done[kSeqs];                 // per warpgroup: no jobs left
    float red2[kSeqs];               // per warpgroup: chunk sum of log P
};
static_assert(sizeof(Misc) <= MISC_BYTES, "misc block too large");
static_assert(offsetof(Misc, mbar) == 0, "mbarriers open the misc block");

// --------------------------------------------------- epilogue arithmetic
// Writes 8 sites (one 16-byte chunk, logical index c) of row k of an
// MN-major swizzled B tile: the swizzle XORs the chunk index with address
// bits 7.. of the row, so the chunk sits at c ^ ((k >> 1) & 3) (64-byte rows)
// or c ^ (k & 7) (128-byte rows).
template <class SH>
__device__ __forceinline__ void tile_store8(uint8_t *tile, int k, int c, const float *v) {
    uint4 w;
    w.x = pack_bf16(v[0], v[1]);
    w.y = pack_bf16(v[2], v[3]);
    w.z = pack_bf16(v[4], v[5]);
    w.w = pack_bf16(v[6], v[7]);
    constexpr uint32_t kMask = SH::kRowBytes / 16 - 1;
    const uint32_t sw = ((uint32_t)k * SH::kRowBytes >> 7) & kMask;
    *reinterpret_cast<uint4 *>(tile + k * SH::kRowBytes + ((c ^ sw) << 4)) = w;
}

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


// MMA issue for stream s: group WHAT = 0 (layer-0 output map D0 u + C0 h), 1 / 3
// (projections W_z x, W_h x of layer 1 / 2), 2 / 4 (output map C h + D x of
// layer 1 / 2).  Stream s accumulates in TMEM columns 2N s .. 2N s + 2N - 1
// (Z or the output in the first N, h~ in the second N); the kernel owns all
// 512 columns, so its allocation starts at column 0.
// Descriptors of the k-th K = 16 slice are the slice-0 descriptor plus the
// slice's byte offset >> 4 in the start-address field (no carry: shared
// addresses stay below 2^18 bytes).
__device__ __forceinline__ uint64_t adesc0(uint32_t w) { return sdesc(w, 16, 1024); }
__device__ __forceinline__ uint64_t aoff(int kk) { return (uint64_t)(((kk >> 2) * 16384 + (kk & 3) * 32) >> 4); }
template <class SH>
__device__ __forceinline__ uint64_t boff(int kk) { return (uint64_t)((kk * 16 * SH::kRowBytes) >> 4); }

template <int WHAT, class SH>
__device__ __forceinline__ void issue(int s, uint32_t sbase) {
    constexpr uint32_t ID = SH::kIdesc;
    const uint32_t tX = sbase + OFF_TILES + (uint32_t)(2 * s) * SH::kTileBytes;
    const uint64_t bX = bdesc<SH>(tX), bH = bdesc<SH>(tX + SH::kTileBytes);
    const uint32_t d = 2u * SH::kN * (uint32_t)s;
    if (WHAT == 0) {
        // accumulates onto D0 u, which the layer-0 scan stored in the columns
        const uint64_t aC = adesc0(sbase + OFF_W + SM_C0 * kMatBytes);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) mma_ss<ID>(d, aC + aoff(kk), bH + boff<SH>(kk), 1);
    } else if (WHAT == 1 || WHAT == 3) {
        const uint32_t wz = kTmemWeightCol + (WHAT == 1 ? TM_WZ1 : TM_WZ2) * 64;
        const uint32_t wh = kTmemWeightCol + (WHAT == 1 ? TM_WH1 : TM_WH2) * 64;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) mma_ts<ID>(d, wz + kk * 8, bX + boff<SH>(kk), kk > 0);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) mma_ts<ID>(d + SH::kN, wh + kk * 8, bX + boff<SH>(kk), kk > 0);
    } else {
        const uint64_t aC = adesc0(sbase + OFF_W + (WHAT == 2 ? SM_C1 : SM_C2) * kMatBytes);
        const uint64_t aD = adesc0(sbase + OFF_W + (WHAT == 2 ? SM_D1 : SM_D2) * kMatBytes);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) mma_ss<ID>(d, aC + aoff(kk), bH + boff<SH>(kk), kk > 0);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) mma_ss<ID>(d, aD + aoff(kk), bX + boff<SH>(kk), 1);
    }
    mma_commit(sbase + OFF_MISC + 8 * (uint32_t)s);
}

// Gates and scan of 16 sites (half hh of the chunk) from their Z and h~
// accumulators: a = sigmoid(z + b_z), h_t = a_t h_{t-1} + (1 - a_t)(h~_t + b_h).
// The sites go to chunks 2 hh, 2 hh + 1 of this sequence's part (cbase) of
// the tile row.
template <int L, class SH>
__device__ __forceinline__ void gates_scan16(const uint32_t (&rz)[16], const uint32_t (&rc)[16], int hh,
                                             float2 hbz2, float2 bh2, float &h, float (&h1)[32],
                                             uint8_t *tileH, int j, int cbase) {
#pragma unroll
    for (int gg = 0; gg < 2; ++gg) {
        float hv[8];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            const int k = 8 * gg + i;
            float2 a, b;
            gates2(make_float2(__uint_as_float(rz[k]), __uint_as_float(rz[k + 1])),
                   make_float2(__uint_as_float(rc[k]), __uint_as_float(rc[k + 1])), hbz2, bh2, a, b);
            h = fmaf(a.x, h, b.x);
            hv[i] = h;
            h = fmaf(a.y, h, b.y);
            hv[i + 1] = h;
        }
        if (L == 1) {
#pragma unroll
            for (int i = 0; i < 8; ++i) h1[16 * hh + 8 * gg + i] = hv[i];
        }
        tile_store8<SH>(tileH, j, cbase + 2 * hh + gg, hv);
    }
}

// One dense layer (l = 1 or 2) of one stream's step, from the projection
// MMAs to the output epilogue.  act: this warpgroup's sequence has a chunk in
// this step (an idle warpgroup keeps the stream's barriers and waits but
// computes nothing).  h1: layer 1 writes its FP32 h there (the residual of
// layer 2); layer 2 adds it and overwrites it with the layer output x3.
template <int L, class SH, class WaitF, class PubF>
__device__ __forceinline__ void dense_layer(bool act, float hbz, float bh, uint8_t *tileX, uint8_t *tileH,
                                            uint32_t sbase, int s, uint32_t accZ, uint32_t accC,
                                            bool issuer, int j, int cbase, float &carry, float (&h1)[32],
                                            WaitF &sync_wait, PubF &publish) {
    if (issuer) issue<L == 1 ? 1 : 3, SH>(s, sbase);
    sync_wait();
    if (act) {
        const float2 hbz2 = make_float2(hbz, hbz), bh2 = make_float2(bh, bh);
        float h = carry;
        if (L == 1) {
            // sites 0..15, with the loads of sites 16..31 in flight meanwhile
            uint32_t z0[16], c0[16], z1[16], c1[16];
            tmem_ld16(accZ, z0);
            tmem_ld16(accC, c0);
            tmem_wait_ld16x2(z0, c0);
            tmem_ld16(accZ + 16, z1);
            tmem_ld16(accC + 16, c1);
            gates_scan16<L, SH>(z0, c0, 0, hbz2, bh2, h, h1, tileH, j, cbase);
            tmem_wait_ld16x2(z1, c1);
            gates_scan16<L, SH>(z1, c1, 1, hbz2, bh2, h, h1, tileH, j, cbase);
        } else {
            // layer 2 keeps the residual h1 live: one half at a time
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                uint32_t z[16], cc[16];
                tmem_ld16(accZ + 16 * hh, z);
                tmem_ld16(accC + 16 * hh, cc);
                tmem_wait_ld16x2(z, cc);
                gates_scan16<L, SH>(z, cc, hh, hbz2, bh2, h, h1, tileH, j, cbase);
            }
        }
        carry = h;
    }
    publish();
    if (issuer) issue<L == 1 ? 2 : 4, SH>(s, sbase);
    sync_wait();
    if (act) {
        uint32_t r[32];
        tmem_ld32(accZ, r);
        tmem_wait_ld32(r);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            float xv[8];
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
                const int k = 8 * g + i;
                float2 y = make_float2(__uint_as_float(r[k]), __uint_as_float(r[k + 1]));
                if (L == 2) y = __fadd2_rn(y, make_float2(h1[k], h1[k + 1]));
                const float2 x = (L == 1) ? gelu_bf16out2(y) : gelu_fast2(y);
                xv[i] = x.x;
                xv[i + 1] = x.y;
                if (L == 2) {
                    h1[k] = x.x;
                    h1[k + 1] = x.y;
                }
            }
            if (L == 1) tile_store8<SH>(tileX, j, cbase + g, xv);
        }
    }
    if (L == 1) publish();
}

// One sequence per MMA stream (shape 1): four streams per CTA, one warpgroup
// each; thread j of a stream's warpgroup owns hidden unit j (TMEM lane j) for
// the 32 sites of the chunk.  Each stream walks the chunks of one job at a
// time (its own job loop, no step-synchronous bookkeeping).
__global__ void __launch_bounds__(kThreads, 1)
fwd_bf16_kernel1(const __grid_constant__ FwdJobs jb, const uint8_t *__restrict__ pkb,
                 const float *__restrict__ pk, F32Layout fl) {
    using SH = Shape<1>;
    constexpr int kStreams = SH::kStreams;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    Misc &M = *reinterpret_cast<Misc *>(smem + OFF_MISC);

    const int tid = threadIdx.x;
    const int s = tid >> 7;          // stream = warpgroup
    const int j = tid & 127;         // hidden unit = TMEM lane
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int lane_base = (warp & 3) * 32;
    // one MMA-issuing thread per stream, each on its own SM sub-partition
    // (lane 0 of warp s of the stream's warpgroup)
    const bool issuer = (j == 32 * s);

    uint8_t *tileX = smem + OFF_TILES + (2 * s) * SH::kTileBytes;
    uint8_t *tileH = tileX + SH::kTileBytes;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar = smem_u32(&M.mbar[s]);

    // ------------------------------------------------------------- set-up
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&M.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kStreams; ++i) {
            mbar_init(smem_u32(&M.mbar[i]), 1);
            M.abort_flag[i] = 0;
        }
        long long b = 0;
        M.base[0] = 0;
        for (int i = 0; i < jb.n_groups; ++i) {
            b += jb.mode == 1 ? (long long)*jb.g[i].n_jobs_dev : (long long)jb.g[i].n_jobs;
            M.base[i + 1] = b;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(pkb + PK_SMEM);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + OFF_W);
        for (int i = tid; i < (int)(kSmemMats * kMatBytes / 16); i += kThreads) dst[i] = src[i];
    }
    fence_proxy_async();
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = M.tmem_base;  // 0: the kernel owns all 512 columns
    if (s == 0) {
#pragma unroll 1
        for (int m = 0; m < kTmemMats; ++m) {
            const uint32_t *row =
                reinterpret_cast<const uint32_t *>(pkb + PK_TMEM + (size_t)m * kMatBytes + j * 256);
#pragma unroll 1
            for (int part = 0; part < 2; ++part) {
                uint32_t r[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) r[q] = row[part * 32 + q];
                tmem_st32(tmem + ((uint32_t)lane_base << 16) + kTmemWeightCol + m * 64 + part * 32, r);
            }
        }
        tmem_wait_st();
    }
    tc_before();
    __syncthreads();
    tc_after();

    // per-unit constants, read once (shared memory holds no room for them and
    // the L1 left beside 227 KB of shared memory does not keep them)
    const float a0_0 = pk[fl.A0 + j], a0_1 = pk[fl.A0 + H + j], a0_2 = pk[fl.A0 + 2 * H + j];
    const float b0_0 = pk[fl.B0 + j], b0_1 = pk[fl.B0 + H + j], b0_2 = pk[fl.B0 + 2 * H + j];
    const float d0_0 = pk[fl.DU0 + j], d0_1 = pk[fl.DU0 + H + j], d0_2 = pk[fl.DU0 + 2 * H + j];
    const float hbz1 = 0.5f * pk[fl.bz[1] + j], bh1 = pk[fl.bh[1] + j];
    const float hbz2 = 0.5f * pk[fl.bz[2] + j], bh2 = pk[fl.bh[2] + j];
    const float wdj = pk[fl.wd + j];
    const float bd = pk[fl.bd];

    const uint32_t lane_off = (uint32_t)lane_base << 16;
    const uint32_t accZ = lane_off + 64 * s;  // this stream's Z (and output) columns
    const uint32_t accC = accZ + 32;          // this stream's h~ columns

    // all 512 columns belong to this CTA, so the allocation starts at column 0;
    // anything else is reported and no work is done
    const long long njobs = (tmem == 0) ? M.base[jb.n_groups] : 0;
    if (tmem != 0 && tid == 0) set_status(jb.status, PSR_EDEVICE);
    const int bar_id = 1 + s;
    uint32_t phase = 0;
    bool aborted = false;
    float *red = reinterpret_cast<float *>(tileX);  // readout scratch [4][32]

    auto sbar = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory"); };
    // Waits for this stream's MMAs.  A wait that expires records
    // PSR_ETIMEOUT and the stream's abort flag but keeps the control flow
    // of every thread identical (all later waits are bounded too); the flag
    // is acted on at the end of the chunk, after a stream-wide barrier.
    auto sync_wait = [&]() {
        const bool ok = mbar_wait(bar, phase);
        phase ^= 1u;
        if (!ok) {
            M.abort_flag[s] = 1;
            set_status(jb.status, PSR_ETIMEOUT);
        }
        tc_after();
    };
    auto publish = [&]() {
        fence_proxy_async();
        tc_before();
        sbar();
        tc_after();
    };

    for (;;) {
        if (issuer) M.job[s] = (long long)atomicAdd(jb.job_counter, 1ull);
        sbar();
        const long long job = M.job[s];
        sbar();
        if (job >= njobs) break;
        int gi = 0;
        while (gi + 1 < jb.n_groups && job >= M.base[gi + 1]) ++gi;
        const FwdGroup &G = jb.g[gi];
        const long long lj = job - M.base[gi];
        const int N = G.N;
        const int nch = (N + CH - 1) / CH;

        int sample, p = -1, q = -1, c0 = 0;
        if (jb.mode == 0) {
            sample = (int)lj;
        } else {
            const int32_t *e = G.entries + 3 * lj;
            sample = e[0];
            p = e[1];
            q = e[2];
            c0 = p / CH;
        }
        const uint64_t *row = G.bits + (int64_t)sample * G.W;
        float cr[NL] = {0.0f, 0.0f, 0.0f};  // scan carries
        if (c0 > 0) {
            const float *cin = G.carries_in + (((int64_t)sample * nch + c0) * NL) * H + j;
            cr[0] = cin[0];
            cr[1] = cin[H];
            cr[2] = cin[2 * H];
        }
        int n_up = G.u1 ? count_up_before(row, c0 * CH) : 0;
        float acc = 0.0f;
        // the 64-bit word holding the current chunk's 32 spins; the spin
        // before the chunk (s_{t0-1}) of the unflipped sample
        float h1[32];  // FP32 h of layer 1 (residual of layer 2), then the layer-2 output x3
        uint32_t rd_cur = 0u;  // spins, first site and reference log P of the chunk read out next
        int rd_t0 = 0;
        float rd_lpref = 0.0f;
        // readout of the last finished chunk: d_t = wd . x3_t + bd over the
        // 128 units, log P, and the chunk's sum into acc
        auto readout = [&]() {
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
                const float2 w = __fmul2_rn(make_float2(wdj, wdj), make_float2(h1[i], h1[i + 1]));
                v[i] = w.x;
                v[i + 1] = w.y;
            }
#pragma unroll
            for (int st = 0; st < 5; ++st) {
                const int m = 16 >> st;
                const int half = 16 >> st;
                const bool upper = (lane & m) != 0;
#pragma unroll
                for (int i = 0; i < half; ++i) {
                    const float send = upper ? v[i] : v[i + half];
                    const float keep = upper ? v[i + half] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
                }
            }
            // lane L holds site L, summed over its warp's units; the X tile is
            // free while the layer-0 MMAs (which read only the H tile) run
            red[(warp & 3) * 32 + lane] = v[0];
            sbar();
            if ((warp & 3) == 0) {
                const float d = bd + red[lane] + red[32 + lane] + red[64 + lane] + red[96 + lane];
                const int tt = rd_t0 + lane;
                float sv = 0.0f;
                if (tt < N) {
                    const int sbit = (int)((rd_cur >> lane) & 1u);
                    const int nu = n_up + __popc(rd_cur & ((1u << lane) - 1u));
                    const float lp = site_logp_fast(d, sbit, u1_forced(G.u1, N, tt, nu));
                    if (G.logp_out) G.logp_out[(int64_t)sample * N + tt] = lp;
                    sv = (jb.mode == 1) ? lp - rd_lpref : lp;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
                acc += sv;  // kept by thread j == 0 of the stream
            }
            n_up += __popc(rd_cur);
            if (M.abort_flag[s]) aborted = true;  // uniform: read after the barrier
        };
        uint64_t word = row[c0 >> 1];
        uint32_t next_prev =
            (c0 == 0) ? 0u : (uint32_t)(((c0 & 1) ? (word >> 31) : (row[(c0 >> 1) - 1] >> 63)) & 1ull);

        for (int c = c0; c < nch && !aborted; ++c) {
            const int t0 = c * CH;
            if (G.carries_out) {
                float *co = G.carries_out + (((int64_t)sample * nch + c) * NL) * H + j;
                co[0] = cr[0];
                co[H] = cr[1];
                co[2 * H] = cr[2];
            }
            uint32_t cur = (uint32_t)(word >> (32 * (c & 1)));
            uint32_t prev = next_prev;
            next_prev = cur >> 31;
            // the next word of spins and this chunk's reference log P are
            // fetched now, long before they are needed
            if ((c & 1) && c + 1 < nch) word = row[(c + 1) >> 1];
            float lp_ref = 0.0f;
            if (jb.mode == 1 && (warp & 3) == 0 && t0 + lane < N)
                lp_ref = G.logp_ref[(int64_t)sample * N + t0 + lane];
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const int x = f ? q : p;
                if (x >= t0 && x < t0 + CH) cur ^= 1u << (x - t0);
                else if (x >= 0 && x == t0 - 1) prev ^= 1u;
            }
            const int nvalid = min(CH, N - t0);
            if (nvalid < 32) cur &= (1u << nvalid) - 1u;
            // bit i = s_{t-1} for site t = t0 + i
            const uint32_t inbits = (cur << 1) | prev;
            const bool seq_start = (t0 == 0);  // site 0 has no predecessor

            // ---------------- layer 0: lookup gates, scan -> tile H; the
            // one-hot input's output term D0 u -> this stream's accumulator
            // columns, which the layer-0 MMAs then add C0 h to
            {
                float h = cr[0];
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    float hv[8];
                    uint32_t du[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const bool sb = (inbits >> (8 * g + i)) & 1u;
                        float a = sb ? a0_2 : a0_1, b = sb ? b0_2 : b0_1, dd = sb ? d0_2 : d0_1;
                        if (g == 0 && i == 0 && seq_start) { a = a0_0; b = b0_0; dd = d0_0; }
                        h = fmaf(a, h, b);
                        hv[i] = h;
                        du[i] = __float_as_uint(dd);
                    }
                    tile_store8<SH>(tileH, j, g, hv);
                    tmem_st8(accZ + 8 * g, du);
                }
                cr[0] = h;
                tmem_wait_st();
            }
            publish();
            if (issuer) issue<0, SH>(s, sbase);
            if (c > c0) readout();  // the previous chunk, while the MMAs run
            sync_wait();
            // epilogue: x1 = GELU(C0 h0 + D0 u) -> tile X
            {
                uint32_t r[32];
                tmem_ld32(accZ, r);
                tmem_wait_ld32(r);
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    float xv[8];
#pragma unroll
                    for (int i = 0; i < 8; i += 2) {
                        const int k = 8 * g + i;
                        const float2 x = gelu_bf16out2(make_float2(__uint_as_float(r[k]), __uint_as_float(r[k + 1])));
                        xv[i] = x.x;
                        xv[i + 1] = x.y;
                    }
                    tile_store8<SH>(tileX, j, g, xv);
                }
            }
            publish();

            // ---------------- layers 1 and 2
            dense_layer<1, SH>(true, hbz1, bh1, tileX, tileH, sbase, s, accZ, accC, issuer, j, 0, cr[1], h1,
                               sync_wait, publish);
            dense_layer<2, SH>(true, hbz2, bh2, tileX, tileH, sbase, s, accZ, accC, issuer, j, 0, cr[2], h1,
                               sync_wait, publish);
            // x3 (in h1) is read out while the next chunk's layer-0 MMAs run
            rd_cur = cur;
            rd_t0 = t0;
            rd_lpref = lp_ref;
        }
        if (!aborted) readout();
        if (aborted) break;
        if (j == 0) G.out[lj] = 0.5f * acc;
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

// Two sequences per MMA stream (shape 2; the template also covers HALVES = 1
// but that shape runs fwd_bf16_kernel1): four warpgroups per CTA, one
// sequence each; thread j of a warpgroup owns hidden unit j (TMEM lane j) for
// the 32 sites of its sequence's chunk.  The sequences of a stream advance
// one chunk per step together; each takes a new job from the counter when
// its job ends, and a stream stops when all of its sequences have run out.
template <int HALVES>
__global__ void __launch_bounds__(kThreads, 1)
fwd_bf16_kernel(const __grid_constant__ FwdJobs jb, const uint8_t *__restrict__ pkb,
                const float *__restrict__ pk, F32Layout fl) {
    using SH = Shape<HALVES>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    Misc &M = *reinterpret_cast<Misc *>(smem + OFF_MISC);

    const int tid = threadIdx.x;
    const int wg = tid >> 7;         // warpgroup = sequence slot
    const int s = wg / HALVES;       // stream
    const int half = wg % HALVES;    // position of the sequence in the stream's tiles
    const int j = tid & 127;         // hidden unit = TMEM lane
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int lane_base = (warp & 3) * 32;
    // one MMA-issuing thread per stream, each on its own SM sub-partition
    const bool issuer = (half == 0) && (j == 32 * s);
    const bool leader = (j == 0);    // per warpgroup: job fetch, sums, output
    const int cbase = 4 * half;      // first 16-byte chunk of this sequence in a tile row

    uint8_t *tileX = smem + OFF_TILES + (2 * s) * SH::kTileBytes;
    uint8_t *tileH = tileX + SH::kTileBytes;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar = smem_u32(&M.mbar[s]);

    // ------------------------------------------------------------- set-up
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&M.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kSeqs; ++i) {
            mbar_init(smem_u32(&M.mbar[i]), 1);
            M.abort_flag[i] = 0;
            M.done[i] = 0;
        }
        long long b = 0;
        M.base[0] = 0;
        for (int i = 0; i < jb.n_groups; ++i) {
            b += jb.mode == 1 ? (long long)*jb.g[i].n_jobs_dev : (long long)jb.g[i].n_jobs;
            M.base[i + 1] = b;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(pkb + PK_SMEM);
        uint4 *dst = reinterpret_cast<uint4 *>(smem + OFF_W);
        for (int i = tid; i < (int)(kSmemMats * kMatBytes / 16); i += kThreads) dst[i] = src[i];
    }
    fence_proxy_async();
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = M.tmem_base;  // 0: the kernel owns all 512 columns
    if (wg == 0) {
#pragma unroll 1
        for (int m = 0; m < kTmemMats; ++m) {
            const uint32_t *row =
                reinterpret_cast<const uint32_t *>(pkb + PK_TMEM + (size_t)m * kMatBytes + j * 256);
#pragma unroll 1
            for (int part = 0; part < 2; ++part) {
                uint32_t r[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) r[q] = row[part * 32 + q];
                tmem_st32(tmem + ((uint32_t)lane_base << 16) + kTmemWeightCol + m * 64 + part * 32, r);
            }
        }
        tmem_wait_st();
    }
    tc_before();
    __syncthreads();
    tc_after();

    // per-unit constants, read once (shared memory holds no room for them and
    // the L1 left beside 227 KB of shared memory does not keep them)
    const float a0_0 = pk[fl.A0 + j], a0_1 = pk[fl.A0 + H + j], a0_2 = pk[fl.A0 + 2 * H + j];
    const float b0_0 = pk[fl.B0 + j], b0_1 = pk[fl.B0 + H + j], b0_2 = pk[fl.B0 + 2 * H + j];
    const float d0_0 = pk[fl.DU0 + j], d0_1 = pk[fl.DU0 + H + j], d0_2 = pk[fl.DU0 + 2 * H + j];
    const float hbz1 = 0.5f * pk[fl.bz[1] + j], bh1 = pk[fl.bh[1] + j];
    const float hbz2 = 0.5f * pk[fl.bz[2] + j], bh2 = pk[fl.bh[2] + j];
    const float wdj = pk[fl.wd + j];
    const float bd = pk[fl.bd];

    const uint32_t lane_off = (uint32_t)lane_base << 16;
    const uint32_t accZ = lane_off + 2u * SH::kN * s + 32u * half;  // this sequence's Z (and output) columns
    const uint32_t accC = accZ + SH::kN;                            // this sequence's h~ columns

    // all 512 columns belong to this CTA, so the allocation starts at column 0;
    // anything else is reported and no work is done
    const long long njobs = (tmem == 0) ? M.base[jb.n_groups] : 0;
    if (tmem != 0 && tid == 0) set_status(jb.status, PSR_EDEVICE);
    uint32_t phase = 0;

    // readout scratch [4 warps][32 sites] of this warpgroup: a part of its
    // stream's X tile that only this warpgroup writes (free while the layer-0
    // MMAs, which read only the H tile, run).  With two sequences per stream
    // a 128-byte tile row holds 64 bytes of each, at offset 64 (half ^ bit 2
    // of the row) after the swizzle.
    auto red_addr = [&](int i) -> float * {
        if (HALVES == 1) return reinterpret_cast<float *>(tileX) + i;
        const int k = i >> 4;
        return reinterpret_cast<float *>(tileX + k * SH::kRowBytes + 64 * (half ^ ((k >> 2) & 1))) + (i & 15);
    };

    const int sbar_id = 1 + s, sbar_n = 128 * HALVES;
    const int hbar_id = (HALVES == 1) ? sbar_id : 1 + SH::kStreams + wg;
    auto sbar = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(sbar_id), "r"(sbar_n) : "memory"); };
    auto hbar = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(hbar_id) : "memory"); };
    // Waits for this stream's MMAs.  A wait that expires records
    // PSR_ETIMEOUT and the stream's abort flag but keeps the control flow
    // of every thread identical (all later waits are bounded too); the flag
    // is acted on at the start of the next step, after a stream-wide barrier.
    auto sync_wait = [&]() {
        const bool ok = mbar_wait(bar, phase);
        phase ^= 1u;
        if (!ok) {
            M.abort_flag[s] = 1;
            set_status(jb.status, PSR_ETIMEOUT);
        }
        tc_after();
    };
    auto publish = [&]() {
        fence_proxy_async();
        tc_before();
        sbar();
        tc_after();
    };

    // ---- this warpgroup's job (uniform within the warpgroup)
    enum { kNeed = 0, kActive = 1, kDone = 2 };
    int state = kNeed;
    int slot = 1;             // RdInfo slot of the current job
    int N = 0, nch = 0, c = 0, p = -1, q = -1, n_up = 0;
    const uint64_t *row = nullptr;
    const float *lpref_row = nullptr;  // mode 1: log P of the sample, per site
    float *co_row = nullptr;           // mode 0: chunk carries out of this sample
    uint64_t word = 0;
    uint32_t next_prev = 0;
    float cr[NL] = {0.0f, 0.0f, 0.0f};  // scan carries
    float h1[32];  // FP32 h of layer 1 (residual of layer 2), then the layer-2 output x3

    // ---- the chunk read out next (during the next step's layer-0 MMAs)
    bool rd_valid = false, rd_final = false;
    uint32_t rd_cur = 0u;
    int rd_t0 = 0, rd_nup = 0, rd_slot = 0;
    float rd_lpref = 0.0f;
    float acc = 0.0f;  // running sum of log P of the job being read out (leader)

    // readout of the last finished chunk: d_t = wd . x3_t + bd over the 128
    // units, log P, and the chunk's sum into acc; the job's result after its
    // last chunk
    auto readout = [&]() {
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; i += 2) {
            const float2 w = __fmul2_rn(make_float2(wdj, wdj), make_float2(h1[i], h1[i + 1]));
            v[i] = w.x;
            v[i + 1] = w.y;
        }
#pragma unroll
        for (int st = 0; st < 5; ++st) {
            const int m = 16 >> st;
            const int hw = 16 >> st;
            const bool upper = (lane & m) != 0;
#pragma unroll
            for (int i = 0; i < hw; ++i) {
                const float send = upper ? v[i] : v[i + hw];
                const float keep = upper ? v[i + hw] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
            }
        }
        // lane L holds site L, summed over its warp's units
        *red_addr((warp & 3) * 32 + lane) = v[0];
        hbar();
        if ((warp & 3) == 0) {
            const RdInfo &ri = M.info[wg][rd_slot];
            const float d = bd + *red_addr(lane) + *red_addr(32 + lane) + *red_addr(64 + lane) +
                            *red_addr(96 + lane);
            const int tt = rd_t0 + lane;
            float sv = 0.0f;
            if (tt < ri.N) {
                const int sbit = (int)((rd_cur >> lane) & 1u);
                const int nu = rd_nup + __popc(rd_cur & ((1u << lane) - 1u));
                const float lp = site_logp_fast(d, sbit, u1_forced(ri.u1, ri.N, tt, nu));
                if (ri.logp) ri.logp[tt] = lp;
                sv = (jb.mode == 1) ? lp - rd_lpref : lp;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
            if (lane == 0) M.red2[wg] = sv;
        }
        hbar();
        if (leader) {
            acc += M.red2[wg];
            if (rd_final) *M.info[wg][rd_slot].out = 0.5f * acc;
        }
        if (rd_final) acc = 0.0f;
        rd_valid = false;
    };

    bool stop = false;
    for (;;) {
        // ---------------- this warpgroup's next job, if its last one ended
        if (state == kNeed) {
            if (leader) M.job[wg] = (long long)atomicAdd(jb.job_counter, 1ull);
            hbar();
            const long long job = M.job[wg];
            hbar();
            if (job >= njobs) {
                state = kDone;
            } else {
                int gi = 0;
                while (gi + 1 < jb.n_groups && job >= M.base[gi + 1]) ++gi;
                const FwdGroup &G = jb.g[gi];
                const long long lj = job - M.base[gi];
                N = G.N;
                nch = (N + CH - 1) / CH;
                int sample, c0 = 0;
                p = -1;
                q = -1;
                if (jb.mode == 0) {
                    sample = (int)lj;
                } else {
                    const int32_t *e = G.entries + 3 * lj;
                    sample = e[0];
                    p = e[1];
                    q = e[2];
                    c0 = p / CH;
                }
                row = G.bits + (int64_t)sample * G.W;
                cr[0] = cr[1] = cr[2] = 0.0f;
                if (c0 > 0) {
                    const float *cin = G.carries_in + (((int64_t)sample * nch + c0) * NL) * H + j;
                    cr[0] = cin[0];
                    cr[1] = cin[H];
                    cr[2] = cin[2 * H];
                }
                n_up = G.u1 ? count_up_before(row, c0 * CH) : 0;
                lpref_row = (jb.mode == 1) ? G.logp_ref + (int64_t)sample * N : nullptr;
                co_row = (jb.mode == 0 && G.carries_out) ? G.carries_out + (int64_t)sample * nch * NL * H + j
                                                         : nullptr;
                word = row[c0 >> 1];
                next_prev = (c0 == 0) ? 0u
                                      : (uint32_t)(((c0 & 1) ? (word >> 31) : (row[(c0 >> 1) - 1] >> 63)) & 1ull);
                c = c0;
                slot ^= 1;
                if (leader) {
                    RdInfo &ri = M.info[wg][slot];
                    ri.logp = (jb.mode == 0 && G.logp_out) ? G.logp_out + (int64_t)sample * N : nullptr;
                    ri.out = G.out + lj;
                    ri.N = N;
                    ri.u1 = G.u1;
                }
                state = kActive;
            }
        }
        const bool act = (state == kActive);
        if (HALVES > 1 && leader) M.done[wg] = (state == kDone);

        // ---------------- layer 0: lookup gates, scan -> tile H; the one-hot
        // input's output term D0 u -> this sequence's accumulator columns,
        // which the layer-0 MMAs then add C0 h to
        const int t0 = c * CH;
        uint32_t cur = 0u;
        float lp_ref = 0.0f;
        if (act) {
            if (co_row) {
                float *co = co_row + (int64_t)c * NL * H;
                co[0] = cr[0];
                co[H] = cr[1];
                co[2 * H] = cr[2];
            }
            cur = (uint32_t)(word >> (32 * (c & 1)));
            uint32_t prev = next_prev;
            next_prev = cur >> 31;
            // the next word of spins and this chunk's reference log P are
            // fetched now, long before they are needed
            if ((c & 1) && c + 1 < nch) word = row[(c + 1) >> 1];
            if (lpref_row && (warp & 3) == 0 && t0 + lane < N) lp_ref = lpref_row[t0 + lane];
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const int x = f ? q : p;
                if (x >= t0 && x < t0 + CH) cur ^= 1u << (x - t0);
                else if (x >= 0 && x == t0 - 1) prev ^= 1u;
            }
            const int nvalid = min(CH, N - t0);
            if (nvalid < 32) cur &= (1u << nvalid) - 1u;
            // bit i = s_{t-1} for site t = t0 + i
            const uint32_t inbits = (cur << 1) | prev;
            const bool seq_start = (t0 == 0);  // site 0 has no predecessor
            float h = cr[0];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                float hv[8];
                uint32_t du[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const bool sb = (inbits >> (8 * g + i)) & 1u;
                    float a = sb ? a0_2 : a0_1, b = sb ? b0_2 : b0_1, dd = sb ? d0_2 : d0_1;
                    if (g == 0 && i == 0 && seq_start) { a = a0_0; b = b0_0; dd = d0_0; }
                    h = fmaf(a, h, b);
                    hv[i] = h;
                    du[i] = __float_as_uint(dd);
                }
                tile_store8<SH>(tileH, j, cbase + g, hv);
                tmem_st8(accZ + 8 * g, du);
            }
            cr[0] = h;
            tmem_wait_st();
        }
        publish();
        // the stream stops when all of its sequences are done, or after an
        // expired wait; both flags were written before the barrier above and
        // are rewritten only after later barriers, so every thread of the
        // stream reads the same values
        {
            bool all_done = !act;
            if (HALVES > 1) {
#pragma unroll
                for (int h = 0; h < HALVES; ++h) all_done = all_done && (M.done[s * HALVES + h] != 0);
            }
            stop = M.abort_flag[s] != 0;
            if (all_done || stop) break;
        }
        if (issuer) issue<0, SH>(s, sbase);
        if (rd_valid) readout();  // the previous chunk, while the MMAs run
        sync_wait();
        // epilogue: x1 = GELU(C0 h0 + D0 u) -> tile X
        if (act) {
            uint32_t r[32];
            tmem_ld32(accZ, r);
            tmem_wait_ld32(r);
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                float xv[8];
#pragma unroll
                for (int i = 0; i < 8; i += 2) {
                    const int k = 8 * g + i;
                    const float2 x = gelu_bf16out2(make_float2(__uint_as_float(r[k]), __uint_as_float(r[k + 1])));
                    xv[i] = x.x;
                    xv[i + 1] = x.y;
                }
                tile_store8<SH>(tileX, j, cbase + g, xv);
            }
        }
        publish();

        // ---------------- layers 1 and 2
        dense_layer<1, SH>(act, hbz1, bh1, tileX, tileH, sbase, s, accZ, accC, issuer, j, cbase, cr[1], h1,
                           sync_wait, publish);
        dense_layer<2, SH>(act, hbz2, bh2, tileX, tileH, sbase, s, accZ, accC, issuer, j, cbase, cr[2], h1,
                           sync_wait, publish);
        // x3 (in h1) is read out while the next step's layer-0 MMAs run
        if (act) {
            rd_valid = true;
            rd_final = (c + 1 == nch);
            rd_cur = cur;
            rd_t0 = t0;
            rd_lpref = lp_ref;
            rd_nup = n_up;
            rd_slot = slot;
            n_up += __popc(cur);
            if (++c == nch) state = kNeed;
        }
    }
    if (!stop && rd_valid) readout();

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

cudaError_t prepare_fwd_bf16() {
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(fwd_bf16_kernel1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fwd_bf16_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemBytes);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

cudaError_t launch_fwd_bf16(const FwdJobs &jobs, const void *packed_bf16, const float *packed_f32,
                            const F32Layout &fl, int num_sms, cudaStream_t stream, int seqs_per_stream) {
    if (fl.H != H || fl.nL != NL) return cudaErrorInvalidValue;
    if (seqs_per_stream != 1 && seqs_per_stream != 2) return cudaErrorInvalidValue;
    cudaError_t e = prepare_fwd_bf16();
    if (e != cudaSuccess) return e;
    int64_t grid = num_sms;
    const int64_t max_jobs_ctas = (max_jobs(jobs) + kSeqs - 1) / kSeqs;
    if (grid > max_jobs_ctas) grid = max_jobs_ctas;
    if (grid < 1) grid = 1;
    const uint8_t *pb = static_cast<const uint8_t *>(packed_bf16);
    if (seqs_per_stream == 1)
        fwd_bf16_kernel1<<<(int)grid, kThreads, kSmemBytes, stream>>>(jobs, pb, packed_f32, fl);
    else
        fwd_bf16_kernel<2><<<(int)grid, kThreads, kSmemBytes, stream>>>(jobs, pb, packed_f32, fl);
    return cudaGetLastError();
}

}  // namespace psr
