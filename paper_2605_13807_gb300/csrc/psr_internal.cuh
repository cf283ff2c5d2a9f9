// Internal declarations of libpsr (GPU side).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/psr.h"

namespace psr {

constexpr int kMaxLayers = 8;
constexpr int kChunkF32 = 32;   // scan chunk of the FP32 SIMT path (sites)
constexpr int kChunkGrad = 16;  // chunk of the gradient path (carries, recompute)
constexpr int kChunkBF16 = 32;  // scan chunk of the tcgen05 path (sites = MMA N)

// Device status word values (first error wins).
constexpr int kStatusOk = 0;

// Offsets (in elements) of each tensor inside the flat theta vector.
struct ThetaLayout {
    int nL, H;
    int64_t Wz[kMaxLayers], bz[kMaxLayers], Wh[kMaxLayers], bh[kMaxLayers];
    int64_t C[kMaxLayers], D[kMaxLayers];
    int64_t Wo, bo;
    int64_t total;
};
ThetaLayout theta_layout(int nL, int H);

// Packed FP32 weights used by the SIMT kernels (offsets in floats).
//   *T tensors are transposed: WzT[k][j] = W_z[j][k] so that thread j reads
//   consecutive addresses for a fixed k.
//   Layer 0 is folded into lookup tables over the input code
//   (0: t = 0, 1: s_{t-1} = 0, 2: s_{t-1} = 1):
//     A0[code][j] = sigmoid(W_z u + b_z), B0 = (1 - A0)(W_h u + b_h), DU0 = D u,
//     CD0 = W_h u + b_h (the candidate, used by the backward).
//   Readout uses the logit difference wd = W_o[1] - W_o[0], bd = b_o[1] - b_o[0].
struct F32Layout {
    int nL, H;
    int64_t WzT[kMaxLayers], WhT[kMaxLayers], CT[kMaxLayers], DT[kMaxLayers];
    int64_t bz[kMaxLayers], bh[kMaxLayers];
    int64_t A0, B0, DU0, CD0;
    int64_t wd, bd;
    int64_t total;
};
F32Layout f32_layout(int nL, int H);

// Sequence evaluations ("jobs") for the forward kernels, in up to
// kMaxGroups groups (one per lattice / sample set).  Jobs are numbered
// across the groups in order; a kernel maps a job to its group with the
// group sizes (read on the device in mode 1).
//   mode 0: job i of a group evaluates sample i from site 0 (full forward).
//   mode 1: job e evaluates the connected configuration of entries[e] =
//           (sample, p, q): the sample with sites p and q (q may be -1)
//           flipped, resuming from the chunk containing p with the stored
//           carries; the result is 1/2 sum_{t >= chunk start} (log P'_t -
//           log P_t(sample)) = log psi(s') - log psi(s).
constexpr int kMaxGroups = 8;
struct FwdGroup {
    int N;                       // sites
    int u1;                      // zero-magnetisation masking
    int W;                       // 64-bit words per bit-packed row (>= ceil(N/64) + 1)
    int64_t n_jobs;              // mode 0: number of samples; mode 1: capacity
    const int64_t *n_jobs_dev;   // mode 1: device count of valid jobs
    const uint64_t *bits;        // [n_samples][W] bit-packed spins
    const int32_t *entries;      // mode 1: [E][3]
    const float *carries_in;     // mode 1: [n][nch][nL][H]
    const float *logp_ref;       // mode 1: [n][N]
    float *out;                  // mode 0: [n] log psi; mode 1: [E] delta
    float *logp_out;             // mode 0, optional: [n][N]
    float *carries_out;          // mode 0, optional: [n][nch][nL][H]
};

// Stash of one sample for the tensor-core backward, written by its own
// forward (launch_fwd_tc): for layer l and quantity q (kStashA: gate a, kStashC:
// candidate c = W_h u + b_h, kStashH: state h, kStashY: output-map
// pre-activation y, residual included) a [H][Npad] block at
// ((l * kStashQ + q) * H) * Npad, then the readout adjoint g [Npad] at
// nL * kStashQ * H * Npad, g_t = 1/2 (s_t - P(1 | s_<t)) (0 where the
// zero-magnetisation mask forces s_t).  Npad = N rounded up to 64; every
// value at t >= N is 0.
enum { kStashA = 0, kStashC = 1, kStashH = 2, kStashY = 3, kStashQ = 4 };
__host__ __device__ inline int stash_npad(int N) { return (N + 63) & ~63; }
__host__ __device__ inline size_t stash_floats_per_sample(int nL, int H, int N) {
    return ((size_t)nL * kStashQ * H + 1) * (size_t)stash_npad(N);
}
struct FwdJobs {
    int mode;
    int n_groups;
    FwdGroup g[kMaxGroups];
    unsigned long long *job_counter;  // zeroed before launch
    int *status;                 // device status word
};

// Upper bound of the job count (mode 1 uses capacities).
inline int64_t max_jobs(const FwdJobs &jb) {
    int64_t n = 0;
    for (int i = 0; i < jb.n_groups; ++i) n += jb.g[i].n_jobs;
    return n;
}

// ---------------------------------------------------------------- launchers
// Every launcher enqueues on `stream` and returns a cudaError_t.

cudaError_t launch_pack_theta_f32(const float *theta, const ThetaLayout &tl, const F32Layout &fl,
                                  float *packed, cudaStream_t stream);
cudaError_t launch_bitpack(const uint8_t *spins, int64_t n, int N, int W, uint64_t *bits,
                           int *status, cudaStream_t stream);
// chunk: kChunkF32 (log psi, E_loc) or kChunkGrad (carries for psr_grad)
cudaError_t launch_fwd_f32(const FwdJobs &jobs, const float *packed, const F32Layout &fl,
                           int num_sms, cudaStream_t stream, int chunk = kChunkF32);

// tcgen05 path (hidden = 128, 3 layers).
size_t bf16_packed_bytes();
cudaError_t launch_pack_theta_bf16(const float *theta, const ThetaLayout &tl, void *packed,
                                   cudaStream_t stream);
// seqs_per_stream: 1 (four MMA streams of one sequence, N = 32) or 2 (two
// streams of two sequences side by side, N = 64); same results bit for bit.
cudaError_t launch_fwd_bf16(const FwdJobs &jobs, const void *packed_bf16, const float *packed_f32,
                            const F32Layout &fl, int num_sms, cudaStream_t stream,
                            int seqs_per_stream = 1);
// Sets the kernel's shared-memory attribute on the current device (once).
cudaError_t prepare_fwd_bf16();

// Hamiltonian side.
struct HamDev {
    int kind;
    int N;
    int nb;
    const int32_t *bonds;  // [nb][2]
    float J, h;
    float coeff;           // off-diagonal element per entry
};
cudaError_t launch_bonds(int Lx, int Ly, int pbc, int32_t *bonds, cudaStream_t stream);
int bond_count(int Lx, int Ly, int pbc);
cudaError_t launch_count_connected(const HamDev &hd, const uint8_t *spins, int64_t n,
                                   int64_t *counts, float *diag, cudaStream_t stream);
cudaError_t launch_exclusive_scan(const int64_t *counts, int64_t n, int64_t *offsets,
                                  cudaStream_t stream);
cudaError_t launch_fill_connected(const HamDev &hd, const uint8_t *spins, int64_t n,
                                  const int64_t *offsets, int32_t *entries, cudaStream_t stream);
cudaError_t launch_eloc_gather(const int64_t *offsets, const float *delta, const float *diag,
                               float coeff, int64_t n, float *eloc, cudaStream_t stream);
cudaError_t launch_stats(const float *eloc, int64_t n, double *stats, cudaStream_t stream);

// Standalone chunked scan h_t = a_t h_{t-1} + b_t over [n][N][H] FP32 arrays
// (psr_scan.cu).  Tile = (sequence, `units` units, `chunk` sites); flags and
// desc are the look-back arrays of n_tiles entries (flags zeroed before the
// launch; only touched when nch > 1).
struct ScanArgs {
    const float *a, *b, *h0;
    float *h;
    int N, H;
    int C;                // chunk length in sites (<= N)
    int nch;              // chunks per column
    int nub;              // unit blocks per sequence (H / units)
    int64_t n_tiles;
    unsigned long long *counter;  // zeroed before launch
    int *flags;           // [n_tiles]
    float *desc;          // [n_tiles][3][units]
    int *status;
};
bool scan_tile_valid(int H, int units, int chunk);
void scan_geometry(int64_t n, int N, int H, int units, int chunk, int *nch, int64_t *n_tiles);
cudaError_t launch_scan(const ScanArgs &g, int units, int num_sms, cudaStream_t stream);

// Exact autoregressive sampler (psr_sample.cu), FP32; per_cta samples per
// CTA: 4, 8, 16 or 32.  unif: [n][N] uniforms in [0, 1).
cudaError_t launch_sample(int per_cta, const float *packed, const F32Layout &fl, const float *unif,
                          int64_t n, int N, int u1, uint8_t *out, float *logpsi,
                          cudaStream_t stream);

// Two-dimensional patched minGRU (psr_fwd2d.cu), FP32.  Packed transposed
// weights: for layer l (din = 32 at l = 0, else H) WzT, WhxT, DT [din][H],
// WhvT, CT [H][H] (h_V and C parts), bz, bh [H]; readout Wo [16][H], bo [16].
struct F2Layout {
    int nL, H;
    int64_t WzT[kMaxLayers], WhxT[kMaxLayers], WhvT[kMaxLayers], CT[kMaxLayers], DT[kMaxLayers];
    int64_t bz[kMaxLayers], bh[kMaxLayers];
    int64_t Wo, bo;
    int64_t total;
};
F2Layout f2_layout(int nL, int H);
int64_t param_count2d(int nL, int H);
// Jobs of the 2D forward.  mode 0: sample i from the first patch row, writing
// out[i] = log psi, optionally logp_out [n][Np] and the row checkpoints
// carries_out [n][Py][fwd2d_checkpoint_floats]; mode 1: entry e = (sample,
// p, q) resumed at the patch row of spin p from carries_in, writing
// out[e] = log psi(s') - log psi(s) from logp_ref.
struct Fwd2Group {
    int Lx, Ly, u1;
    int64_t n_jobs;              // mode 0: samples; mode 1: capacity
    const int64_t *n_jobs_dev;   // mode 1: device count
    const uint8_t *spins;        // [n][Lx*Ly] sequence order
    const int32_t *entries;      // mode 1: [E][3]
    const float *carries_in;
    const float *logp_ref;
    float *out;
    float *logp_out;
    float *carries_out;
};
struct Fwd2Jobs {
    int mode;
    Fwd2Group g;
    unsigned long long *job_counter;
    int *status;
};
// Patches per row held in registers by the 2D kernels (8, 12, 16, 24, 28 or
// 32, the first >= Lx / 2);
// shared rows and row checkpoints are row2d_width + 4 floats wide.
int row2d_width(int Lx);
size_t fwd2d_checkpoint_floats(int nL, int H, int Lx);
cudaError_t launch_pack_theta_f2(const float *theta, const F2Layout &f, float *packed,
                                 cudaStream_t stream);
cudaError_t launch_fwd2d_f32(const Fwd2Jobs &jobs, const float *packed, const F2Layout &f,
                             int num_sms, cudaStream_t stream);

// Offsets of the 2D model's tensors in the flat theta (psr_bwd2d.cu).
struct T2Layout {
    int nL, H;
    int64_t Wz[kMaxLayers], bz[kMaxLayers], Wh[kMaxLayers], bh[kMaxLayers];
    int64_t C[kMaxLayers], D[kMaxLayers];
    int64_t Wo, bo;
    int64_t total;
};
T2Layout t2_layout(int nL, int H);

// Two-dimensional patched minGRU on the tensor cores (psr_fwd2d_tc.cu):
// FP16 or BF16 operands, FP32 accumulation, gates, scan, GELU and softmax; hidden
// 128 or 256, Lx <= 64.  The weights are streamed as 16 KB slices in MMA
// order (launch_pack2d_tc writes them); Sched2 lists, per slice, the matrix,
// layer, unit half, K chunk and the synchronisation before it.
enum { kMtWz = 0, kMtWhx = 1, kMtWhv = 2, kMtC = 3, kMtD = 4, kMtWo = 5 };
// Synchronisation before a slice, in this order: commit the MMAs so far to
// unit half 0's / 1's epilogue, wait for half 0's / 1's epilogue, store the
// h tile as the next row's h_V images, wait for the h_V image of the layer.
enum { kSchedC0 = 1, kSchedC1 = 2, kSchedW0 = 4, kSchedW1 = 8, kSchedStoreH = 16, kSchedWaitHv = 32 };
constexpr int kSchedMax = 320;
// op[i], what the MMA thread needs of slice i: bits 0-9 accumulator column,
// bit 10 B operand from the h tile (else x), bit 11 accumulate from the
// first K step, bits 12-13 K chunk, bits 16-23 flags, bits 24-27 layer.
struct Sched2 {
    int n;
    uint8_t type[kSchedMax], l[kSchedMax], g[kSchedMax], kc[kSchedMax], flags[kSchedMax];
    uint32_t op[kSchedMax];
};
Sched2 fwd2d_tc_schedule(int nL, int H);
// Jobs as in Fwd2Group; the row checkpoints are 16-bit h_V images:
// img_out / img_in [n][Py][nL][fwd2d_tc_image_bytes] (mode 0 writes them when
// img_out is set; mode 1 reads img_in).  scratch: fwd2d_tc_scratch_bytes,
// res: fwd2d_tc_res_floats, zero_img: fwd2d_tc_image_bytes of zeros.
struct Fwd2TcArgs {
    int mode, Lx, Ly, u1;
    int f16;            // operands FP16 (1) or BF16 (0)
    int64_t n_jobs;
    const int64_t *n_jobs_dev;
    const uint8_t *spins;
    const int32_t *entries;
    const uint8_t *img_in;
    uint8_t *img_out;
    uint8_t *scratch;
    const uint8_t *zero_img;
    float *res;
    const float *logp_ref;
    float *out;
    float *logp_out;
    const float *theta;
    T2Layout tl;
    const uint8_t *wimg;
    unsigned long long *job_counter;
    int *status;
    // set by launch_fwd2d_tc
    int W, S, R, n_slices;
    Sched2 sched;
};
bool fwd2d_tc_supported(int nL, int H, int Lx);
void fwd2d_tc_geometry(int Lx, int *W, int *S);
size_t fwd2d_tc_image_bytes(int H, int Lx);
size_t fwd2d_tc_weight_bytes(int nL, int H);
size_t fwd2d_tc_ckpt_bytes(int nL, int H, int Lx, int Ly);   // per sample
size_t fwd2d_tc_scratch_bytes(int nL, int H, int Lx, int grid);
size_t fwd2d_tc_res_floats(int H, int grid);
cudaError_t launch_pack2d_tc(const float *theta, const T2Layout &tl, bool f16, uint8_t *wimg,
                             cudaStream_t stream);
cudaError_t launch_fwd2d_tc(Fwd2TcArgs a, int grid, cudaStream_t stream);
// Reverse-mode gradient of the 2D model over n samples from the forward's
// row checkpoints; grad_rows: [n][P] (dout == NULL) or [grid][P] partial
// sums of dout_i O_k(s_i).  scratch: grid * bwd2d_scratch_floats_per_cta.
size_t bwd2d_scratch_floats_per_cta(int nL, int H);
size_t bwd2d_smem_bytes(int nL, int H, int Lx);
cudaError_t launch_bwd2d(const uint8_t *spins, int64_t n, int Lx, int Ly, int u1, const float *theta,
                         const T2Layout &tl, const float *packed, const F2Layout &f, const float *carries,
                         const float *dout, float *grad_rows, int grid, float *scratch,
                         cudaStream_t stream);

// Exact sampler of the 2D patched minGRU (psr_sample2d.cu); per_cta: 1, 2,
// 4 (hidden >= 64) or 8 (hidden >= 128) samples per CTA.  unif: [n][Np].
size_t sample2d_smem_bytes(int per_cta, int nL, int H, int Lx);
cudaError_t launch_sample2d(int per_cta, const float *packed, const F2Layout &f, const float *unif,
                            int64_t n, int Lx, int Ly, int u1, uint8_t *out, float *logpsi,
                            cudaStream_t stream);

// Deep 1D LRU (psr_lru.cu), FP32.  Packed: per layer lambda (Re, Im) and
// e^gamma [H], B^T (Re, Im) [din][H], C^T (Re, Im) [H][H], D ([2][H] at
// layer 0, else [H]), W_a^T, W_g^T [H][H], b_a, b_g [H]; readout as the logit
// difference wd [H], bd.  Jobs use FwdJobs (carries [n][nch][nL][2][H]).
struct LruLayout {
    int nL, H;
    int64_t lre[kMaxLayers], lim[kMaxLayers], gam[kMaxLayers];
    int64_t BreT[kMaxLayers], BimT[kMaxLayers], CreT[kMaxLayers], CimT[kMaxLayers], D[kMaxLayers];
    int64_t WaT[kMaxLayers], ba[kMaxLayers], WgT[kMaxLayers], bg[kMaxLayers];
    int64_t wd, bd;
    int64_t total;
};
LruLayout lru_layout(int nL, int H);
int64_t param_count_lru(int nL, int H);
constexpr int kChunkLru = 32;
// Deep LRU on the tensor cores (psr_lru_tc.cu), hidden 64: FP16 or BF16
// operands, FP32 accumulation, complex scan, GLU and readout.  Jobs and the
// FP32 complex chunk carries as for launch_lru_f32 (group 0 of g only); wimg:
// lru_tc_weight_bytes(nL), written by launch_pack_lru_tc from the packed FP32
// matrices.
constexpr int kLruSchedMax = 36;
struct LruTcArgs {
    int mode, nL, f16;
    FwdGroup g;
    LruLayout f;
    const float *pk;
    const uint8_t *wimg;
    unsigned long long *job_counter;
    int *status;
    // set by launch_lru_tc
    int R, n_slices;
    uint32_t op[kLruSchedMax];
};
bool lru_tc_supported(int nL, int H);
size_t lru_tc_weight_bytes(int nL);
cudaError_t launch_pack_lru_tc(const float *pk, const LruLayout &f, bool f16, uint8_t *wimg, cudaStream_t stream);
cudaError_t launch_lru_tc(LruTcArgs a, int grid, cudaStream_t stream);
// Exact sampler of the chain minGRU on the tensor cores (psr_sample_tc.cu),
// hidden 128, 3 layers, BF16 operands: packs its weight image (wimg:
// sample_tc_weight_bytes()) from the FP32-packed parameters, then draws
// blocks of 32 samples; spins [n][N] and (if logpsi) log psi [n] out.
bool sample_tc_supported(int nL, int H);
size_t sample_tc_weight_bytes();
cudaError_t launch_sample_tc(const float *pk, const F32Layout &fl, uint8_t *wimg, const float *unif, int64_t n,
                             int N, int u1, uint8_t *out, float *logpsi, int *status, int num_sms,
                             cudaStream_t stream);
// Exact sampler of the deep LRU on the tensor cores (psr_sample_lru_tc.cu),
// hidden 64, 1 to 3 layers: blocks of 32 samples, weights from the image
// launch_pack_lru_tc wrote (resident in shared memory), FP16 or BF16
// operands; spins [n][N] and (if logpsi) log psi [n] out.
bool lru_tc_sample_supported(int nL, int H);
size_t sample_lru_tc_smem_bytes(int nL);
cudaError_t launch_sample_lru_tc(const float *pk, const LruLayout &f, bool f16, const uint8_t *wimg,
                                 const float *unif, int64_t n, int N, int u1, uint8_t *out, float *logpsi,
                                 int *status, int num_sms, cudaStream_t stream);
cudaError_t launch_pack_theta_lru(const float *theta, const LruLayout &f, float *packed,
                                  cudaStream_t stream);
cudaError_t launch_lru_f32(const FwdJobs &jobs, const float *packed, const LruLayout &f, int num_sms,
                           cudaStream_t stream);

// Offsets of the LRU's tensors in the flat theta (psr_bwd_lru.cu).
struct TLruLayout {
    int nL, H;
    int64_t nu[kMaxLayers], th[kMaxLayers], ga[kMaxLayers], Bre[kMaxLayers], Bim[kMaxLayers];
    int64_t Cre[kMaxLayers], Cim[kMaxLayers], D[kMaxLayers], Wa[kMaxLayers], ba[kMaxLayers];
    int64_t Wg[kMaxLayers], bg[kMaxLayers];
    int64_t Wo, bo;
    int64_t total;
};
TLruLayout tlru_layout(int nL, int H);
// Reverse-mode gradient of the LRU over n samples from the forward's complex
// chunk carries [n][nch][nL][2][H]; grad_rows: [n][P] (dout == NULL) or
// [grid][P] partial sums of dout_i O_k(s_i), zeroed by the caller.
// scratch: grid * bwd_lru_scratch_floats_per_cta.
size_t bwd_lru_scratch_floats_per_cta(int nL, int H);
size_t bwd_lru_smem_bytes(int H);
cudaError_t launch_bwd_lru(const uint64_t *bits, int64_t n, int N, int W, int u1, const float *theta,
                           const TLruLayout &tl, const float *packed, const LruLayout &f,
                           const float *carries, const float *dout, float *grad_rows, int grid,
                           float *scratch, cudaStream_t stream);
// Exact sampler of the LRU (psr_sample_lru.cu); per_cta 4, 8 or 16.
size_t sample_lru_smem_bytes(int per_cta, int nL, int H);
cudaError_t launch_sample_lru(int per_cta, const float *packed, const LruLayout &f, const float *unif,
                              int64_t n, int N, int u1, uint8_t *out, float *logpsi, cudaStream_t stream);

// c4v symmetrisation and VMC-step kernels (psr_vmc.cu).
cudaError_t launch_c4v_images(const uint8_t *s, int64_t n, int L, uint8_t *out, cudaStream_t st);
cudaError_t launch_c4v_pick(const uint8_t *s, const float *u, int64_t n, int L, uint8_t *out,
                            cudaStream_t st);
cudaError_t launch_c4v_entries(const int32_t *entries, const int64_t *count, int64_t cap, int L,
                               int32_t *out, cudaStream_t st);
cudaError_t launch_sym_logpsi(const float *lp8, int64_t n, float *out, cudaStream_t st);
cudaError_t launch_sym_delta(const int32_t *entries, const int64_t *count, int64_t cap,
                             const float *lp8, int64_t n, const float *delta8, float *out,
                             cudaStream_t st);
cudaError_t launch_vmc_dout(const float *eloc, const double *stats, const float *lp8, int64_t n,
                            int n_img, float *dout, cudaStream_t st);
cudaError_t launch_adam(const float *theta, const float *grad, int64_t P, float lr, float b1, float b2,
                        float eps, int step, float *m, float *v, float *out, cudaStream_t st);

// Backward (FP32).  Samples of up to kMaxGroups sample sets (one lattice
// each) in one launch: group g holds samples first[g] .. first[g+1]-1 of the
// launch; its chunk carries come from a forward on kChunkGrad-site chunks;
// rows: [n][P] O_k rows (dout == NULL) or per-CTA partial sums of
// dout_i O_k(s_i) ([grid][P], zeroed by the caller).
struct BwdGroup {
    const uint64_t *bits;  // [n][W] bit-packed spins
    int N, W, u1;
    const float *carries;  // [n][nch][nL][H]
    const float *dout;     // [n] or NULL
    float *rows;
};
struct BwdJobs {
    int n_groups;
    int64_t first[kMaxGroups + 1];
    BwdGroup g[kMaxGroups];
};
// Tensor-core backward (hidden 128; psr_bwd_tc.cu): one layer at a time over
// the samples of a batch, from the FP32 forward's stash.  Arrays [n][H][Np]
// FP32 (unit-major, Np = stash_npad(N)).
struct BwdTcArgs {
    int n, N, Np, W, nL, l;
    int64_t P;
    ThetaLayout tl;
    const float *stash;      // batch stash, stash_stride floats per sample
    int64_t stash_stride;
    const float *wd;         // readout logit-difference weights [H]
    const uint8_t *images;   // launch_pack_bwd_tc output
    const uint64_t *bits;    // [n][W] bit-packed spins of the batch
    const float *gx_in;      // gradient w.r.t. this layer's output x^{l+1} (l < nL - 1)
    float *gx_out;           // gradient w.r.t. its input x^l (l >= 1)
    float *gy;               // gx_in (.) GELU'(y) of this layer
    const float *gy_up;      // gy of layer l + 1 (its residual input is h^l)
    float *gh;               // C^T gy
    float *dz, *dc;          // gate and candidate adjoints
    float *rows;             // [n][P] O_k rows of the batch
    const float *pk;         // packed FP32 weights (layer-0 tables, biases, readout)
    F32Layout fl;
    int u1;
    int *status;
};
// The forward that fills the stash of a batch (all layers and the readout
// adjoint) with the same split-BF16 tensor-core products.
cudaError_t launch_fwd_tc(const BwdTcArgs &A, int num_sms, cudaStream_t stream);
size_t bwd_tc_image_bytes(int nL);
cudaError_t launch_pack_bwd_tc(const float *theta, const ThetaLayout &tl, void *images, cudaStream_t stream);
cudaError_t launch_bwd_tc_layer(const BwdTcArgs &A, int num_sms, cudaStream_t stream);
// Sets the tensor-core backward kernels' shared-memory attributes (once per
// device; call before a stream capture that will contain their launches).
cudaError_t prepare_bwd_tc();

// Sets the backward kernel's shared-memory attribute (done by every launch;
// call it before a stream capture that will contain a launch).
cudaError_t prepare_bwd_f32(int H, int nL);
cudaError_t launch_bwd_f32_groups(const BwdJobs &bj, const float *theta, const ThetaLayout &tl,
                                  const float *packed, const F32Layout &fl, int grid, float *tape,
                                  int *status, cudaStream_t stream);
size_t bwd_tape_floats_per_cta(int nL, int H);
cudaError_t launch_bwd_f32(const uint64_t *bits, int64_t n, int N, int W, int u1,
                           const float *theta, const ThetaLayout &tl, const float *packed,
                           const F32Layout &fl, const float *carries, const float *dout,
                           float *grad_rows, int grid, float *tape, int *status,
                           cudaStream_t stream);
size_t bwd_smem_bytes(int H, int nL);
cudaError_t launch_reduce_rows(const float *partial, int rows, int64_t P, float *out,
                               cudaStream_t stream);

}  // namespace psr
