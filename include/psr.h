/*
 * psr.h -- C ABI of libpsr, the GB300 (sm_103a) hot path of PSR-NQS
 * variational Monte Carlo (parallel-scan recurrent neural quantum states,
 * arXiv 2605.13807).
 *
 * The library evaluates, for many spin configurations at once,
 *   - the autoregressive log-amplitude log psi(s) of a stack of minGRU layers
 *     (Sec. II.C, Eq. minGRU) run along the zigzag ordering of the lattice
 *     (Sec. II.F), with output map x~ = C h + D u, GELU and the residual
 *     s^(l) = h^(l-1) for l >= 2 (Sec. II.F-G); the recurrence
 *     h_t = a_t * h_{t-1} + b_t is evaluated as a chunked scan (Sec. II.A);
 *   - the local energy of the Heisenberg model (Sec. III.C) or the
 *     transverse-field Ising model (Sec. III.B) over every configuration
 *     connected to a sample by an off-diagonal term (Sec. II.A, local-energy
 *     paragraph);
 *   - the parameter gradient d log psi / d theta per sample (O_k) or its
 *     weighted sum, as used by the VMC energy-gradient estimator
 *     (Sec. III.B, optimisation paragraph).
 *
 * Conventions shared by every call
 * --------------------------------
 * Pointers.  Every array argument may be a device pointer or a host pointer;
 * the library asks CUDA which it is.  Device arrays are used in place and the
 * call is asynchronous on the context's stream.  Host inputs are copied to
 * the device and host outputs are copied back inside the call, which then
 * synchronises the stream before returning.  The caller owns every array;
 * the library never frees caller memory.  Scratch memory comes from the
 * context's workspace, which grows on demand (cudaMalloc) and is released by
 * psr_context_destroy.
 *
 * Spins.  uint8 [n][N] row-major, one byte per site with value 0 (down,
 * sigma^z = -1) or 1 (up, sigma^z = +1), given in SEQUENCE order: lattice
 * site (i, j) (column i, row j, 0-based) sits at position
 *   pos(i, j) = j * Lx + (j even ? i : Lx - 1 - i)
 * which is the zigzag path of Sec. II.F (predecessor (i - (-1)^j, j)).
 * For a chain Ly = 1 and pos = i.
 *
 * Parameters theta.  float32, P = psr_param_count(n_layers, hidden) values,
 * for each layer l = 0 .. n_layers-1 with d_in = 2 for l = 0 and hidden
 * otherwise, row-major:
 *   W_z[hidden][d_in], b_z[hidden], W_h[hidden][d_in], b_h[hidden],
 *   C[hidden][hidden], D[hidden][d_in]
 * followed by the readout W_o[2][hidden], b_o[2].  Layer 0 sees
 * onehot(s_{t-1}) (the zero vector at t = 0); layer l >= 1 sees the output of
 * layer l-1.  The conditional of site t is softmax(W_o x_t + b_o) over
 * s_t in {0, 1}, and log psi = 1/2 sum_t log P(s_t | s_<t).  With n_layers = 3
 * and hidden = H, P = 9 H^2 + 14 H + 2.
 *
 * u1_mask.  When set, once N/2 up (or N/2 down) spins precede site t the
 * conditional forces the other value (probability one), so log psi is
 * finite exactly on the zero-magnetisation sector.  Requires N even.
 *
 * Precision.  PSR_FP32: every projection in FP32 on CUDA cores (the plain
 * path).  PSR_BF16: the dense projections of layers >= 1 and the output maps
 * run on the tensor cores (tcgen05) with BF16 operands and FP32
 * accumulation; the gates, scan carry, softmax, log-psi sums and every
 * reduction stay in FP32 (hidden = 128 only).  psr_grad always computes in
 * FP32.  PSR_FP16 (FP16 operands, FP32 accumulation) applies to the 2D
 * patched model's forward only (PSR_EUNSUPPORTED elsewhere).
 *
 * Errors.  Every call returns PSR_OK or an error code; nothing traps.
 * Asynchronous device-side failures (a bounded wait that expired, an
 * invalid spin value) are recorded in the context's status word and
 * returned by the next call that synchronises (psr_context_sync or a call
 * with host buffers).
 */
#ifndef PSR_H
#define PSR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PSR_OK = 0,
    PSR_EINVAL = 1,      /* bad argument: null pointer, size, shape, Hamiltonian */
    PSR_ENOMEM = 2,      /* device allocation failed */
    PSR_ECUDA = 3,       /* a CUDA runtime call failed */
    PSR_ETIMEOUT = 4,    /* a bounded device-side wait expired */
    PSR_EDEVICE = 5,     /* a device-side check failed (e.g. spin byte not 0/1) */
    PSR_EUNSUPPORTED = 6 /* valid request the library does not implement */
};

enum { PSR_FP32 = 0, PSR_BF16 = 1, PSR_FP16 = 2 };
enum { PSR_HEISENBERG = 0, PSR_TFIM = 1 };

typedef struct psr_context psr_context;

/* Model description.  theta: P floats (host or device), caller-owned. */
typedef struct {
    int32_t n_layers;  /* >= 1, <= 8 */
    int32_t hidden;    /* 32, 64 or 128 (PSR_BF16: 128) */
    int32_t u1_mask;   /* 0 or 1 */
    int32_t precision; /* PSR_FP32, PSR_BF16 or (2D model only) PSR_FP16 */
    const float *theta;
    psr_context *ctx;
} psr_params;

/* Lattice Hamiltonian.  N = Lx * Ly sites.
 *   PSR_HEISENBERG: H = J sum_<pq> S_p . S_q, S = sigma / 2 (Sec. III.C).
 *     Diagonal (J/4) sum sigma_p sigma_q; each antiparallel bond (p, q)
 *     connects s to s with both spins exchanged, element J/2, times -1 when
 *     marshall = 1 (the Marshall sign of Sec. III.C; bipartite lattices only).
 *   PSR_TFIM: H = -J sum_<pq> sigma^z_p sigma^z_q - h sum_p sigma^x_p
 *     (Sec. III.B); every site flip is connected with element -h.
 * Bonds: nearest neighbours of the Lx x Ly square lattice (a chain when
 * Ly = 1); with pbc = 1 each dimension of length >= 3 wraps around.
 * Canonical bond order: lattice sites in row-major order (row j major,
 * column i minor), for each the bond to (i+1, j) then to (i, j+1); each
 * stored as (min pos, max pos). */
typedef struct {
    int32_t kind;
    int32_t Lx, Ly;
    int32_t pbc;
    int32_t marshall;
    double J;
    double h;
} psr_hamiltonian;

/* Creates a context bound to a CUDA stream (a cudaStream_t passed as
 * void*; NULL selects the legacy default stream) on the current device.
 * Returns PSR_EINVAL for a null out pointer, PSR_ECUDA if the device cannot
 * be queried. */
int psr_context_create(psr_context **out, void *stream);

/* Synchronises the context's stream, frees its workspace and the context. */
int psr_context_destroy(psr_context *ctx);

/* Synchronises the context's stream and returns (then clears) the first
 * device-side error recorded since the last synchronising call. */
int psr_context_sync(psr_context *ctx);

/* Number of float parameters of the layout described above. */
int psr_param_count(int32_t n_layers, int32_t hidden, int64_t *P);

/* log psi of n configurations of N = L sites (Sec. III.B: psi = prod_t
 * sqrt(P(s_t | s_<t)), Sec. II.C recurrence, Sec. II.A scan).
 * spins: uint8 [n][L]; out: float [n].  n >= 1, L >= 1.
 * Configurations outside the support (u1_mask) give -inf. */
int psr_logpsi(const psr_params *params, const uint8_t *spins, int64_t n, int32_t L,
               float *out);

/* Local energy of n samples (Sec. II.A, local-energy paragraph):
 *   E_loc(s) = diag(s) + sum_{s'} H_{s s'} psi(s') / psi(s)
 * summed over every connected configuration s' (ragged: Heisenberg has one
 * per antiparallel bond, TFIM one per site).  Each psi(s')/psi(s) is
 * exp(log psi(s') - log psi(s)); the forward of s' resumes from the scan
 * chunk that contains the first changed site, reusing the sample's stored
 * chunk carries (identical result, fewer site evaluations).
 * samples: uint8 [n][Lx*Ly]; out: float [n] E_loc; stats: double [3]
 * {mean, unbiased variance, standard error sqrt(var/n)} accumulated in FP64,
 * or NULL.  PSR_EINVAL for marshall = 1 on a non-bipartite lattice (a
 * wrapped dimension of odd length). */
int psr_local_energy(const psr_params *params, const uint8_t *samples, int64_t n,
                     const psr_hamiltonian *ham, float *out, double *stats);

/* Connected-configuration generator on its own (bit-exact, deterministic):
 * offsets: int64 [n+1] (CSR over samples), entries: int32 [capacity][3]
 * rows (sample, p, q) in sample-major then canonical bond order (TFIM: site
 * order, q = -1), diag: float [n] diagonal energy, total: int64 on the HOST
 * receiving the number of entries.  capacity must be at least n times the
 * bond count (Heisenberg) or n * N (TFIM); PSR_EINVAL otherwise.
 * This call synchronises the stream to report total. */
int psr_connected(psr_context *ctx, const uint8_t *samples, int64_t n,
                  const psr_hamiltonian *ham, int64_t *offsets, int32_t *entries,
                  int64_t capacity, float *diag, int64_t *total);

/* One sample set of a mixed batch: its own lattice, size and Hamiltonian,
 * the model shared with the other items. */
typedef struct {
    const uint8_t *samples; /* uint8 [n][Lx*Ly] in sequence order, host or device */
    int64_t n;              /* >= 1 */
    psr_hamiltonian ham;
    int32_t u1_mask;        /* zero-magnetisation masking for this item (params->u1_mask is ignored) */
    float *out;             /* float [n]: E_loc */
    double *stats;          /* double [3] {mean, variance, standard error} or NULL */
} psr_batch_item;

/* Local energy of up to 8 sample sets that share one model (e.g. several
 * lattice sizes and both Hamiltonians).  Each item gets exactly what
 * psr_local_energy would give it, but the sample forwards of all items run
 * in one launch and the connected configurations of all items (ragged over
 * samples and lattices) in one persistent launch.  When graphs are enabled
 * on the context (psr_context_set_graphs), the context's stream is not the
 * legacy default stream and every array is a device array, the launch
 * sequence is captured into a CUDA graph on the first call and replayed by
 * later calls with the same arguments (same pointers and sizes; the arrays'
 * contents may change).  PSR_EINVAL for n_items outside 1..8 or any item
 * psr_local_energy would reject. */
int psr_local_energy_batch(const psr_params *params, const psr_batch_item *items,
                           int32_t n_items);

/* One sample set of a full mixed-batch step: its own lattice, size and
 * Hamiltonian, the model shared with the other items.  Each output may be
 * NULL (not computed); at least one must be given. */
typedef struct {
    const uint8_t *samples; /* uint8 [n][Lx*Ly] in sequence order, host or device */
    int64_t n;              /* >= 1 */
    psr_hamiltonian ham;    /* lattice (and, for eloc, the Hamiltonian) */
    int32_t u1_mask;        /* zero-magnetisation masking for this item (params->u1_mask is ignored) */
    float *logpsi;          /* float [n]: log psi, as psr_logpsi gives it, or NULL */
    float *eloc;            /* float [n]: E_loc, as psr_local_energy gives it, or NULL */
    double *stats;          /* double [3] {mean, variance, standard error} of E_loc, or NULL (needs eloc) */
    float *grad;            /* float [n][P]: O_k rows, as psr_grad with dout = NULL gives them, or NULL */
} psr_step_item;

/* The hot path of one VMC step (log psi, per-sample O_k = d log psi / d theta
 * and E_loc over every connected configuration; Sec. II.A local-energy
 * paragraph, Sec. III.B) for up to 8 sample sets that share one model, e.g.
 * several lattice sizes and both Hamiltonians.  Each item gets what
 * psr_logpsi, psr_local_energy and psr_grad (dout = NULL) would give it with
 * the same forward shape (psr_context_set_fwd_shape): bit for bit.  One
 * launch covers the sample forwards of all items, one persistent launch the
 * connected configurations of all items (ragged over samples and lattices),
 * one launch the gradient forwards and one the reverse-scan gradients; the
 * generator, packing and gather kernels run per item.  The forward shape is
 * tuned per batch (sizes of all items) when the autotuner is on.  With
 * graphs enabled (psr_context_set_graphs), a non-default stream and device
 * arrays only, the launch sequence is captured into a CUDA graph on the
 * first call (after the autotuner, if on, has tuned the batch on an earlier
 * uncaptured call) and replayed by later calls with the same arguments.
 * PSR_EINVAL for n_items outside 1..8, an item with no output, stats without
 * eloc, or any item the single calls would reject. */
int psr_step_batch(const psr_params *params, const psr_step_item *items, int32_t n_items);

/* Enables (1) or disables (0) CUDA-graph capture and replay of
 * psr_local_energy_batch and psr_step_batch on this context. */
int psr_context_set_graphs(psr_context *ctx, int enable);

/* Gradient of log psi (Sec. III.B: stochastic energy-gradient estimates).
 * dout == NULL: dparams is float [n][P] with row i = O_k(s_i) = d log psi(s_i)
 *   / d theta (per-sample, e.g. for a covariance / SR solve).
 * dout != NULL (float [n]): dparams is float [P] = sum_i dout_i O_k(s_i).
 * The forward is recomputed chunk by chunk from stored chunk-boundary carries
 * and the recurrence is differentiated by a reverse scan
 * lambda_t = dL/dh_t + a_{t+1} lambda_{t+1}.  Computed in FP32. */
int psr_grad(const psr_params *params, const uint8_t *spins, int64_t n, int32_t L,
             const float *dout, float *dparams);

/* log psi exactly as psr_logpsi computes it, for callers that may not
 * allocate device memory (the paper has no counterpart; this is a service of
 * the library).  Such callers include programs whose device memory belongs
 * to another runtime's pool, latency-critical loops that cannot take the
 * synchronisation an allocation may imply, and plug-ins that are not given
 * the allocation API.  Nothing is allocated: all scratch lives in one fixed
 * 8 MiB array per device inside the library (held from module load until the
 * process exits).  params->ctx is ignored; the work is queued on `stream`
 * (a cudaStream_t passed as void*, NULL = legacy default stream) and the call
 * returns without synchronising.
 * theta, spins and out must all be device arrays (PSR_EINVAL otherwise).
 * Any n is accepted (samples are processed in batches that fit the array);
 * a configuration longer than 33,554,368 sites is rejected with PSR_EINVAL.
 * The first call on a device, with that device current, performs a one-time
 * set-up (it looks up the array's device address); make that first call
 * before any stream capture begins.  Every call shares the array and leaves
 * its contents behind; calls whose work overlaps on one device race on it.
 * The call returns before its kernels run, so device-side failures (a spin
 * byte other than 0/1: PSR_EDEVICE; an expired bounded wait: PSR_ETIMEOUT; a
 * tensor-memory allocation not at column 0: PSR_EDEVICE) are not in its
 * return code: they are recorded in a status word inside the array, and
 * `out` may then be partly or wholly unwritten.  Read that word with
 * psr_noalloc_status before the next call on the device clears it. */
int psr_logpsi_noalloc(const psr_params *params, const uint8_t *spins, int64_t n, int32_t L,
                       float *out, void *stream);

/* Device-side status of the most recent psr_logpsi_noalloc call on the
 * current device (service of the library; the paper has no counterpart).
 * Synchronises `stream` (the stream that call used), then returns the
 * status word: PSR_OK, PSR_EDEVICE or PSR_ETIMEOUT as described above, or
 * PSR_ECUDA if the stream or the read failed.  Allocates nothing; the word
 * is left as it is (the next psr_logpsi_noalloc call clears it). */
int psr_noalloc_status(void *stream);

/* Standalone scan of the diagonal linear recurrence at the heart of the
 * minGRU layer (Eq. minGRU with a_t = 1 - z_t, b_t = z_t h~_t), evaluated as
 * a chunked parallel scan (Sec. II.A, parallel-scan paragraph):
 *     h_t = a_t * h_{t-1} + b_t,  t = 0 .. N-1,  h_{-1} = h0 (zero if NULL),
 * element-wise over H units, independently for each of n sequences.
 * a, b, h: float [n][N][H] row-major (H contiguous); h0: float [n][H] or
 * NULL.  Host or device arrays (device arrays must be 16-byte aligned);
 * h may alias a or b.  The kernel reads a and b and writes h once each
 * (12 bytes per element from HBM); between chunks of one sequence the carry
 * is passed through a look-back array in the workspace.
 * PSR_EINVAL: null a, b or h, n < 1, N outside 1 .. 2^30, H not a positive
 * multiple of 4, or a misaligned device array. */
typedef struct {
    int32_t units; /* units per tile: 4, 16, 32 or 128, dividing H */
    int32_t chunk; /* sites per tile (>= N: one chunk per sequence) */
} psr_scan_tile;

int psr_scan(psr_context *ctx, const float *a, const float *b, const float *h0, int64_t n,
             int32_t N, int32_t H, float *h);

/* psr_scan with an explicit tile shape (PSR_EINVAL for an invalid one). */
int psr_scan_tiled(psr_context *ctx, const float *a, const float *b, const float *h0, int64_t n,
                   int32_t N, int32_t H, float *h, const psr_scan_tile *tile);

/* The tile shape psr_scan will use for (n, N, H) on this context: the
 * autotuned one if (n, N, H) has been tuned (*tuned = 1), else the built-in
 * default (*tuned = 0).  tuned may be NULL. */
int psr_scan_tile_for(psr_context *ctx, int64_t n, int32_t N, int32_t H, psr_scan_tile *tile,
                      int32_t *tuned);

/* Exact autoregressive sampling (Sec. II.A and Sec. III.B: the conditionals
 * P(s_t | s_<t) of the model are drawn site by site along the zigzag
 * sequence, so the n samples are exact and independent).  The caller
 * supplies the random numbers: uniforms float [n][L] in [0, 1), and site t
 * of sample i is s_t = 1 iff uniforms[i][t] < P(s_t = 1 | s_<t) (with
 * u1_mask, the forced value where the mask forces one).  spins: uint8
 * [n][L] output in sequence order; logpsi: float [n] output (log psi of the
 * drawn sample) or NULL.  PSR_FP32: FP32 on CUDA cores.  PSR_BF16 at the
 * BF16 forward's shape (hidden 128, 3 layers): on the tensor cores, the
 * conditionals of the BF16 model psr_logpsi evaluates (BF16 operands, FP32
 * gates, scan and readout; a draw can differ from the exact model's only
 * where u lies within the BF16 error of P); other BF16 shapes draw in FP32.
 * The result does not depend on how samples are grouped into CTAs (a tile
 * shape the autotuner chooses, or blocks of 32 on the tensor cores), so
 * equal uniforms give equal samples.
 * PSR_EINVAL: what psr_logpsi rejects, or null uniforms / spins. */
int psr_sample(const psr_params *params, const float *uniforms, int64_t n, int32_t L,
               uint8_t *spins, float *logpsi);

/* Samples per CTA psr_sample will use for (n, L, n_layers, hidden) on this
 * context: the autotuned value if that shape has been tuned (*tuned = 1),
 * else the default 8 (*tuned = 0).  tuned may be NULL. */
int psr_sample_tile_for(psr_context *ctx, int64_t n, int32_t L, int32_t n_layers, int32_t hidden,
                        int32_t *per_cta, int32_t *tuned);

/* Self-test of the bounded device waits (failure detection without a GPU
 * fault).  Runs a two-chunk scan of one short sequence whose first chunk is
 * deliberately left unprocessed, so the second chunk's look-back wait finds
 * a flag that nothing sets and gives up at its 2 s limit.  Returns
 * PSR_ETIMEOUT (read from, and cleared in, the context's status word) when
 * the bound works; the context stays usable afterwards.  elapsed_ms (may be
 * NULL) receives the device time of the scan.  Synchronises the stream.
 * PSR_EINVAL during stream capture.  The paper has no counterpart. */
int psr_selftest_wait_timeout(psr_context *ctx, float *elapsed_ms);

/* Enables (1) or disables (0) the autotuner of this context.  While enabled,
 * the first call of psr_scan, psr_sample, psr_logpsi, psr_local_energy,
 * psr_local_energy_batch or psr_step_batch for a shape it has not seen
 * (scan: n, N, H; sample: n, L, layers, hidden; the forwards: precision,
 * kind of call and the sizes of every sample set), when not being captured
 * into a graph, times every candidate (scan: unit-block width x chunk
 * length; sample: samples per CTA; the fused forwards: their shape, see
 * psr_context_set_fwd_shape) on its own inputs with CUDA events, keeps the
 * fastest for the context's lifetime and then computes its result with it;
 * that first call synchronises the stream.  Every scan tile computes the
 * same recurrence (results differ only by FP32 rounding of the composed
 * maps); every sampler tile gives identical samples; the BF16 forward shapes
 * give identical results, the FP32 chunk lengths results that differ by FP32
 * summation order. */
int psr_context_set_autotune(psr_context *ctx, int enable);

/* Shape of the fused forward kernels (log psi, and the sample and connected
 * forwards of E_loc).  precision PSR_BF16: sequences per MMA stream of the
 * tcgen05 kernel, 1 (four streams per SM, MMA N = 32 sites) or 2 (two
 * streams, N = 64: each shared-memory weight slice serves twice the sites);
 * PSR_FP32: scan chunk of the SIMT kernel, 32 or 16 sites.  shape 0 returns
 * the choice to the context (the autotuned shape, else the built-in
 * default); any other value fixes it for every later call.  PSR_EINVAL for
 * another shape.  The paper has no counterpart (a tuning choice). */
int psr_context_set_fwd_shape(psr_context *ctx, int32_t precision, int32_t shape);

/* The forward shape a call would use on this context: what = 0 for
 * psr_logpsi of n[0] configurations of L[0] sites, 1 for psr_local_energy
 * of n[0] samples of L[0] sites (n_sets = 1 for both), 2 for
 * psr_local_energy_batch or a psr_step_batch whose n_sets items all ask
 * for E_loc (n[i] samples of L[i] sites each, in item order).  *tuned = 1
 * when it comes from the autotuner.  tuned may be NULL. */
int psr_fwd_shape_for(psr_context *ctx, int32_t precision, int32_t what, int32_t n_sets,
                      const int64_t *n, const int32_t *L, int32_t *shape, int32_t *tuned);

/* ---------------------------------------------------------------------
 * The paper's two-dimensional patched minGRU (Sec. II.F, two-dimensional
 * recurrences; Sec. II.G, residual connections).  The Lx x Ly spin lattice
 * (Lx, Ly even) is cut into 2 x 2 patches; patch (i, j) holds the spins
 * (2i + dx, 2j + dy) and takes the value v = sum s 2^(2 dy + dx) in 0..15.
 * Patches are visited along the zigzag path of the patch lattice (row j left
 * to right when j is even) with causal predecessors H = (i - (-1)^j, j) and
 * V = (i, j - 1) (zero outside the lattice).  Layer input u_0 =
 * (onehot16(v_H), onehot16(v_V)), u_l = x_l for l >= 1;
 *   z = sigma(W_z u + b_z),  h~ = W_h [u, h_V] + b_h,  h = z h_H + (1 - z) h~,
 *   x_{l+1} = GELU(C h + D u + s_l),  s_l = h_{l-1} for l >= 2, else 0;
 * the conditional of a patch is softmax(W_o x_{nL} + b_o) over its 16
 * values (with u1_mask: over the values that keep both the up and the down
 * count at most N/2), log psi = 1/2 sum log P.
 * Spins are uint8 [n][Lx * Ly] in the sequence order of the SPIN lattice,
 * as for the calls above.  theta: float, per layer l (din = 32 at l = 0,
 * else hidden) W_z[hidden][din], b_z[hidden], W_h[hidden][din + hidden]
 * (the last hidden columns act on h_V), b_h[hidden], C[hidden][hidden],
 * D[hidden][din]; then W_o[16][hidden], b_o[16]; psr2d_param_count gives
 * the length (12 H^2 + 118 H + 16 for three layers).
 * Evaluated row by row: within a patch row all sites share one batched
 * projection and one scan (the row starts from h_H = 0).  hidden may also
 * be 256 (the paper's 52 x 52 model) with at most 4 layers.
 * Precision PSR_FP32: every product in FP32 on CUDA cores.  PSR_FP16 and
 * PSR_BF16: every product (W_z u, W_h [u, h_V], C h, D u, W_o x) on the
 * tensor cores (tcgen05) with 16-bit operands (FP16, 11-bit significand;
 * BF16, 8-bit) and FP32 accumulation; the gates, scan, residual, GELU,
 * softmax and log-psi sums in FP32; hidden 128 or 256.  The stored row
 * states (the h_V of the next row, the checkpoints connected
 * configurations resume from) are 16-bit in that format.  Measured against
 * the FP64 oracle at hidden 256: FP16 meets the BF16 path's stated bounds
 * (|d log psi| <= 2e-2 + 2e-5 |log psi|, E_loc 1e-3 relative); BF16
 * operands meet the log psi bound but reach about 2e-3 on E_loc.
 * psr2d_sample and psr2d_grad compute in FP32 at every precision.
 * PSR_EUNSUPPORTED for Lx > 64 (more than 32 patches per row), hidden 256
 * with more than 4 layers, or a 16-bit precision with hidden 32 or 64;
 * PSR_EINVAL for odd Lx or Ly and what psr_logpsi rejects. */
int psr2d_param_count(int32_t n_layers, int32_t hidden, int64_t *P);

int psr2d_logpsi(const psr_params *params, const uint8_t *spins, int64_t n, int32_t Lx, int32_t Ly,
                 float *out);

/* Exact samples of the 2D model (Sec. III.B): patch t of sample i takes the
 * smallest value v whose cumulative conditional probability (values in
 * increasing order, masked ones skipped) exceeds uniforms[i][t]; uniforms
 * float [n][Np], Np = (Lx/2)(Ly/2), in path order.  spins: uint8 [n][Lx*Ly]
 * output in sequence order; logpsi: float [n] or NULL.  FP32; the result
 * does not depend on how samples are grouped into CTAs (a tile shape the
 * autotuner chooses).  Requirements as psr2d_logpsi. */
int psr2d_sample(const psr_params *params, const float *uniforms, int64_t n, int32_t Lx, int32_t Ly,
                 uint8_t *spins, float *logpsi);

/* Gradient of log psi of the 2D model, as psr_grad for the chain model:
 * dout == NULL gives per-sample O_k rows [n][P], otherwise the dout-weighted
 * sum [P].  Rows of patches are recomputed from the forward's row
 * checkpoints and differentiated from the last row to the first, the
 * adjoint of each row's states reaching the row above through
 * W_h^T (the h_V columns).  FP32; every hidden size psr2d_logpsi takes. */
int psr2d_grad(const psr_params *params, const uint8_t *spins, int64_t n, int32_t Lx, int32_t Ly,
               const float *dout, float *dparams);

/* Local energy of the 2D model over every connected configuration, as
 * psr_local_energy computes it for the chain model; a connected
 * configuration is resumed at the patch row of its first flipped spin from
 * the sample's stored row states. */
int psr2d_local_energy(const psr_params *params, const uint8_t *samples, int64_t n,
                       const psr_hamiltonian *hamiltonian, float *out, double *stats);

/* c4v-symmetrised 2D model on an L x L lattice (Lx == Ly, else
 * PSR_EINVAL): psi_sym(s) = sqrt(1/8 sum_g psi(g s)^2) over the 8
 * operations of c4v (as psr_sym_logpsi, with the 2D model's psi), and its
 * local energy E_loc(s) = diag(s) + sum_e c_e psi_sym(s'_e) / psi_sym(s).
 * Every image of a connected configuration is a connected configuration
 * of the sample's image and resumes from that image's stored row states.
 * Requirements, arrays and errors as psr2d_logpsi / psr2d_local_energy;
 * 8x the work of the unsymmetrised calls. */
int psr2d_sym_logpsi(const psr_params *params, const uint8_t *spins, int64_t n, int32_t Lx, int32_t Ly,
                     float *out);
int psr2d_sym_local_energy(const psr_params *params, const uint8_t *samples, int64_t n,
                           const psr_hamiltonian *hamiltonian, float *out, double *stats);

/* ---------------------------------------------------------------------
 * The paper's deep 1D LRU ansatz (Sec. II.B Eq. lru; Sec. II.G 1D residual;
 * Sec. III.B: each layer an LRU followed by a single-layer GLU feed-forward
 * network).  With d = d_h = hidden and layer input u_t (onehot(s_{t-1}) at
 * layer 0, zero at t = 0; x_t of the layer below otherwise):
 *   h_t = lambda h_{t-1} + e^gamma (B u_t),  lambda = exp(-e^nu + i e^theta),
 *   y_t = Re(C h_t) + D u_t,
 *   x_t = (W_a y_t + b_a) sigmoid(W_g y_t + b_g) + [layer >= 1] u_t,
 * with complex B, C; D is a hidden x 2 matrix at layer 0 (one-hot input) and
 * diagonal (hidden entries) above.  Readout, u1_mask and spins as for
 * psr_logpsi.  theta: float, per layer nu[H], theta[H], gamma[H],
 * B_re[H][din], B_im[H][din], C_re[H][H], C_im[H][H], D ([H][2] at layer 0,
 * else [H]), W_a[H][H], b_a[H], W_g[H][H], b_g[H] (din = 2 at layer 0, else
 * H), then W_o[2][H], b_o[2]; 16 H^2 + 25 H + 2 values for three layers.
 * Precision: PSR_FP32 computes in FP32 on CUDA cores (hidden 32, 64 or 128,
 * up to 8 layers).  PSR_FP16 and PSR_BF16 run psr_lru_logpsi and
 * psr_lru_local_energy on the tensor cores at hidden 64 with 1 to 4 layers:
 * the products e^gamma B u, Re(C h) and [W_a; W_g] y and the readout with
 * 16-bit operands (FP16 or BF16) and FP32 accumulation; the complex scan,
 * D u, GLU, residual, softmax and sums in FP32.  Bounds of the 16-bit path
 * against the exact model: |d log psi| <= 2e-2 + 2e-5 |log psi| and E_loc
 * within 1e-3 (|diag| + |E_loc - diag|) with FP16 operands (BF16: about
 * twice that).  Other shapes at 16-bit precision return PSR_EUNSUPPORTED.
 * psr_lru_sample at 16-bit precision draws from the conditionals of that
 * tensor-core model (up to 3 layers; 4 layers draw in FP32); psr_lru_grad
 * computes in FP32 at every precision. */
int psr_lru_param_count(int32_t n_layers, int32_t hidden, int64_t *P);

int psr_lru_logpsi(const psr_params *params, const uint8_t *spins, int64_t n, int32_t L, float *out);

/* Local energy of the LRU ansatz over every connected configuration
 * (connected configurations resume at their first flipped site's chunk from
 * the sample's complex chunk carries), as psr_local_energy. */
int psr_lru_local_energy(const psr_params *params, const uint8_t *samples, int64_t n,
                         const psr_hamiltonian *hamiltonian, float *out, double *stats);

/* Exact samples of |psi|^2 of the LRU ansatz from uniforms [n][L] (float,
 * host or device): s_t = 1 iff u_t < P(s_t = 1 | s_<t), the forced value at
 * sites the zero-magnetisation mask fixes (Sec. II.A).  spins: uint8 [n][L]
 * out; logpsi: float [n] out (NULL to skip).  PSR_FP32: FP32 on CUDA cores.
 * PSR_FP16 / PSR_BF16 at hidden 64 with 1 to 3 layers: on the tensor cores,
 * the conditionals of the 16-bit model psr_lru_logpsi evaluates at that
 * precision (a draw can differ from the FP32 one only where u_t lies within
 * the 16-bit rounding of P).  The result does not depend on how samples are
 * grouped into CTAs.  Requirements as psr_lru_logpsi. */
int psr_lru_sample(const psr_params *params, const float *uniforms, int64_t n, int32_t L, uint8_t *spins,
                   float *logpsi);

/* Gradient of log psi of the LRU ansatz, as psr_grad for the chain model:
 * dout == NULL gives per-sample O_k rows [n][P] (P = psr_lru_param_count),
 * otherwise the dout-weighted sum [P].  Chunks of 32 sites are recomputed
 * from the forward's complex chunk carries and differentiated from the last
 * to the first; the complex recurrence's adjoint runs backwards as
 * mu_t = dL/dh_t + conj(lambda) mu_{t+1}.  FP32. */
int psr_lru_grad(const psr_params *params, const uint8_t *spins, int64_t n, int32_t L, const float *dout,
                 float *dparams);

/* ---------------------------------------------------------------------
 * c4v symmetrisation (the point-group symmetry the paper imposes on its 2D
 * runs, Sec. III.C, in the form of the RNN wave-function work it cites):
 *   psi_sym(s) = sqrt(1/8 sum_g psi(g s)^2)
 * over the 8 operations g of c4v on an L x L lattice (identity, rotations by
 * 90, 180, 270 degrees, reflections in x, in y and in both diagonals), image
 * g of a configuration being (g s)(g(x)) = s(x).  Model, parameters and
 * precision as psr_logpsi (chain minGRU along the zigzag path); every call
 * evaluates the 8 images (8 x the work).  PSR_EINVAL unless Lx == Ly. */
int psr_sym_logpsi(const psr_params *params, const uint8_t *spins, int64_t n, int32_t Lx, int32_t Ly,
                   float *out);

/* E_loc of psi_sym: E_loc(s) = diag(s) + sum_e c_e psi_sym(s'_e) / psi_sym(s).
 * The images of a connected configuration are connected configurations of
 * the sample's images (sites g(p), g(q) flipped), so each resumes from the
 * stored carries of its image sample.  Otherwise as psr_local_energy;
 * PSR_EINVAL unless Lx == Ly. */
int psr_sym_local_energy(const psr_params *params, const uint8_t *samples, int64_t n,
                         const psr_hamiltonian *hamiltonian, float *out, double *stats);

/* Adam state (Sec. III.B; Kingma and Ba): m = beta1 m + (1 - beta1) g,
 * v = beta2 v + (1 - beta2) g^2, theta -= lr m^ / (sqrt(v^) + eps) with the
 * bias corrections m^ = m / (1 - beta1^step), v^ = v / (1 - beta2^step).
 * m, v: device float [P], zero before the first step, updated in place. */
typedef struct {
    float lr, beta1, beta2, eps;
    int32_t step; /* 1-based count of this update */
    float *m, *v;
} psr_adam;

/* One VMC step on the device (Sec. III.B: exact sampling, local energy,
 * stochastic energy gradient, Adam):
 *   1. n exact samples s_i of |psi|^2 from uniforms [n][N] (psr_sample); with
 *      symmetrize = 1, sample i is replaced by its c4v image
 *      g_i = floor(8 sym_uniforms[i]), which makes it a sample of |psi_sym|^2;
 *   2. E_loc (psr_local_energy or psr_sym_local_energy) and its FP64 mean,
 *      variance and standard error;
 *   3. the energy gradient 2/n sum_i (E_loc(s_i) - mean) d log psi / d theta
 *      (for psi_sym: d log psi_sym = sum_g w_g d log psi(g s), w_g the
 *      images' normalised weights psi(g s)^2), by the FP32 reverse scan;
 *   4. theta_out = the Adam update of params->theta (theta_out may alias it).
 * Every array is a device array: uniforms, sym_uniforms (float [n], only with
 * symmetrize), theta_out [P], adam->m, adam->v; optional outputs (NULL to
 * skip): spins_out uint8 [n][N] (the samples used), eloc_out float [n],
 * stats_out double [3], grad_out float [P].  Asynchronous on the context's
 * stream.  PSR_EINVAL for host arrays, a non-square lattice with
 * symmetrize, step < 1 or out-of-range Adam constants. */
int psr_vmc_step(const psr_params *params, const psr_hamiltonian *hamiltonian, int32_t symmetrize,
                 const float *uniforms, const float *sym_uniforms, int64_t n, const psr_adam *adam,
                 float *theta_out, uint8_t *spins_out, float *eloc_out, double *stats_out,
                 float *grad_out);

/* One VMC step of the 2D patched minGRU on the device, as psr_vmc_step:
 * exact samples from uniforms [n][Np] (Np patches in path order,
 * psr2d_sample); with symmetrize = 1 each sample is replaced by its c4v
 * image floor(8 sym_uniforms[i]) and E_loc and the gradient are those of
 * psi_sym (psr2d_sym_local_energy; the gradient by psr2d_grad over the 8
 * images with the images' weights); otherwise E_loc by psr2d_local_energy
 * and the gradient by psr2d_grad; then Adam.  Same array rules as
 * psr_vmc_step; symmetrize needs a square lattice. */
int psr2d_vmc_step(const psr_params *params, const psr_hamiltonian *hamiltonian, int32_t symmetrize,
                   const float *uniforms, const float *sym_uniforms, int64_t n, const psr_adam *adam,
                   float *theta_out, uint8_t *spins_out, float *eloc_out, double *stats_out,
                   float *grad_out);

/* One VMC step of the LRU ansatz on the device, as psr_vmc_step without
 * symmetrisation: exact samples from uniforms [n][N] (psr_lru_sample),
 * E_loc (psr_lru_local_energy), the energy gradient by psr_lru_grad, Adam.
 * At PSR_FP16 / PSR_BF16 the samples and the local energies come from the
 * tensor cores (the sampler at up to 3 layers); the gradient is FP32.  Same
 * array rules as psr_vmc_step. */
int psr_lru_vmc_step(const psr_params *params, const psr_hamiltonian *hamiltonian, const float *uniforms,
                     int64_t n, const psr_adam *adam, float *theta_out, uint8_t *spins_out,
                     float *eloc_out, double *stats_out, float *grad_out);

/* Stages of the launch sequence, for per-stage device timing. */
enum {
    PSR_STAGE_PACK = 0,          /* parameter packing and spin bit-packing */
    PSR_STAGE_GENERATOR = 1,     /* bond list, count, scan, emit (connected set) */
    PSR_STAGE_FWD_SAMPLES = 2,   /* forward over the samples */
    PSR_STAGE_FWD_CONNECTED = 3, /* forward over the connected configurations */
    PSR_STAGE_GATHER = 4,        /* E_loc gather and FP64 statistics */
    PSR_STAGE_BWD = 5,           /* reverse-scan gradient and its reduction */
    PSR_STAGE_SCAN = 6,          /* psr_scan / psr_scan_tiled kernel */
    PSR_STAGE_SAMPLE = 7,        /* psr_sample kernel */
    PSR_STAGE_COUNT = 8
};

/* Enables (1) or disables (0) per-stage CUDA-event timing on the context's
 * stream.  When enabled every call records an event pair around each stage;
 * the cost is a few event records per call. */
int psr_context_set_profiling(psr_context *ctx, int enable);

/* Device time in milliseconds of one stage of the most recent call on this
 * context (0 if the stage did not run).  Synchronises on the stage's end
 * event.  PSR_EINVAL if profiling is off or the stage is out of range. */
int psr_context_stage_ms(psr_context *ctx, int stage, float *ms);

/* Static description of an error code. */
const char *psr_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* PSR_H */
