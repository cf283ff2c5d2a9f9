/*
 * psr_oracle.c -- plain FP64 CPU oracle for the PSR-NQS hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA library; the two are written
 * independently from the paper.
 *
 * Everything here is the plain definition, evaluated strictly sequentially in
 * double precision:
 *   - minGRU recurrence (Sec. II.C, Eq. minGRU):
 *       z_t = sigma(W_z x_{t-1} + b_z),  h~_t = W_h x_{t-1} + b_h,
 *       h_t = z_t * h_{t-1} + (1 - z_t) * h~_t
 *   - output map x~ = C h + D u and GELU block with residual s = h^{(l-1)} for
 *     l >= 2 (Sec. II.F output map; Sec. II.G 2D residual equations)
 *   - lattice ordering: zigzag (snake) path, predecessor (i-(-1)^j, j) and
 *     anything outside the lattice is zero (Sec. II.F)
 *   - autoregressive amplitude psi = prod_t sqrt(P(s_t | s_<t)), exact
 *     sampling (Sec. III.B, VMC paragraph)
 *   - Heisenberg H = sum S_i.S_j with S = sigma/2 and the Marshall sign
 *     (Sec. III.C); TFIM H = -sum zz - h sum x (Sec. III.B)
 *   - local energy over the connected off-diagonal configurations
 *     (Sec. II.A, last paragraph)
 *   - the parallel (Blelloch) scan of an affine diagonal recurrence
 *     (Sec. II.A, parallel scan paragraph), used only to pin the sequential
 *     form against the associative re-ordering.
 *
 * Parameter layout (flat theta, documented in include/psr.h as well, but not
 * shared with it): per layer l = 0..n_layers-1 with d_in = 2 (l = 0) or H:
 *   W_z[H][d_in], b_z[H], W_h[H][d_in], b_h[H], C[H][H], D[H][d_in]
 * then the readout W_o[2][H], b_o[2].
 *
 * Readings of points the paper leaves open:
 *   - layer-0 input at site t is onehot(s_{t-1}) (2-dim), zero at t = 0;
 *   - the readout is a linear map to 2 logits followed by a softmax;
 *   - GELU is the exact erf form;
 *   - u1 masking: once N/2 up (or down) spins have been placed, the
 *     conditional forces the other value (probability 1).
 *
 * Parity: every function here is pinned by tests/test_oracle_pins.py
 * (normalisation, closed forms, exact diagonalisation, finite differences,
 * brute-force bond enumeration, sampler chi^2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------ */
/* Parameter layout                                                    */
/* ------------------------------------------------------------------ */

typedef struct {
    const double *Wz, *bz, *Wh, *bh, *C, *D;
    int din;
} orc_layer;

static long orc_layer_size(int l, int H) {
    long din = (l == 0) ? 2 : H;
    return 3L * H * din + 2L * H + (long)H * H;
}

ORC_EXPORT long psro_param_count(int n_layers, int H) {
    long P = 0;
    for (int l = 0; l < n_layers; ++l) P += orc_layer_size(l, H);
    return P + 2L * H + 2;
}

static void orc_get_layer(const double *theta, int H, int l, orc_layer *L) {
    long off = 0;
    for (int k = 0; k < l; ++k) off += orc_layer_size(k, H);
    int din = (l == 0) ? 2 : H;
    const double *p = theta + off;
    L->din = din;
    L->Wz = p; p += (long)H * din;
    L->bz = p; p += H;
    L->Wh = p; p += (long)H * din;
    L->bh = p; p += H;
    L->C = p;  p += (long)H * H;
    L->D = p;
}

static const double *orc_readout(const double *theta, int n_layers, int H) {
    long off = 0;
    for (int k = 0; k < n_layers; ++k) off += orc_layer_size(k, H);
    return theta + off; /* W_o[2][H] then b_o[2] */
}

static double orc_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }
static double orc_gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
/* d/dx GELU(x) = Phi(x) + x phi(x) */
static double orc_gelu_grad(double x) {
    const double inv_sqrt_2pi = 0.39894228040143267794;
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * inv_sqrt_2pi * exp(-0.5 * x * x);
}

/* ------------------------------------------------------------------ */
/* Forward pass, strictly sequential over sites                        */
/* ------------------------------------------------------------------ */

/* Per-site record kept for the reverse pass and for traces.
 * Arrays are [N][n_layers][H] unless stated. */
typedef struct {
    int N, nL, H;
    double *u;     /* [N][nL][H]  layer input (layer 0 uses the first 2 entries) */
    double *a;     /* gate z_t */
    double *c;     /* candidate h~_t */
    double *h;     /* hidden state h_t */
    double *y;     /* pre-activation x~ + s */
    double *x;     /* [N][H] output of the last layer (readout input) */
    double *logit; /* [N][2] */
    int *mask;     /* [N]: 0 free, 1 forced to 0, 2 forced to 1 */
} orc_tape;

static size_t orc_idx(const orc_tape *T, int t, int l) {
    return ((size_t)t * T->nL + l) * T->H;
}

static int orc_tape_alloc(orc_tape *T, int N, int nL, int H) {
    size_t n3 = (size_t)N * nL * H;
    T->N = N; T->nL = nL; T->H = H;
    T->u = calloc(n3, sizeof(double));
    T->a = calloc(n3, sizeof(double));
    T->c = calloc(n3, sizeof(double));
    T->h = calloc(n3, sizeof(double));
    T->y = calloc(n3, sizeof(double));
    T->x = calloc((size_t)N * H, sizeof(double));
    T->logit = calloc((size_t)N * 2, sizeof(double));
    T->mask = calloc((size_t)N, sizeof(int));
    return (T->u && T->a && T->c && T->h && T->y && T->x && T->logit && T->mask) ? 0 : -1;
}

static void orc_tape_free(orc_tape *T) {
    free(T->u); free(T->a); free(T->c); free(T->h); free(T->y);
    free(T->x); free(T->logit); free(T->mask);
}

/* One site through every layer.  s_prev = -1 means "no predecessor" (t = 0). */
static void orc_site(const double *theta, int nL, int H, orc_tape *T, int t, int s_prev) {
    double *xin = malloc(sizeof(double) * (size_t)H);
    double *xout = malloc(sizeof(double) * (size_t)H);
    for (int l = 0; l < nL; ++l) {
        orc_layer L;
        orc_get_layer(theta, H, l, &L);
        double *u = T->u + orc_idx(T, t, l);
        if (l == 0) {
            u[0] = (s_prev == 0) ? 1.0 : 0.0;
            u[1] = (s_prev == 1) ? 1.0 : 0.0;
        } else {
            for (int k = 0; k < H; ++k) u[k] = xin[k];
        }
        double *a = T->a + orc_idx(T, t, l);
        double *c = T->c + orc_idx(T, t, l);
        double *h = T->h + orc_idx(T, t, l);
        double *y = T->y + orc_idx(T, t, l);
        const double *hprev = (t > 0) ? T->h + orc_idx(T, t - 1, l) : NULL;
        for (int j = 0; j < H; ++j) {
            double zp = L.bz[j], cj = L.bh[j];
            for (int k = 0; k < L.din; ++k) {
                zp += L.Wz[(size_t)j * L.din + k] * u[k];
                cj += L.Wh[(size_t)j * L.din + k] * u[k];
            }
            a[j] = orc_sigmoid(zp);
            c[j] = cj;
            double hp = hprev ? hprev[j] : 0.0;
            h[j] = a[j] * hp + (1.0 - a[j]) * cj;
        }
        for (int j = 0; j < H; ++j) {
            double v = 0.0;
            for (int k = 0; k < H; ++k) v += L.C[(size_t)j * H + k] * h[k];
            for (int k = 0; k < L.din; ++k) v += L.D[(size_t)j * L.din + k] * u[k];
            if (l >= 2) v += T->h[orc_idx(T, t, l - 1) + j];
            y[j] = v;
            xout[j] = orc_gelu(v);
        }
        double *tmp = xin; xin = xout; xout = tmp;
    }
    for (int k = 0; k < H; ++k) T->x[(size_t)t * H + k] = xin[k];
    const double *ro = orc_readout(theta, nL, H);
    for (int o = 0; o < 2; ++o) {
        double v = ro[2 * H + o];
        for (int k = 0; k < H; ++k) v += ro[(size_t)o * H + k] * xin[k];
        T->logit[t * 2 + o] = v;
    }
    free(xin);
    free(xout);
}

/* log P(s_t | s_<t) from the two logits, with the optional u1 mask. */
static double orc_logp(const double *logit, int mask, int s) {
    if (mask == 1) return (s == 0) ? 0.0 : -INFINITY;
    if (mask == 2) return (s == 1) ? 0.0 : -INFINITY;
    double m = logit[0] > logit[1] ? logit[0] : logit[1];
    double lse = m + log(exp(logit[0] - m) + exp(logit[1] - m));
    return logit[s] - lse;
}

static int orc_mask(int u1, int N, int t, int n_up) {
    if (!u1) return 0;
    if (n_up == N / 2) return 1;
    if (t - n_up == N / 2) return 2;
    return 0;
}

/* Full forward on a tape; returns log psi and fills per-site log P. */
static double orc_forward(const double *theta, int nL, int H, int u1,
                          const uint8_t *s, int N, orc_tape *T, double *logP) {
    double acc = 0.0;
    int n_up = 0;
    for (int t = 0; t < N; ++t) {
        orc_site(theta, nL, H, T, t, t == 0 ? -1 : (int)s[t - 1]);
        T->mask[t] = orc_mask(u1, N, t, n_up);
        double lp = orc_logp(T->logit + 2 * t, T->mask[t], (int)s[t]);
        if (logP) logP[t] = lp;
        acc += lp;
        n_up += s[t];
    }
    return 0.5 * acc;
}

/* log psi(s) of one configuration in sequence order; logP may be NULL. */
ORC_EXPORT double psro_logpsi(const double *theta, int n_layers, int H, int u1,
                              const uint8_t *s, int N, double *logP) {
    orc_tape T;
    if (orc_tape_alloc(&T, N, n_layers, H)) return NAN;
    double r = orc_forward(theta, n_layers, H, u1, s, N, &T, logP);
    orc_tape_free(&T);
    return r;
}

/* Batched log psi over n configurations [n][N]. */
ORC_EXPORT void psro_logpsi_batch(const double *theta, int n_layers, int H, int u1,
                                  const uint8_t *s, int N, long n, double *out) {
    for (long i = 0; i < n; ++i)
        out[i] = psro_logpsi(theta, n_layers, H, u1, s + (size_t)i * N, N, NULL);
}

/* Forward trace for tests: h[N][nL][H] and the per-layer outputs
 * xl[N][nL][H] (x^{(l+1)}), plus logits[N][2]. Any pointer may be NULL. */
ORC_EXPORT double psro_trace(const double *theta, int n_layers, int H, int u1,
                             const uint8_t *s, int N, double *h_out, double *x_out,
                             double *logit_out) {
    orc_tape T;
    if (orc_tape_alloc(&T, N, n_layers, H)) return NAN;
    double r = orc_forward(theta, n_layers, H, u1, s, N, &T, NULL);
    for (int t = 0; t < N; ++t)
        for (int l = 0; l < n_layers; ++l)
            for (int j = 0; j < H; ++j) {
                size_t i = orc_idx(&T, t, l) + j;
                if (h_out) h_out[i] = T.h[i];
                if (x_out) x_out[i] = orc_gelu(T.y[i]);
            }
    if (logit_out) memcpy(logit_out, T.logit, sizeof(double) * 2 * (size_t)N);
    orc_tape_free(&T);
    return r;
}

/* ------------------------------------------------------------------ */
/* Reverse mode: d log psi / d theta, hand-written over the same loop  */
/* ------------------------------------------------------------------ */

ORC_EXPORT double psro_grad(const double *theta, int n_layers, int H, int u1,
                            const uint8_t *s, int N, double *grad) {
    const int nL = n_layers;
    long P = psro_param_count(nL, H);
    memset(grad, 0, sizeof(double) * (size_t)P);
    orc_tape T;
    if (orc_tape_alloc(&T, N, nL, H)) return NAN;
    double lpsi = orc_forward(theta, nL, H, u1, s, N, &T, NULL);

    /* gradient slots, same layout as theta */
    long off_layer[64];
    long off = 0;
    for (int l = 0; l < nL; ++l) { off_layer[l] = off; off += orc_layer_size(l, H); }
    double *gWo = grad + off;
    double *gbo = gWo + 2 * H;
    const double *ro = orc_readout(theta, nL, H);

    /* gx[t][l][H]: gradient w.r.t. the OUTPUT of layer l at site t (x^{(l+1)}) */
    size_t n3 = (size_t)N * nL * H;
    double *gx = calloc(n3, sizeof(double));
    double *gh_direct = calloc(n3, sizeof(double)); /* dL/dh_t from the outputs */
    double *gy = calloc(n3, sizeof(double));
    double *lam = malloc(sizeof(double) * (size_t)H);

    /* readout: log psi = 1/2 sum_t log P_t */
    for (int t = 0; t < N; ++t) {
        if (T.mask[t]) continue; /* forced sites carry no parameter dependence */
        const double *lg = T.logit + 2 * t;
        double m = lg[0] > lg[1] ? lg[0] : lg[1];
        double e0 = exp(lg[0] - m), e1 = exp(lg[1] - m);
        double p[2] = {e0 / (e0 + e1), e1 / (e0 + e1)};
        for (int o = 0; o < 2; ++o) {
            double g = 0.5 * (((int)s[t] == o ? 1.0 : 0.0) - p[o]);
            gbo[o] += g;
            for (int k = 0; k < H; ++k) {
                gWo[(size_t)o * H + k] += g * T.x[(size_t)t * H + k];
                gx[orc_idx(&T, t, nL - 1) + k] += g * ro[(size_t)o * H + k];
            }
        }
    }

    /* layers top to bottom */
    for (int l = nL - 1; l >= 0; --l) {
        orc_layer L;
        orc_get_layer(theta, H, l, &L);
        double *g = grad + off_layer[l];
        double *gWz = g;
        double *gbz = gWz + (size_t)H * L.din;
        double *gWh = gbz + H;
        double *gbh = gWh + (size_t)H * L.din;
        double *gC = gbh + H;
        double *gD = gC + (size_t)H * H;
        /* output block: x^{(l+1)} = GELU(C h + D u + [l>=2] h^{(l-1)}) */
        for (int t = 0; t < N; ++t) {
            size_t b = orc_idx(&T, t, l);
            for (int j = 0; j < H; ++j) gy[b + j] = gx[b + j] * orc_gelu_grad(T.y[b + j]);
            for (int j = 0; j < H; ++j) {
                double gyj = gy[b + j];
                for (int k = 0; k < H; ++k) {
                    gC[(size_t)j * H + k] += gyj * T.h[b + k];
                    gh_direct[b + k] += L.C[(size_t)j * H + k] * gyj;
                }
                for (int k = 0; k < L.din; ++k) gD[(size_t)j * L.din + k] += gyj * T.u[b + k];
            }
            if (l >= 2) {
                size_t bm = orc_idx(&T, t, l - 1);
                for (int j = 0; j < H; ++j) gh_direct[bm + j] += gy[b + j];
            }
        }
        /* reverse scan over sites: lam_t = dL/dh_t = direct + a_{t+1} lam_{t+1} */
        for (int j = 0; j < H; ++j) lam[j] = 0.0;
        for (int t = N - 1; t >= 0; --t) {
            size_t b = orc_idx(&T, t, l);
            for (int j = 0; j < H; ++j) {
                double next = 0.0;
                if (t + 1 < N) next = T.a[orc_idx(&T, t + 1, l) + j] * lam[j];
                lam[j] = gh_direct[b + j] + next;
            }
            for (int j = 0; j < H; ++j) {
                double hprev = (t > 0) ? T.h[orc_idx(&T, t - 1, l) + j] : 0.0;
                double aj = T.a[b + j];
                double ga = lam[j] * (hprev - T.c[b + j]);
                double gc = lam[j] * (1.0 - aj);
                double gz = ga * aj * (1.0 - aj);
                gbz[j] += gz;
                gbh[j] += gc;
                for (int k = 0; k < L.din; ++k) {
                    gWz[(size_t)j * L.din + k] += gz * T.u[b + k];
                    gWh[(size_t)j * L.din + k] += gc * T.u[b + k];
                }
                if (l >= 1) {
                    /* input of layer l is the output of layer l-1 */
                    size_t bo = orc_idx(&T, t, l - 1);
                    for (int k = 0; k < H; ++k)
                        gx[bo + k] += L.Wz[(size_t)j * H + k] * gz + L.Wh[(size_t)j * H + k] * gc;
                }
            }
        }
        /* D u term feeds the input gradient of layer l as well */
        if (l >= 1) {
            for (int t = 0; t < N; ++t) {
                size_t b = orc_idx(&T, t, l);
                size_t bo = orc_idx(&T, t, l - 1);
                for (int j = 0; j < H; ++j)
                    for (int k = 0; k < H; ++k) gx[bo + k] += L.D[(size_t)j * H + k] * gy[b + j];
            }
        }
    }
    free(gx); free(gh_direct); free(gy); free(lam);
    orc_tape_free(&T);
    return lpsi;
}

/* ------------------------------------------------------------------ */
/* Exact autoregressive sampling                                       */
/* ------------------------------------------------------------------ */

/* Draws n configurations of N sites.  uniforms[n][N] in [0,1) are inputs:
 * s_t = 1 iff u_t < P(s_t = 1 | s_<t).  Also returns log psi per sample. */
ORC_EXPORT void psro_sample(const double *theta, int n_layers, int H, int u1, int N, long n,
                            const double *uniforms, uint8_t *out, double *logpsi) {
    orc_tape T;
    if (orc_tape_alloc(&T, N, n_layers, H)) return;
    for (long i = 0; i < n; ++i) {
        uint8_t *s = out + (size_t)i * N;
        int n_up = 0;
        double acc = 0.0;
        for (int t = 0; t < N; ++t) {
            orc_site(theta, n_layers, H, &T, t, t == 0 ? -1 : (int)s[t - 1]);
            int mask = orc_mask(u1, N, t, n_up);
            double p1 = exp(orc_logp(T.logit + 2 * t, mask, 1));
            s[t] = (uniforms[(size_t)i * N + t] < p1) ? 1 : 0;
            acc += orc_logp(T.logit + 2 * t, mask, s[t]);
            n_up += s[t];
        }
        if (logpsi) logpsi[i] = 0.5 * acc;
    }
    orc_tape_free(&T);
}

/* ------------------------------------------------------------------ */
/* Lattice, bonds, connected configurations, local energy              */
/* ------------------------------------------------------------------ */

/* zigzag path: row j (0-based) runs left to right when j is even */
ORC_EXPORT int psro_seq_pos(int Lx, int i, int j) {
    return j * Lx + ((j % 2 == 0) ? i : (Lx - 1 - i));
}

/* Nearest-neighbour bonds in canonical order: sites in row-major order
 * (j major, i minor), right bond then down bond; each stored as
 * (min pos, max pos).  Periodic wrap only when the dimension is >= 3
 * (and only in y when Ly > 1).  Returns the bond count. */
ORC_EXPORT int psro_bonds(int Lx, int Ly, int pbc, int32_t *pq) {
    int nb = 0;
    for (int j = 0; j < Ly; ++j) {
        for (int i = 0; i < Lx; ++i) {
            int here = psro_seq_pos(Lx, i, j);
            int nbr[2] = {-1, -1};
            if (i + 1 < Lx) nbr[0] = psro_seq_pos(Lx, i + 1, j);
            else if (pbc && Lx >= 3) nbr[0] = psro_seq_pos(Lx, 0, j);
            if (j + 1 < Ly) nbr[1] = psro_seq_pos(Lx, i, j + 1);
            else if (pbc && Ly >= 3) nbr[1] = psro_seq_pos(Lx, i, 0);
            for (int d = 0; d < 2; ++d) {
                if (nbr[d] < 0) continue;
                int p = here < nbr[d] ? here : nbr[d];
                int q = here < nbr[d] ? nbr[d] : here;
                if (pq) { pq[2 * nb] = p; pq[2 * nb + 1] = q; }
                ++nb;
            }
        }
    }
    return nb;
}

/* kind: 0 = Heisenberg, 1 = TFIM.
 * Counts the connected entries of each sample (counts[n]) and the diagonal
 * energy (diag[n]).  Heisenberg: diag = (J/4) sum_b sigma_p sigma_q, one entry
 * per antiparallel bond.  TFIM: diag = -J sum_b sigma_p sigma_q, N entries. */
ORC_EXPORT void psro_count_connected(int kind, double J, const int32_t *pq, int nb,
                                     const uint8_t *s, int N, long n, int64_t *counts,
                                     double *diag) {
    for (long i = 0; i < n; ++i) {
        const uint8_t *x = s + (size_t)i * N;
        double zz = 0.0;
        int64_t cnt = 0;
        for (int b = 0; b < nb; ++b) {
            int sp = 2 * x[pq[2 * b]] - 1, sq = 2 * x[pq[2 * b + 1]] - 1;
            zz += (double)(sp * sq);
            if (kind == 0 && sp != sq) ++cnt;
        }
        if (kind == 0) { diag[i] = 0.25 * J * zz; counts[i] = cnt; }
        else { diag[i] = -J * zz; counts[i] = N; }
    }
}

/* Writes the entries (sample, p, q) sample-major, then bond order (or site
 * order for TFIM, q = -1).  entries must hold 3 * sum(counts) int32. */
ORC_EXPORT void psro_fill_connected(int kind, const int32_t *pq, int nb, const uint8_t *s,
                                    int N, long n, int32_t *entries) {
    long e = 0;
    for (long i = 0; i < n; ++i) {
        const uint8_t *x = s + (size_t)i * N;
        if (kind == 0) {
            for (int b = 0; b < nb; ++b) {
                int p = pq[2 * b], q = pq[2 * b + 1];
                if (x[p] != x[q]) {
                    entries[3 * e] = (int32_t)i; entries[3 * e + 1] = p; entries[3 * e + 2] = q; ++e;
                }
            }
        } else {
            for (int p = 0; p < N; ++p) {
                entries[3 * e] = (int32_t)i; entries[3 * e + 1] = p; entries[3 * e + 2] = -1; ++e;
            }
        }
    }
}

/* Off-diagonal matrix element c_e of one entry.  Heisenberg: S+S- + S-S+
 * gives J/2 per antiparallel bond, times -1 under the Marshall sign.
 * TFIM: -h per site flip. */
ORC_EXPORT double psro_offdiag_coeff(int kind, double J, double h, int marshall) {
    if (kind == 0) return marshall ? -0.5 * J : 0.5 * J;
    return -h;
}

/* E_loc(s) = diag(s) + sum_e c * psi(s'_e)/psi(s), given log psi values. */
ORC_EXPORT double psro_eloc_combine(double diag, double coeff, double logpsi_s,
                                    const double *logpsi_sp, long m) {
    double acc = diag;
    for (long e = 0; e < m; ++e) acc += coeff * exp(logpsi_sp[e] - logpsi_s);
    return acc;
}

/* Local energy of n samples with the network amplitude: every connected
 * configuration is evaluated by a full sequential forward (no reuse). */
ORC_EXPORT void psro_local_energy(const double *theta, int n_layers, int H, int u1, int kind,
                                  int Lx, int Ly, int pbc, int marshall, double J, double hfield,
                                  const uint8_t *s, int N, long n, double *eloc) {
    int maxb = 2 * Lx * Ly + 2;
    int32_t *pq = malloc(sizeof(int32_t) * 2 * (size_t)maxb);
    int nb = psro_bonds(Lx, Ly, pbc, pq);
    uint8_t *sp = malloc((size_t)N);
    double *lps = malloc(sizeof(double) * ((size_t)nb + N + 1));
    int32_t *ent = malloc(sizeof(int32_t) * 3 * ((size_t)nb + N + 1));
    double coeff = psro_offdiag_coeff(kind, J, hfield, marshall);
    for (long i = 0; i < n; ++i) {
        const uint8_t *x = s + (size_t)i * N;
        int64_t cnt; double diag;
        psro_count_connected(kind, J, pq, nb, x, N, 1, &cnt, &diag);
        psro_fill_connected(kind, pq, nb, x, N, 1, ent);
        double l0 = psro_logpsi(theta, n_layers, H, u1, x, N, NULL);
        for (int64_t e = 0; e < cnt; ++e) {
            memcpy(sp, x, (size_t)N);
            int p = ent[3 * e + 1], q = ent[3 * e + 2];
            sp[p] ^= 1;
            if (q >= 0) sp[q] ^= 1;
            lps[e] = psro_logpsi(theta, n_layers, H, u1, sp, N, NULL);
        }
        eloc[i] = psro_eloc_combine(diag, coeff, l0, lps, cnt);
    }
    free(pq); free(sp); free(lps); free(ent);
}

/* Mean, unbiased variance and standard error sqrt(var/n). */
ORC_EXPORT void psro_stats(const double *e, long n, double *out3) {
    double m = 0.0;
    for (long i = 0; i < n; ++i) m += e[i];
    m /= (double)n;
    double v = 0.0;
    for (long i = 0; i < n; ++i) v += (e[i] - m) * (e[i] - m);
    v = (n > 1) ? v / (double)(n - 1) : 0.0;
    out3[0] = m; out3[1] = v; out3[2] = sqrt(v / (double)n);
}

/* ------------------------------------------------------------------ */
/* Scan forms of h_t = a_t h_{t-1} + b_t (h_{-1} = h0)                  */
/* ------------------------------------------------------------------ */

ORC_EXPORT void psro_scan_sequential(const double *a, const double *b, int N, double h0,
                                     double *h) {
    double cur = h0;
    for (int t = 0; t < N; ++t) { cur = a[t] * cur + b[t]; h[t] = cur; }
}

/* Work-efficient (Blelloch) exclusive scan over the affine maps
 * f_t(x) = a_t x + b_t with composition (f after g) = (a_f a_g, a_f b_g + b_f);
 * the identity is (1, 0).  h_t = (F_t)(h0) where F_t = f_t o ... o f_0. */
ORC_EXPORT void psro_scan_blelloch(const double *a, const double *b, int N, double h0,
                                   double *h) {
    int M = 1;
    while (M < N) M <<= 1;
    double *A = malloc(sizeof(double) * (size_t)M);
    double *B = malloc(sizeof(double) * (size_t)M);
    for (int i = 0; i < M; ++i) {
        A[i] = (i < N) ? a[i] : 1.0;
        B[i] = (i < N) ? b[i] : 0.0;
    }
    /* up-sweep: node r = r o l (the right element applied after the left) */
    for (int d = 1; d < M; d <<= 1) {
        for (int i = 2 * d - 1; i < M; i += 2 * d) {
            int l = i - d;
            double na = A[i] * A[l];
            double nb = A[i] * B[l] + B[i];
            A[i] = na; B[i] = nb;
        }
    }
    /* down-sweep to an exclusive prefix */
    A[M - 1] = 1.0; B[M - 1] = 0.0;
    for (int d = M >> 1; d >= 1; d >>= 1) {
        for (int i = 2 * d - 1; i < M; i += 2 * d) {
            int l = i - d;
            double ta = A[l], tb = B[l];
            /* left child receives the parent's prefix */
            A[l] = A[i]; B[l] = B[i];
            /* right child: its left sibling's subtree applied after the prefix */
            double na = ta * A[i];
            double nb = ta * B[i] + tb;
            A[i] = na; B[i] = nb;
        }
    }
    /* inclusive result: apply f_t after the exclusive prefix */
    for (int t = 0; t < N; ++t) {
        double pa = A[t], pb = B[t];
        double ia = a[t] * pa, ib = a[t] * pb + b[t];
        h[t] = ia * h0 + ib;
    }
    free(A); free(B);
}
