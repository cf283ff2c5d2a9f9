/*
 * psr_oracle2d.c -- plain FP64 CPU oracle for the paper's two-dimensional
 * patched minGRU (Sec. II.F "Two-dimensional Recurrences", Sec. II.G
 * residual connections).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * The model, written out as the paper defines it and evaluated strictly
 * sequentially along the zigzag path of the patch lattice, in double
 * precision:
 *   - the Lx x Ly spin lattice is cut into 2 x 2 patches; patch (i, j) holds
 *     the spins (2i + dx, 2j + dy), dx, dy in {0, 1}, and its value is
 *     v = sum s(2i+dx, 2j+dy) 2^(2 dy + dx) in 0..15; x0_{i,j} = onehot16(v);
 *   - patches are visited along the zigzag path (row j left to right when j
 *     is even), with causal predecessors H = (i - (-1)^j, j) and
 *     V = (i, j - 1); anything outside the lattice is zero;
 *   - layer input u0 = (x0_H, x0_V) (32 entries), u_l = x_l for l >= 1;
 *   - z = sigma(W_z u + b_z), h~ = W_h [u, h_V] + b_h,
 *     h = z * h_H + (1 - z) * h~, with h_H, h_V the same layer's states at
 *     the predecessors;
 *   - x_{l+1} = GELU(C h + D u + s_l), s_l = h_{l-1} (same patch) for l >= 2;
 *   - the conditional of patch t is softmax(W_o x_{nL} + b_o) over its 16
 *     values, log psi = 1/2 sum_t log P(v_t | v_<t).
 *
 * Readings of points the paper leaves open:
 *   - the bit order of a patch value (above) and the readout (a linear map
 *     to 16 logits and a softmax);
 *   - zero magnetisation (u1): a patch value is allowed while neither the
 *     up count nor the down count exceeds N/2 after it; the softmax is taken
 *     over the allowed values;
 *   - spins are given in the sequence order of the SPIN lattice (the same
 *     layout as the one-dimensional model), pos(i, j) = j Lx + (j even ? i :
 *     Lx - 1 - i), so the connected-configuration generator is shared.
 *
 * Parameter layout (flat theta), per layer l with din = 32 (l = 0) or H:
 *   W_z[H][din], b_z[H], W_h[H][din + H], b_h[H], C[H][H], D[H][din]
 * (the last H columns of W_h act on h_V), then W_o[16][H], b_o[16].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))

static double o2_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }
static double o2_gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }

static long o2_layer_size(int l, int H) {
    const long din = l == 0 ? 32 : H;
    return H * din + H + H * (din + H) + H + (long)H * H + H * din;
}

ORC_EXPORT long psro2d_param_count(int nL, int H) {
    long P = 0;
    for (int l = 0; l < nL; ++l) P += o2_layer_size(l, H);
    return P + 16L * H + 16;
}

typedef struct {
    const double *Wz, *bz, *Wh, *bh, *C, *D;
    int din;
} o2_layer;

static void o2_get_layer(const double *theta, int H, int l, o2_layer *L) {
    const double *p = theta;
    for (int k = 0; k < l; ++k) p += o2_layer_size(k, H);
    const int din = l == 0 ? 32 : H;
    L->din = din;
    L->Wz = p; p += (size_t)H * din;
    L->bz = p; p += H;
    L->Wh = p; p += (size_t)H * (din + H);
    L->bh = p; p += H;
    L->C = p; p += (size_t)H * H;
    L->D = p;
}

static int o2_pos(int Lx, int i, int j) { return j * Lx + ((j % 2 == 0) ? i : (Lx - 1 - i)); }

/* value of patch (pi, pj) of a spin configuration in sequence order */
static int o2_patch_value(const uint8_t *s, int Lx, int pi, int pj) {
    int v = 0;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx)
            if (s[o2_pos(Lx, 2 * pi + dx, 2 * pj + dy)]) v |= 1 << (2 * dy + dx);
    return v;
}

/* t-th patch of the zigzag path of a Px x Py patch lattice */
static void o2_patch_at(int Px, int t, int *pi, int *pj) {
    *pj = t / Px;
    const int k = t % Px;
    *pi = (*pj % 2 == 0) ? k : Px - 1 - k;
}

static int o2_popcount4(int v) { return (v & 1) + ((v >> 1) & 1) + ((v >> 2) & 1) + ((v >> 3) & 1); }

/* Forward state of one configuration: h[pj][pi][l][H] and the output x of
 * the last layer, written as patches are visited. */
typedef struct {
    int Px, Py, nL, H;
    double *h;      /* [Py][Px][nL][H] */
    double *u, *xin, *xout, *z, *ht;
} o2_state;

static int o2_alloc(o2_state *S, int Px, int Py, int nL, int H) {
    S->Px = Px; S->Py = Py; S->nL = nL; S->H = H;
    S->h = calloc((size_t)Px * Py * nL * H, sizeof(double));
    S->u = malloc(sizeof(double) * (size_t)(H > 32 ? H : 32));
    S->xin = malloc(sizeof(double) * (size_t)H);
    S->xout = malloc(sizeof(double) * (size_t)H);
    S->z = malloc(sizeof(double) * (size_t)H);
    S->ht = malloc(sizeof(double) * (size_t)H);
    return !(S->h && S->u && S->xin && S->xout && S->z && S->ht);
}

static void o2_free(o2_state *S) {
    free(S->h); free(S->u); free(S->xin); free(S->xout); free(S->z); free(S->ht);
}

static double *o2_h(o2_state *S, int pi, int pj, int l) {
    return S->h + (((size_t)pj * S->Px + pi) * S->nL + l) * S->H;
}

/* Runs every layer at patch (pi, pj) given the patch values vals[pj][pi]
 * of the configuration (only predecessors are read), and writes the 16
 * logits of its conditional. */
static void o2_patch(const double *theta, o2_state *S, const int *vals, int pi, int pj,
                     double *logits) {
    const int H = S->H, Px = S->Px;
    const int hi = pi - ((pj % 2 == 0) ? 1 : -1);  /* horizontal predecessor column */
    const int has_h = (hi >= 0 && hi < Px), has_v = (pj > 0);
    for (int l = 0; l < S->nL; ++l) {
        o2_layer L;
        o2_get_layer(theta, H, l, &L);
        double *u = S->u;
        if (l == 0) {
            for (int k = 0; k < 32; ++k) u[k] = 0.0;
            if (has_h) u[vals[pj * Px + hi]] = 1.0;
            if (has_v) u[16 + vals[(pj - 1) * Px + pi]] = 1.0;
        } else {
            for (int k = 0; k < H; ++k) u[k] = S->xin[k];
        }
        const double *hH = has_h ? o2_h(S, hi, pj, l) : NULL;
        const double *hV = has_v ? o2_h(S, pi, pj - 1, l) : NULL;
        double *h = o2_h(S, pi, pj, l);
        for (int j = 0; j < H; ++j) {
            double zp = L.bz[j], c = L.bh[j];
            for (int k = 0; k < L.din; ++k) {
                zp += L.Wz[(size_t)j * L.din + k] * u[k];
                c += L.Wh[(size_t)j * (L.din + H) + k] * u[k];
            }
            if (hV)
                for (int m = 0; m < H; ++m) c += L.Wh[(size_t)j * (L.din + H) + L.din + m] * hV[m];
            const double z = o2_sigmoid(zp);
            h[j] = z * (hH ? hH[j] : 0.0) + (1.0 - z) * c;
        }
        for (int j = 0; j < H; ++j) {
            double y = 0.0;
            for (int k = 0; k < H; ++k) y += L.C[(size_t)j * H + k] * h[k];
            for (int k = 0; k < L.din; ++k) y += L.D[(size_t)j * L.din + k] * u[k];
            if (l >= 2) y += o2_h(S, pi, pj, l - 1)[j];
            S->xout[j] = o2_gelu(y);
        }
        double *tmp = S->xin; S->xin = S->xout; S->xout = tmp;
    }
    const double *Wo = theta + psro2d_param_count(S->nL, H) - 16L * H - 16;
    for (int o = 0; o < 16; ++o) {
        double v = Wo[16L * H + o];
        for (int k = 0; k < H; ++k) v += Wo[(size_t)o * H + k] * S->xin[k];
        logits[o] = v;
    }
}

/* allowed[v] under the zero-magnetisation mask given the counts so far */
static void o2_mask(int u1, int N, int n_up, int n_down, int *allowed) {
    for (int v = 0; v < 16; ++v) {
        const int up = o2_popcount4(v);
        allowed[v] = !u1 || (n_up + up <= N / 2 && n_down + 4 - up <= N / 2);
    }
}

/* log P(v) over the allowed values (-inf if v is not allowed) */
static double o2_logp(const double *logits, const int *allowed, int v) {
    if (!allowed[v]) return -INFINITY;
    double m = -INFINITY;
    for (int o = 0; o < 16; ++o)
        if (allowed[o] && logits[o] > m) m = logits[o];
    double s = 0.0;
    for (int o = 0; o < 16; ++o)
        if (allowed[o]) s += exp(logits[o] - m);
    return logits[v] - m - log(s);
}

/* log psi of one configuration (spins in sequence order of the Lx x Ly
 * spin lattice, Lx and Ly even).  logP, if not NULL, receives the log
 * conditional of every patch in path order [Px * Py]. */
ORC_EXPORT double psro2d_logpsi(const double *theta, int nL, int H, int u1, int Lx, int Ly,
                                const uint8_t *s, double *logP) {
    const int Px = Lx / 2, Py = Ly / 2, N = Lx * Ly;
    o2_state S;
    int *vals = malloc(sizeof(int) * (size_t)Px * Py);
    if (!vals || o2_alloc(&S, Px, Py, nL, H)) {
        free(vals);
        return NAN;
    }
    for (int pj = 0; pj < Py; ++pj)
        for (int pi = 0; pi < Px; ++pi) vals[pj * Px + pi] = o2_patch_value(s, Lx, pi, pj);
    double acc = 0.0, logits[16];
    int n_up = 0, n_down = 0, allowed[16];
    for (int t = 0; t < Px * Py; ++t) {
        int pi, pj;
        o2_patch_at(Px, t, &pi, &pj);
        o2_patch(theta, &S, vals, pi, pj, logits);
        o2_mask(u1, N, n_up, n_down, allowed);
        const int v = vals[pj * Px + pi];
        const double lp = o2_logp(logits, allowed, v);
        if (logP) logP[t] = lp;
        acc += lp;
        n_up += o2_popcount4(v);
        n_down += 4 - o2_popcount4(v);
    }
    o2_free(&S);
    free(vals);
    return 0.5 * acc;
}

/* Exact samples: patch t takes the smallest value v whose cumulative
 * conditional probability exceeds uniforms[i][t] ([n][Px * Py]).  out
 * receives the spins in sequence order [n][N], logpsi the log amplitude. */
ORC_EXPORT void psro2d_sample(const double *theta, int nL, int H, int u1, int Lx, int Ly, long n,
                              const double *uniforms, uint8_t *out, double *logpsi) {
    const int Px = Lx / 2, Py = Ly / 2, N = Lx * Ly, Np = Px * Py;
    o2_state S;
    int *vals = malloc(sizeof(int) * (size_t)Np);
    if (!vals || o2_alloc(&S, Px, Py, nL, H)) {
        free(vals);
        return;
    }
    for (long i = 0; i < n; ++i) {
        memset(S.h, 0, sizeof(double) * (size_t)Np * nL * H);
        double acc = 0.0, logits[16];
        int n_up = 0, n_down = 0, allowed[16];
        for (int t = 0; t < Np; ++t) {
            int pi, pj;
            o2_patch_at(Px, t, &pi, &pj);
            o2_patch(theta, &S, vals, pi, pj, logits);
            o2_mask(u1, N, n_up, n_down, allowed);
            const double u = uniforms[(size_t)i * Np + t];
            double cum = 0.0;
            int v = -1, last = -1;
            for (int o = 0; o < 16; ++o) {
                if (!allowed[o]) continue;
                last = o;
                cum += exp(o2_logp(logits, allowed, o));
                if (u < cum) {
                    v = o;
                    break;
                }
            }
            if (v < 0) v = last;  /* u above the rounded total */
            vals[pj * Px + pi] = v;
            acc += o2_logp(logits, allowed, v);
            n_up += o2_popcount4(v);
            n_down += 4 - o2_popcount4(v);
            uint8_t *row = out + (size_t)i * N;
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx)
                    row[o2_pos(Lx, 2 * pi + dx, 2 * pj + dy)] = (uint8_t)((v >> (2 * dy + dx)) & 1);
        }
        if (logpsi) logpsi[i] = 0.5 * acc;
    }
    o2_free(&S);
    free(vals);
}

/* The 16-way conditional of every patch of one configuration, in path
 * order: probs[t][v] = P(v_t = v | v_<t) under the mask (0 for values the
 * mask excludes). */
ORC_EXPORT void psro2d_conditionals(const double *theta, int nL, int H, int u1, int Lx, int Ly,
                                    const uint8_t *s, double *probs) {
    const int Px = Lx / 2, Py = Ly / 2, N = Lx * Ly;
    o2_state S;
    int *vals = malloc(sizeof(int) * (size_t)Px * Py);
    if (!vals || o2_alloc(&S, Px, Py, nL, H)) {
        free(vals);
        return;
    }
    for (int pj = 0; pj < Py; ++pj)
        for (int pi = 0; pi < Px; ++pi) vals[pj * Px + pi] = o2_patch_value(s, Lx, pi, pj);
    double logits[16];
    int n_up = 0, n_down = 0, allowed[16];
    for (int t = 0; t < Px * Py; ++t) {
        int pi, pj;
        o2_patch_at(Px, t, &pi, &pj);
        o2_patch(theta, &S, vals, pi, pj, logits);
        o2_mask(u1, N, n_up, n_down, allowed);
        for (int v = 0; v < 16; ++v) probs[(size_t)t * 16 + v] = exp(o2_logp(logits, allowed, v));
        const int v = vals[pj * Px + pi];
        n_up += o2_popcount4(v);
        n_down += 4 - o2_popcount4(v);
    }
    o2_free(&S);
    free(vals);
}
