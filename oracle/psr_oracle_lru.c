/*
 * psr_oracle_lru.c -- plain FP64 CPU oracle for the paper's deep 1D LRU
 * ansatz (Sec. II.B "Linear Recurrent Unit", Eq. lru; Sec. II.G 1D residual;
 * Sec. III.B: three layers, each an LRU followed by a single-layer GLU
 * feed-forward network acting on each site).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Written out as the paper defines it and evaluated strictly sequentially in
 * double precision (complex arithmetic spelled out as real and imaginary
 * parts), for layers l = 0 .. nL-1 with input u_t (u_t = onehot(s_{t-1}) at
 * l = 0, zero at t = 0; u_t = x_t^(l) for l >= 1):
 *   lambda = exp(-exp(nu) + i exp(theta))            (per hidden unit)
 *   h_t = lambda * h_{t-1} + exp(gamma) * (B u_t),   h_{-1} = 0,  B complex
 *   y_t = Re(C h_t) + D u_t,                          C complex
 *   x_t^(l+1) = GLU(y_t) + [l >= 1] x_t^(l),
 *   GLU(y) = (W_a y + b_a) * sigmoid(W_g y + b_g)
 * then softmax(W_o x^(nL) + b_o) over s_t and log psi = 1/2 sum log P.
 *
 * Readings of points the paper leaves open:
 *   - D is elementwise (D in R^d) for l >= 1 as written; at l = 0 the input
 *     is the 2-entry one-hot, so D^(0) is a d x 2 matrix;
 *   - the single-layer GLU is (W_a y + b_a) * sigmoid(W_g y + b_g);
 *   - the input shift x_{t-1} of Eq. lru happens once, at the one-hot input;
 *   - the readout is the two-logit softmax of the minGRU model, and the u1
 *     mask (if asked for) is the same as there.
 *
 * Parameter layout (flat theta), d = d_h = H, din = 2 (l = 0) or H:
 *   nu[H], theta[H], gamma[H], B_re[H][din], B_im[H][din],
 *   C_re[H][H], C_im[H][H], D (l = 0: [H][2]; l >= 1: [H]),
 *   W_a[H][H], b_a[H], W_g[H][H], b_g[H]
 * then W_o[2][H], b_o[2].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))

static double ol_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

static long ol_layer_size(int l, int H) {
    const long din = l == 0 ? 2 : H;
    const long dsize = l == 0 ? 2L * H : H;
    return 3L * H + 2L * H * din + 2L * H * H + dsize + 2L * H * H + 2L * H;
}

ORC_EXPORT long psro_lru_param_count(int nL, int H) {
    long P = 0;
    for (int l = 0; l < nL; ++l) P += ol_layer_size(l, H);
    return P + 2L * H + 2;
}

typedef struct {
    const double *nu, *th, *ga, *Bre, *Bim, *Cre, *Cim, *D, *Wa, *ba, *Wg, *bg;
    int din;
} ol_layer;

static void ol_get_layer(const double *theta, int H, int l, ol_layer *L) {
    const double *p = theta;
    for (int k = 0; k < l; ++k) p += ol_layer_size(k, H);
    const int din = l == 0 ? 2 : H;
    L->din = din;
    L->nu = p; p += H;
    L->th = p; p += H;
    L->ga = p; p += H;
    L->Bre = p; p += (size_t)H * din;
    L->Bim = p; p += (size_t)H * din;
    L->Cre = p; p += (size_t)H * H;
    L->Cim = p; p += (size_t)H * H;
    L->D = p; p += (l == 0) ? 2 * (size_t)H : (size_t)H;
    L->Wa = p; p += (size_t)H * H;
    L->ba = p; p += H;
    L->Wg = p; p += (size_t)H * H;
    L->bg = p;
}

static int ol_mask(int u1, int N, int t, int n_up) {
    if (!u1) return 0;
    if (n_up == N / 2) return 1;
    if (t - n_up == N / 2) return 2;
    return 0;
}

static double ol_logp(const double *logit, int mask, int s) {
    if (mask == 1) return (s == 0) ? 0.0 : -INFINITY;
    if (mask == 2) return (s == 1) ? 0.0 : -INFINITY;
    double m = logit[0] > logit[1] ? logit[0] : logit[1];
    return logit[s] - (m + log(exp(logit[0] - m) + exp(logit[1] - m)));
}

/* State of one configuration: complex hidden states per layer (the previous
 * site's), and work vectors. */
typedef struct {
    int nL, H;
    double *hre, *him;       /* [nL][H] */
    double *u, *x, *y, *xn;  /* [H] each (u holds 2 entries at l = 0) */
} ol_state;

static int ol_alloc(ol_state *S, int nL, int H) {
    S->nL = nL;
    S->H = H;
    S->hre = calloc((size_t)nL * H, sizeof(double));
    S->him = calloc((size_t)nL * H, sizeof(double));
    S->u = malloc(sizeof(double) * (size_t)(H > 2 ? H : 2));
    S->x = malloc(sizeof(double) * (size_t)H);
    S->y = malloc(sizeof(double) * (size_t)H);
    S->xn = malloc(sizeof(double) * (size_t)H);
    return !(S->hre && S->him && S->u && S->x && S->y && S->xn);
}

static void ol_free(ol_state *S) {
    free(S->hre); free(S->him); free(S->u); free(S->x); free(S->y); free(S->xn);
}

/* Runs all layers at site t (s_prev = s_{t-1}, -1 at t = 0) and writes the
 * two logits. */
static void ol_site(const double *theta, ol_state *S, int s_prev, double *logit) {
    const int H = S->H;
    for (int l = 0; l < S->nL; ++l) {
        ol_layer L;
        ol_get_layer(theta, H, l, &L);
        double *u = S->u;
        if (l == 0) {
            u[0] = (s_prev == 0) ? 1.0 : 0.0;
            u[1] = (s_prev == 1) ? 1.0 : 0.0;
        } else {
            for (int k = 0; k < H; ++k) u[k] = S->x[k];
        }
        double *hre = S->hre + (size_t)l * H, *him = S->him + (size_t)l * H;
        for (int j = 0; j < H; ++j) {
            const double r = exp(-exp(L.nu[j])), ph = exp(L.th[j]);
            const double lre = r * cos(ph), lim = r * sin(ph);
            double bre = 0.0, bim = 0.0;
            for (int k = 0; k < L.din; ++k) {
                bre += L.Bre[(size_t)j * L.din + k] * u[k];
                bim += L.Bim[(size_t)j * L.din + k] * u[k];
            }
            const double g = exp(L.ga[j]);
            const double nre = lre * hre[j] - lim * him[j] + g * bre;
            const double nim = lre * him[j] + lim * hre[j] + g * bim;
            hre[j] = nre;
            him[j] = nim;
        }
        for (int i = 0; i < H; ++i) {
            double v = 0.0;
            for (int j = 0; j < H; ++j)
                v += L.Cre[(size_t)i * H + j] * hre[j] - L.Cim[(size_t)i * H + j] * him[j];
            if (l == 0) v += L.D[(size_t)i * 2 + 0] * u[0] + L.D[(size_t)i * 2 + 1] * u[1];
            else v += L.D[i] * u[i];
            S->y[i] = v;
        }
        for (int i = 0; i < H; ++i) {
            double a = L.ba[i], gt = L.bg[i];
            for (int k = 0; k < H; ++k) {
                a += L.Wa[(size_t)i * H + k] * S->y[k];
                gt += L.Wg[(size_t)i * H + k] * S->y[k];
            }
            S->xn[i] = a * ol_sigmoid(gt) + ((l >= 1) ? u[i] : 0.0);
        }
        for (int i = 0; i < H; ++i) S->x[i] = S->xn[i];
    }
    const double *ro = theta + psro_lru_param_count(S->nL, H) - 2L * H - 2;
    for (int o = 0; o < 2; ++o) {
        double v = ro[2L * H + o];
        for (int k = 0; k < H; ++k) v += ro[(size_t)o * H + k] * S->x[k];
        logit[o] = v;
    }
}

/* log psi of one configuration (sequence order); logP may be NULL. */
ORC_EXPORT double psro_lru_logpsi(const double *theta, int nL, int H, int u1, const uint8_t *s, int N,
                                  double *logP) {
    ol_state S;
    if (ol_alloc(&S, nL, H)) return NAN;
    double acc = 0.0, logit[2];
    int n_up = 0;
    for (int t = 0; t < N; ++t) {
        ol_site(theta, &S, t == 0 ? -1 : (int)s[t - 1], logit);
        const double lp = ol_logp(logit, ol_mask(u1, N, t, n_up), (int)s[t]);
        if (logP) logP[t] = lp;
        acc += lp;
        n_up += s[t];
    }
    ol_free(&S);
    return 0.5 * acc;
}

/* Exact samples from uniforms [n][N]: s_t = 1 iff u < P(s_t = 1 | s_<t). */
ORC_EXPORT void psro_lru_sample(const double *theta, int nL, int H, int u1, int N, long n,
                                const double *uniforms, uint8_t *out, double *logpsi) {
    ol_state S;
    if (ol_alloc(&S, nL, H)) return;
    for (long i = 0; i < n; ++i) {
        memset(S.hre, 0, sizeof(double) * (size_t)nL * H);
        memset(S.him, 0, sizeof(double) * (size_t)nL * H);
        uint8_t *s = out + (size_t)i * N;
        double acc = 0.0, logit[2];
        int n_up = 0;
        for (int t = 0; t < N; ++t) {
            ol_site(theta, &S, t == 0 ? -1 : (int)s[t - 1], logit);
            const int mask = ol_mask(u1, N, t, n_up);
            const double p1 = exp(ol_logp(logit, mask, 1));
            s[t] = (uniforms[(size_t)i * N + t] < p1) ? 1 : 0;
            acc += ol_logp(logit, mask, s[t]);
            n_up += s[t];
        }
        if (logpsi) logpsi[i] = 0.5 * acc;
    }
    ol_free(&S);
}
