/*
 * Candidate-classifier oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain CPU statement of the small convolutional classifier that scores
 * 64x64 DM-time snippets around search candidates as astrophysical or not.
 * The paper (Section 2.1) motivates separating true signals from radio
 * frequency interference; the learned classifier itself is not in the paper.
 * Only the test-suite may load this library; it shares nothing with the CUDA
 * path.
 *
 * Network (parameters in one flat float vector, in this order):
 *   conv1 w[16][1][3][3] b[16]   conv2 w[32][16][3][3] b[32]
 *   conv3 w[64][32][3][3] b[64]  conv4 w[64][64][3][3] b[64]
 *   fc1 w[128][1024] b[128]      fc2 w[1][128] b[1]            (191553 values)
 * Each conv: 3x3, zero padding 1, stride 1, then ReLU, then 2x2 max pooling.
 * conv4's pooled output [64][4][4] is flattened as c*16 + y*4 + x into fc1;
 * fc1 is followed by ReLU; fc2 gives the logit.
 *
 * Precision (round = 1): weights, biases and the input are bfloat16 values
 * (weights rounded from the float master copy, nearest-even); every sum is
 * accumulated in float starting from the bias, over (input channel, ky, kx)
 * for convs and over inputs for the dense layers, in increasing index order,
 * with padded taps skipped; a product of two bfloat16 values is exact in
 * float so each step rounds once.  Conv and fc1 outputs are rounded to
 * bfloat16 after the ReLU; pooling takes the first maximum in (0,0), (0,1),
 * (1,0), (1,1) order; the logit stays float.  With round = 0 nothing is
 * rounded (used for finite-difference checks of the backward pass).
 *
 * Loss: mean over the batch of binary cross-entropy with logits,
 *   max(z,0) - z*y + log(1 + exp(-|z|)).
 * Backward: float gradients of that loss w.r.t. the (rounded) parameters,
 * treating each bfloat16 rounding as the identity; max-pool routes the
 * gradient to its first maximum, ReLU passes it where the output is > 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NCONV 4
static const int CIN[NCONV] = {1, 16, 32, 64};
static const int COUT[NCONV] = {16, 32, 64, 64};
static const int HIN[NCONV] = {64, 32, 16, 8};
#define FC1_IN 1024
#define FC1_OUT 128

static float bf16_round(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return f;
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

static float bf16_to_float(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

/* offsets of each tensor in the flat parameter vector */
typedef struct {
    long cw[NCONV], cb[NCONV], f1w, f1b, f2w, f2b, total;
} layout;

static layout make_layout(void)
{
    layout L;
    long o = 0;
    for (int l = 0; l < NCONV; ++l) {
        L.cw[l] = o;
        o += (long)COUT[l] * CIN[l] * 9;
        L.cb[l] = o;
        o += COUT[l];
    }
    L.f1w = o;
    o += (long)FC1_OUT * FC1_IN;
    L.f1b = o;
    o += FC1_OUT;
    L.f2w = o;
    o += FC1_OUT;
    L.f2b = o;
    o += 1;
    L.total = o;
    return L;
}

long oracle_nn_param_count(void) { return make_layout().total; }

/* activations kept for the backward pass */
typedef struct {
    float *in[NCONV];     /* layer inputs [N][Cin][H][H] */
    float *pooled[NCONV]; /* [N][Cout][H/2][H/2] */
    int *arg[NCONV];      /* argmax quad position 0..3 */
    float *h1;            /* fc1 output after ReLU (rounded) [N][128] */
    float *z;             /* logits [N] */
    float *w;             /* parameters as used (rounded when round) */
} acts;

static void free_acts(acts *a)
{
    for (int l = 0; l < NCONV; ++l) {
        free(a->in[l]);
        free(a->pooled[l]);
        free(a->arg[l]);
    }
    free(a->h1);
    free(a->z);
    free(a->w);
}

static int forward(const float *params, int N, const uint16_t *x, int round, acts *a)
{
    layout L = make_layout();
    memset(a, 0, sizeof(*a));
    a->w = (float *)malloc(sizeof(float) * L.total);
    if (!a->w) return -2;
    for (long i = 0; i < L.total; ++i) a->w[i] = round ? bf16_round(params[i]) : params[i];
    const float *w = a->w;
    for (int l = 0; l < NCONV; ++l) {
        long H = HIN[l];
        a->in[l] = (float *)malloc(sizeof(float) * N * CIN[l] * H * H);
        a->pooled[l] = (float *)malloc(sizeof(float) * N * COUT[l] * (H / 2) * (H / 2));
        a->arg[l] = (int *)malloc(sizeof(int) * N * COUT[l] * (H / 2) * (H / 2));
        if (!a->in[l] || !a->pooled[l] || !a->arg[l]) return -2;
    }
    a->h1 = (float *)malloc(sizeof(float) * N * FC1_OUT);
    a->z = (float *)malloc(sizeof(float) * N);
    if (!a->h1 || !a->z) return -2;
    for (long i = 0; i < (long)N * 64 * 64; ++i) a->in[0][i] = bf16_to_float(x[i]);

    for (int l = 0; l < NCONV; ++l) {
        const int Ci = CIN[l], Co = COUT[l], H = HIN[l], Ho = H / 2;
        const float *wl = w + L.cw[l], *bl = w + L.cb[l];
        for (int n = 0; n < N; ++n)
            for (int co = 0; co < Co; ++co)
                for (int yo = 0; yo < Ho; ++yo)
                    for (int xo = 0; xo < Ho; ++xo) {
                        float best = 0.0f;
                        int arg = -1;
                        for (int q = 0; q < 4; ++q) {
                            const int y = 2 * yo + q / 2, xx = 2 * xo + q % 2;
                            float acc = bl[co];
                            for (int ci = 0; ci < Ci; ++ci)
                                for (int ky = 0; ky < 3; ++ky)
                                    for (int kx = 0; kx < 3; ++kx) {
                                        const int yy = y + ky - 1, xi = xx + kx - 1;
                                        if (yy < 0 || yy >= H || xi < 0 || xi >= H) continue;
                                        acc += wl[((long)co * Ci + ci) * 9 + ky * 3 + kx] *
                                               a->in[l][(((long)n * Ci + ci) * H + yy) * H + xi];
                                    }
                            float v = acc > 0.0f ? acc : 0.0f;
                            if (round) v = bf16_round(v);
                            if (arg < 0 || v > best) {
                                best = v;
                                arg = q;
                            }
                        }
                        const long o = (((long)n * Co + co) * Ho + yo) * Ho + xo;
                        a->pooled[l][o] = best;
                        a->arg[l][o] = arg;
                    }
        if (l + 1 < NCONV) memcpy(a->in[l + 1], a->pooled[l], sizeof(float) * N * Co * Ho * Ho);
    }
    const float *feat = a->pooled[NCONV - 1]; /* [N][1024] in c*16 + y*4 + x order */
    for (int n = 0; n < N; ++n) {
        for (int o = 0; o < FC1_OUT; ++o) {
            float acc = w[L.f1b + o];
            for (int i = 0; i < FC1_IN; ++i) acc += w[L.f1w + (long)o * FC1_IN + i] * feat[(long)n * FC1_IN + i];
            float v = acc > 0.0f ? acc : 0.0f;
            a->h1[n * FC1_OUT + o] = round ? bf16_round(v) : v;
        }
        float acc = w[L.f2b];
        for (int i = 0; i < FC1_OUT; ++i) acc += w[L.f2w + i] * a->h1[n * FC1_OUT + i];
        a->z[n] = acc;
    }
    return 0;
}

int oracle_nn_forward(const float *params, int N, const uint16_t *x, float *logits, int round)
{
    acts a;
    int rc = forward(params, N, x, round, &a);
    if (rc == 0) memcpy(logits, a.z, sizeof(float) * N);
    free_acts(&a);
    return rc;
}

float oracle_nn_loss(const float *logits, const float *labels, int N)
{
    double s = 0.0;
    for (int n = 0; n < N; ++n) {
        const double z = logits[n], y = labels[n];
        s += (z > 0 ? z : 0) - z * y + log1p(exp(-fabs(z)));
    }
    return (float)(s / N);
}

/* Gradients of the mean loss (grads: param_count floats). Returns the loss. */
float oracle_nn_backward(const float *params, int N, const uint16_t *x, const float *labels, float *grads,
                         float *logits_out, int round)
{
    layout L = make_layout();
    acts a;
    if (forward(params, N, x, round, &a) != 0) {
        free_acts(&a);
        return NAN;
    }
    const float *w = a.w;
    memset(grads, 0, sizeof(float) * L.total);
    if (logits_out) memcpy(logits_out, a.z, sizeof(float) * N);
    float *dz = (float *)malloc(sizeof(float) * N);
    float *dh = (float *)malloc(sizeof(float) * N * FC1_OUT);
    float *dfeat = (float *)calloc((size_t)N * FC1_IN, sizeof(float));
    for (int n = 0; n < N; ++n) {
        const float s = 1.0f / (1.0f + expf(-a.z[n]));
        dz[n] = (s - labels[n]) / (float)N;
    }
    for (int n = 0; n < N; ++n) {
        grads[L.f2b] += dz[n];
        for (int i = 0; i < FC1_OUT; ++i) {
            grads[L.f2w + i] += dz[n] * a.h1[n * FC1_OUT + i];
            dh[n * FC1_OUT + i] = a.h1[n * FC1_OUT + i] > 0.0f ? dz[n] * w[L.f2w + i] : 0.0f;
        }
    }
    const float *feat = a.pooled[NCONV - 1];
    for (int n = 0; n < N; ++n)
        for (int o = 0; o < FC1_OUT; ++o) {
            const float g = dh[n * FC1_OUT + o];
            grads[L.f1b + o] += g;
            for (int i = 0; i < FC1_IN; ++i) {
                grads[L.f1w + (long)o * FC1_IN + i] += g * feat[(long)n * FC1_IN + i];
                dfeat[(long)n * FC1_IN + i] += g * w[L.f1w + (long)o * FC1_IN + i];
            }
        }
    float *dpool = dfeat; /* gradient w.r.t. the current layer's pooled output */
    for (int l = NCONV - 1; l >= 0; --l) {
        const int Ci = CIN[l], Co = COUT[l], H = HIN[l], Ho = H / 2;
        const float *wl = w + L.cw[l];
        float *din = l > 0 ? (float *)calloc((size_t)N * Ci * H * H, sizeof(float)) : NULL;
        for (int n = 0; n < N; ++n)
            for (int co = 0; co < Co; ++co)
                for (int yo = 0; yo < Ho; ++yo)
                    for (int xo = 0; xo < Ho; ++xo) {
                        const long o = (((long)n * Co + co) * Ho + yo) * Ho + xo;
                        if (!(a.pooled[l][o] > 0.0f)) continue;
                        const float g = dpool[o];
                        const int q = a.arg[l][o];
                        const int y = 2 * yo + q / 2, xx = 2 * xo + q % 2;
                        grads[L.cb[l] + co] += g;
                        for (int ci = 0; ci < Ci; ++ci)
                            for (int ky = 0; ky < 3; ++ky)
                                for (int kx = 0; kx < 3; ++kx) {
                                    const int yy = y + ky - 1, xi = xx + kx - 1;
                                    if (yy < 0 || yy >= H || xi < 0 || xi >= H) continue;
                                    const long wi = ((long)co * Ci + ci) * 9 + ky * 3 + kx;
                                    const long ii = (((long)n * Ci + ci) * H + yy) * H + xi;
                                    grads[L.cw[l] + wi] += g * a.in[l][ii];
                                    if (din) din[ii] += g * wl[wi];
                                }
                    }
        if (dpool != dfeat) free(dpool);
        dpool = din;
    }
    free(dfeat);
    free(dz);
    free(dh);
    float loss = oracle_nn_loss(a.z, labels, N);
    free_acts(&a);
    return loss;
}

/* One AdamW step on the float master parameters; writes the bfloat16 copy
 * (nearest even) the forward pass uses.  step counts from 1. */
void oracle_adamw_step(long count, float *master, const float *grads, float *m, float *v, uint16_t *bf16_out,
                       float lr, float beta1, float beta2, float eps, float wd, int step)
{
    const float c1 = 1.0f - powf(beta1, (float)step);
    const float c2 = 1.0f - powf(beta2, (float)step);
    for (long i = 0; i < count; ++i) {
        const float g = grads[i];
        m[i] = beta1 * m[i] + (1.0f - beta1) * g;
        v[i] = beta2 * v[i] + (1.0f - beta2) * g * g;
        const float mh = m[i] / c1, vh = v[i] / c2;
        master[i] -= lr * (mh / (sqrtf(vh) + eps) + wd * master[i]);
        const float r = bf16_round(master[i]);
        uint32_t u;
        memcpy(&u, &r, 4);
        bf16_out[i] = (uint16_t)(u >> 16);
    }
}
