/*
 * FPIC oracle, learned part: the multilayer perceptron that predicts the
 * implicit scheme's converged step and the hybrid's scheme choice (the
 * learned-guess component of the workload; the paper has no network).
 *
 * TEST INFRASTRUCTURE ONLY (see fpic_oracle.c).  Plain serial loops.
 *
 * Network: x (14) -> 128 -> 128 -> 128 -> y (9), ReLU between layers.
 * Layer l: z_l = W_l a_{l-1} + b_l, W_l row-major [out][in].
 * Precision model of the tensor-core path ("BF16 weights, FP32
 * accumulate"): every GEMM operand (weights, the input, the activations fed
 * to the next layer, the backward deltas) is rounded to bfloat16
 * (round-to-nearest-even); products are accumulated in FP32; biases,
 * pre-activations, outputs and gradients are FP32.  mode 0 uses that model;
 * mode 1 evaluates the same network in FP64 without rounding (for the
 * finite-difference pin of the gradients).
 *
 * Loss per sample: sum over the 8 regression outputs k of m_k (y_k - t_k)^2
 * plus the logistic loss of the scheme logit y_6 against the label s in
 * {0,1}; averaged over the batch.  Regression outputs: 0..5 the corrections,
 * 7, 8 auxiliary; output 6 is the logit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MLP_IN 14
#define MLP_H 128
#define MLP_OUT 9

/* bfloat16 round-to-nearest-even of a float (NaN kept). */
static float bf16r(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

static const int dims[5] = {MLP_IN, MLP_H, MLP_H, MLP_H, MLP_OUT};

/* Parameter vector layout: W1 b1 W2 b2 W3 b3 W4 b4. */
int64_t or_mlp_nparams(void)
{
    int64_t n = 0;
    for (int l = 0; l < 4; ++l) n += (int64_t)dims[l + 1] * dims[l] + dims[l + 1];
    return n;
}

static void offsets(int64_t *oW, int64_t *ob)
{
    int64_t o = 0;
    for (int l = 0; l < 4; ++l) {
        oW[l] = o;
        o += (int64_t)dims[l + 1] * dims[l];
        ob[l] = o;
        o += dims[l + 1];
    }
}

/* Forward pass of B samples.  acts (optional, B x 3 x 128): post-activation
 * of the hidden layers (as fed to the next GEMM, i.e. rounded in mode 0);
 * pre (optional, B x 3 x 128): hidden pre-activations. */
static void fwd1(const double *P, const double *x, int mode, double *y, double *act, double *pre)
{
    int64_t oW[4], ob[4];
    offsets(oW, ob);
    double a[MLP_H], z[MLP_H], in[MLP_H];
    for (int i = 0; i < MLP_IN; ++i) in[i] = mode == 0 ? bf16r((float)x[i]) : x[i];
    for (int l = 0; l < 4; ++l) {
        int ni = dims[l], no = dims[l + 1];
        for (int o = 0; o < no; ++o) {
            if (mode == 0) {
                float acc = 0.0f;
                for (int i = 0; i < ni; ++i)
                    acc += bf16r((float)P[oW[l] + (int64_t)o * ni + i]) * (float)in[i];
                z[o] = (double)(acc + (float)P[ob[l] + o]);
            } else {
                double acc = 0.0;
                for (int i = 0; i < ni; ++i) acc += P[oW[l] + (int64_t)o * ni + i] * in[i];
                z[o] = acc + P[ob[l] + o];
            }
        }
        if (l == 3) {
            for (int o = 0; o < no; ++o) y[o] = z[o];
            break;
        }
        for (int o = 0; o < no; ++o) {
            double h = z[o] > 0.0 ? z[o] : 0.0;
            a[o] = mode == 0 ? bf16r((float)h) : h;
            if (pre) pre[l * MLP_H + o] = z[o];
            if (act) act[l * MLP_H + o] = a[o];
        }
        memcpy(in, a, sizeof(double) * no);
    }
}

void or_mlp_forward(const double *P, int64_t B, const double *x, int mode, double *y, double *act, double *pre)
{
    for (int64_t b = 0; b < B; ++b)
        fwd1(P, x + b * MLP_IN, mode, y + b * MLP_OUT, act ? act + b * 3 * MLP_H : NULL,
             pre ? pre + b * 3 * MLP_H : NULL);
}

/* d loss / d y for one sample; returns the sample's loss. */
static double dloss(const double *y, const double *t, const double *m, double s, double *dy)
{
    double L = 0.0;
    for (int k = 0; k < MLP_OUT; ++k) {
        if (k == 6) {
            /* logistic loss log(1 + e^y) - s y, stable form */
            double v = y[6];
            double sp = v > 0 ? v + log1p(exp(-v)) : log1p(exp(v));
            L += sp - s * v;
            dy[6] = 1.0 / (1.0 + exp(-v)) - s;
        } else {
            double d = y[k] - t[k];
            L += m[k] * d * d;
            dy[k] = 2.0 * m[k] * d;
        }
    }
    return L;
}

/* Loss and gradient (averaged over the batch).  t: B x 9 targets (entry 6
 * unused), s: B labels, m: 9 regression weights.  grad: nparams. */
double or_mlp_loss_grad(const double *P, int64_t B, const double *x, const double *t, const double *s,
                        const double *m, int mode, double *grad)
{
    int64_t oW[4], ob[4];
    offsets(oW, ob);
    int64_t np = or_mlp_nparams();
    if (grad) memset(grad, 0, sizeof(double) * np);
    double Ltot = 0.0;
    double y[MLP_OUT], dy[MLP_OUT], act[3 * MLP_H], pre[3 * MLP_H];
    for (int64_t b = 0; b < B; ++b) {
        const double *xb = x + b * MLP_IN;
        fwd1(P, xb, mode, y, act, pre);
        Ltot += dloss(y, t + b * MLP_OUT, m, s[b], dy);
        if (!grad) continue;
        /* backward: delta of layer 4 = dy (scaled by 1/B at the end) */
        double delta[MLP_H], dprev[MLP_H], in0[MLP_IN];
        for (int i = 0; i < MLP_IN; ++i) in0[i] = mode == 0 ? bf16r((float)xb[i]) : xb[i];
        int no = MLP_OUT;
        for (int k = 0; k < no; ++k) delta[k] = dy[k];
        for (int l = 3; l >= 0; --l) {
            int ni = dims[l];
            const double *ain = l == 0 ? in0 : act + (l - 1) * MLP_H;
            double dr[MLP_H];    /* delta as a GEMM operand */
            for (int o = 0; o < no; ++o) dr[o] = mode == 0 ? bf16r((float)delta[o]) : delta[o];
            for (int o = 0; o < no; ++o) {
                grad[ob[l] + o] += delta[o];
                for (int i = 0; i < ni; ++i) grad[oW[l] + (int64_t)o * ni + i] += dr[o] * ain[i];
            }
            if (l == 0) break;
            for (int i = 0; i < ni; ++i) {
                if (mode == 0) {
                    float acc = 0.0f;
                    for (int o = 0; o < no; ++o) acc += (float)dr[o] * bf16r((float)P[oW[l] + (int64_t)o * ni + i]);
                    dprev[i] = acc;
                } else {
                    double acc = 0.0;
                    for (int o = 0; o < no; ++o) acc += dr[o] * P[oW[l] + (int64_t)o * ni + i];
                    dprev[i] = acc;
                }
            }
            for (int i = 0; i < ni; ++i) delta[i] = pre[(l - 1) * MLP_H + i] > 0.0 ? dprev[i] : 0.0;
            no = ni;
        }
    }
    if (grad)
        for (int64_t k = 0; k < np; ++k) grad[k] /= (double)B;
    return Ltot / (double)B;
}

/* One Adam step (Kingma & Ba 2015) on the FP32 master parameters:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; P -= lr mhat / (sqrt(vhat) + eps),
 * mhat = m / (1 - b1^t), vhat = v / (1 - b2^t); all in FP32. */
void or_mlp_adam(float *P, float *mom, float *vel, const float *g, int64_t n, int t, float lr, float b1, float b2,
                 float eps)
{
    float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    for (int64_t k = 0; k < n; ++k) {
        mom[k] = b1 * mom[k] + (1.0f - b1) * g[k];
        vel[k] = b2 * vel[k] + (1.0f - b2) * g[k] * g[k];
        float mh = mom[k] / c1, vh = vel[k] / c2;
        P[k] -= lr * mh / (sqrtf(vh) + eps);
    }
}

/* bfloat16 rounding of n floats (exposed for its pin). */
void or_bf16_round(int64_t n, const float *x, float *out)
{
    for (int64_t k = 0; k < n; ++k) out[k] = bf16r(x[k]);
}
