/*
 * Oracle: the surrogate source network (spec item 4 reshaping the black
 * box of Sec. 4 step 4 into a learned field) in plain FP64.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Network: x in R^3 -> 256 -> 256 -> 256 -> 256 -> 1, SiLU after each hidden
 * layer: h_1 = s(W_1 x + c_1), h_l = s(W_l h_{l-1} + c_l) (l = 2..4),
 * y = w_5 . h_4 + c_5, s(z) = z / (1 + exp(-z)).
 * Parameter vector layout (ORC_MLP_NPARAM doubles):
 *   W1 [256][3], c1 [256], W2 [256][256], c2, W3, c3, W4, c4, w5 [256], c5 [1]
 * (weights row-major [out][in]).
 * act_bf16 = 1 rounds every hidden activation to bfloat16 (round to nearest
 * even), as a network that stores its activations in bfloat16 does.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define H 256

static const int64_t OFF_W1 = 0;
static const int64_t OFF_C1 = OFF_W1 + H * 3;
static const int64_t OFF_W2 = OFF_C1 + H;
static const int64_t OFF_C2 = OFF_W2 + H * H;
static const int64_t OFF_W3 = OFF_C2 + H;
static const int64_t OFF_C3 = OFF_W3 + H * H;
static const int64_t OFF_W4 = OFF_C3 + H;
static const int64_t OFF_C4 = OFF_W4 + H * H;
static const int64_t OFF_W5 = OFF_C4 + H;
static const int64_t OFF_C5 = OFF_W5 + H;

int64_t orc_mlp_nparam(void) { return OFF_C5 + 1; }

double orc_bf16_round(double x)
{
    /* round-to-nearest-even to 8 significant bits (bfloat16), via float bits */
    union { float f; uint32_t u; } v;
    v.f = (float)x;
    if ((v.u & 0x7f800000u) == 0x7f800000u) return x;   /* inf / nan unchanged */
    const uint32_t lsb = (v.u >> 16) & 1u;
    v.u = (v.u + 0x7fffu + lsb) & 0xffff0000u;
    return (double)v.f;
}

static double silu(double z) { return z / (1.0 + exp(-z)); }
static double silu_d(double z)
{
    const double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 + z * (1.0 - s));
}

/* forward of one point; keeps pre-activations z[4][H] and activations h[4][H] */
static double forward_one(const double* p, const double* x, int act_bf16, double z[4][H], double h[4][H])
{
    for (int o = 0; o < H; ++o) {
        double s = p[OFF_C1 + o];
        for (int i = 0; i < 3; ++i) s += p[OFF_W1 + o * 3 + i] * x[i];
        z[0][o] = s;
        h[0][o] = act_bf16 ? orc_bf16_round(silu(s)) : silu(s);
    }
    const int64_t offW[3] = {OFF_W2, OFF_W3, OFF_W4}, offC[3] = {OFF_C2, OFF_C3, OFF_C4};
    for (int l = 1; l < 4; ++l) {
        for (int o = 0; o < H; ++o) {
            double s = p[offC[l - 1] + o];
            const double* w = p + offW[l - 1] + (int64_t)o * H;
            for (int i = 0; i < H; ++i) s += w[i] * h[l - 1][i];
            z[l][o] = s;
            h[l][o] = act_bf16 ? orc_bf16_round(silu(s)) : silu(s);
        }
    }
    double y = p[OFF_C5];
    for (int i = 0; i < H; ++i) y += p[OFF_W5 + i] * h[3][i];
    return y;
}

void orc_mlp_forward(const double* params, int64_t n, const double* X, int act_bf16, double* y_out)
{
    double (*z)[H] = (double(*)[H])malloc(sizeof(double) * 4 * H);
    double (*h)[H] = (double(*)[H])malloc(sizeof(double) * 4 * H);
    for (int64_t k = 0; k < n; ++k) y_out[k] = forward_one(params, X + 3 * k, act_bf16, z, h);
    free(z);
    free(h);
}

/* mean squared error L = 1/n sum_k (y_k - t_k)^2 and its gradient with
 * respect to every parameter (backpropagation through the SiLU layers) */
double orc_mlp_loss_grad(const double* params, int64_t n, const double* X, const double* t, int act_bf16,
                         double* grad)
{
    const int64_t np = orc_mlp_nparam();
    memset(grad, 0, sizeof(double) * (size_t)np);
    double (*z)[H] = (double(*)[H])malloc(sizeof(double) * 4 * H);
    double (*h)[H] = (double(*)[H])malloc(sizeof(double) * 4 * H);
    double* dz = (double*)malloc(sizeof(double) * H);
    double* dh = (double*)malloc(sizeof(double) * H);
    double loss = 0.0;
    const int64_t offW[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4}, offC[4] = {OFF_C1, OFF_C2, OFF_C3, OFF_C4};
    for (int64_t k = 0; k < n; ++k) {
        const double* x = X + 3 * k;
        const double y = forward_one(params, x, act_bf16, z, h);
        const double e = y - t[k];
        loss += e * e;
        const double dy = 2.0 * e / (double)n;
        grad[OFF_C5] += dy;
        for (int i = 0; i < H; ++i) {
            grad[OFF_W5 + i] += dy * h[3][i];
            dh[i] = dy * params[OFF_W5 + i];
        }
        for (int l = 3; l >= 0; --l) {
            for (int o = 0; o < H; ++o) dz[o] = dh[o] * silu_d(z[l][o]);
            for (int o = 0; o < H; ++o) grad[offC[l] + o] += dz[o];
            if (l == 0) {
                for (int o = 0; o < H; ++o)
                    for (int i = 0; i < 3; ++i) grad[OFF_W1 + o * 3 + i] += dz[o] * x[i];
            } else {
                for (int o = 0; o < H; ++o)
                    for (int i = 0; i < H; ++i) grad[offW[l] + (int64_t)o * H + i] += dz[o] * h[l - 1][i];
                for (int i = 0; i < H; ++i) {
                    double s = 0.0;
                    for (int o = 0; o < H; ++o) s += params[offW[l] + (int64_t)o * H + i] * dz[o];
                    dh[i] = s;
                }
            }
        }
    }
    free(z); free(h); free(dz); free(dh);
    return loss / (double)n;
}

/* one Adam step (Kingma & Ba 2015) on every parameter, step count t >= 1 */
void orc_adam_step(int64_t np, double* params, const double* grad, double* m, double* v, int64_t t,
                   double lr, double beta1, double beta2, double eps)
{
    const double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < np; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        const double mh = m[i] / c1, vh = v[i] / c2;
        params[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
