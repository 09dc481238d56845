/*
 * Oracle: loss and gradient of the learned smoothness indicator network,
 * FP64, plain loops (an extension of the method: the paper has no such
 * component). Test infrastructure only (see oracle.h).
 *
 * For each sample s with data vector x (63 entries, column s of the
 * [63][ld] array) and label y:
 *   xh = x / (max_c |x_c| + 1e-30)
 *   z_j = sum_c W1[j][c] xh_c + b1_j,  h_j = max(z_j, 0)   (8 units)
 *   logit = sum_j w2_j h_j + b2
 *   loss_s = w_y (log(1 + exp(logit)) - y logit),  w_1 = 1, w_0 = neg_weight
 * Loss = mean_s loss_s; the gradient follows by the chain rule.
 * Parameter layout: W1 [8][63] row major, b1 [8], w2 [8], b2.
 */
#include <cmath>
#include <vector>

#include "oracle_internal.h"

namespace {
constexpr int kD = 63, kH = 8;
}

extern "C" int orc_mlp_nparams(void) { return kH * kD + 2 * kH + 1; }

extern "C" int orc_mlp_loss_grad(const double *params, const double *x, const double *y, int n,
                                 long long ld, double neg_weight, double *loss, double *grad) {
    if (n <= 0 || ld < n) return -1;
    const int np = kH * kD + 2 * kH + 1;
    const double *W1 = params, *b1 = params + kH * kD, *w2 = b1 + kH, b2 = w2[kH];
    for (int p = 0; p < np; ++p) grad[p] = 0.0;
    double total = 0.0;
    std::vector<double> xh(kD), z(kH), h(kH);
    for (int s = 0; s < n; ++s) {
        double m = 0.0;
        for (int c = 0; c < kD; ++c) m = std::fmax(m, std::fabs(x[(long long)c * ld + s]));
        for (int c = 0; c < kD; ++c) xh[c] = x[(long long)c * ld + s] / (m + 1e-30);
        double logit = b2;
        for (int j = 0; j < kH; ++j) {
            double a = b1[j];
            for (int c = 0; c < kD; ++c) a += W1[j * kD + c] * xh[c];
            z[j] = a;
            h[j] = a > 0.0 ? a : 0.0;
            logit += w2[j] * h[j];
        }
        const double wt = y[s] > 0.5 ? 1.0 : neg_weight;
        total += wt * (std::log1p(std::exp(logit)) - y[s] * logit);
        const double p = 1.0 / (1.0 + std::exp(-logit));
        const double dl = wt * (p - y[s]) / n;
        for (int j = 0; j < kH; ++j) {
            grad[kH * kD + kH + j] += dl * h[j];
            const double dz = z[j] > 0.0 ? dl * w2[j] : 0.0;
            grad[kH * kD + j] += dz;
            for (int c = 0; c < kD; ++c) grad[j * kD + c] += dz * xh[c];
        }
        grad[kH * kD + 2 * kH] += dl;
    }
    *loss = total / n;
    return 0;
}
