/*
 * FP64 oracle of the learned preconditioner scale (test infrastructure only).
 *
 * The model is not in the paper: the paper's preconditioner study (Sec. 4.4, Table 1)
 * motivates correcting the diagonal preconditioner (diag(A) - theta)^-1 of Sec. 2.  Per
 * (row i, column j) a 3 -> 64 -> 64 -> 1 perceptron with ReLU hidden layers maps the
 * features f = (f1, f2, f3) to z, and s = softplus(z) > 0 scales the diagonal step:
 *     w_ij = s_ij * r_ij / (d_i - theta_j).
 * Because s > 0 the preconditioner stays symmetric positive (definite where the
 * diagonal one is).  Features (computed by the caller):
 *     f1 = (d_i - theta_j) / (8 c),  f2 = rho_i / c,  f3 = r_ij / max_i |r_ij|,
 * with rho_i the off-diagonal 2-norm of row i and c the mean of rho over the rows.
 *
 * Parameter vector layout (float64 here, float on the GPU), 4481 entries:
 *     W1 [64][3], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1]   (row-major, out x in)
 *
 * Training loss per column j (scale-invariant, like the span LOBPCG uses):
 *     L_j = 1 - (w.e)^2 / (|w|^2 |e|^2)
 * with e the exact correction x* - x made orthogonal to x.  Rows outside the learned
 * region contribute fixed parts (w.e)_far and |w|^2_far to the column sums.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define H 64
#define NPARAM (H * 3 + H + H * H + H + H + 1)

int oracle_mlp_num_params(void) { return NPARAM; }

static double softplus(double z) { return z > 30.0 ? z : log1p(exp(z)); }
static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

/* Forward pass of one sample; fills h1/h2 (post-ReLU) and a1/a2 (pre-activation) when non-NULL. */
static double forward1(const double* P, const double* f, double* a1, double* h1, double* a2, double* h2,
                       double* zout) {
  const double *W1 = P, *b1 = W1 + H * 3, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H, *b3 = W3 + H;
  double la1[H], lh1[H], la2[H], lh2[H];
  for (int i = 0; i < H; ++i) {
    double s = b1[i];
    for (int k = 0; k < 3; ++k) s += W1[i * 3 + k] * f[k];
    la1[i] = s;
    lh1[i] = s > 0.0 ? s : 0.0;
  }
  for (int i = 0; i < H; ++i) {
    double s = b2[i];
    for (int k = 0; k < H; ++k) s += W2[i * H + k] * lh1[k];
    la2[i] = s;
    lh2[i] = s > 0.0 ? s : 0.0;
  }
  double z = b3[0];
  for (int k = 0; k < H; ++k) z += W3[k] * lh2[k];
  if (a1) memcpy(a1, la1, sizeof la1);
  if (h1) memcpy(h1, lh1, sizeof lh1);
  if (a2) memcpy(a2, la2, sizeof la2);
  if (h2) memcpy(h2, lh2, sizeof lh2);
  if (zout) *zout = z;
  return softplus(z);
}

/* s_i for N samples (features N x 3, row-major). */
void oracle_mlp_forward(const double* P, int64_t N, const double* F, double* s) {
  for (int64_t i = 0; i < N; ++i) s[i] = forward1(P, F + 3 * i, NULL, NULL, NULL, NULL, NULL);
}

/* Adds sum_i g_i * ds_i/dP to grad (length NPARAM). */
void oracle_mlp_backward(const double* P, int64_t N, const double* F, const double* g, double* grad) {
  const double *W2 = P + H * 3 + H, *W3 = W2 + H * H + H;
  double *gW1 = grad, *gb1 = gW1 + H * 3, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gW3 = gb2 + H, *gb3 = gW3 + H;
  for (int64_t n = 0; n < N; ++n) {
    const double* f = F + 3 * n;
    double a1[H], h1[H], a2[H], h2[H], z;
    forward1(P, f, a1, h1, a2, h2, &z);
    const double dz = g[n] * sigmoid(z); /* d softplus / dz = sigmoid */
    double d2[H], d1[H];
    gb3[0] += dz;
    for (int k = 0; k < H; ++k) {
      gW3[k] += dz * h2[k];
      d2[k] = a2[k] > 0.0 ? dz * W3[k] : 0.0;
    }
    for (int i = 0; i < H; ++i) {
      gb2[i] += d2[i];
      for (int k = 0; k < H; ++k) gW2[i * H + k] += d2[i] * h1[k];
    }
    for (int k = 0; k < H; ++k) {
      double s = 0.0;
      for (int i = 0; i < H; ++i) s += W2[i * H + k] * d2[i];
      d1[k] = a1[k] > 0.0 ? s : 0.0;
    }
    for (int i = 0; i < H; ++i) {
      gb1[i] += d1[i];
      for (int k = 0; k < 3; ++k) gW1[i * 3 + k] += d1[i] * f[k];
    }
  }
}

/* Column losses and dL/ds.  Samples are grouped by column: col[i] in [0, ncol).
 *   q_i = r_i / (d_i - theta), e_i = exact correction component, s_i = scale.
 *   far_we[c], far_ww[c]: contributions of the rows outside the learned region;
 *   ee[c] = |e|^2 over all rows of column c.
 * Returns the mean loss over columns; dLds[i] = d(mean loss)/ds_i. */
double oracle_mlp_loss(int64_t N, int ncol, const int32_t* col, const double* q, const double* e,
                       const double* s, const double* far_we, const double* far_ww, const double* ee,
                       double* dLds) {
  double* we = (double*)calloc((size_t)ncol, sizeof(double));
  double* ww = (double*)calloc((size_t)ncol, sizeof(double));
  for (int c = 0; c < ncol; ++c) we[c] = far_we[c], ww[c] = far_ww[c];
  for (int64_t i = 0; i < N; ++i) {
    const double w = s[i] * q[i];
    we[col[i]] += w * e[i];
    ww[col[i]] += w * w;
  }
  double loss = 0.0;
  for (int c = 0; c < ncol; ++c) loss += 1.0 - we[c] * we[c] / (ww[c] * ee[c]);
  loss /= ncol;
  for (int64_t i = 0; i < N; ++i) {
    const int c = col[i];
    const double w = s[i] * q[i];
    /* L_c = 1 - we^2 / (ww ee):  dL/dw = -2 we e / (ww ee) + 2 we^2 w / (ww^2 ee) */
    const double dLdw = (-2.0 * we[c] * e[i] / (ww[c] * ee[c]) + 2.0 * we[c] * we[c] * w / (ww[c] * ww[c] * ee[c]));
    dLds[i] = dLdw * q[i] / ncol;
  }
  free(we);
  free(ww);
  return loss;
}
