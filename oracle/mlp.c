/*
 * mlp.c - FP64 oracle of the neural radiance cache network.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain loops, no blocking.
 *
 * The paper has no learned component; this network is the radiance cache
 * the tracer is extended with: a frequency encoding of the hit (position,
 * normal, view direction), a 96-64-64-64-64-3 MLP with ReLU hidden layers
 * and an exp output, a relative-L2 loss and Adam.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define N_FREQ 12
static const int DIMS[6] = {96, 64, 64, 64, 64, 3};

/* features: [x_hat(3), n(3), v(3), then for k = 0..11:
 *            sin(2^k pi x_hat_j) j=0..2, cos(2^k pi x_hat_j) j=0..2], 0-pad */
void orc_nrc_encode(int64_t n, const double* in, const double* lo, const double* hi, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    const double* q = in + 9 * i;
    double* f = out + 96 * i;
    memset(f, 0, sizeof(double) * 96);
    double xh[3];
    for (int j = 0; j < 3; ++j) {
      xh[j] = (q[j] - lo[j]) / (hi[j] - lo[j]);
      f[j] = xh[j];
      f[3 + j] = q[3 + j];
      f[6 + j] = q[6 + j];
    }
    for (int k = 0; k < N_FREQ; ++k) {
      double w = ldexp(M_PI, k);
      for (int j = 0; j < 3; ++j) {
        f[9 + 6 * k + j] = sin(w * xh[j]);
        f[9 + 6 * k + 3 + j] = cos(w * xh[j]);
      }
    }
  }
}

/* Round to the nearest BF16 value (ties to even), through FP32.  Used when
 * the network's activations are stored in BF16 between layers. */
double orc_round_bf16(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}

static int64_t w_off(int l) {
  int64_t o = 0;
  for (int k = 0; k < l; ++k) o += (int64_t)DIMS[k] * DIMS[k + 1];
  return o;
}
static int64_t b_off(int l) {
  int64_t o = 0;
  for (int k = 0; k < l; ++k) o += DIMS[k + 1];
  return o;
}

/* forward for one sample; keeps pre-activations z[l] and activations a[l];
 * bf16: hidden activations are rounded to BF16 after the ReLU */
static void fwd1(const double* x, const double* W, const double* B, double a[6][96], double z[6][96], int bf16) {
  for (int j = 0; j < DIMS[0]; ++j) a[0][j] = x[j];
  for (int l = 0; l < 5; ++l) {
    const double* Wl = W + w_off(l);
    const double* Bl = B + b_off(l);
    for (int o = 0; o < DIMS[l + 1]; ++o) {
      double s = Bl[o];
      for (int k = 0; k < DIMS[l]; ++k) s += Wl[(int64_t)o * DIMS[l] + k] * a[l][k];
      z[l + 1][o] = s;
      double h = (l < 4) ? (s > 0 ? s : 0) : exp(s);
      a[l + 1][o] = (bf16 && l < 4) ? orc_round_bf16(h) : h;
    }
  }
}

void orc_mlp_forward_ex(int64_t n, const double* x, const double* W, const double* B, double* y, int bf16) {
  double a[6][96], z[6][96];
  for (int64_t i = 0; i < n; ++i) {
    fwd1(x + 96 * i, W, B, a, z, bf16);
    for (int c = 0; c < 3; ++c) y[3 * i + c] = a[5][c];
  }
}

void orc_mlp_forward(int64_t n, const double* x, const double* W, const double* B, double* y) {
  orc_mlp_forward_ex(n, x, W, B, y, 0);
}

double orc_mlp_loss_grad_ex(int64_t n, const double* x, const double* target, const double* W,
                            const double* B, double* dW, double* dB, int bf16) {
  memset(dW, 0, sizeof(double) * (size_t)w_off(5));
  memset(dB, 0, sizeof(double) * (size_t)b_off(5));
  double loss = 0;
  double a[6][96], z[6][96], g[6][96];
  double inv = 1.0 / (3.0 * (double)n);
  for (int64_t i = 0; i < n; ++i) {
    fwd1(x + 96 * i, W, B, a, z, bf16);
    for (int c = 0; c < 3; ++c) {
      double y = a[5][c], t = target[3 * i + c];
      double den = y * y + 0.01;          /* sg(y)^2 + 0.01: no gradient through it */
      loss += (y - t) * (y - t) / den * inv;
      double dy = 2.0 * (y - t) / den * inv;
      g[5][c] = dy * y;                   /* d exp(z)/dz = exp(z) */
    }
    for (int l = 4; l >= 0; --l) {
      const double* Wl = W + w_off(l);
      double* dWl = dW + w_off(l);
      double* dBl = dB + b_off(l);
      double gr[96];   /* the backward signal as stored: what every gradient of this layer uses */
      for (int o = 0; o < DIMS[l + 1]; ++o) gr[o] = bf16 ? orc_round_bf16(g[l + 1][o]) : g[l + 1][o];
      for (int o = 0; o < DIMS[l + 1]; ++o) {
        dBl[o] += gr[o];
        for (int k = 0; k < DIMS[l]; ++k) dWl[(int64_t)o * DIMS[l] + k] += gr[o] * a[l][k];
      }
      if (l > 0) {
        for (int k = 0; k < DIMS[l]; ++k) {
          double s = 0;
          for (int o = 0; o < DIMS[l + 1]; ++o) s += Wl[(int64_t)o * DIMS[l] + k] * gr[o];
          g[l][k] = z[l][k] > 0 ? s : 0.0;
        }
      }
    }
  }
  return loss;
}

double orc_mlp_loss_grad(int64_t n, const double* x, const double* target, const double* W,
                         const double* B, double* dW, double* dB) {
  return orc_mlp_loss_grad_ex(n, x, target, W, B, dW, dB, 0);
}

void orc_adam(int64_t n, double* w, const double* g, double* m, double* v, int64_t step, double lr,
              double b1, double b2, double eps) {
  double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    w[i] -= lr * mh / (sqrt(vh) + eps);
  }
}
