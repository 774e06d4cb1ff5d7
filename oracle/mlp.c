/*
 * FP64 oracle of the learned Riemann-flux network (TEST INFRASTRUCTURE ONLY,
 * see oracle.h).  The paper has no learned flux; the network is the small
 * multilayer perceptron of the learned-flux configuration: dense layers with
 * SiLU activations on every hidden layer and a linear output layer.
 *
 * Parameters are packed per layer l = 0..nl-1 as W_l[out][in] (row-major)
 * followed by b_l[out]; dims[0..nl] are the layer widths.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static double silu(double z) { return z / (1.0 + exp(-z)); }
static double dsilu(double z) {
  double s = 1.0 / (1.0 + exp(-z));
  return s * (1.0 + z * (1.0 - s));
}

static long n_params(int nl, const int* dims) {
  long n = 0;
  for (int l = 0; l < nl; ++l) n += (long)dims[l + 1] * dims[l] + dims[l + 1];
  return n;
}

/* forward pass of one sample keeping pre-activations z[l] and activations a[l] */
static void forward_one(int nl, const int* dims, const double* params, const double* x,
                        double** z, double** a) {
  memcpy(a[0], x, sizeof(double) * dims[0]);
  const double* p = params;
  for (int l = 0; l < nl; ++l) {
    int nin = dims[l], nout = dims[l + 1];
    const double* W = p;
    const double* b = p + (long)nout * nin;
    for (int o = 0; o < nout; ++o) {
      double s = b[o];
      for (int i = 0; i < nin; ++i) s += W[(long)o * nin + i] * a[l][i];
      z[l + 1][o] = s;
      a[l + 1][o] = (l + 1 < nl) ? silu(s) : s;
    }
    p += (long)nout * nin + nout;
  }
}

static int max_width(int nl, const int* dims) {
  int m = 0;
  for (int l = 0; l <= nl; ++l) if (dims[l] > m) m = dims[l];
  return m;
}

void orc_mlp_forward(int nl, const int* dims, const double* params, int n, const double* x,
                     double* y) {
  int mw = max_width(nl, dims);
  double* buf = (double*)malloc(sizeof(double) * 2 * (nl + 1) * mw);
  double *z[16], *a[16];
  for (int l = 0; l <= nl; ++l) { z[l] = buf + 2 * l * mw; a[l] = z[l] + mw; }
  for (int s = 0; s < n; ++s) {
    forward_one(nl, dims, params, x + (long)s * dims[0], z, a);
    memcpy(y + (long)s * dims[nl], a[nl], sizeof(double) * dims[nl]);
  }
  free(buf);
}

/* Backpropagation of L = 0.5/n sum_s |y_s - t_s|^2. */
double orc_mlp_grad(int nl, const int* dims, const double* params, int n, const double* x,
                    const double* target, double* grad) {
  long np = n_params(nl, dims);
  memset(grad, 0, sizeof(double) * np);
  int mw = max_width(nl, dims);
  double* buf = (double*)malloc(sizeof(double) * 3 * (nl + 1) * mw);
  double *z[16], *a[16], *dz[16];
  for (int l = 0; l <= nl; ++l) {
    z[l] = buf + 3 * l * mw; a[l] = z[l] + mw; dz[l] = a[l] + mw;
  }
  /* start of each layer's parameters */
  long off[16];
  off[0] = 0;
  for (int l = 0; l < nl; ++l) off[l + 1] = off[l] + (long)dims[l + 1] * dims[l] + dims[l + 1];
  double loss = 0.0;
  for (int s = 0; s < n; ++s) {
    forward_one(nl, dims, params, x + (long)s * dims[0], z, a);
    const double* t = target + (long)s * dims[nl];
    for (int o = 0; o < dims[nl]; ++o) {
      double e = a[nl][o] - t[o];
      loss += 0.5 * e * e;
      dz[nl][o] = e / n;                      /* linear output layer */
    }
    for (int l = nl - 1; l >= 0; --l) {
      int nin = dims[l], nout = dims[l + 1];
      const double* W = params + off[l];
      double* gW = grad + off[l];
      double* gb = gW + (long)nout * nin;
      for (int o = 0; o < nout; ++o) {
        gb[o] += dz[l + 1][o];
        for (int i = 0; i < nin; ++i) gW[(long)o * nin + i] += dz[l + 1][o] * a[l][i];
      }
      if (l > 0) {
        for (int i = 0; i < nin; ++i) {
          double s2 = 0.0;
          for (int o = 0; o < nout; ++o) s2 += W[(long)o * nin + i] * dz[l + 1][o];
          dz[l][i] = s2 * dsilu(z[l][i]);
        }
      }
    }
  }
  free(buf);
  return loss / n;
}
