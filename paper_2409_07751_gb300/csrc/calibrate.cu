// Host-side model preparation: the task-specific SiLU approximation of the
// paper (Eq. 11: range [max(mu - 5 sigma, x_min), min(mu + 5 sigma, x_max)]
// from the layer's input statistics under the plaintext KAN; Eq. 12:
// weighted least squares with weight 10 inside mu +- 3 sigma and 1 outside)
// and the comparison bound R of Algorithm 2.
//
// Readings: samples are n evenly spaced points including both ends; the
// polynomial is in the Chebyshev basis of the range mapped to [-1, 1]; the
// least-squares problem is solved by Householder QR; R = 1.1 (max|x| +
// max|t|) / 2 so that every comparison input |x - t| / (2R) stays in [-1, 1].
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace {

double silu(double x) { return x / (1.0 + exp(-x)); }

std::vector<double> knots(const kan_layer_desc& d) {
  const double h = (d.grid_hi - d.grid_lo) / d.G;
  std::vector<double> t;
  for (int m = 0; m <= d.G + 2 * d.k; m++) t.push_back(d.grid_lo + (double)(m - d.k) * h);
  return t;
}

// Cox-de Boor (Eqs. 2-3), half-open intervals; B has G+k entries
void bspline(double x, const std::vector<double>& t, int k, std::vector<double>& B) {
  const int nk = (int)t.size();
  B.assign(nk - 1, 0.0);
  for (int m = 0; m + 1 < nk; m++) B[m] = (t[m] <= x && x < t[m + 1]) ? 1.0 : 0.0;
  for (int j = 1; j <= k; j++) {
    for (int m = 0; m + j + 1 < nk; m++) {
      const double left = (x - t[m]) / (t[m + j] - t[m]) * B[m];
      const double right = (t[m + j + 1] - x) / (t[m + j + 1] - t[m + 1]) * B[m + 1];
      B[m] = left + right;
    }
    B.pop_back();
  }
}

// y[b][o] for x[b][i] through one exact layer (Eqs. 1-5)
void layer_forward(const kan_layer_desc& d, const std::vector<double>& x, size_t n,
                   std::vector<double>& y) {
  const std::vector<double> t = knots(d);
  const int nb = d.G + d.k;
  y.assign(n * d.n_out, 0.0);
  std::vector<double> B;
  for (size_t b = 0; b < n; b++)
    for (int i = 0; i < d.n_in; i++) {
      const double xi = x[b * d.n_in + i];
      bspline(xi, t, d.k, B);
      const double s = silu(xi);
      for (int o = 0; o < d.n_out; o++) {
        double sp = 0;
        for (int m = 0; m < nb; m++) sp += d.coef[((size_t)o * d.n_in + i) * nb + m] * B[m];
        y[b * d.n_out + o] += d.w_b[(size_t)o * d.n_in + i] * s + d.w_s[(size_t)o * d.n_in + i] * sp;
      }
    }
}

// least squares min ||A a - r|| by Householder QR (A: m x n, row-major)
std::vector<double> lstsq_qr(std::vector<double> A, std::vector<double> r, int m, int n) {
  for (int k = 0; k < n; k++) {
    double norm = 0;
    for (int i = k; i < m; i++) norm += A[(size_t)i * n + k] * A[(size_t)i * n + k];
    norm = sqrt(norm);
    if (norm == 0) continue;
    const double alpha = A[(size_t)k * n + k] > 0 ? -norm : norm;
    std::vector<double> v(m - k);
    for (int i = k; i < m; i++) v[i - k] = A[(size_t)i * n + k];
    v[0] -= alpha;
    double vv = 0;
    for (double e : v) vv += e * e;
    if (vv == 0) continue;
    for (int j = k; j < n; j++) {
      double s = 0;
      for (int i = k; i < m; i++) s += v[i - k] * A[(size_t)i * n + j];
      s = 2 * s / vv;
      for (int i = k; i < m; i++) A[(size_t)i * n + j] -= s * v[i - k];
    }
    double s = 0;
    for (int i = k; i < m; i++) s += v[i - k] * r[i];
    s = 2 * s / vv;
    for (int i = k; i < m; i++) r[i] -= s * v[i - k];
  }
  std::vector<double> a(n);
  for (int k = n - 1; k >= 0; k--) {
    double s = r[k];
    for (int j = k + 1; j < n; j++) s -= A[(size_t)k * n + j] * a[j];
    a[k] = s / A[(size_t)k * n + k];
  }
  return a;
}

}  // namespace

extern "C" {

int kan_silu_fit(double lo, double hi, double mu, double sigma, int degree, int n_samples,
                 double* cheb) {
  if (!(hi > lo) || degree < 1 || n_samples <= degree || !cheb) return CKKS_ERR_INVALID_ARG;
  const int n = degree + 1;
  std::vector<double> A((size_t)n_samples * n), r(n_samples);
  for (int s = 0; s < n_samples; s++) {
    const double x = lo + (hi - lo) * (double)s / (double)(n_samples - 1);
    const double y = (2.0 * x - (lo + hi)) / (hi - lo);
    const double sw = sqrt(fabs(x - mu) <= 3.0 * sigma ? 10.0 : 1.0);
    double t0 = 1.0, t1 = y;
    for (int j = 0; j < n; j++) {
      double tj;
      if (j == 0) tj = 1.0;
      else if (j == 1) tj = y;
      else {
        tj = 2.0 * y * t1 - t0;
        t0 = t1;
        t1 = tj;
      }
      A[(size_t)s * n + j] = sw * tj;
    }
    r[s] = sw * silu(x);
  }
  std::vector<double> a = lstsq_qr(A, r, n_samples, n);
  for (int j = 0; j < n; j++) cheb[j] = a[j];
  return CKKS_OK;
}

int kan_calibrate(const kan_layer_desc* layers, size_t n_layers, const double* X, size_t n,
                  int silu_degree, const double* fixed_range, int n_fit_samples, double* R,
                  double* silu_lo, double* silu_hi, double* cheb) {
  if (!layers || !X || n == 0 || !R || !silu_lo || !silu_hi || !cheb) return CKKS_ERR_INVALID_ARG;
  std::vector<double> h(X, X + n * layers[0].n_in), y;
  for (size_t li = 0; li < n_layers; li++) {
    const kan_layer_desc& d = layers[li];
    double sum = 0, mn = h[0], mx = h[0], amax = 0;
    for (double v : h) {
      sum += v;
      mn = std::min(mn, v);
      mx = std::max(mx, v);
      amax = std::max(amax, fabs(v));
    }
    const double mu = sum / (double)h.size();
    double var = 0;
    for (double v : h) var += (v - mu) * (v - mu);
    const double sigma = sqrt(var / (double)h.size());
    double lo, hi;
    if (fixed_range) {
      lo = fixed_range[0];
      hi = fixed_range[1];
    } else {
      lo = std::max(mu - 5.0 * sigma, mn);
      hi = std::min(mu + 5.0 * sigma, mx);
    }
    silu_lo[li] = lo;
    silu_hi[li] = hi;
    const int rc = kan_silu_fit(lo, hi, mu, sigma, silu_degree, n_fit_samples,
                                cheb + li * (size_t)(silu_degree + 1));
    if (rc != CKKS_OK) return rc;
    double tmax = 0;
    for (double t : knots(d)) tmax = std::max(tmax, fabs(t));
    R[li] = 1.1 * (amax + tmax) / 2.0;
    layer_forward(d, h, n, y);
    h.swap(y);
  }
  return CKKS_OK;
}

}  // extern "C"
