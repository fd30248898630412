// Host-side model preparation: the task-specific SiLU approximation of the
// paper (Eq. 11: range [max(mu - 5 sigma, x_min), min(mu + 5 sigma, x_max)]
// from the statistics of the layer's inputs as the encrypted network computes
// them, i.e. under the HE-friendly KAN with the earlier layers calibrated; Eq. 12:
// weighted least squares with weight 10 inside mu +- 3 sigma and 1 outside)
// and the comparison bound R of Algorithm 2. The SiLU fits the paper compares
// against (Table 5) on the same range and degree: OLS (unit weights) and the
// minimax polynomial by the Remez exchange.
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

// odd monomial coefficients of f_n(x) = sum_i 4^-i C(2i,i) x (1-x^2)^i (exact dyadics)
std::vector<double> fn_odd(int n) {
  auto C = [](int a, int b) {
    int64_t r = 1;
    for (int i = 1; i <= b; i++) r = r * (a - b + i) / i;
    return r;
  };
  std::vector<double> c(n + 1);
  for (int l = 0; l <= n; l++) {
    int64_t num = 0;
    for (int i = l; i <= n; i++) num += C(2 * i, i) * C(i, l) * ((int64_t)1 << (2 * (n - i)));
    if (l & 1) num = -num;
    c[l] = (double)num / (double)((int64_t)1 << (2 * n));
  }
  return c;
}

// PolyComp(a, 0) = (1 + f(a)) / 2 with f = f_{n_d} o ... o f_{n_1}
double polycomp0(double a, const int* comp, int n_comp) {
  double u = a;
  for (int s = 0; s < n_comp; s++) {
    const std::vector<double> c = fn_odd(comp[s]);
    double acc = 0, p = u;
    const double u2 = u * u;
    for (double cl : c) {
      acc += cl * p;
      p *= u2;
    }
    u = acc;
  }
  return 0.5 + 0.5 * u;
}

// Algorithm 2 on plaintext values: soft order-0 indicators, the same recursion
void bspline_hef(double x, const std::vector<double>& t, int k, double R, const int* comp,
                 int n_comp, std::vector<double>& B) {
  const int nk = (int)t.size();
  B.assign(nk - 1, 0.0);
  for (int m = 0; m + 1 < nk; m++)
    B[m] = polycomp0((x - t[m]) / (2.0 * R), comp, n_comp) *
           polycomp0((t[m + 1] - x) / (2.0 * R), comp, n_comp);
  for (int j = 1; j <= k; j++) {
    for (int m = 0; m + j + 1 < nk; m++) {
      const double left = (x - t[m]) / (t[m + j] - t[m]) * B[m];
      const double right = (t[m + j + 1] - x) / (t[m + j + 1] - t[m + 1]) * B[m + 1];
      B[m] = left + right;
    }
    B.pop_back();
  }
}

// sum_j c_j T_j(y) by Clenshaw's recurrence
double cheb_sum(const double* c, int deg, double y) {
  double b1 = 0, b2 = 0;
  for (int j = deg; j >= 1; j--) {
    const double b = 2.0 * y * b1 - b2 + c[j];
    b2 = b1;
    b1 = b;
  }
  return y * b1 - b2 + c[0];
}

// one layer of the HE-friendly KAN: fitted SiLU on [lo, hi], PolyComp basis
void layer_forward_hef(const kan_layer_desc& d, double lo, double hi, const double* cheb, int deg,
                       double R, const std::vector<double>& x, size_t n, std::vector<double>& y) {
  const std::vector<double> t = knots(d);
  const int nb = d.G + d.k;
  y.assign(n * d.n_out, 0.0);
  std::vector<double> B;
  for (size_t b = 0; b < n; b++)
    for (int i = 0; i < d.n_in; i++) {
      const double xi = x[b * d.n_in + i];
      bspline_hef(xi, t, d.k, R, d.comp, d.n_comp, B);
      const double s = cheb_sum(cheb, deg, (2.0 * xi - (lo + hi)) / (hi - lo));
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

// sum_j c_j T_j(y) by Clenshaw's recurrence
double cheb_val(const std::vector<double>& c, double y) {
  double b1 = 0, b2 = 0;
  for (int j = (int)c.size() - 1; j >= 1; j--) {
    const double b = 2.0 * y * b1 - b2 + c[j];
    b2 = b1;
    b1 = b;
  }
  return y * b1 - b2 + c[0];
}

// Minimax Chebyshev coefficients of silu on [lo, hi] (mapped to [-1, 1]) by
// the Remez exchange over the n_samples grid: a reference of d + 2 points,
// first the Chebyshev extrema; solve p(y_i) + (-1)^i E = f(y_i); move the
// reference to the alternating extrema of the error (one per run of equal
// sign, the smaller end run dropped while there are more than d + 2); stop
// when the reference repeats.
std::vector<double> remez_fit(double lo, double hi, int d, int n_samples) {
  const int n = d + 2;
  auto fx = [&](double y) { return silu(0.5 * (hi - lo) * y + 0.5 * (hi + lo)); };
  std::vector<double> grid(n_samples);
  for (int s = 0; s < n_samples; s++) {
    const double x = lo + (hi - lo) * (double)s / (double)(n_samples - 1);
    grid[s] = (2.0 * x - (lo + hi)) / (hi - lo);
  }
  std::vector<double> ref(n), c(d + 1, 0.0);
  for (int i = 0; i < n; i++) ref[i] = -cos(M_PI * i / (n - 1));
  std::vector<int> prev;
  for (int it = 0; it < 60; it++) {
    std::vector<double> A((size_t)n * n), r(n);
    for (int i = 0; i < n; i++) {
      double t0 = 1.0, t1 = ref[i];
      for (int j = 0; j <= d; j++) {
        double tj;
        if (j == 0) tj = 1.0;
        else if (j == 1) tj = ref[i];
        else {
          tj = 2.0 * ref[i] * t1 - t0;
          t0 = t1;
          t1 = tj;
        }
        A[(size_t)i * n + j] = tj;
      }
      A[(size_t)i * n + d + 1] = (i & 1) ? -1.0 : 1.0;
      r[i] = fx(ref[i]);
    }
    const std::vector<double> sol = lstsq_qr(A, r, n, n);
    c.assign(sol.begin(), sol.begin() + d + 1);
    // runs of equal error sign and their extremum
    std::vector<std::pair<int, double>> runs;
    int st = 0;
    double prev_sign = 0;
    std::vector<double> e(n_samples);
    for (int s = 0; s < n_samples; s++) e[s] = fx(grid[s]) - cheb_val(c, grid[s]);
    for (int s = 0; s <= n_samples; s++) {
      double sg = 0;
      if (s < n_samples) {
        sg = e[s] > 0 ? 1.0 : (e[s] < 0 ? -1.0 : 0.0);
        if (sg == 0) sg = prev_sign;
      }
      if (s == 0) {
        prev_sign = sg;
        continue;
      }
      if (s == n_samples || sg != prev_sign) {
        int best = st;
        for (int k = st; k < s; k++)
          if (fabs(e[k]) > fabs(e[best])) best = k;
        runs.push_back({best, fabs(e[best])});
        st = s;
      }
      prev_sign = sg;
    }
    if ((int)runs.size() < n) break;
    while ((int)runs.size() > n) {
      if (runs.front().second < runs.back().second)
        runs.erase(runs.begin());
      else
        runs.pop_back();
    }
    std::vector<int> idx;
    for (auto& rr : runs) idx.push_back(rr.first);
    if (idx == prev) break;
    prev = idx;
    for (int i = 0; i < n; i++) ref[i] = grid[idx[i]];
  }
  return c;
}

}  // namespace

extern "C" {

int kan_silu_fit(double lo, double hi, double mu, double sigma, int degree, int n_samples,
                 int method, double* cheb) {
  if (!(hi > lo) || degree < 1 || n_samples <= degree + 1 || !cheb || method < 0 || method > 2)
    return CKKS_ERR_INVALID_ARG;
  const int n = degree + 1;
  if (method == KAN_FIT_REMEZ) {
    const std::vector<double> c = remez_fit(lo, hi, degree, n_samples);
    for (int j = 0; j < n; j++) cheb[j] = c[j];
    return CKKS_OK;
  }
  std::vector<double> A((size_t)n_samples * n), r(n_samples);
  for (int s = 0; s < n_samples; s++) {
    const double x = lo + (hi - lo) * (double)s / (double)(n_samples - 1);
    const double y = (2.0 * x - (lo + hi)) / (hi - lo);
    const double sw = method == KAN_FIT_OLS ? 1.0 : sqrt(fabs(x - mu) <= 3.0 * sigma ? 10.0 : 1.0);
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
                  int silu_degree, const double* fixed_range, int n_fit_samples, int fit_method,
                  double* R, double* silu_lo, double* silu_hi, double* cheb) {
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
    const int rc = kan_silu_fit(lo, hi, mu, sigma, silu_degree, n_fit_samples, fit_method,
                                cheb + li * (size_t)(silu_degree + 1));
    if (rc != CKKS_OK) return rc;
    double tmax = 0;
    for (double t : knots(d)) tmax = std::max(tmax, fabs(t));
    R[li] = 1.1 * (amax + tmax) / 2.0;
    // the next layer's inputs as the encrypted network computes them
    layer_forward_hef(d, lo, hi, cheb + li * (size_t)(silu_degree + 1), silu_degree, R[li], h, n,
                      y);
    h.swap(y);
  }
  return CKKS_OK;
}

}  // extern "C"
