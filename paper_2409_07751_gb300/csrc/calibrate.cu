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
#include <utility>
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

// The comparison composite of a layer as odd monomial coefficient lists,
// first stage first: explicit stages, or f_n by order.
std::vector<std::vector<double>> comp_stages(const kan_layer_desc& d) {
  std::vector<std::vector<double>> st;
  if (d.n_comp_poly > 0) {
    const double* p = d.comp_poly;
    for (int s = 0; s < d.n_comp_poly; s++) {
      st.emplace_back(p, p + d.comp_poly_len[s]);
      p += d.comp_poly_len[s];
    }
  } else {
    for (int s = 0; s < d.n_comp; s++) st.push_back(fn_odd(d.comp[s]));
  }
  return st;
}

// sum_l c_l u^(2l+1)
double odd_val(const std::vector<double>& c, double u) {
  double acc = 0, p = u;
  const double u2 = u * u;
  for (double cl : c) {
    acc += cl * p;
    p *= u2;
  }
  return acc;
}

// PolyComp(a, 0) = (1 + f(a)) / 2 with f the composite of the stages
double polycomp0(double a, const std::vector<std::vector<double>>& stages) {
  double u = a;
  for (const auto& c : stages) u = odd_val(c, u);
  return 0.5 + 0.5 * u;
}

// Algorithm 2 on plaintext values: soft order-0 indicators (product form,
// or the difference of neighbouring knot comparisons), the same recursion
void bspline_hef(double x, const std::vector<double>& t, int k, double R,
                 const std::vector<std::vector<double>>& stages, int b0_form,
                 std::vector<double>& B) {
  const int nk = (int)t.size();
  B.assign(nk - 1, 0.0);
  if (b0_form == 1) {
    std::vector<double> sm(nk);
    for (int m = 0; m < nk; m++) sm[m] = polycomp0((x - t[m]) / (2.0 * R), stages);
    for (int m = 0; m + 1 < nk; m++) B[m] = sm[m] - sm[m + 1];
  } else {
    for (int m = 0; m + 1 < nk; m++)
      B[m] = polycomp0((x - t[m]) / (2.0 * R), stages) *
             polycomp0((t[m + 1] - x) / (2.0 * R), stages);
  }
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
  const std::vector<std::vector<double>> stages = comp_stages(d);
  for (size_t b = 0; b < n; b++)
    for (int i = 0; i < d.n_in; i++) {
      const double xi = x[b * d.n_in + i];
      bspline_hef(xi, t, d.k, R, stages, d.b0_form, B);
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

// ---------------------------------------------------------------- PolyComp
// Composite minimax comparison (Lee et al. 2021, cited by Algorithm 2's
// PolyComp): stage 1 is the odd polynomial of the given degree with the
// least maximum error against 1 on [eps, A] (so against sign on
// [-A, -eps] u [eps, A]); each further stage the same on the image of the
// previous stage's interval. Each stage by the Remez exchange over 40001
// evenly spaced points in the basis T_1, T_3, .. of x / hi (the reference
// starts at the Chebyshev points of the interval; the new reference takes
// the largest error of each run of equal sign, an exact zero joining the run
// before it, dropping the smaller end run while there are too many; the
// loop stops when the reference stops moving). Images are the extreme values
// over the ends and the stationary points inside (sign changes of p' on the
// grid, refined by bisection).

// Gaussian elimination with partial pivoting; A is n x n row-major
std::vector<double> solve_dense(std::vector<double> A, std::vector<double> b, int n) {
  for (int k = 0; k < n; k++) {
    int piv = k;
    for (int i = k + 1; i < n; i++)
      if (fabs(A[(size_t)i * n + k]) > fabs(A[(size_t)piv * n + k])) piv = i;
    if (piv != k) {
      for (int j = 0; j < n; j++) std::swap(A[(size_t)k * n + j], A[(size_t)piv * n + j]);
      std::swap(b[k], b[piv]);
    }
    for (int i = k + 1; i < n; i++) {
      const double f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      for (int j = k; j < n; j++) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
      b[i] -= f * b[k];
    }
  }
  std::vector<double> x(n);
  for (int k = n - 1; k >= 0; k--) {
    double s = b[k];
    for (int j = k + 1; j < n; j++) s -= A[(size_t)k * n + j] * x[j];
    x[k] = s / A[(size_t)k * n + k];
  }
  return x;
}

// T_1(t), T_3(t), .., T_{2m-1}(t)
void odd_cheb(double t, int m, double* out) {
  double t0 = 1.0, t1 = t;
  out[0] = t;
  for (int j = 2, l = 1; l < m; j++) {
    const double tj = 2.0 * t * t1 - t0;
    t0 = t1;
    t1 = tj;
    if (j & 1) out[l++] = tj;
  }
}

// derivative of sum_l c_l u^(2l+1)
double odd_deriv(const std::vector<double>& c, double u) {
  double acc = 0, p = 1.0;
  const double u2 = u * u;
  for (size_t l = 0; l < c.size(); l++) {
    acc += (double)(2 * l + 1) * c[l] * p;
    p *= u2;
  }
  return acc;
}

// [min, max] of the odd polynomial over [lo, hi]
std::pair<double, double> odd_image(const std::vector<double>& c, double lo, double hi) {
  double mn = std::min(odd_val(c, lo), odd_val(c, hi)), mx = std::max(odd_val(c, lo), odd_val(c, hi));
  const int G = 40000;
  double xa = lo, da = odd_deriv(c, lo);
  for (int g = 1; g <= G; g++) {
    const double xb = lo + (hi - lo) * (double)g / G, db = odd_deriv(c, xb);
    if ((da < 0) != (db < 0) && da != 0) {
      double a = xa, b = xb, fa = da;
      for (int it = 0; it < 200 && b - a > 0; it++) {
        const double mid = 0.5 * (a + b);
        if (mid <= a || mid >= b) break;
        const double fm = odd_deriv(c, mid);
        if ((fm < 0) == (fa < 0)) {
          a = mid;
          fa = fm;
        } else {
          b = mid;
        }
      }
      for (double x : {a, b}) {
        mn = std::min(mn, odd_val(c, x));
        mx = std::max(mx, odd_val(c, x));
      }
    }
    xa = xb;
    da = db;
  }
  return {mn, mx};
}

// the odd minimax polynomial of `degree` against 1 on [lo, hi], as odd
// monomial coefficients in x
std::vector<double> odd_minimax(double lo, double hi, int degree) {
  const int m = (degree + 1) / 2, n = m + 1, NG = 40001;
  std::vector<double> xs(NG), B((size_t)NG * m);
  for (int g = 0; g < NG; g++) {
    xs[g] = lo + (hi - lo) * (double)g / (double)(NG - 1);
    odd_cheb(xs[g] / hi, m, &B[(size_t)g * m]);
  }
  std::vector<double> ref(n), sol;
  for (int i = 0; i < n; i++) ref[i] = lo + (hi - lo) * (1.0 - cos(M_PI * i / (n - 1))) / 2.0;
  std::vector<double> e(NG), row(m);
  for (int it = 0; it < 100; it++) {
    std::vector<double> A((size_t)n * n);
    for (int i = 0; i < n; i++) {
      odd_cheb(ref[i] / hi, m, &A[(size_t)i * n]);
      A[(size_t)i * n + m] = (i & 1) ? -1.0 : 1.0;
    }
    sol = solve_dense(A, std::vector<double>(n, 1.0), n);
    for (int g = 0; g < NG; g++) {
      double v = 0;
      for (int l = 0; l < m; l++) v += B[(size_t)g * m + l] * sol[l];
      e[g] = v - 1.0;
    }
    std::vector<std::pair<int, double>> runs;
    int st = 0;
    double sg_prev = e[0] > 0 ? 1.0 : (e[0] < 0 ? -1.0 : 0.0);
    for (int g = 1; g <= NG; g++) {
      double sg = sg_prev;
      if (g < NG && e[g] != 0) sg = e[g] > 0 ? 1.0 : -1.0;
      if (g == NG || sg != sg_prev) {
        int best = st;
        for (int k = st; k < g; k++)
          if (fabs(e[k]) > fabs(e[best])) best = k;
        runs.push_back({best, fabs(e[best])});
        st = g;
      }
      sg_prev = sg;
    }
    if ((int)runs.size() < n) break;
    while ((int)runs.size() > n) {
      if (runs.front().second < runs.back().second)
        runs.erase(runs.begin());
      else
        runs.pop_back();
    }
    bool same = true;
    std::vector<double> nw(n);
    for (int i = 0; i < n; i++) {
      nw[i] = xs[runs[i].first];
      if (fabs(nw[i] - ref[i]) > (hi - lo) * 1e-12) same = false;
    }
    if (same) break;
    ref = nw;
  }
  // sum_l s_l T_{2l+1}(x / hi) -> monomials: coefficients of T_j from the
  // recurrence T_{j+1} = 2 t T_j - T_{j-1}, then t = x / hi
  const int D = 2 * m;
  std::vector<std::vector<double>> T(D, std::vector<double>(D, 0.0));
  T[0][0] = 1.0;
  if (D > 1) T[1][1] = 1.0;
  for (int j = 2; j < D; j++)
    for (int k = 0; k < D; k++) T[j][k] = (k > 0 ? 2.0 * T[j - 1][k - 1] : 0.0) - T[j - 2][k];
  std::vector<double> c(m, 0.0);
  for (int l = 0; l < m; l++) {
    double a = 0;
    for (int j = 0; j < m; j++) a += sol[j] * T[2 * j + 1][2 * l + 1];
    c[l] = a * pow(1.0 / hi, 2 * l + 1);
  }
  return c;
}

}  // namespace

extern "C" {

int kan_comp_minimax(double eps, double A, const int* degrees, int n_stages, double* coef,
                     double* taus) {
  if (!degrees || n_stages < 1 || !coef || !(eps > 0) || !(A > eps)) return CKKS_ERR_INVALID_ARG;
  double lo = eps, hi = A;
  size_t off = 0;
  for (int s = 0; s < n_stages; s++) {
    if (degrees[s] < 1 || degrees[s] % 2 == 0 || degrees[s] > 63) return CKKS_ERR_INVALID_ARG;
    if (!(lo > 0)) return CKKS_ERR_INVALID_ARG;  // the previous stage does not separate the signs
    const std::vector<double> c = odd_minimax(lo, hi, degrees[s]);
    for (double v : c) coef[off++] = v;
    const std::pair<double, double> im = odd_image(c, lo, hi);
    lo = im.first;
    hi = im.second;
    if (taus) taus[s] = std::max(1.0 - lo, hi - 1.0);
  }
  return CKKS_OK;
}

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
